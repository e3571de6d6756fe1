"""The C-ABI library builds, loads and exports every symbol include/gcoreccd.h
declares; host-side validation works without a GPU (no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_11043_gb300 import build
    build.build()
    import paper_2203_11043_gb300 as gc
    return gc.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gcoreccd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gc_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gc_create", "gc_load_carriers", "gc_run", "gc_collect", "gc_image", "gc_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    import paper_2203_11043_gb300 as gc
    names = declared_functions()
    assert sorted(gc.EXPORTS) == names
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", gc.library_path()], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (gc_\w+)", out))
    assert set(names) <= exported


def test_library_targets_sm103a_only():
    from paper_2203_11043_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_param_struct_layout(lib):
    """ctypes mirror of gc_params matches the C layout (defaults round-trip)."""
    import paper_2203_11043_gb300 as gc
    p = gc.gc_default_params()
    assert p.abi_version == gc.GC_ABI_VERSION
    assert (p.thickness_um, p.z_well_um, p.a1_V_cm_um, p.a2_V_cm, p.T_K) == (675.0, 0.0, 2.0, 1500.0, 140.0)
    assert (p.eps_si_rel, p.softening_um, p.dt_s) == (11.7, 0.01, 1e-11)
    assert (p.max_steps, p.coulomb, p.diffusion, p.reflect_back) == (100000, 1, 1, 1)
    assert (p.img_w, p.img_h, p.pixel_um) == (64, 64, 15.0)
    assert (p.graph_steps, p.autotune, p.newton, p.jchunk, p.pair_R, p.timing) == (32, 1, 0, 0, 0, 0)
    assert p.precision == gc.GC_FP32_KAHAN
    assert (p.stored_charge, p.stored_z_um, p.tile_frames) == (0, 0.0, 0)


@pytest.mark.parametrize("field,value", [
    ("abi_version", 99), ("precision", 7), ("precision", -1), ("dt_s", 0.0), ("dt_s", float("nan")),
    ("T_K", -1.0), ("thickness_um", 0.0), ("z_well_um", 700.0), ("pixel_um", 0.0), ("img_w", 0),
    ("img_h", -3), ("max_steps", -1), ("softening_um", 0.0), ("eps_si_rel", 0.0),
    ("graph_steps", -1), ("jchunk", -5), ("coulomb", 2), ("pair_R", 3), ("timing", 2),
    ("stored_charge", 2), ("stored_z_um", float("inf")), ("tile_frames", 2), ("tile_frames", -1),
])
def test_invalid_params_rejected_before_any_cuda_call(lib, field, value):
    import paper_2203_11043_gb300 as gc
    p = gc.gc_default_params()
    setattr(p, field, value)
    h = ctypes.c_void_p()
    assert lib.gc_create(ctypes.byref(p), None, ctypes.byref(h)) == gc.GC_ERR_PARAM
    assert not h.value


def test_fp16x2_without_newton_step(lib):
    """The FP16x2 form has no Newton step (a padding pair would give inf * 0)."""
    import paper_2203_11043_gb300 as gc
    p = gc.gc_default_params(precision=gc.GC_FP16X2, newton=1)
    h = ctypes.c_void_p()
    assert lib.gc_create(ctypes.byref(p), None, ctypes.byref(h)) == gc.GC_ERR_PARAM


def test_status_strings(lib):
    import paper_2203_11043_gb300 as gc
    for st in (gc.GC_OK, gc.GC_INCOMPLETE, gc.GC_ERR_PARAM, gc.GC_ERR_ALLOC, gc.GC_ERR_CUDA,
               gc.GC_ERR_STATE, gc.GC_ERR_DEVICE_TIMEOUT, gc.GC_ERR_NO_DEVICE):
        assert gc.gc_status_string(st).startswith("GC_")
    assert "unknown" in gc.gc_status_string(12345)


def test_null_handles_are_rejected(lib):
    import paper_2203_11043_gb300 as gc
    assert lib.gc_run(None, 1, None) == gc.GC_ERR_PARAM
    assert lib.gc_collect(None, None, None, None, None, None) == gc.GC_ERR_PARAM
    assert lib.gc_image(None, None, 0) == gc.GC_ERR_PARAM
    assert lib.gc_positions(None, None) == gc.GC_ERR_PARAM
    assert lib.gc_load_carriers(None, None, 0, None, 1, None, None) == gc.GC_ERR_PARAM
    lib.gc_destroy(None)
    assert lib.gc_coulomb_field(None, -1, 0.01, 11.7, 2, None, None) == gc.GC_ERR_PARAM
    assert lib.gc_coulomb_field(None, 10, 0.0, 11.7, 2, None, None) == gc.GC_ERR_PARAM


def test_binding_fails_loudly_without_the_library(monkeypatch):
    """No CPU fallback: a missing shared library is an error."""
    import paper_2203_11043_gb300.gcoreccd as g
    monkeypatch.setattr(g, "_lib", None)
    monkeypatch.setattr(g, "library_path", lambda: "/nonexistent/libgcoreccd.so")
    with pytest.raises(RuntimeError, match="not built"):
        g.load()


def test_product_code_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2203_11043_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "oracle.h" not in src, f
