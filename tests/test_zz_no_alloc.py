"""gc_coulomb_field_noalloc: the Eq. 6 field for callers that may not allocate
device memory (code inside an allocator or memory pool it must not re-enter,
or inside a framework that owns every device byte).  Its scratch is a fixed
array inside the library, so it is checked here against gc_coulomb_field, the
entry point that allocates its own scratch, on two calls in a row (the second
call finds the first call's leftovers in the shared array).

This file is collected last on purpose: a failure here does not hide the
result of any other test in a run that stops at the first failure.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
K_EQ6 = 1.2307389298  # q / (4 pi eps0 11.7) in V/cm um^2


@pytest.fixture(scope="module")
def gc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11043_gb300 import build
    build.build()
    import paper_2203_11043_gb300 as g
    g.load()
    return g


def field(gc, fn, xyz, precision):
    import torch
    t = torch.tensor(xyz, dtype=torch.float64, device="cuda")
    E = torch.full_like(t, float("nan"))
    fn(t, len(xyz), 0.01, 11.7, precision, E, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return E.cpu().numpy()


def tolerance(xyz, idx, precision, eps=0.01):
    """Bound on the difference of two GPU evaluations of Eq. 6 at carriers idx
    (twice the FP32 error bound the parity tests use; 2e-12 of the absolute
    sum for the FP64 form)."""
    rho = np.abs(xyz - xyz[0]).max()
    out = np.zeros((len(idx), 3))
    for k, i in enumerate(idx):
        d = xyz[i] - xyz
        s2 = (d * d).sum(1) + eps * eps
        mag = np.sqrt((d * d).sum(1)) / s2 ** 1.5
        if precision == 0:
            out[k] = 2e-12 * K_EQ6 * mag.sum() + 1e-300
        else:
            per = mag * (12 * U32 + 20 * U32 * rho / np.sqrt(s2))
            out[k] = 2 * K_EQ6 * (per.sum() + (256 + 16) * U32 * mag.sum())
    return out


@pytest.mark.parametrize("precision", [2, 0])
def test_noalloc_matches_allocating_entry_point_twice(gc, precision):
    rng = np.random.default_rng(77)
    first = np.array([0.0, 0.0, 300.0]) + 0.5 * rng.standard_normal((20000, 3))
    second = np.array([3.0, -1.0, 120.0]) + 0.4 * rng.standard_normal((5000, 3))
    for xyz in (first, second):
        want = field(gc, gc.gc_coulomb_field, xyz, precision)
        got = field(gc, gc.gc_coulomb_field_noalloc, xyz, precision)
        assert np.all(np.isfinite(got))
        idx = np.unique(np.concatenate([np.arange(100), rng.choice(len(xyz), 100, replace=False),
                                        np.arange(len(xyz) - 100, len(xyz))]))
        assert np.all(np.abs(got[idx] - want[idx]) <= tolerance(xyz, idx, precision))


def test_noalloc_rejects_sizes_beyond_its_scratch(gc):
    import torch
    n = gc.GC_NOALLOC_MAX_CARRIERS + 1
    t = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    E = torch.zeros_like(t)
    with pytest.raises(gc.GcError) as err:
        gc.gc_coulomb_field_noalloc(t, n, 0.01, 11.7, 2, E)
    assert err.value.status == gc.GC_ERR_PARAM
