"""gc_coulomb_field_noalloc: the Eq. 6 field for callers that may not allocate
device memory (code inside an allocator or memory pool it must not re-enter,
or inside a framework that owns every device byte).  Its scratch is a fixed
array inside the library, so it is checked here against gc_coulomb_field, the
entry point that allocates its own scratch, on two calls in a row (the second
call finds the first call's leftovers in the shared array), and on sampled
carriers against the FP64 oracle.

Sizes: 32,768 (GC_NOALLOC_MAX_CARRIERS, where the partial-sum area is exactly
full), 20,000 and 5,000 (one lane per i-group), 1,573 (the 4-lane path of
small events).

This file is collected last on purpose: a failure here does not hide the
result of any other test in a run that stops at the first failure.
"""
import numpy as np
import pytest

import oracle as O

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


def bound(xyz, idx, precision, eps=0.01):
    """Error bound of one GPU evaluation of Eq. 6 at carriers idx: the FP32
    bound of the parity tests (per term 12 u plus the rounding of the FP32
    shadow, (256 + 16) u of the absolute sum with Kahan), plus the f16
    rounding of r^2 for FP16x2, and 1e-12 of the absolute sum in FP64."""
    rho = np.abs(xyz - xyz[0]).max()
    out = np.zeros((len(idx), 3))
    for k, i in enumerate(idx):
        d = xyz[i] - xyz
        s2 = (d * d).sum(1) + eps * eps
        mag = np.sqrt((d * d).sum(1)) / s2 ** 1.5
        if precision == 0:
            out[k] = 1e-12 * K_EQ6 * mag.sum() + 1e-300
            continue
        per = mag * (12 * U32 + 20 * U32 * rho / np.sqrt(s2))
        if precision == 3:
            sc = 2.0 ** np.floor(np.log2(52.0 / max(rho, 1e-6)))
            per = per + mag * 1.5 * (6 * 2.0 ** -11 + 2.0 ** -25 / (s2 * sc * sc))
        acc = (len(xyz) + 16) if precision == 1 else (256 + 16)
        out[k] = K_EQ6 * (per.sum() + acc * U32 * mag.sum())
    return out


def sample(rng, n):
    return np.unique(np.concatenate([np.arange(min(n, 64)), rng.choice(n, min(n, 64), replace=False),
                                     np.arange(max(0, n - 64), n)]))


@pytest.mark.parametrize("precision", [2, 0, 3, 1])
@pytest.mark.parametrize("sizes", [(20000, 5000), (32768, 1573)])
def test_noalloc_matches_allocating_entry_point_twice(gc, precision, sizes):
    rng = np.random.default_rng(77 + sizes[0])
    first = np.array([0.0, 0.0, 300.0]) + 0.5 * rng.standard_normal((sizes[0], 3))
    second = np.array([3.0, -1.0, 120.0]) + 0.4 * rng.standard_normal((sizes[1], 3))
    for xyz in (first, second):
        want = field(gc, gc.gc_coulomb_field, xyz, precision)
        got = field(gc, gc.gc_coulomb_field_noalloc, xyz, precision)
        assert np.all(np.isfinite(got))
        idx = sample(rng, len(xyz))
        # two evaluations, each within its bound of the exact field
        assert np.all(np.abs(got[idx] - want[idx]) <= 2 * bound(xyz, idx, precision))
        ref = O.coulomb_field(xyz, targets=idx)
        assert np.all(np.abs(got[idx] - ref) <= bound(xyz, idx, precision))
        if len(xyz) <= 5000:
            # same j-chunks as the allocating call: the same bits
            assert np.array_equal(got, want)


def test_noalloc_rejects_sizes_beyond_its_scratch(gc):
    import torch
    n = gc.GC_NOALLOC_MAX_CARRIERS + 1
    t = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    E = torch.zeros_like(t)
    with pytest.raises(gc.GcError) as err:
        gc.gc_coulomb_field_noalloc(t, n, 0.01, 11.7, 2, E)
    assert err.value.status == gc.GC_ERR_PARAM
