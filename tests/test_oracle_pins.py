"""Pins of the FP64 oracle to things the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check uses a printed or
hand-evaluated value, a closed form, an independent library routine
(scipy.constants, scipy quadrature / ODE integration, finite differences of
the potential), or an invariant of the equations.
"""
import math

import numpy as np
import pytest
import scipy.constants as sc
from scipy import stats
from scipy.integrate import quad, solve_ivp

import oracle as O
from conftest import load_golden

T140 = 140.0


# ---- Eq. 2: mobility ------------------------------------------------------------------

def test_mobility_hand_values():
    """Eq. 2 against hand-evaluated points (golden/mobility_eq2.txt)."""
    for E, T, mu in load_golden("mobility_eq2.txt"):
        got = O.mobility(float(E), float(T))
        assert got == pytest.approx(float(mu), rel=1e-8), (E, T)


@pytest.mark.parametrize("T", [100.0, 140.0, 173.0, 300.0])
def test_mobility_closed_form_limits(T):
    """Eq. 2 special cases: mu(0) = 1.31e8 T^-2.2; at E = E_c = 1.24 T^1.68 the
    bracket is 2, so mu = mu0 / 2^(1/beta); at high field mu E -> mu0 E_c."""
    mu0 = 1.31e8 * T ** -2.2
    Ec = 1.24 * T ** 1.68
    beta = 0.46 * T ** 0.17
    assert O.mobility(0.0, T) == pytest.approx(mu0, rel=1e-14)
    assert O.mobility(Ec, T) == pytest.approx(mu0 / 2 ** (1 / beta), rel=1e-13)
    E = 1e12
    assert O.mobility(E, T) * E == pytest.approx(mu0 * Ec, rel=1e-6)


def test_mobility_monotone_decreasing():
    Es = np.linspace(0, 2e5, 400)
    mus = [O.mobility(e, T140) for e in Es]
    assert all(a > b for a, b in zip(mus, mus[1:]))


# ---- constants: Eq. 4 and Eq. 6 -------------------------------------------------------

def test_coulomb_constant_against_codata():
    """K of Eq. 6 for eps_Si = 11.7, from scipy's CODATA constants, in V/cm um^2."""
    K = sc.e / (4 * math.pi * sc.epsilon_0 * 11.7)  # V m
    assert O.coulomb_K(11.7) == pytest.approx(K * 1e10, rel=1e-9)
    assert O.coulomb_K(11.7) == pytest.approx(1.2307389298, rel=1e-9)


def test_thermal_voltage_against_codata():
    """k_B T / q of Eq. 4."""
    assert O.thermal_voltage(T140) == pytest.approx(sc.k * T140 / sc.e, rel=1e-12)


# ---- Philox-4x32-10 and Box-Muller ------------------------------------------------------

def test_philox_known_answers():
    """Published Random123 known-answer vectors (golden/philox4x32_10_kat.txt)."""
    for row in load_golden("philox4x32_10_kat.txt"):
        v = [int(h, 16) for h in row]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_box_muller_normal_statistics():
    """The diffusion normals are N(0, 1), mutually uncorrelated, and differ
    between steps, carriers and seeds."""
    ids = np.arange(40000)
    n = O.diffusion_normals(1, ids, 7)
    for c in range(3):
        col = n[:, c]
        assert abs(col.mean()) < 4 / math.sqrt(len(col))
        assert abs(col.var() - 1.0) < 5 * math.sqrt(2 / len(col))
        assert stats.kstest(col, "norm").pvalue > 1e-3
    cc = np.corrcoef(n.T)
    assert np.all(np.abs(cc[np.triu_indices(3, 1)]) < 4 / math.sqrt(len(ids)))
    m = O.diffusion_normals(1, ids[:1000], 8)
    s = O.diffusion_normals(2, ids[:1000], 7)
    assert abs(np.corrcoef(n[:1000, 0], m[:, 0])[0, 1]) < 0.15
    assert abs(np.corrcoef(n[:1000, 0], s[:, 0])[0, 1]) < 0.15


def test_normals_use_the_specified_counter():
    """Counter (id, lo32(step), hi32(step), 0), key (lo32(seed), hi32(seed)),
    then Box-Muller on (x0, x1) and (x2, x3)."""
    seed, cid, step = 0x0123456789ABCDEF, 77, (5 << 32) + 9
    r = O.philox4x32_10([cid, step & 0xFFFFFFFF, step >> 32, 0], [seed & 0xFFFFFFFF, seed >> 32])
    ua, ub = (int(r[0]) + 1) / 2 ** 32, int(r[1]) / 2 ** 32
    ua2, ub2 = (int(r[2]) + 1) / 2 ** 32, int(r[3]) / 2 ** 32
    want = [math.sqrt(-2 * math.log(ua)) * math.cos(2 * math.pi * ub),
            math.sqrt(-2 * math.log(ua)) * math.sin(2 * math.pi * ub),
            math.sqrt(-2 * math.log(ua2)) * math.cos(2 * math.pi * ub2)]
    got = O.diffusion_normals(seed, [cid], step)[0]
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15)


# ---- Eq. 6: softened Coulomb field ------------------------------------------------------

def _potential(xyz, t, eps, K):
    """Softened potential at carrier t: K sum_j 1 / sqrt(|r_t - r_j|^2 + eps^2)."""
    d = xyz[t][None, :] - xyz
    return K * np.sum(1.0 / np.sqrt(np.sum(d * d, axis=1) + eps * eps))


def test_field_is_minus_gradient_of_softened_potential():
    """E = -grad(phi) with phi the softened Coulomb potential (central
    differences): fixes the sign, the exponent 3/2 and where eps enters."""
    rng = np.random.default_rng(3)
    xyz = rng.normal(size=(40, 3)) * np.array([0.4, 0.3, 0.5]) + np.array([0, 0, 300.0])
    eps, K = 0.05, O.coulomb_K(11.7)
    E = O.coulomb_field(xyz, softening_um=eps)
    h = 1e-5
    for t in [0, 7, 19, 39]:
        for c in range(3):
            xp, xm = xyz.copy(), xyz.copy()
            xp[t, c] += h
            xm[t, c] -= h
            g = (_potential(xp, t, eps, K) - _potential(xm, t, eps, K)) / (2 * h)
            assert E[t, c] == pytest.approx(-g, rel=2e-6, abs=1e-6 * np.abs(E).max())


def test_field_pairwise_antisymmetry():
    """sum_i E_i = 0 (each pair contributes equal and opposite terms)."""
    rng = np.random.default_rng(5)
    xyz = rng.normal(size=(500, 3)) * 2.0 + np.array([0, 0, 200.0])
    E = O.coulomb_field(xyz, softening_um=0.01)
    assert np.abs(E.sum(axis=0)).max() <= 1e-12 * np.abs(E).sum()


def test_two_body_closed_form():
    """Two holes at separation d: E = +-K d / (d^2 + eps^2)^(3/2) along the axis."""
    K = O.coulomb_K(11.7)
    for d, eps in [(0.1, 0.01), (1.0, 0.01), (0.02, 0.05)]:
        xyz = np.array([[0.0, 0.0, 100.0], [d, 0.0, 100.0]])
        E = O.coulomb_field(xyz, softening_um=eps)
        mag = K * d / (d * d + eps * eps) ** 1.5
        np.testing.assert_allclose(E, [[-mag, 0, 0], [mag, 0, 0]], rtol=1e-13, atol=1e-15 * mag)


def test_three_body_equilateral_closed_form():
    """Equilateral triangle of side s: each field is radial outward with
    magnitude sqrt(3) K s / (s^2 + eps^2)^(3/2)."""
    K, s, eps = O.coulomb_K(11.7), 0.3, 0.01
    c = np.array([1.0, -2.0, 50.0])
    R = s / math.sqrt(3)
    ang = np.array([0.1, 0.1 + 2 * math.pi / 3, 0.1 + 4 * math.pi / 3])
    xyz = c + R * np.stack([np.cos(ang), np.sin(ang), np.zeros(3)], axis=1)
    E = O.coulomb_field(xyz, softening_um=eps)
    mag = math.sqrt(3) * K * s / (s * s + eps * eps) ** 1.5
    radial = (xyz - c) / R
    np.testing.assert_allclose(E, mag * radial, rtol=1e-12, atol=1e-12 * mag)


def test_self_term_vanishes_and_sources_subset():
    """A lone carrier feels no field; the field from a subset of sources is
    the sum over that subset."""
    one = np.array([[0.0, 0.0, 10.0]])
    assert np.all(O.coulomb_field(one) == 0.0)
    rng = np.random.default_rng(9)
    xyz = rng.normal(size=(30, 3))
    a = O.coulomb_field(xyz, src=np.arange(0, 12), targets=[3, 20])
    b = O.coulomb_field(xyz, src=np.arange(12, 30), targets=[3, 20])
    full = O.coulomb_field(xyz, targets=[3, 20])
    np.testing.assert_allclose(a + b, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())


# ---- the whole step: Coulomb off ----------------------------------------------------------

def _drift_time(z0, a1=2.0, a2=1500.0, T=T140):
    f = lambda z: 1.0 / (1e4 * O.mobility(a2 - a1 * z, T) * (a2 - a1 * z))
    return quad(f, 0.0, z0, epsabs=0.0, epsrel=1e-12, limit=200)[0]


@pytest.mark.parametrize("z0", [300.0, 647.0, 675.0])
def test_drift_time_coulomb_and_diffusion_off(z0):
    """Collection step equals the drift time t(z0) = int_0^z0 dz / (mu E) of
    Eqs. 1-2 (FP64 quadrature) within the explicit-Euler error, which halves
    with dt."""
    t_exact = _drift_time(z0)
    errs = []
    for dt in (1e-11, 5e-12):
        p = O.make_params(coulomb=0, diffusion=0, dt_s=dt, max_steps=10 ** 7)
        sim = O.Simulation(p, np.array([[0.0, 0.0, z0 - 1e-9]]))
        sim.run()
        t_sim = sim.collect_step[0] * dt
        assert abs(t_sim - t_exact) <= 2 * dt
        errs.append(abs(t_sim - t_exact))
    assert t_exact * 1e9 == pytest.approx({300.0: 12.3143, 647.0: 44.2003, 675.0: 50.7462}[z0],
                                          abs=1e-4)


def test_lateral_spread_coulomb_off():
    """sigma_x^2 = sigma_y^2 = 2 int D dt = 2e4 (kT/q) / a1 ln(a2 / (a2 - a1 z0)) um^2
    (Eqs. 3-4 with the mobility cancelling), for a point source at z0 = 300 um."""
    n, z0 = 40000, 300.0
    p = O.make_params(coulomb=0, diffusion=1, img_w=64, img_h=64)
    xyz = np.tile(np.array([[0.0, 0.0, z0]]), (n, 1))
    sim = O.Simulation(p, xyz, img_origin=[[-480.0, -480.0]])
    sim.run()
    assert np.all(sim.collect_step > 0)
    want = 2e4 * (sc.k * T140 / sc.e) / 2.0 * math.log(1500.0 / (1500.0 - 2.0 * z0))
    assert want == pytest.approx(61.627, rel=1e-4)
    tol = 5 * math.sqrt(2 / n) + 5e-3
    assert sim.x.var() == pytest.approx(want, rel=tol)
    assert sim.y.var() == pytest.approx(want, rel=tol)
    assert abs(sim.x.mean()) < 5 * math.sqrt(want / n)
    # all charge is accounted for: image + off-image + still active = n
    assert int(sim.image.sum()) + int(sim.off_image.sum()) == n


# ---- the whole step: Coulomb on, small systems -------------------------------------------

def test_two_body_separation_matches_ode():
    """Two holes, no depletion field (a1 = a2 = 0), no diffusion: the
    separation obeys d' = 2 * 1e4 mu(E(d)) E(d) with E(d) = K d / (d^2 + eps^2)^(3/2).
    The simulation converges to an independent high-order ODE solution at
    first order in dt."""
    K, eps, d0 = O.coulomb_K(11.7), 0.01, 0.5
    t_end = 2e-8

    def rhs(t, d):
        E = K * d[0] / (d[0] ** 2 + eps ** 2) ** 1.5
        return [2 * 1e4 * O.mobility(E, T140) * E]

    ref = solve_ivp(rhs, (0, t_end), [d0], method="DOP853", rtol=1e-12, atol=1e-15).y[0, -1]
    errs = []
    for dt in (1e-11, 5e-12):
        p = O.make_params(a1=0.0, a2=0.0, diffusion=0, dt_s=dt, z_well_um=-1.0)
        sim = O.Simulation(p, np.array([[-d0 / 2, 0.0, 300.0], [d0 / 2, 0.0, 300.0]]))
        sim.run(int(round(t_end / dt)))
        pos = sim.positions()
        assert np.all(pos[:, 1:] == np.array([[0.0, 300.0], [0.0, 300.0]]))
        assert pos[0, 0] == pytest.approx(-pos[1, 0], rel=1e-13)
        errs.append(abs((pos[1, 0] - pos[0, 0]) - ref))
    assert ref > d0 * 1.5
    assert errs[0] < 1e-3 * ref
    assert errs[1] == pytest.approx(errs[0] / 2, rel=0.1)


def test_three_body_stays_equilateral():
    """With no depletion field and no diffusion an equilateral triangle
    expands but stays equilateral (to rounding)."""
    s = 0.2
    R = s / math.sqrt(3)
    ang = np.array([0.3, 0.3 + 2 * math.pi / 3, 0.3 + 4 * math.pi / 3])
    xyz = np.stack([R * np.cos(ang), R * np.sin(ang), np.full(3, 400.0)], axis=1)
    p = O.make_params(a1=0.0, a2=0.0, diffusion=0, z_well_um=-1.0)
    sim = O.Simulation(p, xyz)
    sim.run(500)
    q = sim.positions()
    d = [np.linalg.norm(q[a] - q[b]) for a, b in [(0, 1), (1, 2), (0, 2)]]
    assert min(d) > 2 * s
    assert max(d) - min(d) < 1e-12 * max(d)
    np.testing.assert_allclose(q.mean(axis=0), [0, 0, 400.0], atol=1e-13)


def test_step_zero_collection_and_pixel_edges():
    """Carriers already in the well are collected at step 0 at their own x, y
    and binned with half-open pixel bins [k p, (k+1) p) (Fig. 5)."""
    p = O.make_params(img_w=4, img_h=3, pixel_um=15.0)
    ox, oy = -30.0, -22.5
    pts = [
        (ox + 0.0, oy + 0.0),          # (0, 0) lower edge inclusive
        (ox + 15.0, oy + 15.0),        # (1, 1) exactly on the edge -> upper bin
        (np.nextafter(ox + 15.0, -1e9), oy + 1.0),  # just below the edge -> (0, 0)
        (ox + 59.999, oy + 44.999),    # (3, 2) last pixel
        (ox + 60.0, oy + 1.0),         # x == W p -> off image
        (ox - 1e-9, oy + 1.0),         # x < 0 -> off image
    ]
    xyz = np.array([[x, y, -0.5] for x, y in pts])
    sim = O.Simulation(p, xyz, img_origin=[[ox, oy]])
    assert np.all(sim.collect_step == 0)
    img = sim.image[0]
    assert img[0, 0] == 2 and img[1, 1] == 1 and img[2, 3] == 1
    assert img.sum() == 4 and sim.off_image[0] == 2
    np.testing.assert_array_equal(sim.positions()[:, :2], xyz[:, :2])


def test_back_surface_reflection():
    """A carrier pushed past z = thickness is reflected: z' = 2 thickness - z."""
    a2 = -1000.0  # field +1000 V/cm everywhere (a1 = 0): holes move to larger z
    p = O.make_params(a1=0.0, a2=a2, coulomb=0, diffusion=0, z_well_um=-1.0)
    sim = O.Simulation(p, np.array([[0.0, 0.0, 674.99], [0.0, 0.0, 676.0]]))
    assert sim.z[1] == pytest.approx(674.0, abs=1e-12)  # reflected at load
    sim.run(1)
    step = 1e4 * O.mobility(1000.0, T140) * 1000.0 * 1e-11
    assert sim.z[0] == pytest.approx(2 * 675.0 - (674.99 + step), abs=1e-9)


def test_counts_conserved_batched():
    """image + off-image + active = N for every event, at every stage."""
    rng = np.random.default_rng(11)
    sizes = [5, 17, 40]
    xyz = np.concatenate([rng.normal(size=(n, 3)) * 0.4 + np.array([0, 0, z])
                          for n, z in zip(sizes, [3.0, 8.0, 1.0])])
    ev = np.concatenate([[0], np.cumsum(sizes)])
    p = O.make_params(img_w=8, img_h=8, pixel_um=1.0)
    sim = O.Simulation(p, xyz, ev, seeds=[1, 2, 3], img_origin=[[-4.0, -4.0]] * 3)
    for steps in (0, 50, 10 ** 6):
        sim.run(steps)
        act = sim.n_active()
        for e in range(3):
            assert int(sim.image[e].sum()) + int(sim.off_image[e]) + int(act[e]) == sizes[e]
    assert sim.n_active().sum() == 0


def test_event_independent_of_batch():
    """Events are independent (Sec. 5.1: one interaction produces one cloud):
    an event simulated alone and behind other events of a batch gives
    identical results, because its random vectors are keyed by its own seed
    and the carrier's index within the event."""
    rng = np.random.default_rng(13)
    a = rng.normal(size=(40, 3)) * 0.4 + np.array([0, 0, 6.0])
    b = rng.normal(size=(25, 3)) * 0.4 + np.array([0, 0, 3.0])
    p = O.make_params(img_w=8, img_h=8, pixel_um=2.0)
    alone = O.Simulation(p, a, seeds=[5], img_origin=[[-8.0, -8.0]])
    alone.run()
    both = O.Simulation(p, np.concatenate([b, a]), ev_off=[0, 25, 65], seeds=[9, 5],
                        img_origin=[[-8.0, -8.0]] * 2)
    both.run()
    assert np.array_equal(alone.positions(), both.positions()[25:])
    assert np.array_equal(alone.collect_step, both.collect_step[25:])
    assert np.array_equal(alone.image[0], both.image[1])


# ---- stored charge (Sec. 1: charge already in a pixel deflects later charges) -------------

def _stored_image():
    img = np.zeros((4, 5), dtype=np.uint32)
    img[1, 2], img[3, 0], img[0, 4] = 7, 2, 5
    return img, np.array([-30.0, -20.0])


def test_stored_field_is_minus_gradient_of_its_potential():
    """The stored-charge field is minus the gradient (central differences) of
    K sum_p q_p / sqrt(|r - c_p|^2 + eps^2) over the pixel centres c_p at
    (ox + (ix + 1/2) p, oy + (iy + 1/2) p, stored_z)."""
    p = O.make_params(img_w=5, img_h=4, pixel_um=15.0, softening_um=0.05, stored_z_um=-0.5)
    img, org = _stored_image()
    K = O.coulomb_K(11.7)
    iy, ix = np.nonzero(img)
    centres = np.stack([org[0] + (ix + 0.5) * 15.0, org[1] + (iy + 0.5) * 15.0,
                        np.full(len(ix), -0.5)], axis=1)
    q = img[iy, ix].astype(float)

    def phi(r):
        d = r[None, :] - centres
        return K * np.sum(q / np.sqrt((d * d).sum(1) + 0.05 ** 2))

    pts = np.array([[3.0, -1.0, 4.0], [-22.0, 27.0, 0.7], [40.0, -15.0, 30.0]])
    E = O.stored_field(p, img, org, pts)
    h = 1e-5
    for t, r in enumerate(pts):
        for c in range(3):
            rp, rm = r.copy(), r.copy()
            rp[c] += h
            rm[c] -= h
            assert E[t, c] == pytest.approx(-(phi(rp) - phi(rm)) / (2 * h), rel=2e-6, abs=1e-9)


def test_stored_field_equals_point_sources_at_pixel_centres():
    """The same field as Eq. 6 from q_p carriers placed at each pixel centre."""
    p = O.make_params(img_w=5, img_h=4, pixel_um=15.0, stored_z_um=0.0)
    img, org = _stored_image()
    iy, ix = np.nonzero(img)
    src = np.concatenate([np.tile([[org[0] + (a + 0.5) * 15.0, org[1] + (b + 0.5) * 15.0, 0.0]],
                                  (int(img[b, a]), 1)) for b, a in zip(iy, ix)])
    pts = np.array([[1.0, 2.0, 3.0], [-10.0, 5.0, 0.2]])
    E = O.stored_field(p, img, org, pts)
    allp = np.concatenate([pts, src])
    ref = O.coulomb_field(allp, targets=[0, 1], src=np.arange(2, len(allp)))
    np.testing.assert_allclose(E, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_stored_charge_one_step_closed_form_and_off_switch():
    """A hole above a pixel holding q collected holes (no depletion field, no
    diffusion) moves by 1e4 mu(|E|) E dt with E the stored-charge field; with
    stored_charge = 0 the collected charge exerts nothing."""
    K = O.coulomb_K(11.7)
    q = 40
    # q holes start in the well under pixel (1, 1) of a 3 x 3 image; one hole at 2 um above it
    centre = np.array([-7.5, -7.5]) + 1.5 * 15.0
    xyz = np.concatenate([np.tile([[centre[0], centre[1], -0.1]], (q, 1)),
                          [[centre[0] + 1.0, centre[1], 2.0]]])
    for stored in (0, 1):
        p = O.make_params(a1=0.0, a2=0.0, diffusion=0, coulomb=1, img_w=3, img_h=3, pixel_um=15.0,
                          stored_charge=stored, stored_z_um=-0.1, z_well_um=-0.05)
        sim = O.Simulation(p, xyz, img_origin=[[-7.5, -7.5]])
        assert sim.image[0, 1, 1] == q  # collected at step 0
        sim.run(1)
        d = np.array([1.0, 0.0, 2.1])
        E = stored * K * q * d / (d @ d + 1e-4) ** 1.5
        mu = O.mobility(np.linalg.norm(E), 140.0)
        want = np.array([centre[0] + 1.0, centre[1], 2.0]) + 1e4 * mu * E * 1e-11
        np.testing.assert_allclose(sim.positions()[-1], want, rtol=1e-12, atol=1e-12)


def test_stored_charge_broadens_the_image():
    """Sec. 1: charge already stored deflects the charges that follow, so a
    dense cloud ends wider with the stored-charge field on."""
    rng = np.random.default_rng(2)
    xyz = rng.normal(size=(600, 3)) * 0.3 + np.array([0.0, 0.0, 40.0])
    sig = []
    for stored in (0, 1):
        p = O.make_params(img_w=16, img_h=16, pixel_um=3.0, stored_charge=stored, stored_z_um=0.0)
        sim = O.Simulation(p, xyz, img_origin=[[-24.0, -24.0]])
        sim.run()
        sig.append(np.hypot(sim.x.std(), sim.y.std()))
    assert sig[1] > sig[0] * 1.001


def test_step_targets_matches_a_committed_step():
    """The sampled large-N parity tests take their expected positions from
    step_targets.  It shares the field and update routines with orc_run, so
    this is no physics pin: it checks the helper's own indexing (targets,
    sources, step counter, per-event random-number index) against a committed
    step of a single event, bit for bit, for every hole active before it."""
    rng = np.random.default_rng(12)
    xyz = np.array([0.0, 0.0, 4.0]) + 1.5 * rng.standard_normal((300, 3))
    xyz[:5, 2] = 674.0 + rng.random(5)                  # near the back surface: reflections
    p = O.make_params(img_w=16, img_h=16)
    sim = O.Simulation(p, xyz, seeds=np.array([77], dtype=np.uint64))
    sim.run(3)
    x0 = sim.positions().copy()
    active = np.nonzero(sim.collect_step < 0)[0]
    assert 0 < len(active) < len(xyz)
    want = O.step_targets(p, x0, active, active, 77, sim.step + 1)
    sim.run(1)
    assert np.any(sim.collect_step == sim.step)          # some holes were collected in this step
    assert np.array_equal(sim.positions()[active], want)
