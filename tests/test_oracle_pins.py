"""Pins for the CPU oracle: checks against facts the mathematics fixes, never against itself.

Each test names what it pins.  A plausible slip in the oracle (a dropped term, a sign, a swapped
sinh/cosh, a transposed matrix, a wrong packing index) fails at least one of them:
  * hand-derived cases (tests/golden/hand_cases.txt),
  * the massless closed form m^2 = 2 pt1 pt2 (cosh d_eta - cos d_phi) and its derivatives,
  * invariance of the pair mass under rotations about z and boosts along z (eta shifts),
  * agreement of the binary128 definition (O1) with the cancellation-free FP64 identity (O2),
  * boost inverse, rest frame, collinear velocity addition, metric preservation, mass invariance,
  * central finite differences for the gradients,
  * integer prefix sums and pair enumeration for the jagged form.
"""
import math
import os

import numpy as np
import pytest

import gvx_synth as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.txt")


def _golden_rows(kind):
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line.startswith(kind + " "):
                rows.append([float(x) for x in line.split()[1:]])
    assert rows
    return rows


def test_binary128(orc):
    assert orc.precision_bits() == 113


# ------------------------------------------------------------------------------------------ mass

def test_mass_hand_cases(orc):
    for r in _golden_rows("mass"):
        a, b, want, rtol, atol = np.array(r[0:4]), np.array(r[4:8]), r[8], r[9], r[10]
        for m in (orc.mass_def(a, b)[0], orc.mass_fp64(a, b)[0]):
            assert abs(m - want) <= rtol * abs(want) + atol, (r, m)


def _massless_pairs(n, seed):
    g = syn.rng(seed)
    a, b = syn.ptetaphim(g, n), syn.ptetaphim(g, n)
    a[:, 3] = 0.0
    b[:, 3] = 0.0
    return a, b


def test_mass_massless_closed_form(orc):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    a, b = _massless_pairs(400, 101)
    got1, got2 = orc.mass_def(a, b), orc.mass_fp64(a, b)
    for i in range(len(a)):
        pt1, e1, f1, _ = (mp.mpf(x) for x in a[i])
        pt2, e2, f2, _ = (mp.mpf(x) for x in b[i])
        want = float(mp.sqrt(2 * pt1 * pt2 * (mp.cosh(e1 - e2) - mp.cos(f1 - f2))))
        assert abs(got1[i] - want) <= 2.5e-16 * want
        assert abs(got2[i] - want) <= 4e-15 * want


def test_mass_symmetric_and_invariant(orc):
    g = syn.rng(102)
    a, b = syn.ptetaphim(g, 2000), syn.ptetaphim(g, 2000)
    m = orc.mass_def(a, b)
    assert np.array_equal(m, orc.mass_def(b, a))
    # a rotation about z (phi -> phi + alpha) leaves m unchanged; for massless legs eta is the
    # rapidity, so a boost along z (eta -> eta + y) does too.  The shifted inputs are rounded,
    # so compare at the conditioning of the angular term.
    a0, b0 = a.copy(), b.copy()
    a0[:, 3] = 0.0
    b0[:, 3] = 0.0
    for (x, y), col, shift in (((a, b), 2, 0.7), ((a0, b0), 1, 0.3)):
        m = orc.mass_def(x, y)
        x2, y2 = x.copy(), y.copy()
        x2[:, col] += shift
        y2[:, col] += shift
        m2 = orc.mass_def(x2, y2)
        E = x[:, 0] * np.cosh(x[:, 1]) + y[:, 0] * np.cosh(y[:, 1]) + x[:, 3] + y[:, 3]
        tol = 1e-14 * m + 1e-15 * E * E / np.maximum(m, 1e-300)
        assert np.all(np.abs(m2 - m) <= tol)
    # for massive legs an eta shift is not a boost: it must change m (guards a mass term dropped)
    a2, b2 = a.copy(), b.copy()
    a2[:, 1] += 0.3
    b2[:, 1] += 0.3
    assert np.median(np.abs(orc.mass_def(a2, b2) / orc.mass_def(a, b) - 1)) > 1e-6


def _adversarial_pairs(n, seed):
    """Near-collinear, light legs: the E^2/m^2 cancellation regime."""
    g = syn.rng(seed)
    a = syn.ptetaphim(g, n)
    a[:, 0] = np.exp(g.uniform(np.log(50), np.log(1000), n))
    a[:, 3] = g.uniform(0, 1e-2, n)
    b = a.copy()
    b[:, 0] *= np.exp(g.uniform(-1, 1, n))
    b[:, 1] += g.choice([1e-7, 1e-5, 1e-3], n) * g.uniform(-1, 1, n)
    b[:, 2] += g.choice([1e-7, 1e-5, 1e-3], n) * g.uniform(-1, 1, n)
    b[:, 3] = g.uniform(0, 1e-2, n)
    return a, b


def test_mass_definition_vs_identity(orc):
    """O1 (binary128 definition) and O2 (FP64 all-positive identity) are different formulas."""
    g = syn.rng(103)
    a, b = syn.ptetaphim(g, 20000), syn.ptetaphim(g, 20000)
    rel = np.abs(orc.mass_fp64(a, b) / orc.mass_def(a, b) - 1)
    assert rel.max() <= 1e-14
    a, b = _adversarial_pairs(20000, 104)
    m1 = orc.mass_def(a, b)
    rel = np.abs(orc.mass_fp64(a, b) / m1 - 1)
    assert rel.max() <= 1e-14
    # the plain definition in double is not good enough on these pairs: this is why O1 runs in
    # binary128 (information, but also a check that the adversarial set is adversarial)
    naive = np.abs(orc.mass_naive_fp64(a, b) / m1 - 1)
    assert naive.max() > 1e-9
    # azimuths on either side of +-pi, 2 pi - |d_phi| down to 1e-8 (massless legs at equal eta,
    # where the azimuthal term is the whole mass): O2's half-angle from exact brackets; the
    # rounded phi1 - phi2 (~4e-16 absolute) would be off by up to ~1e-8 relative here.  Compared
    # where O1 itself keeps 1e-14 (m >= 1e-9 (E1 + E2)).
    g = syn.rng(106)
    n = 4000
    a, b = syn.ptetaphim(g, n), syn.ptetaphim(g, n)
    a[:, 1] = g.uniform(-1, 1, n)
    b[:, 1] = a[:, 1]
    gap = 10 ** g.uniform(-8, -1, n)
    a[:, 2] = np.pi - gap * g.random(n)
    b[:, 2] = -np.pi + gap * g.random(n)
    a[::2, 3] = 0.0
    b[::2, 3] = 0.0
    m1 = orc.mass_def(a, b)
    e = lambda x: np.sqrt((x[:, 0] * np.cosh(x[:, 1])) ** 2 + x[:, 3] ** 2)
    cond = m1 >= 1e-9 * (e(a) + e(b))
    assert cond.mean() > 0.9
    rel = np.abs(orc.mass_fp64(a, b)[cond] / m1[cond] - 1)
    assert rel.max() <= 1e-14


def test_mass_threads_agree(orc):
    g = syn.rng(105)
    a, b = syn.ptetaphim(g, 5000), syn.ptetaphim(g, 5000)
    assert np.array_equal(orc.mass_def(a, b, 1), orc.mass_def(a, b, 4))
    assert np.array_equal(orc.mass_fp64(a, b, 1), orc.mass_fp64(a, b, 3))


# ------------------------------------------------------------------------------------ mass grad

def test_mass_grad_massless_closed_form(orc):
    """m = sqrt(2 pt1 pt2 (cosh d - cos f)):  dm/dpt1 = m/(2 pt1),
    dm/deta1 = pt1 pt2 sinh(d)/m, dm/dphi1 = pt1 pt2 sin(f)/m, with d = eta1-eta2, f = phi1-phi2;
    the derivative in m1 at m1 = 0 is 0."""
    a, b = _massless_pairs(300, 106)
    gm = syn.upstream(syn.rng(107), 300)
    ga, gb = orc.mass_grad_def(a, b, gm)
    m = orc.mass_def(a, b)
    d, f = a[:, 1] - b[:, 1], a[:, 2] - b[:, 2]
    pp = a[:, 0] * b[:, 0]
    want_a = np.stack([m / (2 * a[:, 0]), pp * np.sinh(d) / m, pp * np.sin(f) / m,
                       np.zeros_like(m)], axis=1) * gm[:, None]
    want_b = np.stack([m / (2 * b[:, 0]), -pp * np.sinh(d) / m, -pp * np.sin(f) / m,
                       np.zeros_like(m)], axis=1) * gm[:, None]
    scale = np.abs(want_a).max(axis=1, keepdims=True)
    assert np.all(np.abs(ga - want_a) <= 1e-12 * scale)
    assert np.all(np.abs(gb - want_b) <= 1e-12 * scale)


def test_mass_grad_finite_differences(orc):
    g = syn.rng(108)
    n = 200
    a, b = syn.ptetaphim(g, n), syn.ptetaphim(g, n)
    gm = syn.upstream(g, n)
    ga, gb = orc.mass_grad_def(a, b, gm)
    for legs, grad, which in ((a, ga, 0), (b, gb, 1)):
        for k in range(4):
            h = 1e-6 * np.maximum(np.abs(legs[:, k]), 1.0)
            hi, lo = legs.copy(), legs.copy()
            hi[:, k] += h
            lo[:, k] -= h
            if which == 0:
                fd = (orc.mass_def(hi, b) - orc.mass_def(lo, b)) / (hi[:, k] - lo[:, k])
            else:
                fd = (orc.mass_def(a, hi) - orc.mass_def(a, lo)) / (hi[:, k] - lo[:, k])
            fd *= gm
            scale = np.abs(grad).max(axis=1) + 1e-300
            assert np.all(np.abs(fd - grad[:, k]) <= 2e-6 * scale), (which, k)


def test_mass_grad_leg_symmetry_and_zero_mass(orc):
    g = syn.rng(109)
    a, b = syn.ptetaphim(g, 500), syn.ptetaphim(g, 500)
    gm = syn.upstream(g, 500)
    ga, gb = orc.mass_grad_def(a, b, gm)
    gb2, ga2 = orc.mass_grad_def(b, a, gm)
    assert np.array_equal(ga, ga2) and np.array_equal(gb, gb2)
    # m = 0 (collinear massless legs): zero subgradient
    z = np.array([[10.0, 0.7, -1.0, 0.0]])
    ga, gb = orc.mass_grad_def(z, z * [2, 1, 1, 1], [1.0])
    assert abs(orc.mass_def(z, z * [2, 1, 1, 1])[0]) < 1e-12
    assert np.all(np.abs(ga) <= 1e-3) and np.all(np.abs(gb) <= 1e-3)


# ----------------------------------------------------------------------------------------- boost

def test_boost_hand_cases(orc):
    for r in _golden_rows("boost"):
        v, beta, want, rtol = np.array(r[0:4]), np.array(r[4:7]), np.array(r[7:11]), r[11]
        for out in (orc.boost_def(v, beta)[0], orc.boost_fp64(v, beta)[0]):
            assert np.all(np.abs(out - want) <= rtol * want[3]), (r, out)
    v = np.array([[1.0, 2.0, 3.0, 10.0]])
    assert np.array_equal(orc.boost_def(v, np.zeros(3)), v)


def _kappa(beta):
    b = np.sqrt(np.sum(beta * beta, axis=-1))
    return (1 + b) / (1 - b)


def test_boost_inverse_and_rest_frame(orc):
    g = syn.rng(110)
    n = 3000
    v = syn.pxpypze(g, n)
    beta = syn.velocities(g, n, 0.99)
    out = orc.boost_def(v, beta)
    back = orc.boost_def(out, -beta)
    k = _kappa(beta)
    assert np.all(np.abs(back - v).max(axis=1) <= 4e-16 * k * k * v[:, 3])
    # rest frame of v: boosting by -p/E leaves (0, 0, 0, m)
    rest = orc.boost_def(v, -v[:, :3] / v[:, 3:4])
    m = orc.lv_mass_def(v)
    gam = v[:, 3] / np.maximum(m, 1e-300)
    ok = gam < 1e6
    err = np.abs(rest - np.stack([0 * m, 0 * m, 0 * m, m], axis=1)).max(axis=1)
    assert np.all(err[ok] <= 1e-15 * v[ok, 3] * gam[ok] + 1e-13 * m[ok])


def test_boost_velocity_addition(orc):
    """Two boosts along one axis compose to one with (b1 + b2)/(1 + b1 b2)."""
    g = syn.rng(111)
    n = 2000
    v = syn.pxpypze(g, n)
    u = syn.velocities(g, n, 1.0)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    b1, b2 = g.uniform(-0.9, 0.9, n), g.uniform(-0.9, 0.9, n)
    two = orc.boost_def(orc.boost_def(v, u * b1[:, None]), u * b2[:, None])
    one = orc.boost_def(v, u * ((b1 + b2) / (1 + b1 * b2))[:, None])
    ab1, ab2 = np.abs(b1), np.abs(b2)
    k = ((1 + ab1) / (1 - ab1) * (1 + ab2) / (1 - ab2))[:, None]
    assert np.all(np.abs(two - one) <= 1e-15 * k * v[:, 3:4])


def test_boost_matrix_preserves_metric(orc):
    g = syn.rng(112)
    G = np.diag([-1.0, -1.0, -1.0, 1.0])
    for beta in syn.velocities(g, 200, 0.999):
        L = orc.boost_matrix_def(beta)
        assert np.allclose(L, L.T, rtol=0, atol=0)
        gam = L[3, 3]
        assert np.abs(L.T @ G @ L - G).max() <= 1e-14 * gam * gam
        # the double-precision comparison value carries the conditioning of 1 - b2 (~gamma^2)
        assert abs(gam - 1 / math.sqrt(1 - float(beta @ beta))) <= 1e-15 * gam ** 3


def test_boost_preserves_mass(orc):
    g = syn.rng(113)
    n = 2000
    v = syn.pxpypze(g, n)
    v[:, 3] = np.sqrt(np.sum(v[:, :3] ** 2, axis=1) + (0.5 * np.linalg.norm(v[:, :3], axis=1)) ** 2)
    beta = syn.velocities(g, n, 0.9)
    m0 = orc.lv_mass_def(v)
    m1 = orc.lv_mass_def(orc.boost_def(v, beta))
    assert np.all(np.abs(m1 / m0 - 1) <= 1e-13)


def test_boost_definition_vs_vector_form(orc):
    g = syn.rng(114)
    n = 20000
    v = syn.pxpypze(g, n)
    beta = syn.velocities(g, n, 0.99)
    o1, o2 = orc.boost_def(v, beta), orc.boost_fp64(v, beta)
    assert np.all(np.abs(o1 - o2).max(axis=1) <= 1e-14 * o1[:, 3])
    shared = beta[7]
    assert np.array_equal(orc.boost_def(v, shared), orc.boost_def(v, np.tile(shared, (n, 1))))


def test_boost_superluminal_is_nan(orc):
    v = np.array([[1.0, 2.0, 3.0, 10.0]])
    for beta in ([1.0, 0, 0], [0.8, 0.8, 0], [0, 0, -2.0]):
        assert np.all(np.isnan(orc.boost_def(v, np.array(beta))))
        assert np.all(np.isnan(orc.boost_fp64(v, np.array(beta))))


def test_boost_grad_finite_differences(orc):
    g = syn.rng(115)
    n = 200
    v = syn.pxpypze(g, n) / 100.0
    beta = syn.velocities(g, n, 0.9)
    gout = syn.upstream(g, (n, 4))
    gv, gb = orc.boost_grad_def(v, beta, gout)

    def f(vv, bb):
        return np.sum(orc.boost_def(vv, bb) * gout, axis=1)

    for k in range(4):
        h = 1e-6 * np.maximum(np.abs(v[:, k]), 1.0)
        hi, lo = v.copy(), v.copy()
        hi[:, k] += h
        lo[:, k] -= h
        fd = (f(hi, beta) - f(lo, beta)) / (hi[:, k] - lo[:, k])
        assert np.all(np.abs(fd - gv[:, k]) <= 1e-7 * np.abs(gv).max(axis=1))
    for k in range(3):
        h = 1e-7
        hi, lo = beta.copy(), beta.copy()
        hi[:, k] += h
        lo[:, k] -= h
        fd = (f(v, hi) - f(v, lo)) / (hi[:, k] - lo[:, k])
        assert np.all(np.abs(fd - gb[:, k]) <= 1e-6 * np.abs(gb).max(axis=1))
    # shared velocity: its gradient is the sum of the per-vector ones
    gv_s, gb_s = orc.boost_grad_def(v, beta[3], gout)
    gv_t, gb_t = orc.boost_grad_def(v, np.tile(beta[3], (n, 1)), gout)
    assert np.array_equal(gv_s, gv_t)
    assert np.allclose(gb_s, gb_t.sum(axis=0), rtol=1e-14, atol=0)
    # beta = 0: grad_v = gout (identity), grad_beta_k = gout_k E + gout_t p_k
    gv0, gb0 = orc.boost_grad_def(v, np.zeros((n, 3)), gout)
    assert np.array_equal(gv0, gout)
    t1, t2 = gout[:, :3] * v[:, 3:4], gout[:, 3:4] * v[:, :3]
    assert np.all(np.abs(gb0 - (t1 + t2)) <= 4e-16 * (np.abs(t1) + np.abs(t2)))


# ---------------------------------------------------------------------------------------- jagged

def test_event_pairs(orc):
    g = syn.rng(116)
    off = syn.jagged_offsets(g, 300, lam=4.0, n_max=12)
    off = np.concatenate([off, off[-1:] + [0, 1, 3, 6]])  # append events of size 0, 1, 2, 3
    p = syn.ptetaphim(g, int(off[-1]))
    pair_off, pair_m, sums = orc.event_pairs_def(p, off)
    counts = np.diff(off)
    want_off = np.concatenate([[0], np.cumsum(counts * (counts - 1) // 2)])
    assert np.array_equal(pair_off, want_off)
    assert pair_m.shape[0] == want_off[-1]
    cart = orc.to_cartesian_def(p)
    for e in range(len(counts)):
        n, base = counts[e], off[e]
        ii, jj = np.triu_indices(n, 1)  # row-major i < j
        got = pair_m[pair_off[e]:pair_off[e + 1]]
        assert np.array_equal(got, orc.mass_def(p[base + ii], p[base + jj]))
        want_sum = cart[base:base + n].sum(axis=0) if n else np.zeros(4)
        assert np.all(np.abs(sums[e] - want_sum) <= 1e-15 * (np.abs(cart[base:base + n]).sum() + 1e-300))
        if n == 2:  # the event's total mass is its one pair mass
            assert abs(orc.lv_mass_def(sums[e])[0] - got[0]) <= 1e-9 * got[0] + 1e-9
    # the multi-body mass of the last (3-particle) event from the pair masses:
    # M^2 = sum_{i<j} m_ij^2 - (n-2) sum_i m_i^2
    e = len(counts) - 1
    mi = p[off[e]:off[e + 1], 3]
    M2 = np.sum(pair_m[pair_off[e]:pair_off[e + 1]] ** 2) - (3 - 2) * np.sum(mi ** 2)
    assert abs(orc.lv_mass_def(sums[e])[0] ** 2 - M2) <= 1e-9 * M2


def test_event_pairs_rejects_bad_offsets(orc):
    p = syn.ptetaphim(syn.rng(117), 5)
    with pytest.raises(ValueError):
        orc.event_pairs_def(p, [0, 3, 2, 5])
    with pytest.raises(ValueError):
        orc.event_pairs_def(p, [0, 2, 4])


def _event_losses(orc, p, off, gpm, gsum):
    """Per-event L_e = sum of gpm * pair masses + gsum . event sum, from the forward oracle."""
    pair_off, pair_m, sums = orc.event_pairs_def(p, off)
    n_ev = len(off) - 1
    pair_ev = np.repeat(np.arange(n_ev), np.diff(pair_off))
    L = np.bincount(pair_ev, weights=gpm * pair_m, minlength=n_ev)
    return L + np.sum(gsum * sums, axis=1)


def test_event_pairs_grad_finite_differences(orc):
    """Central differences of the forward oracle's per-event losses.  Events are independent, so
    perturbing the r-th particle of every event at once gives each event's derivative in one
    pair of forward calls."""
    g = syn.rng(118)
    off = syn.jagged_offsets(g, 80, lam=4.0, n_max=8)
    off = np.concatenate([off, off[-1:] + [0, 1, 3, 6]])
    p = syn.ptetaphim(g, int(off[-1]))
    counts = np.diff(off)
    n_pairs = int(np.sum(counts * (counts - 1) // 2))
    gpm, gsum = syn.upstream(g, n_pairs), syn.upstream(g, (len(counts), 4))
    grad = orc.event_pairs_grad_def(p, off, gpm, gsum)
    for r in range(counts.max()):
        ev = np.flatnonzero(counts > r)
        idx = off[ev] + r
        for k in range(4):
            h = 1e-6 * np.maximum(np.abs(p[idx, k]), 1.0)
            hi, lo = p.copy(), p.copy()
            hi[idx, k] += h
            lo[idx, k] -= h
            fd = (_event_losses(orc, hi, off, gpm, gsum) - _event_losses(orc, lo, off, gpm, gsum))[ev]
            fd /= hi[idx, k] - lo[idx, k]
            scale = np.abs(grad[idx]).max(axis=1) + np.abs(gsum[ev]).sum(axis=1) * 10
            assert np.all(np.abs(fd - grad[idx, k]) <= 2e-6 * scale), (r, k)


def test_event_pairs_grad_sum_part_closed_form(orc):
    """With only an event-sum gradient along one axis, each particle gets one row of the
    PtEtaPhiM -> PxPyPzE Jacobian: d px = (cos phi, 0, -pt sin phi, 0), d pz = (sinh eta,
    pt cosh eta, 0, 0), d E = (pt cosh^2 eta, pt^2 cosh eta sinh eta, 0, m) / E."""
    g = syn.rng(119)
    off = syn.jagged_offsets(g, 50, lam=5.0, n_max=10)
    p = syn.ptetaphim(g, int(off[-1]))
    counts = np.diff(off)
    gpm = np.zeros(int(np.sum(counts * (counts - 1) // 2)))
    pt, eta, phi, m = p.T
    ch, sh = np.cosh(eta), np.sinh(eta)
    E = np.sqrt((pt * ch) ** 2 + m ** 2)
    zero = np.zeros_like(pt)
    want = {0: np.stack([np.cos(phi), zero, -pt * np.sin(phi), zero], axis=1),
            2: np.stack([sh, pt * ch, zero, zero], axis=1),
            3: np.stack([pt * ch * ch / E, pt * pt * ch * sh / E, zero, m / E], axis=1)}
    for axis, w in want.items():
        gsum = np.zeros((len(counts), 4))
        gsum[:, axis] = 1.0
        got = orc.event_pairs_grad_def(p, off, gpm, gsum)
        assert np.all(np.abs(got - w) <= 1e-14 * np.abs(w).max(axis=1, keepdims=True)), axis


def test_event_pairs_grad_massless_pairs_closed_form(orc):
    """Two-particle events of massless legs: m = sqrt(2 pt1 pt2 (cosh d - cos f)) gives
    dm/dpt1 = m/(2 pt1), dm/deta1 = pt1 pt2 sinh(d)/m, dm/dphi1 = pt1 pt2 sin(f)/m, dm/dm1 = 0,
    and the opposite signs of the angle terms for the second particle."""
    a, b = _massless_pairs(200, 120)
    p = np.empty((400, 4))
    p[0::2], p[1::2] = a, b
    off = np.arange(0, 401, 2)
    gpm = syn.upstream(syn.rng(121), 200)
    got = orc.event_pairs_grad_def(p, off, gpm)
    m = orc.mass_def(a, b)
    d, f = a[:, 1] - b[:, 1], a[:, 2] - b[:, 2]
    pp = a[:, 0] * b[:, 0]
    zero = np.zeros_like(m)
    want_a = np.stack([m / (2 * a[:, 0]), pp * np.sinh(d) / m, pp * np.sin(f) / m, zero], axis=1)
    want_b = np.stack([m / (2 * b[:, 0]), -pp * np.sinh(d) / m, -pp * np.sin(f) / m, zero], axis=1)
    for got_l, w in ((got[0::2], want_a), (got[1::2], want_b)):
        w = w * gpm[:, None]
        assert np.all(np.abs(got_l - w) <= 1e-12 * np.abs(w).max(axis=1, keepdims=True))


def test_event_pairs_grad_permutation(orc):
    """Reordering the particles of every event (and the pair gradients with them) reorders the
    particle gradients."""
    g = syn.rng(122)
    off = syn.jagged_offsets(g, 60, lam=6.0, n_max=12)
    p = syn.ptetaphim(g, int(off[-1]))
    counts = np.diff(off)
    n_pairs = int(np.sum(counts * (counts - 1) // 2))
    gpm, gsum = syn.upstream(g, n_pairs), syn.upstream(g, (len(counts), 4))
    grad = orc.event_pairs_grad_def(p, off, gpm, gsum)
    perm = np.arange(len(p))
    gpm2 = np.empty_like(gpm)
    pbase = 0
    for e, n in enumerate(counts):
        local = g.permutation(n)  # new position q holds old particle local[q]
        perm[off[e]:off[e + 1]] = off[e] + local
        ii, jj = np.triu_indices(n, 1)
        old = {}
        for k, (i, j) in enumerate(zip(ii, jj)):
            old[(i, j)] = gpm[pbase + k]
        for k, (i, j) in enumerate(zip(ii, jj)):
            a, b = sorted((local[i], local[j]))
            gpm2[pbase + k] = old[(a, b)]
        pbase += n * (n - 1) // 2
    grad2 = orc.event_pairs_grad_def(p[perm], off, gpm2, gsum)
    assert np.all(np.abs(grad2 - grad[perm]) <= 1e-15 * np.abs(grad[perm]).max(axis=1, keepdims=True))


def test_event_pairs_grad_rejects_bad_input(orc):
    p = syn.ptetaphim(syn.rng(123), 5)
    with pytest.raises(ValueError):
        orc.event_pairs_grad_def(p, [0, 3, 2, 5], np.zeros(4))
    with pytest.raises(ValueError):
        orc.event_pairs_grad_def(p, [0, 2, 5], np.zeros(3))  # 1 + 3 pairs expected


# ------------------------------------------------------------- fused selection + histogram

def _mp_pair_mass(mp, a, b):
    """The pair mass from the definition in mpmath (50 digits)."""
    def cart(x):
        pt, eta, phi, m = (mp.mpf(float(v)) for v in x)
        px, py, pz = pt * mp.cos(phi), pt * mp.sin(phi), pt * mp.sinh(eta)
        return px, py, pz, mp.sqrt(px * px + py * py + pz * pz + m * m)
    u, w = cart(a), cart(b)
    s = [u[k] + w[k] for k in range(4)]
    return mp.sqrt(s[3] ** 2 - s[0] ** 2 - s[1] ** 2 - s[2] ** 2)


def test_pair_select_brute_force_mpmath(orc):
    """Counts and best candidates against a brute-force loop with masses in mpmath: the slot of
    every pair from its 50-digit mass rounded to double, the best pair from exact |m - target|."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    g = syn.rng(124)
    off = syn.jagged_offsets(g, 40, lam=4.0, n_max=7)
    p = syn.ptetaphim(g, int(off[-1]))
    pt_min, eta_max, lo, hi, nb, target = 15.0, 2.0, 0.0, 300.0, 30, 91.1876
    counts, near, bk, bm = orc.pair_select_def(p, off, pt_min, eta_max, lo, hi, nb, target)
    want = np.zeros(nb + 2, dtype=np.uint64)
    inv_w = nb / (hi - lo)
    for e in range(len(off) - 1):
        best = None
        k = 0
        n = off[e + 1] - off[e]
        for i in range(n):
            for j in range(i + 1, n):
                a, b = p[off[e] + i], p[off[e] + j]
                if a[0] >= pt_min and abs(a[1]) <= eta_max and b[0] >= pt_min and abs(b[1]) <= eta_max:
                    mq = _mp_pair_mass(mp, a, b)
                    m = float(mq)
                    slot = 0 if m < lo else nb + 1 if m >= hi else 1 + min(int(np.floor((m - lo) * inv_w)), nb - 1)
                    want[slot] += 1
                    d = abs(mq - target)
                    if best is None or d < best[0]:
                        best = (d, k, m)
                k += 1
        assert bk[e] == (best[1] if best else -1), e
        if best:
            assert abs(bm[e] - best[2]) <= 1e-15 * best[2]
        else:
            assert np.isnan(bm[e])
    assert near.sum() == 0  # no mass of this sample sits on a bin edge
    assert np.array_equal(counts, want)


def test_pair_select_invariants(orc):
    """Every passing pair is counted once (total = sum over events of C(n_pass, 2)); no cut
    counts all pairs and one bin over everything holds them all; an impossible cut counts
    nothing and leaves every event without a candidate."""
    g = syn.rng(125)
    off = syn.jagged_offsets(g, 500, lam=6.0, n_max=20)
    p = syn.ptetaphim(g, int(off[-1]))
    counts, _, bk, _ = orc.pair_select_def(p, off, 30.0, 1.5, 0.0, 500.0, 50, 91.19)
    passing = (p[:, 0] >= 30.0) & (np.abs(p[:, 1]) <= 1.5)
    n_pass = np.add.reduceat(passing.astype(np.int64), off[:-1]) if len(p) else 0
    n_pass = np.where(np.diff(off) > 0, n_pass, 0)
    assert int(counts.sum()) == int(np.sum(n_pass * (n_pass - 1) // 2))
    assert np.array_equal(bk >= 0, n_pass >= 2)
    c = np.diff(off)
    counts, _, bk, _ = orc.pair_select_def(p, off, 0.0, np.inf, 0.0, 1e9, 1, 91.19)
    assert counts[1] == np.sum(c * (c - 1) // 2) and counts[0] == 0 and counts[2] == 0
    counts, _, bk, bm = orc.pair_select_def(p, off, 1e9, np.inf, 0.0, 1e9, 4, 91.19)
    assert counts.sum() == 0 and np.all(bk == -1) and np.all(np.isnan(bm))


def test_pair_select_hand_case_and_ties(orc):
    """Two massless particles back to back at eta = 0 with pt = 45.5 have m = 91 exactly (bin
    91 of 1-GeV bins); a duplicated particle makes two pairs with equal masses, and the smaller
    packed index wins the tie."""
    p = np.array([[45.5, 0.0, 0.0, 0.0], [45.5, 0.0, -np.pi, 0.0], [10.0, 0.0, 0.5, 0.0],
                  [20.0, 0.3, 1.0, 0.0], [20.0, 0.3, 1.0, 0.0], [35.0, -0.4, -2.0, 0.0]])
    off = np.array([0, 3, 6])
    counts, near, bk, bm = orc.pair_select_def(p, off, 0.0, np.inf, 0.0, 200.0, 200, 91.0)
    assert bk[0] == 0 and abs(bm[0] - 91.0) <= 1e-13  # k(0, 1) = 0
    assert counts[1 + 91] >= 1 or near[1 + 91] + near[1 + 90] >= 1
    # event 1: particles 0 and 1 identical, so pairs (0, 2) and (1, 2) have the same mass
    m02 = orc.mass_def(p[3:4], p[5:6])[0]
    counts, _, bk, bm = orc.pair_select_def(p, off, 0.0, np.inf, 0.0, 200.0, 20, m02)
    assert bk[1] == 1 and bm[1] == m02  # k(0, 2) = 1 beats k(1, 2) = 2
    # the cuts are inclusive: pt = pt_min and |eta| = eta_max pass (event 0: one pair, event 1:
    # three pairs)
    counts, _, _, _ = orc.pair_select_def(p, off, 20.0, 0.4, 0.0, 200.0, 20, 91.0)
    assert counts.sum() == 4


# ------------------------------------------------- other coordinate systems, general transformations

def _mp_matvec(mp, L, v):
    return [sum(mp.mpf(float(L[r, k])) * mp.mpf(float(v[k])) for k in range(4)) for r in range(4)]


def test_lorentz_apply_identity_rotation_and_brute_force(orc):
    """The identity returns the input exactly; a rotation about z matches its closed form; on
    random matrices every component equals the 50-digit product rounded (within one ulp); a
    per-vector matrix array gives each vector its own matrix."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    g = syn.rng(126)
    v = syn.pxpypze(g, 200)
    assert np.array_equal(orc.lorentz_apply_def(np.eye(4), v), v)
    th = 0.7
    R = np.eye(4)
    R[0, 0], R[0, 1], R[1, 0], R[1, 1] = np.cos(th), -np.sin(th), np.sin(th), np.cos(th)
    out = orc.lorentz_apply_def(R, v)
    want = np.stack([v[:, 0] * R[0, 0] + v[:, 1] * R[0, 1], v[:, 0] * R[1, 0] + v[:, 1] * R[1, 1],
                     v[:, 2], v[:, 3]], axis=1)
    assert np.all(np.abs(out - want) <= 4e-16 * np.abs(v).sum(axis=1, keepdims=True))
    Ls = g.uniform(-2, 2, (50, 4, 4))
    out = orc.lorentz_apply_def(Ls, v[:50])
    for i in range(50):
        ref = _mp_matvec(mp, Ls[i], v[i])
        for r in range(4):
            assert abs(out[i, r] - float(ref[r])) <= np.spacing(abs(float(ref[r]))), (i, r)


def test_lorentz_apply_composition_and_metric(orc):
    """L1 (L2 v) = (L1 L2) v up to rounding (the product taken in mpmath), and a boost matrix
    keeps the mass of the vector."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    g = syn.rng(127)
    v = syn.pxpypze(g, 100)
    L1 = orc.boost_matrix_def(np.array([0.3, -0.2, 0.5]))
    L2 = orc.boost_matrix_def(np.array([-0.6, 0.1, 0.0]))
    L12 = np.array([[float(sum(mp.mpf(L1[r, k]) * mp.mpf(L2[k, c]) for k in range(4)))
                     for c in range(4)] for r in range(4)])
    a = orc.lorentz_apply_def(L1, orc.lorentz_apply_def(L2, v))
    b = orc.lorentz_apply_def(L12, v)
    scale = np.abs(v).sum(axis=1, keepdims=True) * 10
    assert np.all(np.abs(a - b) <= 1e-14 * scale)
    m0, m1 = orc.lv_mass_def(v), orc.lv_mass_def(orc.lorentz_apply_def(L1, v))
    assert np.all(np.abs(m1 - m0) <= 1e-10 * v[:, 3])


def _mp_cart_mass(mp, a, b, coords):
    def leg(x):
        px, py, pz, w = (mp.mpf(float(t)) for t in x)
        E = w if coords == "pxpypze" else mp.sqrt(px * px + py * py + pz * pz + w * w)
        return px, py, pz, E
    u, w = leg(a), leg(b)
    s = [u[k] + w[k] for k in range(4)]
    m2 = s[3] ** 2 - s[0] ** 2 - s[1] ** 2 - s[2] ** 2
    return mp.sqrt(m2) if m2 >= 0 else -mp.sqrt(-m2)


def test_mass_cart_brute_force_and_closed_form(orc):
    """Cartesian pair masses (E or m stored) against 50-digit brute force on random and
    near-collinear light pairs; massless legs (E = |p| exactly representable: Pythagorean
    momenta) against 2 (|p1||p2| - p1.p2) in closed form."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    g = syn.rng(128)
    v = syn.pxpypze(g, 400)
    a, b = v[:200], v[200:].copy()
    b[:50, :3] = a[:50, :3] * (1 + 1e-7)  # near-collinear
    b[:50, 3] = np.sqrt(np.sum(b[:50, :3] ** 2, axis=1) + 1e-6)
    for coords in ("pxpypze", "pxpypzm"):
        aa, bb = a.copy(), b.copy()
        if coords == "pxpypzm":
            aa[:, 3], bb[:, 3] = g.uniform(0, 10, 200), g.uniform(0, 1e-3, 200)
        m = orc.mass_cart_def(aa, bb, coords)
        for i in range(0, 200, 3):
            ref = _mp_cart_mass(mp, aa[i], bb[i], coords)
            assert abs(m[i] - float(ref)) <= 1e-15 * abs(float(ref)) + 1e-300, (coords, i)
    # massless legs: (3, 4, 12) has |p| = 13 exactly
    a = np.array([[3.0, 4.0, 12.0, 13.0], [0.0, 0.0, 5.0, 5.0]])
    b = np.array([[-4.0, 3.0, 12.0, 13.0], [0.0, 3.0, 4.0, 5.0]])
    m = orc.mass_cart_def(a, b)
    p1, p2 = a[:, :3], b[:, :3]
    want = np.sqrt(2 * (np.linalg.norm(p1, axis=1) * np.linalg.norm(p2, axis=1) - np.sum(p1 * p2, axis=1)))
    assert np.all(np.abs(m - want) <= 1e-15 * want)


def test_mass_cart_rotation_invariance(orc):
    """A rotation by 90 degrees about z maps doubles to doubles exactly and leaves every pair
    mass unchanged; the stored m of the PxPyPzM form enters through m^2 only."""
    g = syn.rng(129)
    v = syn.pxpypze(g, 600)
    a, b = v[:300], v[300:]
    rot = lambda x: np.stack([-x[:, 1], x[:, 0], x[:, 2], x[:, 3]], axis=1)
    assert np.array_equal(orc.mass_cart_def(a, b), orc.mass_cart_def(rot(a), rot(b)))
    am = a.copy()
    am[:, 3] = g.uniform(0, 10, 300)
    neg = am.copy()
    neg[:, 3] *= -1
    assert np.array_equal(orc.mass_cart_def(am, b, "pxpypzm"), orc.mass_cart_def(neg, b, "pxpypzm"))


def _mp_ptetaphie_leg(mp, x):
    pt, eta, phi, E = (mp.mpf(float(t)) for t in x)
    return [pt * mp.cos(phi), pt * mp.sin(phi), pt * mp.sinh(eta), E]


def test_ptetaphie_conversion_and_mass_brute_force(orc):
    """PtEtaPhiE legs (E stored) against 50-digit brute force: the conversion to PxPyPzE component
    by component (one rounding) and the pair mass of the converted sum, on random and on
    near-collinear pairs; the PtEtaPhiM conversion through the same entry agrees with
    to_cartesian_def bit for bit."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    g = syn.rng(190)
    p = syn.ptetaphim(g, 300)
    cart = orc.to_cartesian_def(p)
    legs = p.copy()
    legs[:, 3] = cart[:, 3]  # on-shell energies of the PtEtaPhiM draws
    out = orc.to_pxpypze_def(legs, "ptetaphie")
    for i in range(0, 300, 7):
        ref = _mp_ptetaphie_leg(mp, legs[i])
        for c in range(4):
            assert abs(out[i, c] - float(ref[c])) <= 2.0 ** -53 * abs(float(ref[c])) + 1e-300
    assert np.array_equal(orc.to_pxpypze_def(p, "ptetaphim"), cart)
    a, b = legs[:150], legs[150:].copy()
    b[:40, 1] = a[:40, 1] + 1e-7  # near-collinear
    b[:40, 2] = a[:40, 2]
    m = orc.mass_cart_def(a, b, "ptetaphie")
    for i in range(0, 150, 3):
        va, vb = _mp_ptetaphie_leg(mp, a[i]), _mp_ptetaphie_leg(mp, b[i])
        w = [va[k] + vb[k] for k in range(4)]
        m2 = w[3] ** 2 - (w[0] ** 2 + w[1] ** 2 + w[2] ** 2)
        ref = mp.sqrt(m2) if m2 >= 0 else -mp.sqrt(-m2)
        assert abs(m[i] - float(ref)) <= 1e-15 * abs(float(ref)) + 1e-300, i


def test_ptetaphie_mass_closed_forms(orc):
    """Back-to-back legs of equal pt and opposite eta (p1 + p2 = 0 up to the rounding of pi) have
    m = E1 + E2; equal legs have m = 2 sqrt(E^2 - pt^2 cosh^2 eta); a common rotation in phi and
    a common sign flip of eta leave every mass unchanged; on-shell PtEtaPhiE legs give the
    PtEtaPhiM pair mass where the pair is well conditioned."""
    g = syn.rng(191)
    pt, eta, phi = g.uniform(1, 100, 50), g.uniform(-3, 3, 50), g.uniform(-3, 3, 50)
    E1, E2 = pt * np.cosh(eta) * 1.5, pt * np.cosh(eta) * 2.0
    a = np.stack([pt, eta, phi, E1], axis=1)
    b = np.stack([pt, -eta, np.where(phi > 0, phi - np.pi, phi + np.pi), E2], axis=1)
    m = orc.mass_cart_def(a, b, "ptetaphie")
    assert np.all(np.abs(m - (E1 + E2)) <= 1e-14 * (E1 + E2))
    m_eq = orc.mass_cart_def(a, a, "ptetaphie")
    want = 2 * pt * np.cosh(eta) * np.sqrt(1.5 ** 2 - 1)
    assert np.all(np.abs(m_eq - want) <= 1e-14 * want)
    p = syn.ptetaphim(g, 400)
    legs = p.copy()
    legs[:, 3] = orc.to_cartesian_def(p)[:, 3]
    a, b = legs[:200], legs[200:]
    m = orc.mass_cart_def(a, b, "ptetaphie")
    ar, br = a.copy(), b.copy()
    ar[:, 2] = np.mod(a[:, 2] + 0.7 + np.pi, 2 * np.pi) - np.pi
    br[:, 2] = np.mod(b[:, 2] + 0.7 + np.pi, 2 * np.pi) - np.pi
    ar[:, 1], br[:, 1] = -a[:, 1], -b[:, 1]
    assert np.all(np.abs(orc.mass_cart_def(ar, br, "ptetaphie") - m) <= 1e-12 * m)
    mm = orc.mass_def(p[:200], p[200:])
    assert np.all(np.abs(m - mm) <= 1e-12 * mm)


# ----------------------------------------------------------------- O2 adjoint and jagged forms

def _grad_err(g, r, x):
    """Normwise: components weighted by max(|x_k|, 1), relative to the weighted 1-norm of r."""
    s = np.maximum(np.abs(x), 1.0)
    den = np.sum(np.abs(r) * s, axis=1)
    return np.max(np.abs(g - r) * s, axis=1) / np.where(den > 0, den, 1.0)


def test_mass_grad_fp64_vs_definition(orc):
    """O2's adjoint (the O2 identity differentiated term by term, in double) against O1's (the
    chain rule through the binary128 definition): within 1e-14 normwise on the workload, on light
    and heavy mixes, on near-collinear light legs (where m is resolved by O1), with azimuths
    across +-pi, and with massless and zero-pt legs; zero where the mass is zero."""
    e = lambda x: np.sqrt((x[:, 0] * np.cosh(x[:, 1])) ** 2 + x[:, 3] ** 2)
    g = syn.rng(120)
    n = 20000
    wrap_a, wrap_b = syn.ptetaphim(g, n), syn.ptetaphim(g, n)
    gap = 10 ** g.uniform(-6, -1, n)
    wrap_a[:, 2] = np.pi - gap * g.random(n)
    wrap_b[:, 2] = -np.pi + gap * g.random(n)
    deg_a, deg_b = syn.ptetaphim(g, n), syn.ptetaphim(g, n)
    deg_a[::3, 3] = 0.0          # massless legs
    deg_b[1::5, 3] = 0.0
    deg_a[2::7, 0] = 0.0         # pt = 0 legs (with mass)
    cases = [(syn.ptetaphim(g, n), syn.ptetaphim(g, n)),
             (syn.ptetaphim_light_mix(g, n), syn.ptetaphim_light_mix(g, n)),
             _adversarial_pairs(n, 121), (wrap_a, wrap_b), (deg_a, deg_b)]
    for k, (a, b) in enumerate(cases):
        gm = syn.upstream(g, n)
        ra, rb = orc.mass_grad_def(a, b, gm, nthreads=4)
        oa, ob = orc.mass_grad_fp64(a, b, gm, nthreads=4)
        m1 = orc.mass_def(a, b, nthreads=4)
        sel = m1 >= 1e-9 * (e(a) + e(b))
        assert sel.mean() > 0.9, k
        err = _grad_err(np.hstack([oa, ob])[sel], np.hstack([ra, rb])[sel], np.hstack([a, b])[sel])
        assert err.max() <= 1e-14, (k, err.max())
    a = np.array([[10.0, 0.3, 0.1, 0.0], [0.0, 0.0, 0.0, 0.0]])
    oa, ob = orc.mass_grad_fp64(a, a, np.ones(2))  # identical massless legs, zero vectors: m = 0
    assert np.all(oa == 0) and np.all(ob == 0)
    # a planted sign error in the azimuthal term fails the comparison (the pin is sensitive)
    a, b = cases[0]
    gm = syn.upstream(syn.rng(122), n)
    ra, _ = orc.mass_grad_def(a, b, gm)
    oa, _ = orc.mass_grad_fp64(a, b, gm)
    bad = oa.copy()
    bad[:, 2] = -bad[:, 2]
    assert _grad_err(bad, ra, a).max() > 1e-3


def test_mass_grad_fp64_threads_agree(orc):
    g = syn.rng(123)
    a, b, gm = syn.ptetaphim(g, 5000), syn.ptetaphim(g, 5000), syn.upstream(g, 5000)
    r1, r3 = orc.mass_grad_fp64(a, b, gm, 1), orc.mass_grad_fp64(a, b, gm, 3)
    assert np.array_equal(r1[0], r3[0]) and np.array_equal(r1[1], r3[1])


def test_event_pairs_fp64_vs_definition(orc):
    """O2 jagged forms against O1 on 3000 Poisson(8) events plus empty, single-particle and
    65-particle events: offsets equal, pair masses within 1e-14 relative, event sums within
    1e-14 of the summed component magnitudes, the adjoint within 1e-14 of the summed
    contribution magnitudes (which the magnitudes mode returns, checked against an explicit
    sum over the pairs); thread counts do not change the bits."""
    g = syn.rng(124)
    counts = np.concatenate([np.diff(syn.jagged_offsets(g, 3000)), [0, 1, 2, 65]])
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    p = syn.ptetaphim(g, int(off[-1]))
    p[7::31, 3] = 0.0
    po1, pm1, s1 = orc.event_pairs_def(p, off)
    po2, pm2, s2 = orc.event_pairs_fp64(p, off, nthreads=4)
    assert np.array_equal(po1, po2)
    assert np.all(np.abs(pm2 - pm1) <= 1e-14 * pm1)
    cart = np.abs(orc.to_cartesian_def(p))
    ev = np.repeat(np.arange(len(counts)), counts)
    mag = np.zeros((len(counts), 4))
    np.add.at(mag, ev, cart)
    assert np.all(np.abs(s2 - s1) <= 1e-14 * mag)
    _, pm3, s3 = orc.event_pairs_fp64(p, off, nthreads=1)
    assert np.array_equal(pm2, pm3) and np.array_equal(s2, s3)
    gpm = syn.upstream(g, len(pm1))
    gsum = syn.upstream(g, (len(counts), 4))
    r1 = orc.event_pairs_grad_def(p, off, gpm, gsum)
    r2 = orc.event_pairs_grad_fp64(p, off, gpm, gsum, nthreads=4)
    mg = orc.event_pairs_grad_fp64(p, off, gpm, gsum, magnitudes=True, nthreads=4)
    s = np.maximum(np.abs(p), 1.0)
    den = np.sum(mg * s, axis=1)
    err = np.max(np.abs(r2 - r1) * s, axis=1) / np.where(den > 0, den, 1.0)
    assert err.max() <= 1e-14
    assert np.array_equal(r2, orc.event_pairs_grad_fp64(p, off, gpm, gsum, nthreads=1))
    # the magnitudes: for a sample of events, the sum over the event's pairs of |gpm| |dm/dp|
    # (the elementwise O2 adjoint) plus |J|^T |gsum| (O1's sum part, unit by unit)
    po = po1
    for e in (0, 5, 17, len(counts) - 1):
        lo, hi = off[e], off[e + 1]
        n = hi - lo
        want = np.zeros((n, 4))
        if n >= 2:
            ii, jj = np.triu_indices(n, 1)
            ga, gb = orc.mass_grad_fp64(p[lo + ii], p[lo + jj], np.abs(gpm[po[e]:po[e + 1]]))
            np.add.at(want, ii, np.abs(ga))
            np.add.at(want, jj, np.abs(gb))
        for r in range(4):
            unit = np.zeros((1, 4))
            unit[0, r] = 1.0
            J_r = orc.event_pairs_grad_def(p[lo:hi], [0, n], np.zeros(n * (n - 1) // 2), unit)
            want += np.abs(J_r) * abs(gsum[e, r])
        assert np.allclose(mg[lo:hi], want, rtol=1e-12, atol=0), e
    # without sums: the pair part alone
    r1 = orc.event_pairs_grad_def(p, off, gpm)
    r2 = orc.event_pairs_grad_fp64(p, off, gpm)
    mg = orc.event_pairs_grad_fp64(p, off, gpm, magnitudes=True)
    den = np.sum(mg * s, axis=1)
    assert (np.max(np.abs(r2 - r1) * s, axis=1) / np.where(den > 0, den, 1.0)).max() <= 1e-14
    with pytest.raises(ValueError):
        orc.event_pairs_fp64(p, off[::-1])
    with pytest.raises(ValueError):
        orc.event_pairs_grad_fp64(p, off, gpm[:-1])
