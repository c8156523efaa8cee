"""CPU checks of the float-float arithmetic the FP64 kernels use (csrc/ff.cuh, csrc/mass_ff.cuh),
compiled for the host from the same source: elementary functions against mpmath, the pair mass
against the binary128 oracle.  The GPU parity tests then check the device build of the same code.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import gvx_synth as syn

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ffh(tmp_path_factory):
    from helpers import build_ff_harness
    return build_ff_harness(tmp_path_factory.mktemp("ffh"))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _unary(lib, op, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out, ok = np.empty_like(x), np.empty(len(x), np.uint8)
    lib.ffh_unary(op, _p(x), ctypes.c_int64(len(x)), _p(out), _p(ok))
    return out, ok.astype(bool)


def _binary(lib, op, x, y):
    x, y = (np.ascontiguousarray(v, dtype=np.float64) for v in (x, y))
    out, ok = np.empty_like(x), np.empty(len(x), np.uint8)
    lib.ffh_binary(op, _p(x), _p(y), ctypes.c_int64(len(x)), _p(out), _p(ok))
    return out, ok.astype(bool)


def _mass(lib, a, b):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    m, ok = np.empty(len(a)), np.empty(len(a), np.uint8)
    lib.ffh_mass(_p(a), _p(b), ctypes.c_int64(len(a)), _p(m), _p(ok))
    return m, ok.astype(bool)


def test_ff_elementary_functions(ffh):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    g = np.random.default_rng(5)
    x = np.concatenate([g.uniform(-16, 16, 600), g.uniform(-1e-2, 1e-2, 200),
                        10 ** g.uniform(-20, -2, 200) * g.choice([-1, 1], 200), [0.0]])
    for op, f, tol in ((0, mp.cosh, 6e-14), (1, mp.sinh, 6e-14)):  # |x| < 16: 16 * 2^-48
        out, ok = _unary(ffh, op, x)
        ref = np.array([float(f(mp.mpf(v))) for v in x])
        assert ok.all()
        err = np.abs(out - ref) / np.maximum(np.abs(ref), 1e-300)
        assert err.max() <= tol, (op, x[np.argmax(err)])
    h = np.concatenate([g.uniform(0, np.pi / 2, 800), 10 ** g.uniform(-20, 0, 200), [0.0]])
    out, _ = _unary(ffh, 2, h)
    ref = np.array([float(mp.sin(mp.mpf(v))) for v in h])
    assert np.all(np.abs(out - ref) <= 3e-14 * np.abs(ref))
    y = 10 ** g.uniform(-15, 15, 1000) * g.choice([-1, 1], 1000)
    out, ok = _unary(ffh, 3, y)           # double -> ff -> double
    assert ok.all() and np.all(np.abs(out / y - 1) <= 2 ** -47)
    out, _ = _unary(ffh, 4, np.abs(y))    # sqrt
    ref = np.array([float(mp.sqrt(mp.mpf(abs(v)))) for v in y])
    assert np.all(np.abs(out / ref - 1) <= 3e-14)
    z = 10 ** g.uniform(-10, 10, 1000)
    out, _ = _binary(ffh, 2, y, z)        # division
    ref = np.array([float(mp.mpf(u) / mp.mpf(v)) for u, v in zip(y, z)])
    assert np.all(np.abs(out / ref - 1) <= 4e-14)


def test_ff_exact_differences(ffh):
    """An FP64 difference converted to ff is exact where a and b are within a factor 2 (where
    cancellation happens), and within 2^-47 relative elsewhere."""
    g = np.random.default_rng(6)
    a = g.uniform(-4, 4, 4000)
    b = a + g.choice([1e-15, 1e-12, 1e-6, 1e-2], 4000) * g.uniform(-1, 1, 4000)
    out, ok = _binary(ffh, 0, a, b)
    assert ok.all()
    from fractions import Fraction
    for i in range(0, 4000, 7):
        exact = Fraction(a[i]) - Fraction(b[i])
        if exact != 0:
            assert abs(Fraction(out[i]) - exact) <= abs(exact) * Fraction(1, 2 ** 47)


def test_ff_pair_mass_against_oracle(ffh, orc):
    from test_oracle_pins import _adversarial_pairs
    from helpers import edge_pairs
    n = 100_000
    cases = [(syn.ptetaphim(syn.rng(0), n), syn.ptetaphim(syn.rng(7), n)),
             _adversarial_pairs(50_000, 104),
             (syn.ptetaphim_light_mix(syn.rng(2), n), syn.ptetaphim_light_mix(syn.rng(3), n)),
             edge_pairs()]
    for k, (a, b) in enumerate(cases):
        m, ok = _mass(ffh, a, b)
        ref = orc.mass_def(a, b, nthreads=8)
        e = lambda x: np.sqrt((x[:, 0] * np.cosh(x[:, 1])) ** 2 + x[:, 3] ** 2)
        bound = 1e-13 * np.abs(ref) + 1e-16 * (e(a) + e(b))
        assert np.all(np.abs(m - ref)[ok] <= bound[ok]), k
        if k < 3:
            assert ok.mean() > 0.998, k  # the fast path covers the collider-like workloads


def _mass_lc(lib, a, b):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    m, ok = np.empty(len(a)), np.empty(len(a), np.uint8)
    lib.ffh_mass_lc(_p(a), _p(b), ctypes.c_int64(len(a)), _p(m), _p(ok))
    return m, ok.astype(bool)


def test_lc_pair_mass_against_oracle(ffh, orc):
    """The light-cone fast path of the FP64 mass kernel (mass_lc.cuh), built for the host with the
    hardware approximations' worst-case error modelled: pure relative error against O1 wherever
    O1 is accurate (m >= 1e-9 (E1 + E2)) and against O2, on every value it accepts; it accepts all
    but a few of the collider-like pairs."""
    from test_oracle_pins import _adversarial_pairs
    from helpers import edge_pairs
    n = 100_000
    cases = [(syn.ptetaphim(syn.rng(0), n), syn.ptetaphim(syn.rng(7), n)),
             _adversarial_pairs(50_000, 104),
             (syn.ptetaphim_light_mix(syn.rng(2), n), syn.ptetaphim_light_mix(syn.rng(3), n)),
             edge_pairs()]
    e = lambda x: np.sqrt((x[:, 0] * np.cosh(x[:, 1])) ** 2 + x[:, 3] ** 2)
    for k, (a, b) in enumerate(cases):
        m, ok = _mass_lc(ffh, a, b)
        o1, o2 = orc.mass_def(a, b, nthreads=8), orc.mass_fp64(a, b, nthreads=8)
        cond = ok & (o1 >= 1e-9 * (e(a) + e(b)))
        assert np.all(np.abs(m - o1)[cond] <= 2.5e-13 * o1[cond]), k
        pos = ok & (o2 > 0)
        assert np.all(np.abs(m - o2)[pos] <= 2.5e-13 * o2[pos]), k
        assert np.all(m[ok & (o2 == 0)] == 0), k
        if k < 3:
            assert ok.mean() > 0.9999, k


def test_lc_to_double_conversion(ffh):
    """The adjoint's ff -> double conversion (mass_lc.cuh lc_to_double) against the exact sum
    hi + lo (fractions): the correctly rounded double of hi + lo, times 2^shift, for lo of every
    relative size and sign, power-of-two hi included; exactly hi where lo is 0 or denormal (a
    denormal lo counts as 0); 0 for a zero hi."""
    from fractions import Fraction
    g = syn.rng(80)
    n = 20000
    e = g.integers(-100, 100, n)
    hi = np.ldexp(g.uniform(1, 2, n), e).astype(np.float32)
    hi[: n // 4] = np.ldexp(1.0, e[: n // 4]).astype(np.float32)       # powers of two
    hi *= np.where(g.random(n) < 0.5, -1, 1).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    lo = (g.uniform(-2, 2, n) * ulp * np.ldexp(1.0, -g.integers(0, 40, n))).astype(np.float32)
    lo[::11] = 0.0
    hi, lo = np.ascontiguousarray(hi), np.ascontiguousarray(lo)
    for shift in (0, -300, 500):
        out = np.empty(n)
        ffh.ffh_lc_to_double(hi.ctypes.data_as(ctypes.c_void_p), lo.ctypes.data_as(ctypes.c_void_p),
                             ctypes.c_int64(n), ctypes.c_int(shift), _p(out))
        for h, l, o in zip(hi, lo, out):
            lo_eff = float(l) if abs(float(l)) >= 2.0 ** -126 else 0.0
            exact = (Fraction(float(h)) + Fraction(lo_eff)) * Fraction(2) ** shift
            assert o == float(exact), (h, l, o)
    tiny = np.array([0.0, -0.0], np.float32)
    out = np.empty(2)
    z = np.zeros(2, np.float32)
    ffh.ffh_lc_to_double(tiny.ctypes.data_as(ctypes.c_void_p), z.ctypes.data_as(ctypes.c_void_p),
                         ctypes.c_int64(2), ctypes.c_int(0), _p(out))
    assert np.all(out == 0)


def test_lc_to_double_int_conversion(ffh):
    """The jagged pair mass's integer ff -> double conversion (mass_lc.cuh lc_to_double_int)
    against the exact sum hi + lo (fractions): below one ulp of the result on normalized pairs of
    every relative size and sign, in the binade below a power-of-two hi too; exactly hi where lo
    is 0; a denormal lo counts as 0; 0 for a zero or denormal hi."""
    from fractions import Fraction
    g = syn.rng(81)
    n = 20000
    e = g.integers(-100, 100, n)
    hi = np.ldexp(g.uniform(1, 2, n), e).astype(np.float32)
    hi[: n // 4] = np.ldexp(1.0, e[: n // 4]).astype(np.float32)       # powers of two
    hi *= np.where(g.random(n) < 0.5, -1, 1).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    lo = (g.uniform(-0.5, 0.5, n) * ulp * np.ldexp(1.0, -g.integers(0, 40, n)))
    lo[::7] = 0.5 * ulp[::7] * np.sign(g.uniform(-1, 1, n)[::7])      # exactly half an ulp
    lo = lo.astype(np.float32)
    lo[::11] = 0.0

    def normalized(h, l):
        h, l = float(h), float(l)
        below = l * h < 0 and abs(h) == 2.0 ** np.floor(np.log2(abs(h)))
        return abs(l) <= float(np.spacing(np.float32(abs(h) / 2 if below else abs(h)))) / 2
    keep = np.array([normalized(h, l) for h, l in zip(hi, lo)])
    hi, lo = np.ascontiguousarray(hi[keep]), np.ascontiguousarray(lo[keep])
    assert len(hi) > 0.9 * n
    for shift in (0, -300, 500):
        out = np.empty(len(hi))
        ffh.ffh_lc_to_double_int(hi.ctypes.data_as(ctypes.c_void_p), lo.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.c_int64(len(hi)), ctypes.c_int(shift), _p(out))
        for h, l, o in zip(hi, lo, out):
            exact = (Fraction(float(h)) + Fraction(float(l))) * Fraction(2) ** shift
            # a denormal lo counts as 0: an absolute error below 2^-126 (times 2^shift)
            bound = Fraction(float(np.spacing(abs(o)))) + Fraction(2) ** (shift - 126)
            assert abs(Fraction(float(o)) - exact) < bound, (h, l, o)
            if l == 0:
                assert o == np.ldexp(float(h), shift)
    tiny = np.array([0.0, -0.0, 1e-40], np.float32)
    out = np.empty(3)
    z = np.zeros(3, np.float32)
    ffh.ffh_lc_to_double_int(tiny.ctypes.data_as(ctypes.c_void_p), z.ctypes.data_as(ctypes.c_void_p),
                             ctypes.c_int64(3), ctypes.c_int(0), _p(out))
    assert np.all(out == 0)


def _mass_grad_lc(lib, a, b, gm, ms=None):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    gm = np.ascontiguousarray(gm, dtype=np.float64)
    ga, gb, ok = np.empty_like(a), np.empty_like(b), np.empty(len(a), np.uint8)
    msp = None if ms is None else _p(np.ascontiguousarray(ms, dtype=np.float64))
    lib.ffh_mass_grad_lc(_p(a), _p(b), _p(gm), msp, ctypes.c_int64(len(a)), _p(ga), _p(gb),
                         _p(ok))
    return ga, gb, ok.astype(bool)


def test_lc_pair_mass_gradient_against_oracle(ffh, orc):
    """The light-cone adjoint of the FP64 mass kernel (mass_lc_grad.cuh), host build: both legs'
    gradients against the binary128 chain rule, normwise (components weighted by max(|x|, 1))
    within 1e-12 of the weighted reference wherever it runs, with the forward's masses recomputed
    and with the oracle's masses given as the saved ones; zero where m = 0 or gm = 0."""
    from test_oracle_pins import _adversarial_pairs
    from helpers import scaled_grad_err
    cases = [(syn.ptetaphim(syn.rng(60), 50000), syn.ptetaphim(syn.rng(61), 50000)),
             (syn.ptetaphim_light_mix(syn.rng(62), 20000), syn.ptetaphim_light_mix(syn.rng(63), 20000)),
             _adversarial_pairs(10000, 64)]
    e = lambda x: np.sqrt((x[:, 0] * np.cosh(x[:, 1])) ** 2 + x[:, 3] ** 2)
    for k, (a, b) in enumerate(cases):
        gm = syn.upstream(syn.rng(65 + k), len(a))
        ra, rb = orc.mass_grad_def(a, b, gm, nthreads=8)
        o1 = orc.mass_def(a, b, nthreads=8)
        for ms in (None, o1):
            ga, gb, ok = _mass_grad_lc(ffh, a, b, gm, ms)
            assert ok.mean() > 0.999, k
            # O1's gradient is exact only where m is resolved (the m = 0 pairs get 0 here)
            sel = ok & (o1 >= 1e-9 * (e(a) + e(b)))
            err = scaled_grad_err(np.hstack([ga, gb])[sel], np.hstack([ra, rb])[sel],
                                  np.hstack([a, b])[sel])
            assert err.max() <= 1e-12, (k, ms is None, err.max())
    # gm = 0 and saved m = 0 give exact zeros
    a, b = syn.ptetaphim(syn.rng(68), 1000), syn.ptetaphim(syn.rng(69), 1000)
    gm = syn.upstream(syn.rng(70), 1000)
    gm[::3] = 0.0
    ms = orc.mass_def(a, b)
    ms[1::3] = 0.0
    ga, gb, ok = _mass_grad_lc(ffh, a, b, gm, ms)
    zero = np.zeros(1000, bool)
    zero[::3] = zero[1::3] = True
    assert ok.all() and np.all(ga[zero] == 0) and np.all(gb[zero] == 0)
    assert np.all(np.abs(ga[~zero]).max(axis=1) > 0)


def test_lc_pair_mass_tiny_and_degenerate_legs(ffh, orc):
    """Scale ratios at and beyond the fast path's 2^-40 rule, zero and denormal components, and
    |d_phi| in and out of the band around 2 pi that the fast path leaves to FP64: whatever it
    accepts is within its bound."""
    g = syn.rng(12)
    n = 20_000
    a, b = syn.ptetaphim(g, n), syn.ptetaphim(g, n)
    shrink = np.ldexp(1.0, -g.integers(0, 80, n))
    a[:, 0] *= np.where(g.random(n) < 0.3, shrink, 1.0)
    a[:, 3] *= np.where(g.random(n) < 0.3, shrink, 1.0)
    b[:, 3] = np.where(g.random(n) < 0.2, 0.0, b[:, 3])
    a[:, 0] = np.where(g.random(n) < 0.05, 0.0, a[:, 0])
    b[:, 0] = np.where(g.random(n) < 0.02, 5e-324, b[:, 0])
    w = g.random(n) < 0.2  # opposite azimuths near +-pi
    a[w, 2] = np.pi - 10 ** g.uniform(-12, 0, w.sum())
    b[w, 2] = -np.pi + 10 ** g.uniform(-12, 0, w.sum())
    m, ok = _mass_lc(ffh, a, b)
    o2 = orc.mass_fp64(a, b, nthreads=8)
    pos = ok & (o2 > 0)
    assert np.all(np.abs(m - o2)[pos] <= 2.5e-13 * o2[pos])
    assert np.all(m[ok & (o2 == 0)] == 0)
    assert 0.5 < ok.mean() < 1.0  # both branches are exercised


def test_ff_unchecked_conversion_and_tiny_legs(ffh):
    """pt and m (and the boost's inputs) enter the ff paths through the unchecked conversion:
    bitwise the checked one on every value that one accepts, a signed zero for zeros, denormals
    and values that scale below 2^-74.  The mass domain keeps out nonzero denormals and scale
    exponents at or below 2^-993; exact zeros stay in."""
    g = syn.rng(11)
    x = np.concatenate([np.ldexp(g.uniform(1, 2, 20000), g.integers(-80, 1, 20000)),
                        [0.0, -0.0, 1.0, 2.0 - 2.0 ** -52, 2.0 ** -30, 2.0 ** -74,
                         2.0 ** -75 * (2 - 2.0 ** -52), 1.0 - 2.0 ** -53, 1.0 + 2.0 ** -29]])
    x[::2] *= -1
    for shift in (-940, -3, 0, 7, 1000):
        xs = np.ldexp(x, shift)
        hi, lo, same = np.empty(len(xs)), np.empty(len(xs)), np.empty(len(xs), np.uint8)
        ffh.ffh_conv_ranged(_p(xs), ctypes.c_int64(len(xs)), shift, _p(hi), _p(lo), _p(same))
        small = np.abs(x) < 2.0 ** -74
        assert np.all(same[~small | (x == 0)] == 1), shift
        assert np.all(same[small & (x != 0)] == 2), shift
        assert np.all((hi[small] == 0) & (lo[small] == 0)), shift
        assert np.array_equal(np.signbit(hi[small]), np.signbit(xs[small])), shift
    ffh.ffh_conv_ranged(_p(np.array([5e-324])), ctypes.c_int64(1), 0, _p(hi), _p(lo), _p(same))
    assert hi[0] == 0.0 and lo[0] == 0.0 and same[0] == 2
    den = 5e-324
    a = np.array([[den, 0.1, 0.2, 1e-290], [1e-290, 0.1, 0.2, den], [0.0, 0.1, 0.2, 1e-290],
                  [1e-289, 0.3, -0.2, 0.0], [2.0 ** -990, 0.0, 0.0, 0.0], [2.0 ** -994, 0, 0, 0],
                  [3.0, 0.5, 1.0, 0.0], [den, 0.5, 1.0, 2.0]])
    b = np.array([[0.0, 0.0, 0.0, 0.0]] * 6 + [[4.0, -0.5, -1.0, 0.0], [1.0, 0.0, 0.0, 0.0]])
    m, ok = _mass(ffh, a, b)
    assert ok.tolist() == [False, False, True, True, True, False, True, False]
    assert m[2] == 1e-290 and m[3] == 0.0 and m[4] == 0.0  # a massless leg alone has m = 0


def test_ff_pair_mass_tiny_angles(ffh, orc):
    """Angles and angle differences below 2^-74 enter the ff path as exact zeros (their share of
    m^2 is below 2^-148 of pt1 pt2): such pairs stay on the fast path and keep the gate."""
    pi_d = float(np.pi)
    a = np.array([[50.0, 1e-30, 0.3, 1.0], [50.0, 1e-300, 0.3, 0.0], [40.0, 2.0, pi_d, 0.5],
                  [40.0, 2.0, 1e-300, 0.5], [10.0, -3.0, -pi_d, 2.0], [7.0, 1e-25, -1e-25, 0.0]])
    b = np.array([[60.0, -1e-30, 1.3, 2.0], [50.0, -1e-300, 0.3, 0.0], [30.0, 2.0, -pi_d, 0.0],
                  [30.0, 2.0 + 1e-20, -1e-300, 0.5], [12.0, -3.0, pi_d, 3.0], [9.0, -1e-25, 1e-25, 0.0]])
    m, ok = _mass(ffh, a, b)
    ref = orc.mass_def(a, b)
    assert ok.all()
    e = lambda x: np.sqrt((x[:, 0] * np.cosh(x[:, 1])) ** 2 + x[:, 3] ** 2)
    assert np.all(np.abs(m - ref) <= 1e-13 * np.abs(ref) + 1e-16 * (e(a) + e(b)))


def test_ff_pair_mass_gradient_against_oracle(ffh, orc):
    """The FP64 adjoint's ff pair gradient (both legs) against the binary128 chain rule, on the
    workload, the light/heavy mix and the adversarial near-collinear pairs: normwise (components
    weighted by max(|x|, 1)) within 1e-12 of the weighted reference where the fast path runs."""
    from test_oracle_pins import _adversarial_pairs
    from helpers import scaled_grad_err
    cases = [(syn.ptetaphim(syn.rng(50), 20000), syn.ptetaphim(syn.rng(51), 20000)),
             (syn.ptetaphim_light_mix(syn.rng(52), 20000), syn.ptetaphim_light_mix(syn.rng(53), 20000)),
             _adversarial_pairs(5000, 54)]
    for k, (a, b) in enumerate(cases):
        a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
        gm = syn.upstream(syn.rng(55 + k), len(a))
        ga, gb = np.empty_like(a), np.empty_like(b)
        ok = np.empty(len(a), np.uint8)
        ffh.ffh_mass_grad(_p(a), _p(b), _p(gm), ctypes.c_int64(len(a)), _p(ga), _p(gb), _p(ok))
        ok = ok.astype(bool)
        ra, rb = orc.mass_grad_def(a, b, gm, nthreads=8)
        assert ok.mean() > 0.99, k
        assert scaled_grad_err(ga[ok], ra[ok], a[ok]).max() <= 1e-12, k
        assert scaled_grad_err(gb[ok], rb[ok], b[ok]).max() <= 1e-12, k


def test_ff_boost_coefficients(ffh):
    """gamma = 1/sqrt(1 - b2) and w = gamma/(1 + gamma) of the FP64 boost, from the exact
    fixed-point 1 - b2, against mpmath."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    b = np.concatenate([syn.velocities(syn.rng(8), 1500, 0.99),
                        syn.velocities(syn.rng(9), 500, 0.99998),
                        [[0, 0, 0], [1e-9, -2e-9, 3e-9], [0.6, 0.8, 0.0]]])
    g, w = np.empty(len(b)), np.empty(len(b))
    ok = np.empty(len(b), np.uint8)
    ffh.ffh_boost_coef(_p(b), ctypes.c_int64(len(b)), _p(g), _p(w), _p(ok))
    ok = ok.astype(bool)
    assert not ok[-1] and ok[:-1].all()  # |beta| = 1 leaves the fast path
    for i in np.flatnonzero(ok):
        b2 = sum(mp.mpf(x) ** 2 for x in b[i])
        G = 1 / mp.sqrt(1 - b2)
        assert abs(g[i] / float(G) - 1) <= 3e-14
        assert abs(w[i] / float(G / (1 + G)) - 1) <= 3e-14


def test_ff_to_double_by_integers(ffh):
    """The integer ff -> double conversion against the exact sum hi + lo (rounded once by an FP64
    add): within 2 ulps, signs and carries across a power of two included."""
    g = syn.rng(12)
    n = 200_000
    hi = (np.ldexp(g.uniform(1, 2, n), g.integers(-60, 60, n)) * g.choice([-1, 1], n)).astype(np.float32)
    hi[:64] = np.float32(1.0)
    hi[64:128] = np.float32(-2.0)
    hi[128:192] = np.nextafter(np.float32(2.0), np.float32(0))
    rel = np.ldexp(g.uniform(-1, 1, n), -g.integers(21, 60, n))
    lo = (hi.astype(np.float64) * rel).astype(np.float32)
    lo[::7] = 0
    lo[1::97] = np.float32(1e-45)  # denormal lo: counts as 0
    for shift in (-700, 0, 5, 700):
        oi, oa = np.empty(n), np.empty(n)
        ffh.ffh_to_double(hi.ctypes.data_as(ctypes.c_void_p), lo.ctypes.data_as(ctypes.c_void_p),
                          ctypes.c_int64(n), shift, _p(oi), _p(oa))
        exact = np.ldexp(hi.astype(np.float64), shift)
        assert np.all(np.abs(oi - oa) <= 2 * np.spacing(np.abs(oa))), shift
        assert np.all(np.sign(oi) == np.sign(exact)), shift


def _boost(lib, v, beta):
    v, beta = np.ascontiguousarray(v), np.ascontiguousarray(beta)
    out, ok = np.empty_like(v), np.empty(len(v), np.uint8)
    lib.ffh_boost(_p(v), _p(beta), ctypes.c_int64(len(v)), _p(out), _p(ok))
    return out, ok.astype(bool)


def test_ff_boost_fast_path_against_oracle(ffh, orc):
    """The FP64 boost's fast path (beta.p and E + beta.p in FP64, gamma, w, E' and f in ff)
    against the binary128 boost.  Its error model: a few ulps of FP64 amplified by the condition
    C = (E + |beta| |p|) / (E + beta.p) of E + beta.p, plus a few 2^-47 from the ff steps, so the
    normwise error vs E' stays below 4e-14 + 2e-15 C (C <= 199 for |beta| <= 0.99)."""
    g = syn.rng(1)
    v, b = syn.pxpypze(g, 1 << 18), syn.velocities(g, 1 << 18, 0.99)
    cond = (v[:, 3] + np.linalg.norm(b, axis=1) * np.linalg.norm(v[:, :3], axis=1)) / (
        v[:, 3] + np.sum(b * v[:, :3], axis=1))
    idx = np.union1d(np.arange(0, len(v), 16), np.argpartition(cond, -2048)[-2048:])
    out, ok = _boost(ffh, v[idx], b[idx])
    assert ok.all()
    ref = orc.boost_def(v[idx], b[idx], nthreads=8)
    err = np.abs(out - ref).max(axis=1) / ref[:, 3]
    assert np.all(err <= 4e-14 + 2e-15 * cond[idx])
    assert cond[idx].max() > 50  # the sample reaches the ill-conditioned end
    # beta orthogonal to p at gamma up to 158: beta.p cancels, E + beta.p does not
    m = 2000
    w = syn.pxpypze(syn.rng(5), m)
    d = syn.velocities(syn.rng(6), m, 1.0)
    d -= (np.sum(d * w[:, :3], axis=1) / np.sum(w[:, :3] ** 2, axis=1))[:, None] * w[:, :3]
    d *= (syn.rng(7).uniform(0.9, 0.99998, m) / np.linalg.norm(d, axis=1))[:, None]
    out, ok = _boost(ffh, w, d)
    ref = orc.boost_def(w, d)
    assert ok.all()
    assert np.all(np.abs(out - ref).max(axis=1) <= 4e-14 * ref[:, 3])
    # rest frame (beta = -p/E): absolute error within a few 2^-47 of gamma (E + |beta| |p|)
    bw = -w[:, :3] / w[:, 3:4]
    out, ok = _boost(ffh, w, bw)
    ref = orc.boost_def(w, bw)
    gam = 1 / np.sqrt(1 - np.sum(bw * bw, axis=1))
    sc = gam * (w[:, 3] + np.linalg.norm(bw, axis=1) * np.linalg.norm(w[:, :3], axis=1))
    assert ok.any() and np.all(np.abs(out - ref)[ok].max(axis=1) <= 3e-14 * sc[ok])
    # domain: 1 - b2 below 2^-16, a zero vector, magnitudes outside [2^-823, 2^1013), non-finite
    one = np.array([[0.0, 0.0, 0.3]])
    cases = [([1.0, 2.0, 3.0, 4.0], [0.0, 0.0, 0.999995]), ([0.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.3]),
             ([1.0, 2.0, 3.0, 2.0 ** 1013], [0.0, 0.0, 0.3]), ([2.0 ** -824, 0, 0, 0], [0, 0, 0.3]),
             ([1.0, np.inf, 0.0, 4.0], [0.0, 0.0, 0.3]), ([1.0, 2.0, 3.0, 4.0], [np.nan, 0, 0]),
             ([1.0, 2.0, 3.0, 2.0 ** 1012], [0.0, 0.0, 0.3]), ([2.0 ** -823, 0, 0, 0], [0, 0, 0.3])]
    out, ok = _boost(ffh, np.array([c[0] for c in cases], float), np.array([c[1] for c in cases], float))
    assert ok.tolist() == [False] * 6 + [True, True]
    ref = orc.boost_def(np.array([c[0] for c in cases[6:]], float), np.repeat(one, 2, axis=0))
    assert np.all(np.abs(out[6:] - ref).max(axis=1) <= 4e-14 * ref[:, 3])
    # beta = 0 is the identity, bit for bit (gamma = 1 and p + f 0 are exact)
    out, ok = _boost(ffh, w, np.zeros((m, 3)))
    assert ok.all() and np.array_equal(out, w)


def test_ff_boost_adjoint_against_oracle(ffh, orc):
    """The FP64 boost adjoint's fast path (FP64 dot products and sums that can cancel, A, B, f and
    the boost of the upstream gradient in ff) against the binary128 chain rule, on the FP64
    workload: normwise, components weighted by max(|x|, 1), within 1e-12 of the weighted
    reference.  A zero upstream gradient gives exact zeros; inputs outside the domain are left
    to the FP64 formulas."""
    from helpers import scaled_grad_err
    g = syn.rng(60)
    n = 1 << 15
    v, b, q = syn.pxpypze(g, n), syn.velocities(g, n, 0.99), syn.upstream(g, (n, 4))
    v, b, q = (np.ascontiguousarray(x) for x in (v, b, q))
    gv, gb = np.empty_like(v), np.empty_like(b)
    ok = np.empty(n, np.uint8)
    ffh.ffh_boost_bwd(_p(v), _p(b), _p(q), ctypes.c_int64(n), _p(gv), _p(gb), _p(ok))
    assert ok.all()
    rv, rb = orc.boost_grad_def(v, b, q)
    assert scaled_grad_err(gv, rv, q).max() <= 1e-12
    assert scaled_grad_err(gb, rb, b).max() <= 1e-12
    z = np.zeros((3, 4))
    v3, b3 = np.ascontiguousarray(v[:3]), np.ascontiguousarray(b[:3])
    gv, gb, ok = np.empty((3, 4)), np.empty((3, 3)), np.empty(3, np.uint8)
    ffh.ffh_boost_bwd(_p(v3), _p(b3), _p(z), ctypes.c_int64(3), _p(gv), _p(gb), _p(ok))
    assert ok.all() and not gv.any() and not gb.any()
    bad_q = np.array([[1e-300, 0, 0, 0], [1.0, 2.0, 3.0, np.inf], [1e300, 0, 0, 1e300]])
    bad_b = np.array([[0.0, 0.0, 0.3], [0.0, 0.0, 0.3], [0.0, 0.0, 0.999995]])
    ffh.ffh_boost_bwd(_p(v3), _p(np.ascontiguousarray(bad_b)), _p(bad_q), ctypes.c_int64(3),
                      _p(gv), _p(gb), _p(ok))
    assert not ok.any()


def _cart_inputs(seed, n):
    g = syn.rng(seed)
    a, b = syn.pxpypze(g, n), syn.pxpypze(g, n)
    k = n // 4  # near-collinear light pairs: the cancellation the form is for
    b[:k, :3] = a[:k, :3] * g.uniform(0.5, 2.0, (k, 1))
    b[:k, :3] += a[:k, :3] * g.uniform(-1e-9, 1e-9, (k, 3))
    mb = g.uniform(0, 1e-3, k)
    b[:k, 3] = np.sqrt(np.sum(b[:k, :3] ** 2, axis=1) + mb * mb)
    return a, b


def test_ff_cartesian_mass_against_oracle(ffh, orc):
    """The FP64 Cartesian pair mass (FMA-exact cross product and E^2 - |p|^2) against the
    binary128 definition, PxPyPzE and PxPyPzM legs, including near-collinear light pairs:
    within 1e-12 relative."""
    for coords, code in (("pxpypze", 0), ("pxpypzm", 1)):
        a, b = _cart_inputs(130 + code, 20000)
        if code == 1:
            g = syn.rng(140)
            a[:, 3] = g.uniform(0, 10, len(a))
            b[: len(b) // 4, 3] = g.uniform(0, 1e-3, len(b) // 4)
        a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
        m, ok = np.empty(len(a)), np.empty(len(a), np.uint8)
        ffh.ffh_mass_cart(_p(a), _p(b), ctypes.c_int64(len(a)), code, _p(m), _p(ok))
        ok = ok.astype(bool)
        ref = orc.mass_cart_def(a, b, coords)
        assert ok.all(), coords
        err = np.abs(m[ok] - ref[ok]) / ref[ok]
        assert err.max() <= 1e-12, (coords, err.max())


def _cart_fixed(ffh, a, b, coords=0):
    a, b = np.ascontiguousarray(a, dtype=np.float64), np.ascontiguousarray(b, dtype=np.float64)
    n = len(a)
    m, ok = np.empty(n), np.empty(n, np.uint8)
    m32, ok32 = np.empty(n, np.float32), np.empty(n, np.uint8)
    ffh.ffh_mass_cart_fixed(_p(a), _p(b), ctypes.c_int64(n), coords, _p(m), _p(ok), _p(m32),
                            _p(ok32))
    return m, ok.astype(bool), m32, ok32.astype(bool)


def test_fixed_point_pxpypze_mass_against_oracle(ffh, orc):
    """The exact fixed-point PxPyPzE pair mass (FP64 legs) against the binary128 definition:
    within 2^-44 relative wherever it takes the pair, and it takes every random pair; the
    near-collinear light pairs it takes are just as accurate."""
    g = syn.rng(150)
    n = 40000
    a, b = syn.pxpypze(g, n), syn.pxpypze(g, n)
    m, ok, _, _ = _cart_fixed(ffh, a, b)
    ref = orc.mass_cart_def(a, b, "pxpypze")
    assert ok.all()
    assert np.max(np.abs(m - ref) / ref) <= 2.0 ** -44
    a, b = _cart_inputs(151, 20000)
    m, ok, _, _ = _cart_fixed(ffh, a, b)
    ref = orc.mass_cart_def(a, b, "pxpypze")
    assert ok[len(a) // 4:].all()  # the unrelated pairs
    assert np.max(np.abs(m[ok] - ref[ok]) / np.abs(ref[ok])) <= 2.0 ** -44


def test_fixed_point_pxpypze_mass_threshold_and_edges(ffh, orc):
    """Pairs are taken exactly when |m^2| >= 2^-31 of the squared scale (the power of two
    2^(2 sc) with the largest component in [2^sc, 2^(sc+1))), so a zero or vanishing mass goes
    to the FP64 form; a spacelike sum gives -sqrt(-m^2); a component 2^-100 below the others is
    dropped below the fixed-point resolution; non-finite or far out-of-range inputs are refused."""
    E = 1.5  # scale exponent 0
    rows = []
    for r in (2.0 ** -15.4, 2.0 ** -15.6, 2.0 ** -10, 0.5):  # m / 2^sc around the 2^-15.5 edge
        rows.append(([0.0, 0.0, 1.0, np.hypot(1.0, r / 2)], [0.0, 0.0, 1.0, np.hypot(1.0, r / 2)]))
    rows.append(([0.0, 0.0, E, E], [0.0, 0.0, E, E]))                 # massless, collinear: 0
    rows.append(([1.0, 0.0, 0.0, 0.1], [1.0, 0.0, 0.0, 0.1]))         # spacelike sum
    rows.append(([1e-30, 2.0, -1.0, 3.0], [0.5, -1e-300, 0.25, 1.25]))  # tiny components
    rows.append(([np.inf, 0.0, 0.0, 1.0], [0.0, 0.0, 0.0, 1.0]))
    rows.append(([0.0, 0.0, 0.0, 1e300], [0.0, 0.0, 0.0, 1e300]))
    rows.append(([0.0, 0.0, 0.0, 1e-300], [0.0, 0.0, 0.0, 1e-300]))
    a = np.array([r[0] for r in rows])
    b = np.array([r[1] for r in rows])
    m, ok, _, _ = _cart_fixed(ffh, a, b)
    ref = orc.mass_cart_def(a, b, "pxpypze")
    # E = sqrt(1 + r^2/4) in [1, 2): scale exponent 0 and m^2 = 4 (E^2 - 1) = r^2, so the
    # threshold 2^-31 falls at r = 2^-15.5
    assert ok[:4].tolist() == [True, False, True, True]
    assert not ok[4]
    assert ok[5] and m[5] < 0
    assert ok[6]
    assert not ok[7:].any()
    sel = ok & np.isfinite(ref)
    assert np.all(np.abs(m[sel] - ref[sel]) <= 2.0 ** -44 * np.abs(ref[sel]))


def test_fixed_point_pxpypze_mass_f32(ffh, orc):
    """FP32 legs through the same fixed-point path, rounded once to float: within one rounding
    of the binary128 mass of the float inputs."""
    g = syn.rng(152)
    a, b = syn.to_f32(syn.pxpypze(g, 40000)), syn.to_f32(syn.pxpypze(g, 40000))
    _, _, m32, ok32 = _cart_fixed(ffh, a.astype(np.float64), b.astype(np.float64))
    ref = orc.mass_cart_def(a.astype(np.float64), b.astype(np.float64), "pxpypze")
    assert ok32.all()
    assert np.max(np.abs(m32.astype(np.float64) - ref) / np.abs(ref)) <= 2.0 ** -24 * 1.01


def _apply(ffh, L, v):
    L = np.ascontiguousarray(L, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out, ok = np.full(v.shape, np.nan), np.zeros(len(v), np.uint8)
    c = ffh.ffh_apply(_p(L), _p(v), ctypes.c_int64(len(v)), _p(out), _p(ok))
    return c, out, ok.astype(bool)


def _apply_bound(L, v):
    """2^-42 sum_j |L_ij v_j| + 2^-70 max_j |L_ij| max_j |v_j|, per component."""
    Lf = np.broadcast_to(L, (len(v), 4, 4))
    s = np.einsum("nrk,nk->nr", np.abs(Lf), np.abs(v))
    floor = np.max(np.abs(Lf), axis=2) * np.max(np.abs(v), axis=1)[:, None]
    return 2.0 ** -42 * s + 2.0 ** -70 * floor


def test_ff_lorentz_apply_against_oracle(ffh, orc):
    """The float-float shared-matrix transformation against the binary128 product, for a dense
    random matrix, a large boost (gamma ~ 700: rows that cancel) and a rotation whose entries
    include the FP64 remnants of cos(pi/2): within the stated bound, every vector taken."""
    g = syn.rng(160)
    v = syn.pxpypze(g, 20000)
    v[:100, 0] = 1e-30  # a component far below the others
    mats = [g.uniform(-2, 2, (4, 4)), orc.boost_matrix_def(np.array([0.6, -0.5, np.sqrt(0.389998)]))]
    c, s = np.cos(np.pi / 2), np.sin(np.pi / 2)
    R = np.eye(4)
    R[:2, :2] = [[c, -s], [s, c]]
    mats.append(R)
    for L in mats:
        cnt, out, ok = _apply(ffh, L, v)
        assert cnt == len(v) and ok.all()
        ref = orc.lorentz_apply_def(L, v)
        assert np.all(np.abs(out - ref) <= _apply_bound(L, v)), np.max(np.abs(out - ref) / _apply_bound(L, v))


def test_ff_lorentz_apply_domain(ffh, orc):
    """Zero rows are exact; a matrix with a non-finite entry, a row of denormals alone or a
    row scale beyond 2^400 is refused as a whole; a vector that is all zero, non-finite or
    scaled beyond 2^400 is refused alone."""
    g = syn.rng(161)
    L = g.uniform(-2, 2, (4, 4))
    L[2] = 0.0
    v = syn.pxpypze(g, 8)
    v[1] = 0.0
    v[2, 3] = np.inf
    v[3] *= 2.0 ** 420
    v[4] *= 2.0 ** -420
    cnt, out, ok = _apply(ffh, L, v)
    assert ok.tolist() == [True, False, False, False, False, True, True, True]
    assert np.all(out[ok][:, 2] == 0.0)
    ref = orc.lorentz_apply_def(L, v[ok])
    assert np.all(np.abs(out[ok] - ref) <= _apply_bound(L, v[ok]))
    for bad in (np.inf, 5e-324, 2.0 ** 410):
        L2 = L.copy()
        L2[1] = [bad, 0.0, 0.0, 0.0]
        assert _apply(ffh, L2, v)[0] == -1


def _pxpypzm_inputs(seed, n):
    """PxPyPzM legs: random pairs, then a quarter near-collinear with light second legs, and a
    quarter soft-hard (|p| ratios up to 3e4)."""
    g = syn.rng(seed)
    a, b = syn.pxpypze(g, n), syn.pxpypze(g, n)
    a[:, 3] = g.uniform(0, 10, n)
    b[:, 3] = g.uniform(0, 10, n)
    k = n // 4
    b[:k, :3] = a[:k, :3] * g.uniform(0.5, 2.0, (k, 1)) + a[:k, :3] * g.uniform(-1e-6, 1e-6, (k, 3))
    b[:k, 3] = g.uniform(0, 1e-3, k)
    b[k:2 * k, :3] *= 1e-4
    return a, b


def test_fixed_point_pxpypzm_mass_against_oracle(ffh, orc):
    """The PxPyPzM fast path (per-leg fixed point, float-float on non-negative terms) against the
    binary128 definition: within 2^-43 relative wherever it takes the pair; it takes every
    random pair and every soft-hard pair, FP64 and FP32 (one rounding)."""
    a, b = _pxpypzm_inputs(170, 40000)
    m, ok, m32, ok32 = _cart_fixed(ffh, a, b, coords=1)
    ref = orc.mass_cart_def(a, b, "pxpypzm")
    k = len(a) // 4
    assert ok[k:].all()
    assert np.max(np.abs(m[ok] - ref[ok]) / ref[ok]) <= 2.0 ** -43
    a32, b32 = syn.to_f32(a).astype(np.float64), syn.to_f32(b).astype(np.float64)
    _, _, m32, ok32 = _cart_fixed(ffh, a32, b32, coords=1)
    ref32 = orc.mass_cart_def(a32, b32, "pxpypzm")
    assert ok32[k:].all()
    assert np.max(np.abs(m32[ok32].astype(np.float64) - ref32[ok32]) / ref32[ok32]) <= 2.0 ** -24 * 1.01


def test_fixed_point_pxpypzm_mass_edges(ffh, orc):
    """Collinear massless legs (m = 0: refused), back-to-back legs, legs at rest, a dot product
    of exactly zero, scales 61 binades apart (refused) and a non-finite leg (refused)."""
    rows = [([0.0, 0.0, 1.0, 0.0], [0.0, 0.0, 3.0, 0.0]),
            ([1.0, 2.0, 3.0, 0.5], [-1.0, -2.0, -3.0, 0.5]),
            ([0.0, 0.0, 0.0, 2.0], [0.0, 0.0, 0.0, 3.0]),
            ([1.0, 0.0, 0.0, 0.1], [0.0, 1.0, 0.0, 0.2]),
            ([1.0, 0.0, 0.0, 0.0], [2.0 ** -61, 0.0, 0.0, 2.0 ** -61]),
            ([np.nan, 0.0, 0.0, 1.0], [1.0, 0.0, 0.0, 1.0])]
    a = np.array([r[0] for r in rows])
    b = np.array([r[1] for r in rows])
    m, ok, _, _ = _cart_fixed(ffh, a, b, coords=1)
    assert ok.tolist() == [False, True, True, True, False, False]
    ref = orc.mass_cart_def(a[ok], b[ok], "pxpypzm")
    assert np.all(np.abs(m[ok] - ref) <= 2.0 ** -43 * ref)
    assert m[2] == 5.0


def _convert(ffh, p, code):
    p = np.ascontiguousarray(p, dtype=np.float64)
    out, ok = np.full(p.shape, np.nan), np.zeros(len(p), np.uint8)
    ffh.ffh_convert(_p(p), ctypes.c_int64(len(p)), code, _p(out), _p(ok))
    return out, ok.astype(bool)


def conversion_scale(p, coords):
    """max(|E|, |p|) of each row, from the stored values (the conversion's error unit)."""
    if coords == "pxpypzm":
        pm = np.sqrt(np.sum(p[:, :3] ** 2, axis=1))
        return np.maximum(pm, np.sqrt(pm ** 2 + p[:, 3] ** 2))
    pm = np.abs(p[:, 0]) * np.cosh(p[:, 1])
    E = np.abs(p[:, 3]) if coords == "ptetaphie" else np.sqrt(pm ** 2 + p[:, 3] ** 2)
    return np.maximum(pm, E)


def test_ff_conversion_pxpypzm_to_pxpypze(ffh, orc):
    """The float-float conversion of PxPyPzM rows to PxPyPzE (E = sqrt(|p|^2 + m^2)) against the
    binary128 conversion: every component within 2^-44 max(|E|, |p|)."""
    g = syn.rng(192)
    c = syn.pxpypze(g, 20000)
    c[:, 3] = g.uniform(0, 10, len(c))
    out, ok = _convert(ffh, c, 2)
    assert ok.all()
    ref = orc.to_pxpypze_def(c, "pxpypzm")
    err = np.max(np.abs(out - ref), axis=1) / conversion_scale(c, "pxpypzm")
    assert err.max() <= 2.0 ** -44, np.log2(err.max())


def test_lc_conversion_to_pxpypze(ffh, orc):
    """The FP64 kernel's conversion (convert_ff.cuh ptetaphi_to_cart_lc: one paired reduction of
    (|eta|, |phi|) on the light-cone tables) of PtEtaPhiM and PtEtaPhiE rows against the binary128
    conversion: every component within 2^-43 max(|E|, |p|) (the bound gvx_to_pxpypze states), on
    the collider-like draws, tiny eta (sinh(eta) ~ eta kept), azimuths up to 3.5 and rows at
    the edges of the domain (negative pt, |eta| >= 8, NaN: refused; pt = 0 with a mass: taken)."""
    def conv(rows, code):
        rows = np.ascontiguousarray(rows, dtype=np.float64)
        out, ok = np.full(rows.shape, np.nan), np.zeros(len(rows), np.uint8)
        ffh.ffh_convert(_p(rows), ctypes.c_int64(len(rows)), code, _p(out), _p(ok))
        return out, ok.astype(bool)
    g = syn.rng(195)
    p = syn.ptetaphim_light_mix(g, 20000)
    p[::7, 1] = g.choice([1e-300, 1e-20, 1e-9, -1e-5], len(p[::7]))
    p[1::11, 2] = g.uniform(-3.5, 3.5, len(p[1::11])) * 0.9999
    e_on = orc.to_cartesian_def(p)[:, 3]
    pe = p.copy()
    pe[:, 3] = e_on * g.uniform(0.999, 1.5, len(p))
    for rows, coords, code in ((p, "ptetaphim", 0), (pe, "ptetaphie", 3)):
        out, ok = conv(rows, code)
        assert ok.all(), coords
        ref = orc.to_pxpypze_def(rows, coords)
        err = np.max(np.abs(out - ref), axis=1) / conversion_scale(rows, coords)
        assert err.max() <= 2.0 ** -43, (coords, np.log2(err.max()))
    edge = np.array([[0.0, 1.0, 0.5, 2.0], [-1.0, 1.0, 0.5, 2.0], [1.0, 8.0, 0.5, 2.0],
                     [1.0, 1.0, 3.1415927, 2.0], [1.0, np.nan, 0.5, 2.0], [1.0, 7.9, -np.pi, 0.0]])
    out, ok = conv(edge, 0)
    assert ok.tolist() == [True, False, False, True, False, True]
    ref = orc.to_pxpypze_def(edge[ok], "ptetaphim")
    assert np.all(np.abs(out[ok] - ref) <= 2.0 ** -43 * conversion_scale(edge[ok], "ptetaphim")[:, None])
    _, ok = conv(edge, 3)
    assert not ok[0]  # E stored: a zero pt leaves no scale


def test_fixed_point_masses_adversarial_property(ffh, orc):
    """Randomised adversarial legs for the fixed-point PxPyPzE and PxPyPzM masses (hypothesis):
    components with random signs, exact zeros and exponents spread over 2^-60 .. 2^60 of each
    other, second legs nearly collinear and nearly massless.  Wherever the fast path takes a pair
    it is within its bound of the binary128 definition (2^-44 and 2^-43 relative)."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    comp = st.tuples(st.sampled_from([-1.0, 0.0, 1.0]), st.floats(1.0, 2.0), st.integers(-60, 60))

    @hyp.settings(max_examples=300, deadline=None, derandomize=True)
    @hyp.given(st.lists(comp, min_size=4, max_size=4), st.floats(1e-12, 1e-3),
               st.floats(-1e-6, 1e-6), st.sampled_from([0, 1]))
    def check(c, mfrac, eps, coords):
        a = np.array([s * m * 2.0 ** e for s, m, e in c])
        p = a[:3]
        pn = np.sqrt(np.sum(p * p))
        if coords == 0:
            a[3] = abs(a[3]) + pn  # timelike or on the light cone
        b = a.copy()
        b[:3] = p * (1.0 + eps)
        b[3] = (np.sqrt(np.sum(b[:3] ** 2) + (mfrac * max(pn, 1e-300)) ** 2) if coords == 0
                else mfrac * max(pn, abs(a[3]), 1e-300))
        A, B = a[None, :], b[None, :]
        m, ok, _, _ = _cart_fixed(ffh, A, B, coords)
        if ok[0]:
            ref = orc.mass_cart_def(A, B, ("pxpypze", "pxpypzm")[coords])[0]
            tol = 2.0 ** -44 if coords == 0 else 2.0 ** -43
            assert abs(m[0] - ref) <= tol * abs(ref), (a, b, m[0], ref)

    check()


def test_lc_ptetaphie_mass_against_oracle(ffh, orc):
    """The light-cone PtEtaPhiE pair mass of the FP64 kernel (ptetaphie_lc.cuh: D = E - P,
    Y = E + P with the stored E) against the binary128 definition: within 2^-40 (M1 + M2)^2 in
    m|m| wherever it takes the pair, on on-shell and off-shell energies, near-collinear pairs,
    light/heavy mixes, azimuths across +-pi; it takes the random pairs; negative energies, -0,
    negative pt and legs with pt = E = 0 are left to the other route."""
    g = syn.rng(194)
    n = 40000
    p = syn.ptetaphim_light_mix(g, n)
    e = orc.to_cartesian_def(p)[:, 3]
    p[:, 3] = e * np.where(g.random(n) < 0.5, 1.0, g.uniform(1.0, 1.5, n))
    a, b = np.ascontiguousarray(p[: n // 2]), p[n // 2:].copy()
    b[:5000, 1] = a[:5000, 1] + 1e-7
    b[:5000, 2] = a[:5000, 2]
    b[5000:7000, 2] = -np.sign(a[5000:7000, 2]) * (np.pi - 1e-6 * g.random(2000))
    b = np.ascontiguousarray(b)
    m, ok = np.empty(len(a)), np.zeros(len(a), np.uint8)
    ffh.ffh_mass_e_lc(_p(a), _p(b), ctypes.c_int64(len(a)), _p(m), _p(ok))
    ok = ok.astype(bool)
    assert ok[7000:].mean() > 0.99
    ref = orc.mass_cart_def(a, b, "ptetaphie")
    M = conversion_scale(a, "ptetaphie") + conversion_scale(b, "ptetaphie")
    err = np.abs(m * np.abs(m) - ref * np.abs(ref)) / M ** 2
    assert err[ok].max() <= 2.0 ** -40, np.log2(err[ok].max())
    bad = np.ascontiguousarray(np.repeat(a[:1], 5, axis=0))
    bad[0, 3] = -bad[0, 3]
    bad[1, 3] = -0.0
    bad[2, 0] = -bad[2, 0]
    bad[3, 0] = bad[3, 3] = 0.0
    bad[4, 1] = 8.5
    m2, ok2 = np.empty(5), np.zeros(5, np.uint8)
    ffh.ffh_mass_e_lc(_p(bad), _p(np.ascontiguousarray(b[:5])), ctypes.c_int64(5), _p(m2), _p(ok2))
    assert not ok2.any()


def test_leg_paired_pair_mass_is_bit_identical(ffh):
    """The pair mass with its two legs on paired FP32 operations (the FP64 kernel's path) gives the
    scalar pair_mass_ff's bits, and takes the same pairs, on the collider-like draws, the
    light/heavy mix, near-collinear pairs, azimuthal wrap-around, negative and zero eta and tiny
    masses."""
    g = syn.rng(194)
    n = 40000
    a = syn.ptetaphim_light_mix(g, n)
    b = syn.ptetaphim_light_mix(g, n)
    k = n // 4
    b[:k, 1] = a[:k, 1] + g.uniform(-1e-7, 1e-7, k)
    b[:k, 2] = a[:k, 2] + g.uniform(-1e-7, 1e-7, k)
    b[k:2 * k, 2] = np.where(a[k:2 * k, 2] > 0, a[k:2 * k, 2] - 3.1, a[k:2 * k, 2] + 3.1)
    b[2 * k:2 * k + 500, 3] = 0.0
    a[2 * k + 500:2 * k + 1000, 3] = a[2 * k + 500:2 * k + 1000, 0] * 2.0 ** -29
    a[2 * k + 1000:2 * k + 1500, 1] = 0.0
    b[2 * k + 1000:2 * k + 1250, 1] = -a[2 * k + 1000:2 * k + 1250, 1]
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    m1, ok1 = _mass(ffh, a, b)
    assert ok1.mean() > 0.99
    m3, ok3 = np.empty(n), np.zeros(n, np.uint8)
    ffh.ffh_mass_lp(_p(a), _p(b), ctypes.c_int64(n), _p(m3), _p(ok3))
    ok3 = ok3.astype(bool)
    assert np.array_equal(ok3, ok1)
    assert np.array_equal(m1[ok1].view(np.uint64), m3[ok1].view(np.uint64))
