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
    from paper_2312_02756_gb300 import gen_tables
    d = tmp_path_factory.mktemp("ffh")
    gen_tables.write(str(d / "gvx_tables.inc"))
    out = str(d / "ffh.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-I" + str(d), os.path.join(HERE, "ff_harness.cpp"), "-o", out],
                   check=True)
    lib = ctypes.CDLL(out)
    lib.ffh_mass.restype = ctypes.c_int64
    return lib


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


def test_ff_boost_coefficients(ffh):
    """gamma = 1/sqrt(1 - b2) and k = gamma^2/(1 + gamma) of the FP64 boost, from the exact
    fixed-point 1 - b2, against mpmath."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    b = np.concatenate([syn.velocities(syn.rng(8), 1500, 0.99),
                        syn.velocities(syn.rng(9), 500, 0.99998),
                        [[0, 0, 0], [1e-9, -2e-9, 3e-9], [0.6, 0.8, 0.0]]])
    g, k = np.empty(len(b)), np.empty(len(b))
    ok = np.empty(len(b), np.uint8)
    ffh.ffh_boost_coef(_p(b), ctypes.c_int64(len(b)), _p(g), _p(k), _p(ok))
    ok = ok.astype(bool)
    assert not ok[-1] and ok[:-1].all()  # |beta| = 1 leaves the fast path
    for i in np.flatnonzero(ok):
        b2 = sum(mp.mpf(x) ** 2 for x in b[i])
        G = 1 / mp.sqrt(1 - b2)
        assert abs(g[i] / float(G) - 1) <= 3e-14
        assert abs(k[i] / float(G * G / (1 + G)) - 1) <= 3e-14
