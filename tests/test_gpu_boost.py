"""GPU parity of gvx_boost against the binary128 definition oracle (O1: the 4x4 matrix built
and applied in binary128).

Error measure (per vector, normwise): max_k |x'_k - ref_k| / E'_ref -- a component can vanish,
the energy cannot (E' >= |p'|).  FP64 gate 1e-12; FP32 error measured and bounded.
"""
import os

import numpy as np
import pytest

import gvx_synth as syn
from helpers import TOL_F64, dev, host, normwise, summary, torch_cuda

pytestmark = pytest.mark.gpu

N0 = 65_536
N_FULL = 1 << 26


def _run(v, beta, lv="aos", lb="aos", dtype=None):
    import paper_2312_02756_gb300 as gvx
    if beta.ndim == 2:
        bt = dev(beta, lb, dtype)
        out = gvx.boost(dev(v, lv, dtype), bt, layout=lv, beta_layout=lb)
    else:
        bt = dev(beta.reshape(1, 3), "aos", dtype)[0]
        out = gvx.boost(dev(v, lv, dtype), bt, layout=lv)
    return host(out, lv)


@pytest.mark.parametrize("lv,lb", [("aos", "aos"), ("soa", "soa"), ("soa", "aos"), ("aos", "soa")])
def test_boost_f64_small_workload(orc, lv, lb):
    torch_cuda()
    g = syn.rng(3)
    v, beta = syn.pxpypze(g, N0), syn.velocities(g, N0, 0.99)
    ref = orc.boost_def(v, beta, nthreads=8)
    out = _run(v, beta, lv, lb)
    err = normwise(out, ref, ref[:, 3])
    print("FP64 boost vs O1 (%s/%s): %s" % (lv, lb, summary(err)))
    assert err.max() <= TOL_F64


def test_boost_f64_shared_velocity_and_edges(orc):
    torch_cuda()
    g = syn.rng(4)
    n = 10_007
    v = syn.pxpypze(g, n)
    for beta in (np.array([0.3, -0.5, 0.2]), np.zeros(3), np.array([0.0, 0.0, 0.999999])):
        out = _run(v, beta)
        ref = orc.boost_def(v, beta, nthreads=8)
        if not beta.any():
            assert np.array_equal(out, v)  # identity, bit for bit
        assert normwise(out, ref, ref[:, 3]).max() <= TOL_F64
    # |beta| close to 1 per vector, and superluminal velocities -> NaN
    beta = syn.velocities(g, n, 0.999999)
    beta[::97] *= 1.0 / np.linalg.norm(beta[::97], axis=1, keepdims=True)  # |beta| = 1
    beta[1::97] *= 1.5 / np.linalg.norm(beta[1::97], axis=1, keepdims=True)
    out, ref = _run(v, beta), orc.boost_def(v, beta, nthreads=8)
    fin = np.isfinite(ref[:, 3])
    assert np.array_equal(np.isnan(out).all(axis=1), ~fin)
    assert normwise(out[fin], ref[fin], ref[fin, 3]).max() <= TOL_F64
    # rest frame: boosting by -p/E gives (0, 0, 0, m).  Here |beta| -> 1 (gamma = E/m up to
    # ~1e4), so the gate is the forward error bound of the vector form: gamma and w carry a
    # relative error below 3e-14 (float-float, pinned by the host tests) and the multiply-adds
    # round in FP64,  |x'_k - ref_k| <= (3e-14 + 16 u) gamma (E + |beta| |p|),  u = 2^-53
    w = v[:1000]
    bw = -w[:, :3] / w[:, 3:4]
    rest, ref = _run(w, bw), orc.boost_def(w, bw)
    gam = 1 / np.sqrt(1 - np.sum(bw * bw, axis=1))
    scale = gam * (w[:, 3] + np.linalg.norm(bw, axis=1) * np.linalg.norm(w[:, :3], axis=1))
    tol = 3e-14 + 16 * 2.0 ** -53
    assert np.all(normwise(rest, ref, scale) <= tol)
    assert np.all(np.abs(rest[:, 3] - orc.lv_mass_def(w)) <= tol * scale)


@pytest.mark.parametrize("n", [1, 3, 33, 257, 65_539])
def test_boost_f64_ragged(orc, n):
    torch_cuda()
    g = syn.rng(20 + n)
    v, beta = syn.pxpypze(g, n), syn.velocities(g, n, 0.99)
    ref = orc.boost_def(v, beta)
    for lv in ("aos", "soa"):
        assert normwise(_run(v, beta, lv, lv), ref, ref[:, 3]).max() <= TOL_F64


@pytest.mark.parametrize("layout", ["soa", "aos"])
def test_boost_f64_full_size(orc, layout):
    """All 2^26 boosts by per-vector beta (|beta| <= 0.99) against O2 (the FP64 vector form,
    pinned to O1 at 1e-14), normwise relative to E'; plus a uniform sample and the 4096
    worst-conditioned vectors against O1."""
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    g = syn.rng(1)
    v, beta = syn.pxpypze(g, N_FULL), syn.velocities(g, N_FULL, 0.99)
    dv, db = dev(v, layout), dev(beta, layout)
    out = gvx.boost(dv, db, layout=layout, beta_layout=layout)
    torch.cuda.synchronize()
    del dv, db
    oh = host(out, layout)
    del out
    torch.cuda.empty_cache()
    assert np.all(np.isfinite(oh))
    ref2 = orc.boost_fp64(v, beta, nthreads=os.cpu_count() or 8)
    err2 = normwise(oh, ref2, ref2[:, 3])
    print("FP64 boost 2^26 (%s) vs O2, every element: %s" % (layout, summary(err2)))
    assert err2.max() <= TOL_F64
    del ref2, err2
    # a uniform sample plus the 4096 worst-conditioned vectors: there p' nearly cancels (the
    # boost lands close to the vector's rest frame) and (E + |beta| |p|) / (E + beta.p) is largest
    cond = (v[:, 3] + np.linalg.norm(beta, axis=1) * np.linalg.norm(v[:, :3], axis=1)) / (
        v[:, 3] + np.sum(beta * v[:, :3], axis=1))
    worst = np.argpartition(cond, -4096)[-4096:]
    del cond
    idx = np.union1d(syn.rng(102).choice(N_FULL, 1 << 16, replace=False), worst)
    ref = orc.boost_def(v[idx], beta[idx], nthreads=8)
    err1 = normwise(oh[idx], ref, ref[:, 3])
    print("FP64 boost 2^26 (%s) vs O1, sample + worst-conditioned: %s" % (layout, summary(err1)))
    assert err1.max() <= TOL_F64


def test_boost_f32_error_per_output(orc):
    """FP32 vectors, |beta| up to 0.999999 (gamma ~ 707): 1 - beta^2 from exact FP32 products."""
    torch = torch_cuda()
    g = syn.rng(5)
    n = 1 << 20
    v32 = syn.to_f32(syn.pxpypze(g, n))
    b32 = syn.to_f32(syn.velocities(g, n, 0.999999))
    ok = np.sum(b32.astype(np.float64) ** 2, axis=1) < 1
    ref = orc.boost_def(v32.astype(np.float64), b32.astype(np.float64), nthreads=8)
    # forward error bound of the vector form with every operation rounded to FP32: each output
    # component is a sum of terms bounded by gamma (E + |beta| |p|), so
    #   |x'_k - ref_k| <= c u gamma (E + |beta| |p|),  u = 2^-24;  c = 16 covers the ~8 roundings
    vd, bd = v32.astype(np.float64)[ok], b32.astype(np.float64)[ok]
    gam = 1 / np.sqrt(1 - np.sum(bd * bd, axis=1))
    scale = gam * (vd[:, 3] + np.linalg.norm(bd, axis=1) * np.linalg.norm(vd[:, :3], axis=1))
    for lv in ("aos", "soa"):
        out = _run(v32, b32, lv, lv, torch.float32)
        assert out.dtype == np.float32
        err = normwise(out[ok], ref[ok], ref[ok, 3])
        print("FP32 boost vs O1 (%s), relative to E': %s" % (lv, summary(err)))
        print("   in units of u gamma (E + |beta||p|): %s"
              % summary(normwise(out[ok], ref[ok], scale * 2.0 ** -24)))
        assert np.all(normwise(out[ok], ref[ok], scale) <= 16 * 2.0 ** -24)
