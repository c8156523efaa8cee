"""GPU parity of the Cartesian-input pair mass (gvx_invariant_mass_cart) and of the general
Lorentz transformation (gvx_lorentz_apply) against the binary128 oracle.

Cartesian mass, FP64: 1e-12 relative (the cancellation-free form with an FMA-exact cross product
and E^2 - |p|^2).  FP32 legs are evaluated in FP64 and rounded once: within one float ulp of the
oracle on the exact upcast inputs.  Lorentz apply: each component within a few ulps of sum_k |L_rk v_k|
(no structure of L is assumed: 4 u for FP64, 4 u for FP32 with u the unit roundoff).
"""
import numpy as np
import pytest

import gvx_synth as syn
from helpers import TOL_F64, dev, host, summary, torch_cuda

pytestmark = pytest.mark.gpu


def _legs(seed, n, coords):
    g = syn.rng(seed)
    a, b = syn.pxpypze(g, n), syn.pxpypze(g, n)
    k = n // 4  # near-collinear light pairs
    b[:k, :3] = a[:k, :3] * g.uniform(0.5, 2.0, (k, 1))
    b[:k, :3] += a[:k, :3] * g.uniform(-1e-9, 1e-9, (k, 3))
    mb = g.uniform(0, 1e-3, k)
    b[:k, 3] = np.sqrt(np.sum(b[:k, :3] ** 2, axis=1) + mb * mb)
    if coords == "pxpypzm":
        a[:, 3] = g.uniform(0, 10, n)
        b[:, 3] = g.uniform(0, 10, n)
        b[:k, 3] = mb
    return a, b


def _mass(a, b, coords, la="aos", lb="aos", dtype=None):
    import paper_2312_02756_gb300 as gvx
    torch_cuda()
    m = gvx.invariant_mass_cart(dev(a, la, dtype), dev(b, lb, dtype), coords, layout_a=la, layout_b=lb)
    return m.cpu().numpy()


@pytest.mark.parametrize("coords", ["pxpypze", "pxpypzm"])
@pytest.mark.parametrize("la,lb", [("aos", "aos"), ("soa", "soa"), ("soa", "aos")])
def test_cart_mass_f64(orc, coords, la, lb):
    a, b = _legs(80, 65_537, coords)
    m = _mass(a, b, coords, la, lb)
    ref = orc.mass_cart_def(a, b, coords)
    err = np.abs(m - ref) / np.abs(ref)
    print("FP64 %s mass vs O1: %s" % (coords, summary(err)))
    assert err.max() <= TOL_F64


def test_cart_mass_f64_edges(orc):
    """Spacelike legs (E stored below |p|), massless legs, a zero leg, back-to-back legs and a
    pair whose sum is spacelike (negative mass by GenVector's convention)."""
    a = np.array([[3.0, 4.0, 12.0, 13.0], [0.0, 0.0, 0.0, 0.0], [1.0, 2.0, 3.0, 3.5],
                  [5.0, 0.0, 0.0, 5.0], [3.0, 4.0, 12.0, 12.999999], [1.0, 0.0, 0.0, 0.1]])
    b = np.array([[-4.0, 3.0, 12.0, 13.0], [1.0, 2.0, 3.0, 10.0], [0.0, 0.0, 0.0, 0.0],
                  [-5.0, 0.0, 0.0, 5.0], [3.0, 4.0, 12.0, 13.0], [1.0, 0.0, 0.0, 0.1]])
    m = _mass(a, b, "pxpypze")
    ref = orc.mass_cart_def(a, b, "pxpypze")
    assert np.all(np.abs(m - ref) <= TOL_F64 * np.abs(ref) + 1e-300)
    assert m[-1] < 0  # |p| = 2 > E = 0.2: spacelike sum


def test_cart_mass_f64_full_size_sampled(orc):
    torch = torch_cuda()
    n = 1 << 24
    a, b = _legs(81, n, "pxpypze")
    m = _mass(a, b, "pxpypze")
    idx = np.sort(syn.rng(181).choice(n, 1 << 15, replace=False))
    ref = orc.mass_cart_def(a[idx], b[idx], "pxpypze")
    assert np.all(np.isfinite(m))
    assert np.max(np.abs(m[idx] - ref) / np.abs(ref)) <= TOL_F64
    torch.cuda.empty_cache()


@pytest.mark.parametrize("coords", ["pxpypze", "pxpypzm"])
def test_cart_mass_f32_error(orc, coords):
    import torch
    a, b = _legs(82, 1 << 18, coords)
    a32, b32 = syn.to_f32(a), syn.to_f32(b)
    m = _mass(a32, b32, coords, dtype=torch.float32)
    ref = orc.mass_cart_def(a32.astype(np.float64), b32.astype(np.float64), coords)
    err = np.abs(m - ref) / np.abs(ref)
    print("FP32 %s mass vs O1: %s" % (coords, summary(err)))
    assert err.max() <= 2.0 ** -24 * 1.01  # the one final rounding to float


@pytest.mark.parametrize("dtype,u", [("f64", 2.0 ** -53), ("f32", 2.0 ** -24)])
@pytest.mark.parametrize("shared", [True, False])
def test_lorentz_apply(orc, dtype, u, shared):
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    g = syn.rng(83)
    n = 50_001
    v = syn.pxpypze(g, n)
    L = g.uniform(-2, 2, (4, 4)) if shared else g.uniform(-2, 2, (n, 4, 4))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":
        v, L = syn.to_f32(v).astype(np.float64), syn.to_f32(L).astype(np.float64)
    for layout in ("aos", "soa"):
        out = gvx.lorentz_apply(torch.as_tensor(L, dtype=tdt).cuda(), dev(v, layout, tdt), layout=layout)
        got = host(out, layout).astype(np.float64)
        ref = orc.lorentz_apply_def(L, v)
        Lf = np.broadcast_to(L, (n, 4, 4))
        scale = np.einsum("nrk,nk->nr", np.abs(Lf), np.abs(v))
        assert np.all(np.abs(got - ref) <= 4 * u * scale + 1e-300), (dtype, shared, layout)


def test_lorentz_apply_boost_matrix_matches_boost(orc):
    """A boost matrix applied as a general transformation agrees with gvx_boost within the
    general transformation's bound."""
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    g = syn.rng(84)
    v = syn.pxpypze(g, 10_000)
    beta = np.array([0.3, -0.45, 0.6])
    L = orc.boost_matrix_def(beta)
    out = gvx.lorentz_apply(torch.as_tensor(L).cuda(), dev(v)).cpu().numpy()
    ref = gvx.boost(dev(v), torch.as_tensor(beta).cuda()).cpu().numpy()
    scale = np.abs(v) @ np.abs(L).T
    assert np.all(np.abs(out - ref) <= 1e-14 * scale)
