"""GPU parity of the Cartesian-input pair mass (gvx_invariant_mass_cart) and of the general
Lorentz transformation (gvx_lorentz_apply) against the binary128 oracle.

Cartesian mass, FP64: 1e-12 relative (PxPyPzE pairs through the exact fixed-point evaluation,
the others through the cancellation-free FP64 form).  FP32 legs: within one rounding of the
oracle on the exact upcast inputs.  Lorentz apply: each component within 4 u sum_k |L_rk v_k|
(u the unit roundoff) for the FMA chains (FP32, a matrix per vector), and within
2^-42 sum_k |L_rk v_k| + 2^-70 max_k |L_rk| max_k |v_k| for one shared FP64 matrix (float-float).
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
        assert np.all(np.abs(got - ref) <= _apply_bound(L, v, dtype == "f64" and shared, u)), \
            (dtype, shared, layout)


def _apply_bound(L, v, ff, u=2.0 ** -53):
    Lf = np.broadcast_to(L, (len(v), 4, 4))
    scale = np.einsum("nrk,nk->nr", np.abs(Lf), np.abs(v))
    if not ff:
        return 4 * u * scale + 1e-300
    floor = np.max(np.abs(Lf), axis=2) * np.max(np.abs(v), axis=1)[:, None]
    # + the absolute rounding of a result that underflows (the FMA chains on a denormal row)
    return 2.0 ** -42 * scale + 2.0 ** -70 * floor + 2.0 ** -1074


def test_lorentz_apply_f64_shared_domain(orc):
    """Vectors outside the float-float domain (all zero, scaled beyond 2^400 either way) and a
    matrix outside it (a row of denormals alone) take the FP64 FMA chains: every component
    within the bound either way, zero rows exact."""
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    g = syn.rng(85)
    v = syn.pxpypze(g, 4096)
    v[::7] = 0.0
    v[1::7] *= 2.0 ** 420
    v[2::7] *= 2.0 ** -420
    v[3::7, 0] = 1e-30
    L = g.uniform(-2, 2, (4, 4))
    L[2] = 0.0
    L_den = L.copy()
    L_den[1] = [5e-324, 0.0, -1e-310, 0.0]
    for M in (L, L_den):
        out = gvx.lorentz_apply(torch.as_tensor(M).cuda(), dev(v)).cpu().numpy()
        ref = orc.lorentz_apply_def(M, v)
        assert np.all(np.abs(out - ref) <= _apply_bound(M, v, True))
        assert np.all(out[:, 2] == 0.0)


def test_lorentz_apply_boost_matrix_matches_boost(orc):
    """A boost matrix applied as a general transformation agrees with gvx_boost within the sum
    of the two kernels' bounds."""
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    g = syn.rng(84)
    v = syn.pxpypze(g, 10_000)
    beta = np.array([0.3, -0.45, 0.6])
    L = orc.boost_matrix_def(beta)
    out = gvx.lorentz_apply(torch.as_tensor(L).cuda(), dev(v)).cpu().numpy()
    ref = gvx.boost(dev(v), torch.as_tensor(beta).cuda()).cpu().numpy()
    scale = np.abs(v) @ np.abs(L).T
    # the transformation's float-float bound plus the boost's own (normwise on E')
    assert np.all(np.abs(out - ref) <= 2.0 ** -42 * (scale + scale[:, 3:4]))


def test_device_fast_paths_match_host_build(orc, tmp_path):
    """The device builds of the fixed-point pair masses and of the float-float transformation
    agree with the same headers compiled for the host (whose accuracy the CPU tests check case by
    case), wherever the host build takes the fast path: the transformation bit for bit, the masses
    within 2^-44 relative (FP32: one float ulp), since the float-float square root starts from the
    device's approximate reciprocal square root and from the host's own."""
    import ctypes
    import paper_2312_02756_gb300 as gvx
    from helpers import build_ff_harness
    torch = torch_cuda()
    ffh = build_ff_harness(tmp_path)
    P = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    g = syn.rng(86)
    n = 1 << 16
    for coords, code in (("pxpypze", 0), ("pxpypzm", 1)):
        a, b = _legs(87 + code, n, coords)
        m = _mass(a, b, coords)
        hm, ok = np.empty(n), np.empty(n, np.uint8)
        m32, ok32 = np.empty(n, np.float32), np.empty(n, np.uint8)
        ffh.ffh_mass_cart_fixed(P(a), P(b), ctypes.c_int64(n), code, P(hm), P(ok), P(m32), P(ok32))
        ok = ok.astype(bool)
        assert ok.mean() > 0.7
        assert np.all(np.abs(m[ok] - hm[ok]) <= 2.0 ** -44 * np.abs(hm[ok])), coords
        d32 = _mass(a.astype(np.float32), b.astype(np.float32), coords, dtype=torch.float32)
        ok32 = ok32.astype(bool)
        dm = np.abs(d32[ok32].astype(np.float64) - m32[ok32].astype(np.float64))
        assert np.all(dm <= 2.0 ** -23 * np.abs(m32[ok32].astype(np.float64))), coords
    v = syn.pxpypze(g, n)
    L = np.ascontiguousarray(g.uniform(-2, 2, (4, 4)))
    out = gvx.lorentz_apply(torch.as_tensor(L).cuda(), dev(v)).cpu().numpy()
    hout, hok = np.empty_like(v), np.empty(n, np.uint8)
    assert ffh.ffh_apply(P(L), P(v), ctypes.c_int64(n), P(hout), P(hok)) == n
    assert np.array_equal(out, hout)


def _conv_inputs(seed, n):
    """PtEtaPhiM (light/heavy mix), PtEtaPhiE (energies from on-shell to 1.5x) and PxPyPzM rows."""
    g = syn.rng(seed)
    p = syn.ptetaphim_light_mix(g, n)
    pe = p.copy()
    pe[:, 3] = orc_energy(p) * g.uniform(0.999, 1.5, n)
    c = syn.pxpypze(g, n)
    c[:, 3] = g.uniform(0, 10, n)
    return {"ptetaphim": p, "ptetaphie": pe, "pxpypzm": c}


def orc_energy(p):
    import oracle
    return oracle.to_cartesian_def(p)[:, 3]


def _scale(p, coords):
    if coords == "pxpypzm":
        pm = np.sqrt(np.sum(p[:, :3] ** 2, axis=1))
        return np.sqrt(pm ** 2 + p[:, 3] ** 2)
    pm = np.abs(p[:, 0]) * np.cosh(p[:, 1])
    E = np.abs(p[:, 3]) if coords == "ptetaphie" else np.sqrt(pm ** 2 + p[:, 3] ** 2)
    return np.maximum(pm, E)


@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_to_pxpypze(orc, layout):
    """Conversion of PtEtaPhiM, PtEtaPhiE and PxPyPzM vectors to PxPyPzE against the binary128
    conversion: FP64 within 2^-43 max(|E|, |p|) per component, FP32 (CUDA's float functions, on
    the float inputs) within 2^-20 of it."""
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    for coords, p in _conv_inputs(93, 50_001).items():
        ref = orc.to_pxpypze_def(p, coords)
        out = host(gvx.to_pxpypze(dev(p, layout), coords, layout=layout), layout)
        err = np.max(np.abs(out - ref), axis=1) / _scale(p, coords)
        print("FP64 %s -> PxPyPzE: %s" % (coords, summary(err)))
        assert err.max() <= 2.0 ** -43, coords
        p32 = syn.to_f32(p).astype(np.float64)
        ref32 = orc.to_pxpypze_def(p32, coords)
        out32 = host(gvx.to_pxpypze(dev(p32, layout, torch.float32), coords, layout=layout), layout)
        err32 = np.max(np.abs(out32.astype(np.float64) - ref32), axis=1) / _scale(p32, coords)
        assert err32.max() <= 2.0 ** -20, coords


def test_to_pxpypze_edges_and_boost(orc):
    """Rows outside the float-float domain (negative pt, |eta| >= 16, pt = 0 with E stored) take
    the FP64 formulas; a PtEtaPhiM array converted and then boosted matches the binary128
    conversion and boost within 1e-12 gamma (E + |beta| |p|) per component (the conversion's
    error times the boost's amplification, plus the boost's own)."""
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    edge = np.array([[-2.0, 1.0, 0.5, 2.0], [1.0, 17.0, 0.5, 2.0], [0.0, 1.0, 0.5, 3.0],
                     [5.0, -16.5, -3.0, 1e-3], [1.0, 0.0, 0.0, 0.0]])
    for coords in ("ptetaphim", "ptetaphie"):
        out = gvx.to_pxpypze(dev(edge), coords).cpu().numpy()
        ref = orc.to_pxpypze_def(edge, coords)
        assert np.all(np.abs(out - ref) <= 2.0 ** -43 * _scale(edge, coords)[:, None] + 1e-300)
    g = syn.rng(94)
    p = syn.ptetaphim(g, 20_000)
    beta = syn.velocities(g, 20_000)
    v = gvx.to_pxpypze(dev(p), "ptetaphim")
    got = gvx.boost(v, torch.as_tensor(beta).cuda()).cpu().numpy()
    vin = orc.to_pxpypze_def(p, "ptetaphim")
    ref = orc.boost_def(vin, beta)
    bn = np.linalg.norm(beta, axis=1)
    scale = (vin[:, 3] + bn * np.linalg.norm(vin[:, :3], axis=1)) / np.sqrt(1 - bn * bn)
    assert np.all(np.max(np.abs(got - ref), axis=1) <= 1e-12 * scale)


def test_ptetaphie_mass(orc):
    """PtEtaPhiE pair masses: within 2^-40 (M1 + M2)^2 in m|m| of the binary128 definition
    (M_i = max(|E_i|, pt_i cosh eta_i)), FP64 (the float-float identity, else both legs converted
    and the exact fixed-point mass), AoS and SoA, random and near-collinear pairs; FP32 (the
    additive form m1^2 + m2^2 + 2 (E1 E2 - P1 P2) + 4 pt1 pt2 S with CUDA's float functions)
    within 2^-19 (M1 + M2)^2, both layouts."""
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    p = _conv_inputs(95, 40_000)["ptetaphie"]
    a, b = p[:20_000], p[20_000:].copy()
    b[:5000, 1] = a[:5000, 1] + 1e-6
    b[:5000, 2] = a[:5000, 2]
    ref = orc.mass_cart_def(a, b, "ptetaphie")
    M = _scale(a, "ptetaphie") + _scale(b, "ptetaphie")
    for la, lb in (("aos", "aos"), ("soa", "soa")):
        m = _mass(a, b, "ptetaphie", la, lb)
        err = np.abs(m * np.abs(m) - ref * np.abs(ref)) / M ** 2
        print("FP64 ptetaphie mass, normwise in m|m|: %s" % summary(err))
        assert err.max() <= 2.0 ** -40
    a32, b32 = syn.to_f32(a).astype(np.float64), syn.to_f32(b).astype(np.float64)
    ref32 = orc.mass_cart_def(a32, b32, "ptetaphie")
    for la, lb in (("aos", "aos"), ("soa", "soa")):
        m32 = _mass(a32, b32, "ptetaphie", la, lb, dtype=torch.float32).astype(np.float64)
        err32 = np.abs(m32 * np.abs(m32) - ref32 * np.abs(ref32)) / M ** 2
        print("FP32 ptetaphie mass (%s), normwise in m|m|, units of 2^-24 (M1 + M2)^2: %s"
              % (la, summary(err32 * 2.0 ** 24)))
        assert err32.max() <= 2.0 ** -19


@pytest.mark.parametrize("coords", ["pxpypze", "pxpypzm", "ptetaphie"])
def test_cart_mass_nan_propagates_and_mixed_layouts(orc, coords):
    """A NaN in any component of either leg gives a NaN mass (the fast paths refuse the pair and
    the FP64 form propagates it), in FP64 and FP32; SoA against AoS legs give the same bits."""
    import torch
    g = syn.rng(96)
    if coords == "ptetaphie":
        a, b = _conv_inputs(97, 2 * 4096)["ptetaphie"][:4096], _conv_inputs(97, 2 * 4096)["ptetaphie"][4096:]
    else:
        a, b = _legs(98, 4096, coords)
    rows = g.choice(4096, 64, replace=False)
    for t, r in enumerate(rows):
        (a if t % 2 else b)[r, t % 4] = np.nan
    for dtype in (None, torch.float32):
        m = _mass(a, b, coords, "soa", "aos", dtype=dtype)
        assert np.all(np.isnan(m[rows]))
        others = np.setdiff1d(np.arange(4096), rows)
        assert np.all(np.isfinite(m[others]))
        m2 = _mass(a, b, coords, "aos", "soa", dtype=dtype)
        assert np.array_equal(np.isnan(m2), np.isnan(m)) and np.array_equal(m2[others], m[others])


def test_coordinates_workload_full_size_sampled(orc):
    """The benchmark's coordinate-system workload at its full size (2^26 FP64 elements, SoA, the
    same seeded inputs as bench.py's coords form): 2^14 sampled outputs of every kernel -- the
    PxPyPzE, PxPyPzM and PtEtaPhiE pair masses, the conversion and the shared-matrix
    transformation -- against the oracle within each kernel's bound."""
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    n = 1 << 26
    idx = np.sort(syn.rng(187).choice(n, 1 << 14, replace=False))
    g = syn.rng(5)
    a, b = syn.pxpypze(g, n), syn.pxpypze(g, n)
    m = gvx.invariant_mass_cart(dev(a, "soa"), dev(b, "soa"), "pxpypze", "soa", "soa").cpu().numpy()
    ref = orc.mass_cart_def(a[idx], b[idx], "pxpypze")
    assert np.max(np.abs(m[idx] - ref) / np.abs(ref)) <= 2.0 ** -44
    gm = syn.rng(6)
    a[:, 3], b[:, 3] = gm.uniform(0.0, 10.0, n), gm.uniform(0.0, 10.0, n)
    m = gvx.invariant_mass_cart(dev(a, "soa"), dev(b, "soa"), "pxpypzm", "soa", "soa").cpu().numpy()
    ref = orc.mass_cart_def(a[idx], b[idx], "pxpypzm")
    assert np.max(np.abs(m[idx] - ref) / np.abs(ref)) <= 2.0 ** -43
    del a, b, m
    torch.cuda.empty_cache()
    gp = syn.rng(7)
    pa, pb = syn.ptetaphim(gp, n), syn.ptetaphim(gp, n)
    for x in (pa, pb):
        x[:, 3] = np.sqrt((x[:, 0] * np.cosh(x[:, 1])) ** 2 + x[:, 3] ** 2)
    m = gvx.invariant_mass_cart(dev(pa, "soa"), dev(pb, "soa"), "ptetaphie", "soa", "soa").cpu().numpy()
    ref = orc.mass_cart_def(pa[idx], pb[idx], "ptetaphie")
    M = _scale(pa[idx], "ptetaphie") + _scale(pb[idx], "ptetaphie")
    assert np.max(np.abs(m[idx] * np.abs(m[idx]) - ref * np.abs(ref)) / M ** 2) <= 2.0 ** -40
    vd = gvx.to_pxpypze(dev(pa, "soa"), "ptetaphie", layout="soa")
    v = host(vd, "soa")
    ref = orc.to_pxpypze_def(pa[idx], "ptetaphie")
    assert np.max(np.max(np.abs(v[idx] - ref), axis=1) / _scale(pa[idx], "ptetaphie")) <= 2.0 ** -43
    L = np.array([[1.2, 0.1, 0.0, 0.5], [0.1, 1.1, 0.2, 0.0], [0.0, 0.2, 1.3, 0.4], [0.5, 0.0, 0.4, 1.5]])
    w = host(gvx.lorentz_apply(torch.as_tensor(L).cuda(), vd, layout="soa"), "soa")
    ref = orc.lorentz_apply_def(L, v[idx])
    assert np.all(np.abs(w[idx] - ref) <= _apply_bound(L, v[idx], True))
    del pa, pb, m, v, vd, w
    torch.cuda.empty_cache()
