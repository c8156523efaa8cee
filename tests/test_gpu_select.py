"""GPU parity of gvx_event_pair_select (fused selection, pair-mass histogram and best candidate
per event) against the binary128 oracle.

Histogram: the totals are exact; a slot may differ from the oracle only by masses that sit within
1e-12 (relative) of one of its edges or its neighbours' (the oracle counts those), because the
two sides round the same mass differently.  Best candidate: the same pair, or one whose oracle
|m - target| is within 1e-12 relative of the oracle's best; best_m is that pair's mass to 1e-12.
"""
import numpy as np
import pytest

import gvx_synth as syn
from helpers import TOL_F64, dev, torch_cuda

pytestmark = pytest.mark.gpu

CUTS = dict(pt_min=20.0, eta_max=2.5, lo=0.0, hi=400.0, n_bins=200, target=91.1876)


def _run(p, off, layout="aos", counts=None, **cuts):
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    c, bk, bm = gvx.event_pair_select(dev(p, layout), torch.as_tensor(off).cuda(), counts=counts,
                                      layout=layout, **cuts)
    assert gvx.device_status() == 0
    return c.cpu().numpy().astype(np.uint64), bk.cpu().numpy(), bm.cpu().numpy()


def _check(orc, p, off, counts, bk, bm, **cuts):
    rc, near, rk, rm = orc.pair_select_def(p, off, cuts["pt_min"], cuts["eta_max"], cuts["lo"],
                                           cuts["hi"], cuts["n_bins"], cuts["target"])
    assert counts.sum() == rc.sum()
    slack = near + np.roll(near, 1) + np.roll(near, -1)
    assert np.all(np.abs(counts.astype(np.int64) - rc.astype(np.int64)) <= slack.astype(np.int64))
    assert np.array_equal(bk < 0, rk < 0)
    diff = np.flatnonzero(bk != rk)
    if len(diff):  # only near-ties may differ
        _, pm, _ = orc.event_pairs_def(p, off)
        c = np.diff(off)
        po = np.concatenate([[0], np.cumsum(c * (c - 1) // 2)])
        t = cuts["target"]
        for e in diff:
            m_got = pm[po[e] + bk[e]]
            assert abs(abs(m_got - t) - abs(rm[e] - t)) <= 1e-12 * max(m_got, t), e
    has = bk >= 0
    if has.any():
        _, pm, _ = orc.event_pairs_def(p, off)
        c = np.diff(off)
        po = np.concatenate([[0], np.cumsum(c * (c - 1) // 2)])
        want = pm[po[:-1][has] + bk[has]]
        assert np.all(np.abs(bm[has] - want) <= TOL_F64 * want)
    assert np.all(np.isnan(bm[~has]))


@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_select_small(orc, layout):
    g = syn.rng(70)
    counts = np.diff(syn.jagged_offsets(g, 3000))
    counts = np.concatenate([counts, [0, 1, 2, 65, 100, 300]])  # big events take the global path
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    p = syn.ptetaphim(g, int(off[-1]))
    p[3::101, 1] = 17.0  # outside the float-float domain (and the eta cut)
    c, bk, bm = _run(p, off, layout, **CUTS)
    _check(orc, p, off, c, bk, bm, **CUTS)


def test_select_edges_of_the_cuts_and_accumulation(orc):
    """No cut (every pair), cuts with particles exactly at pt_min and |eta| = eta_max, a single
    bin, and two calls adding into the same counts."""
    import torch
    g = syn.rng(71)
    off = syn.jagged_offsets(g, 800, lam=6.0, n_max=30)
    p = syn.ptetaphim(g, int(off[-1]))
    p[::13, 0] = 30.0
    p[1::17, 1] = -1.5
    cuts = dict(pt_min=30.0, eta_max=1.5, lo=50.0, hi=60.0, n_bins=1, target=55.0)
    c, bk, bm = _run(p, off, **cuts)
    _check(orc, p, off, c, bk, bm, **cuts)
    c2, _, _ = _run(p, off, counts=torch.as_tensor(c.astype(np.int64)).cuda(), **cuts)
    assert np.array_equal(c2, 2 * c)
    nocut = dict(pt_min=0.0, eta_max=np.inf, lo=0.0, hi=1e9, n_bins=4000, target=0.0)
    c, bk, bm = _run(p, off, **nocut)
    k = np.diff(off)
    assert c.sum() == np.sum(k * (k - 1) // 2)
    _check(orc, p, off, c, bk, bm, **nocut)


def test_select_full_size(orc):
    """2^20 events, Poisson(8): total count exact against the integer count of selected pairs,
    and 300 sampled events against the oracle."""
    g = syn.rng(72)
    off = syn.jagged_offsets(g, 1 << 20)
    p = syn.ptetaphim(g, int(off[-1]))
    c, bk, bm = _run(p, off, **CUTS)
    sel = (p[:, 0] >= CUTS["pt_min"]) & (np.abs(p[:, 1]) <= CUTS["eta_max"])
    cs = np.concatenate([[0], np.cumsum(sel)])
    n_sel = cs[off[1:]] - cs[off[:-1]]
    assert int(c.sum()) == int(np.sum(n_sel * (n_sel - 1) // 2))
    assert np.array_equal(bk >= 0, n_sel >= 2)
    for e in np.sort(syn.rng(172).choice(1 << 20, 300, replace=False)):
        lo, hi = off[e], off[e + 1]
        sub = np.array([0, hi - lo])
        _, _, rk, rm = orc.pair_select_def(p[lo:hi], sub, CUTS["pt_min"], CUTS["eta_max"],
                                           CUTS["lo"], CUTS["hi"], CUTS["n_bins"], CUTS["target"])
        if rk[0] < 0:
            assert bk[e] == -1 and np.isnan(bm[e])
        elif bk[e] == rk[0]:
            assert abs(bm[e] - rm[0]) <= TOL_F64 * rm[0]
        else:
            _, pm, _ = orc.event_pairs_def(p[lo:hi], sub)
            t = CUTS["target"]
            assert abs(abs(pm[bk[e]] - t) - abs(rm[0] - t)) <= 1e-12 * max(pm[bk[e]], t)


def test_select_rejects_bad_arguments():
    import ctypes
    import paper_2312_02756_gb300 as gvx
    from paper_2312_02756_gb300 import _lib
    torch = torch_cuda()
    lib = gvx.load_library()
    p = dev(syn.ptetaphim(syn.rng(73), 10))
    off = torch.as_tensor(np.array([0, 4, 10])).cuda()
    counts = torch.zeros(8, dtype=torch.int64, device="cuda")
    lv = ctypes.byref(gvx._lv(p, _lib.AOS, 4))
    args = lambda nb, lo, hi: (lv, ctypes.c_void_p(off.data_ptr()), 2, 10, 0.0, 5.0, lo, hi, nb,
                               91.0, ctypes.c_void_p(counts.data_ptr()), None, None, gvx._stream())
    assert lib.gvx_event_pair_select(*args(0, 0.0, 1.0)) == 2     # GVX_ERR_SIZE
    assert lib.gvx_event_pair_select(*args(5000, 0.0, 1.0)) == 2  # more bins than the maximum
    assert lib.gvx_event_pair_select(*args(6, 1.0, 1.0)) == 11    # GVX_ERR_ARG: empty range
    assert lib.gvx_event_pair_select(*args(6, 0.0, 100.0)) == 0   # NULL best_k / best_m allowed
    assert gvx.device_status() == 0 and int(counts.sum()) == 6 + 15
