"""GPU parity of gvx_event_pair_masses_bwd (the adjoint of the jagged pair masses and event sums)
against the binary128 oracle.

Error measure: per particle, the largest component error weighted by max(|x_k|, 1), relative to
the same weighting of the summed magnitudes of the contributions (|upstream| * |dm/dp| over the
particle's pairs, plus |J|^T |grad_event_sum|) -- the scale a correct summation in any order
reaches.  Gate 1e-12 (as the elementwise FP64 adjoint).
"""
import os

import numpy as np
import pytest

import gvx_synth as syn
from helpers import TOL_F64, dev, host, summary, torch_cuda

pytestmark = pytest.mark.gpu


def _n_pairs(off):
    c = np.diff(off)
    return int(np.sum(c * (c - 1) // 2))


def _pair_offsets(off):
    c = np.diff(off)
    return np.concatenate([[0], np.cumsum(c * (c - 1) // 2)]).astype(np.int64)


def _magnitudes(orc, p, off, gpm, gsum):
    """Per particle and component: sum of |contribution| over its pairs and the sum part."""
    mag = np.zeros_like(p)
    po = _pair_offsets(off)
    for e in range(len(off) - 1):
        n = off[e + 1] - off[e]
        if n < 2:
            continue
        ii, jj = np.triu_indices(n, 1)
        ii, jj = ii + off[e], jj + off[e]
        ga, gb = orc.mass_grad_def(p[ii], p[jj], np.abs(gpm[po[e]:po[e + 1]]))
        np.add.at(mag, ii, np.abs(ga))
        np.add.at(mag, jj, np.abs(gb))
    if gsum is not None:
        ev = np.repeat(np.arange(len(off) - 1), np.diff(off))
        zero = np.zeros_like(gpm)
        for r in range(4):
            unit = np.zeros((len(off) - 1, 4))
            unit[:, r] = 1.0
            J_r = orc.event_pairs_grad_def(p, off, zero, unit)
            mag += np.abs(J_r) * np.abs(gsum[ev, r])[:, None]
    return mag


def _err(got, ref, mag, p):
    s = np.maximum(np.abs(p), 1.0)
    den = np.sum(mag * s, axis=1)
    return np.max(np.abs(got - ref) * s, axis=1) / np.where(den > 0, den, 1.0)


def _gpu_bwd(p, off, gpm, gsum, layout="aos", sums_layout="aos", grad_layout="aos"):
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    gs = None if gsum is None else dev(gsum, sums_layout)
    out = gvx.event_pair_masses_bwd(dev(p, layout), torch.as_tensor(off).cuda(),
                                    torch.as_tensor(_pair_offsets(off)).cuda(),
                                    torch.as_tensor(np.ascontiguousarray(gpm)).cuda(), gs,
                                    layout=layout, sums_layout=sums_layout,
                                    grad_layout=grad_layout)
    assert gvx.device_status() == 0
    return host(out, grad_layout)


def _inputs(seed, n_events, extra_sizes=(0, 1, 2, 3, 65, 130)):
    g = syn.rng(seed)
    counts = np.diff(syn.jagged_offsets(g, n_events))
    counts = np.concatenate([counts, extra_sizes]).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    p = syn.ptetaphim(g, int(off[-1]))
    # a few particles outside the float-float domain and massless ones
    p[5::97, 1] = g.choice([-17.0, 18.5], len(p[5::97]))
    p[7::31, 3] = 0.0
    gpm = syn.upstream(g, _n_pairs(off))
    gsum = syn.upstream(g, (len(counts), 4))
    # upstream values outside the float-float ranges (FP64 pair and event-sum paths)
    gpm[::211] *= 1e-30
    gpm[1::307] *= 1e7
    gsum[3::50, :] *= 1e-100
    gsum[4::50, 2] *= 1e120
    return p, off, gpm, gsum


@pytest.mark.parametrize("layout,sums_layout,grad_layout",
                         [("aos", "aos", "aos"), ("soa", "soa", "soa"), ("aos", "soa", "soa")])
def test_event_pairs_bwd_small(orc, layout, sums_layout, grad_layout):
    p, off, gpm, gsum = _inputs(40, 1500)
    got = _gpu_bwd(p, off, gpm, gsum, layout, sums_layout, grad_layout)
    ref = orc.event_pairs_grad_def(p, off, gpm, gsum)
    err = _err(got, ref, _magnitudes(orc, p, off, gpm, gsum), p)
    assert np.all(np.isfinite(got))
    assert err.max() <= TOL_F64


def test_event_pairs_bwd_without_sum_gradient_and_deterministic(orc):
    p, off, gpm, _ = _inputs(41, 1000)
    a = _gpu_bwd(p, off, gpm, None)
    b = _gpu_bwd(p, off, gpm, None)
    assert np.array_equal(a, b)  # fixed summation order: bitwise repeatable
    ref = orc.event_pairs_grad_def(p, off, gpm)
    assert _err(a, ref, _magnitudes(orc, p, off, gpm, None), p).max() <= TOL_F64


def test_event_pairs_bwd_through_autograd(orc):
    """torch.autograd through event_pair_masses gives the kernel's gradient."""
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    p, off, gpm, gsum = _inputs(42, 400)
    x = dev(p).requires_grad_(True)
    toff = torch.as_tensor(off).cuda()
    po, pm, sums = gvx.event_pair_masses(x, toff, _n_pairs(off))
    loss = (pm * torch.as_tensor(gpm).cuda()).sum() + (sums * dev(gsum)).sum()
    loss.backward()
    assert gvx.device_status() == 0
    direct = _gpu_bwd(p, off, gpm, gsum)
    assert np.array_equal(x.grad.cpu().numpy(), direct)
    ref = orc.event_pairs_grad_def(p, off, gpm, gsum)
    assert _err(direct, ref, _magnitudes(orc, p, off, gpm, gsum), p).max() <= TOL_F64


def test_event_pairs_bwd_full_size(orc):
    """2^20 events, Poisson(8) multiplicities clamped to [0, 64]: every gradient against O2
    (pinned to O1 at 1e-14), each particle's error relative to its summed contribution
    magnitudes (O2's magnitudes mode); 300 sampled events against O1."""
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    g = syn.rng(43)
    off = syn.jagged_offsets(g, 1 << 20)
    p = syn.ptetaphim(g, int(off[-1]))
    gpm = syn.upstream(g, _n_pairs(off))
    gsum = syn.upstream(g, (1 << 20, 4))
    got = _gpu_bwd(p, off, gpm, gsum)
    assert np.all(np.isfinite(got))
    nt = os.cpu_count() or 8
    ref2 = orc.event_pairs_grad_fp64(p, off, gpm, gsum, nthreads=nt)
    mag2 = orc.event_pairs_grad_fp64(p, off, gpm, gsum, magnitudes=True, nthreads=nt)
    err2 = _err(got, ref2, mag2, p)
    print("jagged adjoint (%d particles) vs O2, every element: %s" % (len(p), summary(err2)))
    assert err2.max() <= TOL_F64
    del ref2, mag2, err2
    po = _pair_offsets(off)
    for e in np.sort(syn.rng(143).choice(1 << 20, 300, replace=False)):
        lo, hi = off[e], off[e + 1]
        sub = np.array([0, hi - lo])
        ref = orc.event_pairs_grad_def(p[lo:hi], sub, gpm[po[e]:po[e + 1]], gsum[e:e + 1])
        mag = _magnitudes(orc, p[lo:hi], sub, gpm[po[e]:po[e + 1]], gsum[e:e + 1])
        if hi > lo:
            assert _err(got[lo:hi], ref, mag, p[lo:hi]).max() <= TOL_F64, e
    del got
    torch.cuda.empty_cache()


def test_event_pairs_bwd_rejects_mismatched_pair_offsets():
    """Pair offsets that do not match the event sizes: GVX_ERR_OFFSETS on the device, no fault;
    the events of the other tiles (tiles hold at most 64 events) still get their gradients."""
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    p, off, gpm, gsum = _inputs(44, 500, extra_sizes=())
    po = _pair_offsets(off)
    bad = po.copy()
    bad[3] += 1  # event 2 and 3 no longer have n(n-1)/2 pairs
    grad = torch.full((len(p), 4), -7.0, dtype=torch.float64, device="cuda")
    lib = gvx.load_library()
    import ctypes
    from paper_2312_02756_gb300 import _lib
    lv = lambda t: ctypes.byref(gvx._lv(t, _lib.AOS, 4))
    tp, toff, tbad, tg = dev(p), torch.as_tensor(off).cuda(), torch.as_tensor(bad).cuda(), \
        torch.as_tensor(gpm).cuda()
    ws_bytes = lib.gvx_event_pair_masses_bwd_workspace(len(off) - 1)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    st = lib.gvx_event_pair_masses_bwd(lv(tp), ctypes.c_void_p(toff.data_ptr()),
                                       ctypes.c_void_p(tbad.data_ptr()), len(off) - 1, len(p),
                                       ctypes.c_void_p(tg.data_ptr()), len(gpm), None, lv(grad),
                                       ctypes.c_void_p(ws.data_ptr()), ws_bytes, gvx._stream())
    assert st == 0
    assert gvx.device_status() == 6
    g = grad.cpu().numpy()
    assert np.all(g[off[2]:off[4]] == -7.0)  # the tile holding events 2 and 3 was skipped
    assert np.all(g[off[64]:] != -7.0)  # tiles hold at most 64 events: the rest was written
    # an empty batch launches nothing and succeeds
    st = lib.gvx_event_pair_masses_bwd(lv(tp), ctypes.c_void_p(toff.data_ptr()),
                                       ctypes.c_void_p(tbad.data_ptr()), 0, 0, None, 0, None,
                                       lv(grad), None, 0, gvx._stream())
    assert st == 0 and gvx.device_status() == 0
    # a missing, short or misaligned workspace is refused before any launch
    args = (lv(tp), ctypes.c_void_p(toff.data_ptr()), ctypes.c_void_p(toff.data_ptr()),
            len(off) - 1, len(p), ctypes.c_void_p(tg.data_ptr()), len(gpm), None, lv(grad))
    assert lib.gvx_event_pair_masses_bwd(*args, None, ws_bytes, gvx._stream()) == 7
    assert lib.gvx_event_pair_masses_bwd(*args, ctypes.c_void_p(ws.data_ptr()), ws_bytes - 8,
                                         gvx._stream()) == 7
    assert lib.gvx_event_pair_masses_bwd(*args, ctypes.c_void_p(ws.data_ptr() + 8), ws_bytes,
                                         gvx._stream()) == 5
    assert gvx.device_status() == 0
