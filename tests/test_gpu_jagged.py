"""GPU parity of gvx_event_pair_masses (jagged events, one persistent launch) against the oracle.

pair_offsets: bit-exact against the integer running sum.  Pair masses: 1e-12 relative (as the
elementwise FP64 mass).  Event sums: normwise, |sum - ref| <= 1e-12 * sum_i |E_i| (any summation
order is correct).
"""
import ctypes
import os

import numpy as np
import pytest

import gvx_synth as syn
from helpers import TOL_F64, dev, host, summary, torch_cuda

pytestmark = pytest.mark.gpu


def _n_pairs(off):
    c = np.diff(off)
    return int(np.sum(c * (c - 1) // 2))


def _run(p, off, layout="aos", sums_layout="aos"):
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    po, pm, s = gvx.event_pair_masses(dev(p, layout), torch.as_tensor(off).cuda(), _n_pairs(off),
                                      sums_layout=sums_layout)
    assert gvx.device_status() == 0
    return po.cpu().numpy(), pm.cpu().numpy(), host(s, sums_layout)


def _check(orc, p, off, po, pm, sums, events=None):
    c = np.diff(off)
    want_off = np.concatenate([[0], np.cumsum(c * (c - 1) // 2)])
    assert np.array_equal(po, want_off)
    cart = orc.to_cartesian_def(p) if len(p) else np.zeros((0, 4))
    events = range(len(c)) if events is None else events
    for e in events:
        lo, hi = off[e], off[e + 1]
        sub = off[e:e + 2] - lo
        r_off, r_m, r_s = orc.event_pairs_def(p[lo:hi], sub)
        got = pm[po[e]:po[e + 1]]
        assert np.all(np.abs(got - r_m) <= TOL_F64 * r_m + 1e-300), e
        mag = np.abs(cart[lo:hi]).sum() if hi > lo else 0.0
        assert np.all(np.abs(sums[e] - r_s[0]) <= TOL_F64 * mag), e


@pytest.mark.parametrize("layout,sums_layout", [("aos", "aos"), ("soa", "soa"), ("aos", "soa")])
def test_event_pairs_small(orc, layout, sums_layout):
    g = syn.rng(3)
    off = syn.jagged_offsets(g, 3000)
    p = syn.ptetaphim(g, int(off[-1]))
    po, pm, sums = _run(p, off, layout, sums_layout)
    _check(orc, p, off, po, pm, sums)


def test_event_pairs_match_elementwise_mass():
    """Each pair mass agrees with gvx_invariant_mass of the same two particles: both kernels take
    the same light-cone float-float arithmetic (each within ~1.2e-13 of the exact mass), the
    jagged one with per-particle terms at its event's scale; on the device their last bits may
    differ, so the bound is the two paths' combined error, 2.5e-13 relative."""
    import paper_2312_02756_gb300 as gvx
    g = syn.rng(30)
    off = syn.jagged_offsets(g, 500)
    p = syn.ptetaphim(g, int(off[-1]))
    po, pm, _ = _run(p, off)
    ia, ib = [], []
    for e in range(500):
        ii, jj = np.triu_indices(off[e + 1] - off[e], 1)
        ia.append(off[e] + ii)
        ib.append(off[e] + jj)
    ia, ib = np.concatenate(ia), np.concatenate(ib)
    m = gvx.invariant_mass(dev(p[ia]), dev(p[ib])).cpu().numpy()
    rel = np.abs(pm - m) / m
    print("jagged vs elementwise FP64 masses: max rel diff %.3e, equal bits %.4f"
          % (rel.max(), np.mean(pm == m)))
    assert rel.max() <= 2.5e-13


def test_event_pairs_edge_events(orc):
    g = syn.rng(31)
    counts = np.array([0, 1, 2, 0, 0, 64, 1, 3, 0, 1100, 5, 0, 2, 1], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    p = syn.ptetaphim(g, int(off[-1]))
    po, pm, sums = _run(p, off)
    small = [e for e in range(len(counts)) if counts[e] != 1100]
    _check(orc, p, off, po, pm, sums, small)
    # the 1100-particle event (larger than the shared-memory stage): sampled pairs
    e = int(np.flatnonzero(counts == 1100)[0])
    n = 1100
    k = np.sort(syn.rng(32).choice(n * (n - 1) // 2, 4000, replace=False))
    ii, jj = np.triu_indices(n, 1)
    ref = orc.mass_def(p[off[e] + ii[k]], p[off[e] + jj[k]])
    got = pm[po[e] + k]
    assert np.all(np.abs(got - ref) <= TOL_F64 * ref)
    cart = orc.to_cartesian_def(p[off[e]:off[e + 1]])
    assert np.all(np.abs(sums[e] - cart.sum(axis=0)) <= TOL_F64 * np.abs(cart).sum())
    # all events empty, and no events at all
    off0 = np.zeros(9, dtype=np.int64)
    po, pm, sums = _run(np.zeros((0, 4)), off0)
    assert np.array_equal(po, off0) and np.all(sums == 0)
    po, pm, sums = _run(np.zeros((0, 4)), np.zeros(1, dtype=np.int64))
    assert np.array_equal(po, [0])


def test_event_pairs_full_size(orc):
    """2^20 events, Poisson(8) multiplicities: offsets exact everywhere; every pair mass and
    every event sum against O2 (pinned to O1 at 1e-14); 400 events against O1."""
    g = syn.rng(3)
    off = syn.jagged_offsets(g, 1 << 20)
    p = syn.ptetaphim(g, int(off[-1]))
    po, pm, sums = _run(p, off)
    assert np.all(np.isfinite(pm)) and np.all(pm >= 0)
    r_off, r_m, r_s = orc.event_pairs_fp64(p, off, nthreads=os.cpu_count() or 8)
    assert np.array_equal(po, r_off)
    pos = r_m > 0
    rel = np.abs(pm[pos] - r_m[pos]) / r_m[pos]
    print("jagged pair masses (%d) vs O2, every element: %s" % (len(pm), summary(rel)))
    assert rel.max() <= TOL_F64 and np.all(pm[~pos] == 0)
    cart = np.abs(orc.to_cartesian_def(p))
    ev = np.repeat(np.arange(len(off) - 1), np.diff(off))
    mag = np.zeros((len(off) - 1, 4))
    np.add.at(mag, ev, cart)
    mag = mag.sum(axis=1)
    es = np.max(np.abs(sums - r_s), axis=1) / np.where(mag > 0, mag, 1.0)
    print("jagged event sums (%d) vs O2, relative to sum |components|: %s" % (len(sums), summary(es)))
    assert es.max() <= TOL_F64
    events = np.sort(syn.rng(33).choice(1 << 20, 400, replace=False))
    _check(orc, p, off, po, pm, sums, events)


def test_event_pairs_graph_and_autotune(orc):
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    g = syn.rng(34)
    off = syn.jagged_offsets(g, 20_000)
    p = syn.ptetaphim(g, int(off[-1]))
    po, pm, sums = _run(p, off)
    dp, doff = dev(p), torch.as_tensor(off).cuda()
    shape, (te, nt), ms = gvx.autotune_event_pair_masses(dp, doff, _n_pairs(off), reps=2,
                                                         cache=False)
    assert 0 <= shape and te <= nt and ms > 0
    graph = gvx.EventPairMassesGraph(dp, doff, _n_pairs(off))
    graph.pair_m.fill_(-1.0)
    graph.launch()
    graph.launch()
    torch.cuda.synchronize()
    assert gvx.device_status() == 0
    assert np.array_equal(graph.pair_offsets.cpu().numpy(), po)
    assert np.array_equal(graph.pair_m.cpu().numpy(), pm)
    assert np.array_equal(graph.sums.cpu().numpy(), sums)
    graph.close()


def _raw_call(p_dev, off_dev, n_events, n_particles, capacity, pair_m):
    """Direct C-ABI call with an explicit pair capacity (the Python wrapper sizes it exactly)."""
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    from paper_2312_02756_gb300 import _lib
    lib = gvx.load_library()
    po = torch.empty(n_events + 1, dtype=torch.int64, device="cuda")
    sums = torch.empty((n_events, 4), dtype=torch.float64, device="cuda")
    wsb = lib.gvx_event_pair_masses_workspace(n_events)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    lv_p, lv_s = _lib.LV(), _lib.LV()
    lv_p.layout = lv_s.layout = _lib.AOS
    lv_p.c[0], lv_s.c[0] = p_dev.data_ptr(), sums.data_ptr()
    st = lib.gvx_event_pair_masses(ctypes.byref(lv_p), ctypes.c_void_p(off_dev.data_ptr()),
                                   n_events, n_particles, ctypes.c_void_p(po.data_ptr()),
                                   ctypes.c_void_p(pair_m.data_ptr()), capacity,
                                   ctypes.byref(lv_s), ctypes.c_void_p(ws.data_ptr()), wsb,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(st)
    return po


def test_event_pairs_device_detected_errors():
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    g = syn.rng(35)
    off = syn.jagged_offsets(g, 1000)
    p = syn.ptetaphim(g, int(off[-1]))
    total = _n_pairs(off)
    dp, doff = dev(p), torch.as_tensor(off).cuda()
    # capacity: nothing is written past it, and GVX_ERR_CAPACITY is recorded
    buf = torch.full((total + 1000,), -7.0, dtype=torch.float64, device="cuda")
    cap = total - 500
    _raw_call(dp, doff, 1000, len(p), cap, buf)
    assert gvx.device_status() == 10
    assert torch.all(buf[cap:] == -7.0).item()
    # malformed offsets (decreasing, beyond the particle count): GVX_ERR_OFFSETS, no fault
    bad = off.copy()
    bad[500] = bad[502] + 3
    bad[700] = len(p) + 10
    buf = torch.full((total + 1000,), -7.0, dtype=torch.float64, device="cuda")
    _raw_call(dp, torch.as_tensor(bad).cuda(), 1000, len(p), total + 1000, buf)
    assert gvx.device_status() == 6
    # the context is still good
    po, pm, _ = _run(p, off)
    assert po[-1] == total


def test_event_pairs_bounded_wait_times_out():
    """A tile whose predecessor never publishes (tile 0 skipped through the test hook) makes its
    look-back wait run out: GVX_ERR_TIMEOUT is recorded, the kernel finishes, the context stays
    usable."""
    torch = torch_cuda()
    import time
    import paper_2312_02756_gb300 as gvx
    g = syn.rng(36)
    off = syn.jagged_offsets(g, 600)
    p = syn.ptetaphim(g, int(off[-1]))
    lib = gvx.load_library()
    lib.gvx_testing_skip_first_tile(1)
    try:
        t0 = time.time()
        gvx.event_pair_masses(dev(p), torch.as_tensor(off).cuda(), _n_pairs(off))
        code = gvx.device_status()
        dt = time.time() - t0
    finally:
        lib.gvx_testing_skip_first_tile(0)
    assert code == 9
    assert dt < 30
    po, pm, _ = _run(p, off)
    assert po[-1] == _n_pairs(off)


def test_sharded_shares_reassemble_the_packed_output(orc):
    """Two shards of an event array, each run through event_pair_masses_sharded on this GPU (no
    process group: each share is computed as its rank would, with the base of the shard before it
    given by the same exclusive scan), reassemble the single-call pair offsets and pair masses
    exactly."""
    import paper_2312_02756_gb300 as gvx
    from paper_2312_02756_gb300 import sharding
    torch = torch_cuda()
    g = syn.rng(302)
    off = syn.jagged_offsets(g, 3000)
    p = syn.ptetaphim(g, int(off[-1]))
    po_all, pm_all, _ = _run(p, off)
    base = 0
    for r in range(2):
        e_lo, e_hi, p_lo, p_hi = sharding.shard_events(off, r, 2)
        local = off[e_lo:e_hi + 1] - off[e_lo]
        po, pm, sums, b, grand = sharding.event_pair_masses_sharded(
            dev(p[p_lo:p_hi]), torch.as_tensor(local).cuda())
        assert b == 0 and grand == len(pm)  # a single process: its own share only
        po = po.cpu().numpy() + base
        assert np.array_equal(po, po_all[e_lo:e_hi + 1])
        assert np.array_equal(pm.cpu().numpy(), pm_all[po[0]:po[-1]])
        base += len(pm)
