"""gvx_event_pair_masses_noalloc: the jagged-event entry point for callers that cannot allocate
device memory (its scratch is a fixed array inside the library).  Called through the C ABI, two
calls in a row on different inputs, each checked against gvx_event_pair_masses (the entry point
with a caller-provided workspace) at the tolerances the jagged parity tests use.  This file is
collected last on purpose, and also passes when run alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import gvx_synth as syn
from helpers import TOL_F64, torch_cuda

pytestmark = pytest.mark.gpu


def _lv(t):
    from paper_2312_02756_gb300 import _lib
    v = _lib.LV()
    v.layout = _lib.AOS
    v.c[0] = t.data_ptr()
    return v


def _inputs(seed, n_events):
    g = syn.rng(seed)
    off = syn.jagged_offsets(g, n_events)
    p = syn.ptetaphim(g, int(off[-1]))
    c = np.diff(off)
    return p, off, int(np.sum(c * (c - 1) // 2))


def _call(lib, torch, p, off, n_pairs, noalloc):
    from paper_2312_02756_gb300 import _lib
    n_events = len(off) - 1
    dp = torch.as_tensor(p).cuda()
    doff = torch.as_tensor(off).cuda()
    po = torch.full((n_events + 1,), -1, dtype=torch.int64, device="cuda")
    pm = torch.full((max(n_pairs, 1),), -1.0, dtype=torch.float64, device="cuda")
    sums = torch.full((n_events, 4), -1.0, dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    common = (ctypes.byref(_lv(dp)), ctypes.c_void_p(doff.data_ptr()), n_events, len(p),
              ctypes.c_void_p(po.data_ptr()), ctypes.c_void_p(pm.data_ptr()), n_pairs,
              ctypes.byref(_lv(sums)))
    if noalloc:
        st = lib.gvx_event_pair_masses_noalloc(*common, s)
    else:
        wsb = lib.gvx_event_pair_masses_workspace(n_events)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        st = lib.gvx_event_pair_masses(*common, ctypes.c_void_p(ws.data_ptr()), wsb, s)
    _lib.check(st)
    code = ctypes.c_int32(-1)
    _lib.check(lib.gvx_device_status(s, ctypes.byref(code)))
    assert code.value == 0
    return po.cpu().numpy(), pm.cpu().numpy()[:n_pairs], sums.cpu().numpy()


def test_noalloc_matches_workspace_entry_point():
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    lib = gvx.load_library()
    # two calls in a row (different sizes and contents): the shared scratch is reset each time
    for seed, n_events in ((60, 7000), (61, 3001)):
        p, off, n_pairs = _inputs(seed, n_events)
        po, pm, sums = _call(lib, torch, p, off, n_pairs, noalloc=True)
        ro, rm, rs = _call(lib, torch, p, off, n_pairs, noalloc=False)
        # the same kernel and tile shape on the same inputs: the same bits
        assert np.array_equal(po, ro)
        assert np.array_equal(pm, rm)
        assert np.array_equal(sums, rs)
        assert np.all(np.abs(pm - rm) <= TOL_F64 * np.abs(rm))


def test_noalloc_at_its_largest_size():
    """Exactly GVX_NOALLOC_MAX_EVENTS events (all empty): the largest call the fixed scratch
    takes, its last look-back descriptor included."""
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    from paper_2312_02756_gb300 import _lib
    lib = gvx.load_library()
    n_events = 1 << 21
    off = torch.zeros(n_events + 1, dtype=torch.int64, device="cuda")
    po = torch.full((n_events + 1,), -1, dtype=torch.int64, device="cuda")
    sums = torch.full((n_events, 4), -1.0, dtype=torch.float64, device="cuda")
    pm = torch.empty(1, dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.gvx_event_pair_masses_noalloc(
        ctypes.byref(_lv(sums)), ctypes.c_void_p(off.data_ptr()), n_events, 0,
        ctypes.c_void_p(po.data_ptr()), ctypes.c_void_p(pm.data_ptr()), 0,
        ctypes.byref(_lv(sums)), s)
    assert st == 0
    code = ctypes.c_int32(-1)
    _lib.check(lib.gvx_device_status(s, ctypes.byref(code)))
    assert code.value == 0
    assert torch.all(po == 0).item() and torch.all(sums == 0).item()


def test_noalloc_rejects_more_events_than_its_scratch():
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    lib = gvx.load_library()
    n_events = (1 << 21) + 1
    off = torch.zeros(n_events + 1, dtype=torch.int64, device="cuda")
    po = torch.empty(n_events + 1, dtype=torch.int64, device="cuda")
    sums = torch.empty((n_events, 4), dtype=torch.float64, device="cuda")
    pm = torch.empty(1, dtype=torch.float64, device="cuda")
    st = lib.gvx_event_pair_masses_noalloc(
        ctypes.byref(_lv(sums)), ctypes.c_void_p(off.data_ptr()), n_events, 0,
        ctypes.c_void_p(po.data_ptr()), ctypes.c_void_p(pm.data_ptr()), 0,
        ctypes.byref(_lv(sums)), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 2  # GVX_ERR_SIZE, nothing launched
