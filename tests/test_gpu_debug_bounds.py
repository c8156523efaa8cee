"""The GVX_DEBUG_BOUNDS build on the GPU: the jagged forward and adjoint, with every explicit index
check compiled in, record no GVX_ERR_BOUNDS on valid inputs (events of every size, including ones
larger than a staged sub-batch) and return the bits of the normal build."""
import os
import subprocess
import sys

import numpy as np
import pytest

import gvx_synth as syn
from helpers import dev, torch_cuda

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RUN = r"""
import sys, numpy as np, torch
sys.path.insert(0, %(root)r); sys.path.insert(0, %(tests)r)
import paper_2312_02756_gb300 as gvx
from paper_2312_02756_gb300 import build as b
assert b.DEBUG_BOUNDS and "libgvx_dbg_" in b.LIB_PATH
d = np.load(%(inp)r)
p, off, gpm, gsum = d["p"], d["off"], d["gpm"], d["gsum"]
c = np.diff(off); npairs = int(np.sum(c * (c - 1) // 2))
dp = torch.as_tensor(p).cuda(); doff = torch.as_tensor(off).cuda()
po, pm, s = gvx.event_pair_masses(dp, doff, npairs)
st1 = gvx.device_status()
g = gvx.event_pair_masses_bwd(dp, doff, po, torch.as_tensor(gpm).cuda(), torch.as_tensor(gsum).cuda())
st2 = gvx.device_status()
np.savez(%(out)r, po=po.cpu().numpy(), pm=pm.cpu().numpy(), s=s.cpu().numpy(),
         g=g.cpu().numpy(), st=np.array([st1, st2]))
"""


def test_debug_bounds_build_matches(tmp_path):
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    g = syn.rng(71)
    counts = np.concatenate([np.diff(syn.jagged_offsets(g, 3000)), [0, 1, 2, 65, 130, 300]])
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    p = syn.ptetaphim(g, int(off[-1]))
    p[5::97, 1] = 18.5  # outside the float-float domain
    npairs = int(np.sum(counts * (counts - 1) // 2))
    gpm, gsum = syn.upstream(g, npairs), syn.upstream(g, (len(counts), 4))
    np.savez(tmp_path / "in.npz", p=p, off=off, gpm=gpm, gsum=gsum)
    code = _RUN % dict(root=ROOT, tests=os.path.join(ROOT, "tests"), inp=str(tmp_path / "in.npz"),
                       out=str(tmp_path / "out.npz"))
    env = dict(os.environ, GVX_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    dbg = np.load(tmp_path / "out.npz")
    assert list(dbg["st"]) == [0, 0]
    dp, doff = dev(p), torch.as_tensor(off).cuda()
    po, pm, s = gvx.event_pair_masses(dp, doff, npairs)
    grad = gvx.event_pair_masses_bwd(dp, doff, po, torch.as_tensor(gpm).cuda(),
                                     torch.as_tensor(gsum).cuda())
    assert gvx.device_status() == 0
    assert np.array_equal(dbg["po"], po.cpu().numpy())
    assert np.array_equal(dbg["pm"].view(np.uint64), pm.cpu().numpy().view(np.uint64))
    assert np.array_equal(dbg["s"].view(np.uint64), s.cpu().numpy().view(np.uint64))
    assert np.array_equal(dbg["g"].view(np.uint64), grad.cpu().numpy().view(np.uint64))
