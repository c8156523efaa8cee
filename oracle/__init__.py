"""CPU oracle for the gvx kernels -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It wraps ``gvx_oracle.c`` (compiled with the host C compiler) through ctypes and
shares no code with the CUDA library in ``paper_2312_02756_gb300``.

Two tiers (see the C file's header for the formulas and the paper passages they follow):

* ``*_def``  -- O1, the plain definitions evaluated in IEEE binary128, rounded once to double.
* ``*_fp64`` -- O2, cancellation-free identities in double; fast, used for whole-input checks
  and as the timed CPU baseline.

All array arguments are numpy float64 arrays of shape (n, 4) (PtEtaPhiM or PxPyPzE rows) or
(n, 3) (velocities); float32 inputs are upcast exactly before the call.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gvx_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_%s.so" % platform.machine())
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build`` (host gcc, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", _LIB_PATH + ".tmp", "-lm", "-lpthread"]
    if platform.machine() in ("x86_64", "AMD64"):
        cmd.append("-lquadmath")
    subprocess.run(cmd, check=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    INT = ctypes.c_int
    sigs = {
        "orc_precision_bits": ([], INT),
        "orc_mass_def": ([P, P, I64, P, INT], None),
        "orc_mass_naive_fp64": ([P, P, I64, P], None),
        "orc_mass_grad_def": ([P, P, P, I64, P, P, INT], None),
        "orc_boost_matrix_def": ([P, P], None),
        "orc_boost_def": ([P, P, I64, I64, P, INT], None),
        "orc_boost_grad_def": ([P, P, I64, P, I64, P, P], None),
        "orc_event_pairs_def": ([P, P, I64, P, P, P], INT),
        "orc_event_pairs_grad_def": ([P, P, I64, P, P, P], INT),
        "orc_lorentz_apply_def": ([P, I64, P, I64, P], None),
        "orc_mass_cart_def": ([P, P, I64, INT, P], None),
        "orc_to_pxpypze_def": ([P, I64, INT, P], None),
        "orc_pair_select_def": ([P, P, I64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                 P, P, P, P], INT),
        "orc_to_cartesian_def": ([P, I64, P], None),
        "orc_lv_mass_def": ([P, I64, P], None),
        "orc_mass_fp64": ([P, P, I64, P, INT], None),
        "orc_boost_fp64": ([P, P, I64, I64, P, INT], None),
        "orc_mass_grad_fp64": ([P, P, P, I64, P, P, INT], None),
        "orc_event_pairs_fp64": ([P, P, I64, P, P, P, INT], INT),
        "orc_event_pairs_grad_fp64": ([P, P, I64, P, P, INT, P, INT], INT),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _rows(x, width):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if a.ndim == 1 and a.size == width:
        a = a.reshape(1, width)
    if a.ndim != 2 or a.shape[1] != width:
        raise ValueError("expected an (n, %d) array, got shape %s" % (width, a.shape))
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def precision_bits() -> int:
    return _load().orc_precision_bits()


def mass_def(a, b, nthreads: int = 1) -> np.ndarray:
    """O1 pair mass: m[i] = mass(cartesian(a[i]) + cartesian(b[i])) in binary128."""
    a, b = _rows(a, 4), _rows(b, 4)
    assert a.shape == b.shape
    m = np.empty(a.shape[0])
    _load().orc_mass_def(_ptr(a), _ptr(b), a.shape[0], _ptr(m), nthreads)
    return m


def mass_naive_fp64(a, b) -> np.ndarray:
    """The definition in plain double (information only: shows the cancellation error)."""
    a, b = _rows(a, 4), _rows(b, 4)
    m = np.empty(a.shape[0])
    _load().orc_mass_naive_fp64(_ptr(a), _ptr(b), a.shape[0], _ptr(m))
    return m


def mass_grad_def(a, b, gm, nthreads: int = 1):
    """O1 gradient of the pair mass: (ga, gb), each (n, 4), scaled by the upstream gm."""
    a, b = _rows(a, 4), _rows(b, 4)
    gm = np.ascontiguousarray(np.asarray(gm, dtype=np.float64).reshape(-1))
    n = a.shape[0]
    assert gm.shape[0] == n
    ga, gb = np.empty((n, 4)), np.empty((n, 4))
    _load().orc_mass_grad_def(_ptr(a), _ptr(b), _ptr(gm), n, _ptr(ga), _ptr(gb), nthreads)
    return ga, gb


def boost_matrix_def(beta) -> np.ndarray:
    b = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(3))
    L = np.empty(16)
    _load().orc_boost_matrix_def(_ptr(b), _ptr(L))
    return L.reshape(4, 4)


def _beta_arg(beta, n):
    b = np.ascontiguousarray(np.asarray(beta, dtype=np.float64))
    if b.ndim == 1:
        if b.size != 3:
            raise ValueError("a shared velocity has 3 components")
        return b, 0
    if b.shape != (n, 3):
        raise ValueError("per-vector velocities must be (n, 3)")
    return b, 1


def boost_def(v, beta, nthreads: int = 1) -> np.ndarray:
    """O1 boost: out[i] = L(beta_i) v[i]; beta is (n, 3) or a single (3,) velocity."""
    v = _rows(v, 4)
    n = v.shape[0]
    b, stride = _beta_arg(beta, n)
    out = np.empty((n, 4))
    _load().orc_boost_def(_ptr(v), _ptr(b), stride, n, _ptr(out), nthreads)
    return out


def boost_grad_def(v, beta, gout):
    """O1 boost gradient: (gv (n,4), gbeta (n,3) or (3,) summed for a shared velocity)."""
    v = _rows(v, 4)
    n = v.shape[0]
    b, stride = _beta_arg(beta, n)
    g = _rows(gout, 4)
    gv = np.empty((n, 4))
    gb = np.empty((n, 3)) if stride else np.empty(3)
    _load().orc_boost_grad_def(_ptr(v), _ptr(b), stride, _ptr(g), n, _ptr(gv), _ptr(gb))
    return gv, gb


def event_pairs_def(p, offsets):
    """O1 jagged pair masses: (pair_offsets int64[n_ev+1], pair_m, sums (n_ev, 4))."""
    p = _rows(p, 4) if len(p) else np.zeros((0, 4))
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    n_ev = off.shape[0] - 1
    if n_ev < 0 or off[-1] != p.shape[0]:
        raise ValueError("offsets must have n_events+1 entries ending at the particle count")
    counts = np.diff(off)
    if np.any(counts < 0):
        raise ValueError("offsets must be non-decreasing")
    n_pairs = int(np.sum(counts * (counts - 1) // 2))
    pair_off = np.empty(n_ev + 1, dtype=np.int64)
    pair_m = np.empty(max(n_pairs, 1))
    sums = np.empty((max(n_ev, 1), 4))
    rc = _load().orc_event_pairs_def(_ptr(p), _ptr(off), n_ev, _ptr(pair_off), _ptr(pair_m),
                                     _ptr(sums))
    if rc != 0:
        raise ValueError("malformed offsets")
    return pair_off, pair_m[:n_pairs], sums[:n_ev]


def event_pairs_grad_def(p, offsets, grad_pair_m, grad_sums=None) -> np.ndarray:
    """O1 adjoint of event_pairs_def: d/dp of sum(grad_pair_m * pair_m) + sum(grad_sums * sums),
    as (n_particles, 4) PtEtaPhiM rows.  grad_sums None means zero."""
    p = _rows(p, 4) if len(p) else np.zeros((0, 4))
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    n_ev = off.shape[0] - 1
    if n_ev < 0 or off[-1] != p.shape[0]:
        raise ValueError("offsets must have n_events+1 entries ending at the particle count")
    counts = np.diff(off)
    if np.any(counts < 0):
        raise ValueError("offsets must be non-decreasing")
    n_pairs = int(np.sum(counts * (counts - 1) // 2))
    gpm = np.ascontiguousarray(np.asarray(grad_pair_m, dtype=np.float64)).reshape(-1)
    if gpm.shape[0] != n_pairs:
        raise ValueError("grad_pair_m must hold one value per pair")
    gpm = gpm if n_pairs else np.zeros(1)
    gs = None if grad_sums is None else _rows(grad_sums, 4)
    if gs is not None and gs.shape[0] != n_ev:
        raise ValueError("grad_sums must hold one row per event")
    out = np.zeros((max(p.shape[0], 1), 4))
    rc = _load().orc_event_pairs_grad_def(_ptr(p), _ptr(off), n_ev, _ptr(gpm),
                                          None if gs is None else _ptr(gs), _ptr(out))
    if rc != 0:
        raise ValueError("malformed offsets")
    return out[:p.shape[0]]


def pair_select_def(p, offsets, pt_min, eta_max, lo, hi, n_bins, target, rel_tol=1e-12):
    """O1 fused selection + pair-mass histogram + best candidate per event (see the C function).
    Returns (counts uint64[n_bins + 2], near_edge uint64[n_bins + 2], best_k int64[n_events],
    best_m float64[n_events])."""
    p = _rows(p, 4) if len(p) else np.zeros((0, 4))
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    n_ev = off.shape[0] - 1
    if n_ev < 0 or off[-1] != p.shape[0]:
        raise ValueError("offsets must have n_events+1 entries ending at the particle count")
    counts = np.zeros(n_bins + 2, dtype=np.uint64)
    near = np.zeros(n_bins + 2, dtype=np.uint64)
    best_k = np.empty(max(n_ev, 1), dtype=np.int64)
    best_m = np.empty(max(n_ev, 1))
    rc = _load().orc_pair_select_def(_ptr(p), _ptr(off), n_ev, float(pt_min), float(eta_max),
                                     float(lo), float(hi), int(n_bins), float(target),
                                     float(rel_tol), _ptr(counts), _ptr(near), _ptr(best_k),
                                     _ptr(best_m))
    if rc != 0:
        raise ValueError("malformed offsets or histogram range")
    return counts, near, best_k[:n_ev], best_m[:n_ev]


def lorentz_apply_def(L, v) -> np.ndarray:
    """O1 general Lorentz transformation: L (4, 4) shared or (n, 4, 4) per vector, applied to
    PxPyPzE rows v (n, 4), in binary128, rounded once."""
    v = _rows(v, 4)
    Lm = np.ascontiguousarray(np.asarray(L, dtype=np.float64))
    if Lm.shape == (4, 4):
        stride = 0
    elif Lm.shape == (v.shape[0], 4, 4):
        stride = 1
    else:
        raise ValueError("L must be (4, 4) or (n, 4, 4)")
    out = np.empty_like(v)
    _load().orc_lorentz_apply_def(_ptr(Lm), stride, _ptr(v), v.shape[0], _ptr(out))
    return out


COORDS = {"pxpypze": 0, "pxpypzm": 1, "ptetaphie": 2, "ptetaphim": 3}


def mass_cart_def(a, b, coords="pxpypze") -> np.ndarray:
    """O1 pair mass for legs in any of the coordinate systems 'pxpypze' (E stored), 'pxpypzm'
    (m stored), 'ptetaphie' (pt, eta, phi, E) or 'ptetaphim'."""
    a, b = _rows(a, 4), _rows(b, 4)
    code = COORDS[coords]
    m = np.empty(a.shape[0])
    _load().orc_mass_cart_def(_ptr(a), _ptr(b), a.shape[0], code, _ptr(m))
    return m


def to_pxpypze_def(p, coords) -> np.ndarray:
    """O1 conversion of rows in any of the coordinate systems of mass_cart_def to PxPyPzE."""
    p = _rows(p, 4)
    out = np.empty_like(p)
    _load().orc_to_pxpypze_def(_ptr(p), p.shape[0], COORDS[coords], _ptr(out))
    return out


def to_cartesian_def(p) -> np.ndarray:
    p = _rows(p, 4)
    out = np.empty_like(p)
    _load().orc_to_cartesian_def(_ptr(p), p.shape[0], _ptr(out))
    return out


def lv_mass_def(v) -> np.ndarray:
    v = _rows(v, 4)
    m = np.empty(v.shape[0])
    _load().orc_lv_mass_def(_ptr(v), v.shape[0], _ptr(m))
    return m


def mass_fp64(a, b, nthreads: int = 1) -> np.ndarray:
    """O2 pair mass from the cancellation-free identity, in double."""
    a, b = _rows(a, 4), _rows(b, 4)
    m = np.empty(a.shape[0])
    _load().orc_mass_fp64(_ptr(a), _ptr(b), a.shape[0], _ptr(m), nthreads)
    return m


def boost_fp64(v, beta, nthreads: int = 1) -> np.ndarray:
    """O2 boost in vector form, in double."""
    v = _rows(v, 4)
    n = v.shape[0]
    b, stride = _beta_arg(beta, n)
    out = np.empty((n, 4))
    _load().orc_boost_fp64(_ptr(v), _ptr(b), stride, n, _ptr(out), nthreads)
    return out


def mass_grad_fp64(a, b, gm, nthreads: int = 1):
    """O2 adjoint of the pair mass: (ga, gb) = gm * dm/d(pt, eta, phi, m) of each leg, from the
    O2 identity differentiated term by term, in double."""
    a, b = _rows(a, 4), _rows(b, 4)
    gm = np.ascontiguousarray(np.asarray(gm, dtype=np.float64)).reshape(-1)
    if gm.shape[0] != a.shape[0] or b.shape[0] != a.shape[0]:
        raise ValueError("a, b and gm must have the same length")
    ga, gb = np.empty_like(a), np.empty_like(b)
    _load().orc_mass_grad_fp64(_ptr(a), _ptr(b), _ptr(gm), a.shape[0], _ptr(ga), _ptr(gb),
                               nthreads)
    return ga, gb


def _offsets(p, offsets):
    p = _rows(p, 4) if len(p) else np.zeros((0, 4))
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    n_ev = off.shape[0] - 1
    if n_ev < 0 or off[-1] != p.shape[0]:
        raise ValueError("offsets must have n_events+1 entries ending at the particle count")
    counts = np.diff(off)
    if np.any(counts < 0):
        raise ValueError("offsets must be non-decreasing")
    return p, off, n_ev, int(np.sum(counts * (counts - 1) // 2))


def event_pairs_fp64(p, offsets, nthreads: int = 1):
    """O2 jagged pair masses, as event_pairs_def: (pair_offsets, pair_m, sums (n_ev, 4))."""
    p, off, n_ev, n_pairs = _offsets(p, offsets)
    pair_off = np.empty(n_ev + 1, dtype=np.int64)
    pair_m = np.empty(max(n_pairs, 1))
    sums = np.empty((max(n_ev, 1), 4))
    rc = _load().orc_event_pairs_fp64(_ptr(p), _ptr(off), n_ev, _ptr(pair_off), _ptr(pair_m),
                                      _ptr(sums), nthreads)
    if rc != 0:
        raise ValueError("malformed offsets")
    return pair_off, pair_m[:n_pairs], sums[:n_ev]


def event_pairs_grad_fp64(p, offsets, grad_pair_m, grad_sums=None, magnitudes=False,
                          nthreads: int = 1) -> np.ndarray:
    """O2 adjoint of the jagged pair masses and event sums, as event_pairs_grad_def; with
    magnitudes, the per-particle sums of the contributions' magnitudes instead."""
    p, off, n_ev, n_pairs = _offsets(p, offsets)
    gpm = np.ascontiguousarray(np.asarray(grad_pair_m, dtype=np.float64)).reshape(-1)
    if gpm.shape[0] != n_pairs:
        raise ValueError("grad_pair_m must hold one value per pair")
    gpm = gpm if n_pairs else np.zeros(1)
    gs = None if grad_sums is None else _rows(grad_sums, 4)
    if gs is not None and gs.shape[0] != n_ev:
        raise ValueError("grad_sums must hold one row per event")
    out = np.zeros((max(p.shape[0], 1), 4))
    rc = _load().orc_event_pairs_grad_fp64(_ptr(p), _ptr(off), n_ev, _ptr(gpm),
                                           None if gs is None else _ptr(gs), int(magnitudes),
                                           _ptr(out), nthreads)
    if rc != 0:
        raise ValueError("malformed offsets")
    return out[:p.shape[0]]
