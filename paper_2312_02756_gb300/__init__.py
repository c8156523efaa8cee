"""gvx: Lorentz-vector kernels for one GB300, after GenVectorX (arXiv 2312.02756).

Thin Python layer over the C ABI in ``include/gvx.h`` (libgvx, hand-written CUDA for sm_103a).
PyTorch provides device memory, streams and autograd plumbing; every step of the computation
runs in libgvx kernels.  There is no CPU fallback: without the built library every call raises.

Vector arrays are torch tensors on the GPU, float64 or float32:
  * AoS: shape (n, 4), contiguous -- rows (pt, eta, phi, m) or (px, py, pz, E);
  * SoA: shape (4, n) with unit stride along n -- one row per component.
The layout is inferred from the shape ((n, 4) wins when n = 4) unless ``layout`` is given.
Velocities are (n, 3) / (3, n) in the same way, or a single (3,) velocity shared by all vectors.
"""
from __future__ import annotations

import ctypes
import json
import os

import torch

from . import _lib
from ._lib import AOS, F32, F64, SOA, GvxError, LV

__all__ = [
    "invariant_mass", "boost", "event_pair_masses", "EventPairMassesGraph",
    "autotune_event_pair_masses", "device_status", "check_device_status", "GvxError",
    "load_library", "library_path", "version", "event_pair_masses_bwd", "event_pair_select",
    "invariant_mass_cart", "lorentz_apply", "to_pxpypze",
]


def load_library():
    """Load (building if needed) libgvx; raises if it cannot be built or loaded."""
    return _lib.load()


def library_path() -> str:
    return _lib.library_path()


def version() -> str:
    return load_library().gvx_version().decode()


# ----------------------------------------------------------------------------------- marshalling

def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError("gvx works on float64 or float32 tensors, got %s" % t.dtype)


def _layout_of(t: torch.Tensor, width: int, layout=None) -> int:
    if layout is not None:
        code = {"soa": SOA, "aos": AOS, SOA: SOA, AOS: AOS}[layout]
    elif t.dim() == 2 and t.shape[1] == width:
        code = AOS
    elif t.dim() == 2 and t.shape[0] == width:
        code = SOA
    else:
        raise ValueError("expected an (n, %d) or (%d, n) tensor, got %s"
                         % (width, width, tuple(t.shape)))
    if code == AOS and not (t.dim() == 2 and t.shape[1] == width and t.is_contiguous()):
        raise ValueError("AoS arrays must be contiguous (n, %d) tensors" % width)
    if code == SOA and not (t.dim() == 2 and t.shape[0] == width
                            and (t.shape[1] <= 1 or t.stride(1) == 1)):
        raise ValueError("SoA arrays must be (%d, n) tensors with unit stride along n" % width)
    return code


def _count(t: torch.Tensor, code: int) -> int:
    return t.shape[0] if code == AOS else t.shape[1]


def _lv(t: torch.Tensor, code: int, width: int) -> LV:
    v = LV()
    v.layout = code
    if code == AOS:
        v.c[0] = t.data_ptr()
    else:
        for k in range(width):
            v.c[k] = t[k].data_ptr()
    return v


def _require_cuda(*ts):
    for t in ts:
        if not t.is_cuda:
            raise ValueError("gvx kernels take CUDA tensors (got a tensor on %s)" % t.device)


# ------------------------------------------------------------------------------- invariant mass

class _InvariantMass(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, b, la, lb):
        lib = load_library()
        n = _count(a, la)
        m = torch.empty(n, dtype=a.dtype, device=a.device)
        st = lib.gvx_invariant_mass(ctypes.byref(_lv(a, la, 4)), ctypes.byref(_lv(b, lb, 4)),
                                    ctypes.c_void_p(m.data_ptr()), n, _dtype_code(a), _stream())
        _lib.check(st, "gvx_invariant_mass")
        ctx.save_for_backward(a, b, m)
        ctx.la, ctx.lb = la, lb
        return m

    @staticmethod
    def backward(ctx, gm):
        lib = load_library()
        a, b, m = ctx.saved_tensors
        gm = gm.contiguous().to(a.dtype)
        ga, gb = torch.empty_like(a), torch.empty_like(b)
        n = _count(a, ctx.la)
        st = lib.gvx_invariant_mass_bwd(
            ctypes.byref(_lv(a, ctx.la, 4)), ctypes.byref(_lv(b, ctx.lb, 4)),
            ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(gm.data_ptr()),
            ctypes.byref(_lv(ga, ctx.la, 4)),
            ctypes.byref(_lv(gb, ctx.lb, 4)), n, _dtype_code(a), _stream())
        _lib.check(st, "gvx_invariant_mass_bwd")
        return ga, gb, None, None


def invariant_mass(a: torch.Tensor, b: torch.Tensor, layout_a=None, layout_b=None):
    """Mass of each pair of PtEtaPhiM vectors (GenVectorX Sec. 4.1, Fig. 1).

    Differentiable with respect to both legs (hand-written adjoint kernel)."""
    _require_cuda(a, b)
    la, lb = _layout_of(a, 4, layout_a), _layout_of(b, 4, layout_b)
    if a.dtype != b.dtype:
        raise TypeError("both legs must have the same dtype")
    if _count(a, la) != _count(b, lb):
        raise ValueError("both legs must hold the same number of vectors")
    return _InvariantMass.apply(a, b, la, lb)


# ---------------------------------------------------------------------------------------- boost

_COORDS = {"ptetaphim": 0, "pxpypze": 1, "pxpypzm": 2, "ptetaphie": 3}


def _coords_code(coords: str) -> int:
    try:
        return _COORDS[coords]
    except KeyError:
        raise ValueError("coords must be one of %s, got %r" % (sorted(_COORDS), coords)) from None


def invariant_mass_cart(a: torch.Tensor, b: torch.Tensor, coords: str = "pxpypze",
                        layout_a=None, layout_b=None) -> torch.Tensor:
    """Pair masses of legs in another coordinate system (gvx_invariant_mass_cart): coords
    'pxpypze' (E stored), 'pxpypzm' (m stored) or 'ptetaphie' (pt, eta, phi, E), FP64 or FP32,
    SoA or AoS like invariant_mass."""
    _require_cuda(a, b)
    la, lb = _layout_of(a, 4, layout_a), _layout_of(b, 4, layout_b)
    if a.dtype != b.dtype:
        raise TypeError("both legs must have the same dtype")
    n = _count(a, la)
    if _count(b, lb) != n:
        raise ValueError("both legs must hold the same number of vectors")
    m = torch.empty(n, dtype=a.dtype, device=a.device)
    st = load_library().gvx_invariant_mass_cart(
        ctypes.byref(_lv(a, la, 4)), ctypes.byref(_lv(b, lb, 4)), ctypes.c_void_p(m.data_ptr()), n,
        _coords_code(coords), _dtype_code(a), _stream())
    _lib.check(st, "gvx_invariant_mass_cart")
    return m


def to_pxpypze(v: torch.Tensor, coords: str, layout=None) -> torch.Tensor:
    """Vectors in coords 'ptetaphim', 'ptetaphie' or 'pxpypzm' converted to PxPyPzE
    (gvx_to_pxpypze), same shape and layout; the input of boost and lorentz_apply."""
    _require_cuda(v)
    lv = _layout_of(v, 4, layout)
    n = _count(v, lv)
    out = torch.empty_like(v)
    st = load_library().gvx_to_pxpypze(ctypes.byref(_lv(v, lv, 4)), ctypes.byref(_lv(out, lv, 4)),
                                       n, _coords_code(coords), _dtype_code(v), _stream())
    _lib.check(st, "gvx_to_pxpypze")
    return out


def lorentz_apply(L: torch.Tensor, v: torch.Tensor, layout=None) -> torch.Tensor:
    """A general Lorentz transformation (gvx_lorentz_apply): L (4, 4) for every vector or
    (n, 4, 4) one per vector, applied to PxPyPzE vectors v ((n, 4) or (4, n))."""
    _require_cuda(L, v)
    lv = _layout_of(v, 4, layout)
    n = _count(v, lv)
    if L.dtype != v.dtype:
        raise TypeError("L and v must have the same dtype")
    L = L.contiguous()
    if tuple(L.shape) == (4, 4):
        stride = 0
    elif tuple(L.shape) == (n, 4, 4):
        stride = 1
    else:
        raise ValueError("L must be (4, 4) or (n, 4, 4)")
    out = torch.empty_like(v)
    st = load_library().gvx_lorentz_apply(ctypes.c_void_p(L.data_ptr()), stride,
                                          ctypes.byref(_lv(v, lv, 4)), ctypes.byref(_lv(out, lv, 4)),
                                          n, _dtype_code(v), _stream())
    _lib.check(st, "gvx_lorentz_apply")
    return out


def _beta_args(beta: torch.Tensor, n: int, layout=None):
    if beta.dim() == 1:
        if beta.numel() != 3 or not beta.is_contiguous():
            raise ValueError("a shared velocity is a contiguous (3,) tensor")
        return AOS, 0
    code = _layout_of(beta, 3, layout)
    if _count(beta, code) != n:
        raise ValueError("per-vector velocities must hold one velocity per vector")
    return code, 1


class _Boost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, beta, lv_code, lb_code, stride):
        lib = load_library()
        n = _count(v, lv_code)
        out = torch.empty_like(v)
        st = lib.gvx_boost(ctypes.byref(_lv(v, lv_code, 4)), ctypes.byref(_lv(beta, lb_code, 3)),
                           stride, ctypes.byref(_lv(out, lv_code, 4)), n, _dtype_code(v),
                           _stream())
        _lib.check(st, "gvx_boost")
        ctx.save_for_backward(v, beta)
        ctx.codes = (lv_code, lb_code, stride)
        return out

    @staticmethod
    def backward(ctx, g):
        lib = load_library()
        v, beta = ctx.saved_tensors
        lv_code, lb_code, stride = ctx.codes
        g = g.to(v.dtype)
        if lv_code == AOS:
            g = g.contiguous()
        elif g.stride(1) != 1:
            g = g.contiguous()
        n = _count(v, lv_code)
        gv, gbeta = torch.empty_like(v), torch.empty_like(beta)
        ws_bytes = lib.gvx_boost_bwd_workspace(n, stride, _dtype_code(v))
        ws = torch.empty(max(ws_bytes, 8), dtype=torch.uint8, device=v.device)
        st = lib.gvx_boost_bwd(
            ctypes.byref(_lv(v, lv_code, 4)), ctypes.byref(_lv(beta, lb_code, 3)), stride,
            ctypes.byref(_lv(g, lv_code, 4)), ctypes.byref(_lv(gv, lv_code, 4)),
            ctypes.byref(_lv(gbeta, lb_code, 3)), n, _dtype_code(v),
            ctypes.c_void_p(ws.data_ptr()), ws_bytes, _stream())
        _lib.check(st, "gvx_boost_bwd")
        return gv, gbeta, None, None, None


def boost(v: torch.Tensor, beta: torch.Tensor, layout=None, beta_layout=None):
    """Boost PxPyPzE vectors by velocities beta (GenVectorX Sec. 4.1, ApplyBoost).

    ``beta`` is one velocity per vector ((n, 3) or (3, n)) or one shared (3,) velocity.
    Differentiable with respect to v and beta (hand-written adjoint kernel)."""
    _require_cuda(v, beta)
    lv_code = _layout_of(v, 4, layout)
    if beta.dtype != v.dtype:
        raise TypeError("v and beta must have the same dtype")
    lb_code, stride = _beta_args(beta, _count(v, lv_code), beta_layout)
    return _Boost.apply(v, beta, lv_code, lb_code, stride)


# --------------------------------------------------------------------------------------- jagged

def _jagged_buffers(particles, offsets, n_pairs, layout, sums_layout):
    _require_cuda(particles, offsets)
    if particles.dtype != torch.float64:
        raise TypeError("the jagged form takes float64 particles")
    if offsets.dtype != torch.int64 or not offsets.is_contiguous():
        raise TypeError("offsets must be a contiguous int64 tensor")
    lp = _layout_of(particles, 4, layout)
    n_events = offsets.numel() - 1
    if n_events < 0:
        raise ValueError("offsets needs n_events + 1 entries")
    dev = particles.device
    pair_off = torch.empty(n_events + 1, dtype=torch.int64, device=dev)
    pair_m = torch.empty(max(int(n_pairs), 1), dtype=torch.float64, device=dev)
    ls = AOS if sums_layout in (None, "aos", AOS) else SOA
    sums = torch.empty((n_events, 4) if ls == AOS else (4, n_events), dtype=torch.float64,
                       device=dev)
    lib = load_library()
    ws_bytes = lib.gvx_event_pair_masses_workspace(n_events)
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=dev)
    return lp, ls, n_events, pair_off, pair_m, sums, ws, ws_bytes


def _jagged_args(particles, lp, offsets, n_events, pair_off, pair_m, n_pairs, sums, ls, ws,
                 ws_bytes):
    return (ctypes.byref(_lv(particles, lp, 4)), ctypes.c_void_p(offsets.data_ptr()), n_events,
            _count(particles, lp), ctypes.c_void_p(pair_off.data_ptr()),
            ctypes.c_void_p(pair_m.data_ptr()), int(n_pairs), ctypes.byref(_lv(sums, ls, 4)),
            ctypes.c_void_p(ws.data_ptr()), ws_bytes)


class _EventPairMasses(torch.autograd.Function):
    @staticmethod
    def forward(ctx, particles, offsets, n_pairs, layout, sums_layout, stream):
        lp, ls, n_events, pair_off, pair_m, sums, ws, ws_bytes = _jagged_buffers(
            particles, offsets, n_pairs, layout, sums_layout)
        lib = load_library()
        st = lib.gvx_event_pair_masses(*_jagged_args(particles, lp, offsets, n_events, pair_off,
                                                     pair_m, n_pairs, sums, ls, ws, ws_bytes),
                                       _stream(stream))
        _lib.check(st, "gvx_event_pair_masses")
        ctx.save_for_backward(particles, offsets, pair_off)
        ctx.codes = (lp, ls, int(n_pairs), stream)
        ctx.mark_non_differentiable(pair_off)
        return pair_off, pair_m[:int(n_pairs)], sums

    @staticmethod
    def backward(ctx, _g_off, g_pm, g_sums):
        particles, offsets, pair_off = ctx.saved_tensors
        lp, ls, n_pairs, stream = ctx.codes
        n_events = offsets.numel() - 1
        gp = torch.empty_like(particles)
        if g_pm is None:
            g_pm = torch.zeros(max(n_pairs, 1), dtype=torch.float64, device=particles.device)
        g_pm = g_pm.to(torch.float64).contiguous()
        gs_arg = None
        if g_sums is not None:
            g_sums = g_sums.to(torch.float64).contiguous()
            gs_arg = ctypes.byref(_lv(g_sums, ls, 4))
        ws, ws_bytes = _bwd_workspace(n_events, particles.device)
        st = load_library().gvx_event_pair_masses_bwd(
            ctypes.byref(_lv(particles, lp, 4)), ctypes.c_void_p(offsets.data_ptr()),
            ctypes.c_void_p(pair_off.data_ptr()), n_events, _count(particles, lp),
            ctypes.c_void_p(g_pm.data_ptr()), n_pairs, gs_arg, ctypes.byref(_lv(gp, lp, 4)),
            ctypes.c_void_p(ws.data_ptr()), ws_bytes, _stream(stream))
        _lib.check(st, "gvx_event_pair_masses_bwd")
        return gp, None, None, None, None, None


def event_pair_masses(particles: torch.Tensor, offsets: torch.Tensor, n_pairs: int, layout=None,
                      sums_layout=None, stream=None):
    """All in-event pair masses and per-event summed 4-vectors of jagged events (FP64).

    ``offsets`` (int64, n_events + 1, on the GPU) delimits the events; ``n_pairs`` is the
    capacity of the pair output (the exact total sum n(n-1)/2 when known).  Returns
    (pair_offsets, pair_m[:n_pairs], event_sums).  Differentiable with respect to the particles
    (hand-written adjoint kernel, gvx_event_pair_masses_bwd).  Device-detected problems
    (malformed offsets, capacity) are reported by ``check_device_status``."""
    return _EventPairMasses.apply(particles, offsets, int(n_pairs), layout, sums_layout, stream)


def _bwd_workspace(n_events, device):
    """Scratch of gvx_event_pair_masses_bwd (the list of tiles for its FP64 pass): a fresh
    allocation per call (the caching allocator's blocks are 512-byte aligned)."""
    ws_bytes = load_library().gvx_event_pair_masses_bwd_workspace(n_events)
    return torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=device), ws_bytes


def event_pair_masses_bwd(particles, offsets, pair_offsets, grad_pair_m, grad_sums=None,
                          layout=None, sums_layout=None, grad_layout=None, stream=None):
    """gvx_event_pair_masses_bwd: d/dparticles of sum(grad_pair_m * pair_m) +
    sum(grad_sums * event_sums); ``grad_sums`` None means zero.  Returns the gradient with the
    particles' shape (or ``grad_layout``)."""
    _require_cuda(particles, offsets, pair_offsets, grad_pair_m)
    lp = _layout_of(particles, 4, layout)
    lg = lp if grad_layout is None else (AOS if grad_layout in ("aos", AOS) else SOA)
    n = _count(particles, lp)
    gp = torch.empty((n, 4) if lg == AOS else (4, n), dtype=torch.float64,
                     device=particles.device)
    gs_arg = None
    if grad_sums is not None:
        ls = _layout_of(grad_sums, 4, sums_layout)
        gs_arg = ctypes.byref(_lv(grad_sums, ls, 4))
    ws, ws_bytes = _bwd_workspace(offsets.numel() - 1, particles.device)
    st = load_library().gvx_event_pair_masses_bwd(
        ctypes.byref(_lv(particles, lp, 4)), ctypes.c_void_p(offsets.data_ptr()),
        ctypes.c_void_p(pair_offsets.data_ptr()), offsets.numel() - 1, n,
        ctypes.c_void_p(grad_pair_m.data_ptr()), grad_pair_m.numel(), gs_arg,
        ctypes.byref(_lv(gp, lg, 4)), ctypes.c_void_p(ws.data_ptr()), ws_bytes, _stream(stream))
    _lib.check(st, "gvx_event_pair_masses_bwd")
    return gp


def event_pair_select(particles, offsets, pt_min, eta_max, lo, hi, n_bins, target, counts=None,
                      layout=None, stream=None):
    """gvx_event_pair_select: the fused selection + pair-mass histogram + best candidate per
    event (FP64, one launch, no pair mass stored).  Returns (counts, best_k, best_m): counts is
    an int64 tensor of n_bins + 2 slots (under, bins, over) that this call adds to (a new zero
    tensor when ``counts`` is None); best_k the packed pair index per event (-1 when none),
    best_m its mass (NaN when none)."""
    _require_cuda(particles, offsets)
    if particles.dtype != torch.float64:
        raise TypeError("the jagged form takes float64 particles")
    if offsets.dtype != torch.int64 or not offsets.is_contiguous():
        raise TypeError("offsets must be a contiguous int64 tensor")
    lp = _layout_of(particles, 4, layout)
    n_events = offsets.numel() - 1
    dev = particles.device
    if counts is None:
        counts = torch.zeros(int(n_bins) + 2, dtype=torch.int64, device=dev)
    elif counts.dtype != torch.int64 or counts.numel() != int(n_bins) + 2 or not counts.is_contiguous():
        raise ValueError("counts must be a contiguous int64 tensor of n_bins + 2 slots")
    best_k = torch.empty(max(n_events, 1), dtype=torch.int64, device=dev)
    best_m = torch.empty(max(n_events, 1), dtype=torch.float64, device=dev)
    st = load_library().gvx_event_pair_select(
        ctypes.byref(_lv(particles, lp, 4)), ctypes.c_void_p(offsets.data_ptr()), n_events,
        _count(particles, lp), float(pt_min), float(eta_max), float(lo), float(hi), int(n_bins),
        float(target), ctypes.c_void_p(counts.data_ptr()), ctypes.c_void_p(best_k.data_ptr()),
        ctypes.c_void_p(best_m.data_ptr()), _stream(stream))
    _lib.check(st, "gvx_event_pair_select")
    return counts, best_k[:n_events], best_m[:n_events]


class EventPairMassesGraph:
    """gvx_event_pair_masses captured once into a CUDA graph for fixed inputs and outputs.

    ``launch()`` replays the whole call (workspace reset + one persistent kernel) as one graph
    launch; results land in ``pair_offsets``, ``pair_m`` and ``sums``."""

    def __init__(self, particles, offsets, n_pairs, layout=None, sums_layout=None):
        lp, ls, n_events, pair_off, pair_m, sums, ws, ws_bytes = _jagged_buffers(
            particles, offsets, n_pairs, layout, sums_layout)
        self._keep = (particles, offsets, ws)
        self.pair_offsets, self.sums = pair_off, sums
        self._pair_m, self.n_pairs = pair_m, int(n_pairs)
        lib = load_library()
        h = ctypes.c_void_p()
        st = lib.gvx_event_pair_masses_graph_create(
            *_jagged_args(particles, lp, offsets, n_events, pair_off, pair_m, n_pairs, sums, ls, ws,
                          ws_bytes), ctypes.byref(h))
        _lib.check(st, "gvx_event_pair_masses_graph_create")
        self._h = h

    @property
    def pair_m(self):
        return self._pair_m[:self.n_pairs]

    def launch(self, stream=None):
        _lib.check(load_library().gvx_graph_launch(self._h, _stream(stream)), "gvx_graph_launch")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().gvx_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _tune_cache_path():
    return os.environ.get("GVX_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gvx_autotune.json"))


def _bucket(n):
    return max(int(n), 1).bit_length() - 1


def autotune_event_pair_masses(particles, offsets, n_pairs, reps: int = 3, layout=None,
                               sums_layout=None, cache: bool = True):
    """Pick the jagged kernel's tile shape for this problem size by timing every shape.

    The choice is recorded in libgvx for the power-of-two bucket of n_events on the current
    device and, with ``cache``, in a JSON file keyed by device name and bucket (reloaded by later
    processes through ``load_tuning``).  Returns (shape, (events_per_tile, threads), mean ms)."""
    lp, ls, n_events, pair_off, pair_m, sums, ws, ws_bytes = _jagged_buffers(
        particles, offsets, n_pairs, layout, sums_layout)
    lib = load_library()
    best, best_ms = ctypes.c_int32(-1), ctypes.c_float(0)
    st = lib.gvx_event_pair_masses_autotune(
        *_jagged_args(particles, lp, offsets, n_events, pair_off, pair_m, n_pairs, sums, ls, ws,
                      ws_bytes), reps, _stream(), ctypes.byref(best), ctypes.byref(best_ms))
    _lib.check(st, "gvx_event_pair_masses_autotune")
    te, nt = ctypes.c_int32(), ctypes.c_int32()
    _lib.check(lib.gvx_event_pair_masses_shape(best.value, ctypes.byref(te), ctypes.byref(nt)))
    if cache:
        path = _tune_cache_path()
        try:
            data = json.load(open(path)) if os.path.exists(path) else {}
        except (OSError, ValueError):
            data = {}
        key = "%s|%d" % (torch.cuda.get_device_name(), _bucket(n_events))
        data[key] = int(best.value)
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
    return int(best.value), (te.value, nt.value), float(best_ms.value)


def load_tuning(path=None):
    """Apply the cached autotuner choices for the current device to libgvx."""
    path = path or _tune_cache_path()
    if not os.path.exists(path):
        return 0
    data = json.load(open(path))
    name = torch.cuda.get_device_name()
    lib = load_library()
    applied = 0
    for key, shape in data.items():
        dev, _, bucket = key.rpartition("|")
        if dev == name:
            _lib.check(lib.gvx_event_pair_masses_set_shape(1 << int(bucket), int(shape)))
            applied += 1
    return applied


# ------------------------------------------------------------------------------------- status

def device_status(stream=None) -> int:
    """Synchronise the stream; return and clear the device status word (0 = GVX_OK)."""
    v = ctypes.c_int32(0)
    _lib.check(load_library().gvx_device_status(_stream(stream), ctypes.byref(v)),
               "gvx_device_status")
    return int(v.value)


def check_device_status(stream=None):
    code = device_status(stream)
    if code != 0:
        raise GvxError(code, "device")
