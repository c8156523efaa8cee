#!/usr/bin/env python3
"""Benchmark of the gvx hot path on GB300.

One step = the FP64 workload at N = 2^26: invariant mass of 2^26 PtEtaPhiM pairs in SoA, the
same in AoS (32-byte structs), and the boost of 2^26 PxPyPzE vectors, each by its own velocity
(the two kernels GenVectorX benchmarks in Sec. 5.1: pair masses from two particle arrays, and the
boost of a single array).  Inputs are resident in HBM and larger than L2, so no flush is needed
between steps.

Printed on rank 0 as one JSON line: whole-job outputs/s (pair masses + boosted vectors), the
roofline of the dominant kernel (per-launch CUDA events on the launching stream), the CPU
oracle's throughput on the host cores, the end-to-end rate with host buffers (copies inside the
timed region), SM clocks sampled during the timed region, and the other forms of the method
(FP32, jagged events, forward+backward) measured on the same GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gvx|reference]
Under torchrun (N > 1) each rank runs an independent replica of the workload (weak scaling).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "inv-mass & boost vectors/s at N=2^26 FP64/FP32, % roofline; fwd+bwd vs fwd"
UNIT = "vectors/s"
N_FULL = 1 << 26
LOAD_WINDOW_S = 1.5  # seconds of back-to-back untimed steps under the clock sampler
FORMS = ("fp32", "jagged", "fwd_bwd", "coords")
WORKLOAD = ("FP64 invariant mass of 2^26 PtEtaPhiM pairs in SoA and in AoS, plus FP64 boost of "
            "2^26 PxPyPzE vectors by per-vector beta (|beta| <= 0.99)")
BYTES_MASS_F64 = 72    # 2 legs x 4 doubles in + 1 double out, per pair
BYTES_BOOST_F64 = 88   # 4 doubles in + 3 doubles beta + 4 doubles out, per vector
BYTES_MASS_F32 = 36
BYTES_BOOST_F32 = 44


def max_over_ranks(torch, dist, value, device):
    """The largest per-rank value (a step time) over the process group; the value itself when
    there is no group.  Whole-job rates divide all ranks' units by this time."""
    if dist is None:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (ms * 1e-3)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# --------------------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self, settle=0.3):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(settle)

    def stop(self, settle=0.25):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(settle)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------- workload

def make_inputs(n, seed_stream=1):
    import gvx_synth as syn
    g = syn.rng(seed_stream)
    a, b = syn.ptetaphim(g, n), syn.ptetaphim(g, n)
    v, beta = syn.pxpypze(g, n), syn.velocities(g, n, 0.99)
    return a, b, v, beta


def cpu_oracle_rate(a, b, v, beta, reps=1):
    """O2 (FP64 oracle) over the given rows on all host cores: outputs/s for the step's mix
    (two mass launches + one boost launch)."""
    import oracle
    cores = _cores()
    oracle.build()
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.mass_fp64(a, b, nthreads=cores)
    t_mass = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.boost_fp64(v, beta, nthreads=cores)
    t_boost = (time.perf_counter() - t0) / reps
    n = a.shape[0]
    return 3 * n / (2 * t_mass + t_boost), cores, t_mass, t_boost


def cpu_oracle_rate_1t(a, b, v, beta, sample=1 << 22):
    """O2 on one host thread (the paper measures its speed-ups against a single-threaded CPU run,
    Sec. 5.2) over the first `sample` rows: outputs/s for the step's mix."""
    import oracle
    oracle.build()
    a, b, v, beta = a[:sample], b[:sample], v[:sample], beta[:sample]
    t0 = time.perf_counter()
    oracle.mass_fp64(a, b, nthreads=1)
    t_mass = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.boost_fp64(v, beta, nthreads=1)
    t_boost = time.perf_counter() - t0
    return 3 * a.shape[0] / (2 * t_mass + t_boost), t_mass, t_boost


class Step:
    """The timed step: mass SoA, mass AoS, boost, called through the C ABI with preallocated
    outputs, one CUDA-event pair around every launch."""

    def __init__(self, torch, gvx, a, b, v, beta):
        from paper_2312_02756_gb300 import _lib
        self.torch, self.lib, self._lib = torch, gvx.load_library(), _lib
        n = a.shape[0]
        self.n = n
        dev = "cuda"
        self.a_soa = torch.as_tensor(a.T.copy()).to(dev)
        self.b_soa = torch.as_tensor(b.T.copy()).to(dev)
        self.a_aos = torch.as_tensor(a).to(dev)
        self.b_aos = torch.as_tensor(b).to(dev)
        self.v = torch.as_tensor(v.T.copy()).to(dev)
        self.beta = torch.as_tensor(beta.T.copy()).to(dev)
        self.m1 = torch.empty(n, dtype=torch.float64, device=dev)
        self.m2 = torch.empty(n, dtype=torch.float64, device=dev)
        self.out = torch.empty((4, n), dtype=torch.float64, device=dev)
        L = _lib.LV
        mk = lambda t, layout, k: self._lv(t, layout, k)
        self.lv = [mk(self.a_soa, 0, 4), mk(self.b_soa, 0, 4), mk(self.a_aos, 1, 4),
                   mk(self.b_aos, 1, 4), mk(self.v, 0, 4), mk(self.beta, 0, 3),
                   mk(self.out, 0, 4)]
        self.names = ["mass_f64_soa", "mass_f64_aos", "boost_f64_soa"]
        self.events = None

    @staticmethod
    def _lv(t, layout, k):
        from paper_2312_02756_gb300 import _lib
        x = _lib.LV()
        x.layout = layout
        if layout == 1:
            x.c[0] = t.data_ptr()
        else:
            for i in range(k):
                x.c[i] = t[i].data_ptr()
        return x

    def __call__(self, stream, ev=None):
        lib, r, P = self.lib, ctypes.byref, ctypes.c_void_p
        s = P(stream.cuda_stream)
        lv = self.lv
        calls = [
            lambda: lib.gvx_invariant_mass(r(lv[0]), r(lv[1]), P(self.m1.data_ptr()), self.n, 0, s),
            lambda: lib.gvx_invariant_mass(r(lv[2]), r(lv[3]), P(self.m2.data_ptr()), self.n, 0, s),
            lambda: lib.gvx_boost(r(lv[4]), r(lv[5]), 1, r(lv[6]), self.n, 0, s),
        ]
        for k, call in enumerate(calls):
            if ev is not None:
                ev[k][0].record(stream)
            st = call()
            if ev is not None:
                ev[k][1].record(stream)
            self._lib.check(st, self.names[k])


def time_loop(torch, fn, stream, steps, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


# ---------------------------------------------------------------------------------------- forms

def forms(torch, gvx, steps, warmup, fp64_pairs_per_s, fp64_mass_ms, which=FORMS):
    """FP32, jagged and forward+backward forms, each timed alone on the same GPU."""
    import gvx_synth as syn
    from paper_2312_02756_gb300 import _lib
    lib = gvx.load_library()
    stream = torch.cuda.current_stream()
    s = ctypes.c_void_p(stream.cuda_stream)
    r, P = ctypes.byref, ctypes.c_void_p
    res = {}
    if "fp32" in which:
        # FP32: half the particles light and hard; boost with |beta| <= 0.999999
        g = syn.rng(2)
        a = torch.as_tensor(syn.to_f32(syn.ptetaphim_light_mix(g, N_FULL)).T.copy()).cuda()
        b = torch.as_tensor(syn.to_f32(syn.ptetaphim_light_mix(g, N_FULL)).T.copy()).cuda()
        m = torch.empty(N_FULL, dtype=torch.float32, device="cuda")
        la, lb = Step._lv(a, 0, 4), Step._lv(b, 0, 4)
        t_m = time_loop(torch, lambda: _lib.check(lib.gvx_invariant_mass(
            r(la), r(lb), P(m.data_ptr()), N_FULL, 1, s)), stream, steps, warmup)
        del a, b, m
        v = torch.as_tensor(syn.to_f32(syn.pxpypze(g, N_FULL)).T.copy()).cuda()
        be = torch.as_tensor(syn.to_f32(syn.velocities(g, N_FULL, 0.999999)).T.copy()).cuda()
        o = torch.empty_like(v)
        lv_, lbe, lo = Step._lv(v, 0, 4), Step._lv(be, 0, 3), Step._lv(o, 0, 4)
        t_b = time_loop(torch, lambda: _lib.check(lib.gvx_boost(
            r(lv_), r(lbe), 1, r(lo), N_FULL, 1, s)), stream, steps, warmup)
        del v, be, o
        torch.cuda.empty_cache()
        res["fp32"] = {
            "workload": "FP32 mass of 2^26 pairs (half light, pt up to 5 TeV) + FP32 boost of 2^26 "
                        "vectors, |beta| <= 0.999999, SoA",
            "mass_ms": t_m, "boost_ms": t_b,
            "mass_pairs_per_s": N_FULL / (t_m * 1e-3), "boost_vectors_per_s": N_FULL / (t_b * 1e-3),
            "mass_GBps": BYTES_MASS_F32 * N_FULL / (t_m * 1e-3) / 1e9,
            "boost_GBps": BYTES_BOOST_F32 * N_FULL / (t_b * 1e-3) / 1e9,
            "mass_speedup_vs_fp64": fp64_mass_ms / t_m,
        }
    if "jagged" in which:
        # jagged: 2^20 events, Poisson(8) multiplicities, one persistent launch in a CUDA graph
        g = syn.rng(3)
        off = syn.jagged_offsets(g, 1 << 20)
        p = torch.as_tensor(syn.ptetaphim(g, int(off[-1]))).cuda()
        c = np.diff(off)
        n_pairs = int(np.sum(c * (c - 1) // 2))
        doff = torch.as_tensor(off).cuda()
        shape, (te, nt), _ = gvx.autotune_event_pair_masses(p, doff, n_pairs, reps=3, cache=False)
        graph = gvx.EventPairMassesGraph(p, doff, n_pairs)
        t_j = time_loop(torch, lambda: graph.launch(stream), stream, steps, warmup)
        status = gvx.device_status()
        # the adjoint (gvx_event_pair_masses_bwd) on the same events, upstream gradients U[-1, 1]
        n_ev = len(off) - 1
        gpm = torch.as_tensor(syn.upstream(g, n_pairs)).cuda()
        gsum = torch.as_tensor(syn.upstream(g, (n_ev, 4))).cuda()
        gp = torch.empty_like(p)
        lp, lgs, lgp = Step._lv(p, 1, 4), Step._lv(gsum, 1, 4), Step._lv(gp, 1, 4)
        ws_b = lib.gvx_event_pair_masses_bwd_workspace(n_ev)
        ws = torch.empty(ws_b, dtype=torch.uint8, device="cuda")
        jbwd = lambda: _lib.check(lib.gvx_event_pair_masses_bwd(
            r(lp), P(doff.data_ptr()), P(graph.pair_offsets.data_ptr()), n_ev, int(off[-1]),
            P(gpm.data_ptr()), n_pairs, r(lgs), r(lgp), P(ws.data_ptr()), ws_b, s))
        t_jb = time_loop(torch, jbwd, stream, steps, warmup)
        status_b = gvx.device_status()
        # the fused analysis step on the same events: cuts pt >= 20, |eta| <= 2.5, 200 bins of
        # the selected pair masses over [0, 400), best candidate for 91.1876
        hist = torch.zeros(202, dtype=torch.int64, device="cuda")
        bk = torch.empty(n_ev, dtype=torch.int64, device="cuda")
        bm = torch.empty(n_ev, dtype=torch.float64, device="cuda")
        jsel = lambda: _lib.check(lib.gvx_event_pair_select(
            r(lp), P(doff.data_ptr()), n_ev, int(off[-1]), 20.0, 2.5, 0.0, 400.0, 200, 91.1876,
            P(hist.data_ptr()), P(bk.data_ptr()), P(bm.data_ptr()), s))
        t_js = time_loop(torch, jsel, stream, steps, warmup)
        status_s = gvx.device_status()
        sel_pairs = int(hist.sum().item()) // (steps + warmup)
        del hist, bk, bm
        graph.close()
        del p, doff, graph, gpm, gsum, gp
        torch.cuda.empty_cache()
        jag_bytes = 32 * int(off[-1]) + 8 * n_pairs + 8 * (len(off)) * 2 + 32 * (len(off) - 1)
        # adjoint: particles, pair gradients, event-sum gradients and offsets in, gradients out
        jag_bwd_bytes = 64 * int(off[-1]) + 8 * n_pairs + 16 * (len(off)) + 32 * n_ev
        res["jagged"] = {
            "workload": "2^20 events, multiplicity Poisson(8) clamped to [0,64]; all in-event pair "
                        "masses + per-event sums; one persistent kernel replayed as a CUDA graph",
            "ms": t_j, "pairs": n_pairs, "particles": int(off[-1]),
            "pairs_per_s": n_pairs / (t_j * 1e-3), "events_per_s": (len(off) - 1) / (t_j * 1e-3),
            "GBps": jag_bytes / (t_j * 1e-3) / 1e9, "shape": {"events_per_tile": te, "threads": nt},
            "pairs_per_s_vs_fp64_mass": (n_pairs / (t_j * 1e-3)) / fp64_pairs_per_s,
            "device_status": status,
            "bwd": {"ms": t_jb, "pairs_per_s": n_pairs / (t_jb * 1e-3),
                    "GBps": jag_bwd_bytes / (t_jb * 1e-3) / 1e9, "bwd_over_fwd": t_jb / t_j,
                    "device_status": status_b,
                    "how": "gvx_event_pair_masses_bwd, pair-mass and event-sum gradients U[-1, 1]"},
        "select": {"ms": t_js, "events_per_s": n_ev / (t_js * 1e-3),
                   "pairs_per_s": n_pairs / (t_js * 1e-3), "selected_pairs": sel_pairs,
                   "device_status": status_s,
                   "how": "gvx_event_pair_select: pt >= 20, |eta| <= 2.5, 200 bins over "
                          "[0, 400), best candidate for 91.1876; no pair mass stored"},
        }
    if "fwd_bwd" in which:
        # forward + backward, FP64 and FP32, N = 2^24
        n = 1 << 24
        out = {}
        for dt, code, tdt in (("f64", 0, torch.float64), ("f32", 1, torch.float32)):
            g = syn.rng(4)
            a = torch.as_tensor(syn.ptetaphim(g, n).T.copy(), dtype=tdt).cuda()
            b = torch.as_tensor(syn.ptetaphim(g, n).T.copy(), dtype=tdt).cuda()
            gm = torch.as_tensor(syn.upstream(g, n), dtype=tdt).cuda()
            m = torch.empty(n, dtype=tdt, device="cuda")
            ga, gb = torch.empty_like(a), torch.empty_like(b)
            la, lb, lga, lgb = (Step._lv(t, 0, 4) for t in (a, b, ga, gb))
            fwd = lambda: _lib.check(lib.gvx_invariant_mass(r(la), r(lb), P(m.data_ptr()), n, code, s))
            bwd = lambda: _lib.check(lib.gvx_invariant_mass_bwd(
                r(la), r(lb), P(m.data_ptr()), P(gm.data_ptr()), r(lga), r(lgb), n, code, s))
            t_f = time_loop(torch, fwd, stream, steps, warmup)
            t_fb = time_loop(torch, lambda: (fwd(), bwd()), stream, steps, warmup)
            del a, b, gm, m, ga, gb
            v = torch.as_tensor(syn.pxpypze(g, n).T.copy(), dtype=tdt).cuda()
            be = torch.as_tensor(syn.velocities(g, n, 0.99).T.copy(), dtype=tdt).cuda()
            go = torch.as_tensor(syn.upstream(g, (n, 4)).T.copy(), dtype=tdt).cuda()
            o, gv, gbe = torch.empty_like(v), torch.empty_like(v), torch.empty_like(be)
            lv_, lbe, lgo, lo, lgv, lgbe = (Step._lv(t, 0, k) for t, k in
                                            ((v, 4), (be, 3), (go, 4), (o, 4), (gv, 4), (gbe, 3)))
            bf = lambda: _lib.check(lib.gvx_boost(r(lv_), r(lbe), 1, r(lo), n, code, s))
            bb = lambda: _lib.check(lib.gvx_boost_bwd(r(lv_), r(lbe), 1, r(lgo), r(lgv), r(lgbe), n,
                                                      code, None, 0, s))
            t_bf = time_loop(torch, bf, stream, steps, warmup)
            t_bfb = time_loop(torch, lambda: (bf(), bb()), stream, steps, warmup)
            del v, be, go, o, gv, gbe
            torch.cuda.empty_cache()
            out[dt] = {"mass_fwd_ms": t_f, "mass_fwd_bwd_ms": t_fb, "mass_ratio": t_fb / t_f,
                       "mass_fwd_bwd_GBps": 208 * n / (t_fb * 1e-3) / 1e9 * (1 if code == 0 else 0.5),
                       "boost_fwd_ms": t_bf, "boost_fwd_bwd_ms": t_bfb, "boost_ratio": t_bfb / t_bf}
        out["workload"] = "N = 2^24 pairs / vectors, SoA, upstream gradients uniform in [-1, 1]"
        res["fwd_bwd"] = out
    if "coords" in which:
        # other coordinate systems: FP64 pair masses of 2^26 Cartesian pairs (E, then m stored) and a
        # general Lorentz transformation (one shared 4x4 matrix) of 2^26 PxPyPzE vectors
        g = syn.rng(5)
        a = torch.as_tensor(syn.pxpypze(g, N_FULL).T.copy()).cuda()
        b = torch.as_tensor(syn.pxpypze(g, N_FULL).T.copy()).cuda()
        m = torch.empty(N_FULL, dtype=torch.float64, device="cuda")
        la, lb = Step._lv(a, 0, 4), Step._lv(b, 0, 4)
        t_c = time_loop(torch, lambda: _lib.check(lib.gvx_invariant_mass_cart(
            r(la), r(lb), P(m.data_ptr()), N_FULL, 1, 0, s)), stream, steps, warmup)
        # the same legs with the fourth component read as a mass in [0, 10] (PxPyPzM)
        gm = syn.rng(6)
        a[3] = torch.as_tensor(gm.uniform(0.0, 10.0, N_FULL)).cuda()
        b[3] = torch.as_tensor(gm.uniform(0.0, 10.0, N_FULL)).cuda()
        t_cm = time_loop(torch, lambda: _lib.check(lib.gvx_invariant_mass_cart(
            r(la), r(lb), P(m.data_ptr()), N_FULL, 2, 0, s)), stream, steps, warmup)
        # PtEtaPhiE legs (on-shell energies of the PtEtaPhiM draws): pair masses, and the
        # conversion of one array to PxPyPzE
        gp = syn.rng(7)
        pe_a, pe_b = syn.ptetaphim(gp, N_FULL), syn.ptetaphim(gp, N_FULL)
        for x in (pe_a, pe_b):
            x[:, 3] = np.sqrt((x[:, 0] * np.cosh(x[:, 1])) ** 2 + x[:, 3] ** 2)
        a.copy_(torch.as_tensor(pe_a.T.copy()))
        b.copy_(torch.as_tensor(pe_b.T.copy()))
        del pe_a, pe_b
        t_ce = time_loop(torch, lambda: _lib.check(lib.gvx_invariant_mass_cart(
            r(la), r(lb), P(m.data_ptr()), N_FULL, 3, 0, s)), stream, steps, warmup)
        # FP32 copies of the PtEtaPhiE legs: the same pair masses in single precision
        a32, b32 = a.float(), b.float()
        m32 = torch.empty(N_FULL, dtype=torch.float32, device="cuda")
        la32, lb32 = Step._lv(a32, 0, 4), Step._lv(b32, 0, 4)
        t_ce32 = time_loop(torch, lambda: _lib.check(lib.gvx_invariant_mass_cart(
            r(la32), r(lb32), P(m32.data_ptr()), N_FULL, 3, 1, s)), stream, steps, warmup)
        del a32, b32, m32
        o = torch.empty_like(a)
        lo = Step._lv(o, 0, 4)
        t_cv = time_loop(torch, lambda: _lib.check(lib.gvx_to_pxpypze(
            r(la), r(lo), N_FULL, 3, 0, s)), stream, steps, warmup)
        L = torch.as_tensor(np.array([[1.2, 0.1, 0.0, 0.5], [0.1, 1.1, 0.2, 0.0],
                                      [0.0, 0.2, 1.3, 0.4], [0.5, 0.0, 0.4, 1.5]])).cuda()
        t_l = time_loop(torch, lambda: _lib.check(lib.gvx_lorentz_apply(  # on the converted vectors
            P(L.data_ptr()), 0, r(lo), r(la), N_FULL, 0, s)), stream, steps, warmup)
        del a, b, m, o, L
        torch.cuda.empty_cache()
        res["coords"] = {
            "workload": "FP64, 2^26 elements, SoA: pair masses of PxPyPzE legs, of PxPyPzM "
                        "legs (masses in [0, 10]) and of PtEtaPhiE legs (on-shell; also in FP32); the "
                        "PtEtaPhiE -> PxPyPzE conversion; a shared 4x4 Lorentz transformation "
                        "of PxPyPzE vectors",
            "mass_pxpypze_ms": t_c, "mass_pxpypze_pairs_per_s": N_FULL / (t_c * 1e-3),
            "mass_pxpypze_GBps": 72 * N_FULL / (t_c * 1e-3) / 1e9,
            "mass_pxpypzm_ms": t_cm, "mass_pxpypzm_pairs_per_s": N_FULL / (t_cm * 1e-3),
            "mass_pxpypzm_GBps": 72 * N_FULL / (t_cm * 1e-3) / 1e9,
            "mass_ptetaphie_ms": t_ce, "mass_ptetaphie_pairs_per_s": N_FULL / (t_ce * 1e-3),
            "mass_ptetaphie_GBps": 72 * N_FULL / (t_ce * 1e-3) / 1e9,
            "mass_ptetaphie_f32_ms": t_ce32,
            "mass_ptetaphie_f32_GBps": 36 * N_FULL / (t_ce32 * 1e-3) / 1e9,
            "to_pxpypze_ms": t_cv, "to_pxpypze_vectors_per_s": N_FULL / (t_cv * 1e-3),
            "to_pxpypze_GBps": 64 * N_FULL / (t_cv * 1e-3) / 1e9,
            "lorentz_apply_ms": t_l, "lorentz_apply_vectors_per_s": N_FULL / (t_l * 1e-3),
            "lorentz_apply_GBps": 64 * N_FULL / (t_l * 1e-3) / 1e9,
        }
    return res


# ------------------------------------------------------------------------------------------ e2e

def e2e(torch, gvx, a, b, v, beta, steps=3, warmup=1, dist=None, world=1):
    """The step through the C ABI with HOST buffers: the same three calls, given pinned host
    pointers for every input and output, so each kernel streams its inputs over the host link
    and writes its outputs back over it (both directions at once) inside the timed region.
    (Explicit cudaMemcpyAsync copies in and out on one stream measured ~2x slower: they do not
    overlap the two directions.)"""
    stream = torch.cuda.current_stream()
    pin = lambda x: torch.as_tensor(x).pin_memory()
    n = a.shape[0]
    host = {
        "a_soa": pin(a.T.copy()), "b_soa": pin(b.T.copy()), "a_aos": pin(a), "b_aos": pin(b),
        "v": pin(v.T.copy()), "beta": pin(beta.T.copy()),
        "m1": torch.empty(n, dtype=torch.float64).pin_memory(),
        "m2": torch.empty(n, dtype=torch.float64).pin_memory(),
        "out": torch.empty((4, n), dtype=torch.float64).pin_memory(),
    }
    h2d = sum(host[k].numel() * 8 for k in ("a_soa", "b_soa", "a_aos", "b_aos", "v", "beta"))
    d2h = sum(host[k].numel() * 8 for k in ("m1", "m2", "out"))
    step = Step.__new__(Step)  # the timed step, pointed at the host buffers
    from paper_2312_02756_gb300 import _lib
    step.torch, step.lib, step._lib, step.n = torch, gvx.load_library(), _lib, n
    for k, t in host.items():
        setattr(step, k, t)
    step.lv = [Step._lv(host["a_soa"], 0, 4), Step._lv(host["b_soa"], 0, 4),
               Step._lv(host["a_aos"], 1, 4), Step._lv(host["b_aos"], 1, 4),
               Step._lv(host["v"], 0, 4), Step._lv(host["beta"], 0, 3), Step._lv(host["out"], 0, 4)]
    step.names = ["mass_f64_soa", "mass_f64_aos", "boost_f64_soa"]
    if dist:
        dist.barrier()
    ms = max_over_ranks(torch, dist, time_loop(torch, lambda: step(stream), stream, steps, warmup),
                        "cuda")
    res = {"value": job_rate(3 * n, world, ms), "unit": UNIT, "ms_per_step": ms,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "how": "the C-ABI calls given pinned host pointers: inputs read and outputs written by "
                  "the kernels across the host link inside the timed region"}
    return res


# ----------------------------------------------------------------------------------------- arms

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    sample = 1 << 24
    a, b, v, beta = make_inputs(sample)
    for _ in range(args.warmup):
        cpu_oracle_rate(a[:1 << 16], b[:1 << 16], v[:1 << 16], beta[:1 << 16])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rate, cores, _, _ = cpu_oracle_rate(a, b, v, beta)
    dt = (time.perf_counter() - t0) / args.steps
    value = 3 * sample / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_FULL},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "each step: 2^24 pairs twice (the SoA and AoS launches) and "
                                   "2^24 boosts through the FP64 oracle tier O2 on all host "
                                   "cores; the GPU workload is 2^26 of each"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_gvx(args):
    import torch
    import paper_2312_02756_gb300 as gvx

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    gvx.load_library()
    a, b, v, beta = make_inputs(N_FULL)
    step = Step(torch, gvx, a, b, v, beta)
    stream = torch.cuda.current_stream()
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    for _ in range(args.warmup):
        step(stream)
    w1.record(stream)
    torch.cuda.synchronize()
    warm_ms = w0.elapsed_time(w1) / max(args.warmup, 1)
    ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(3)]
          for _ in range(args.steps)]
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    uuid = getattr(props, "uuid", None)
    clocks = ClockSampler(("GPU-%s" % uuid) if uuid else torch.cuda.current_device())
    # the clocks are sampled (every 200 ms) over a load window of back-to-back untimed steps,
    # --clock-window seconds long, that runs straight into the timed region: a timed region of a few
    # steps alone is shorter than one sample interval
    n_load = int(math.ceil(args.clock_window * 1e3 / max(warm_ms, 1e-3)))
    clocks.start(settle=0.0)
    for _ in range(n_load):
        step(stream)
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(stream, ev[k])
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop(settle=0.0)
    if isinstance(clk, dict):
        clk["window"] = ("nvidia-smi every 200 ms over %d untimed steps (%.2f s) running straight "
                         "into the %d timed steps" % (n_load, n_load * warm_ms / 1e3, args.steps))
    ms = max_over_ranks(torch, dist, e0.elapsed_time(e1) / args.steps, "cuda")
    per_kernel = [statistics.mean(ev[k][j][0].elapsed_time(ev[k][j][1]) for k in range(args.steps))
                  for j in range(3)]
    units = 3 * N_FULL
    value = job_rate(units, world, ms)
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs")
    kern = {}
    for name, t, nb in zip(step.names, per_kernel, (BYTES_MASS_F64, BYTES_MASS_F64,
                                                    BYTES_BOOST_F64)):
        kern[name] = {"ms": t, "GBps": nb * N_FULL / (t * 1e-3) / 1e9,
                      "outputs_per_s": N_FULL / (t * 1e-3)}
    dom = max(kern, key=lambda k: kern[k]["ms"])
    achieved = kern[dom]["GBps"]
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": (achieved / hbm) if hbm else None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"
                if hbm else "fallback 6800 GB/s",
                "traffic": None,
                "algorithmic_bytes_per_unit": BYTES_MASS_F64 if "mass" in dom else BYTES_BOOST_F64}
    if not hbm:
        roofline["peak"] = 6800.0
        roofline["frac"] = achieved / 6800.0
    traffic = _profile_traffic(dom, N_FULL)
    if traffic is not None:
        roofline["traffic"] = traffic
    issue = issue_roofline(dom, kern[dom]["ms"], clk.get("sm_mhz") if isinstance(clk, dict) else None,
                           props.multi_processor_count, N_FULL)
    if issue is not None:
        roofline["issue"] = issue
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_FULL, "layouts": ["soa", "aos", "soa"],
                   "l2": "no flush: every launch reads >= 3.7 GB, far above the 129 MB L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "kernels": kern, "roofline": roofline, "gpu_launches": 3 * args.steps, "clocks": clk,
    }
    if not args.no_e2e:  # every rank streams its own replica over its host link
        res = e2e(torch, gvx, a, b, v, beta, dist=dist, world=world)
        if rank == 0:
            line["e2e"] = res
    if rank == 0 and not args.no_cpu:
        rate, cores, tm, tb = cpu_oracle_rate(a, b, v, beta)
        r1, tm1, tb1 = cpu_oracle_rate_1t(a, b, v, beta)
        line["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "the whole 2^26 workload (mass twice, boost once) through the FP64 oracle "
                      "tier O2 on all host cores: mass %.0f ms, boost %.0f ms" % (tm * 1e3, tb * 1e3),
            "single_thread": {"value": r1, "unit": UNIT, "cores": 1,
                              "sample": "2^22 pairs and 2^22 boosts through O2 on one thread: "
                                        "mass %.0f ms, boost %.0f ms" % (tm1 * 1e3, tb1 * 1e3)}}
    del step
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_forms:
        which = tuple(f for f in args.forms.split(",") if f)
        unknown = set(which) - set(FORMS)
        if unknown:
            raise SystemExit("unknown --forms entries: %s" % ",".join(sorted(unknown)))
        line["forms"] = forms(torch, gvx, max(3, args.steps // 2), 2,
                              N_FULL / (per_kernel[0] * 1e-3), per_kernel[0], which)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# The sources each timed kernel's device code is built from (the committed counters are valid
# while these match; gvx_internal.h, which only declares the host-side launch functions, is left
# out).
_MASS_SRC = ("mass.cu", "mass_lc.cuh", "mass_lc_grad.cuh", "ff2.cuh", "ff_tables.cuh", "ff.cuh",
             "pair_math.cuh", "common.cuh", "../gen_tables.py")
KERNEL_SOURCES = {
    "mass_f64_soa": _MASS_SRC,
    "mass_f64_aos": _MASS_SRC,
    "boost_f64_soa": ("boost.cu", "boost_ff.cuh", "mass_lc.cuh", "ff2.cuh", "ff_tables.cuh", "ff.cuh",
                      "common.cuh", "../gen_tables.py"),
}


def sources_hash(kernel, read=None):
    """Short hash of the sources `kernel` is built from; `read(relpath) -> bytes` defaults to the
    working tree (paths relative to the package's csrc folder)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2312_02756_gb300", "csrc")
    read = read or (lambda rel: open(os.path.join(csrc, rel), "rb").read())
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kernel]:
        h.update(rel.encode())
        h.update(read(rel))
    return h.hexdigest()[:16]


def _profile_entry(kernel):
    """The committed ncu figures for `kernel` (profiles/traffic.json), only while the kernel's
    sources are the ones the counters were taken from."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return None
    entry = data.get(kernel)
    if not isinstance(entry, dict) or kernel not in KERNEL_SOURCES:
        return None
    if entry.get("sources_hash") != sources_hash(kernel):
        return None
    return entry


PROFILE_N = 1 << 26  # the element count the committed per-launch figures are given for


def _profile_traffic(kernel, n):
    """DRAM bytes per launch of `kernel` at n elements (see _profile_entry), scaled from the
    committed figure by the element count (every element is read once)."""
    entry = _profile_entry(kernel)
    b = entry.get("bytes_per_launch") if entry else None
    return None if b is None else b * n / PROFILE_N


def issue_roofline(kernel, ms, sm_mhz, n_sms, n):
    """The instruction-issue view of a kernel bound by issue rather than by DRAM: warp
    instructions per launch (ncu, scaled like the traffic) over the launch time, against the
    issue peak of the GPU -- four warp instructions per SM per clock at the sampled SM clock."""
    entry = _profile_entry(kernel)
    inst = entry.get("warp_inst_per_launch") if entry else None
    if inst is None or not sm_mhz or not n_sms:
        return None
    inst = inst * n / PROFILE_N
    achieved = inst / (ms * 1e-3)
    peak = 4.0 * n_sms * sm_mhz * 1e6
    return {"bound": "issue", "unit": "warp instructions/s", "achieved": achieved, "peak": peak,
            "frac": achieved / peak, "warp_inst_per_launch": inst,
            "peak_source": "4 issue slots x %d SMs x median sampled SM clock %.0f MHz"
                           % (n_sms, sm_mhz)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gvx", choices=["gvx", "reference"])
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--forms", default=",".join(FORMS),
                    help="comma-separated subset of %s" % ",".join(FORMS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--clock-window", type=float, default=LOAD_WINDOW_S,
                    help="seconds of untimed back-to-back steps sampled for clocks before the "
                         "timed region (0 under a profiler)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--n-log2", type=int, default=26,
                    help="problem size for profiling captures only (the benchmark is 2^26)")
    args = ap.parse_args()
    global N_FULL
    N_FULL = 1 << args.n_log2
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gvx(args)


if __name__ == "__main__":
    sys.exit(main())
