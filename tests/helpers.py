"""Shared helpers for the GPU parity tests (tolerances, device transfer, error measures)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

# FP64 gate: relative error of every pair mass against the binary128 definition.
TOL_F64 = 1e-12
PI_D = float(np.pi)


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def dev(x, layout="aos", dtype=None):
    """(n, k) numpy rows -> CUDA tensor, AoS (n, k) or SoA (k, n)."""
    import torch
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    if layout == "soa":
        t = t.t().contiguous()
    return t.cuda()


def host(t, layout="aos"):
    x = t.detach().cpu().numpy()
    return x.T.copy() if layout == "soa" else x


def rel_err(got, ref):
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    den = np.abs(ref)
    out = np.abs(got - ref) / np.where(den > 0, den, 1.0)
    return np.where(np.isnan(ref) & np.isnan(got), 0.0, out)


def normwise(got, ref, scale):
    """max_k |got_k - ref_k| / scale per row."""
    return np.max(np.abs(np.asarray(got) - np.asarray(ref)), axis=1) / scale


def scaled_grad_err(g, r, x):
    """Normwise error of a gradient, each component weighted by max(|x_k|, 1) (so that all
    components carry the unit of the output), relative to the weighted 1-norm of the reference."""
    s = np.maximum(np.abs(x), 1.0)
    den = np.sum(np.abs(r) * s, axis=1)
    return np.max(np.abs(g - r) * s, axis=1) / np.where(den > 0, den, 1.0)


def summary(err):
    err = np.asarray(err)
    return "max %.3e  p99.9 %.3e  p50 %.3e" % (err.max(), np.quantile(err, 0.999),
                                               np.quantile(err, 0.5))


def edge_pairs():
    """Degenerate and adversarial PtEtaPhiM pairs (rows of a and b)."""
    rows = [
        # identical legs, zero vectors, legs at rest, massless collinear
        ([7, 1.5, 0.3, 2], [7, 1.5, 0.3, 2]),
        ([0, 0, 0, 0], [0, 0, 0, 0]),
        ([12, 0, 0, 5], [0, 0, 0, 0]),
        ([0, 0.3, 1, 3], [0, -2, 2, 4]),
        ([10, 0.7, -1, 0], [20, 0.7, -1, 0]),
        # back to back, perpendicular
        ([50, 1.2, 0.4, 0], [50, 1.2, 0.4 - PI_D, 0]),
        ([1, 0, 0, 0], [1, 0, PI_D / 2, 0]),
        # azimuthal wrap: |d_phi| close to 2 pi
        ([100, 0.1, PI_D, 0], [80, 0.1, -PI_D, 0]),
        ([100, 0.1, PI_D - 1e-9, 0], [80, 0.1, -PI_D + 1e-9, 0]),
        ([100, 0.1, PI_D - 1e-6, 1e-4], [80, 0.1, -PI_D + 3e-6, 0]),
        ([100, 2.0, -PI_D + 1e-5, 0], [80, 2.0, PI_D - 2e-5, 0]),
        ([5, 0.0, 3.0, 0.1], [5, 0.0, -3.0, 0.1]),
        # near collinear in eta only, in phi only
        ([300, 2.5, 1.0, 0], [200, 2.5 + 1e-8, 1.0, 0]),
        ([300, -3.9, 1.0, 1e-3], [200, -3.9, 1.0 + 1e-8, 1e-3]),
        # large |eta|, tiny pt, heavy legs
        ([10, 10.0, 0.5, 1], [20, -12.0, -0.5, 2]),
        ([1e-3, 0.1, 0.2, 1e3], [2e-3, -0.1, 2.2, 5e2]),
        ([1000, 4.0, 3.1, 10], [1000, -4.0, -3.1, 10]),
        ([1, -4.0, -PI_D, 0], [1000, 4.0, PI_D - 1e-12, 0]),
    ]
    a = np.array([r[0] for r in rows], dtype=np.float64)
    b = np.array([r[1] for r in rows], dtype=np.float64)
    return a, b


def build_ff_harness(out_dir):
    """Compile tests/ff_harness.cpp (the library's float-float and fixed-point headers built for
    the host) into out_dir and load it."""
    from paper_2312_02756_gb300 import gen_tables
    out_dir = str(out_dir)
    gen_tables.write(os.path.join(out_dir, "gvx_tables.inc"))
    out = os.path.join(out_dir, "ffh.so")
    here = os.path.dirname(os.path.abspath(__file__))
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-I" + out_dir, os.path.join(here, "ff_harness.cpp"), "-o", out],
                   check=True)
    lib = ctypes.CDLL(out)
    for name in ("ffh_mass", "ffh_mass_grad", "ffh_boost", "ffh_boost_bwd", "ffh_mass_cart",
                 "ffh_mass_cart_fixed", "ffh_apply", "ffh_convert", "ffh_mass_lp",
                 "ffh_mass_lc", "ffh_mass_lc_event",
                 "ffh_mass_grad_lc", "ffh_mass_e_lc"):
        getattr(lib, name).restype = ctypes.c_int64
    return lib
