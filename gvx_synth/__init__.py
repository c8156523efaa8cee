"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws random numbers with the shapes and distributions of the paper's
workloads (two arrays of particles for the invariant mass, one array for the boost, Sec. 5.1);
it holds none of the arithmetic under test.  Every generator takes a numpy Generator so that the
CUDA path and the oracle can be fed the identical bytes.

Distributions ("collider-like"):
  * PtEtaPhiM: pt log-uniform in [1, 1000] GeV, eta uniform in [-4, 4], phi uniform in
    [-pi, pi), m uniform in [0, 10] GeV.
  * light/heavy mix: a Bernoulli(1/2) mask per particle; masked particles have m uniform in
    [0, 1e-3] GeV and pt log-uniform in [100, 5000] GeV, the others are as above.
  * PxPyPzE (boost inputs): isotropic direction, |p| log-uniform in [1, 3e4] GeV (the range of
    pt cosh(eta) above), m uniform in [0, 10] GeV, E on the mass shell.
  * velocities: isotropic direction, |beta| uniform in [0, beta_max].
  * jagged multiplicities: Poisson(lam) clamped to [0, n_max]; offsets are their running sum.
  * upstream gradients: uniform in [-1, 1].
"""
from __future__ import annotations

import numpy as np

SEED = 2312_02756


def rng(stream_id: int = 0) -> np.random.Generator:
    """The generator for one named input stream (seed 2312_02756 + stream_id)."""
    return np.random.Generator(np.random.PCG64(SEED + int(stream_id)))


def _log_uniform(g, lo, hi, n):
    return np.exp(g.uniform(np.log(lo), np.log(hi), n))


def ptetaphim(g: np.random.Generator, n: int) -> np.ndarray:
    """(n, 4) float64 rows (pt, eta, phi, m)."""
    out = np.empty((n, 4))
    out[:, 0] = _log_uniform(g, 1.0, 1000.0, n)
    out[:, 1] = g.uniform(-4.0, 4.0, n)
    out[:, 2] = g.uniform(-np.pi, np.pi, n)
    out[:, 3] = g.uniform(0.0, 10.0, n)
    return out


def ptetaphim_light_mix(g: np.random.Generator, n: int) -> np.ndarray:
    """(n, 4) float64 rows; half of the particles near-massless and hard (see module doc)."""
    out = ptetaphim(g, n)
    light = g.random(n) < 0.5
    k = int(light.sum())
    out[light, 0] = _log_uniform(g, 100.0, 5000.0, k)
    out[light, 3] = g.uniform(0.0, 1e-3, k)
    return out


def _unit_vectors(g, n):
    d = g.standard_normal((n, 3))
    norm = np.sqrt(np.sum(d * d, axis=1))
    norm[norm == 0] = 1.0
    return d / norm[:, None]


def pxpypze(g: np.random.Generator, n: int) -> np.ndarray:
    """(n, 4) float64 rows (px, py, pz, E) of on-shell vectors."""
    p = _log_uniform(g, 1.0, 3.0e4, n)
    m = g.uniform(0.0, 10.0, n)
    out = np.empty((n, 4))
    out[:, :3] = _unit_vectors(g, n) * p[:, None]
    out[:, 3] = np.sqrt(p * p + m * m)
    return out


def velocities(g: np.random.Generator, n: int, beta_max: float = 0.99) -> np.ndarray:
    """(n, 3) float64 velocities with |beta| uniform in [0, beta_max]."""
    return _unit_vectors(g, n) * g.uniform(0.0, beta_max, n)[:, None]


def jagged_offsets(g: np.random.Generator, n_events: int, lam: float = 8.0,
                   n_max: int = 64) -> np.ndarray:
    """int64 offsets[n_events + 1] of Poisson(lam) multiplicities clamped to [0, n_max]."""
    counts = np.minimum(g.poisson(lam, n_events), n_max).astype(np.int64)
    off = np.zeros(n_events + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off


def upstream(g: np.random.Generator, shape) -> np.ndarray:
    """Upstream gradients, uniform in [-1, 1]."""
    return g.uniform(-1.0, 1.0, shape)


def to_f32(x: np.ndarray) -> np.ndarray:
    """Round-to-nearest float32 copy (the FP32 workloads store these)."""
    return np.asarray(x, dtype=np.float32)
