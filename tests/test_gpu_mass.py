"""GPU parity of gvx_invariant_mass against the binary128 definition oracle (O1).

FP64: every element within 1e-12 relative (plus an absolute floor of 1e-16 (E1 + E2), far below
1e-12 m unless the pair is exactly degenerate, where the definition itself rounds to +-1e-17 E).
FP32: the error per output against O1 on the exact upcast of the FP32 inputs is measured and held
to the bound derived from the arithmetic (all terms non-negative: a few ulps).
"""
import numpy as np
import pytest

import gvx_synth as syn
from helpers import TOL_F64, dev, edge_pairs, host, rel_err, summary, torch_cuda

pytestmark = pytest.mark.gpu

N0 = 65_536  # the small FP64 workload: 65,536 pairs
N_FULL = 1 << 26
TOL_F32 = 2.0e-6  # ~34 ulp of FP32; measured max is reported by the test


def _energy_scale(a, b):
    e = lambda x: np.sqrt((x[:, 0] * np.cosh(x[:, 1])) ** 2 + x[:, 3] ** 2)
    return e(a) + e(b)


def _check_f64(got, ref, a, b):
    bound = TOL_F64 * np.abs(ref) + 1e-16 * _energy_scale(a, b)
    bad = np.abs(got - ref) > bound
    assert not bad.any(), (np.flatnonzero(bad)[:5], got[bad][:5], ref[bad][:5])


@pytest.fixture(scope="module")
def cfg0(orc):
    g = syn.rng(0)
    a, b = syn.ptetaphim(g, N0), syn.ptetaphim(g, N0)
    return a, b, orc.mass_def(a, b, nthreads=8)


@pytest.mark.parametrize("la,lb", [("soa", "soa"), ("aos", "aos"), ("soa", "aos"), ("aos", "soa")])
def test_mass_f64_small_workload(cfg0, la, lb):
    torch_cuda()
    import paper_2312_02756_gb300 as gvx
    a, b, ref = cfg0
    m = gvx.invariant_mass(dev(a, la), dev(b, lb), la, lb).cpu().numpy()
    _check_f64(m, ref, a, b)
    print("FP64 mass vs O1 (%s/%s): %s" % (la, lb, summary(rel_err(m, ref))))


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 255, 256, 257, 4097, 77_777])
def test_mass_f64_ragged_sizes(orc, n):
    torch_cuda()
    import paper_2312_02756_gb300 as gvx
    g = syn.rng(10 + n)
    a, b = syn.ptetaphim(g, n), syn.ptetaphim(g, n)
    for layout in ("soa", "aos"):
        m = gvx.invariant_mass(dev(a, layout), dev(b, layout), layout, layout).cpu().numpy()
        assert m.shape == (n,)
        _check_f64(m, orc.mass_def(a, b, nthreads=8), a, b)


def test_mass_f64_edge_cases(orc):
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    a, b = edge_pairs()
    ref = orc.mass_def(a, b)
    for layout in ("soa", "aos"):
        m = gvx.invariant_mass(dev(a, layout), dev(b, layout), layout, layout).cpu().numpy()
        _check_f64(m, ref, a, b)
    # adversarial near-collinear light pairs: the plain FP64 form loses up to 1e-8 here
    from test_oracle_pins import _adversarial_pairs
    a, b = _adversarial_pairs(50_000, 104)
    m = gvx.invariant_mass(dev(a), dev(b)).cpu().numpy()
    _check_f64(m, orc.mass_def(a, b, nthreads=8), a, b)
    # n = 0
    e = torch.empty((0, 4), dtype=torch.float64, device="cuda")
    assert gvx.invariant_mass(e, e).shape == (0,)


def test_mass_f64_full_size_sampled(orc):
    """2^26 pairs in both layouts (the benchmark launch): 2^16 sampled outputs against O1,
    and properties of all outputs."""
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    g = syn.rng(1)
    a, b = syn.ptetaphim(g, N_FULL), syn.ptetaphim(g, N_FULL)
    idx = np.sort(syn.rng(101).choice(N_FULL, 1 << 16, replace=False))
    ref = orc.mass_def(a[idx], b[idx], nthreads=8)
    for layout in ("soa", "aos"):
        da, db = dev(a, layout), dev(b, layout)
        m = gvx.invariant_mass(da, db, layout, layout)
        torch.cuda.synchronize()
        del da, db
        mh = m.cpu().numpy()
        assert np.all(np.isfinite(mh)) and np.all(mh >= 0)
        _check_f64(mh[idx], ref, a[idx], b[idx])
        del m
        torch.cuda.empty_cache()


def test_mass_f32_error_per_output(orc):
    """FP32 in and out, half of the particles light and hard: report and bound the relative
    error of every output against O1 on the exact upcast inputs."""
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    g = syn.rng(2)
    n = 1 << 20
    a32 = syn.to_f32(syn.ptetaphim_light_mix(g, n))
    b32 = syn.to_f32(syn.ptetaphim_light_mix(g, n))
    ref = orc.mass_def(a32.astype(np.float64), b32.astype(np.float64), nthreads=8)
    for layout in ("soa", "aos"):
        m = gvx.invariant_mass(dev(a32, layout), dev(b32, layout), layout, layout).cpu().numpy()
        assert m.dtype == np.float32
        err = rel_err(m, ref)
        print("FP32 mass vs O1 (%s): %s" % (layout, summary(err)))
        assert err.max() <= TOL_F32
    # the plain FP32 definition on the same inputs, for comparison (information)
    naive = orc.mass_naive_fp64(a32.astype(np.float64), b32.astype(np.float64))
    del naive
