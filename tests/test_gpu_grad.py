"""GPU parity of the hand-written adjoints (gvx_invariant_mass_bwd, gvx_boost_bwd) against the
binary128 chain-rule gradients of the oracle, against central finite differences, and through
torch.autograd.

Mass gradient error measure: per pair, components weighted by max(|x_k|, 1) (so all carry the
unit of m), normwise relative to the weighted 1-norm of the reference (helpers.scaled_grad_err).
FP64 gate 1e-12.  Boost: normwise relative to the largest reference component, FP64 gate 1e-12.
"""
import os

import numpy as np
import pytest

import gvx_synth as syn
from helpers import TOL_F64, dev, host, scaled_grad_err, summary, torch_cuda

pytestmark = pytest.mark.gpu

N_GRAD = 1 << 16


def _mass_grads(a, b, gm, layout="aos", dtype=None):
    import paper_2312_02756_gb300 as gvx
    torch = torch_cuda()
    ta = dev(a, layout, dtype).requires_grad_(True)
    tb = dev(b, layout, dtype).requires_grad_(True)
    m = gvx.invariant_mass(ta, tb, layout, layout)
    m.backward(torch.as_tensor(gm, dtype=m.dtype, device="cuda"))
    return host(ta.grad, layout), host(tb.grad, layout), m.detach().cpu().numpy()


@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_mass_grad_f64_vs_oracle(orc, layout):
    g = syn.rng(40)
    a, b = syn.ptetaphim(g, N_GRAD), syn.ptetaphim(g, N_GRAD)
    gm = syn.upstream(g, N_GRAD)
    ga, gb, _ = _mass_grads(a, b, gm, layout)
    ra, rb = orc.mass_grad_def(a, b, gm, nthreads=8)
    err = scaled_grad_err(np.hstack([ga, gb]), np.hstack([ra, rb]), np.hstack([a, b]))
    print("FP64 mass grad vs O1 (%s): %s" % (layout, summary(err)))
    assert err.max() <= TOL_F64


def test_mass_grad_f64_full_size(orc):
    """2^24 pairs (SoA, the saved masses passed to the adjoint as autograd does): every gradient
    against O2's adjoint (pinned to O1 at 1e-14), normwise as above."""
    g = syn.rng(39)
    n = 1 << 24
    a, b = syn.ptetaphim(g, n), syn.ptetaphim(g, n)
    gm = syn.upstream(g, n)
    ga, gb, _ = _mass_grads(a, b, gm, "soa")
    ra, rb = orc.mass_grad_fp64(a, b, gm, nthreads=os.cpu_count() or 8)
    err = scaled_grad_err(np.hstack([ga, gb]), np.hstack([ra, rb]), np.hstack([a, b]))
    print("FP64 mass grad 2^24 vs O2, every element: %s" % summary(err))
    assert err.max() <= TOL_F64


def test_mass_grad_f64_edges(orc):
    from helpers import edge_pairs
    from test_oracle_pins import _adversarial_pairs
    for a, b in (edge_pairs(), _adversarial_pairs(20_000, 41)):
        gm = np.linspace(-1, 1, len(a))
        ga, gb, m = _mass_grads(a, b, gm)
        ra, rb = orc.mass_grad_def(a, b, gm)
        mref = orc.mass_def(a, b)
        ok = mref > 1e-9 * (a[:, 0] + b[:, 0] + a[:, 3] + b[:, 3] + 1e-300)  # m = 0: see below
        err = scaled_grad_err(np.hstack([ga, gb]), np.hstack([ra, rb]), np.hstack([a, b]))
        assert err[ok].max() <= TOL_F64
        # where m = 0 the gradient is defined as 0
        assert np.all(ga[m == 0] == 0) and np.all(gb[m == 0] == 0)


def test_mass_grad_f64_finite_differences():
    """Central differences of the GPU forward, h = 1e-6 relative (the FD truncation and rounding
    error of that step is ~1e-9 relative, hence the looser bound)."""
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    g = syn.rng(42)
    n = 4096
    a, b = syn.ptetaphim(g, n), syn.ptetaphim(g, n)
    gm = syn.upstream(g, n)
    ga, gb, _ = _mass_grads(a, b, gm)
    for legs, grad, which in ((a, ga, 0), (b, gb, 1)):
        for k in range(4):
            h = 1e-6 * np.maximum(np.abs(legs[:, k]), 1.0)
            hi, lo = legs.copy(), legs.copy()
            hi[:, k] += h
            lo[:, k] -= h
            pair = (lambda x: (dev(x), dev(b))) if which == 0 else (lambda x: (dev(a), dev(x)))
            mh = gvx.invariant_mass(*pair(hi)).cpu().numpy()
            ml = gvx.invariant_mass(*pair(lo)).cpu().numpy()
            fd = (mh - ml) / (hi[:, k] - lo[:, k]) * gm
            scale = np.abs(grad).max(axis=1) + 1e-300
            assert np.all(np.abs(fd - grad[:, k]) <= 1e-6 * scale), (which, k)


def test_mass_grad_autograd_gradcheck():
    """The autograd wiring, against torch's central differences of the forward with its absolute
    step 1e-6: the forward's rounding (~1e-13 relative) becomes ~m 1e-7 of noise in the numerical
    Jacobian, so the pairs are kept moderate (pt in [1, 10], |eta| <= 1: m <= ~20); the 1e-12
    gates are the oracle and relative-step tests above."""
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    g = syn.rng(43)
    def legs():
        x = syn.ptetaphim(g, 64)
        x[:, 0] = 1 + 9 * g.random(64)
        x[:, 1] = g.uniform(-1, 1, 64)
        return x
    a = dev(legs()).requires_grad_(True)
    b = dev(legs()).requires_grad_(True)
    assert torch.autograd.gradcheck(gvx.invariant_mass, (a, b), eps=1e-6, atol=1e-5, rtol=1e-6)


def test_mass_grad_f32_error(orc):
    torch = torch_cuda()
    g = syn.rng(44)
    n = 1 << 18
    a32 = syn.to_f32(syn.ptetaphim(g, n))
    b32 = syn.to_f32(syn.ptetaphim(g, n))
    gm32 = syn.to_f32(syn.upstream(g, n))
    ga, gb, _ = _mass_grads(a32, b32, gm32, "aos", torch.float32)
    ra, rb = orc.mass_grad_def(a32.astype(np.float64), b32.astype(np.float64),
                               gm32.astype(np.float64), nthreads=8)
    err = scaled_grad_err(np.hstack([ga, gb]).astype(np.float64), np.hstack([ra, rb]),
                          np.hstack([a32, b32]).astype(np.float64))
    print("FP32 mass grad vs O1: %s" % summary(err))
    assert err.max() <= 1e-5


def _boost_grads(v, beta, gout, layout="aos", dtype=None):
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    tv = dev(v, layout, dtype).requires_grad_(True)
    if beta.ndim == 1:
        tb = dev(beta.reshape(1, 3), "aos", dtype)[0].detach().requires_grad_(True)
    else:
        tb = dev(beta, layout, dtype).requires_grad_(True)
    out = gvx.boost(tv, tb, layout=layout, beta_layout=None if beta.ndim == 1 else layout)
    out.backward(dev(gout, layout, dtype))
    gb = tb.grad.cpu().numpy() if beta.ndim == 1 else host(tb.grad, layout)
    return host(tv.grad, layout), gb


@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_boost_grad_f64_vs_oracle(orc, layout):
    g = syn.rng(45)
    v, beta = syn.pxpypze(g, N_GRAD), syn.velocities(g, N_GRAD, 0.99)
    gout = syn.upstream(g, (N_GRAD, 4))
    gv, gb = _boost_grads(v, beta, gout, layout)
    rv, rb = orc.boost_grad_def(v, beta, gout)
    ev = np.max(np.abs(gv - rv), axis=1) / np.max(np.abs(rv), axis=1)
    eb = np.max(np.abs(gb - rb), axis=1) / np.max(np.abs(rb), axis=1)
    print("FP64 boost grad_v vs O1 (%s): %s" % (layout, summary(ev)))
    print("FP64 boost grad_beta vs O1 (%s): %s" % (layout, summary(eb)))
    assert ev.max() <= TOL_F64 and eb.max() <= TOL_F64


def test_boost_grad_f64_shared_velocity(orc):
    g = syn.rng(46)
    n = 100_003
    v = syn.pxpypze(g, n) / 100.0
    gout = syn.upstream(g, (n, 4))
    beta = np.array([0.2, -0.6, 0.3])
    gv, gb = _boost_grads(v, beta, gout)
    rv, rb = orc.boost_grad_def(v, beta, gout)
    assert np.max(np.abs(gv - rv)) <= TOL_F64 * np.max(np.abs(rv))
    # the shared gradient is a sum of n terms of both signs: bound by the sum of magnitudes
    _, rb_each = orc.boost_grad_def(v, np.tile(beta, (n, 1)), gout)
    assert np.all(np.abs(gb - rb) <= TOL_F64 * np.sum(np.abs(rb_each), axis=0))


def test_boost_grad_f64_finite_differences():
    """Central differences of the GPU boost, h = 1e-6 relative (max(|x|, 1)), for the loss
    sum(gout . boost(v, beta)): the gradients with respect to the 4-vector and to beta, per
    vector within 1e-6 of the largest gradient component (FD truncation and rounding at this step
    are far below that)."""
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    g = syn.rng(49)
    n = 4096
    v, beta = syn.pxpypze(g, n), syn.velocities(g, n, 0.99)
    gout = syn.upstream(g, (n, 4))
    gv, gb = _boost_grads(v, beta, gout)
    loss = lambda vv, bb: np.sum(gvx.boost(dev(vv), dev(bb)).cpu().numpy() * gout, axis=1)
    for x, grad, width, which in ((v, gv, 4, "v"), (beta, gb, 3, "beta")):
        scale = np.abs(grad).max(axis=1) + 1e-300
        for k in range(width):
            h = 1e-6 * np.maximum(np.abs(x[:, k]), 1.0) if which == "v" else np.full(n, 1e-6)
            hi, lo = x.copy(), x.copy()
            hi[:, k] += h
            lo[:, k] -= h
            if which == "v":
                fd = (loss(hi, beta) - loss(lo, beta)) / (hi[:, k] - lo[:, k])
            else:
                fd = (loss(v, hi) - loss(v, lo)) / (hi[:, k] - lo[:, k])
            err = np.abs(fd - grad[:, k]) / scale
            assert err.max() <= 1e-6, (which, k, err.max())


def test_boost_grad_autograd_gradcheck():
    torch = torch_cuda()
    import paper_2312_02756_gb300 as gvx
    g = syn.rng(47)
    v = dev(syn.pxpypze(g, 32) / 100.0).requires_grad_(True)
    beta = dev(syn.velocities(g, 32, 0.9)).requires_grad_(True)
    assert torch.autograd.gradcheck(gvx.boost, (v, beta), eps=1e-7, atol=1e-5, rtol=1e-5)


def test_boost_grad_f32_error(orc):
    torch = torch_cuda()
    g = syn.rng(48)
    n = 1 << 18
    v32 = syn.to_f32(syn.pxpypze(g, n) / 100.0)
    b32 = syn.to_f32(syn.velocities(g, n, 0.99))
    g32 = syn.to_f32(syn.upstream(g, (n, 4)))
    gv, gb = _boost_grads(v32, b32, g32, "aos", torch.float32)
    rv, rb = orc.boost_grad_def(v32.astype(np.float64), b32.astype(np.float64),
                                g32.astype(np.float64))
    ev = np.max(np.abs(gv - rv), axis=1) / np.max(np.abs(rv), axis=1)
    eb = np.max(np.abs(gb - rb), axis=1) / np.max(np.abs(rb), axis=1)
    print("FP32 boost grad_v vs O1: %s" % summary(ev))
    print("FP32 boost grad_beta vs O1: %s" % summary(eb))
    assert ev.max() <= 1e-4 and eb.max() <= 1e-3
