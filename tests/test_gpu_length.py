"""Differentiable form on the GPU (relearn_mean_length / _backward and the torch
autograd op) against the FP64 oracle.

Tolerances (derived from the arithmetic): every attraction, distance and product
is one or two FP32 roundings (relative 2^-24 each; the special-function unit adds
a few 2^-24); the forward sums are Kahan-compensated and the ratios formed in FP64,
so a source's length l_i, the mean and dL/dsigma carry relative errors of a few
1e-7: all within 1e-5 (the stated floating-point bar).

The position gradient is a sum of terms of both signs. It is compared element by
element in two ways:
  |g_gpu - g_orc| <= 1e-5 |g_orc| + 1e-5 max|g_orc| / sqrt(n)       (a)
  |g_gpu - g_orc| <= 1e-5 a_orc                                       (b)
where a_orc is the oracle's sum of the magnitudes of the same terms (the scale of
the rounding error of any evaluation of the sum). (a) holds at 2^12 and 2^14; its
floor shrinks like 1/sqrt(n) while FP32 term errors do not, so at 2^18 the bound
is (b), the componentwise relative error of a sum.

At theta > 0 a criterion test within FP32 rounding of its tie can put a node in or
out of a source's frontier on one side only. The forward exempts exactly the
sources with a root-frontier criterion test within 1e-5 of its tie (the oracle
reports the margin per source). A flip changes that source's contributions to
every node of its frontier, so the gradient of many neurons, and the gradient
checks at theta > 0 therefore run on the same network with those sources'
searches removed (vac_ax = 0 for every source with a margin below 1e-4, on both
sides), which leaves a tree and frontiers that FP32 reproduces.
"""
import numpy as np
import pytest

import oracle
from gpu_common import dev
from paper_2509_26193_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_26193_gb300 import build
    build.build()
    oracle.build()


def _gpu(net, theta, sigma=None, grad=True):
    import torch
    from paper_2509_26193_gb300 import relearn as R
    ctx = R.relearn_create(net.n, 64)
    x, y, z = dev(net.x), dev(net.y), dev(net.z)
    va, vd = dev(net.vac_ax), dev(net.vac_de)
    R.relearn_build_octree(ctx, x, y, z)
    prm = R.params(net.sigma if sigma is None else sigma, theta, 0, 0)
    mean = torch.empty(1, dtype=torch.float64, device="cuda")
    ell = torch.empty(net.n, dtype=torch.float32, device="cuda")
    R.relearn_mean_length(ctx, prm, va, vd, mean, ell)
    out = {"mean": float(mean.item()), "ell": ell.cpu().numpy().astype(np.float64)}
    if grad:
        g = [torch.empty(net.n, dtype=torch.float32, device="cuda") for _ in range(3)]
        gs = torch.empty(1, dtype=torch.float64, device="cuda")
        R.relearn_mean_length_backward(ctx, va, vd, *g, gsigma=gs)
        out["g"] = np.stack([t.cpu().numpy() for t in g], 1).astype(np.float64)
        out["dsigma"] = float(gs.item())
    ctx.close()
    return out


def _orc(net, theta, sigma=None, grad=True):
    t = oracle.Tree(net.x, net.y, net.z)
    t.reduce(net.vac_de)
    r = oracle.mean_length(t, net.sigma if sigma is None else sigma, theta, net.vac_ax,
                           net.vac_de, grad=grad, threads=16)
    t.close()
    return r


def _compare_forward(g, o, theta):
    assert abs(g["mean"] - o["mean"]) <= 1e-5 * o["mean"]
    ok = np.isfinite(o["ell"])
    assert np.array_equal(np.isfinite(g["ell"]), ok)
    rel = np.abs(g["ell"][ok] - o["ell"][ok]) / o["ell"][ok]
    near = o["margin_ac"][ok] < 1e-5   # a criterion test within 1e-5 of its tie
    if theta == 0.0:
        assert not near.any()
    assert rel[~near].max() <= 1e-5, rel[~near].max()
    print(f"forward: max rel {rel[~near].max():.2e}, {int(near.sum())} of {int(ok.sum())} "
          f"sources exempt (criterion margin < 1e-5)")


def _compare_gradient(g, o, n, floor_rule=True):
    assert abs(g["dsigma"] - o["dsigma"]) <= 1e-5 * abs(o["dsigma"])
    err = np.abs(g["g"] - o["g"])
    ra = err / (np.abs(o["g"]) + np.abs(o["g"]).max() / np.sqrt(n))
    rb = err / np.maximum(o["g_abs"], 1e-300)
    print(f"gradient n={n}: (a) max {ra.max():.2e}, (b) max {rb.max():.2e}, "
          f"norm {np.linalg.norm(err) / np.linalg.norm(o['g']):.2e}")
    assert rb.max() <= 1e-5, rb.max()
    if floor_rule:
        assert ra.max() <= 1e-5, ra.max()


def _tie_free(net, theta, cut=1e-4):
    """The same network without the searches of sources whose root frontier has a
    criterion test within `cut` of its tie (their vac_ax set to 0)."""
    o = _orc(net, theta, grad=False)
    near = o["margin_ac"] < cut
    net.vac_ax = np.where(near, 0, net.vac_ax).astype(np.int32)
    return net, int(near.sum())


@pytest.mark.parametrize("n", [1 << 12, 1 << 14])
@pytest.mark.parametrize("theta", [0.0, 0.3])
def test_forward_and_adjoint_match_oracle(theta, n):
    net = workloads.differentiable_cube(n=n)
    _compare_forward(_gpu(net, theta, grad=False), _orc(net, theta, grad=False), theta)
    if theta > 0:
        net, removed = _tie_free(net, theta)
        print(f"{removed} sources near a criterion tie removed for the gradient check")
    _compare_gradient(_gpu(net, theta), _orc(net, theta), n, floor_rule=n <= 1 << 12)


def test_sigma_gradient_matches_fp64_central_difference():
    """d mean / d sigma on the GPU against the oracle's FP64 central difference
    (h = 1e-3 sigma) at theta = 0.3 (the criterion does not depend on sigma)."""
    net = workloads.differentiable_cube(n=1 << 12)
    h = 1e-3 * net.sigma
    fd = (_orc(net, 0.3, net.sigma + h, grad=False)["mean"]
          - _orc(net, 0.3, net.sigma - h, grad=False)["mean"]) / (2 * h)
    g = _gpu(net, 0.3)
    assert abs(g["dsigma"] - fd) <= 1e-3 * abs(fd), (g["dsigma"], fd)


def test_full_size_2p18():
    net = workloads.differentiable_cube()
    _compare_forward(_gpu(net, 0.3, grad=False), _orc(net, 0.3, grad=False), 0.3)
    net, removed = _tie_free(net, 0.3)
    print(f"{removed} sources near a criterion tie removed for the gradient check")
    _compare_gradient(_gpu(net, 0.3), _orc(net, 0.3), net.n, floor_rule=False)


def test_edge_cases():
    from paper_2509_26193_gb300 import relearn as R
    # nobody to connect to: mean is NaN, gradients zero
    net = workloads.differentiable_cube(n=100, seed=31)
    net.vac_de[:] = 0
    g = _gpu(net, 0.3)
    assert np.isnan(g["mean"]) and np.all(np.isnan(g["ell"]))
    assert np.all(g["g"] == 0.0) and g["dsigma"] == 0.0
    # two neurons: the length is their distance
    net = workloads.differentiable_cube(n=2, seed=32)
    net.x[:] = [100.0, 400.0]
    net.y[:] = [50.0, 450.0]
    net.z[:] = [7.0, 7.0]
    net.vac_ax[:] = [3, 0]
    net.vac_de[:] = [0, 2]
    g = _gpu(net, 0.3)
    assert g["mean"] == pytest.approx(500.0, rel=1e-6)
    u = np.array([-300.0, -400.0, 0.0]) / 500.0
    assert np.allclose(g["g"][0], u, atol=1e-6) and np.allclose(g["g"][1], -u, atol=1e-6)
    # the backward needs its forward
    ctx = R.relearn_create(16, 16)
    t = dev(np.zeros(16, np.int32))
    with pytest.raises(R.RelearnError):
        R.relearn_mean_length_backward(ctx, t, t, *(dev(np.zeros(16, np.float32))
                                                     for _ in range(3)))
    ctx.close()


def test_autograd_op_and_sigma_calibration():
    """The torch op returns the C-ABI values; 50 Adam steps bring the mean expected
    synapse length of the 2^18-neuron cube from its sigma = 800 um value to 600 um."""
    import torch
    from paper_2509_26193_gb300 import relearn as R
    from paper_2509_26193_gb300.differentiable import calibrate_sigma, mean_synapse_length
    net = workloads.differentiable_cube()
    ctx = R.relearn_create(net.n, 64)
    x, y, z = (dev(a).requires_grad_(True) for a in (net.x, net.y, net.z))
    va, vd = dev(net.vac_ax), dev(net.vac_de)
    sigma = torch.tensor([net.sigma], dtype=torch.float32, device="cuda", requires_grad=True)
    m = mean_synapse_length(ctx, x, y, z, sigma, va, vd, 0.3)
    m.backward()
    ref = _gpu(net, 0.3)
    assert float(m.detach()) == pytest.approx(ref["mean"], rel=1e-12)
    assert float(sigma.grad) == pytest.approx(ref["dsigma"], rel=1e-6)
    assert np.allclose(x.grad.cpu().numpy(), ref["g"][:, 0], rtol=0, atol=1e-9 + 1e-5 *
                       np.abs(ref["g"]).max())
    sig, means = calibrate_sigma(ctx, x.detach(), y.detach(), z.detach(), va, vd, net.sigma,
                                 600.0, steps=50)
    final = float(means[-1])
    assert abs(final - 600.0) < 2.0, final
    # the calibrated sigma checked by the oracle
    o = _orc(net, 0.3, float(sig[-1]), grad=False)
    assert abs(o["mean"] - 600.0) < 3.0, o["mean"]
    ctx.close()
