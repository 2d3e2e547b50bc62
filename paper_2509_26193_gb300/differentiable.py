"""Differentiable form: the mean expected synapse length as a torch autograd op.

``mean_synapse_length(ctx, x, y, z, sigma, vac_ax, vac_de, theta)`` builds the
octree of the given positions, runs the bottom-up update and the forward
kernel of ``relearn_mean_length``, and returns the mean as a 0-d float64 tensor;
its backward is the hand-written adjoint ``relearn_mean_length_backward``
(gradients for x, y, z and sigma). sigma stays on the device (a 1-element
float32 tensor), so a training loop never synchronises with the host.
Every step runs in the library's kernels; there is no fallback.
"""
from __future__ import annotations

import torch

from . import relearn as R


class MeanSynapseLength(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x, y, z, sigma, rctx, vac_ax, vac_de, theta):
        R.relearn_build_octree(rctx, x.detach(), y.detach(), z.detach())
        sig = sigma.detach().reshape(1).to(torch.float32).contiguous()
        prm = R.params(1.0, theta, 0, 0, net_sigma=sig)
        mean = torch.empty(1, dtype=torch.float64, device=x.device)
        R.relearn_mean_length(rctx, prm, vac_ax, vac_de, mean)
        fctx.rctx, fctx.vac_ax, fctx.vac_de = rctx, vac_ax, vac_de
        fctx.keep = sig  # the forward's sigma stays alive until the backward
        fctx.sigma_shape, fctx.sigma_dtype = sigma.shape, sigma.dtype
        return mean.reshape(())

    @staticmethod
    def backward(fctx, gout):
        n = fctx.rctx.n
        dev = fctx.vac_ax.device
        gx, gy, gz = (torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3))
        gs = torch.empty(1, dtype=torch.float64, device=dev)
        g = gout.detach().reshape(1).to(torch.float64).contiguous()
        R.relearn_mean_length_backward(fctx.rctx, fctx.vac_ax, fctx.vac_de, gx, gy, gz,
                                       grad_mean=g, gsigma=gs)
        gsig = gs.to(fctx.sigma_dtype).reshape(fctx.sigma_shape)
        return gx, gy, gz, gsig, None, None, None, None


def mean_synapse_length(rctx, x, y, z, sigma, vac_ax, vac_de, theta=0.3):
    """x, y, z: float32 CUDA tensors [n]; sigma: CUDA tensor with one element (float32 or
    float64); vac_ax, vac_de: int32 CUDA tensors [n]."""
    return MeanSynapseLength.apply(x, y, z, sigma, rctx, vac_ax, vac_de, float(theta))


def calibrate_sigma(rctx, x, y, z, vac_ax, vac_de, sigma0, target, steps=50, lr=30.0,
                    betas=(0.5, 0.999), theta=0.3):
    """Adam on sigma (um) so that the mean expected synapse length approaches ``target``
    (loss ((mean - target) / target)^2). A short first-moment memory (beta1 = 0.5) keeps
    the one-parameter problem from overshooting. Returns (sigma history, mean history)."""
    sigma = torch.tensor([float(sigma0)], dtype=torch.float32, device=x.device,
                         requires_grad=True)
    opt = torch.optim.Adam([sigma], lr=lr, betas=betas)
    sig_hist, mean_hist = [], []
    for _ in range(steps):
        opt.zero_grad(set_to_none=True)
        m = mean_synapse_length(rctx, x, y, z, sigma, vac_ax, vac_de, theta)
        loss = ((m - float(target)) / float(target)) ** 2
        loss.backward()
        opt.step()
        sig_hist.append(sigma.detach().clone())
        mean_hist.append(m.detach().clone())
    return torch.cat(sig_hist), torch.stack(mean_hist)
