"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare with the oracle. Imported by test modules only."""
import numpy as np

# A search may legitimately differ between FP32 (GPU) and FP64 (oracle) only when
# one of its criterion tests is within 1e-5 (relative to len^2) of a tie or one
# of its draws lies within 1e-5 of a cumulative-probability boundary.
AC_MARGIN = 1e-5
DRAW_MARGIN = 1e-5
LNS_TOL = 1e-5   # |ln S_gpu - ln S_oracle| = relative error of the attraction sum


def torch_mod():
    import torch
    return torch


def dev(a):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


class GpuNet:
    """One network on the GPU: context, positions, vacancies, types."""

    def __init__(self, net, max_synapses=None, max_searches=0, box=None):
        from paper_2509_26193_gb300 import build, relearn as R
        build.build()
        self.R = R
        self.net = net
        n = net.n
        cap = max_synapses or max(4 * int(net.vac_ax.sum()) + 16, 64)
        self.ctx = R.relearn_create(n, cap, max_searches)
        self.x, self.y, self.z = dev(net.x), dev(net.y), dev(net.z)
        self.vac_ax = dev(net.vac_ax.astype(np.int32))
        self.vac_de = dev(net.vac_de.astype(np.int32))
        self.type = dev(net.type.astype(np.uint8))
        lo, hi = (None, None) if box is None else box
        R.relearn_build_octree(self.ctx, self.x, self.y, self.z, self.vac_de, lo, hi)

    def update(self, step, theta=None, diag=True, stats=True):
        R = self.R
        p = R.params(self.net.sigma, self.net.theta if theta is None else theta, self.net.seed,
                     step, R.FLAG_DIAG if diag else 0)
        return R.relearn_update_connectivity(self.ctx, p, self.vac_ax, self.vac_de, self.type,
                                             stats=stats)

    def requests(self):
        return self.R.relearn_get_requests(self.ctx)

    def synapses(self):
        return self.R.relearn_get_synapses(self.ctx)

    def vacancies(self):
        return self.vac_ax.cpu().numpy(), self.vac_de.cpu().numpy()

    def close(self):
        self.ctx.close()


def compare_targets(gpu_tgt, orc_tgt, orc_diag):
    """Returns (mismatches outside the exemption, exempt searches, exempt mismatches)."""
    exempt = (orc_diag["margin_ac"] < AC_MARGIN) | (orc_diag["margin_draw"] < DRAW_MARGIN)
    diff = gpu_tgt != orc_tgt
    return int((diff & ~exempt).sum()), int(exempt.sum()), int((diff & exempt).sum())
