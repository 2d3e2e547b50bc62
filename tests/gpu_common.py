"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare with the oracle. Imported by test modules only."""
import numpy as np

# A search may legitimately differ between FP32 (GPU) and FP64 (oracle) only when
# one of its criterion tests is within 1e-5 (relative to len^2) of a tie or one
# of its draws lies within 1e-5 of a cumulative-probability boundary.
AC_MARGIN = 1e-5
DRAW_MARGIN = 1e-5
LNS_TOL = 1e-5   # |ln S_gpu - ln S_oracle| = relative error of the attraction sum
TIGHT_MARGIN = 1e-6  # see check_targets


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


def check_targets(gpu_tgt, orc_tgt, orc_diag, label=""):
    """Asserts the search parity rule and returns its counts.

    No search may differ outside the exemption, and the exempt searches that do
    differ are bounded: at most a tenth of the exempt ones (or 2). A search whose
    criterion test or draw lies within 1e-5 of a tie may go either way in FP32, but
    only a small share of them actually should; an exempt search that could return
    any target would otherwise pass unnoticed.

    Second, tighter check: no search differs whose margins (criterion and draw) are
    both at least TIGHT_MARGIN = 1e-6. The GPU's cumulative sums are Kahan-compensated
    FP32 with an FP64 normaliser (relative error a few 1e-7) and its centroids FP32
    roundings of exact sums, so a real disagreement needs a tie far closer than the
    stated 1e-5; this check exempts about ten times fewer searches (0.1 to 0.8 % on the
    clustered and uniform workloads against 2 to 7 %) and so has more power. Also
    reports, for the searches that differ, the largest oracle margin seen."""
    bad, exempt, exempt_diff = compare_targets(gpu_tgt, orc_tgt, orc_diag)
    diff = gpu_tgt != orc_tgt
    m_ac = float(orc_diag["margin_ac"][diff].max()) if diff.any() else 0.0
    m_dr = float(orc_diag["margin_draw"][diff].max()) if diff.any() else 0.0
    m = np.minimum(orc_diag["margin_ac"][diff], orc_diag["margin_draw"][diff])
    worst = float(m.max()) if diff.any() else 0.0
    n = len(gpu_tgt)
    info = dict(searches=n, exempt=exempt, exempt_share=exempt / max(n, 1), bad=bad,
                exempt_diff=exempt_diff, worst_margin_of_diff=worst, max_ac=m_ac, max_draw=m_dr,
                share_ac=float(np.mean(orc_diag["margin_ac"] < AC_MARGIN)),
                share_draw=float(np.mean(orc_diag["margin_draw"] < DRAW_MARGIN)))
    for tol in (1e-6, 1e-7):   # how the exempt share and the mismatches shrink with the margin
        tight = (orc_diag["margin_ac"] < tol) | (orc_diag["margin_draw"] < tol)
        info[f"share_{tol:g}"] = float(np.mean(tight))
        info[f"diff_outside_{tol:g}"] = int((diff & ~tight).sum())
        tight_d = (orc_diag["margin_ac"] < AC_MARGIN) | (orc_diag["margin_draw"] < tol)
        info[f"share_draw_{tol:g}"] = float(np.mean(tight_d))
        info[f"diff_outside_draw_{tol:g}"] = int((diff & ~tight_d).sum())
    tight = (orc_diag["margin_ac"] < TIGHT_MARGIN) | (orc_diag["margin_draw"] < TIGHT_MARGIN)
    info["exempt_share_tight"] = float(np.mean(tight))
    info["diff_outside_tight"] = int((diff & ~tight).sum())
    print(f"parity {label}: {info}")
    assert bad == 0, info
    assert exempt_diff <= max(2, exempt // 10), info
    assert info["diff_outside_tight"] == 0, info
    return info
