"""Pins the oracle's Barnes-Hut partner search (Sec. III-B "Division of work";
criterion and the theta = 0 direct solution from Sec. II).

* theta = 0 must be the exact O(n^2) draw over all neurons (brute force below).
* hand-built layouts whose outcome probabilities have closed forms.
* chi-square of sampled targets against the exact outcome distribution.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2509_26193_gb300 import workloads


def _u(orc, seed, step, i, e, depth):
    w = orc.philox4x32_10([i, step & 0xFFFFFFFF, (e << 8) | depth, 0],
                          [seed & 0xFFFFFFFF, seed >> 32])[0]
    return int(w) / 2.0 ** 32


def test_theta_zero_is_brute_force(orc):
    net = workloads.uniform_cube(n=4096, seed=1)
    t = orc.Tree(net.x, net.y, net.z)
    t.reduce(net.vac_de)
    qi, qe = orc.queries(net.vac_ax)
    step = 7
    tgt, diag = t.search_batch(net.sigma, 0.0, net.seed, step, qi, qe)
    # brute force: every neuron in canonical (Morton code, id) order
    codes, _, _ = orc.morton(net.x, net.y, net.z)
    order = np.lexsort((np.arange(net.n), codes))
    P = np.stack([net.x, net.y, net.z], 1).astype(np.float64)[order]
    w = net.vac_de.astype(np.float64)[order]
    s2 = net.sigma ** 2
    mism = 0
    for q in range(len(qi)):
        i, e = int(qi[q]), int(qe[q])
        d2 = ((P - P[np.where(order == i)[0][0]]) ** 2).sum(1)
        a = w * np.exp(-d2 / s2)
        a[order == i] = 0.0
        C = np.cumsum(a)
        if C[-1] == 0:
            assert tgt[q] == -1
            continue
        u = _u(orc, net.seed, step, i, e, 0)
        k = int(np.searchsorted(C, u * C[-1], side="right"))
        want = int(order[k])
        if want != tgt[q]:
            assert diag["margin_draw"][q] < 1e-9
            mism += 1
        assert diag["restarts"][q] == 0
    assert mism <= 2
    assert len(qi) > 7000


def test_theta_zero_marginals_equal_kernel(orc):
    net = workloads.uniform_cube(n=300, seed=3)
    t = orc.Tree(net.x, net.y, net.z)
    t.reduce(net.vac_de)
    P = np.stack([net.x, net.y, net.z], 1).astype(np.float64)
    for i in (0, 17, 123):
        a = net.vac_de * np.exp(-((P - P[i]) ** 2).sum(1) / net.sigma ** 2)
        a[i] = 0
        p = t.marginals(net.sigma, 0.0, i)
        assert np.allclose(p[:-1], a / a.sum(), rtol=1e-12, atol=1e-15)


def test_two_neurons(orc):
    p = np.array([[0, 0, 0], [3, 4, 0]], np.float32)
    t = orc.Tree(p[:, 0], p[:, 1], p[:, 2])
    t.reduce(np.array([2, 5], np.int32))
    for step in range(20):
        for theta in (0.0, 0.3, 0.9):
            assert t.search(10.0, theta, 1, step, 0, 0)["target"] == 1
            assert t.search(10.0, theta, 1, step, 1, 3)["target"] == 0


def test_three_collinear_closed_form(orc):
    # box [0,4]^3: the source (0.5) and neuron 1 (1.5) share octant 0, neuron 2 (3.5)
    # is alone in octant 1. Source has no vacant dendrites (count 0).
    pts = np.array([[0.5, 0.5, 0.5], [1.5, 0.5, 0.5], [3.5, 0.5, 0.5]], np.float32)
    vac = np.array([0, 2, 3], np.int32)
    lo, hi = np.zeros(3, np.float32), np.full(3, 4, np.float32)
    t = orc.Tree(pts[:, 0], pts[:, 1], pts[:, 2], lo, hi)
    t.reduce(vac)
    sigma = 2.0
    a1 = 2 * math.exp(-1.0 / sigma ** 2)
    a2 = 3 * math.exp(-9.0 / sigma ** 2)
    for theta in (0.0, 0.3, 0.8):
        p = t.marginals(sigma, theta, 0)
        assert p[1] == pytest.approx(a1 / (a1 + a2), rel=1e-12)
        assert p[2] == pytest.approx(a2 / (a1 + a2), rel=1e-12)


def test_far_cluster_is_one_candidate(orc):
    # box [0,16]^3; source (no vacancies) and one near neuron in octant 0; a
    # 3-neuron cluster in octant 7, which is accepted as one node at theta = 0.5
    # (cell length 8 < 0.5 * distance ~ 24.6) and entered by a restart.
    pts = np.array([[0.5, 0.5, 0.5], [1.5, 0.5, 0.5],
                    [14.5, 14.5, 14.5], [15.5, 14.5, 14.5], [14.5, 15.5, 14.5]], np.float32)
    vac = np.array([0, 1, 1, 2, 1], np.int32)
    t = orc.Tree(pts[:, 0], pts[:, 1], pts[:, 2], np.zeros(3, np.float32),
                 np.full(3, 16, np.float32))
    t.reduce(vac)
    sigma = 20.0
    s2 = sigma ** 2
    x0 = pts[0].astype(np.float64)
    w = vac[2:].astype(np.float64)
    cen = (w[:, None] * pts[2:].astype(np.float64)).sum(0) / w.sum()
    a_near = 1.0 * math.exp(-1.0 / s2)
    a_cl = w.sum() * math.exp(-((x0 - cen) ** 2).sum() / s2)
    p_cl = a_cl / (a_near + a_cl)
    dj = ((pts[2:].astype(np.float64) - x0) ** 2).sum(1)
    inner = w * np.exp(-dj / s2)
    want = np.array([0.0, 1 - p_cl, *(p_cl * inner / inner.sum()), 0.0])
    got = t.marginals(sigma, 0.5, 0)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-15)
    # at theta = 0 the cluster members are individual candidates instead
    a = np.concatenate([[0.0, a_near], w * np.exp(-dj / s2)])
    got0 = t.marginals(sigma, 0.0, 0)
    assert np.allclose(got0[:-1], a / a.sum(), rtol=1e-12)
    # the sampler draws from that distribution: restarts happen for the cluster
    diags = [t.search(sigma, 0.5, 9, s, 0, 0) for s in range(3000)]
    tg = np.array([d["target"] for d in diags])
    assert all(d["restarts"] >= 1 for d in diags if d["target"] >= 2)
    assert all(d["restarts"] == 0 for d in diags if d["target"] == 1)
    obs = np.array([(tg == j).sum() for j in range(1, 5)])
    exp_ = 3000 * want[1:5]
    assert stats.chisquare(obs, exp_).pvalue > 1e-3


def test_chi_square_small_network(orc):
    net = workloads.uniform_cube(n=24, side=100.0, seed=4, sigma=60.0)
    vac = np.maximum(net.vac_de, 1)
    t = orc.Tree(net.x, net.y, net.z)
    t.reduce(vac)
    i = 5
    exact = t.marginals(net.sigma, 0.5, i)
    assert exact[i] == 0 and abs(exact.sum() - 1) < 1e-12
    ns = 20000
    # independent draws: the step index changes every Philox counter
    tg = np.array([t.search(net.sigma, 0.5, 77, s, i, 0)["target"] for s in range(ns)])
    obs = np.bincount(tg, minlength=net.n).astype(float)
    exp_ = ns * exact[:net.n]
    keep = exp_ >= 5
    obs_k, exp_k = obs[keep], exp_[keep]
    if exp_[~keep].sum() > 0:
        obs_k = np.append(obs_k, obs[~keep].sum())
        exp_k = np.append(exp_k, exp_[~keep].sum())
    assert stats.chisquare(obs_k, exp_k).pvalue > 1e-3


def test_approximation_vanishes_as_theta_goes_to_zero(orc):
    net = workloads.gaussian_clusters(n=200, clusters=4, side=1500, std=80, seed=6,
                                      sigma=300.0)
    vac = np.maximum(net.vac_de, 1)
    t = orc.Tree(net.x, net.y, net.z)
    t.reduce(vac)
    P = np.stack([net.x, net.y, net.z], 1).astype(np.float64)
    tv = {}
    for theta in (0.8, 0.5, 0.3, 0.1, 0.0):
        acc = 0.0
        for i in range(0, 200, 10):
            a = vac * np.exp(-((P - P[i]) ** 2).sum(1) / net.sigma ** 2)
            a[i] = 0
            acc += 0.5 * np.abs(t.marginals(net.sigma, theta, i)[:-1] - a / a.sum()).sum()
        tv[theta] = acc / 20
    assert tv[0.0] < 1e-12
    assert tv[0.1] < tv[0.8]
    assert tv[0.1] < 0.02


def test_zero_mass_fails(orc):
    net = workloads.uniform_cube(n=50, seed=8)
    t = orc.Tree(net.x, net.y, net.z)
    t.reduce(np.zeros(50, np.int32))
    assert t.search(net.sigma, 0.3, 1, 0, 3, 0)["target"] == -1
    only_self = np.zeros(50, np.int32)
    only_self[3] = 4
    t.reduce(only_self)
    assert t.search(net.sigma, 0.3, 1, 0, 3, 0)["target"] == -1
    assert t.search(net.sigma, 0.3, 1, 0, 4, 0)["target"] == 3


def test_far_source_does_not_underflow(orc):
    # neighbours ~ 60 sigma away: exp(-3600) underflows FP64 without the shift
    pts = np.array([[0, 0, 0], [6000, 0, 0], [6000, 10, 0]], np.float32)
    t = orc.Tree(pts[:, 0], pts[:, 1], pts[:, 2])
    t.reduce(np.array([1, 1, 1], np.int32))
    p = t.marginals(100.0, 0.0, 0)
    # relative weights exp(-(d_j^2 - d_min^2) / sigma^2): d_2^2 - d_1^2 = 100
    a = np.array([0.0, 1.0, math.exp(-100.0 / 1e4)])
    assert np.allclose(p[:3], a / a.sum(), rtol=1e-9)
    assert t.search(100.0, 0.3, 3, 0, 0, 0)["target"] in (1, 2)


@pytest.mark.parametrize("long_axis", [0, 1, 2])
def test_cell_length_is_longest_edge(orc, long_axis):
    """Reading R2 (Sec. II criterion, Sec. III-B cells): in an anisotropic box the cell
    "length" is the longest edge of the cell. Box 4 x 16 x 4 (long axis rotated through
    x, y, z). A source with no vacancies and one near neuron sit in the first depth-1
    cell (2 x 8 x 2); a three-neuron cluster sits alone in a second one, each member
    alone in its own depth-2 cell. The cluster cell's centroid is at distance d from
    the source; theta is chosen so that theta * d falls between two edge readings:
      theta = 0.4:  theta d = 5.20: longest edge 8 rejects (members drawn one by one);
                    the short edges (2), the cube root of the volume (3.17) accept;
      theta = 0.63: theta d = 8.20: longest edge 8 accepts (one candidate, then a
                    restart inside the cluster); the cell diagonal (8.49) rejects.
    Closed-form marginals, written out per case."""
    def put(p):   # (short, long, short) -> long axis at long_axis
        p = np.asarray(p, np.float64)
        out = np.empty_like(p)
        short = [a for a in range(3) if a != long_axis]
        out[:, long_axis] = p[:, 1]
        out[:, short[0]] = p[:, 0]
        out[:, short[1]] = p[:, 2]
        return out
    base = np.array([[0.5, 0.5, 0.5],     # source (no vacant dendritic elements)
                     [0.5, 1.5, 0.5],     # near neuron
                     [0.5, 14.5, 0.5],    # cluster member c1
                     [1.5, 14.5, 0.5],    # c2
                     [0.5, 10.5, 0.5]])   # c3
    pts = put(base).astype(np.float32)
    lo = np.zeros(3, np.float32)
    hi = put([[4.0, 16.0, 4.0]])[0].astype(np.float32)
    vac = np.array([0, 1, 1, 2, 1], np.int32)
    t = orc.Tree(pts[:, 0], pts[:, 1], pts[:, 2], lo, hi)
    t.reduce(vac)
    sigma = 10.0
    s2 = sigma ** 2
    x0 = base[0]
    d2 = ((base - x0) ** 2).sum(1)             # 0, 1, 196, 197, 100
    w = vac[2:].astype(np.float64)
    cen = (w[:, None] * base[2:]).sum(0) / w.sum()   # (1.0, 13.5, 0.5)
    dc = math.sqrt(((cen - x0) ** 2).sum())    # 13.0096...
    assert 8.0 < 0.63 * dc < math.sqrt(2 * 2 + 8 * 8 + 2 * 2)
    assert (2 * 8 * 2) ** (1 / 3) < 0.4 * dc < 8.0
    a_near = math.exp(-d2[1] / s2)
    a_mem = w * np.exp(-d2[2:] / s2)
    # theta = 0.4: every member is a candidate of the root frontier
    want = np.array([0.0, a_near, *a_mem]) / (a_near + a_mem.sum())
    got = t.marginals(sigma, 0.4, 0)
    assert np.allclose(got[:5], want, rtol=1e-12, atol=1e-15)
    # theta = 0.63: the cluster cell is one candidate (count 4 at its centroid)
    a_cl = w.sum() * math.exp(-dc ** 2 / s2)
    p_cl = a_cl / (a_near + a_cl)
    want = np.array([0.0, 1 - p_cl, *(p_cl * a_mem / a_mem.sum())])
    got = t.marginals(sigma, 0.63, 0)
    assert np.allclose(got[:5], want, rtol=1e-12, atol=1e-15)
