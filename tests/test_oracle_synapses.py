"""Pins the oracle's acceptance, apply, deletion and spike delivery
(Sec. III-A "Update of synapses" and "Update of electrical activity")."""
import numpy as np
import pytest
from scipy import sparse, stats

from paper_2509_26193_gb300 import workloads


# ------------------------------------------------------------------ acceptance
def test_accept_rule_small(orc):
    # target 0: 3 requests, 1 vacancy; target 1: 2 requests, 5 vacancies; target 2: none
    src = np.array([4, 5, 6, 7, 8, 9], np.int32)
    elem = np.array([0, 0, 1, 0, 2, 0], np.int32)
    tgt = np.array([0, 0, 0, 1, 1, -1], np.int32)
    vac_de = np.array([1, 5, 3, 0, 0, 0, 0, 0, 0, 0], np.int32)
    acc = orc.accept(10, src, elem, tgt, vac_de, seed=3, step=2)
    assert list(acc[3:]) == [1, 1, 0]
    pr = [orc.request_priority(3, 2, int(s), int(e)) for s, e in zip(src[:3], elem[:3])]
    assert list(acc[:3]) == [1 if k == int(np.argmin(pr)) else 0 for k in range(3)]


def test_accept_is_uniform_over_requests(orc):
    # four requests compete for one vacancy: each wins with probability 1/4
    src = np.array([1, 2, 3, 4], np.int32)
    elem = np.zeros(4, np.int32)
    tgt = np.zeros(4, np.int32)
    vac = np.array([1, 0, 0, 0, 0], np.int32)
    wins = np.zeros(4)
    for step in range(4000):
        wins += orc.accept(5, src, elem, tgt, vac, seed=11, step=step)
    assert wins.sum() == 4000
    assert stats.chisquare(wins, np.full(4, 1000.0)).pvalue > 1e-3


def test_update_invariants(orc):
    net = workloads.gaussian_clusters(n=3000, clusters=6, side=3000, std=150, seed=31,
                                      sigma=200.0)
    t = orc.Tree(net.x, net.y, net.z)
    syn = orc.Synapses(10 * net.n)
    vac_ax, vac_de = net.vac_ax.copy(), net.vac_de.copy()
    for step in range(4):
        ax0, de0, m0 = vac_ax.copy(), vac_de.copy(), syn.count
        r = orc.update_connectivity(t, vac_ax, vac_de, net.type, net.sigma, net.theta,
                                    net.seed, step, syn)
        tg, acc = r["tgt"], r["accept"].astype(bool)
        # every vacant axonal element searched once; accepted <= vacancies per target
        assert len(tg) == ax0.sum()
        per_t = np.bincount(tg[acc], minlength=net.n)
        req_t = np.bincount(tg[tg >= 0], minlength=net.n)
        assert np.array_equal(per_t, np.minimum(req_t, de0))
        # conservation: formed = lost axonal vacancies = lost dendritic vacancies
        assert r["formed"] == acc.sum() == (ax0 - vac_ax).sum() == (de0 - vac_de).sum()
        assert syn.count - m0 == r["formed"]
        assert vac_ax.min() >= 0 and vac_de.min() >= 0
        s, d, g = syn.arrays()
        assert np.all(s != d)                               # no autapse (theta < 0.577)
        assert np.all(np.diff(s.astype(np.int64) * net.n + d) >= 0)   # canonical order
        assert np.array_equal(g, np.where(net.type[s] == 1, -1, 1))
        # out-degree of each neuron = axonal elements it has bound so far
        assert np.array_equal(np.bincount(s, minlength=net.n), net.vac_ax - vac_ax)
        assert np.array_equal(np.bincount(d, minlength=net.n), net.vac_de - vac_de)


# -------------------------------------------------------------------- deletion
def _store(orc, pairs, n, types=None):
    src = np.array([p[0] for p in pairs], np.int32)
    tgt = np.array([p[1] for p in pairs], np.int32)
    sign = np.ones(len(pairs), np.int8) if types is None else np.where(types[src], -1, 1)
    return orc.Synapses(len(pairs) + 4, src, tgt, sign.astype(np.int8))


def test_delete_vacant_first(orc):
    syn = _store(orc, [(0, 1), (0, 2)], 3)
    vac_ax = np.array([3, 0, 0], np.int32)
    vac_de = np.array([0, 0, 0], np.int32)
    broken = orc.delete(np.array([2, 0, 0], np.int32), np.zeros(3, np.int32), vac_ax, vac_de,
                        1, 0, syn)
    assert broken == 0 and list(vac_ax) == [1, 0, 0] and syn.count == 2


def test_delete_bound_returns_partner_vacancy(orc):
    syn = _store(orc, [(0, 1), (0, 2), (0, 3)], 4)
    vac_ax = np.array([1, 0, 0, 0], np.int32)
    vac_de = np.zeros(4, np.int32)
    broken = orc.delete(np.array([2, 0, 0, 0], np.int32), np.zeros(4, np.int32), vac_ax,
                        vac_de, 5, 0, syn)
    assert broken == 1 and vac_ax[0] == 0 and vac_de.sum() == 1
    s, d, _ = syn.arrays()
    lost = ({1, 2, 3} - set(d.tolist())).pop()
    assert vac_de[lost] == 1


def test_delete_mutual_pick_returns_nothing(orc):
    syn = _store(orc, [(0, 1)], 2)
    vac_ax = np.zeros(2, np.int32)
    vac_de = np.zeros(2, np.int32)
    broken = orc.delete(np.array([1, 0], np.int32), np.array([0, 1], np.int32), vac_ax, vac_de,
                        5, 0, syn)
    assert broken == 1 and syn.count == 0
    assert vac_ax.sum() == 0 and vac_de.sum() == 0


def test_delete_one_sided_dendrite(orc):
    syn = _store(orc, [(0, 2), (1, 2)], 3)
    vac_ax = np.zeros(3, np.int32)
    vac_de = np.zeros(3, np.int32)
    broken = orc.delete(np.zeros(3, np.int32), np.array([0, 0, 1], np.int32), vac_ax, vac_de,
                        5, 0, syn)
    assert broken == 1 and syn.count == 1
    s, _, _ = syn.arrays()
    assert vac_ax[1 - s[0]] == 1 and vac_ax.sum() == 1


def test_delete_is_uniform(orc):
    wins = np.zeros(4)
    for step in range(4000):
        syn = _store(orc, [(0, 1), (0, 2), (0, 3), (0, 4)], 5)
        vac_ax = np.zeros(5, np.int32)
        vac_de = np.zeros(5, np.int32)
        orc.delete(np.array([1, 0, 0, 0, 0], np.int32), np.zeros(5, np.int32), vac_ax, vac_de,
                   13, step, syn)
        wins += vac_de[1:]
    assert stats.chisquare(wins, np.full(4, 1000.0)).pvalue > 1e-3


def test_delete_element_conservation(orc):
    rng = np.random.default_rng(4)
    n = 400
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, n, (3000, 2)) if a != b]
    syn = _store(orc, pairs, n)
    s, d, _ = syn.arrays()
    vac_ax = rng.integers(0, 3, n).astype(np.int32)
    vac_de = rng.integers(0, 3, n).astype(np.int32)
    tot_ax = vac_ax + np.bincount(s, minlength=n)
    tot_de = vac_de + np.bincount(d, minlength=n)
    ra = rng.integers(0, 6, n).astype(np.int32)
    rd = rng.integers(0, 6, n).astype(np.int32)
    orc.delete(ra, rd, vac_ax, vac_de, 21, 3, syn)
    s2, d2, _ = syn.arrays()
    # each neuron loses exactly min(retraction, total) elements per side; partner
    # breaks only move an element from bound to vacant
    assert np.array_equal(vac_ax + np.bincount(s2, minlength=n), tot_ax - np.minimum(ra, tot_ax))
    assert np.array_equal(vac_de + np.bincount(d2, minlength=n), tot_de - np.minimum(rd, tot_de))
    assert vac_ax.min() >= 0 and vac_de.min() >= 0
    assert np.all(np.diff(s2.astype(np.int64) * n + d2) >= 0)


# ----------------------------------------------------------------------- spikes
def test_spike_delivery_is_signed_adjacency_product(orc):
    rng = np.random.default_rng(9)
    n = 500
    types = (rng.random(n) < 0.2).astype(np.uint8)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, n, (4000, 2))]
    syn = _store(orc, pairs, n, types)
    spiked = (rng.random(n) < 0.1).astype(np.uint8)
    got = orc.deliver_spikes(n, syn, spiked)
    s, d, g = syn.arrays()
    A = sparse.coo_matrix((g.astype(np.int64), (d, s)), shape=(n, n)).tocsr()
    assert np.array_equal(got, A @ spiked.astype(np.int64))


# --------------------------------------------------- firing-rate delivery
def test_rate_delivery_extremes_equal_spike_delivery(orc):
    # rate 1 = always spiked, rate 0 = never: exactly the spike delivery of those flags
    rng = np.random.default_rng(12)
    n = 300
    types = (rng.random(n) < 0.2).astype(np.uint8)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, n, (3000, 2))]
    syn = _store(orc, pairs, n, types)
    spiked = (rng.random(n) < 0.3).astype(np.uint8)
    rate = spiked.astype(np.float32)
    for step in range(3):
        assert np.array_equal(orc.deliver_rates(n, syn, rate, 5, step),
                              orc.deliver_spikes(n, syn, spiked))


def test_rate_delivery_mean_is_expected_input(orc):
    # E[input[t]] = sum over synapses s -> t of sign * rate[s]
    rng = np.random.default_rng(13)
    n = 50
    types = (rng.random(n) < 0.3).astype(np.uint8)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, n, (400, 2))]
    syn = _store(orc, pairs, n, types)
    rate = rng.uniform(0.0, 0.6, n).astype(np.float32)
    steps = 4000
    acc = np.zeros(n)
    for step in range(steps):
        acc += orc.deliver_rates(n, syn, rate, 9, step)
    s, d, g = syn.arrays()
    want = np.zeros(n)
    np.add.at(want, d, g * rate[s].astype(np.float64))
    var = np.zeros(n)
    np.add.at(var, d, (rate[s] * (1 - rate[s])).astype(np.float64))
    # duplicates of one (s, t) pair share the draw: bound their covariance generously
    sd = np.sqrt(np.maximum(var, 1e-9) * 4 / steps)
    assert np.all(np.abs(acc / steps - want) < 5 * sd + 1e-9)
