"""Pins the oracle's typed-dendrite variant (reading R16: excitatory axons search
vacant excitatory dendritic elements, inhibitory axons inhibitory ones).

* a three-neuron layout whose outcome has a closed form in the searching axon's
  own pool (the other pool's counts must not matter);
* pool bookkeeping: every synapse lands in the pool of its source's type, and each
  pool's vacancies drop by exactly the synapses formed onto it;
* a network without inhibitory neurons is the plain update on the excitatory pool.
"""
import math

import numpy as np

from paper_2509_26193_gb300 import workloads


def _u(orc, seed, step, i, e, depth):
    w = orc.philox4x32_10([i, step & 0xFFFFFFFF, (e << 8) | depth, 0],
                          [seed & 0xFFFFFFFF, seed >> 32])[0]
    return int(w) / 2.0 ** 32


def test_search_uses_the_axons_own_pool(orc):
    # A (origin) searches; B 100 um along x, C 50 um along y (three root octants).
    x = np.array([0.0, 100.0, 0.0], np.float32)
    y = np.array([0.0, 0.0, 50.0], np.float32)
    z = np.zeros(3, np.float32)
    exc = np.array([0, 1, 2], np.int32)       # A's excitatory axons see B:1, C:2
    inh = np.array([0, 5, 0], np.int32)       # an inhibitory axon would only see B
    seed, step = 13, 2
    for kind, pool in ((0, exc), (1, inh)):
        t = orc.Tree(x, y, z)
        va = np.array([40, 0, 0], np.int32)
        ve, vi = exc.copy(), inh.copy()
        typ = np.array([kind, 0, 0], np.uint8)
        syn = orc.Synapses(64)
        r = orc.update_connectivity_typed(t, va, ve, vi, typ, 100.0, 0.0, seed, step, syn)
        got = r["exc" if kind == 0 else "inh"]["tgt"]
        a_b, a_c = pool[1] * math.exp(-1.0), pool[2] * math.exp(-0.25)
        want = [1 if _u(orc, seed, step, 0, e, 0) * (a_b + a_c) < a_b else 2 for e in range(40)]
        assert got.tolist() == want
        t.close()


def _typed_net(n=3000, seed=41):
    net = workloads.gaussian_clusters(n=n, clusters=4, side=2000, std=150, seed=seed,
                                      sigma=300.0)
    rng = np.random.default_rng(seed)
    return net, rng.integers(0, 4, n).astype(np.int32)


def test_pool_bookkeeping(orc):
    net, de_inh = _typed_net()
    t = orc.Tree(net.x, net.y, net.z)
    va, ve, vi = net.vac_ax.copy(), net.vac_de.copy(), de_inh.copy()
    syn = orc.Synapses(int(va.sum()) + 16)
    r = orc.update_connectivity_typed(t, va, ve, vi, net.type, net.sigma, net.theta, net.seed,
                                      1, syn)
    s, d, sg = syn.arrays()
    assert len(s) == r["exc"]["formed"] + r["inh"]["formed"] > 0
    assert np.all(s != d)
    assert np.array_equal(sg, np.where(net.type[s] == 1, -1, 1))
    n = net.n
    assert np.array_equal(net.vac_ax - va, np.bincount(s, minlength=n))
    assert np.array_equal(net.vac_de - ve, np.bincount(d[sg > 0], minlength=n))
    assert np.array_equal(de_inh - vi, np.bincount(d[sg < 0], minlength=n))
    assert np.all(va >= 0) and np.all(ve >= 0) and np.all(vi >= 0)
    # every request of a pool targets a neuron with vacancies in that pool
    for name, pool in (("exc", net.vac_de), ("inh", de_inh)):
        tg = r[name]["tgt"]
        assert np.all(pool[tg[tg >= 0]] > 0)
        assert np.all(net.type[r[name]["src"]] == (0 if name == "exc" else 1))


def test_excitatory_only_is_the_plain_update(orc):
    net, de_inh = _typed_net(seed=42)
    net.type[:] = 0
    t1 = orc.Tree(net.x, net.y, net.z)
    va1, vd1 = net.vac_ax.copy(), net.vac_de.copy()
    syn1 = orc.Synapses(int(va1.sum()) + 16)
    r1 = orc.update_connectivity(t1, va1, vd1, net.type, net.sigma, net.theta, net.seed, 4, syn1)
    t2 = orc.Tree(net.x, net.y, net.z)
    va2, ve2, vi2 = net.vac_ax.copy(), net.vac_de.copy(), de_inh.copy()
    syn2 = orc.Synapses(int(va2.sum()) + 16)
    r2 = orc.update_connectivity_typed(t2, va2, ve2, vi2, net.type, net.sigma, net.theta,
                                       net.seed, 4, syn2)
    assert np.array_equal(r1["tgt"], r2["exc"]["tgt"]) and len(r2["inh"]["tgt"]) == 0
    assert np.array_equal(va1, va2) and np.array_equal(vd1, ve2)
    assert np.array_equal(vi2, de_inh)
    for a, b in zip(syn1.arrays(), syn2.arrays()):
        assert np.array_equal(a, b)
