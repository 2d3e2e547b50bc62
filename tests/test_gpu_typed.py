"""Typed dendrite pools on the GPU (excitatory axons search excitatory dendritic
elements, inhibitory axons inhibitory ones), through the C ABI.

* the typed entry point equals two explicit plain updates, one per pool, each on the
  axons of that pool's type, bit for bit (store, vacancies, requests);
* against the oracle: each pool's requests within the search exemption, acceptance and
  apply replayed on the GPU's requests bit-exact, the final store and vacancies equal.
"""
import numpy as np
import pytest

import oracle
from gpu_common import GpuNet, check_targets, dev
from paper_2509_26193_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_26193_gb300 import build
    build.build()
    oracle.build()


def _typed_net(n=40000, seed=71):
    net = workloads.gaussian_clusters(n=n, clusters=6, side=3000, std=180, seed=seed,
                                      sigma=350.0)
    de_inh = np.random.default_rng(seed).integers(0, 4, n).astype(np.int32)
    return net, de_inh


def _typed_update(g, de_inh, step, group=0):
    R = g.R
    p = R.params(g.net.sigma, g.net.theta, g.net.seed, step, R.FLAG_DIAG, group)
    return R.relearn_update_connectivity_typed(g.ctx, p, g.vac_ax, g.vac_de, de_inh, g.type,
                                               stats=True)


@pytest.mark.parametrize("group", [0, 2])
def test_typed_equals_two_masked_plain_updates(group):
    import torch
    from paper_2509_26193_gb300 import relearn as R
    net, de_inh = _typed_net()
    g1, g2 = GpuNet(net), GpuNet(net)
    vi1, vi2 = dev(de_inh), dev(de_inh)
    for step in (0, 1):
        s1 = _typed_update(g1, vi1, step, group)
        t1, a1 = g1.requests()
        # the same two passes spelled out with the plain entry point
        p = R.params(net.sigma, net.theta, net.seed, step, R.FLAG_DIAG, group)
        formed = 0
        for kind, pool in ((0, g2.vac_de), (1, vi2)):
            va = torch.where(g2.type == kind, g2.vac_ax, torch.zeros_like(g2.vac_ax))
            s = R.relearn_update_connectivity(g2.ctx, p, va, pool, g2.type, stats=True)
            formed += s["formed"]
            g2.vac_ax.copy_(torch.where(g2.type == kind, va, g2.vac_ax))
        t2, a2 = g2.requests()
        assert s1["formed"] == formed > 0
        assert np.array_equal(t1, t2) and np.array_equal(a1, a2)
        assert np.array_equal(np.stack(g1.synapses()), np.stack(g2.synapses()))
        assert torch.equal(g1.vac_ax, g2.vac_ax) and torch.equal(g1.vac_de, g2.vac_de)
        assert torch.equal(vi1, vi2)
    g1.close()
    g2.close()


def test_typed_matches_oracle_replay():
    import torch
    from paper_2509_26193_gb300 import relearn as R
    net, de_inh = _typed_net(seed=72)
    g = GpuNet(net)
    # a second context runs the excitatory pass alone, to read its requests
    ge = GpuNet(net)
    vi = dev(de_inh)
    step = 3
    stats = _typed_update(g, vi, step)
    p = R.params(net.sigma, net.theta, net.seed, step, R.FLAG_DIAG)
    va_e = torch.where(ge.type == 0, ge.vac_ax, torch.zeros_like(ge.vac_ax))
    R.relearn_update_connectivity(ge.ctx, p, va_e, ge.vac_de, ge.type)
    gt_e, _ = ge.requests()
    gt_i, gacc_i = g.requests()

    t = oracle.Tree(net.x, net.y, net.z)
    va, ve, vi_o = net.vac_ax.copy(), net.vac_de.copy(), de_inh.copy()
    syn = oracle.Synapses(4 * int(va.sum()) + 16)
    searches = declined = formed = 0
    for kind, pool, gt in ((0, ve, gt_e), (1, vi_o, gt_i)):
        part = np.where(net.type == kind, va, 0).astype(np.int32)
        t.reduce(pool)
        qi, qe = oracle.queries(part)
        ot, od = t.search_batch(net.sigma, net.theta, net.seed, step, qi, qe, threads=8)
        assert len(gt) == len(qi) > 0
        check_targets(gt, ot, od, f"typed pool {kind}")
        assert np.all(pool[gt[gt >= 0]] > 0)
        # acceptance and apply replayed on the GPU's requests
        oacc = oracle.accept(net.n, qi, qe, gt, pool, net.seed, step)
        if kind == 1:
            assert np.array_equal(gacc_i, oacc)
        searches += len(qi)
        declined += int(((gt >= 0) & (oacc == 0)).sum())
        formed += oracle.apply(qi, gt, oacc, net.type, part, pool, syn)
        va[net.type == kind] = part[net.type == kind]
    assert stats["searches"] == searches
    assert stats["requests_declined"] == declined
    assert stats["formed"] == formed
    assert np.array_equal(g.vac_ax.cpu().numpy(), va)
    assert np.array_equal(g.vac_de.cpu().numpy(), ve)
    assert np.array_equal(vi.cpu().numpy(), vi_o)
    s, d, sg = g.synapses()
    assert np.array_equal(np.stack([s, d, sg]), np.stack(syn.arrays()))
    # signs follow the source type; each pool received only its own type's synapses
    assert np.array_equal(sg, np.where(net.type[s] == 1, -1, 1))
    g.close()
    ge.close()


def test_typed_rejects_aliased_pools():
    from paper_2509_26193_gb300 import relearn as R
    net, _ = _typed_net(n=2000)
    g = GpuNet(net)
    p = R.params(net.sigma, net.theta, net.seed, 0)
    with pytest.raises(R.RelearnError):
        R.relearn_update_connectivity_typed(g.ctx, p, g.vac_ax, g.vac_de, g.vac_de, g.type)
    g.close()
