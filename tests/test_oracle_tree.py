"""Pins the oracle's octree build and bottom-up update (Sec. III-B, "Spatial
octree" and "Division of work") against hand-built layouts and direct sums."""
import numpy as np
import pytest

from paper_2509_26193_gb300 import workloads


def _tree(orc, pts, vac=None, lo=None, hi=None):
    p = np.asarray(pts, np.float32)
    t = orc.Tree(p[:, 0], p[:, 1], p[:, 2], lo, hi)
    t.reduce(np.ones(len(p), np.int32) if vac is None else np.asarray(vac, np.int32))
    return t


def test_two_points_opposite_corners(orc):
    t = _tree(orc, [(0, 0, 0), (1, 1, 1)])
    e = t.export()
    assert list(e["depth"]) == [0, 1, 1]
    assert list(e["is_leaf"]) == [0, 1, 1]
    assert list(e["neuron"]) == [-1, 0, 1]


def test_chain_and_compression(orc):
    # both points in octant 0 of octant 0; they first differ at depth 3 (x bit 7)
    box = ([0, 0, 0], [8, 8, 8])
    t = _tree(orc, [(0.1, 0.1, 0.1), (1.1, 0.1, 0.1)], None, *box)
    full = t.export()
    assert list(full["depth"]) == [0, 1, 2, 3, 3]
    comp = t.export(compressed=True)
    assert list(comp["depth"]) == [0, 2, 3, 3]   # root kept, chain collapses to its bottom
    assert list(comp["is_leaf"]) == [0, 0, 1, 1]


def test_coincident_points_make_a_bucket(orc):
    pts = [(5, 5, 5), (0, 0, 0), (5, 5, 5), (5, 5, 5), (9, 9, 9)]
    t = _tree(orc, pts)
    e = t.export()
    bucket = np.where(e["depth"] == 10)[0]
    assert len(bucket) == 1
    b = bucket[0]
    assert e["size"][b] == 3 and not e["is_leaf"][b]
    # children of the bucket: its neurons, in id order, at depth 11
    kids = np.where(e["depth"] == 11)[0]
    assert list(e["neuron"][kids]) == [0, 2, 3]
    assert all(e["is_leaf"][kids])


def _check_structure(orc, net, tree, vac):
    """Structural invariants + counts/centroids by direct FP64 sums over ranges."""
    codes, _, _ = orc.morton(net.x, net.y, net.z)
    order = np.lexsort((np.arange(net.n), codes))
    perm = tree.canonical_order()
    assert np.array_equal(perm, order)           # canonical = (code, id) order
    e = tree.export()
    m = len(e["depth"])
    leaf = e["is_leaf"].astype(bool)
    assert np.all(e["size"][leaf] == 1)          # leaves hold one neuron
    assert np.array_equal(np.sort(e["neuron"][leaf]), np.arange(net.n))
    px, py, pz = (a.astype(np.float64)[perm] for a in (net.x, net.y, net.z))
    w = vac.astype(np.float64)[perm]
    cw = np.concatenate([[0], np.cumsum(w)])
    sc = codes[perm]
    for k in range(m):
        f, s, d = e["first"][k], e["size"][k], e["depth"][k]
        assert e["count"][k] == cw[f + s] - cw[f]
        if not leaf[k]:
            # every neuron of a cell shares its top-d octal digits, and the cell
            # is maximal: the neurons just outside differ there
            if d <= 10:
                sh = 3 * (10 - d)
                pre = sc[f:f + s] >> sh
                assert np.all(pre == pre[0])
                if f > 0:
                    assert (sc[f - 1] >> sh) != pre[0] or d == 0
                if f + s < net.n:
                    assert (sc[f + s] >> sh) != pre[0] or d == 0
        if e["count"][k] > 0:
            ww = w[f:f + s]
            c = np.array([np.dot(ww, px[f:f + s]), np.dot(ww, py[f:f + s]),
                          np.dot(ww, pz[f:f + s])]) / ww.sum()
            got = np.array([e["cx"][k], e["cy"][k], e["cz"][k]])
            assert np.allclose(got, c, rtol=1e-12, atol=0)
        else:
            assert np.isnan(e["cx"][k])
    # pre-order: ranges are nested or disjoint, children partition the parent
    assert e["first"][0] == 0 and e["size"][0] == net.n


@pytest.mark.parametrize("gen", ["cube", "clusters", "slab"])
def test_structure_and_direct_sums(orc, gen):
    if gen == "cube":
        net = workloads.uniform_cube(n=700, seed=11)
    elif gen == "clusters":
        net = workloads.gaussian_clusters(n=900, clusters=5, side=2000, std=60, seed=12)
    else:
        net = workloads.cortical_slab(n=800, sx=500, sy=500, sz=60, seed=13)
    t = orc.Tree(net.x, net.y, net.z)
    t.reduce(net.vac_de)
    _check_structure(orc, net, t, net.vac_de)


def test_root_is_weighted_mean(orc):
    net = workloads.gaussian_clusters(n=2000, clusters=3, side=1000, std=100, seed=5)
    t = orc.Tree(net.x, net.y, net.z)
    t.reduce(net.vac_de)
    e = t.export()
    w = net.vac_de.astype(np.float64)
    assert e["count"][0] == w.sum()
    for a, key in zip((net.x, net.y, net.z), ("cx", "cy", "cz")):
        assert e[key][0] == pytest.approx(np.dot(w, a.astype(np.float64)) / w.sum(), rel=1e-13)


def test_every_multi_neuron_cell_is_subdivided(orc):
    net = workloads.uniform_cube(n=500, seed=21)
    t = orc.Tree(net.x, net.y, net.z)
    e = t.export()
    for k in range(len(e["depth"])):
        if e["size"][k] >= 2:
            assert not e["is_leaf"][k]
    # uncompressed node count >= compressed; compressed inner nodes <= n - 1 (+ root)
    c = t.export(compressed=True)
    assert len(c["depth"]) <= len(e["depth"])
    assert (c["is_leaf"] == 0).sum() <= net.n


def test_single_neuron_and_zero_counts(orc):
    t = _tree(orc, [(1, 2, 3)], [0])
    e = t.export()
    assert list(e["is_leaf"]) == [1] and np.isnan(e["cx"][0])
