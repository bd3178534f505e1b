"""Pins of the oracle's cluster tree, block tree and admissibility (Sec. 2).

No test retypes the oracle's formulas: they check a hand-derived example,
set-partition invariants and brute-force geometric consequences.
"""
import json
import os

import numpy as np
import pytest

from oracle import h2_oracle as O
from workloads import sphere_points

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ptset(points, c):
    return sorted(float(x) for x in points[c.idx, 0])


def test_golden_tiny_line_tree_and_blocks():
    """Hand-derived tree and leaf-block partition (tests/golden/tiny_line_blocks.json)."""
    d = json.load(open(os.path.join(GOLDEN, "tiny_line_blocks.json")))
    pts = np.zeros((len(d["points_x"]), 3))
    pts[:, 0] = d["points_x"]
    root = O.build_cluster_tree(pts, d["leaf_size"])
    assert root.idx.tolist() == d["perm"]
    bt = O.build_block_tree(root, root, d["eta"])
    adm, near = O.leaf_blocks(bt)
    got_adm = sorted((_ptset(pts, b.t), _ptset(pts, b.s)) for b in adm)
    got_near = sorted((_ptset(pts, b.t), _ptset(pts, b.s)) for b in near)
    want_adm = sorted((sorted(map(float, a)), sorted(map(float, b))) for a, b in d["admissible"])
    want_near = sorted((sorted(map(float, a)), sorted(map(float, b))) for a, b in d["inadmissible"])
    assert got_adm == want_adm
    assert got_near == want_near


@pytest.mark.parametrize("n,leaf", [(1, 64), (64, 64), (65, 64), (3000, 64), (2000, 17)])
def test_cluster_tree_is_a_cluster_tree(n, leaf):
    """Def. "Cluster tree": root label = I, sons disjoint and covering; leaves small;
    labels are contiguous pre-order ranges; boxes are tight."""
    pts = sphere_points(n, 3)
    root = O.build_cluster_tree(pts, leaf)
    assert sorted(root.idx.tolist()) == list(range(n))
    for c in O.clusters_preorder(root):
        seg = root.idx[c.offset:c.offset + c.size]
        assert np.array_equal(seg, c.idx)
        assert np.array_equal(c.lo, pts[c.idx].min(0)) and np.array_equal(c.hi, pts[c.idx].max(0))
        if c.is_leaf:
            assert c.size <= leaf
        else:
            assert len(c.sons) == 2
            u = np.concatenate([s.idx for s in c.sons])
            assert sorted(u.tolist()) == sorted(c.idx.tolist())
            assert len(set(c.sons[0].idx.tolist()) & set(c.sons[1].idx.tolist())) == 0
            assert all(s.size > 0 and s.level == c.level + 1 for s in c.sons)


def test_block_leaves_partition_index_square():
    """Sec. 2: the leaves of the block tree form a disjoint partition of I×J."""
    pts = sphere_points(1500, 5)
    root = O.build_cluster_tree(pts, 32)
    adm, near = O.leaf_blocks(O.build_block_tree(root, root, 2.0))
    cover = np.zeros((1500, 1500), dtype=np.int32)
    for b in adm + near:
        cover[np.ix_(b.t.idx, b.s.idx)] += 1
    assert cover.min() == 1 and cover.max() == 1
    for b in near:  # inadmissible leaves are leaf x leaf by the stopping rule
        assert b.t.is_leaf and b.s.is_leaf


def test_admissible_blocks_are_geometrically_separated():
    """Brute force: for every admissible block the true point-set diameters and
    the true minimum distance satisfy the condition too (boxes over-estimate
    diameters and under-estimate distances)."""
    pts = sphere_points(1200, 11)
    root = O.build_cluster_tree(pts, 24)
    eta = 2.0
    adm, near = O.leaf_blocks(O.build_block_tree(root, root, eta))
    assert len(adm) > 50
    rng = np.random.default_rng(0)
    for b in [adm[i] for i in rng.choice(len(adm), 60, replace=False)]:
        P, Q = pts[b.t.idx], pts[b.s.idx]
        dmin = np.sqrt(((P[:, None, :] - Q[None, :, :]) ** 2).sum(-1)).min()
        dt = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)).max()
        ds = np.sqrt(((Q[:, None, :] - Q[None, :, :]) ** 2).sum(-1)).max()
        assert max(dt, ds) <= eta * dmin + 1e-15
        assert dmin > 0


def test_admissibility_boundaries():
    """dist = 0 is never admissible; touching boxes are not admissible; a tie is."""
    def box(lo, hi):
        c = O.Cluster(np.arange(1), np.array(lo, float), np.array(hi, float), 0, 0, None)
        return c
    a = box([0, 0, 0], [1, 0, 0])
    b = box([1, 0, 0], [2, 0, 0])
    assert O.dist(a, b) == 0.0 and not O.admissible(a, b, 10.0)
    c = box([3, 0, 0], [4, 0, 0])  # gap 2, diameters 1 -> 1 <= 0.5*2 tie
    assert O.admissible(a, c, 0.5) and not O.admissible(a, c, 0.49)
    p = box([0, 0, 0], [0, 0, 0])
    assert not O.admissible(p, p, 1.0)
    # 3-D distance between boxes separated along two axes: sqrt(3² + 4²) = 5
    d = box([4, 5, 0], [5, 6, 0])
    e = box([0, 0, 0], [1, 1, 0])
    assert O.dist(d, e) == 5.0 and O.dist(e, d) == 5.0
    assert O.diam(e) == pytest.approx(2 ** 0.5, rel=0, abs=1e-15)


def test_coincident_points_split_by_halving():
    """Coincident points cannot be split geometrically; the index range is halved."""
    pts = np.ones((300, 3)) * 0.25
    root = O.build_cluster_tree(pts, 64)
    leaves = [c for c in O.clusters_preorder(root) if c.is_leaf]
    assert all(c.size <= 64 for c in leaves)
    assert root.idx.tolist() == list(range(300))
    adm, near = O.leaf_blocks(O.build_block_tree(root, root, 2.0))
    assert len(adm) == 0 and len(near) == len(leaves) ** 2


def test_counts_sphere_4096_q3():
    """Sizes of the n=4096 sphere workload (sanity numbers recorded for the build)."""
    H = O.H2Matrix(sphere_points(4096, 0), q=3, leaf_size=64, eta=2.0, sigma=1e-2)
    c = H.counts()
    assert c["n_clusters"] == 195 and c["n_leaves"] == 98
    assert c["n_adm"] == 2130 and c["n_near"] == 1242 and c["nnz_near"] == 2232818
