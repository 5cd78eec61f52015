"""Pins of the oracle's colour transform (paper Section 4) and tree / BFS
numbering (Eq. 1, Section 3.4): exhaustive inversion, the closed form of the
lifting steps, hand-derived values, and BFS checked against networkx."""
import os

import networkx as nx
import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _all_rgb():
    v = np.arange(1 << 24, dtype=np.uint32)
    return np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], axis=-1).astype(np.uint8)


def test_ycocg_r_is_lossless_on_every_rgb_triple():
    rgb = _all_rgb()
    ycc = oracle.ycocg_fwd(rgb)
    back = oracle.ycocg_inv(ycc)
    assert np.array_equal(back, rgb.astype(np.int32))
    assert ycc[:, 0].min() == 0 and ycc[:, 0].max() == 255
    assert ycc[:, 1:].min() == -255 and ycc[:, 1:].max() == 255


def test_ycocg_r_closed_form():
    # the lifting steps collapse to Y = floor((G + floor((R+B)/2)) / 2),
    # Co = R - B, Cg = G - floor((R+B)/2)
    rgb = _all_rgb()[::7].astype(np.int64)
    r, g, b = rgb[:, 0], rgb[:, 1], rgb[:, 2]
    ycc = oracle.ycocg_fwd(rgb.astype(np.uint8)).astype(np.int64)
    half = np.floor_divide(r + b, 2)
    assert np.array_equal(ycc[:, 0], np.floor_divide(g + half, 2))
    assert np.array_equal(ycc[:, 1], r - b)
    assert np.array_equal(ycc[:, 2], g - half)


def test_ycocg_r_hand_values():
    for line in open(os.path.join(GOLDEN, "ycocg_examples.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        a, b = line.split("|")
        rgb = np.array([int(x) for x in a.split()], dtype=np.uint8)
        expect = [int(x) for x in b.split()]
        assert list(oracle.ycocg_fwd(rgb)) == expect
        assert list(oracle.ycocg_inv(np.array(expect))) == list(rgb)


@pytest.mark.parametrize("G", list(range(1, 41)))
def test_cluster_tiling_partitions_each_axis(G):
    for c in range(1, G + 3):
        k = oracle.tile_count(G, c)
        assert k == -(-G // c)
        t = oracle.tree_from_clusters(G, 1, 2, [0, c])
        # parent of node x along u is its tile; tiles contiguous, cover 0..G-1
        par = t["parent"][0]
        assert par == sorted(par) and set(par) == set(range(k))
        sizes = [par.count(a) for a in range(k)]
        assert max(sizes) <= c and max(sizes) - min(sizes) <= 1


def _nx_bfs(t):
    g = nx.DiGraph()
    L = t["L"]
    root = ("root", 0)
    for i in range(t["Gu"][L - 1] * t["Gv"][L - 1]):
        g.add_edge(root, (L - 1, i))
    for l in range(L - 1):
        for i, p in enumerate(t["parent"][l]):
            g.add_edge((l + 1, p), (l, i))
    order = [root] + [v for _, v in nx.bfs_edges(g, root, sort_neighbors=lambda ns: sorted(ns, key=lambda x: x[1]))]
    return [(l, i) for (l, i) in order if l != "root" and l < L - 1]


@pytest.mark.parametrize("U,V,L,c", [
    (5, 5, 2, [0, 5]), (9, 9, 3, [0, 3, 3]), (17, 17, 3, [0, 5, 4]),
    (15, 15, 3, [0, 3, 5]), (5, 5, 3, [0, 2, 3]), (7, 4, 4, [0, 2, 2, 2]),
    (6, 6, 3, [0, 2, 2]),
])
def test_bfs_numbering_matches_networkx(U, V, L, c):
    t = oracle.tree_from_clusters(U, V, L, c)
    ours = list(zip(t["bfs_level"], t["bfs_node"]))
    assert ours == _nx_bfs(t)
    assert t["S"] == len(ours)
    for p, (l, i) in enumerate(ours):
        assert t["pos_of"][l][i] == p


def test_bfs_hand_derived_plain_grid():
    line = [x for x in open(os.path.join(GOLDEN, "bfs_plain_9x9.txt")) if not x.startswith("#")][0]
    expect = [tuple(int(v) for v in tok.split(":")) for tok in line.split()]
    t = oracle.tree_from_clusters(9, 9, 3, [0, 3, 3])
    assert list(zip(t["bfs_level"], t["bfs_node"]))[: len(expect)] == expect
    assert t["Gu"] == [9, 3, 1] and t["S"] == 90 and t["n_top"] == 1


def test_preset_tree_shapes():
    assert oracle.tree_from_clusters(17, 17, 3, [0, 5, 4])["Gu"] == [17, 4, 1]
    assert oracle.tree_from_clusters(15, 15, 3, [0, 3, 5])["Gu"] == [15, 5, 1]
    assert oracle.tree_from_clusters(5, 5, 3, [0, 2, 3])["Gu"] == [5, 3, 1]
    assert oracle.tree_from_clusters(17, 17, 3, [0, 5, 4])["S"] == 289 + 16
