"""Pins for the oracle's mesh builder: brute force, closed forms, invariants."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2307_16758_gb300 import workloads as W


def _brute_adjacency(tris):
    """O(n^2) search: the cell sharing each (unordered) edge."""
    n = len(tris)
    nbr = -np.ones((n, 3), np.int64)
    for i in range(n):
        for k in range(3):
            e = {tris[i][k], tris[i][(k + 1) % 3]}
            for j in range(n):
                if j != i and e <= set(tris[j]):
                    nbr[i, k] = j
    return nbr


def test_adjacency_matches_brute_force():
    nodes, tris, bnd, side = W.structured(7, 5, 7.0, 5.0, jitter=0.3, seed=3)
    m = oracle.Mesh(nodes, tris)
    a = m.arrays
    brute = _brute_adjacency(a["tri"].tolist())
    assert np.array_equal(a["nbr"], brute)
    # neighbour relation is symmetric and the shared edge is walked both ways
    for i, k in itertools.product(range(m.n), range(3)):
        j = a["nbr"][i, k]
        if j < 0:
            continue
        kj = a["nbr_edge"][i, k]
        assert a["nbr"][j, kj] == i
        # opposite outward normals, bit for bit
        assert a["lnx"][j, kj] == -a["lnx"][i, k] and a["lny"][j, kj] == -a["lny"][i, k]


def test_counts_structured():
    nx, ny = 9, 4
    nodes, tris, bnd, side = W.structured(nx, ny, 9.0, 4.0)
    m = oracle.Mesh(nodes, tris, bnd, np.zeros(len(bnd)))
    a = m.arrays
    assert m.n == 2 * nx * ny
    assert (a["nbr"] < 0).sum() == 2 * (nx + ny)
    assert (a["btag"][a["nbr"] < 0] == 0).all()
    assert (a["btag"][a["nbr"] >= 0] == -1).all()


def test_geometry_closed_forms():
    # right isosceles triangle with unit legs, given clockwise
    nodes = np.array([[0.0, 0.0], [0.0, 1.0], [1.0, 0.0]])
    m = oracle.Mesh(nodes, np.array([[0, 1, 2]]))
    a = m.arrays
    assert a["area"][0] == 0.5
    assert math.isclose(a["rin"][0], (2.0 - math.sqrt(2.0)) / 2.0, rel_tol=1e-15)
    assert math.isclose(a["cx"][0], 1.0 / 3.0, rel_tol=1e-15)
    # re-oriented counter-clockwise: outward normals point away from the centroid
    t = a["tri"][0]
    assert list(t) == [0, 2, 1]
    for k in range(3):
        p, q = nodes[t[k]], nodes[t[(k + 1) % 3]]
        mid = 0.5 * (p + q)
        out = np.array([a["lnx"][0, k], a["lny"][0, k]])
        assert np.dot(out, mid - [a["cx"][0], a["cy"][0]]) > 0
        assert math.isclose(np.linalg.norm(out), np.linalg.norm(q - p), rel_tol=1e-15)


def test_normals_close_each_triangle():
    nodes, tris, bnd, side = W.structured(12, 9, 3.0, 2.0, jitter=0.3, seed=11)
    a = oracle.Mesh(nodes, tris).arrays
    assert np.abs(a["lnx"].sum(axis=1)).max() < 1e-15
    assert np.abs(a["lny"].sum(axis=1)).max() < 1e-15
    assert (a["area"] > 0).all()
    # area from the divergence theorem: 1/2 sum_k (x_mid . Ln_k)
    p = nodes[a["tri"]]
    mid = 0.5 * (p + np.roll(p, -1, axis=1))
    a2 = 0.5 * (mid[:, :, 0] * a["lnx"] + mid[:, :, 1] * a["lny"]).sum(axis=1)
    assert np.allclose(a2, a["area"], rtol=1e-12)


def test_cut_edges_become_walls():
    w = W.partial_dam_break(nx=16, ny=8, spacing=1.0, n_gauss=4)
    m = oracle.Mesh(w.nodes, w.tris, w.bnd_edges, w.bnd_tag, w.cut_edges)
    m0 = oracle.Mesh(w.nodes, w.tris, w.bnd_edges, w.bnd_tag)
    a, a0 = m.arrays, m0.arrays
    extra = (a["nbr"] < 0).sum() - (a0["nbr"] < 0).sum()
    assert extra == 2 * len(w.cut_edges)
    assert (a["btag"][(a["nbr"] < 0) & (a0["nbr"] >= 0)] == 0).all()


@pytest.mark.parametrize("case", ["degenerate", "nonmanifold", "bnd_not_boundary"])
def test_bad_meshes_rejected(case):
    nodes = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0], [2.0, 2.0], [0.2, 0.8]])
    tris = np.array([[0, 1, 2], [0, 2, 3]])
    bnd = None
    if case == "degenerate":
        tris = np.array([[0, 2, 4]])
    elif case == "nonmanifold":
        tris = np.array([[0, 1, 2], [0, 2, 3], [0, 2, 5]])
    else:
        bnd = np.array([[0, 2]])
    with pytest.raises(ValueError):
        oracle.Mesh(nodes, tris, bnd, None if bnd is None else np.array([1]))


def _morton_keys(cx, cy):
    ext = max(cx.max() - cx.min(), cy.max() - cy.min())
    s = 2097151.0 / ext
    qx = np.clip(np.floor((cx - cx.min()) * s), 0, 2097151).astype(np.uint64)
    qy = np.clip(np.floor((cy - cy.min()) * s), 0, 2097151).astype(np.uint64)
    key = np.zeros_like(qx)
    for b in range(21):
        key |= ((qx >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
        key |= ((qy >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + 1)
    return key


def test_morton_order_properties():
    nodes, tris, bnd, side = W.structured(20, 13, 20.0, 13.0, jitter=0.3, seed=2)
    m = oracle.Mesh(nodes, tris)
    p = m.morton()
    assert np.array_equal(np.sort(p), np.arange(m.n))
    key = _morton_keys(m.arrays["cx"], m.arrays["cy"])[p]
    assert (np.diff(key.astype(np.float64)) >= 0).all()
    same = key[1:] == key[:-1]
    assert (p[1:][same] > p[:-1][same]).all()


def test_rcm_reduces_bandwidth():
    nodes, tris, bnd, side = W.structured(30, 20, 30.0, 20.0)
    rng = np.random.default_rng(0)
    shuffle = rng.permutation(len(tris))
    m = oracle.Mesh(nodes, tris[shuffle])
    p = m.rcm()
    assert np.array_equal(np.sort(p), np.arange(m.n))
    inv = np.empty_like(p)
    inv[p] = np.arange(m.n)
    nbr = m.arrays["nbr"]
    i = np.repeat(np.arange(m.n), 3)
    j = nbr.ravel()
    ok = j >= 0
    bw_before = np.abs(i[ok] - j[ok]).max()
    bw_after = np.abs(inv[i[ok]] - inv[j[ok]]).max()
    assert bw_after < bw_before / 5
