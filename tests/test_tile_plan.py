"""The tile step's plan, host side (no GPU needed).

The plan is what the one-pass tile kernel indexes instead of the mesh's
adjacency: every slot, halo id and edge record it holds must name the same
cell, local edge and left/right role as the exported adjacency (Sec. 6.1: each
side L_ij of a cell, its neighbour j, and which of the two is the edge's left
state: the lower id in the caller's order).  Each test decodes the plan and
checks it record by record against the adjacency, and checks that every edge
a tile must solve is there exactly once.
"""
import numpy as np
import pytest

from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe
from paper_2307_16758_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    swe.load_library()


def _check_plan(m, tile):
    """Decode the plan of mesh m and compare it with the exported adjacency."""
    a = m.export()
    nbr, nbr_edge, btag, perm = a["nbr"], a["nbr_edge"], a["btag"], a["perm"]
    n = m.n
    info, hdr, words = swe.swe_tile_plan_export(m.handle, tile)
    n_tiles = -(-n // tile)
    assert info["n_tiles"] == n_tiles and hdr.shape == (n_tiles, 8)
    assert info["n_words"] == len(words) and len(words) % 8 == 0
    next_off = 0
    seen = {}                                       # (cell, local edge) -> times solved as the left cell
    for b in range(n_tiles):
        off, n_halo, n_h1, n_edges, n_cross, nw, z0, z1 = (int(v) for v in hdr[b])
        assert (z0, z1) == (0, 0)
        assert off == next_off and nw % 8 == 0
        next_off = off + nw
        s0, s1 = b * tile, min(n, (b + 1) * tile)

        def inside(j):
            return s0 <= j < s1

        # halo: H1 in order of first use, then H2 ascending
        h1 = []
        for i in range(s0, s1):
            for k in range(3):
                j = int(nbr[i, k])
                if j >= 0 and not inside(j) and j not in h1:
                    h1.append(j)
        h2 = sorted({int(q) for j in h1 for q in nbr[j] if q >= 0 and not inside(q) and q not in h1})
        halo = words[off:off + n_halo].tolist()
        assert n_h1 == len(h1) and halo == h1 + h2
        assert tile + n_halo <= 2047

        def cell(slot):
            assert 0 <= slot < tile + n_halo
            return s0 + slot if slot < tile else halo[slot - tile]

        # edge records: crossing edges first, every record names a real side
        rec = words[off + n_halo:off + n_halo + n_edges].astype(np.int64) & 0xFFFFFFFF
        assert (rec >> 28 == 0).all()
        want_cross = {(i, k) for i in range(s0, s1) for k in range(3) if nbr[i, k] >= 0 and not inside(nbr[i, k])}
        want_inner = {(i, k) for i in range(s0, s1) for k in range(3) if nbr[i, k] > i and inside(nbr[i, k])}
        got = []
        for q, r in enumerate(rec.tolist()):
            si, ki, sj, kj = r & 0x7FF, (r >> 11) & 3, (r >> 13) & 0x7FF, (r >> 24) & 3
            own, cross = (r >> 26) & 1, (r >> 27) & 1
            assert si < s1 - s0
            i, j = s0 + si, cell(sj)
            assert nbr[i, ki] == j and nbr_edge[i, ki] == kj and nbr[j, kj] == i
            assert own == (perm[i] < perm[j]) and cross == (not inside(j)) and cross == (q < n_cross)
            got.append((i, ki))
            if own:
                seen[(i, ki)] = seen.get((i, ki), 0) + 1
            else:
                seen[(j, kj)] = seen.get((j, kj), 0) + 1
        assert len(got) == len(set(got)) == n_edges
        assert set(got[:n_cross]) == want_cross and set(got[n_cross:]) == want_inner

        # local words: per tile slot and per H1 cell, each local edge
        lw0 = off + n_halo + n_edges
        lw = words[lw0:off + nw].view(np.int16)
        n_lw = 3 * (tile + n_h1)
        assert len(lw) >= n_lw and (lw[n_lw:] == 0).all()
        for s in range(tile + n_h1):
            c = s0 + s if s < tile else h1[s - tile]
            for k in range(3):
                v = int(lw[3 * s + k])
                if s < tile and c >= n:
                    assert v == -1                  # unused slot: a wall
                    continue
                q = int(nbr[c, k])
                if q < 0:
                    assert v == -1 - int(btag[c, k])
                else:
                    assert v >= 0
                    assert cell(v >> 3) == q and (v >> 1) & 3 == nbr_edge[c, k] and (v & 1) == (perm[c] < perm[q])
    assert next_off == len(words)
    assert info["hmax"] == int(hdr[:, 1].max()) and info["h1max"] == int(hdr[:, 2].max())
    assert info["wmax"] == int(hdr[:, 5].max())
    # across tiles: an edge inside a tile is solved once, an edge between two tiles once from each
    interior = {(i, k) for i in range(n) for k in range(3) if nbr[i, k] >= 0 and perm[i] < perm[nbr[i, k]]}
    assert set(seen) == interior
    for (i, k), t in seen.items():
        assert t == (1 if (i // tile) == (int(nbr[i, k]) // tile) else 2)
    return info


@pytest.mark.parametrize("reorder", ["morton", "rcm", "none"])
@pytest.mark.parametrize("tile", [32, 128, 256])
def test_plan_matches_adjacency_dam_break(reorder, tile):
    """Partial dam break: walls, an internal wall with a breach (cut edges),
    inflow and open boundaries; 1,600 cells, a ragged last tile at 128 and
    256 cells."""
    w = W.partial_dam_break(nx=40, ny=20, spacing=1.0, n_gauss=10, seed=4)
    m = swe.Mesh.from_workload(w, reorder)
    assert m.n % tile != 0 or tile == 32
    _check_plan(m, tile)
    m.close()


@pytest.mark.parametrize("tile", [64, 1024])
def test_plan_matches_adjacency_circular(tile):
    """Circular dam break mesh (alternating diagonals), Morton order; at 1024
    cells per tile the last tile is mostly unused slots."""
    w = W.circular_dam_break(n=24)
    m = swe.Mesh.from_workload(w, "morton")
    _check_plan(m, tile)
    m.close()


def test_plan_of_a_mesh_smaller_than_one_tile():
    w = W.dam_break_1d(5, 2, 5.0, 2.0)
    m = swe.Mesh.from_workload(w, "morton")
    assert m.n < 32
    info = _check_plan(m, 32)
    assert info["n_tiles"] == 1
    m.close()


def _shuffled_mesh(nx, ny, seed):
    nodes, tris, bnd, side = W.structured(nx, ny, float(nx), float(ny))
    tris = tris[np.random.default_rng(seed).permutation(len(tris))]
    return swe.Mesh(nodes, tris, bnd, np.zeros(len(bnd), np.int32), reorder="none")


def test_plan_of_a_scattered_order():
    """No locality at all (cells in random order): nearly every edge crosses
    a tile, halos are as large as they get, and the plan must still hold."""
    m = _shuffled_mesh(30, 20, seed=7)
    info = _check_plan(m, 32)
    assert info["h1max"] > 40
    m.close()


def test_plan_rejects_a_halo_beyond_the_slot_fields():
    """1,024 scattered cells reach more than 1,023 outside cells: the 11-bit
    slots cannot hold them and the plan (and the tile step) refuse."""
    m = _shuffled_mesh(60, 40, seed=8)
    with pytest.raises(swe.SweError) as e:
        swe.swe_tile_plan_info(m.handle, 1024)
    assert e.value.code == -1 and "renumber" in str(e.value)
    m.close()


@pytest.mark.parametrize("tile", [0, 16, 31, 48, 96, 2048, -32])
def test_plan_rejects_bad_tile_sizes(tile):
    w = W.dam_break_1d(10, 2, 10.0, 2.0)
    m = swe.Mesh.from_workload(w)
    with pytest.raises(swe.SweError) as e:
        swe.swe_tile_plan_info(m.handle, tile)
    assert e.value.code == -1 and "power of two" in str(e.value)
    m.close()


def test_plan_rejects_a_null_mesh():
    with pytest.raises(swe.SweError) as e:
        swe.swe_tile_plan_info(None, 128)
    assert e.value.code == -1
