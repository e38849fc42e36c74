"""The seeded synthetic inputs follow their stated recipe (no GPU needed).

The paper's meshes and bathymetry (Sec. 6.5) are not available; the
generators stand in for them.  These tests check, on small versions of each
recipe, the properties that the workloads are chosen for: seeded and
reproducible, beds on the 2^-10 m grid (so that a lake at rest is exact in
FP32 and FP64), the stated wet fractions, boundary tags on the stated sides,
Manning coefficients by zone, the internal wall with its breach, and the
ensemble's member sizes and parameter ranges.
"""
import numpy as np
import pytest

from paper_2307_16758_gb300 import workloads as W


def _arrays(w):
    return [w.nodes, w.tris, w.bnd_edges, w.bnd_tag, w.cut_edges, w.z, w.nman, w.h, w.hu, w.hv]


def _areas(w):
    p = w.nodes[w.tris]
    return 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) -
                  (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))


@pytest.mark.parametrize("make", [lambda s: W.river(120, 45, seed=s),
                                  lambda s: W.partial_dam_break(nx=80, ny=40, n_gauss=12, seed=s)])
def test_generators_are_seeded(make):
    a, b, c = make(11), make(11), make(12)
    for x, y in zip(_arrays(a), _arrays(b)):
        assert np.array_equal(x, y)
    assert not np.array_equal(a.z, c.z)


@pytest.mark.parametrize("make", [lambda: W.river(120, 45, seed=3),
                                  lambda: W.partial_dam_break(nx=80, ny=40, n_gauss=12, seed=3)])
def test_beds_on_the_quantum_make_rest_exact_in_fp32(make):
    """z is a multiple of 2^-10 m, so eta = h + z rounds to nothing in FP32:
    every wet cell of the initial lake gives back its level exactly."""
    w = make()
    q = w.z / W.BED_QUANTUM
    assert np.array_equal(q, np.round(q))
    wet = w.h > 0
    eta = w.h + w.z
    for T in (np.float32, np.float64):
        h, z = w.h.astype(T), w.z.astype(T)
        assert np.array_equal((h + z)[wet], eta[wet].astype(T))
        assert np.array_equal((eta.astype(T) - z)[wet], h[wet])


def test_jitter_keeps_every_triangle_above_a_fifth_of_its_area():
    nodes, tris, bnd, side = W.structured(60, 30, 60.0, 30.0, jitter=0.45, seed=9)
    p = nodes[tris]
    a = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) -
               (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))
    assert a.min() >= 0.2 * 0.5 - 1e-12
    assert abs(a.sum() - 60.0 * 30.0) < 1e-9                # the rectangle is still tiled
    interior = np.ones(len(nodes), bool)
    interior[np.unique(bnd)] = False
    moved = np.abs(nodes - W.structured(60, 30, 60.0, 30.0)[0]).max(axis=1)
    assert (moved[~interior] == 0).all() and (moved[interior] > 0).mean() > 0.9


def test_river_recipe():
    nx, ny, ql = 200, 75, 0.5
    w = W.river(nx, ny, seed=5, q_in=3000.0, n_channel=0.03, n_floodplain=0.06, level_quantile=ql)
    assert w.n_cells == 2 * nx * ny
    assert abs(_areas(w).sum() - 40000.0 * 15000.0) < 1e-3 * 40000.0 * 15000.0 * 1e-6
    # flat initial level at the bed quantile: about that fraction wet, at rest
    eta0 = w.meta["eta0"]
    wet = w.h > 0
    assert abs(wet.mean() - ql) < 0.02
    assert np.array_equal(w.h[wet] + w.z[wet], np.full(wet.sum(), eta0))
    assert (w.z[~wet] >= eta0).all()
    assert not w.hu.any() and not w.hv.any()
    # Manning n by zone; the channel lies below the floodplain around it
    assert set(np.unique(w.nman)) == {0.03, 0.06}
    ch = w.nman == 0.03
    assert 0.01 < ch.mean() < 0.2
    assert np.median(w.z[ch]) < np.median(w.z[~ch]) - 4.0
    # tags: inflow group 0 on the upstream side (x = 0) inside the channel,
    # fixed level downstream (x = 40 km), walls elsewhere
    mid = w.nodes[w.bnd_edges].mean(axis=1)
    kinds = w.bnd_tag & 3
    assert set(np.unique(w.bnd_tag)) == {W.tag(W.WALL), W.tag(W.INFLOW, 0), W.tag(W.LEVEL, 0)}
    assert np.allclose(mid[kinds == W.INFLOW, 0], 0.0)
    assert np.allclose(mid[kinds == W.LEVEL, 0], 40000.0)
    assert (kinds == W.LEVEL).sum() == ny
    y_in = mid[kinds == W.INFLOW, 1]
    assert 0 < len(y_in) < ny and y_in.max() - y_in.min() < 800.0 + 2 * 15000.0 / ny
    assert list(w.q_in) == [3000.0] and list(w.level) == [eta0]


def test_partial_dam_break_recipe():
    nx, ny = 120, 60
    w = W.partial_dam_break(nx=nx, ny=ny, spacing=1.0, n_gauss=20, seed=6)
    assert w.n_cells == 2 * nx * ny
    dam = nx // 4
    # internal wall: vertical grid edges on x = dam except the breach |y - L/2| <= L/10
    e = w.nodes[w.cut_edges]
    assert np.allclose(e[:, :, 0], dam)
    ymid = e[:, :, 1].mean(axis=1)
    assert (np.abs(ymid - ny / 2) > ny / 10).all()
    assert len(w.cut_edges) == ny - np.count_nonzero(np.abs(np.arange(ny) + 0.5 - ny / 2) <= ny / 10)
    # lake at eta 2 downstream with about 30 % of all cells above it, eta 3 upstream
    cx = w.nodes[w.tris][:, :, 0].mean(axis=1)
    up = (np.arange(w.n_cells) // 2) % nx < dam
    assert (cx[up] < dam).all() and (cx[~up] > dam).all()
    wet = w.h > 0
    assert np.allclose((w.h + w.z)[wet & ~up], 2.0, rtol=0, atol=0)
    assert np.allclose((w.h + w.z)[wet & up], 3.0, rtol=0, atol=0)
    assert abs((w.z > 2.0).mean() - 0.30) < 0.01
    assert set(np.unique(w.nman)) == {0.03}
    assert (w.bnd_tag == W.tag(W.WALL)).all()
    # without the breach it is the lake at rest, one level everywhere
    r = W.partial_dam_break(nx=nx, ny=ny, spacing=1.0, n_gauss=20, seed=6, breach=False)
    assert len(r.cut_edges) == 0 and np.array_equal((r.h + r.z)[r.h > 0], np.full((r.h > 0).sum(), 2.0))


def test_dam_break_recipe():
    w = W.dam_break_1d()
    assert w.n_cells == 2000
    cx = w.nodes[w.tris][:, :, 0].mean(axis=1)
    assert np.array_equal(w.h, np.where(cx < 50.0, 1.0, 0.5))
    assert not w.z.any() and not w.hu.any() and not w.hv.any()
    assert (w.bnd_tag == W.tag(W.WALL)).all()


def test_ensemble_sizes_and_members():
    s = W.ensemble_sizes()
    assert len(s) == 64
    assert s.min() >= 50_000 and s.max() <= 2_000_000
    assert abs(int(s.sum()) - 40_000_000) <= 64
    assert np.array_equal(s, W.ensemble_sizes())
    for k in (0, 17, 63):
        n = 4000 + 1000 * k
        m = W.ensemble_member(k, n)
        assert abs(m.n_cells - n) / n < 0.05
        q, nch = float(m.q_in[0]), m.meta["n_channel"]
        assert 1000.0 <= q <= 10000.0 and 0.02 <= nch <= 0.06
        assert m.meta["n_floodplain"] == min(2 * nch, 0.1)
        assert 0.25 < m.meta["wet_fraction"] < 0.75
