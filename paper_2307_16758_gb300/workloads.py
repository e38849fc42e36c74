"""Seeded synthetic workloads: triangle meshes, bathymetry and initial states.

This module only builds inputs (node coordinates, triangles, boundary tags,
bed elevation, Manning coefficients, initial depth and discharge); it holds
none of the solver's arithmetic.  The same arrays feed the CUDA path and the
FP64 oracle.  The paper's meshes and bathymetry (the Mille-Iles river and the
Montreal archipelago, Sec. 6.5) are not available, so these generators stand
in for them at the sizes of the benchmark workloads:

* ``dam_break_1d``  -- the idealised wet-bed dam break of Sec. 6.3, as a strip
  of squares split by their "/" diagonal (the 100 m x 10 m case is 2000 cells).
* ``partial_dam_break`` -- a jittered 1 m structured triangulation, a bed made
  of seeded Gaussians on a 0.1 % slope, a lake at rest at eta = 2 m with about
  30 % of the cells dry, and an internal wall with a breach (1M cells at full size).
* ``river`` -- a meandering channel (sinuosity 1.5, width 200-800 m, bed
  5-15 m below the banks) in a 40 km x 15 km floodplain with 1/f^2 noise, an
  inflow cross-section upstream and a fixed level downstream (13M / 4M cells).
* ``ensemble_sizes`` -- 64 log-uniform member sizes summing to 40M cells.

Bed elevations are rounded to multiples of 2^-10 m.  With such a bed,
h = eta - z and eta = h + z are exact in FP64 and in FP32 (for |z| < 8192 m),
so a lake at rest can be represented exactly in either precision.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

WALL, OPEN, INFLOW, LEVEL = 0, 1, 2, 3
BED_QUANTUM = 2.0 ** -10


def tag(kind: int, group: int = 0) -> int:
    """Boundary tag: kind (WALL/OPEN/INFLOW/LEVEL) + 4 * group."""
    return int(kind) + 4 * int(group)


@dataclass
class Workload:
    name: str
    nodes: np.ndarray            # [n_nodes, 2] float64
    tris: np.ndarray             # [n_cells, 3] int32
    bnd_edges: np.ndarray        # [n_bnd, 2] int32 node pairs
    bnd_tag: np.ndarray          # [n_bnd] int32
    cut_edges: np.ndarray        # [n_cut, 2] int32 node pairs (internal walls)
    z: np.ndarray                # [n_cells] bed elevation, float64
    nman: np.ndarray             # [n_cells] Manning n
    h: np.ndarray                # [n_cells] initial depth
    hu: np.ndarray
    hv: np.ndarray
    q_in: np.ndarray = field(default_factory=lambda: np.zeros(0))    # inflow discharge per group [m^3/s]
    level: np.ndarray = field(default_factory=lambda: np.zeros(0))   # outflow free surface per group [m]
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return int(self.tris.shape[0])

    def centroids(self):
        p = self.nodes[self.tris]
        return p[:, :, 0].mean(axis=1), p[:, :, 1].mean(axis=1)


def quantize_bed(z):
    return np.round(np.asarray(z, dtype=np.float64) / BED_QUANTUM) * BED_QUANTUM


def structured(nx: int, ny: int, lx: float, ly: float, jitter: float = 0.0, seed: int = 0,
               fixed_x_col: int | None = None):
    """Rectangle [0,lx]x[0,ly] of nx*ny squares, each split by its "/" diagonal.

    Interior nodes move by U(-jitter, jitter) spacings per axis (boundary
    nodes stay); nodes of triangles left with less than 20 % of their nominal
    area have their displacement halved until no such triangle remains.  Returns nodes, tris and the boundary edges with their side
    (0 bottom, 1 right, 2 top, 3 left)."""
    dx, dy = lx / nx, ly / ny
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1))
    x = (ii * dx).astype(np.float64).ravel()
    y = (jj * dy).astype(np.float64).ravel()
    if jitter > 0:
        rng = np.random.default_rng(seed)
        jx = rng.uniform(-jitter, jitter, x.shape) * dx
        jy = rng.uniform(-jitter, jitter, y.shape) * dy
        interior = ((ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)).ravel()
        mx = interior.copy()
        if fixed_x_col is not None:
            mx &= (ii.ravel() != fixed_x_col)
        jx = np.where(mx, jx, 0.0)
        jy = np.where(interior, jy, 0.0)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    i, j = i.ravel(), j.ravel()
    p00 = j * (nx + 1) + i
    p10, p01, p11 = p00 + 1, p00 + nx + 1, p00 + nx + 2
    tris = np.empty((2 * nx * ny, 3), np.int32)
    tris[0::2] = np.stack([p00, p10, p11], axis=1)
    tris[1::2] = np.stack([p00, p11, p01], axis=1)
    if jitter > 0:
        # a jitter above 1/6 of the spacing can fold or flatten a triangle:
        # halve the jitter of the nodes of any triangle under 20 % of its
        # nominal area until none is left (deterministic)
        for _ in range(40):
            px, py = (x + jx)[tris], (y + jy)[tris]
            cross = (px[:, 1] - px[:, 0]) * (py[:, 2] - py[:, 0]) - (py[:, 1] - py[:, 0]) * (px[:, 2] - px[:, 0])
            bad = cross < 0.2 * dx * dy
            if not bad.any():
                break
            nodes_bad = np.unique(tris[bad])
            jx[nodes_bad] *= 0.5
            jy[nodes_bad] *= 0.5
        x, y = x + jx, y + jy
    nodes = np.stack([x, y], axis=1)
    # boundary edges, side by side
    b = np.arange(nx)
    bottom = np.stack([b, b + 1], axis=1)
    top = np.stack([ny * (nx + 1) + b, ny * (nx + 1) + b + 1], axis=1)
    c = np.arange(ny)
    left = np.stack([c * (nx + 1), (c + 1) * (nx + 1)], axis=1)
    right = np.stack([c * (nx + 1) + nx, (c + 1) * (nx + 1) + nx], axis=1)
    bnd = np.concatenate([bottom, right, top, left]).astype(np.int32)
    side = np.concatenate([np.zeros(nx), np.ones(ny), np.full(nx, 2), np.full(ny, 3)]).astype(np.int32)
    return nodes, tris, bnd, side


def _empty_edges():
    return np.zeros((0, 2), np.int32)


def dam_break_1d(nx: int = 100, ny: int = 10, lx: float = 100.0, ly: float = 10.0,
                 h_left: float = 1.0, h_right: float = 0.5, v_left: float = 0.0, v_right: float = 0.0,
                 x_dam: float | None = None, open_ends: bool = False) -> Workload:
    """Idealised wet-bed dam break (Sec. 6.3), walls all round by default.

    Optional tangential velocities v_left / v_right add a passive shear layer."""
    nodes, tris, bnd, side = structured(nx, ny, lx, ly)
    x_dam = lx / 2 if x_dam is None else x_dam
    w = Workload("dam_break_1d", nodes, tris, bnd, np.zeros(len(bnd), np.int32), _empty_edges(),
                 np.zeros(len(tris)), np.zeros(len(tris)), None, None, None)
    cx, cy = w.centroids()
    left = cx < x_dam
    w.h = np.where(left, h_left, h_right).astype(np.float64)
    w.hu = np.zeros(len(tris))
    w.hv = w.h * np.where(left, v_left, v_right)
    if open_ends:
        w.bnd_tag = np.where((side == 1) | (side == 3), tag(OPEN), tag(WALL)).astype(np.int32)
    w.meta = dict(nx=nx, ny=ny, lx=lx, ly=ly, h_left=h_left, h_right=h_right, x_dam=x_dam)
    return w


def partial_dam_break(nx: int = 1000, ny: int = 500, spacing: float = 1.0, seed: int = 20230732,
                      n_gauss: int = 200, eta0: float = 2.0, eta_up: float = 3.0,
                      dry_fraction: float = 0.30, manning: float = 0.03, breach: bool = True,
                      jitter: float = 0.3) -> Workload:
    """Lake at rest over Gaussian bathymetry with a partial dam break.

    The bed is 0.001*(L - x) plus n_gauss seeded Gaussians (amplitude U(0,3) m,
    sigma U(5,50) m scaled with the domain), shifted so that ``dry_fraction``
    of the cells lie above eta0.  An internal wall on the grid line x = L/4
    has a breach of half-width ny*spacing/10 about mid-height; upstream of it
    the free surface is eta_up.  With ``breach=False`` the state is the lake at rest."""
    lx, ly = nx * spacing, ny * spacing
    dam_col = nx // 4
    nodes, tris, bnd, side = structured(nx, ny, lx, ly, jitter=jitter, seed=seed, fixed_x_col=dam_col)
    rng = np.random.default_rng(seed + 1)
    p = nodes[tris]
    cx, cy = p[:, :, 0].mean(axis=1), p[:, :, 1].mean(axis=1)
    scale = min(lx / 1000.0, ly / 500.0)
    z = 0.001 * (lx - cx)
    amp = rng.uniform(0.0, 3.0, n_gauss)
    sig = rng.uniform(5.0, 50.0, n_gauss) * max(scale, 0.02)
    gx = rng.uniform(0.0, lx, n_gauss)
    gy = rng.uniform(0.0, ly, n_gauss)
    for a, s, x0, y0 in zip(amp, sig, gx, gy):
        r2 = (cx - x0) ** 2 + (cy - y0) ** 2
        m = r2 < (6 * s) ** 2
        z[m] += a * np.exp(-r2[m] / (2 * s * s))
    z += eta0 - np.quantile(z, 1.0 - dry_fraction)
    z = quantize_bed(z)
    h = np.maximum(0.0, eta0 - z)
    cut = _empty_edges()
    if breach:
        # vertical grid edges on column dam_col, except the breach
        jrow = np.arange(ny)
        ymid = (jrow + 0.5) * spacing
        keep = np.abs(ymid - ly / 2) > ly / 10
        a = jrow[keep] * (nx + 1) + dam_col
        cut = np.stack([a, a + nx + 1], axis=1).astype(np.int32)
        sq_i = (np.arange(len(tris)) // 2) % nx
        up = sq_i < dam_col
        h = np.where(up, np.maximum(0.0, eta_up - z), h)
    w = Workload("partial_dam_break", nodes, tris, bnd, np.zeros(len(bnd), np.int32), cut,
                 z, np.full(len(tris), manning), h, np.zeros(len(tris)), np.zeros(len(tris)))
    w.meta = dict(nx=nx, ny=ny, spacing=spacing, seed=seed, eta0=eta0, eta_up=eta_up, dam_col=dam_col)
    return w


def _fractal_noise(shape, rng, std):
    """Gaussian field with a 1/f^2 power spectrum, scaled to the given std."""
    ny, nx = shape
    white = rng.standard_normal(shape)
    f = np.fft.rfft2(white)
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.rfftfreq(nx)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    k[0, 0] = np.inf
    field_ = np.fft.irfft2(f / k, s=shape)
    field_ -= field_.mean()
    return field_ * (std / field_.std())


def river(nx: int = 4160, ny: int = 1563, lx: float = 40000.0, ly: float = 15000.0,
          seed: int = 20230733, q_in: float = 8000.0, n_channel: float = 0.025,
          n_floodplain: float = 0.05, level_quantile: float = 0.5, jitter: float = 0.25) -> Workload:
    """Meandering river in a floodplain (stand-in for the Mille-Iles mesh of Sec. 6.5).

    Centreline y = ly/2 + A sin(2 pi x / lambda) with A = 0.262 lambda
    (sinuosity 1.5) and lambda = 5.5 km +-20 %; width 200-800 m and depth
    5-15 m vary as seeded sinusoids; the floodplain falls 0.0001 down-valley
    and carries 1/f^2 noise of std 0.5 m.  The initial free surface is flat
    at the ``level_quantile`` of the bed (about half the cells dry at 0.5).
    Inflow Q enters through the channel's upstream cross-section; the
    downstream side holds the initial level."""
    rng = np.random.default_rng(seed)
    nodes, tris, bnd, side = structured(nx, ny, lx, ly, jitter=jitter, seed=seed + 7)
    lam = 5500.0 * rng.uniform(0.8, 1.2)
    amp = 0.262 * lam
    lam_w, ph_w = rng.uniform(8000.0, 15000.0), rng.uniform(0, 2 * np.pi)
    lam_d, ph_d = rng.uniform(6000.0, 12000.0), rng.uniform(0, 2 * np.pi)
    noise_nodes = _fractal_noise((ny + 1, nx + 1), rng, 0.5).ravel()

    def centre(x):
        return ly / 2 + amp * np.sin(2 * np.pi * x / lam)

    def slope(x):
        return amp * 2 * np.pi / lam * np.cos(2 * np.pi * x / lam)

    def width(x):
        return 500.0 + 300.0 * np.sin(2 * np.pi * x / lam_w + ph_w)

    def depth(x):
        return 10.0 + 5.0 * np.sin(2 * np.pi * x / lam_d + ph_d)

    p = nodes[tris]
    cx, cy = p[:, :, 0].mean(axis=1), p[:, :, 1].mean(axis=1)
    zf = 0.0001 * (lx - cx) + noise_nodes[tris].mean(axis=1)
    d = np.abs(cy - centre(cx)) / np.sqrt(1.0 + slope(cx) ** 2)
    w_ = width(cx)
    inch = d < w_ / 2
    z = np.where(inch, zf - depth(cx) * (1.0 - (2 * d / w_) ** 2), zf)
    z = quantize_bed(z)
    eta0 = float(quantize_bed(np.quantile(z, level_quantile)))
    h = np.maximum(0.0, eta0 - z)
    nman = np.where(inch, n_channel, n_floodplain).astype(np.float64)
    # boundary tags: inflow on the channel part of the upstream side, level downstream
    mid = nodes[bnd].mean(axis=1)
    dy = ly / ny
    bin_ = (side == 3) & (np.abs(mid[:, 1] - centre(0.0)) < max(width(0.0) / 2, 0.75 * dy))
    tags = np.where(bin_, tag(INFLOW, 0), np.where(side == 1, tag(LEVEL, 0), tag(WALL)))
    w = Workload("river", nodes, tris, bnd, tags.astype(np.int32), _empty_edges(), z, nman, h,
                 np.zeros(len(tris)), np.zeros(len(tris)),
                 q_in=np.array([q_in]), level=np.array([eta0]))
    w.meta = dict(nx=nx, ny=ny, lx=lx, ly=ly, seed=seed, lam=lam, eta0=eta0, q_in=q_in,
                  n_channel=n_channel, n_floodplain=n_floodplain, wet_fraction=float((h > 0).mean()))
    return w


def river_grid_for_cells(n_cells: int, lx: float = 40000.0, ly: float = 15000.0):
    """Grid (nx, ny) with the river's aspect ratio and about n_cells triangles."""
    nx = max(8, int(round(math.sqrt(n_cells / 2.0 * lx / ly))))
    ny = max(4, int(round(n_cells / (2.0 * nx))))
    return nx, ny


def ensemble_sizes(n_members: int = 64, total: int = 40_000_000, lo: int = 50_000, hi: int = 2_000_000,
                   seed: int = 20230735):
    """Member sizes: log-uniform in [lo, hi], rescaled and clipped to sum to ``total``."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(np.log(lo), np.log(hi), n_members))
    for _ in range(50):
        s = np.clip(s * total / s.sum(), lo, hi)
    return np.round(s).astype(np.int64)


def ensemble_member(k: int, n_cells: int, seed: int = 20230735) -> Workload:
    """Member k of the river ensemble: own size, inflow, Manning n and initial level."""
    rng = np.random.default_rng(seed + 1000 + k)
    q = rng.uniform(1000.0, 10000.0)
    nch = rng.uniform(0.02, 0.06)
    lvl = rng.uniform(0.3, 0.7)
    nx, ny = river_grid_for_cells(n_cells)
    return river(nx, ny, seed=seed + 2000 + k, q_in=q, n_channel=nch,
                 n_floodplain=min(2 * nch, 0.1), level_quantile=lvl)


def circular_dam_break(n: int = 40, radius: float = 10.0, half: float = 25.0, h_in: float = 2.0,
                       h_out: float = 1.0, jitter: float = 0.0, seed: int = 5) -> Workload:
    """Square [-half, half]^2 with a cylinder of water of the given radius.

    The triangulation alternates its diagonal by quadrant so that it is
    mirror-symmetric about both axes (when jitter is 0)."""
    nodes, tris, bnd, side = structured(2 * n, 2 * n, 2 * half, 2 * half, jitter=jitter, seed=seed)
    nodes = nodes - half
    # mirror the diagonal in the quadrants x<0 xor y<0 so the mesh is symmetric
    nx = 2 * n
    sq = np.arange(len(tris)) // 2
    i, j = sq % nx, sq // nx
    p00 = j * (nx + 1) + i
    p10, p01, p11 = p00 + 1, p00 + nx + 1, p00 + nx + 2
    flip = (i < n) ^ (j < n)
    t0 = np.where(flip[:, None], np.stack([p00, p10, p01], 1), np.stack([p00, p10, p11], 1))
    t1 = np.where(flip[:, None], np.stack([p10, p11, p01], 1), np.stack([p00, p11, p01], 1))
    tris = tris.copy()
    tris[0::2] = t0[0::2]
    tris[1::2] = t1[1::2]
    w = Workload("circular_dam_break", nodes, tris.astype(np.int32), bnd, np.zeros(len(bnd), np.int32),
                 _empty_edges(), np.zeros(len(tris)), np.zeros(len(tris)), None, None, None)
    cx, cy = w.centroids()
    w.h = np.where(cx * cx + cy * cy < radius * radius, h_in, h_out).astype(np.float64)
    w.hu = np.zeros(len(tris))
    w.hv = np.zeros(len(tris))
    w.meta = dict(n=n, radius=radius, half=half)
    return w


def gaussian_hump(n: int, l: float = 10.0, amp: float = 0.1, h0: float = 1.0, sigma: float = 1.0) -> Workload:
    """Smooth free-surface hump on a flat bed in a closed square (order studies).

    Grids with n, 2n, 4n squares per side are nested: each coarse triangle is
    exactly four fine ones."""
    nodes, tris, bnd, side = structured(n, n, l, l)
    w = Workload("gaussian_hump", nodes, tris, bnd, np.zeros(len(bnd), np.int32), _empty_edges(),
                 np.zeros(len(tris)), np.zeros(len(tris)), None, None, None)
    cx, cy = w.centroids()
    w.h = h0 + amp * np.exp(-((cx - l / 2) ** 2 + (cy - l / 2) ** 2) / (2 * sigma * sigma))
    w.hu = np.zeros(len(tris))
    w.hv = np.zeros(len(tris))
    w.meta = dict(n=n, l=l)
    return w
