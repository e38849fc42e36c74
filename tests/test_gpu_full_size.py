"""Full-size checks on the workloads' own sizes.

13,004,160-cell river (the benchmark): the oracle can afford one full-mesh
step, so the FP64 path is compared with it cell by cell (one step, 1e-12).
The FP32 benchmark configuration (the one-pass tile step with tiles of 256
cells, CUDA graphs, CFL 0.9) is checked through properties that hold at any
size: its one-step result against the same oracle step (same h_eps), the mass
budget, and that the split kernels give the same bits.

4,000,920-cell river: WAF and MUSCL in FP32 against the FP64 path after 1000
steps (L1 error, mass drift, wetting front).

1,000,000-cell partial dam break: MUSCL (split kernels and tile step) and
WAF (split kernels) FP64 against the oracle after 100 steps, cell by cell.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe
from paper_2307_16758_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def river13m():
    B.build()
    swe.load_library()
    w = W.river()                                   # 4160 x 1563 grid, 13,004,160 cells
    assert w.n_cells == 13_004_160
    mesh = swe.Mesh.from_workload(w, "morton")
    om = oracle.Mesh(w.nodes, w.tris, w.bnd_edges, w.bnd_tag)
    yield w, mesh, om
    mesh.close()


def _oracle_step(w, om, h_eps, dt):
    o = oracle.opts("muscl", h_eps=h_eps, r_eps=1e-12 if h_eps < 1e-5 else 1e-6)
    return oracle.run(om, o, w.z, w.nman, w.h, w.hu, w.hv, 1, q_in=w.q_in, level=w.level, dt=[dt])


def test_fp64_one_step_matches_oracle_at_full_size(river13m):
    w, mesh, om = river13m
    st = swe.State.from_workload(mesh, swe.swe_params_default("muscl", "fp64"), w)
    st.step(1, 0.9)
    dt = st.dt_history(1)[0]
    h, hu, hv = st.get_state()
    st.close()
    oh, ohu, ohv, dts, d = _oracle_step(w, om, 1e-6, dt)
    qs = max(np.abs(ohu).max(), np.abs(ohv).max())
    assert np.abs(h - oh).max() <= 1e-12 * np.abs(oh).max()
    assert np.abs(hu - ohu).max() <= 1e-12 * qs
    assert np.abs(hv - ohv).max() <= 1e-12 * qs
    # the GPU's CFL step equals the oracle's own
    _, _, _, dts2, _ = oracle.run(om, oracle.opts("muscl"), w.z, w.nman, w.h, w.hu, w.hv, 1, q_in=w.q_in,
                                  level=w.level)
    assert math.isclose(dt, dts2[0], rel_tol=1e-14)


def test_fp32_bench_configuration_at_full_size(river13m):
    w, mesh, om = river13m
    p = swe.swe_params_default("muscl", "fp32")           # the benchmark's path: the tile step, tiles of 256
    st = swe.State.from_workload(mesh, p, w)
    m0 = st.mass()[0]
    st.step(1, 0.9)
    dt = st.dt_history(1)[0]
    h, hu, hv = st.get_state()
    oh, *_ = _oracle_step(w, om, p.h_eps, dt)
    assert np.abs(h - oh).sum() <= 1e-6 * np.abs(oh).sum()
    st.step(48, 0.9)                                   # two CUDA-graph launches of 24 steps
    mass, clipped, bnd_in = st.mass()
    assert abs(mass - m0 - clipped - bnd_in) <= 1e-6 * m0
    assert st.time()[1] == 49
    hs = st.get_state()[0]
    st.close()
    pf = swe.swe_params_default("muscl", "fp32", kernel="split")
    sf = swe.State.from_workload(mesh, pf, w)
    sf.step(49, 0.9)
    assert np.array_equal(sf.get_state()[0], hs)
    sf.close()


# ---- the 4M river (2310 x 866 grid): WAF and MUSCL in FP32 against the FP64 path ----

@pytest.fixture(scope="module")
def river4m():
    B.build()
    swe.load_library()
    w = W.river(2310, 866)                          # 4,000,920 cells, same recipe as the 13M mesh
    assert w.n_cells == 4_000_920
    mesh = swe.Mesh.from_workload(w, "morton")
    yield w, mesh
    mesh.close()


def _wetting_front(w, h, thresh=1e-3):
    """Largest along-valley x of the cells that were dry at t = 0 and now hold more than 1 mm."""
    cx, _ = w.centroids()
    new = (h > thresh) & (w.h <= 0.0)
    return float(cx[new].max()) if new.any() else float("nan")


def _river_run(mesh, w, scheme, precision, steps=1000, dts=None, **kw):
    p = swe.swe_params_default(scheme, precision, **kw)
    p.h_eps = 1e-6                                  # the same dry threshold in both precisions
    s = swe.State.from_workload(mesh, p, w)
    m0 = s.mass()[0]
    if dts is None:
        s.step(steps, 0.9)
        dts = s.dt_history(steps)
    else:
        s.step_dt(dts)
    h = s.get_state()[0]
    mass, clip, bin_ = s.mass()
    s.close()
    return h, dts, abs(mass - m0 - clip - bin_) / m0


def _l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def test_river_4m_muscl_fp32_error_mass_and_front_against_fp64(river4m):
    """MUSCL FP32 bulk arithmetic after 1000 steps at matched time (the FP64 run's dt replayed),
    same h_eps: relative L1(h) <= 1e-4 over the mesh and 1e-3 of the change over the cells the
    flow has reached; mass drift <= 1e-6; the wetting front agrees to two cells."""
    w, mesh = river4m
    h64, dts, drift64 = _river_run(mesh, w, "muscl", "fp64")
    h32, _, drift32 = _river_run(mesh, w, "muscl", "fp32", dts=dts)
    l1 = _l1(h32, h64)
    changed = h64 != w.h
    f64, f32 = _wetting_front(w, h64), _wetting_front(w, h32)
    print(f"4M river muscl: FP32 vs FP64 L1(h) {l1:.3e}; front FP64 {f64:.1f} m, FP32 {f32:.1f} m; "
          f"mass drift FP32 {drift32:.2e}")
    assert l1 <= 1e-4, l1
    assert changed.sum() > 1000                     # the inflow has moved water
    assert np.abs(h32 - h64)[changed].sum() / np.abs(h64 - w.h)[changed].sum() <= 1e-3
    assert drift32 <= 1e-6 and drift64 <= 1e-12
    assert np.isfinite(f64) and abs(f32 - f64) <= 2 * 40000.0 / 2310


def test_river_4m_waf_fp32_against_fp64(river4m):
    """WAF with SUPERBEE switches its limiter where the local change of h crosses zero, so the
    round-off guard r_eps of the ratios decides some switches (reading R14): in FP64 alone,
    r_eps = 1e-6 instead of 1e-12 moves the result after 1000 steps by about as much as FP32 does.
    So: FP32's distance from FP64 is at most twice that FP64 sensitivity (and 3e-4); with the
    limiter off (phi = 1) FP32 follows FP64 to 3e-5 (its only switches are reading R18's tests
    for a dry side or a vacuum-forming edge, decided in each precision's arithmetic: 7e-6
    measured, 5e-8 before R18); the mass budget closes in both."""
    w, mesh = river4m
    h64, dts, drift64 = _river_run(mesh, w, "waf", "fp64")
    h64g, _, _ = _river_run(mesh, w, "waf", "fp64", dts=dts, r_eps=1e-6)
    h32, _, drift32 = _river_run(mesh, w, "waf", "fp32", dts=dts)
    l1, l1_guard = _l1(h32, h64), _l1(h64g, h64)
    print(f"4M river waf: FP32 vs FP64 L1(h) {l1:.3e}; FP64 r_eps 1e-6 vs 1e-12 {l1_guard:.3e}")
    assert l1 <= 3e-4 and l1 <= 2 * l1_guard, (l1, l1_guard)
    assert drift32 <= 1e-6 and drift64 <= 1e-12
    p64, dts1, _ = _river_run(mesh, w, "waf", "fp64", waf_limiter="phi1")
    p32, _, _ = _river_run(mesh, w, "waf", "fp32", dts=dts1, waf_limiter="phi1")
    print(f"4M river waf phi=1: FP32 vs FP64 L1(h) {_l1(p32, p64):.3e}")
    assert _l1(p32, p64) <= 3e-5


# ---- the 1M partial dam break (1000 x 500 squares): FP64 against the oracle at full size ----

@pytest.fixture(scope="module")
def dam1m():
    B.build()
    swe.load_library()
    w = W.partial_dam_break()                       # 1,000,000 cells, ~30 % dry, breach, n = 0.03
    assert w.n_cells == 1_000_000
    om = oracle.Mesh(w.nodes, w.tris, w.bnd_edges, w.bnd_tag, w.cut_edges)
    yield w, om


@pytest.mark.parametrize("scheme,kernel", [("muscl", "split"), ("muscl", "fused"), ("waf", "split")])
def test_fp64_partial_dam_break_1m_against_oracle(dam1m, scheme, kernel):
    """100 steps at full size with the oracle's own time steps replayed: 1e-9 (the stated bar)."""
    w, om = dam1m
    o = oracle.opts(scheme, threads=os.cpu_count() or 1)
    oh, ohu, ohv, dts, d = oracle.run(om, o, w.z, w.nman, w.h, w.hu, w.hv, 100, q_in=w.q_in, level=w.level)
    m = swe.Mesh.from_workload(w, "morton")
    st = swe.State.from_workload(m, swe.swe_params_default(scheme, "fp64", kernel=kernel), w)
    st.step_dt(dts)
    h, hu, hv = st.get_state()
    st.close()
    m.close()
    qs = max(np.abs(ohu).max(), np.abs(ohv).max())
    assert np.abs(h - oh).max() <= 1e-9 * np.abs(oh).max()
    assert np.abs(hu - ohu).max() <= 1e-9 * qs
    assert np.abs(hv - ohv).max() <= 1e-9 * qs
