"""Full-size checks on the benchmark workload (13,004,160-cell river mesh).

The oracle can afford one full-mesh step, so the FP64 path is compared with it
cell by cell at full size (one step, 1e-12).  The FP32 benchmark configuration
(split kernels, block 256, CUDA graphs, CFL 0.9) is checked through properties
that hold at any size: its one-step result against the same oracle step (same
h_eps), the mass budget, and that the fused kernel gives the same bits.
"""
import math

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
    p = swe.swe_params_default("muscl", "fp32")           # split kernels, block 256: the benchmark's path
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
    pf = swe.swe_params_default("muscl", "fp32", kernel="fused")
    sf = swe.State.from_workload(mesh, pf, w)
    sf.step(49, 0.9)
    assert np.array_equal(sf.get_state()[0], hs)
    sf.close()
