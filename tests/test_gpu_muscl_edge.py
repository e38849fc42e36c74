"""The paper's own MUSCL (Sec. 6.2.3: slopes along each edge from the upwind means of the two
other neighbours, beta-limited) on the GPU against the FP64 oracle.

The oracle writes the two sides of an edge with the printed left and right formulas; the kernels
reconstruct each cell's own faces (the limiter's symmetry makes the right formula the left one
seen from R), so FP64 parity also checks that step.  Tolerances as for the other schemes:
1e-12 after one step, 1e-9 after 100 steps; invariants bit for bit.
"""
import math

import numpy as np
import pytest

from gpu_common import rel_l1, run_gpu, run_oracle, state_errors
from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe
from paper_2307_16758_gb300 import workloads as W

pytestmark = pytest.mark.gpu
S = "muscl_edge"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    swe.load_library()


def _pdb(nx=90, ny=44, seed=11):
    return W.partial_dam_break(nx=nx, ny=ny, spacing=1.0, n_gauss=30, seed=seed)


@pytest.mark.parametrize("beta", [1.0, 1.5, 2.0])
def test_fp64_one_step_and_100_steps(beta):
    for w in (W.dam_break_1d(), _pdb()):
        g1, o1 = run_gpu(w, S, steps=1, muscl_beta=beta), run_oracle(w, S, steps=1, beta=beta)
        assert max(state_errors(g1, o1)) <= 1e-12
        o = run_oracle(w, S, steps=100, beta=beta)
        g = run_gpu(w, S, dt=o["dts"], muscl_beta=beta)
        assert max(state_errors(g, o)) <= 1e-9
        gc = run_gpu(w, S, steps=100, muscl_beta=beta)
        assert math.isclose(gc["t"], o["t"], rel_tol=1e-9)


def test_fp64_river_inflow_level_friction_and_heun():
    w = W.river(nx=100, ny=38, seed=21, q_in=1500.0)
    o = run_oracle(w, S, steps=100)
    g = run_gpu(w, S, dt=o["dts"])
    assert max(state_errors(g, o)) <= 1e-9
    assert math.isclose(g["bnd_in"], o["bnd_in"], rel_tol=1e-9)
    w = _pdb(60, 30)
    o = run_oracle(w, S, steps=40, time_scheme="heun")
    g = run_gpu(w, S, dt=o["dts"], time_scheme="heun")
    assert max(state_errors(g, o)) <= 1e-9


@pytest.mark.parametrize("block", [64, 128, 512])
def test_fp64_block_sizes(block):
    w = _pdb(33, 17)                                  # 1122 cells: ragged tail at every block size
    o = run_oracle(w, S, steps=10)
    g = run_gpu(w, S, dt=o["dts"], block=block)
    assert max(state_errors(g, o)) <= 1e-11


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lake_at_rest_bitwise(precision):
    w = W.partial_dam_break(nx=80, ny=40, spacing=1.0, n_gauss=40, breach=False, seed=9)
    w.bnd_tag = np.full(len(w.bnd_edges), W.tag(W.LEVEL), np.int32)
    w.level = np.array([2.0])
    g = run_gpu(w, S, precision, steps=1000)
    assert np.array_equal(g["h"], w.h)
    assert not g["hu"].any() and not g["hv"].any()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_mass_conservation(precision, tol):
    w = _pdb()
    m0 = run_oracle(w, S, steps=0)["mass0"]
    g = run_gpu(w, S, precision, steps=300)
    assert abs(g["mass"] - m0 - g["clipped"]) <= tol * m0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_renumbering_is_bitwise_invisible(precision):
    w = _pdb(50, 24)
    ref = run_gpu(w, S, precision, steps=60, reorder="none")
    for r in ("morton", "rcm"):
        g = run_gpu(w, S, precision, steps=60, reorder=r)
        for k in ("h", "hu", "hv"):
            assert np.array_equal(g[k], ref[k]), (r, k)


def test_fp32_error_against_oracle():
    """FP32 state and fluxes, 1000 replayed steps, same h_eps: relative L1(h) <= 1e-4."""
    w = W.river(80, 30, seed=21, q_in=1500.0)
    o = run_oracle(w, S, steps=1000, h_eps=1e-4, r_eps=1e-6)
    g = run_gpu(w, S, "fp32", dt=o["dts"])
    assert rel_l1(g["h"], o["h"]) <= 1e-4
    assert abs(g["mass"] - o["mass0"] - g["clipped"] - g["bnd_in"]) <= 1e-6 * o["mass0"]


def test_fused_kernel_and_bad_beta_are_rejected():
    w = _pdb(20, 10)
    for kw in (dict(kernel="fused"), dict(muscl_beta=0.5), dict(muscl_beta=2.5)):
        with pytest.raises(swe.SweError) as e:
            run_gpu(w, S, "fp64", steps=1, **kw)
        assert e.value.code == -1


def test_autotune_keeps_to_the_split_kernels():
    w = W.river(90, 34, seed=7, q_in=3000.0)
    p = swe.swe_params_default(S, "fp32")
    m = swe.Mesh.from_workload(w)
    a = swe.State.from_workload(m, p, w)
    a.step(5, 0.9)
    kernel, block, ms = a.autotune(m, trial_steps=3)
    assert kernel == "split" and ms > 0
    a.close()
    m.close()
