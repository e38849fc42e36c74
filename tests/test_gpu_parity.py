"""CUDA path against the FP64 oracle, element by element, through the C ABI.

FP64: relative max error <= 1e-12 after one step and <= 1e-9 after 100 steps
(the oracle and the kernels evaluate the same algorithm; they differ only in
rounding order and fused multiply-adds).  FP32: relative L1 error of h and the
mass drift are bounded (see each test).  Integer work (the mesh) is compared
bit for bit in test_abi.py.
"""
import math

import numpy as np
import pytest

from gpu_common import rel_l1, rel_max, run_gpu, run_oracle, state_errors
from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe
from paper_2307_16758_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    swe.load_library()


def _pdb(nx=90, ny=44, seed=11):
    return W.partial_dam_break(nx=nx, ny=ny, spacing=1.0, n_gauss=30, seed=seed)


def _river(nx=100, ny=38, seed=21, q=1500.0):
    return W.river(nx=nx, ny=ny, seed=seed, q_in=q)


# ---- FP64 parity ------------------------------------------------------------

@pytest.mark.parametrize("scheme", ["hllc", "muscl", "waf"])
def test_fp64_one_step_dam_break_2000_cells(scheme):
    w = W.dam_break_1d()                        # 2000 cells: 7 full blocks and a ragged tail
    g = run_gpu(w, scheme, steps=1)
    o = run_oracle(w, scheme, steps=1)
    assert max(state_errors(g, o)) <= 1e-12
    assert math.isclose(g["t"], o["t"], rel_tol=1e-15)


def test_fp64_hllc_config1_200_steps_cfl():
    """First-order HLLC, 2000 cells, CFL 0.9, 200 steps."""
    w = W.dam_break_1d()
    g100, o100 = run_gpu(w, "hllc", steps=100), run_oracle(w, "hllc", steps=100)
    assert max(state_errors(g100, o100)) <= 1e-9
    assert math.isclose(g100["t"], o100["t"], rel_tol=1e-12)
    g, o = run_gpu(w, "hllc", steps=200), run_oracle(w, "hllc", steps=200)
    assert max(state_errors(g, o)) <= 1e-9
    assert g["steps"] == 200


KERNELS = ["split", "fused"]
# the one-pass tile step ("fused") runs LSQ MUSCL and first-order HLLC; WAF runs the split kernels
SCHEME_KERNELS = [("hllc", "split"), ("hllc", "fused"), ("muscl", "split"), ("muscl", "fused"), ("waf", "split")]


@pytest.mark.parametrize("scheme,kernel", SCHEME_KERNELS)
def test_fp64_partial_dam_break(scheme, kernel):
    """Jittered mesh, Gaussian bed, ~30 % dry, breach, Manning: 1 and 100 steps."""
    w = _pdb()
    g1, o1 = run_gpu(w, scheme, steps=1, kernel=kernel), run_oracle(w, scheme, steps=1)
    assert max(state_errors(g1, o1)) <= 1e-12
    o = run_oracle(w, scheme, steps=100)
    g = run_gpu(w, scheme, dt=o["dts"], kernel=kernel)
    errs = state_errors(g, o)
    assert max(errs) <= 1e-9, errs
    gc = run_gpu(w, scheme, steps=100, kernel=kernel)
    assert math.isclose(gc["t"], o["t"], rel_tol=1e-9)


@pytest.mark.parametrize("scheme,kernel", SCHEME_KERNELS)
def test_fp64_river_inflow_level_friction(scheme, kernel):
    w = _river()
    o = run_oracle(w, scheme, steps=100)
    g = run_gpu(w, scheme, dt=o["dts"], kernel=kernel)
    assert max(state_errors(g, o)) <= 1e-9
    assert math.isclose(g["bnd_in"], o["bnd_in"], rel_tol=1e-9)


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp64_heun(kernel):
    w = _pdb(60, 30)
    o = run_oracle(w, "muscl", steps=40, time_scheme="heun")
    g = run_gpu(w, "muscl", dt=o["dts"], time_scheme="heun", kernel=kernel)
    assert max(state_errors(g, o)) <= 1e-9


@pytest.mark.parametrize("kernel,block", [("split", 64), ("split", 128), ("split", 512),
                                          ("fused", 64), ("fused", 128), ("fused", 256)])
def test_fp64_block_sizes(block, kernel):
    """Block (and, for the tile step, tile) sizes; 33x17 squares = 1122 cells, ragged tail."""
    w = _pdb(33, 17)
    o = run_oracle(w, "muscl", steps=10)
    g = run_gpu(w, "muscl", dt=o["dts"], block=block, kernel=kernel)
    assert max(state_errors(g, o)) <= 1e-11


def test_block_above_the_kernel_limit_is_rejected():
    """FP64 tiles of 1024 threads need more registers than a block has: a host error."""
    w = _pdb(20, 10)
    with pytest.raises(swe.SweError) as e:
        run_gpu(w, "muscl", "fp64", steps=1, kernel="fused", block=1024)
    assert e.value.code == -1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme", ["muscl", "hllc"])
def test_split_and_fused_kernels_agree_bitwise(precision, scheme):
    """The one-pass tile step runs the same per-edge and per-cell code as the split kernels, so
    every tile size gives the split kernels' bits (CFL steps, inflow, level, friction, wet/dry)."""
    w = _river(90, 34)
    a = run_gpu(w, scheme, precision, steps=50, kernel="split")
    for block in (64, 128, 256) + ((512,) if precision == "fp32" else ()):
        b = run_gpu(w, scheme, precision, steps=50, kernel="fused", block=block)
        for k in ("h", "hu", "hv"):
            assert np.array_equal(a[k], b[k]), (block, k)


# ---- invariants on the GPU ----------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme,kernel", SCHEME_KERNELS)
def test_lake_at_rest_bitwise(precision, scheme, kernel):
    w = W.partial_dam_break(nx=80, ny=40, spacing=1.0, n_gauss=40, breach=False, seed=9)
    w.bnd_tag = np.full(len(w.bnd_edges), W.tag(W.LEVEL), np.int32)
    w.level = np.array([2.0])
    g = run_gpu(w, scheme, precision, steps=1000, kernel=kernel)
    assert np.array_equal(g["h"], w.h)
    assert not g["hu"].any() and not g["hv"].any()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
@pytest.mark.parametrize("scheme", ["hllc", "muscl", "waf"])
def test_mass_conservation(precision, tol, scheme):
    w = _pdb()
    m0 = run_oracle(w, scheme, steps=0)["mass0"]
    g = run_gpu(w, scheme, precision, steps=300)
    assert abs(g["mass"] - m0 - g["clipped"]) <= tol * m0


def test_mass_budget_with_inflow():
    w = _river()
    o = run_oracle(w, "muscl", steps=0)
    g = run_gpu(w, "muscl", "fp64", steps=300)
    assert abs(g["mass"] - o["mass0"] - g["clipped"] - g["bnd_in"]) <= 1e-12 * o["mass0"]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_renumbering_is_bitwise_invisible(precision, kernel):
    """Morton, RCM and the original order give the same bits (cf. Sec. 6.3.1)."""
    w = _pdb(50, 24)
    ref = run_gpu(w, "muscl", precision, steps=60, reorder="none", kernel=kernel)
    for r in ("morton", "rcm"):
        g = run_gpu(w, "muscl", precision, steps=60, reorder=r, kernel=kernel)
        for k in ("h", "hu", "hv"):
            assert np.array_equal(g[k], ref[k]), (r, k)
        assert g["t"] == ref["t"]


# ---- FP32 against the FP64 oracle ----------------------------------------------

@pytest.mark.parametrize("scheme,kernel", SCHEME_KERNELS)
def test_fp32_error_against_oracle(scheme, kernel):
    """FP32 state and fluxes (FP64 mass and time): relative L1 of h after 1000
    replayed steps <= 1e-4, mass drift <= 1e-6 (same h_eps on both sides)."""
    w = _river(80, 30)
    o = run_oracle(w, scheme, steps=1000, h_eps=1e-4, r_eps=1e-6)
    g = run_gpu(w, scheme, "fp32", dt=o["dts"], kernel=kernel)
    assert rel_l1(g["h"], o["h"]) <= 1e-4
    drift = abs(g["mass"] - o["mass0"] - g["clipped"] - g["bnd_in"]) / o["mass0"]
    assert drift <= 1e-6


# ---- edge cases and error paths ------------------------------------------------

def test_single_triangle_and_tiny_meshes():
    nodes = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    n = 1
    w = W.Workload("one", nodes, np.array([[0, 1, 2]], np.int32), np.zeros((0, 2), np.int32),
                   np.zeros(0, np.int32), np.zeros((0, 2), np.int32), np.zeros(n), np.zeros(n),
                   np.ones(n), np.zeros(n), np.zeros(n))
    for kernel in KERNELS:
        g = run_gpu(w, "muscl", steps=5, kernel=kernel)
        assert np.array_equal(g["h"], [1.0]) and g["hu"][0] == 0 and g["hv"][0] == 0
    for nx in (1, 2, 129):                       # 2, 4 and 258 cells (one block plus a tail)
        w2 = W.dam_break_1d(nx, 1, float(nx), 1.0, 1.0, 0.5, x_dam=nx / 2.0 + 0.1)
        o = run_oracle(w2, "muscl", steps=3)
        for kernel in KERNELS:
            g2 = run_gpu(w2, "muscl", dt=o["dts"], kernel=kernel)
            assert max(state_errors(g2, o)) <= 1e-12, (nx, kernel)


def test_non_finite_input_is_reported():
    w = W.dam_break_1d(20, 2, 20.0, 2.0)
    w.h = w.h.copy()
    w.h[3] = np.nan
    p = swe.swe_params_default("hllc", "fp64")
    m = swe.Mesh.from_workload(w)
    s = swe.State.from_workload(m, p, w)
    s.step_dt([0.01])
    with pytest.raises(swe.SweError) as e:
        s.sync()
    assert e.value.code == -5


def test_all_dry_domain_is_reported():
    w = W.dam_break_1d(20, 2, 20.0, 2.0, 0.0, 0.0)
    p = swe.swe_params_default("hllc", "fp64")
    m = swe.Mesh.from_workload(w)
    s = swe.State.from_workload(m, p, w)
    s.step(1, 0.9)
    with pytest.raises(swe.SweError) as e:
        s.sync()
    assert e.value.code == -4


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tile_states_with_different_plans_coexist(precision):
    """Two states on the tile step whose plans need different shared memory (tiles of 512 and of
    128 cells): configuring the smaller one after the larger must not stop the larger one from
    launching, and both keep the split kernels' bits."""
    w = _pdb(60, 30)
    m = swe.Mesh.from_workload(w)
    big_tile = 512 if precision == "fp32" else 256
    big = swe.State.from_workload(m, swe.swe_params_default("muscl", precision, kernel="fused", block=big_tile), w)
    small = swe.State.from_workload(m, swe.swe_params_default("muscl", precision, kernel="fused", block=128), w)
    ref = swe.State.from_workload(m, swe.swe_params_default("muscl", precision, kernel="split"), w)
    for st in (big, small, ref):
        st.step(12, 0.9)
    r = ref.get_state()
    for st in (big, small):
        for x, y in zip(st.get_state(), r):
            assert np.array_equal(x, y)
    for st in (big, small, ref):
        st.close()
    m.close()


def test_set_state_round_trip_and_resume():
    w = _pdb(40, 20)
    p = swe.swe_params_default("muscl", "fp64")
    m = swe.Mesh.from_workload(w)
    a = swe.State.from_workload(m, p, w)
    a.step(30, 0.9)
    mid = a.get_state()
    a.step(30, 0.9)
    end_a = a.get_state()
    b = swe.State.from_workload(m, p, w)
    b.set_state(*mid)
    b.step(30, 0.9)
    end_b = b.get_state()
    for x, y in zip(end_a, end_b):
        assert np.array_equal(x, y)


# ---- CFL forms (R11: the printed global form, and the local form as an option) ----

@pytest.mark.parametrize("kernel,time_scheme", [("split", "euler"), ("fused", "euler"), ("split", "heun")])
def test_fp64_local_cfl_steps_match_the_oracle(kernel, time_scheme):
    """CFL-driven steps (not replayed) on a jittered mesh with a breach: the GPU's time steps and
    state follow the oracle's under the per-cell form, which differs from the global one there."""
    w = _pdb()
    o = run_oracle(w, "muscl", steps=40, cfl_mode="local", time_scheme=time_scheme)
    og = run_oracle(w, "muscl", steps=1, time_scheme=time_scheme)
    assert o["dts"][0] > og["dts"][0] * (1 + 1e-9)        # the local form takes a longer first step
    p = swe.swe_params_default("muscl", "fp64", kernel=kernel, cfl_mode="local", time_scheme=time_scheme)
    m = swe.Mesh.from_workload(w, "morton")
    s = swe.State.from_workload(m, p, w)
    s.step(40, 0.9)
    dts = s.dt_history(40)
    h, hu, hv = s.get_state()
    s.close()
    m.close()
    assert np.allclose(dts, o["dts"], rtol=1e-12, atol=0)
    assert max(state_errors(dict(h=h, hu=hu, hv=hv), o)) <= 1e-9


def test_fp32_local_cfl_takes_the_oracle_first_step():
    w = _pdb()
    o = run_oracle(w, "muscl", steps=1, cfl_mode="local", h_eps=1e-4, r_eps=1e-6)
    g = swe.swe_params_default("muscl", "fp32", cfl_mode="local")
    m = swe.Mesh.from_workload(w, "morton")
    s = swe.State.from_workload(m, g, w)
    s.step(1, 0.9)
    dt = s.dt_history(1)[0]
    s.close()
    m.close()
    assert math.isclose(dt, o["dts"][0], rel_tol=1e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mass_is_the_correctly_rounded_sum(precision):
    """swe_mass sums area_i * h_i with compensation: within a few ulp of the exactly rounded sum."""
    w = _river(160, 60)
    m = swe.Mesh.from_workload(w, "morton")
    a = m.export()
    s = swe.State.from_workload(m, swe.swe_params_default("muscl", precision), w)
    s.step(30, 0.9)
    h = s.get_state()[0]
    mass = s.mass()[0]
    s.close()
    m.close()
    exact = math.fsum((a["area"] * h[a["perm"]]).tolist())
    assert abs(mass - exact) <= 4 * np.spacing(exact), (mass, exact)


# ---- the clipping flag --------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_clipping_flag_follows_the_clipped_mass(precision):
    """swe_flags: SWE_FLAG_CLIPPED is set exactly when a negative depth was clipped (the clipped
    mass of swe_mass is then positive); a lake at rest sets no flag."""
    rest = W.partial_dam_break(nx=40, ny=20, spacing=1.0, n_gauss=20, breach=False, seed=9)
    p = swe.swe_params_default("muscl", precision)
    m = swe.Mesh.from_workload(rest)
    s = swe.State.from_workload(m, p, rest)
    s.step(50, 0.9)
    assert s.flags() == 0
    s.close()
    m.close()
    w = W.dam_break_1d(h_right=0.0)            # dry-bed dam break: MUSCL with Euler clips at the front
    m = swe.Mesh.from_workload(w)
    s = swe.State.from_workload(m, p, w)
    seen = False
    for _ in range(10):
        s.step(20, 0.9)
        clipped = s.mass()[1]
        f = s.flags()
        assert bool(f & swe.FLAG_CLIPPED) == (clipped > 0), (f, clipped)
        assert not f & (swe.FLAG_NONFINITE | swe.FLAG_DRY)
        seen = seen or clipped > 0
    assert seen, "the dry-bed dam break clipped no depth"
    s.close()
    m.close()
