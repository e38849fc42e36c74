"""WAF with its ratios on the free surface (SWE_WAF_RATIO_SURFACE, the default reading R4) on the GPU
against the FP64 oracle, with the same bars as the cell-depth ratio (option R17), plus the properties
that pin it: the same bits as the depth ratio on a flat bed, an exact lake at rest, mass, and a
bounded run on a river where the depth ratio grows spurious speeds."""
import numpy as np
import pytest

from gpu_common import rel_l1, run_gpu, run_oracle, state_errors
from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe
from paper_2307_16758_gb300 import workloads as W

pytestmark = pytest.mark.gpu
S = dict(waf_ratio="surface")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    swe.load_library()


@pytest.mark.parametrize("workload", ["pdb", "river"])
def test_fp64_one_step_and_100_steps(workload):
    w = W.partial_dam_break(nx=90, ny=44, spacing=1.0, n_gauss=30, seed=11) if workload == "pdb" \
        else W.river(nx=100, ny=38, seed=21, q_in=1500.0)
    g1, o1 = run_gpu(w, "waf", steps=1, **S), run_oracle(w, "waf", steps=1, **S)
    assert max(state_errors(g1, o1)) <= 1e-12
    o = run_oracle(w, "waf", steps=100, **S)
    g = run_gpu(w, "waf", dt=o["dts"], **S)
    assert max(state_errors(g, o)) <= 1e-9
    od = run_oracle(w, "waf", dt=o["dts"], waf_ratio="depth")
    assert max(state_errors(g, od)) > 1e-7           # over a bed the surface ratio is a different scheme


@pytest.mark.parametrize("limiter", ["minbee", "vanleer", "phi1"])
def test_other_limiters_match_the_oracle(limiter):
    """WAF with A(r, c) = 1 - (1 - |c|) phi(r) for MINBEE, van Leer and phi = 1 (Sec. 6.2.2),
    with the edges that have no wet star region on their HLLC flux (R18): a river with dry banks
    and an inflow, FP64 against the oracle after 1 and 100 replayed steps."""
    w = W.river(100, 38, seed=21, q_in=1500.0)
    g1, o1 = run_gpu(w, "waf", steps=1, waf_limiter=limiter), run_oracle(w, "waf", steps=1, waf_limiter=limiter)
    assert max(state_errors(g1, o1)) <= 1e-12
    o = run_oracle(w, "waf", steps=100, waf_limiter=limiter)
    g = run_gpu(w, "waf", dt=o["dts"], waf_limiter=limiter)
    assert max(state_errors(g, o)) <= 1e-9
    osb = run_oracle(w, "waf", dt=o["dts"])
    assert max(state_errors(g, osb)) > 1e-7              # a different limiter, a different scheme


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_flat_bed_gives_the_depth_ratio_bits(precision):
    w = W.dam_break_1d(120, 8, 10.0, 1.0, 1.0, 0.5, x_dam=5.0)
    a = run_gpu(w, "waf", precision, steps=150, waf_ratio="depth")
    b = run_gpu(w, "waf", precision, steps=150, **S)
    for k in ("h", "hu", "hv"):
        assert np.array_equal(a[k], b[k])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lake_at_rest_bitwise(precision):
    w = W.partial_dam_break(nx=80, ny=40, spacing=1.0, n_gauss=40, breach=False, seed=9)
    w.bnd_tag = np.full(len(w.bnd_edges), W.tag(W.LEVEL), np.int32)
    w.level = np.array([2.0])
    g = run_gpu(w, "waf", precision, steps=1000, **S)
    assert np.array_equal(g["h"], w.h)
    assert not g["hu"].any() and not g["hv"].any()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_mass_conservation(precision, tol):
    w = W.partial_dam_break(nx=90, ny=44, spacing=1.0, n_gauss=30, seed=11)
    m0 = run_oracle(w, "waf", steps=0)["mass0"]
    g = run_gpu(w, "waf", precision, steps=300, **S)
    assert abs(g["mass"] - m0 - g["clipped"]) <= tol * m0


def test_fp32_error_against_the_oracle():
    w = W.river(80, 30, seed=21, q_in=1500.0)
    o = run_oracle(w, "waf", steps=100, h_eps=1e-4, r_eps=1e-6, **S)
    g = run_gpu(w, "waf", "fp32", dt=o["dts"], **S)
    assert rel_l1(g["h"], o["h"]) <= 1e-5


def test_ensemble_members_match_stepping_alone():
    ws = [W.river(40, 16, seed=41, q_in=2000.0), W.river(60, 22, seed=42, q_in=5000.0)]
    p = swe.swe_params_default("waf", "fp32", **S)
    meshes = [swe.Mesh.from_workload(w) for w in ws]
    states = [swe.State.from_workload(m, p, w) for m, w in zip(meshes, ws)]
    ens = swe.Ensemble(states)
    ens.step(30, 0.9)
    ens.sync()
    for w, st in zip(ws, states):
        m = swe.Mesh.from_workload(w)
        alone = swe.State.from_workload(m, p, w)
        alone.step(30, 0.9)
        for x, y in zip(st.get_state(), alone.get_state()):
            assert np.array_equal(x, y)
        alone.close()
        m.close()


@pytest.mark.parametrize("kw", [dict(scheme="waf", kernel="fused"), dict(scheme="waf", waf_ratio=2)])
def test_unsupported_combinations_are_rejected(kw):
    kw = dict(kw)
    scheme = kw.pop("scheme")
    kw.setdefault("waf_ratio", "surface")
    w = W.partial_dam_break(nx=20, ny=10, spacing=1.0, n_gauss=8, seed=3)
    with pytest.raises(swe.SweError) as e:
        run_gpu(w, scheme, "fp64", steps=1, **kw)
    assert e.value.code == -1


def test_bounded_speeds_on_a_river():
    """120,000-cell river, 3000 FP32 CFL steps: the free-surface ratio (the default reading) keeps
    every speed below 10 m/s (the cell-depth ratio passes 10^4 m/s on this run in the oracle by
    step 1000)."""
    w = W.river(400, 150)
    m = swe.Mesh.from_workload(w)
    st = swe.State.from_workload(m, swe.swe_params_default("waf", "fp32", **S), w)
    worst = 0.0
    for _ in range(30):
        st.step(100, 0.9)
        h, hu, hv = st.get_state()
        u = np.where(h > 1e-3, np.hypot(hu, hv) / np.maximum(h, 1e-300), 0.0)
        worst = max(worst, float(u.max()))
    st.close()
    m.close()
    assert worst < 10.0, worst


def test_autotune_stays_on_the_split_kernels():
    w = W.river(90, 34, seed=7, q_in=3000.0)
    m = swe.Mesh.from_workload(w)
    a = swe.State.from_workload(m, swe.swe_params_default("waf", "fp32", **S), w)
    kernel, block, ms = a.autotune(m, trial_steps=4)
    assert kernel == "split" and ms > 0
    a.close()
    m.close()
