"""Batched ensemble and autotuner on the GPU (the ensemble row of the hot path).

An ensemble advances independent river scenarios of different sizes, each with
its own inflow, Manning coefficients, initial level and CFL time step, in one
batched launch per step.  It runs the same per-mesh device code as a state
stepped alone, so every member must come out bit for bit as if it had been
stepped alone; the autotuner must leave the simulation untouched.
"""
import math

import numpy as np
import pytest

from gpu_common import run_oracle, state_errors
from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe
from paper_2307_16758_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    swe.load_library()


def _scenarios():
    """Four members of uneven size (900 to 6000 cells), own Q, n and level."""
    specs = [(30, 15, 1200.0, 0.02, 0.4), (60, 22, 5000.0, 0.05, 0.6), (25, 18, 2500.0, 0.03, 0.5),
             (100, 30, 9000.0, 0.06, 0.35)]
    return [W.river(nx, ny, seed=100 + k, q_in=q, n_channel=nc, n_floodplain=min(2 * nc, 0.1),
                    level_quantile=lv) for k, (nx, ny, q, nc, lv) in enumerate(specs)]


def _alone(w, p, steps):
    m = swe.Mesh.from_workload(w)
    st = swe.State.from_workload(m, p, w)
    st.step(steps, 0.9)
    out = st.get_state(), st.time(), st.mass()
    st.close()
    m.close()
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("kernel,scheme", [("split", "muscl"), ("fused", "muscl"), ("split", "waf"),
                                           ("split", "hllc"), ("fused", "hllc"), ("split", "muscl_edge")])
def test_ensemble_members_match_stepping_alone(kernel, scheme, precision):
    ws = _scenarios()
    p = swe.swe_params_default(scheme, precision, kernel=kernel)
    meshes = [swe.Mesh.from_workload(w) for w in ws]
    states = [swe.State.from_workload(m, p, w) for m, w in zip(meshes, ws)]
    ens = swe.Ensemble(states)
    ens.step(40, 0.9)
    ens.step(13, 0.9)                 # 53 steps: not a multiple of the 6-step launch pattern
    ens.sync()
    for w, st in zip(ws, states):
        (h, hu, hv), (t, k), (mass, clip, bin_) = _alone(w, p, 53)
        gh, ghu, ghv = st.get_state()
        assert np.array_equal(gh, h) and np.array_equal(ghu, hu) and np.array_equal(ghv, hv)
        gt, gk = st.time()
        assert gt == t and gk == k == 53
    # the members still work on their own afterwards; the ensemble then refuses to run members
    # that are out of step with one another
    states[1].step(7, 0.9)
    assert states[1].time()[1] == 60
    with pytest.raises(swe.SweError) as e:
        ens.step(1, 0.9)
    assert e.value.code == -1


def test_ensemble_fp64_matches_the_oracle():
    ws = _scenarios()[:2]
    p = swe.swe_params_default("muscl", "fp64")
    meshes = [swe.Mesh.from_workload(w) for w in ws]
    states = [swe.State.from_workload(m, p, w) for m, w in zip(meshes, ws)]
    ens = swe.Ensemble(states)
    ens.step(60, 0.9)
    ens.sync()
    for w, st in zip(ws, states):
        o = run_oracle(w, "muscl", steps=60)
        h, hu, hv = st.get_state()
        assert max(state_errors(dict(h=h, hu=hu, hv=hv), o)) <= 1e-9
        assert math.isclose(st.time()[0], o["t"], rel_tol=1e-9)


def test_ensemble_rejects_mixed_members():
    ws = _scenarios()[:2]
    meshes = [swe.Mesh.from_workload(w) for w in ws]
    a = swe.State.from_workload(meshes[0], swe.swe_params_default("muscl", "fp32", kernel="split"), ws[0])
    b = swe.State.from_workload(meshes[1], swe.swe_params_default("muscl", "fp32", kernel="fused"), ws[1])
    with pytest.raises(swe.SweError) as e:
        swe.Ensemble([a, b])
    assert e.value.code == -1
    c = swe.State.from_workload(meshes[1], swe.swe_params_default("muscl", "fp32", kernel="split"), ws[1])
    c.step(1, 0.9)                    # another step phase
    with pytest.raises(swe.SweError):
        swe.Ensemble([a, c])
    with pytest.raises(swe.SweError) as e:
        swe.Ensemble([a, a])          # one state listed twice
    assert e.value.code == -1


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotune_leaves_the_simulation_unchanged(precision):
    w = W.river(90, 34, seed=7, q_in=3000.0)
    p = swe.swe_params_default("muscl", precision)
    m = swe.Mesh.from_workload(w)
    a = swe.State.from_workload(m, p, w)
    a.step(10, 0.9)
    kernel, block, ms = a.autotune(m, trial_steps=4)
    assert kernel in ("split", "fused") and block in (128, 256, 512) and ms > 0
    assert a.time()[1] == 10
    assert a.info()[2] == block
    a.step(20, 0.9)
    b = swe.State.from_workload(m, p, w)
    b.step(30, 0.9)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert a.time() == b.time()


def test_ensemble_autotune():
    ws = _scenarios()
    p = swe.swe_params_default("muscl", "fp32")
    meshes = [swe.Mesh.from_workload(w) for w in ws]
    states = [swe.State.from_workload(m, p, w) for m, w in zip(meshes, ws)]
    ens = swe.Ensemble(states)
    ens.step(5, 0.9)
    kernel, block, ms = ens.autotune(meshes, trial_steps=3)
    assert ms > 0
    ens.step(15, 0.9)
    ens.sync()
    for w, st in zip(ws, states):
        (h, hu, hv), (t, k), _ = _alone(w, p, 20)
        assert np.array_equal(st.get_state()[0], h)
        assert st.time()[1] == 20


@pytest.mark.parametrize("scheme", ["hllc", "muscl", "waf", "muscl_edge"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ensemble_autotune_every_scheme_and_block_limit(scheme, precision):
    """Every candidate the ensemble autotuner keeps launches (the batched kernels have their own
    register counts and so their own largest block), and the result is still stepping alone."""
    ws = _scenarios()[:2]
    p = swe.swe_params_default(scheme, precision)
    meshes = [swe.Mesh.from_workload(w) for w in ws]
    states = [swe.State.from_workload(m, p, w) for m, w in zip(meshes, ws)]
    ens = swe.Ensemble(states)
    kernel, block, ms = ens.autotune(meshes, trial_steps=2)
    assert ms > 0 and block in (128, 256, 512)
    ens.step(12, 0.9)
    ens.sync()
    p_alone = swe.swe_params_default(scheme, precision, kernel=kernel, block=block)
    for w, st in zip(ws, states):
        (h, hu, hv), (t, k), _ = _alone(w, p_alone, 12)
        assert np.array_equal(st.get_state()[0], h) and k == 12
    # 1024 threads: refused where a kernel cannot launch them, else the same bits as stepping alone
    big = swe.swe_params_default(scheme, precision, kernel="split", block=1024)
    try:
        members = [swe.State.from_workload(m, big, w) for m, w in zip(meshes, ws)]
        e2 = swe.Ensemble(members)
        e2.step(3, 0.9)
        e2.sync()
    except swe.SweError as err:
        assert err.code == -1          # an argument error, not a failed launch
        return
    for w, st in zip(ws, members):
        (h, hu, hv), (t, k), _ = _alone(w, big, 3)
        assert np.array_equal(st.get_state()[0], h)
