"""Second-order hydrostatic reconstruction (the paper's future work, Sec. 7; reading R16) on the GPU
against the FP64 oracle: h reconstructed like eta, the face bed from their difference, the centred
bed source in the own-side pressure term.  Same bars as the other schemes."""
import numpy as np
import pytest

from gpu_common import rel_l1, run_gpu, run_oracle, state_errors
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


@pytest.mark.parametrize("workload", ["pdb", "river"])
def test_fp64_one_step_and_100_steps(workload):
    w = _pdb() if workload == "pdb" else W.river(nx=100, ny=38, seed=21, q_in=1500.0)
    g1, o1 = run_gpu(w, "muscl", steps=1, hr_order=2), run_oracle(w, "muscl", steps=1, hr_order=2)
    assert max(state_errors(g1, o1)) <= 1e-12
    o = run_oracle(w, "muscl", steps=100, hr_order=2)
    g = run_gpu(w, "muscl", dt=o["dts"], hr_order=2)
    assert max(state_errors(g, o)) <= 1e-9
    # and the second-order reconstruction does change the result on these beds
    o1st = run_oracle(w, "muscl", dt=o["dts"])
    assert max(state_errors(g, o1st)) > 1e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", ["wall", "level"])
def test_lake_at_rest_bitwise(precision, bc):
    w = W.partial_dam_break(nx=80, ny=40, spacing=1.0, n_gauss=40, breach=False, seed=9)
    if bc == "level":
        w.bnd_tag = np.full(len(w.bnd_edges), W.tag(W.LEVEL), np.int32)
        w.level = np.array([2.0])
    g = run_gpu(w, "muscl", precision, steps=1000, hr_order=2)
    assert np.array_equal(g["h"], w.h)
    assert not g["hu"].any() and not g["hv"].any()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_mass_conservation(precision, tol):
    w = _pdb()
    m0 = run_oracle(w, "muscl", steps=0)["mass0"]
    g = run_gpu(w, "muscl", precision, steps=300, hr_order=2)
    assert abs(g["mass"] - m0 - g["clipped"]) <= tol * m0


def test_fp32_error_and_renumbering():
    w = W.river(80, 30, seed=21, q_in=1500.0)
    o = run_oracle(w, "muscl", steps=1000, h_eps=1e-4, r_eps=1e-6, hr_order=2)
    g = run_gpu(w, "muscl", "fp32", dt=o["dts"], hr_order=2)
    assert rel_l1(g["h"], o["h"]) <= 1e-4
    p = _pdb(50, 24)
    ref = run_gpu(p, "muscl", "fp32", steps=60, reorder="none", hr_order=2)
    for r in ("morton", "rcm"):
        got = run_gpu(p, "muscl", "fp32", steps=60, reorder=r, hr_order=2)
        assert np.array_equal(got["h"], ref["h"]) and np.array_equal(got["hu"], ref["hu"])


@pytest.mark.parametrize("kw", [dict(scheme="hllc"), dict(scheme="waf"), dict(scheme="muscl_edge"),
                                dict(scheme="muscl", kernel="fused"), dict(scheme="muscl", hr_order=3)])
def test_unsupported_combinations_are_rejected(kw):
    kw = dict(kw)
    scheme = kw.pop("scheme")
    kw.setdefault("hr_order", 2)
    with pytest.raises(swe.SweError) as e:
        run_gpu(_pdb(20, 10), scheme, "fp64", steps=1, **kw)
    assert e.value.code == -1


def _alone(w, p, steps):
    m = swe.Mesh.from_workload(w)
    st = swe.State.from_workload(m, p, w)
    st.step(steps, 0.9)
    out = st.get_state(), st.time()
    st.close()
    m.close()
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_ensemble_members_match_stepping_alone(precision):
    ws = [W.river(40, 16, seed=31, q_in=2000.0), W.river(70, 26, seed=32, q_in=6000.0, level_quantile=0.4)]
    p = swe.swe_params_default("muscl", precision, hr_order=2)
    meshes = [swe.Mesh.from_workload(w) for w in ws]
    states = [swe.State.from_workload(m, p, w) for m, w in zip(meshes, ws)]
    ens = swe.Ensemble(states)
    ens.step(53, 0.9)
    ens.sync()
    for w, st in zip(ws, states):
        (h, hu, hv), tk = _alone(w, p, 53)
        gh, ghu, ghv = st.get_state()
        assert np.array_equal(gh, h) and np.array_equal(ghu, hu) and np.array_equal(ghv, hv)
        assert st.time() == tk
    # members must share the reconstruction order
    a = swe.State.from_workload(meshes[0], swe.swe_params_default("muscl", precision), ws[0])
    b = swe.State.from_workload(meshes[1], p, ws[1])
    with pytest.raises(swe.SweError) as e:
        swe.Ensemble([a, b])
    assert e.value.code == -1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_boundary_first_schedule_same_bits(precision):
    w = W.river(nx=90, ny=34, seed=13, q_in=2500.0)

    def run(n_parts):
        m = swe.Mesh.from_workload(w, "morton")
        st = swe.State.from_workload(m, swe.swe_params_default("muscl", precision, hr_order=2), w)
        part = swe.Partition(m, n_parts) if n_parts else None
        if part is not None:
            st.set_partition(part)
        st.step(60, 0.9)
        out = st.get_state(), st.time()
        st.close()
        if part is not None:
            part.close()
        m.close()
        return out

    (ref, t_ref), (got, t_got) = run(0), run(8)
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)
    assert t_got == t_ref


def test_autotune_stays_on_the_split_kernels():
    w = W.river(90, 34, seed=7, q_in=3000.0)
    m = swe.Mesh.from_workload(w)
    a = swe.State.from_workload(m, swe.swe_params_default("muscl", "fp32", hr_order=2), w)
    kernel, block, ms = a.autotune(m, trial_steps=4)
    assert kernel == "split" and ms > 0
