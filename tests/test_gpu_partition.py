"""Boundary-first schedule on the GPU (the single-GPU rehearsal of the sub-domain schedule of
Sec. 6.4): the same bits as the plain schedule, and each part's exchange buffer holds the new state
of its two halo layers."""
import numpy as np
import pytest

from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe
from paper_2307_16758_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    swe.load_library()


def _run(w, scheme, precision, n_parts, steps=60, dt=None, block=256):
    m = swe.Mesh.from_workload(w, "morton")
    st = swe.State.from_workload(m, swe.swe_params_default(scheme, precision, kernel="split", block=block), w)
    part = swe.Partition(m, n_parts) if n_parts else None
    if part is not None:
        st.set_partition(part)
    if dt is not None:
        st.step_dt(dt)
    else:
        st.step(steps, 0.9)
    out = st.get_state(), st.time(), st.mass()
    halos = [st.halo(part, p) for p in range(n_parts)] if part is not None else None
    lists = [part.export(p) for p in range(n_parts)] if part is not None else None
    perm = m.export()["perm"]
    st.close()
    if part is not None:
        part.close()
    m.close()
    return out, halos, lists, perm


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme", ["hllc", "muscl", "waf", "muscl_edge"])
@pytest.mark.parametrize("n_parts", [3, 8])
def test_same_bits_as_the_plain_schedule(scheme, precision, n_parts):
    w = W.river(nx=90, ny=34, seed=13, q_in=2500.0)          # inflow, level, friction, dry cells
    (ref, t_ref, m_ref), *_ = _run(w, scheme, precision, 0)
    (got, t_got, m_got), halos, lists, perm = _run(w, scheme, precision, n_parts)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    assert t_got == t_ref
    # each part's exchange buffer: the state of its halo1 then halo2 cells after the last step
    h = got[0]
    for p in range(n_parts):
        h1, h2, _ = lists[p]
        cells = np.concatenate([h1, h2])
        assert np.array_equal(halos[p][0], h[perm[cells]])
        assert np.array_equal(halos[p][1], got[1][perm[cells]])
        assert np.array_equal(halos[p][2], got[2][perm[cells]])


def test_replayed_steps_odd_block_and_clearing():
    w = W.partial_dam_break(nx=50, ny=24, spacing=1.0, n_gauss=12, seed=6)
    (ref, _, _), *_ = _run(w, "muscl", "fp64", 0, steps=37)
    (got, _, _), *_ = _run(w, "muscl", "fp64", 5, steps=37, block=128)   # 37 = graph + single steps
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    m = swe.Mesh.from_workload(w)
    st = swe.State.from_workload(m, swe.swe_params_default("muscl", "fp32"), w)
    part = swe.Partition(m, 4)
    st.set_partition(part)
    st.step(10, 0.9)
    st.set_partition(None)                                     # back to the plain schedule
    st.step(10, 0.9)
    assert st.time()[1] == 20
    st.close()
    m.close()


def test_unsupported_configurations_are_rejected():
    w = W.partial_dam_break(nx=30, ny=14, spacing=1.0, n_gauss=6, seed=6)
    m = swe.Mesh.from_workload(w)
    part = swe.Partition(m, 3)
    for kw in (dict(kernel="fused"), dict(time_scheme="heun")):
        st = swe.State.from_workload(m, swe.swe_params_default("muscl", "fp64", **kw), w)
        with pytest.raises(swe.SweError) as e:
            st.set_partition(part)
        assert e.value.code == -1
        st.close()
    other = swe.Mesh.from_workload(W.dam_break_1d(10, 2, 10.0, 2.0))
    st = swe.State.from_workload(other, swe.swe_params_default("hllc", "fp64"), W.dam_break_1d(10, 2, 10.0, 2.0))
    with pytest.raises(swe.SweError):
        st.set_partition(part)                                 # a partition of another mesh
    st.close()
    other.close()
    part.close()
    m.close()


@pytest.mark.parametrize("scheme", ["hllc", "muscl", "waf"])
def test_one_cell_per_part_same_bits(scheme):
    """The degenerate schedule: every cell its own sub-domain, every cell a boundary cell."""
    w = W.dam_break_1d(8, 2, 8.0, 2.0, 1.0, 0.5, x_dam=4.0)
    (ref, t_ref, _), *_ = _run(w, scheme, "fp64", 0, steps=30)
    n = 2 * 8 * 2
    (got, t_got, _), *_ = _run(w, scheme, "fp64", n, steps=30)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    assert t_got == t_ref


@pytest.mark.parametrize("scheme", ["hllc", "muscl", "waf"])
@pytest.mark.parametrize("n_parts", [1, 5, 64])
def test_schedule_against_the_oracle(scheme, n_parts):
    """The boundary-first schedule (Sec. 6.4) against the FP64 oracle, not only against the plain
    schedule: 1e-12 after one step and 1e-9 after 100 steps with the oracle's time steps replayed,
    on a river with inflow, fixed level, friction and dry banks."""
    from gpu_common import run_oracle, state_errors

    w = W.river(nx=90, ny=34, seed=13, q_in=2500.0)
    o1 = run_oracle(w, scheme, steps=1)
    (g1, _, _), *_ = _run(w, scheme, "fp64", n_parts, dt=o1["dts"])
    assert max(state_errors(dict(h=g1[0], hu=g1[1], hv=g1[2]), o1)) <= 1e-12
    o = run_oracle(w, scheme, steps=100)
    (g, (t, k), _), *_ = _run(w, scheme, "fp64", n_parts, dt=o["dts"])
    assert max(state_errors(dict(h=g[0], hu=g[1], hv=g[2]), o)) <= 1e-9
    assert k == 100 and abs(t - o["t"]) <= 1e-12 * o["t"]
