"""swe_muscl_step_noalloc against the regular entry point (GPU).

Some callers cannot allocate device memory -- a plug-in inside an application
that owns the GPU's memory pools, or a real-time loop where an allocation
could block -- so they cannot create a swe_state.  swe_muscl_step_noalloc
serves them: it takes caller-owned device buffers and keeps its only scratch
(the per-cell face values) in an array compiled into the library.  This test
gives it the same mesh and state as a regular state advanced with
swe_step_dt, and compares two calls in a row bit for bit (the second call
reads the first call's output while the shared scratch still holds the
first call's face values).  The file is collected last so that a failing run stops only
after every other test has run; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe
from paper_2307_16758_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _device_layout(mesh, w):
    """The mesh and state in the library's cell order, as the entry point expects."""
    a = mesh.export()
    perm = a["perm"]
    nbr, ne, bt = a["nbr"], a["nbr_edge"], a["btag"]
    inner = nbr >= 0
    owner = np.zeros_like(nbr)
    owner[inner] = (perm[np.repeat(np.arange(mesh.n), 3).reshape(-1, 3)][inner] < perm[nbr[inner]]).astype(np.int32)
    packed = np.where(inner, (nbr << 3) | (ne << 1) | owner, -1 - bt).astype(np.int32)
    ln = np.stack([a["lnx"], a["lny"]], axis=-1).astype(np.float32)
    lens = np.hypot(a["lnx"], a["lny"])
    qlen = []
    for g, q in enumerate(w.q_in):
        sel = (~inner) & ((bt & 3) == W.INFLOW) & ((bt >> 2) == g)
        qlen.append(q / lens[sel].sum())
    cells = {k: getattr(w, k)[perm].astype(np.float32) for k in ("z", "nman", "h", "hu", "hv")}
    return perm, packed, ln, cells, np.array(qlen, np.float32), np.asarray(w.level, np.float32)


def test_noalloc_step_matches_regular_entry_point_twice():
    import torch

    B.build()
    swe.load_library()
    w = W.river(nx=150, ny=56, seed=31, q_in=2500.0)          # 16,800 cells, inflow, level, friction
    mesh = swe.Mesh.from_workload(w, "morton")
    n = mesh.n
    assert n <= swe.NOALLOC_MAX_CELLS
    p = swe.swe_params_default("muscl", "fp32", kernel="split")

    # time steps of the regular path, then two replayed steps one at a time
    probe = swe.State.from_workload(mesh, p, w)
    probe.step(2, 0.9)
    dts = probe.dt_history(2)
    probe.close()
    ref = swe.State.from_workload(mesh, p, w)
    expected = []
    for dt in dts:
        ref.step_dt([dt])
        expected.append(ref.get_state())
    ref.close()

    perm, packed, ln, cells, qlen, level = _device_layout(mesh, w)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    t_nbr, t_ln = dev(packed), dev(ln)
    t_z, t_n = dev(cells["z"]), dev(cells["nman"])
    bufs = [[dev(cells["h"]), dev(cells["hu"]), dev(cells["hv"])],
            [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]]
    torch.cuda.synchronize()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, dt in enumerate(dts):
        src, dst = bufs[call % 2], bufs[(call + 1) % 2]
        swe.swe_muscl_step_noalloc(n, t_nbr.data_ptr(), t_ln.data_ptr(), t_z.data_ptr(),
                                   t_n.data_ptr(), *[b.data_ptr() for b in src], *[b.data_ptr() for b in dst],
                                   float(dt), p, qlen, level, stream)
        torch.cuda.synchronize()
        for k, got in enumerate(dst):
            out = np.empty(n)
            out[perm] = got.cpu().numpy().astype(np.float64)
            # the same kernels on the same inputs and the same dt: the same bits
            assert np.array_equal(out, expected[call][k]), (call, k, np.abs(out - expected[call][k]).max())
    mesh.close()


def test_noalloc_rejects_meshes_above_its_limit():
    B.build()
    swe.load_library()
    p = swe.swe_params_default("muscl", "fp32")
    with pytest.raises(swe.SweError) as e:
        swe.swe_muscl_step_noalloc(swe.NOALLOC_MAX_CELLS + 1, *([1] * 10), 0.1, p, stream=C.c_void_p(None))
    assert e.value.code == -1


def _small_buffers(n):
    """Valid device buffers of n cells (so that a check that failed to reject could not fault)."""
    import torch

    f = lambda: torch.zeros(n, dtype=torch.float32, device="cuda")
    nbr = torch.full((3 * n,), -1, dtype=torch.int32, device="cuda")      # every edge a wall
    ln = torch.zeros(6 * n, dtype=torch.float32, device="cuda")
    return nbr, ln, f(), f(), [f(), f(), f()], [f(), f(), f()]


@pytest.mark.parametrize("case", ["dt_inf", "dt_nan", "dt_negative", "hr_order_2", "out_is_in_hu",
                                  "outs_alias", "out_overlaps_z", "fp64"])
def test_noalloc_rejects_bad_arguments(case):
    B.build()
    swe.load_library()
    n = 64
    nbr, ln, z, nm, src, dst = _small_buffers(n)
    p = swe.swe_params_default("muscl", "fp32")
    dt = 0.01
    outs = [b.data_ptr() for b in dst]
    if case == "dt_inf":
        dt = float("inf")
    elif case == "dt_nan":
        dt = float("nan")
    elif case == "dt_negative":
        dt = -1e-3
    elif case == "hr_order_2":
        p.hr_order = 2
    elif case == "out_is_in_hu":
        outs[1] = src[1].data_ptr()
    elif case == "outs_alias":
        outs[2] = outs[0] + 4 * (n // 2)                                       # overlaps h_out's tail
    elif case == "out_overlaps_z":
        outs[0] = z.data_ptr()
    elif case == "fp64":
        p = swe.swe_params_default("muscl", "fp64")
    with pytest.raises(swe.SweError) as e:
        swe.swe_muscl_step_noalloc(n, nbr.data_ptr(), ln.data_ptr(), z.data_ptr(), nm.data_ptr(),
                                   *[b.data_ptr() for b in src], *outs, dt, p, stream=C.c_void_p(None))
    assert e.value.code == -1, case
