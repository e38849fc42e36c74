"""Helpers for the GPU parity tests: run the CUDA path and the oracle on the same inputs."""
import numpy as np

import oracle
from paper_2307_16758_gb300 import swe


def run_gpu(w, scheme, precision="fp64", steps=0, cfl=0.9, dt=None, reorder="morton", **kw):
    p = swe.swe_params_default(scheme, precision, **kw)
    m = swe.Mesh.from_workload(w, reorder)
    s = swe.State.from_workload(m, p, w)
    if dt is not None:
        s.step_dt(dt)
    elif steps:
        s.step(steps, cfl)
    h, hu, hv = s.get_state()
    t, k = s.time()
    mass, clipped, bin_ = s.mass()
    s.close()
    m.close()
    return dict(h=h, hu=hu, hv=hv, t=t, steps=k, mass=mass, clipped=clipped, bnd_in=bin_)


def run_oracle(w, scheme, steps=0, cfl=0.9, dt=None, h_eps=1e-6, r_eps=1e-12, **kw):
    om = oracle.Mesh(w.nodes, w.tris, w.bnd_edges, w.bnd_tag, w.cut_edges if len(w.cut_edges) else None)
    o = oracle.opts(scheme, h_eps=h_eps, r_eps=r_eps, cfl=cfl, **kw)
    n = len(dt) if dt is not None else steps
    h, hu, hv, dts, d = oracle.run(om, o, w.z, w.nman, w.h, w.hu, w.hv, n, q_in=w.q_in, level=w.level, dt=dt)
    return dict(h=h, hu=hu, hv=hv, dts=dts, t=d["t"], clipped=d["clipped"], bnd_in=d["boundary_in"],
                mass=om.mass(h), mass0=om.mass(w.h), mesh=om)


def rel_max(a, b, scale=None):
    s = scale if scale is not None else max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / s)


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def state_errors(g, o):
    """Max error of h and of the discharges, relative to the largest |h| and |(hu,hv)|."""
    qs = max(np.abs(o["hu"]).max(), np.abs(o["hv"]).max(), 1e-300)
    return (rel_max(g["h"], o["h"]), rel_max(g["hu"], o["hu"], qs), rel_max(g["hv"], o["hv"], qs))
