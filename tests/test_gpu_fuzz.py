"""Seeded random problems against the FP64 oracle: random mesh sizes and jitter, random bathymetry with
dry areas, a random dam-break perturbation and velocities, random boundary kinds per side (wall, open,
inflow, fixed level), random friction, every scheme.  The GPU's FP64 path must match the oracle step
by step (its time steps replayed) to the parity bar of 1e-9."""
import numpy as np
import pytest

from gpu_common import run_gpu, run_oracle, state_errors
from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe
from paper_2307_16758_gb300 import workloads as W

pytestmark = pytest.mark.gpu
SCHEMES = ["hllc", "muscl", "waf", "muscl_edge"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    swe.load_library()


def random_problem(seed):
    rng = np.random.default_rng(20240 + seed)
    nx, ny = int(rng.integers(3, 40)), int(rng.integers(2, 25))
    lx, ly = nx * rng.uniform(0.5, 3.0), ny * rng.uniform(0.5, 3.0)
    nodes, tris, bnd, side = W.structured(nx, ny, lx, ly, jitter=rng.uniform(0.0, 0.3), seed=seed)
    w = W.Workload(f"random{seed}", nodes, tris, bnd, np.zeros(len(bnd), np.int32), np.zeros((0, 2), np.int32),
                   np.zeros(len(tris)), np.zeros(len(tris)), None, None, None)
    cx, cy = w.centroids()
    z = rng.uniform(0.2, 1.5) * np.sin(2 * np.pi * cx / lx * rng.uniform(0.5, 2.0)) * np.cos(np.pi * cy / ly)
    w.z = W.quantize_bed(z + rng.normal(0.0, 0.1, len(tris)))
    eta0 = float(np.quantile(w.z, rng.uniform(0.4, 0.8)))
    h = np.maximum(eta0 - w.z, 0.0) + np.where(cx < lx * rng.uniform(0.2, 0.6), rng.uniform(0.0, 1.0), 0.0)
    h[h < 1e-2] = 0.0                                        # clear margins above the dry threshold
    w.h = h
    w.hu = np.where(h > 0, h * rng.normal(0.0, 0.3, len(tris)), 0.0)
    w.hv = np.where(h > 0, h * rng.normal(0.0, 0.3, len(tris)), 0.0)
    w.nman = rng.uniform(0.0, 0.05, len(tris)) if rng.random() < 0.7 else np.zeros(len(tris))
    kinds = rng.integers(0, 4, 4)                           # per side: wall, open, inflow, level
    w.bnd_tag = np.array([W.tag(int(kinds[s]), int(s % 2) if kinds[s] == W.LEVEL else 0) for s in side], np.int32)
    w.q_in = np.array([rng.uniform(0.0, 2.0) * ly])
    w.level = np.array([eta0 + rng.uniform(-0.3, 0.3), eta0 + rng.uniform(-0.3, 0.3)])
    return w, SCHEMES[seed % 4]


@pytest.mark.parametrize("seed", range(16))
def test_random_problem_fp64_matches_the_oracle(seed):
    w, scheme = random_problem(seed)
    o = run_oracle(w, scheme, steps=15)
    assert np.isfinite(o["h"]).all() and (o["h"] >= 0).all()
    g = run_gpu(w, scheme, dt=o["dts"])
    assert max(state_errors(g, o)) <= 1e-9, (scheme, w.n_cells)


OPTIONS = [("muscl", dict(hr_order=2)), ("waf", dict(waf_ratio="surface")), ("muscl", dict(time_scheme="heun")),
           ("hllc", dict(time_scheme="heun")), ("muscl_edge", dict(beta=1.0)), ("waf", dict(waf_limiter="phi1"))]


@pytest.mark.parametrize("seed", range(12))
def test_random_problem_with_options_fp64_matches_the_oracle(seed):
    """The same random problems with the options: second-order hydrostatic reconstruction, the WAF ratio
    on the free surface, Heun steps, the paper's MUSCL with the MINBEE limiter, WAF without limiting."""
    w, _ = random_problem(100 + seed)
    scheme, kw = OPTIONS[seed % len(OPTIONS)]
    gkw = {("muscl_beta" if k == "beta" else k): v for k, v in kw.items()}
    o = run_oracle(w, scheme, steps=15, **kw)
    assert np.isfinite(o["h"]).all()
    g = run_gpu(w, scheme, dt=o["dts"], **gkw)
    assert max(state_errors(g, o)) <= 1e-9, (scheme, kw, w.n_cells)


@pytest.mark.parametrize("seed", range(12))
def test_random_problem_fp32_stays_close_to_the_oracle(seed):
    """The FP32 path on the random problems (the oracle with FP32's dry and ratio thresholds): after 15
    replayed steps the relative L1 differences stay at the FP32 rounding level, 1e-5 for h and 1e-4
    for the discharges."""
    from gpu_common import rel_l1
    w, scheme = random_problem(200 + seed)
    o = run_oracle(w, scheme, steps=15, h_eps=1e-4, r_eps=1e-6)
    g = run_gpu(w, scheme, "fp32", dt=o["dts"])
    assert rel_l1(g["h"], o["h"]) <= 1e-5, (scheme, w.n_cells)
    assert rel_l1(g["hu"], o["hu"]) <= 1e-4 and rel_l1(g["hv"], o["hv"]) <= 1e-4, (scheme, w.n_cells)
