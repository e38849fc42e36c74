"""C-ABI library: symbols, argument checks and the host mesh builder (no GPU needed).

The mesh builder runs on the host, so it is compared with the oracle's own,
independently written builder here: every exported array must be equal bit
for bit (geometry has a plain definition and both sides evaluate it without
floating-point contraction; the orders are index work).
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe
from paper_2307_16758_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return swe.load_library()


def _declared():
    inc = os.path.join(ROOT, "include")
    txt = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(swe_[a-z_]+)\s*\(", txt))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(swe.EXPORTED)


def test_params_default(lib):
    p = swe.swe_params_default("muscl", "fp32")
    assert p.scheme == 1 and p.precision == 1 and p.g == 9.81 and p.h_eps == 1e-4
    p = swe.swe_params_default("hllc", "fp64")
    assert p.h_eps == 1e-6 and p.r_eps == 1e-12 and p.time_scheme == 0 and p.cfl_mode == 0
    assert swe.swe_params_default("muscl", "fp64", cfl_mode="local").cfl_mode == 1
    with pytest.raises(swe.SweError) as e:
        swe.swe_params_default(7, "fp64")
    assert e.value.code == -1


def _compare_with_oracle(w, reorder):
    m = swe.Mesh.from_workload(w, reorder)
    a = m.export()
    om = oracle.Mesh(w.nodes, w.tris, w.bnd_edges, w.bnd_tag, w.cut_edges if len(w.cut_edges) else None)
    o = om.arrays
    perm = a["perm"]
    if reorder == "morton":
        assert np.array_equal(perm, om.morton())
    elif reorder == "rcm":
        assert np.array_equal(perm, om.rcm())
    else:
        assert np.array_equal(perm, np.arange(m.n))
    inv = np.empty_like(perm)
    inv[perm] = np.arange(m.n)
    onbr = o["nbr"][perm]
    assert np.array_equal(a["nbr"], np.where(onbr >= 0, inv[np.maximum(onbr, 0)], -1))
    for k in ("tri", "nbr_edge", "btag", "lnx", "lny", "area", "cx", "cy", "rin", "dx", "dy"):
        assert np.array_equal(a[k], o[k][perm]), k          # bit for bit
    assert m.r_min == o["rin"].min()
    return m


@pytest.mark.parametrize("reorder", ["none", "morton", "rcm"])
def test_mesh_builder_matches_oracle_bitwise(lib, reorder):
    _compare_with_oracle(W.partial_dam_break(nx=30, ny=14, spacing=1.0, n_gauss=6, seed=3), reorder)
    _compare_with_oracle(W.river(nx=60, ny=22, seed=5), reorder)
    _compare_with_oracle(W.circular_dam_break(n=8), reorder)


def test_mesh_builder_reorients_clockwise_input(lib):
    nodes = np.array([[0.0, 0.0], [0.0, 1.0], [1.0, 0.0], [1.0, 1.0]])
    tris = np.array([[0, 1, 2], [1, 3, 2]])
    m = swe.Mesh(nodes, tris, reorder="none")
    a = m.export()
    assert (a["area"] == 0.5).all()
    assert a["nbr"][0].tolist().count(1) == 1


@pytest.mark.parametrize("case", ["degenerate", "nonmanifold", "bnd_not_boundary", "bad_tag", "node_range"])
def test_mesh_errors(lib, case):
    nodes = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0], [2.0, 2.0], [0.2, 0.8]])
    tris, bnd, tg = np.array([[0, 1, 2], [0, 2, 3]]), None, None
    if case == "degenerate":
        tris = np.array([[0, 2, 4]])
    elif case == "nonmanifold":
        tris = np.array([[0, 1, 2], [0, 2, 3], [0, 2, 5]])
    elif case == "bnd_not_boundary":
        bnd, tg = np.array([[0, 2]]), np.array([1])
    elif case == "bad_tag":
        bnd, tg = np.array([[0, 1]]), np.array([4 * 99])
    else:
        tris = np.array([[0, 1, 9]])
    with pytest.raises(swe.SweError) as e:
        swe.Mesh(nodes, tris, bnd, tg, reorder="none")
    assert e.value.code == -2


def test_argument_errors(lib):
    with pytest.raises(swe.SweError) as e:
        swe.swe_mesh_create(np.zeros((3, 2)), np.zeros((0, 3)))
    assert e.value.code == -1
    with pytest.raises(swe.SweError) as e:
        swe.swe_mesh_create(np.array([[0, 0], [1, 0], [0, 1.0]]), np.array([[0, 1, 2]]), reorder=5)
    assert e.value.code == -1
    rc = lib.swe_step(None, 1, 0.9)
    assert rc == -1
    rc = lib.swe_get_state(None, None, None, None)
    assert rc == -1
    assert lib.swe_mesh_info(None, None, None) == -1
    assert lib.swe_state_destroy(None) == 0


def test_inflow_lengths_and_packed_tags(lib):
    w = W.river(nx=40, ny=15, seed=2)
    m = swe.Mesh.from_workload(w, "morton")
    a = m.export()
    inflow = (a["nbr"] < 0) & (a["btag"] >= 0) & ((a["btag"] & 3) == W.INFLOW)
    assert inflow.sum() >= 1
    lens = np.hypot(a["lnx"], a["lny"])
    assert lens[inflow].sum() > 0


def test_binding_classes_own_their_handles():
    for cls, methods in ((swe.Mesh, ("export", "close")),
                         (swe.State, ("step", "step_dt", "get_state", "mass", "time", "autotune", "close")),
                         (swe.Ensemble, ("step", "sync", "autotune", "close"))):
        for m in methods:
            assert callable(getattr(cls, m, None)), (cls.__name__, m)
    assert swe.State.close is not swe.Ensemble.close


@pytest.mark.parametrize("args", [("fp32", 0), ("fp32", 1 << 21), (7, 100)])
def test_fma_peak_rejects_bad_arguments_before_any_launch(args):
    precision, iters = args
    with pytest.raises(swe.SweError) as e:
        swe.swe_fma_peak(precision, iters)
    assert e.value.code == -1


def _header_constants():
    """Every enumerator and #define of the public headers, by name."""
    inc = os.path.join(ROOT, "include")
    txt = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    vals = {k: int(v) for k, v in re.findall(r"\b(SWE_[A-Z0-9_]+)\s*=\s*(-?\d+)", txt)}
    vals.update({k: int(v) for k, v in re.findall(r"#define\s+(SWE_[A-Z0-9_]+)\s+(-?\d+)", txt)})
    return vals


def test_binding_constants_match_the_header():
    """The binding's name tables carry the header's values (a mismatch would silently select
    another scheme, limiter or kernel)."""
    h = _header_constants()
    for code, name in swe.ERRORS.items():
        assert h[name] == code, name
    assert h["SWE_OK"] == swe.SWE_OK
    tables = {"SWE_REORDER_": swe.REORDER, "SWE_SCHEME_": swe.SCHEME, "SWE_": swe.PRECISION,
              "SWE_KERNEL_": swe.KERNEL, "SWE_CFL_": swe.CFL_MODE, "SWE_WAF_RATIO_": swe.WAF_RATIO,
              "SWE_WAF_": swe.WAF_LIMITER}
    for prefix, table in tables.items():
        for name, value in table.items():
            assert h[prefix + name.upper()] == value, (prefix, name)
    assert h["SWE_EULER"] == swe.TIME_SCHEME["euler"] and h["SWE_HEUN"] == swe.TIME_SCHEME["heun"]
    assert (h["SWE_WALL"], h["SWE_OPEN"], h["SWE_INFLOW"], h["SWE_LEVEL"]) == (
        swe.SWE_WALL, swe.SWE_OPEN, swe.SWE_INFLOW, swe.SWE_LEVEL) == (W.WALL, W.OPEN, W.INFLOW, W.LEVEL)
    assert (h["SWE_FLAG_CLIPPED"], h["SWE_FLAG_NONFINITE"], h["SWE_FLAG_DRY"]) == (
        swe.FLAG_CLIPPED, swe.FLAG_NONFINITE, swe.FLAG_DRY)
    assert h["SWE_MAX_GROUPS"] == swe.MAX_GROUPS
    assert h["SWE_NOALLOC_MAX_CELLS"] == swe.NOALLOC_MAX_CELLS
    assert h["SWE_K_COUNT"] == len(swe.KERNEL_KINDS)
    for k, name in enumerate(swe.KERNEL_KINDS):
        if "SWE_K_" + name.upper() in h:
            assert h["SWE_K_" + name.upper()] == k, name


def test_allocator_pair_is_both_or_neither(lib):
    """swe_set_allocator takes both functions or neither (neither: cudaMalloc/cudaFree); the
    binding keeps every pair it installed alive.  No device memory is allocated here."""
    saved = swe._callbacks
    try:
        with pytest.raises(swe.SweError) as e:
            swe.swe_set_allocator(lambda n, s, c: None)
        assert e.value.code == -1
        assert lib.swe_set_allocator(swe._ALLOC(lambda n, s, c: None), swe._FREE(), None) == -1
        swe.swe_set_allocator()
        assert swe._callbacks is not saved and saved in swe._retired
    finally:
        if saved is not None:
            assert lib.swe_set_allocator(saved[0], saved[1], None) == 0
        swe._callbacks = saved
