"""FP64 CPU oracle for the shallow-water finite-volume step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` (the default run's baseline, ``--impl reference`` and the
per-configuration study ``--configs``) import this package.  The product library never calls it.  The
oracle is plain C (``swe_oracle.c``) compiled with gcc into an in-tree shared
library and called through ctypes.  Arrays are numpy, in the caller's cell
order.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

SCHEMES = {"hllc": 0, "muscl": 1, "waf": 2, "muscl_edge": 3}
BC_WALL, BC_OPEN, BC_INFLOW, BC_LEVEL = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "swe_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Opts(C.Structure):
    _fields_ = [("scheme", C.c_int), ("time_scheme", C.c_int), ("waf_limiter", C.c_int),
                ("threads", C.c_int), ("g", C.c_double), ("h_eps", C.c_double),
                ("r_eps", C.c_double), ("cfl", C.c_double), ("cfl_local", C.c_int),
                ("beta", C.c_double), ("hr_order", C.c_int), ("waf_surface", C.c_int)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
        lib.om_mesh_build.argtypes = [vp, i64, vp, i64, vp, vp, i64, vp, i64, C.POINTER(vp)]
        lib.om_mesh_free.argtypes = [vp]
        lib.om_mesh_ncells.argtypes = [vp]
        lib.om_mesh_ncells.restype = i64
        lib.om_mesh_export.argtypes = [vp] * 13
        lib.om_morton_order.argtypes = [vp, vp]
        lib.om_rcm_order.argtypes = [vp, vp]
        lib.om_run.argtypes = [vp, C.POINTER(_Opts), vp, vp, vp, i32, vp, i32, vp, vp, vp, i32, vp, vp, vp]
        lib.om_gradients.argtypes = [vp, C.POINTER(_Opts), vp, vp, vp, vp, vp, vp]
        lib.om_edge_flux.argtypes = [C.POINTER(_Opts), vp, vp, vp]
        lib.om_mass.argtypes = [vp, vp]
        lib.om_mass.restype = C.c_double
        lib.om_beta_limit.argtypes = [C.c_double, C.c_double, C.c_double]
        lib.om_beta_limit.restype = C.c_double
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def opts(scheme="hllc", time_scheme="euler", waf_limiter="superbee", g=9.81, h_eps=1e-6,
         r_eps=1e-12, cfl=0.9, threads=0, cfl_mode="global", beta=2.0, hr_order=1,
         waf_ratio="surface") -> _Opts:
    """waf_ratio: the quantity of the WAF ratios, "surface" (eta, reading R4, the default) or
    "depth" (the cell depth h, option R17)."""
    return _Opts(SCHEMES[scheme], {"euler": 0, "heun": 1}[time_scheme],
                 {"superbee": 0, "phi1": 1, "phi0": 2, "minbee": 3, "vanleer": 4}[waf_limiter], threads,
                 g, h_eps, r_eps, cfl, {"global": 0, "local": 1}[cfl_mode], beta, hr_order,
                 {"depth": 0, "surface": 1}[waf_ratio])


class Mesh:
    """Oracle mesh (original cell order)."""

    def __init__(self, nodes, tris, bnd_edges=None, bnd_tag=None, cut_edges=None):
        lib = _load()
        self._nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        self._tris = np.ascontiguousarray(tris, dtype=np.int32)
        be = np.ascontiguousarray(bnd_edges if bnd_edges is not None else np.zeros((0, 2)), dtype=np.int32)
        bt = np.ascontiguousarray(bnd_tag if bnd_tag is not None else np.zeros(0), dtype=np.int32)
        ce = np.ascontiguousarray(cut_edges if cut_edges is not None else np.zeros((0, 2)), dtype=np.int32)
        h = C.c_void_p()
        rc = lib.om_mesh_build(_p(self._nodes), len(self._nodes), _p(self._tris), len(self._tris),
                               _p(be), _p(bt), len(bt), _p(ce), len(ce), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle mesh build failed ({rc})")
        self._h = h
        self.n = int(lib.om_mesh_ncells(h))
        self.arrays = self._export()

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.om_mesh_free(self._h)
            self._h = None

    def _export(self):
        n = self.n
        a = {
            "tri": np.empty((n, 3), np.int32), "nbr": np.empty((n, 3), np.int32),
            "nbr_edge": np.empty((n, 3), np.int32), "btag": np.empty((n, 3), np.int32),
            "lnx": np.empty((n, 3)), "lny": np.empty((n, 3)), "area": np.empty(n),
            "cx": np.empty(n), "cy": np.empty(n), "rin": np.empty(n),
            "dx": np.empty((n, 3)), "dy": np.empty((n, 3)),
        }
        _lib.om_mesh_export(self._h, *[_p(a[k]) for k in
                                      ("tri", "nbr", "nbr_edge", "btag", "lnx", "lny", "area",
                                       "cx", "cy", "rin", "dx", "dy")])
        return a

    def morton(self):
        p = np.empty(self.n, np.int32)
        _lib.om_morton_order(self._h, _p(p))
        return p

    def rcm(self):
        p = np.empty(self.n, np.int32)
        _lib.om_rcm_order(self._h, _p(p))
        return p

    def mass(self, h):
        h = np.ascontiguousarray(h, dtype=np.float64)
        return float(_lib.om_mass(self._h, _p(h)))


def run(mesh: Mesh, o: _Opts, z, nman, h, hu, hv, n_steps, q_in=(), level=(), dt=None):
    """Advance a copy of (h, hu, hv) by n_steps.  Returns (h, hu, hv, dts, diag)."""
    lib = _load()
    h = np.array(h, dtype=np.float64, copy=True)
    hu = np.array(hu, dtype=np.float64, copy=True)
    hv = np.array(hv, dtype=np.float64, copy=True)
    z = np.ascontiguousarray(z, dtype=np.float64)
    nman = np.ascontiguousarray(nman if nman is not None else np.zeros(mesh.n), dtype=np.float64)
    qa = np.ascontiguousarray(q_in, dtype=np.float64).reshape(-1)
    la = np.ascontiguousarray(level, dtype=np.float64).reshape(-1)
    dts = np.zeros(n_steps)
    dtg = None if dt is None else np.ascontiguousarray(dt, dtype=np.float64)
    diag = np.zeros(4)
    rc = lib.om_run(mesh._h, C.byref(o), _p(z), _p(nman), _p(qa) if len(qa) else None, len(qa),
                    _p(la) if len(la) else None, len(la), _p(h), _p(hu), _p(hv), int(n_steps),
                    _p(dtg), _p(dts), _p(diag))
    if rc != 0:
        raise RuntimeError(f"oracle run failed ({rc})")
    return h, hu, hv, dts, {"t": diag[0], "clipped": diag[1], "boundary_in": diag[2]}


def gradients(mesh: Mesh, o: _Opts, z, h, hu, hv):
    lib = _load()
    gl = np.empty((mesh.n, 6))
    gu = np.empty((mesh.n, 6))
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (z, h, hu, hv)]
    lib.om_gradients(mesh._h, C.byref(o), *[_p(a) for a in arrs], _p(gl), _p(gu))
    return gl, gu


def edge_flux(o: _Opts, state, waf=None):
    """state = (hface_L, hstar_L, hcell_L, uL, vL, hface_R, hstar_R, hcell_R, uR, vR)."""
    lib = _load()
    a = np.ascontiguousarray(state, dtype=np.float64)
    w = None if waf is None else np.ascontiguousarray(waf, dtype=np.float64)
    out = np.empty(4)
    lib.om_edge_flux(C.byref(o), _p(a), _p(w), _p(out))
    return out


def beta_limit(beta, up, dn):
    """The limited slope of the paper's MUSCL (Sec. 6.2.3); see om_beta_limit."""
    return float(_load().om_beta_limit(float(beta), float(up), float(dn)))
