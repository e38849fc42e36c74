"""Thin Python binding of the C ABI in ``include/swe.h`` (argument marshalling only).

Functions keep the C names (``swe_mesh_create``, ``swe_state_init``,
``swe_step``, ``swe_get_state``, ``swe_mass`` ...).  Arrays are numpy, FP64
for real data and int32 for ids, in the caller's cell order.  Device memory
goes through PyTorch's caching allocator and launches go to PyTorch's current
CUDA stream, so the library interoperates with torch code; every numerical
step runs in the library's CUDA kernels.  There is no CPU fallback: if the
library or a GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libswe.so")

SWE_OK = 0
ERRORS = {-1: "SWE_ERR_ARG", -2: "SWE_ERR_MESH", -3: "SWE_ERR_CUDA", -4: "SWE_ERR_DRY",
          -5: "SWE_ERR_NONFINITE", -6: "SWE_ERR_TIMEOUT",
          -7: "SWE_ERR_NOMEM"}
FLAG_CLIPPED, FLAG_NONFINITE, FLAG_DRY = 1, 2, 4
SWE_WALL, SWE_OPEN, SWE_INFLOW, SWE_LEVEL = 0, 1, 2, 3
REORDER = {"none": 0, "morton": 1, "rcm": 2}
SCHEME = {"hllc": 0, "muscl": 1, "waf": 2, "muscl_edge": 3}
PRECISION = {"fp64": 0, "fp32": 1}
TIME_SCHEME = {"euler": 0, "heun": 1}
WAF_LIMITER = {"superbee": 0, "phi1": 1, "phi0": 2, "minbee": 3, "vanleer": 4}
KERNEL = {"auto": 0, "split": 1, "fused": 2}
CFL_MODE = {"global": 0, "local": 1}
WAF_RATIO = {"depth": 0, "surface": 1}
MAX_GROUPS = 16

EXPORTED = [
    "swe_last_error", "swe_params_default", "swe_set_allocator", "swe_mesh_create", "swe_mesh_destroy",
    "swe_mesh_info", "swe_mesh_export", "swe_state_init", "swe_state_destroy", "swe_set_stream",
    "swe_set_state", "swe_step", "swe_step_dt", "swe_sync", "swe_get_state", "swe_mass", "swe_time",
    "swe_flags", "swe_state_info", "swe_ensemble_create", "swe_ensemble_destroy", "swe_ensemble_step",
    "swe_ensemble_sync", "swe_profile_begin", "swe_profile_end", "swe_dt_history",
    "swe_muscl_step_noalloc", "swe_autotune", "swe_ensemble_autotune",
    "swe_partition_create", "swe_partition_destroy", "swe_partition_info", "swe_partition_export",
    "swe_set_partition", "swe_halo_get", "swe_fma_peak", "swe_probe_bounded_wait",
    "swe_tile_plan_info", "swe_tile_plan_export",
]
NOALLOC_MAX_CELLS = 262144
KERNEL_KINDS = ["prep", "flux", "heun_avg", "smax", "fused", "ensemble", "k6", "k7"]


class SweError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("scheme", C.c_int), ("precision", C.c_int), ("time_scheme", C.c_int),
                ("waf_limiter", C.c_int), ("g", C.c_double), ("h_eps", C.c_double),
                ("r_eps", C.c_double), ("kernel", C.c_int), ("block", C.c_int), ("cfl_mode", C.c_int),
                ("muscl_beta", C.c_double), ("hr_order", C.c_int), ("waf_ratio", C.c_int)]


class BcValues(C.Structure):
    _fields_ = [("n_inflow", C.c_int), ("inflow_q", C.POINTER(C.c_double)),
                ("n_level", C.c_int), ("level", C.POINTER(C.c_double))]


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
_lib = None
_callbacks = None
_retired = []


def load_library(path: str = LIB_PATH, use_torch_allocator: bool = True):
    """Load libswe.so (built by ``build.build()``); raises if it is missing."""
    global _lib, _callbacks
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int, C.c_double
    lib.swe_last_error.restype = C.c_char_p
    lib.swe_params_default.argtypes = [C.POINTER(Params), i32, i32]
    lib.swe_set_allocator.argtypes = [_ALLOC, _FREE, vp]
    lib.swe_mesh_create.argtypes = [vp, i64, vp, i64, vp, vp, i64, vp, i64, i32, C.POINTER(vp)]
    lib.swe_mesh_destroy.argtypes = [vp]
    lib.swe_mesh_info.argtypes = [vp, C.POINTER(i64), C.POINTER(dp)]
    lib.swe_mesh_export.argtypes = [vp] * 14
    lib.swe_state_init.argtypes = [vp, C.POINTER(Params), vp, vp, vp, vp, vp, C.POINTER(BcValues), vp,
                                   C.POINTER(vp)]
    lib.swe_state_destroy.argtypes = [vp]
    lib.swe_set_stream.argtypes = [vp, vp]
    lib.swe_set_state.argtypes = [vp, vp, vp, vp]
    lib.swe_step.argtypes = [vp, i32, dp]
    lib.swe_step_dt.argtypes = [vp, vp, i32]
    lib.swe_sync.argtypes = [vp]
    lib.swe_get_state.argtypes = [vp, vp, vp, vp]
    lib.swe_mass.argtypes = [vp, C.POINTER(dp), C.POINTER(dp), C.POINTER(dp)]
    lib.swe_time.argtypes = [vp, C.POINTER(dp), C.POINTER(i64)]
    lib.swe_flags.argtypes = [vp, C.POINTER(i32)]
    lib.swe_state_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32)]
    lib.swe_ensemble_create.argtypes = [C.POINTER(vp), i32, C.POINTER(vp)]
    lib.swe_ensemble_destroy.argtypes = [vp]
    lib.swe_ensemble_step.argtypes = [vp, i32, dp]
    lib.swe_ensemble_sync.argtypes = [vp]
    lib.swe_profile_begin.argtypes = [vp]
    lib.swe_profile_end.argtypes = [vp, vp, vp]
    lib.swe_dt_history.argtypes = [vp, vp, i32]
    lib.swe_autotune.argtypes = [vp, vp, i32, dp, C.POINTER(i32), C.POINTER(i32), C.POINTER(dp)]
    lib.swe_ensemble_autotune.argtypes = [vp, C.POINTER(vp), i32, dp, C.POINTER(i32), C.POINTER(i32), C.POINTER(dp)]
    lib.swe_muscl_step_noalloc.argtypes = [i64] + [vp] * 10 + [dp, C.POINTER(Params), vp, i32, vp, i32, vp]
    lib.swe_partition_create.argtypes = [vp, i32, C.POINTER(vp)]
    lib.swe_partition_destroy.argtypes = [vp]
    lib.swe_partition_info.argtypes = [vp, i32] + [C.POINTER(i64)] * 5
    lib.swe_partition_export.argtypes = [vp, i32, vp, vp, vp]
    lib.swe_set_partition.argtypes = [vp, vp]
    lib.swe_halo_get.argtypes = [vp, i32, vp, vp, vp]
    lib.swe_fma_peak.argtypes = [i32, i32, vp, C.POINTER(dp)]
    lib.swe_probe_bounded_wait.argtypes = [C.c_uint32, i32, C.POINTER(i32), vp]
    lib.swe_tile_plan_info.argtypes = [vp, i32, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32),
                                       C.POINTER(i32), C.POINTER(i64)]
    lib.swe_tile_plan_export.argtypes = [vp, i32, vp, vp]
    if use_torch_allocator:
        import torch

        def _alloc(nbytes, stream, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream)
            except Exception:        # out of memory: the library reports SWE_ERR_NOMEM
                return None

        def _free(ptr, stream, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        _callbacks = (_ALLOC(_alloc), _FREE(_free))
        lib.swe_set_allocator(_callbacks[0], _callbacks[1], None)
    _lib = lib
    return lib


def _check(rc):
    if rc != SWE_OK:
        raise SweError(rc, _lib.swe_last_error().decode())
    return rc


def _p(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _current_stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# ---- C-named entry points --------------------------------------------------

def swe_set_allocator(alloc=None, free_fn=None):
    """Install a device allocator pair: alloc(nbytes, stream, ctx) -> int address or None, and
    free_fn(ptr, stream, ctx); both None restores cudaMalloc/cudaFree.  Blocks already handed out
    go back to the pair that gave them.  The callbacks are kept alive here."""
    global _callbacks
    lib = load_library()
    if (alloc is None) != (free_fn is None):
        raise SweError(-1, "swe_set_allocator: give both functions or neither")
    pair = (_ALLOC(alloc), _FREE(free_fn)) if alloc is not None else (_ALLOC(), _FREE())
    _check(lib.swe_set_allocator(pair[0], pair[1], None))
    _retired.append(_callbacks)          # the old pair may still be called to free its blocks
    _callbacks = pair


def swe_params_default(scheme="muscl", precision="fp32", **over) -> Params:
    lib = load_library()
    p = Params()
    _check(lib.swe_params_default(C.byref(p), SCHEME.get(scheme, scheme), PRECISION.get(precision, precision)))
    for k, v in over.items():
        if k == "time_scheme":
            v = TIME_SCHEME.get(v, v)
        elif k == "waf_limiter":
            v = WAF_LIMITER.get(v, v)
        elif k == "kernel":
            v = KERNEL.get(v, v)
        elif k == "cfl_mode":
            v = CFL_MODE.get(v, v)
        elif k == "waf_ratio":
            v = WAF_RATIO.get(v, v)
        setattr(p, k, v)
    return p


def swe_mesh_create(nodes, tris, bnd_edges=None, bnd_tag=None, cut_edges=None, reorder="morton"):
    lib = load_library()
    nodes, tris = _f64(nodes), _i32(tris)
    be = _i32(bnd_edges if bnd_edges is not None else np.zeros((0, 2)))
    bt = _i32(bnd_tag if bnd_tag is not None else np.zeros(0))
    ce = _i32(cut_edges if cut_edges is not None else np.zeros((0, 2)))
    h = C.c_void_p()
    _check(lib.swe_mesh_create(_p(nodes), len(nodes), _p(tris), len(tris), _p(be), _p(bt), len(bt),
                               _p(ce) if len(ce) else None, len(ce), REORDER.get(reorder, reorder), C.byref(h)))
    return h


def swe_mesh_destroy(m):
    load_library().swe_mesh_destroy(m)


def swe_mesh_info(m):
    n, r = C.c_int64(), C.c_double()
    _check(load_library().swe_mesh_info(m, C.byref(n), C.byref(r)))
    return n.value, r.value


def swe_mesh_export(m):
    n, _ = swe_mesh_info(m)
    a = {"perm": np.empty(n, np.int32), "tri": np.empty((n, 3), np.int32), "nbr": np.empty((n, 3), np.int32),
         "nbr_edge": np.empty((n, 3), np.int32), "btag": np.empty((n, 3), np.int32),
         "lnx": np.empty((n, 3)), "lny": np.empty((n, 3)), "area": np.empty(n), "cx": np.empty(n),
         "cy": np.empty(n), "rin": np.empty(n), "dx": np.empty((n, 3)), "dy": np.empty((n, 3))}
    _check(load_library().swe_mesh_export(m, *[_p(a[k]) for k in (
        "perm", "tri", "nbr", "nbr_edge", "btag", "lnx", "lny", "area", "cx", "cy", "rin", "dx", "dy")]))
    return a


def swe_state_init(mesh, params: Params, h, hu, hv, z, manning_n=None, q_in=(), level=(), stream=None):
    lib = load_library()
    h, hu, hv, z = _f64(h), _f64(hu), _f64(hv), _f64(z)
    nm = None if manning_n is None else _f64(manning_n)
    qa, la = _f64(np.asarray(q_in, dtype=np.float64).reshape(-1)), _f64(np.asarray(level, dtype=np.float64).reshape(-1))
    bc = BcValues(len(qa), qa.ctypes.data_as(C.POINTER(C.c_double)) if len(qa) else None,
                  len(la), la.ctypes.data_as(C.POINTER(C.c_double)) if len(la) else None)
    out = C.c_void_p()
    _check(lib.swe_state_init(mesh, C.byref(params), _p(h), _p(hu), _p(hv), _p(z), _p(nm), C.byref(bc),
                              stream if stream is not None else _current_stream(), C.byref(out)))
    return out


def swe_state_destroy(s):
    load_library().swe_state_destroy(s)


def swe_set_stream(s, stream=None):
    _check(load_library().swe_set_stream(s, stream if stream is not None else _current_stream()))


def swe_set_state(s, h, hu, hv):
    h, hu, hv = _f64(h), _f64(hu), _f64(hv)
    _check(load_library().swe_set_state(s, _p(h), _p(hu), _p(hv)))


def swe_step(s, n_steps, cfl=0.9):
    _check(load_library().swe_step(s, int(n_steps), float(cfl)))


def swe_step_dt(s, dt):
    dt = _f64(dt)
    _check(load_library().swe_step_dt(s, _p(dt), len(dt)))


def swe_sync(s):
    _check(load_library().swe_sync(s))


def swe_get_state(s, n, out=None):
    if out is None:
        out = (np.empty(n), np.empty(n), np.empty(n))
    _check(load_library().swe_get_state(s, *[_p(a) for a in out]))
    return out


def swe_mass(s):
    m, c, b = C.c_double(), C.c_double(), C.c_double()
    _check(load_library().swe_mass(s, C.byref(m), C.byref(c), C.byref(b)))
    return m.value, c.value, b.value


def swe_time(s):
    t, k = C.c_double(), C.c_int64()
    _check(load_library().swe_time(s, C.byref(t), C.byref(k)))
    return t.value, k.value


def swe_flags(s):
    f = C.c_int()
    _check(load_library().swe_flags(s, C.byref(f)))
    return f.value


def swe_state_info(s):
    b, k, bl = C.c_int64(), C.c_int(), C.c_int()
    _check(load_library().swe_state_info(s, C.byref(b), C.byref(k), C.byref(bl)))
    return b.value, k.value, bl.value


def swe_profile_begin(s):
    _check(load_library().swe_profile_begin(s))


def swe_profile_end(s):
    """Per kernel kind: (summed device ms, launches)."""
    ms = np.zeros(8)
    cnt = np.zeros(8, np.int64)
    _check(load_library().swe_profile_end(s, _p(ms), _p(cnt)))
    return {KERNEL_KINDS[q]: (float(ms[q]), int(cnt[q])) for q in range(8) if cnt[q]}


def swe_dt_history(s, n):
    out = np.empty(n)
    _check(load_library().swe_dt_history(s, _p(out), int(n)))
    return out


def swe_muscl_step_noalloc(n_cells, nbr, ln, z, manning_n, h, hu, hv, h_out, hu_out, hv_out, dt,
                           params: Params, inflow_qlen=(), level=(), stream=None):
    """Device pointers (ints) in, device pointers out; no allocation inside."""
    qa = np.ascontiguousarray(inflow_qlen, dtype=np.float32).reshape(-1)
    la = np.ascontiguousarray(level, dtype=np.float32).reshape(-1)
    _check(load_library().swe_muscl_step_noalloc(
        int(n_cells), nbr, ln, z, manning_n, h, hu, hv, h_out, hu_out, hv_out, float(dt), C.byref(params),
        _p(qa) if len(qa) else None, len(qa), _p(la) if len(la) else None, len(la),
        stream if stream is not None else _current_stream()))


def swe_autotune(s, mesh=None, trial_steps=8, cfl=0.9):
    """Returns (kernel name, block, ms per step) of the fastest configuration, now in use."""
    k, b, ms = C.c_int(), C.c_int(), C.c_double()
    _check(load_library().swe_autotune(s, mesh, int(trial_steps), float(cfl), C.byref(k), C.byref(b), C.byref(ms)))
    return {1: "split", 2: "fused"}.get(k.value, k.value), b.value, ms.value


def swe_ensemble_autotune(e, meshes=None, trial_steps=8, cfl=0.9):
    k, b, ms = C.c_int(), C.c_int(), C.c_double()
    arr = None
    if meshes is not None:
        arr = (C.c_void_p * len(meshes))(*[m.value if isinstance(m, C.c_void_p) else m for m in meshes])
    _check(load_library().swe_ensemble_autotune(e, arr, int(trial_steps), float(cfl), C.byref(k), C.byref(b),
                                                C.byref(ms)))
    return {1: "split", 2: "fused"}.get(k.value, k.value), b.value, ms.value


def swe_ensemble_create(states):
    arr = (C.c_void_p * len(states))(*[s.value if isinstance(s, C.c_void_p) else s for s in states])
    out = C.c_void_p()
    _check(load_library().swe_ensemble_create(arr, len(states), C.byref(out)))
    return out


def swe_ensemble_destroy(e):
    load_library().swe_ensemble_destroy(e)


def swe_ensemble_step(e, n_steps, cfl=0.9):
    _check(load_library().swe_ensemble_step(e, int(n_steps), float(cfl)))


def swe_ensemble_sync(e):
    _check(load_library().swe_ensemble_sync(e))


# ---- convenience wrappers ---------------------------------------------------

def swe_partition_create(mesh, n_parts):
    out = C.c_void_p()
    _check(load_library().swe_partition_create(mesh, int(n_parts), C.byref(out)))
    return out


def swe_partition_destroy(p):
    load_library().swe_partition_destroy(p)


def swe_partition_info(p, part):
    v = [C.c_int64() for _ in range(5)]
    _check(load_library().swe_partition_info(p, int(part), *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)        # owned_begin, owned_end, n_halo1, n_halo2, n_boundary


def swe_partition_export(p, part):
    _, _, n1, n2, nb = swe_partition_info(p, part)
    h1, h2, b = (np.empty(max(k, 1), np.int32) for k in (n1, n2, nb))
    _check(load_library().swe_partition_export(p, int(part), _p(h1), _p(h2), _p(b)))
    return h1[:n1], h2[:n2], b[:nb]


def swe_tile_plan_info(m, tile):
    nt, nw = C.c_int64(), C.c_int64()
    hm, h1, wm = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load_library().swe_tile_plan_info(m, int(tile), C.byref(nt), C.byref(hm), C.byref(h1), C.byref(wm),
                                             C.byref(nw)))
    return {"n_tiles": nt.value, "hmax": hm.value, "h1max": h1.value, "wmax": wm.value, "n_words": nw.value}


def swe_tile_plan_export(m, tile):
    """The tile step's plan of mesh handle m: (info dict, hdr[n_tiles, 8], words)."""
    info = swe_tile_plan_info(m, tile)
    hdr = np.empty(max(8 * info["n_tiles"], 1), np.int32)
    words = np.empty(max(info["n_words"], 1), np.int32)
    _check(load_library().swe_tile_plan_export(m, int(tile), _p(hdr), _p(words)))
    return info, hdr[:8 * info["n_tiles"]].reshape(-1, 8), words[:info["n_words"]]


def swe_set_partition(s, p):
    _check(load_library().swe_set_partition(s, p))


def swe_halo_get(s, part, n):
    h, hu, hv = np.empty(max(n, 1)), np.empty(max(n, 1)), np.empty(max(n, 1))
    _check(load_library().swe_halo_get(s, int(part), _p(h), _p(hu), _p(hv)))
    return h[:n], hu[:n], hv[:n]


def swe_probe_bounded_wait(polls, arrive, stream=None):
    """Run the bounded-wait self-check; True if the wait gave up (see include/swe.h)."""
    out = C.c_int(-1)
    _check(load_library().swe_probe_bounded_wait(int(polls), int(arrive), C.byref(out), stream))
    return out.value == 1


def swe_fma_peak(precision="fp32", iters=None, stream=None):
    """Fused multiply-add rate of the GPU (FLOP/s, an FMA counted as two)."""
    prec = PRECISION.get(precision, precision)
    if iters is None:
        iters = 65536 if prec == PRECISION["fp32"] else 2048
    out = C.c_double(0.0)
    _check(load_library().swe_fma_peak(prec, int(iters), stream, C.byref(out)))
    return out.value


class Mesh:
    """Owning wrapper of a swe_mesh handle."""

    def __init__(self, nodes, tris, bnd_edges=None, bnd_tag=None, cut_edges=None, reorder="morton"):
        self.handle = swe_mesh_create(nodes, tris, bnd_edges, bnd_tag, cut_edges, reorder)
        self.n, self.r_min = swe_mesh_info(self.handle)

    @classmethod
    def from_workload(cls, w, reorder="morton"):
        return cls(w.nodes, w.tris, w.bnd_edges, w.bnd_tag, w.cut_edges if len(w.cut_edges) else None, reorder)

    def export(self):
        return swe_mesh_export(self.handle)

    def close(self):
        if self.handle:
            swe_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """Owning wrapper of a swe_state handle."""

    def __init__(self, mesh: Mesh, params: Params, h, hu, hv, z, manning_n=None, q_in=(), level=(), stream=None):
        self.n = mesh.n
        self.handle = swe_state_init(mesh.handle, params, h, hu, hv, z, manning_n, q_in, level, stream)

    @classmethod
    def from_workload(cls, mesh, params, w):
        return cls(mesh, params, w.h, w.hu, w.hv, w.z, w.nman, w.q_in, w.level)

    def step(self, n_steps, cfl=0.9):
        swe_step(self.handle, n_steps, cfl)

    def step_dt(self, dt):
        swe_step_dt(self.handle, dt)

    def sync(self):
        swe_sync(self.handle)

    def set_state(self, h, hu, hv):
        swe_set_state(self.handle, h, hu, hv)

    def get_state(self, out=None):
        return swe_get_state(self.handle, self.n, out)

    def mass(self):
        return swe_mass(self.handle)

    def time(self):
        return swe_time(self.handle)

    def flags(self):
        """Bit flags since init: FLAG_CLIPPED (a negative depth was clipped), FLAG_NONFINITE, FLAG_DRY."""
        return swe_flags(self.handle)

    def info(self):
        return swe_state_info(self.handle)

    def dt_history(self, n):
        return swe_dt_history(self.handle, n)

    def profile_begin(self):
        swe_profile_begin(self.handle)

    def profile_end(self):
        return swe_profile_end(self.handle)

    def set_partition(self, partition):
        swe_set_partition(self.handle, partition.handle if partition is not None else None)

    def halo(self, partition, part):
        _, _, n1, n2, _ = partition.info(part)
        return swe_halo_get(self.handle, part, n1 + n2)

    def autotune(self, mesh=None, trial_steps=8, cfl=0.9):
        return swe_autotune(self.handle, mesh.handle if mesh is not None else None, trial_steps, cfl)

    def close(self):
        if self.handle:
            swe_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Partition:
    """Owning wrapper of a swe_partition handle (sub-domains with two halo layers)."""

    def __init__(self, mesh: "Mesh", n_parts: int):
        self.n_parts = int(n_parts)
        self.handle = swe_partition_create(mesh.handle, n_parts)

    def info(self, part):
        return swe_partition_info(self.handle, part)

    def export(self, part):
        return swe_partition_export(self.handle, part)

    def close(self):
        if self.handle:
            swe_partition_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Owning wrapper of a swe_ensemble handle (the member states stay owned by the caller)."""

    def __init__(self, states):
        self.states = list(states)
        self.handle = swe_ensemble_create([st.handle for st in self.states])

    def step(self, n_steps, cfl=0.9):
        swe_ensemble_step(self.handle, n_steps, cfl)

    def sync(self):
        swe_ensemble_sync(self.handle)

    def autotune(self, meshes=None, trial_steps=8, cfl=0.9):
        return swe_ensemble_autotune(self.handle, [m.handle for m in meshes] if meshes is not None else None,
                                     trial_steps, cfl)

    def close(self):
        if self.handle:
            swe_ensemble_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
