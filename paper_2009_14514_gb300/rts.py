"""Thin ctypes binding of librts (the C ABI in include/rts.h), same names as the ABI.

Argument marshalling only: every step of the method runs in the CUDA library.  Arrays
may be numpy arrays (host) or torch tensors (host or CUDA); vectors are (n, 3) float32
in the caller's particle order.  The stream defaults to torch's current CUDA stream.
If the library cannot be loaded, every call raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

RTS_OK = 0
RTS_ERR_ARG, RTS_ERR_DOMAIN, RTS_ERR_CUDA, RTS_ERR_OOM, RTS_ERR_CAPACITY = 1, 2, 3, 4, 5
RTS_ERR_NOT_CONVERGED, RTS_ERR_TIMEOUT, RTS_ERR_STATE, RTS_ERR_INTERNAL = 6, 7, 8, 9
STATUS_NAMES = {
    0: "RTS_OK", 1: "RTS_ERR_ARG", 2: "RTS_ERR_DOMAIN", 3: "RTS_ERR_CUDA", 4: "RTS_ERR_OOM",
    5: "RTS_ERR_CAPACITY", 6: "RTS_ERR_NOT_CONVERGED", 7: "RTS_ERR_TIMEOUT", 8: "RTS_ERR_STATE", 9: "RTS_ERR_INTERNAL",
}
EXPORTED = [
    "rts_init", "rts_bin", "rts_classify_blocks", "rts_evaluate", "rts_wcsph_substep",
    "rts_pcisph_step", "rts_advance", "rts_get_state", "rts_set_state", "rts_get_bins",
    "rts_get_blocks", "rts_sync", "rts_num_blocks", "rts_substep_index", "rts_last_error",
    "rts_destroy", "rts_profile_enable", "rts_profile_read", "rts_bin_noalloc",
    "rts_pcisph_last", "rts_get_pcisph_state", "rts_get_neighbors",
    "rts_diff_create", "rts_diff_forward", "rts_diff_backward", "rts_diff_last_error",
    "rts_diff_destroy",
    "rts_batch_init", "rts_batch_scene_info", "rts_batch_layout", "rts_batch_set_launch",
    "rts_batch_get_launch", "rts_batch_autotune",
]


class RtsError(RuntimeError):
    def __init__(self, status, what, msg):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}: {msg}")


class RtsParams(C.Structure):
    _fields_ = [
        ("scheme", C.c_int32), ("mode", C.c_int32), ("force_level", C.c_int32),
        ("spacing", C.c_float), ("support_r", C.c_float), ("block_edge", C.c_float),
        ("domain_min", C.c_float * 3), ("grid_dim", C.c_int32 * 3),
        ("rho0", C.c_float), ("c_s", C.c_float), ("gamma", C.c_float), ("visc_alpha", C.c_float),
        ("gravity", C.c_float * 3),
        ("lambda_v", C.c_float), ("lambda_f", C.c_float), ("alpha", C.c_float),
        ("n_levels", C.c_int32), ("level_mult", C.c_int32 * 8), ("beta", C.c_float * 8),
        ("dt_b", C.c_float), ("max_per_block", C.c_int32),
        ("n_minor", C.c_int32), ("eta", C.c_float), ("eta_T", C.c_float),
        ("max_iters", C.c_int32), ("max_global_iters", C.c_int32), ("max_local_iters", C.c_int32),
        ("expand_layers", C.c_int32), ("r1_search_rings", C.c_int32),
        ("clean_majors", C.c_int32), ("short_minor", C.c_int32),
        ("sched", (C.c_int32 * 8) * 4), ("refresh", C.c_int32 * 8),
        ("max_neighbors", C.c_int32),
        ("wall_project", C.c_int32),
        ("wall_lo", C.c_float * 3),
        ("wall_hi", C.c_float * 3),
        ("level_clock", C.c_int32),
        ("tait_B", C.c_float),
        ("tait_no_clamp", C.c_int32),
        ("serna_off", C.c_int32),
        ("r2_search_rings", C.c_int32),
        ("stale_bins", C.c_int32),
    ]


class RtsStats(C.Structure):
    _fields_ = [
        ("substeps", C.c_int64), ("steps", C.c_int64), ("particle_evals", C.c_int64),
        ("pair_interactions", C.c_int64), ("active_blocks", C.c_int64),
        ("level_count", C.c_int64 * 8), ("candidate_tests", C.c_int64),
        ("tests_performed", C.c_int64),
        ("pcisph_iterations", C.c_int64),
        ("pcisph_local_iterations", C.c_int64), ("pcisph_global_restarts", C.c_int64),
        ("t_sim", C.c_double),
    ]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "level_count"}
        d["level_count"] = list(self.level_count)
        return d


class RtsScene(C.Structure):
    _fields_ = [("n_fluid", C.c_int32), ("n_boundary", C.c_int32),
                ("domain_min", C.c_float * 3), ("grid_dim", C.c_int32 * 3),
                ("wall_lo", C.c_float * 3), ("wall_hi", C.c_float * 3)]


PHASES = ["bin", "classify", "activity", "density", "force", "correct", "iterate", "other"]


class RtsPcisphInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("global_iterations", C.c_int32),
                ("local_iterations", C.c_int32), ("reverts", C.c_int32),
                ("not_converged", C.c_int32), ("minor", C.c_int32),
                ("n_minor_current", C.c_int32), ("clean_majors", C.c_int32),
                ("err_max", C.c_double), ("err_avg", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class RtsProfile(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("launches", C.c_int64 * 8), ("kernels", C.c_int64),
                ("timed", C.c_int64 * 8), ("passes", C.c_int64 * 8)]

    def as_dict(self):
        return {"ms": dict(zip(PHASES, list(self.ms))),
                "launches": dict(zip(PHASES, list(self.launches))), "kernels": self.kernels,
                "timed": dict(zip(PHASES, list(self.timed))),
                "passes": dict(zip(PHASES, list(self.passes)))}


def make_params(d: dict) -> RtsParams:
    P = RtsParams()
    P.scheme = int(d["scheme"])
    P.mode = int(d.get("mode", 0))
    P.force_level = int(d.get("force_level", -1))
    P.spacing = d["spacing"]
    P.support_r = d["support_r"]
    P.block_edge = d["block_edge"]
    for k in range(3):
        P.domain_min[k] = d["domain_min"][k]
        P.grid_dim[k] = int(d["grid_dim"][k])
        P.gravity[k] = d["gravity"][k]
    for f in ("rho0", "c_s", "gamma", "visc_alpha", "lambda_v", "lambda_f", "alpha", "dt_b",
              "eta", "eta_T"):
        setattr(P, f, float(d[f]))
    P.n_levels = int(d["n_levels"])
    for L in range(min(8, len(d["level_mult"]))):
        P.level_mult[L] = int(d["level_mult"][L])
        P.beta[L] = float(d["beta"][L])
    for f in ("max_per_block", "n_minor", "max_iters", "max_global_iters", "max_local_iters",
              "expand_layers", "r1_search_rings", "clean_majors", "short_minor", "max_neighbors"):
        setattr(P, f, int(d[f]))
    for n in range(4):
        for j in range(len(d["sched"][n])):
            P.sched[n][j] = int(d["sched"][n][j])
    for L in range(len(d["refresh"])):
        P.refresh[L] = int(d["refresh"][L])
    P.wall_project = int(d.get("wall_project", 0))
    for k in range(3):
        P.wall_lo[k] = d.get("wall_lo", [0.0] * 3)[k]
        P.wall_hi[k] = d.get("wall_hi", [0.0] * 3)[k]
    P.level_clock = int(d.get("level_clock", 0))
    P.tait_B = float(d.get("tait_B", 0.0))
    P.tait_no_clamp = int(d.get("tait_no_clamp", 0))
    P.serna_off = int(d.get("serna_off", 0))
    P.r2_search_rings = int(d.get("r2_search_rings", 1))
    P.stale_bins = int(d.get("stale_bins", 0))
    return P


_LIB = None


def lib():
    """Load librts (building it in-tree if needed).  Raises if that fails."""
    global _LIB
    if _LIB is None:
        path = _build.build() if not os.environ.get("RTS_NO_BUILD") else _build.LIB
        L = C.CDLL(path)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "rts_init": [vp, i32, vp, vp, i32, vp, vp, vp],
            "rts_bin": [vp], "rts_classify_blocks": [vp], "rts_evaluate": [vp],
            "rts_wcsph_substep": [vp], "rts_pcisph_step": [vp],
            "rts_advance": [vp, C.c_double, vp],
            "rts_get_state": [vp] * 11,
            "rts_set_state": [vp] * 9 + [i64, i32],
            "rts_get_bins": [vp] * 4, "rts_get_blocks": [vp] * 3, "rts_sync": [vp],
            "rts_destroy": [vp], "rts_profile_enable": [vp, i32],
            "rts_profile_read": [vp, vp, i32],
            "rts_bin_noalloc": [vp, i32, vp, vp, vp, vp, vp],
            "rts_pcisph_last": [vp, vp], "rts_get_pcisph_state": [vp, vp, vp, vp],
            "rts_get_neighbors": [vp, vp, vp, i32],
            "rts_diff_create": [vp, i32, vp, i32, vp, i32, i32, vp, vp],
            "rts_diff_forward": [vp, vp, C.c_float, C.c_float, vp, vp],
            "rts_diff_backward": [vp, vp, vp, vp, vp, vp],
            "rts_batch_init": [vp, i32, vp, vp, vp, vp, vp, vp],
            "rts_batch_scene_info": [vp, i32, vp],
            "rts_batch_layout": [vp, vp, vp, vp, vp],
            "rts_batch_set_launch": [vp, i32, i32, i32],
            "rts_batch_get_launch": [vp, vp, vp, vp, vp],
            "rts_batch_autotune": [vp, i32, vp, vp, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.rts_last_error.argtypes = [vp]
        L.rts_last_error.restype = C.c_char_p
        L.rts_num_blocks.argtypes = [vp]
        L.rts_num_blocks.restype = i64
        L.rts_substep_index.argtypes = [vp]
        L.rts_substep_index.restype = i64
        L.rts_diff_last_error.argtypes = [vp]
        L.rts_diff_last_error.restype = C.c_char_p
        L.rts_diff_destroy.argtypes = [vp]
        L.rts_diff_destroy.restype = None
        _LIB = L
    return _LIB


def library_path() -> str:
    return _build.LIB


# ------------------------------------------------------------- marshalling ---

def _ptr(a):
    """Pointer of a numpy array or torch tensor (contiguous), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported array type {type(a)}")


def _f32(a, n, width=3):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, np.float32)
    elif hasattr(a, "dtype"):
        import torch
        if a.dtype != torch.float32:
            raise TypeError("tensors must be float32")
    shape = tuple(a.shape)
    want = (n, width) if width > 1 else (n,)
    if shape != want and not (width > 1 and n == 0):
        raise ValueError(f"expected shape {want}, got {shape}")
    return a


def _i32(a, n):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, np.int32)
    if tuple(a.shape) != (n,):
        raise ValueError(f"expected shape ({n},), got {tuple(a.shape)}")
    return a


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return C.c_void_p(0)


class Ctx:
    """Owner of an rts_ctx handle (destroyed on close / garbage collection)."""

    def __init__(self, handle, params, n, nb):
        self.handle = handle
        self.params = params
        self.n = n
        self.nb = nb

    def close(self):
        if self.handle:
            lib().rts_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_blocks(self):
        return lib().rts_num_blocks(self.handle)

    @property
    def substep_index(self):
        return lib().rts_substep_index(self.handle)


def _check(st, what, ctx=None):
    if st != RTS_OK:
        h = ctx.handle if isinstance(ctx, Ctx) else None
        msg = lib().rts_last_error(h)
        raise RtsError(st, what, msg.decode() if msg else "")
    return st


# ------------------------------------------------------------------- calls ---

def rts_init(params, x, v, xb, stream=None) -> Ctx:
    P = params if isinstance(params, RtsParams) else make_params(params)
    n = int(x.shape[0])
    nb = int(xb.shape[0])
    x, v, xb = _f32(x, n), _f32(v, n), _f32(xb, nb)
    h = C.c_void_p()
    st = lib().rts_init(C.byref(P), n, _ptr(x), _ptr(v), nb, _ptr(xb), _stream(stream), C.byref(h))
    _check(st, "rts_init")
    return Ctx(h, P, n, nb)


def rts_bin(ctx):
    return _check(lib().rts_bin(ctx.handle), "rts_bin", ctx)


def rts_classify_blocks(ctx):
    return _check(lib().rts_classify_blocks(ctx.handle), "rts_classify_blocks", ctx)


def rts_evaluate(ctx):
    return _check(lib().rts_evaluate(ctx.handle), "rts_evaluate", ctx)


def rts_wcsph_substep(ctx):
    return _check(lib().rts_wcsph_substep(ctx.handle), "rts_wcsph_substep", ctx)


def rts_pcisph_step(ctx, allow_not_converged=True):
    st = lib().rts_pcisph_step(ctx.handle)
    if allow_not_converged and st == 6:
        return st
    return _check(st, "rts_pcisph_step", ctx)


def rts_advance(ctx, t_sim, allow_not_converged=True) -> dict:
    s = RtsStats()
    st = lib().rts_advance(ctx.handle, float(t_sim), C.byref(s))
    if not (allow_not_converged and st == 6):
        _check(st, "rts_advance", ctx)
    return s.as_dict()


def rts_sync(ctx, allow_not_converged=True):
    st = lib().rts_sync(ctx.handle)
    if allow_not_converged and st == 6:
        return st
    return _check(st, "rts_sync", ctx)


def rts_get_state(ctx, fields=("x", "v", "a", "rho", "p", "level", "validity", "klast", "nbr",
                               "compute")) -> dict:
    """State in the caller's order as numpy arrays (host)."""
    n = ctx.n
    out = {}
    spec = {"x": (np.float32, 3), "v": (np.float32, 3), "a": (np.float32, 3),
            "rho": (np.float32, 1), "p": (np.float32, 1), "level": (np.int32, 1),
            "validity": (np.int32, 1), "klast": (np.int32, 1), "nbr": (np.int32, 1),
            "compute": (np.uint8, 1)}
    for f in fields:
        dt, w = spec[f]
        out[f] = np.zeros((n, 3) if w == 3 else (n,), dt)
    args = [_ptr(out.get(f)) for f in ("x", "v", "a", "rho", "p", "level", "validity", "klast",
                                      "nbr", "compute")]
    _check(lib().rts_get_state(ctx.handle, *args), "rts_get_state", ctx)
    return out


def rts_get_state_into(ctx, x=None, v=None, a=None, rho=None, p=None, level=None,
                       validity=None, klast=None, nbr=None, compute=None):
    """Copy state into caller-provided buffers (numpy or torch, host or device)."""
    _check(lib().rts_get_state(ctx.handle, _ptr(x), _ptr(v), _ptr(a), _ptr(rho), _ptr(p),
                               _ptr(level), _ptr(validity), _ptr(klast), _ptr(nbr),
                               _ptr(compute)), "rts_get_state", ctx)


def rts_profile_enable(ctx, on=True):
    """on: False/0 off, True/1 every phase, 2 only the density and force passes."""
    level = int(on) if not isinstance(on, bool) else (1 if on else 0)
    return _check(lib().rts_profile_enable(ctx.handle, level), "rts_profile_enable", ctx)


def rts_profile_read(ctx, reset=False) -> dict:
    prof = RtsProfile()
    _check(lib().rts_profile_read(ctx.handle, C.byref(prof), 1 if reset else 0),
           "rts_profile_read", ctx)
    return prof.as_dict()


def rts_set_state(ctx, x, v, a=None, rho=None, p=None, level=None, validity=None, klast=None,
                  k=0, primed=False):
    n = ctx.n
    x, v, a = _f32(x, n), _f32(v, n), _f32(a, n)
    rho, p = _f32(rho, n, 1), _f32(p, n, 1)
    level, validity, klast = _i32(level, n), _i32(validity, n), _i32(klast, n)
    st = lib().rts_set_state(ctx.handle, _ptr(x), _ptr(v), _ptr(a), _ptr(rho), _ptr(p),
                             _ptr(level), _ptr(validity), _ptr(klast), int(k), 1 if primed else 0)
    return _check(st, "rts_set_state", ctx)


def rts_get_bins(ctx):
    n = ctx.n
    B = ctx.num_blocks
    key = np.zeros(n, np.int32)
    perm = np.zeros(n, np.int32)
    cstart = np.zeros(B + 1, np.int32)
    _check(lib().rts_get_bins(ctx.handle, _ptr(key), _ptr(perm), _ptr(cstart)), "rts_get_bins", ctx)
    return key, perm, cstart


def rts_get_blocks(ctx):
    B = ctx.num_blocks
    raw = np.zeros(B, np.int32)
    lev = np.zeros(B, np.int32)
    _check(lib().rts_get_blocks(ctx.handle, _ptr(raw), _ptr(lev)), "rts_get_blocks", ctx)
    return raw, lev


def rts_destroy(ctx):
    ctx.close()


def rts_last_error(ctx=None) -> str:
    h = ctx.handle if isinstance(ctx, Ctx) else None
    return lib().rts_last_error(h).decode()


def _noalloc_args(P, x, key, perm, cstart):
    """Validate rts_bin_noalloc's arguments before any pointer reaches the library: the
    library writes n entries of key and perm and nblocks + 1 of cstart into device memory
    of the current device, so a short or host buffer would be written out of bounds."""
    import torch
    named = (("x", x), ("key", key), ("perm", perm), ("cstart", cstart))
    for name, t in named:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"rts_bin_noalloc: {name} must be a torch tensor, not {type(t).__name__}")
        if not t.is_contiguous():
            raise ValueError(f"rts_bin_noalloc: {name} must be contiguous")
    if x.dtype != torch.float32 or x.dim() != 2 or x.shape[1] != 3:
        raise ValueError(f"rts_bin_noalloc: x must be float32 of shape (n, 3), not "
                         f"{x.dtype} {tuple(x.shape)}")
    n = int(x.shape[0])
    nblocks = int(P.grid_dim[0]) * int(P.grid_dim[1]) * int(P.grid_dim[2])
    for name, t, need in (("key", key, n), ("perm", perm, n), ("cstart", cstart, nblocks + 1)):
        if t.dtype != torch.int32:
            raise ValueError(f"rts_bin_noalloc: {name} must be int32, not {t.dtype}")
        if t.numel() < need:
            raise ValueError(f"rts_bin_noalloc: {name} holds {t.numel()} entries, needs {need}")
    for name, t in named:
        if not t.is_cuda:
            raise ValueError(f"rts_bin_noalloc: {name} must be in device memory (a CUDA tensor)")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"rts_bin_noalloc: {name} is on cuda:{t.device.index}, the current "
                             f"device is cuda:{torch.cuda.current_device()}")
    return n


def rts_bin_noalloc(params, x, key, perm, cstart, stream=None):
    """Binning without device allocation (see rts.h): x (n x 3 float32), key and perm
    (int32, >= n entries) and cstart (int32, >= nblocks + 1 entries) are contiguous CUDA
    tensors on the current device that the caller owns.  For callers that cannot
    allocate device memory.  Raises ValueError on any other argument, before the call."""
    P = params if isinstance(params, RtsParams) else make_params(params)
    n = _noalloc_args(P, x, key, perm, cstart)
    st = lib().rts_bin_noalloc(C.byref(P), n, _ptr(x), _ptr(key), _ptr(perm), _ptr(cstart),
                               _stream(stream))
    return _check(st, "rts_bin_noalloc")


def rts_pcisph_last(ctx) -> dict:
    info = RtsPcisphInfo()
    _check(lib().rts_pcisph_last(ctx.handle, C.byref(info)), "rts_pcisph_last", ctx)
    return info.as_dict()


def rts_get_pcisph_state(ctx) -> dict:
    n = ctx.n
    out = {"ap": np.zeros((n, 3), np.float32), "err": np.zeros(n, np.float32),
           "in_se": np.zeros(n, np.uint8)}
    _check(lib().rts_get_pcisph_state(ctx.handle, _ptr(out["ap"]), _ptr(out["err"]),
                                      _ptr(out["in_se"])), "rts_get_pcisph_state", ctx)
    return out


def rts_get_neighbors(ctx, cap=None):
    """Neighbour lists (caller indices; boundary b as n + b) as a list of arrays."""
    n = ctx.n
    cap = int(cap or ctx.params.max_neighbors)
    counts = np.zeros(n, np.int32)
    idx = np.zeros(max(n, 1) * cap, np.int32)
    _check(lib().rts_get_neighbors(ctx.handle, _ptr(counts), _ptr(idx), cap), "rts_get_neighbors", ctx)
    return [idx[i * cap: i * cap + counts[i]] for i in range(n)]


# ------------------------------------------------------------ batched scenes ---

def rts_batch_init(params, scenes_desc, x, v, xb, stream=None) -> Ctx:
    """Batched RTS-PCISPH over many scenes (see rts.h).  scenes_desc: one dict per scene
    with n_fluid, n_boundary, domain_min, grid_dim, wall_lo, wall_hi; x, v: all scenes'
    fluid particles concatenated, xb: all boundary particles concatenated."""
    P = params if isinstance(params, RtsParams) else make_params(params)
    ns = len(scenes_desc)
    arr = (RtsScene * max(ns, 1))()
    for k, d in enumerate(scenes_desc):
        arr[k].n_fluid = int(d["n_fluid"])
        arr[k].n_boundary = int(d["n_boundary"])
        for a in range(3):
            arr[k].domain_min[a] = float(d["domain_min"][a])
            arr[k].grid_dim[a] = int(d["grid_dim"][a])
            arr[k].wall_lo[a] = float(d.get("wall_lo", [0.0] * 3)[a])
            arr[k].wall_hi[a] = float(d.get("wall_hi", [0.0] * 3)[a])
    n = int(x.shape[0])
    nb = int(xb.shape[0])
    x, v, xb = _f32(x, n), _f32(v, n), _f32(xb, nb)
    h = C.c_void_p()
    st = lib().rts_batch_init(C.byref(P), ns, arr, _ptr(x), _ptr(v), _ptr(xb), _stream(stream),
                              C.byref(h))
    _check(st, "rts_batch_init")
    ctx = Ctx(h, P, n, nb)
    ctx.n_scenes = ns
    return ctx


def rts_batch_scene_info(ctx, scene) -> dict:
    info = RtsPcisphInfo()
    _check(lib().rts_batch_scene_info(ctx.handle, int(scene), C.byref(info)),
           "rts_batch_scene_info", ctx)
    return info.as_dict()


def rts_batch_layout(ctx) -> dict:
    ns = ctx.n_scenes
    dims = np.zeros(3, np.int32)
    z0 = np.zeros(ns + 1, np.int32)
    fb = np.zeros(ns + 1, np.int32)
    bb = np.zeros(ns + 1, np.int32)
    _check(lib().rts_batch_layout(ctx.handle, _ptr(dims), _ptr(z0), _ptr(fb), _ptr(bb)),
           "rts_batch_layout", ctx)
    return {"grid_dim": dims, "z0": z0, "fluid_base": fb, "boundary_base": bb}


def rts_batch_set_launch(ctx, threads=256, tile=128, use_graph=True):
    return _check(lib().rts_batch_set_launch(ctx.handle, int(threads), int(tile),
                                             1 if use_graph else 0), "rts_batch_set_launch", ctx)


def rts_batch_get_launch(ctx) -> dict:
    t, l, g = C.c_int32(), C.c_int32(), C.c_int32()
    it = C.c_int64()
    _check(lib().rts_batch_get_launch(ctx.handle, C.byref(t), C.byref(l), C.byref(g), C.byref(it)),
           "rts_batch_get_launch", ctx)
    return {"threads": t.value, "tile": l.value, "use_graph": bool(g.value),
            "iterations_run": it.value}


def rts_batch_autotune(ctx, reps=3) -> dict:
    t, l = C.c_int32(), C.c_int32()
    ms = C.c_float()
    _check(lib().rts_batch_autotune(ctx.handle, int(reps), C.byref(t), C.byref(l), C.byref(ms)),
           "rts_batch_autotune", ctx)
    return {"threads": t.value, "tile": l.value, "ms_per_iteration": ms.value}
