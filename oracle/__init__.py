"""ctypes wrapper of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  The oracle shares no code with the CUDA library; both are fed
the same seeded inputs from ``paper_2009_14514_gb300.scenes``.

Parameters are rounded to FP32 first (the values the CUDA library receives) and then
widened exactly to double, so both sides decide on the same numbers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build_oracle import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = C.CDLL(_build())
        _declare(_LIB)
    return _LIB


def _f32(v):
    return float(np.float64(np.float32(v)))


class OrcParams(C.Structure):
    _fields_ = [
        ("scheme", C.c_int32), ("mode", C.c_int32), ("force_level", C.c_int32),
        ("s", C.c_double), ("r", C.c_double), ("edge", C.c_double),
        ("origin", C.c_double * 3), ("dim", C.c_int32 * 3),
        ("rho0", C.c_double), ("c_s", C.c_double), ("gamma", C.c_double),
        ("visc_alpha", C.c_double), ("g", C.c_double * 3),
        ("lambda_v", C.c_double), ("lambda_f", C.c_double), ("alpha", C.c_double),
        ("n_levels", C.c_int32), ("mult", C.c_int32 * 8), ("beta", C.c_double * 8),
        ("dt_b", C.c_double), ("max_per_block", C.c_int32),
        ("n_minor", C.c_int32), ("eta", C.c_double), ("eta_T", C.c_double),
        ("max_iters", C.c_int32), ("max_global_iters", C.c_int32),
        ("max_local_iters", C.c_int32), ("expand_layers", C.c_int32),
        ("r1_rings", C.c_int32), ("clean_majors", C.c_int32), ("short_minor", C.c_int32),
        ("sched", (C.c_int32 * 8) * 4), ("refresh", C.c_int32 * 8),
        ("max_neighbors", C.c_int32),
        ("wall_project", C.c_int32),
        ("wall_lo", C.c_double * 3),
        ("wall_hi", C.c_double * 3),
        ("level_clock", C.c_int32),
        ("tait_B", C.c_double),
        ("tait_no_clamp", C.c_int32),
        ("serna_off", C.c_int32),
        ("r2_rings", C.c_int32),
    ]


def make_params(d: dict) -> OrcParams:
    P = OrcParams()
    P.scheme = int(d["scheme"])
    P.mode = int(d.get("mode", 0))
    P.force_level = int(d.get("force_level", -1))
    P.s = _f32(d["spacing"])
    P.r = _f32(d["support_r"])
    P.edge = _f32(d["block_edge"])
    for k in range(3):
        P.origin[k] = _f32(d["domain_min"][k])
        P.dim[k] = int(d["grid_dim"][k])
        P.g[k] = _f32(d["gravity"][k])
    P.rho0 = _f32(d["rho0"])
    P.c_s = _f32(d["c_s"])
    P.gamma = _f32(d["gamma"])
    P.visc_alpha = _f32(d["visc_alpha"])
    P.lambda_v = _f32(d["lambda_v"])
    P.lambda_f = _f32(d["lambda_f"])
    P.alpha = _f32(d["alpha"])
    P.n_levels = int(d["n_levels"])
    for L in range(int(d["n_levels"])):
        P.mult[L] = int(d["level_mult"][L])
        P.beta[L] = _f32(d["beta"][L])
    P.dt_b = _f32(d["dt_b"])
    P.max_per_block = int(d["max_per_block"])
    P.n_minor = int(d["n_minor"])
    P.eta = _f32(d["eta"])
    P.eta_T = _f32(d["eta_T"])
    P.max_iters = int(d["max_iters"])
    P.max_global_iters = int(d["max_global_iters"])
    P.max_local_iters = int(d["max_local_iters"])
    P.expand_layers = int(d["expand_layers"])
    P.r1_rings = int(d["r1_search_rings"])
    P.clean_majors = int(d["clean_majors"])
    P.short_minor = int(d["short_minor"])
    for n in range(4):
        for j in range(len(d["sched"][n])):
            P.sched[n][j] = int(d["sched"][n][j])
    for L in range(len(d["refresh"])):
        P.refresh[L] = int(d["refresh"][L])
    P.max_neighbors = int(d["max_neighbors"])
    P.wall_project = int(d.get("wall_project", 0))
    P.level_clock = int(d.get("level_clock", 0))
    P.tait_B = _f32(d.get("tait_B", 0.0))
    P.tait_no_clamp = int(d.get("tait_no_clamp", 0))
    P.serna_off = int(d.get("serna_off", 0))
    P.r2_rings = int(d.get("r2_search_rings", 1))
    for k in range(3):
        P.wall_lo[k] = _f32(d.get("wall_lo", [0.0] * 3)[k])
        P.wall_hi[k] = _f32(d.get("wall_hi", [0.0] * 3)[k])
    return P


class WState(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("nb", C.c_int32),
        ("x", C.c_void_p), ("v", C.c_void_p), ("a", C.c_void_p),
        ("rho", C.c_void_p), ("p", C.c_void_p),
        ("klast", C.c_void_p), ("validity", C.c_void_p), ("level", C.c_void_p),
        ("compute", C.c_void_p), ("nbr", C.c_void_p), ("xb", C.c_void_p),
        ("block_level", C.c_void_p), ("k", C.c_int64), ("primed", C.c_int32),
    ]


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _declare(L):
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    L.orc_kernel_W.restype = dbl
    L.orc_kernel_W.argtypes = [dbl, dbl]
    L.orc_kernel_dW.restype = dbl
    L.orc_kernel_dW.argtypes = [dbl, dbl]
    L.orc_block_key.argtypes = [vp, vp, vp]
    L.orc_bin.argtypes = [vp, i32, vp, vp, vp, vp]
    L.orc_neighbors_brute.restype = i64
    L.orc_neighbors_brute.argtypes = [i32, vp, i32, vp, dbl, vp, vp]
    L.orc_neighbors_grid.restype = i64
    L.orc_neighbors_grid.argtypes = [vp, i32, vp, i32, vp, i32, vp, vp]
    L.orc_wcsph_density.argtypes = [vp, i32, vp, i32, vp, vp, vp, vp, vp]
    L.orc_wcsph_accel.argtypes = [vp, i32, vp, vp, vp, vp, i32, vp, vp, vp]
    L.orc_level_thresholds.restype = None
    L.orc_level_thresholds.argtypes = [vp, vp, vp, vp]
    L.orc_classify_wcsph.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.orc_wcsph_evaluate.argtypes = [vp, vp]
    L.orc_wcsph_substep.argtypes = [vp, vp]
    L.orc_wcsph_global_step.argtypes = [vp, vp, i32, vp]
    L.orc_pcisph_delta.restype = dbl
    L.orc_pcisph_delta.argtypes = [vp]
    L.orc_classify_pcisph.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.orc_observed_blocks.restype = None
    L.orc_observed_blocks.argtypes = [vp, vp, vp, vp]
    L.orc_pcisph_step.argtypes = [vp, vp]
    L.orc_pcisph_plain_step.argtypes = [vp, vp]
    L.orc_pcisph_global_step.argtypes = [vp, vp, i32, vp]
    L.orc_num_threads.restype = C.c_int
    L.orc_num_threads.argtypes = []
    L.orc_tait.restype = dbl
    L.orc_tait.argtypes = [vp, dbl]
    L.orc_pcisph_pressure_accel.argtypes = [vp, i32, vp, vp, vp, i32, vp, vp]
    L.orc_pcisph_nonpressure_accel.argtypes = [vp, i32, vp, vp, i32, vp, vp]


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != 0:
        raise OracleError(f"{what} returned status {st}")


def d3(a):
    return np.ascontiguousarray(np.asarray(a, np.float64).reshape(-1, 3))


def n_blocks(P: OrcParams) -> int:
    return P.dim[0] * P.dim[1] * P.dim[2]


# ------------------------------------------------------------------ functions ---

def kernel_W(d, h):
    return lib().orc_kernel_W(float(d), float(h))


def kernel_dW(d, h):
    return lib().orc_kernel_dW(float(d), float(h))


def bin_particles(P, x):
    x = d3(x)
    n = x.shape[0]
    key = np.zeros(n, np.int32)
    perm = np.zeros(n, np.int32)
    cstart = np.zeros(n_blocks(P) + 1, np.int32)
    _check(lib().orc_bin(C.byref(P), n, _p(x), _p(key), _p(perm), _p(cstart)), "orc_bin")
    return key, perm, cstart


def neighbors_brute(x, xb, r):
    x, xb = d3(x), d3(xb)
    n = x.shape[0]
    off = np.zeros(n + 1, np.int32)
    tot = lib().orc_neighbors_brute(n, _p(x), xb.shape[0], _p(xb), float(r), _p(off), None)
    idx = np.zeros(max(tot, 1), np.int32)
    lib().orc_neighbors_brute(n, _p(x), xb.shape[0], _p(xb), float(r), _p(off), _p(idx))
    return off, idx[:tot]


def neighbors_grid(P, x, xb, rings=1):
    x, xb = d3(x), d3(xb)
    n = x.shape[0]
    off = np.zeros(n + 1, np.int32)
    tot = lib().orc_neighbors_grid(C.byref(P), n, _p(x), xb.shape[0], _p(xb), rings, _p(off), None)
    if tot < 0:
        raise OracleError(f"orc_neighbors_grid status {-tot}")
    idx = np.zeros(max(tot, 1), np.int32)
    lib().orc_neighbors_grid(C.byref(P), n, _p(x), xb.shape[0], _p(xb), rings, _p(off), _p(idx))
    return off, idx[:tot]


def density(P, x, xb, mask=None):
    x, xb = d3(x), d3(xb)
    n = x.shape[0]
    rho = np.zeros(n)
    prs = np.zeros(n)
    nbr = np.zeros(n, np.int32)
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    _check(lib().orc_wcsph_density(C.byref(P), n, _p(x), xb.shape[0], _p(xb), _p(m), _p(rho),
                                   _p(prs), _p(nbr)), "orc_wcsph_density")
    return rho, prs, nbr


def accel(P, x, v, rho, prs, xb, mask=None):
    x, v, xb = d3(x), d3(v), d3(xb)
    n = x.shape[0]
    rho = np.ascontiguousarray(rho, np.float64)
    prs = np.ascontiguousarray(prs, np.float64)
    a = np.zeros((n, 3))
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    _check(lib().orc_wcsph_accel(C.byref(P), n, _p(x), _p(v), _p(rho), _p(prs), xb.shape[0],
                                 _p(xb), _p(m), _p(a)), "orc_wcsph_accel")
    return a


def num_threads():
    """OpenMP threads of the oracle's parallel loops (omp_get_max_threads)."""
    return int(lib().orc_num_threads())


def tait(P, rho):
    return lib().orc_tait(C.byref(P), float(rho))


def level_thresholds(P):
    v = np.zeros(8)
    a = np.zeros(8)
    e = np.zeros(8, np.int32)
    lib().orc_level_thresholds(C.byref(P), _p(v), _p(a), _p(e))
    nl = P.n_levels
    return v[:nl], a[:nl], e[:nl]


def classify_wcsph(P, x, v, a):
    x, v, a = d3(x), d3(v), d3(a)
    B = n_blocks(P)
    raw = np.zeros(B, np.int32)
    lev = np.zeros(B, np.int32)
    _check(lib().orc_classify_wcsph(C.byref(P), x.shape[0], _p(x), _p(v), _p(a), _p(raw),
                                    _p(lev)), "orc_classify_wcsph")
    return raw, lev


class WCSPH:
    """WCSPH state (user order, FP64) advanced by the oracle."""

    def __init__(self, P, x, v, xb, a=None, rho=None, p=None, klast=None, validity=None,
                 level=None, k=0, primed=False):
        self.P = P
        n = len(x)
        self.x = d3(x).copy()
        self.v = d3(v).copy()
        self.a = d3(a).copy() if a is not None else np.zeros((n, 3))
        self.rho = (np.asarray(rho, np.float64).copy() if rho is not None
                    else np.full(n, P.rho0))
        self.p = np.asarray(p, np.float64).copy() if p is not None else np.zeros(n)
        self.klast = (np.asarray(klast, np.int32).copy() if klast is not None
                      else np.zeros(n, np.int32))
        self.validity = (np.asarray(validity, np.int32).copy() if validity is not None
                         else np.zeros(n, np.int32))
        self.level = (np.asarray(level, np.int32).copy() if level is not None
                      else np.full(n, -1, np.int32))
        self.compute = np.zeros(n, np.uint8)
        self.nbr = np.zeros(n, np.int32)
        self.xb = d3(xb).copy()
        self.block_level = np.full(n_blocks(P), -1, np.int32)
        self.S = WState()
        self.S.n = n
        self.S.nb = self.xb.shape[0]
        for f in ("x", "v", "a", "rho", "p", "klast", "validity", "level", "compute", "nbr",
                  "xb", "block_level"):
            setattr(self.S, f, getattr(self, f).ctypes.data)
        self.S.k = int(k)
        self.S.primed = 1 if primed else 0

    @property
    def k(self):
        return self.S.k

    @property
    def primed(self):
        return bool(self.S.primed)

    def evaluate(self):
        _check(lib().orc_wcsph_evaluate(C.byref(self.P), C.byref(self.S)), "orc_wcsph_evaluate")

    def substep(self):
        _check(lib().orc_wcsph_substep(C.byref(self.P), C.byref(self.S)), "orc_wcsph_substep")

    def global_step(self, max_mult=1 << 30):
        used = C.c_int32(0)
        _check(lib().orc_wcsph_global_step(C.byref(self.P), C.byref(self.S), int(max_mult),
                                           C.byref(used)), "orc_wcsph_global_step")
        return used.value


# ------------------------------------------------------------------ PCISPH ---

class PState(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("nb", C.c_int32),
        ("x", C.c_void_p), ("v", C.c_void_p), ("anp", C.c_void_p), ("ap", C.c_void_p),
        ("p", C.c_void_p), ("rho", C.c_void_p), ("err", C.c_void_p),
        ("level", C.c_void_p), ("validity", C.c_void_p), ("compute", C.c_void_p),
        ("nbr_cnt", C.c_void_p), ("nbr_idx", C.c_void_p), ("cap", C.c_int32),
        ("xb", C.c_void_p), ("pblock", C.c_void_p), ("cs", C.c_void_p), ("pm", C.c_void_p),
        ("bcs", C.c_void_p), ("bpm", C.c_void_p), ("block_level", C.c_void_p),
        ("block_raw", C.c_void_p), ("block_ob", C.c_void_p), ("p_backup", C.c_void_p),
        ("in_se", C.c_void_p), ("minor", C.c_int32), ("n_minor_cur", C.c_int32),
        ("clean", C.c_int32), ("shorten_now", C.c_int32), ("k", C.c_int64),
        ("iters", C.c_int32), ("global_iters", C.c_int32), ("local_iters", C.c_int32),
        ("reverts", C.c_int32), ("not_converged", C.c_int32),
        ("err_max", C.c_double), ("err_avg", C.c_double),
        ("total_iters", C.c_int64), ("total_local", C.c_int64), ("total_restarts", C.c_int64),
    ]


def pcisph_pressure_accel(P, x, prs, rho, xb):
    x, xb = d3(x), d3(xb)
    n = x.shape[0]
    prs = np.ascontiguousarray(prs, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    a = np.zeros((n, 3))
    _check(lib().orc_pcisph_pressure_accel(C.byref(P), n, _p(x), _p(prs), _p(rho), xb.shape[0],
                                           _p(xb), _p(a)), "orc_pcisph_pressure_accel")
    return a


def pcisph_nonpressure_accel(P, x, v, xb):
    x, v, xb = d3(x), d3(v), d3(xb)
    n = x.shape[0]
    a = np.zeros((n, 3))
    _check(lib().orc_pcisph_nonpressure_accel(C.byref(P), n, _p(x), _p(v), xb.shape[0], _p(xb),
                                              _p(a)), "orc_pcisph_nonpressure_accel")
    return a


def pcisph_delta(P):
    return lib().orc_pcisph_delta(C.byref(P))


def classify_pcisph(P, x, v, a):
    x, v, a = d3(x), d3(v), d3(a)
    B = n_blocks(P)
    raw = np.zeros(B, np.int32)
    lev = np.zeros(B, np.int32)
    _check(lib().orc_classify_pcisph(C.byref(P), x.shape[0], _p(x), _p(v), _p(a), _p(raw),
                                     _p(lev)), "orc_classify_pcisph")
    return raw, lev


def observed_blocks(P, block_level, in_re=None):
    lev = np.ascontiguousarray(block_level, np.int32)
    re_ = None if in_re is None else np.ascontiguousarray(in_re, np.uint8)
    ob = np.zeros(len(lev), np.uint8)
    lib().orc_observed_blocks(C.byref(P), _p(lev), _p(re_), _p(ob))
    return ob


class PCISPH:
    """RTS-PCISPH state (user order, FP64) advanced by the oracle."""

    def __init__(self, P, x, v, xb, cap=None):
        self.P = P
        n = len(x)
        B = n_blocks(P)
        self.cap = int(cap or P.max_neighbors)
        self.x = d3(x).copy()
        self.v = d3(v).copy()
        self.anp = np.zeros((n, 3))
        self.ap = np.zeros((n, 3))
        self.p = np.zeros(n)
        self.rho = np.full(n, P.rho0)
        self.err = np.zeros(n)
        self.level = np.zeros(n, np.int32)
        self.validity = np.zeros(n, np.int32)
        self.compute = np.ones(n, np.uint8)
        self.nbr_cnt = np.zeros(n, np.int32)
        self.nbr_idx = np.zeros(max(n, 1) * self.cap, np.int32)
        self.xb = d3(xb).copy()
        self.pblock = np.zeros(max(n, 1), np.int32)
        self.cs = np.zeros(B + 1, np.int32)
        self.pm = np.zeros(max(n, 1), np.int32)
        _, self.bpm, self.bcs = bin_particles(P, self.xb) if len(self.xb) else (
            None, np.zeros(1, np.int32), np.zeros(B + 1, np.int32))
        self.bpm = np.ascontiguousarray(self.bpm, np.int32)
        self.bcs = np.ascontiguousarray(self.bcs, np.int32)
        self.block_level = np.full(B, -1, np.int32)
        self.block_raw = np.full(B, -1, np.int32)
        self.block_ob = np.zeros(B, np.uint8)
        self.p_backup = np.zeros(max(n, 1))
        self.in_se = np.zeros(max(n, 1), np.uint8)
        self.S = PState()
        self.S.n = n
        self.S.nb = self.xb.shape[0]
        self.S.cap = self.cap
        for f in ("x", "v", "anp", "ap", "p", "rho", "err", "level", "validity", "compute",
                  "nbr_cnt", "nbr_idx", "xb", "pblock", "cs", "pm", "bcs", "bpm",
                  "block_level", "block_raw", "block_ob", "p_backup", "in_se"):
            setattr(self.S, f, getattr(self, f).ctypes.data)
        self.S.n_minor_cur = P.n_minor

    def step(self, allow_not_converged=True):
        st = lib().orc_pcisph_step(C.byref(self.P), C.byref(self.S))
        if st == 6 and allow_not_converged:
            return st
        _check(st, "orc_pcisph_step")
        return st

    def plain_step(self, allow_not_converged=True):
        st = lib().orc_pcisph_plain_step(C.byref(self.P), C.byref(self.S))
        if st == 6 and allow_not_converged:
            return st
        _check(st, "orc_pcisph_plain_step")
        return st

    def global_step(self, max_mult=1 << 30, allow_not_converged=True):
        used = C.c_int32(0)
        st = lib().orc_pcisph_global_step(C.byref(self.P), C.byref(self.S), int(max_mult),
                                          C.byref(used))
        if not (st == 6 and allow_not_converged):
            _check(st, "orc_pcisph_global_step")
        return used.value

    def neighbors(self, i):
        return self.nbr_idx[i * self.cap: i * self.cap + self.nbr_cnt[i]]

    @property
    def stats(self):
        S = self.S
        return dict(iters=S.iters, global_iters=S.global_iters, local_iters=S.local_iters,
                    reverts=S.reverts, not_converged=S.not_converged, err_max=S.err_max,
                    err_avg=S.err_avg, minor=S.minor, n_minor_cur=S.n_minor_cur, k=S.k)
