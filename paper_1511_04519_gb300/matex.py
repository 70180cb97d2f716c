"""Thin ctypes binding of the C ABI in ``include/matex.h``.

Argument marshalling only: every step of the integrator runs in the CUDA
library.  Device buffers and the stream come from PyTorch.  Importing this
module loads ``_lib/libmatex.so`` and raises if it is missing; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmatex.so")

MATEX_OK = 0
MATEX_ERR_NOCONV = 5
STATUS = {0: "MATEX_OK", 1: "MATEX_ERR_ARG", 2: "MATEX_ERR_NOT_SPD", 3: "MATEX_ERR_CUDA",
          4: "MATEX_ERR_TIMEOUT", 5: "MATEX_ERR_NOCONV", 6: "MATEX_ERR_OOM", 7: "MATEX_ERR_STATE"}


class MatexError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class MatexOpts(C.Structure):
    _fields_ = [("col_block", C.c_int32), ("group_select", C.c_int32), ("include_dc", C.c_int32),
                ("n_rows", C.c_int32), ("rows", C.POINTER(C.c_int32)),
                ("replay_m", C.POINTER(C.c_int32)), ("n_replay", C.c_int64),
                ("max_width", C.c_int32), ("strict", C.c_int32), ("solve_mode", C.c_int32),
                ("tape", C.c_int32), ("krylov", C.c_int32), ("graph", C.c_int32),
                ("tail_eps", C.c_double), ("tape_window", C.c_int32), ("tape_block", C.c_int32),
                ("recombine", C.c_int32), ("decompose", C.c_int32), ("resident", C.c_int32),
                ("tc_solve", C.c_int32), ("tc_min_width", C.c_int32),
                ("single_column", C.c_int32)]


class MatexStats(C.Structure):
    _fields_ = [("setup_order_ms", C.c_double), ("setup_factor_ms", C.c_double),
                ("setup_upload_ms", C.c_double), ("run_ms", C.c_double), ("nnz_L", C.c_int64),
                ("n_supernodes", C.c_int32), ("n_levels", C.c_int32), ("n_segments", C.c_int32),
                ("krylov_segments", C.c_int32), ("sum_m", C.c_int32), ("max_m", C.c_int32),
                ("nonconv", C.c_int32), ("breakdowns", C.c_int32), ("sweeps_M", C.c_int32),
                ("sweeps_G", C.c_int32), ("solve_columns", C.c_int64),
                ("kernel_launches", C.c_int32), ("rounds", C.c_int32),
                ("graph_replay", C.c_int32), ("graph_capture_ms", C.c_double),
                ("nnz_L_exact", C.c_int64), ("tape_window", C.c_int32), ("tape_block", C.c_int32),
                ("tape_bytes", C.c_int64), ("tc_rounds", C.c_int32), ("resident", C.c_int32),
                ("tc_solve_supernodes", C.c_int32), ("tc_solve_min_cols", C.c_int32),
                ("single_column", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MatexProfile(C.Structure):
    _fields_ = [("ms", C.c_double * 6), ("units", C.c_int64 * 6), ("launches", C.c_int64 * 6),
                ("flops", C.c_double * 6), ("bytes", C.c_double * 6)]

    CLASSES = ["solve", "move", "gram_schmidt", "small_dense", "recombine", "other"]

    def as_dict(self):
        return {name: dict(ms=self.ms[i], units=self.units[i], launches=self.launches[i],
                           flops=self.flops[i], bytes=self.bytes[i])
                for i, name in enumerate(self.CLASSES)}


EXPORTS = ["matex_default_opts", "matex_setup", "matex_run", "matex_run_host", "matex_set_sources",
           "matex_solve", "matex_expm", "matex_get_m", "matex_get_sizes", "matex_get_setup_stats",
           "matex_last_error", "matex_status_string", "matex_destroy", "matex_set_profiling",
           "matex_get_profile", "matex_host_factor_solve", "matex_host_single_column_plan",
           "matex_set_batching",
           "matex_debug_inject_wait", "matex_solve_noalloc", "matex_grad", "matex_set_caps",
           "matex_get_autotune", "matex_batch_create", "matex_batch_run", "matex_batch_last_error",
           "matex_batch_destroy", "matex_measure_fp64_peak", "matex_tr_run",
           "matex_time_solve", "matex_get_level_blocks", "matex_solve_resident"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmatex.so is not built ({LIB_PATH}); run "
                          "paper_1511_04519_gb300.build.build() first")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    i32p, i64p, dp = C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_double)
    lib.matex_default_opts.argtypes = [C.POINTER(MatexOpts)]
    lib.matex_default_opts.restype = None
    lib.matex_setup.argtypes = [C.POINTER(P), C.c_int64, dp, i64p, i32p, dp, dp, C.c_int32, i32p,
                                i32p, dp, dp, i32p, C.c_int32, C.c_double, C.c_double, C.c_int32,
                                C.c_double, C.c_double, C.POINTER(MatexOpts), P]
    lib.matex_setup.restype = C.c_int
    lib.matex_run.argtypes = [P, P, C.POINTER(MatexStats)]
    lib.matex_run.restype = C.c_int
    lib.matex_run_host.argtypes = [P, dp, dp, C.POINTER(MatexStats)]
    lib.matex_run_host.restype = C.c_int
    lib.matex_set_sources.argtypes = [P, dp]
    lib.matex_set_sources.restype = C.c_int
    lib.matex_solve.argtypes = [P, C.c_int32, C.c_int32, P, P]
    lib.matex_solve.restype = C.c_int
    lib.matex_solve_noalloc.argtypes = [P, C.c_int32, C.c_int32, P, P]
    lib.matex_solve_noalloc.restype = C.c_int
    lib.matex_solve_resident.argtypes = [P, C.c_int32, C.c_int32, P, P]
    lib.matex_solve_resident.restype = C.c_int
    lib.matex_get_level_blocks.argtypes = [P, i32p, i32p, C.POINTER(C.c_float), C.c_int32, i32p]
    lib.matex_get_level_blocks.restype = C.c_int
    lib.matex_time_solve.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_float),
                                     C.POINTER(C.c_float)]
    lib.matex_time_solve.restype = C.c_int
    lib.matex_expm.argtypes = [P, C.c_int32, C.c_int32, P, P, P]
    lib.matex_expm.restype = C.c_int
    lib.matex_get_m.argtypes = [P, i32p, C.c_int64, i64p]
    lib.matex_get_m.restype = C.c_int
    lib.matex_get_sizes.argtypes = [P, i32p, i32p, i64p]
    lib.matex_get_sizes.restype = C.c_int
    lib.matex_get_setup_stats.argtypes = [P, C.POINTER(MatexStats)]
    lib.matex_get_setup_stats.restype = C.c_int
    lib.matex_last_error.argtypes = [P]
    lib.matex_last_error.restype = C.c_char_p
    lib.matex_status_string.argtypes = [C.c_int]
    lib.matex_status_string.restype = C.c_char_p
    lib.matex_get_autotune.argtypes = [P, i32p, i32p, C.POINTER(C.c_float), C.c_int32, i32p]
    lib.matex_get_autotune.restype = C.c_int
    lib.matex_set_caps.argtypes = [P, dp]
    lib.matex_set_caps.restype = C.c_int
    lib.matex_grad.argtypes = [P, P, P, P]
    lib.matex_grad.restype = C.c_int
    lib.matex_debug_inject_wait.argtypes = [P, C.c_int32]
    lib.matex_debug_inject_wait.restype = C.c_int
    lib.matex_set_batching.argtypes = [P, C.c_int32]
    lib.matex_set_batching.restype = C.c_int
    lib.matex_set_profiling.argtypes = [P, C.c_int32]
    lib.matex_set_profiling.restype = C.c_int
    lib.matex_get_profile.argtypes = [P, C.POINTER(MatexProfile)]
    lib.matex_get_profile.restype = C.c_int
    lib.matex_destroy.argtypes = [P]
    lib.matex_destroy.restype = None
    lib.matex_batch_create.argtypes = [C.POINTER(P), C.POINTER(P), C.c_int32]
    lib.matex_batch_create.restype = C.c_int
    lib.matex_batch_run.argtypes = [P, C.POINTER(P), C.POINTER(MatexStats), C.POINTER(C.c_float)]
    lib.matex_batch_run.restype = C.c_int
    lib.matex_batch_last_error.argtypes = [P]
    lib.matex_batch_last_error.restype = C.c_char_p
    lib.matex_batch_destroy.argtypes = [P]
    lib.matex_batch_destroy.restype = None
    lib.matex_tr_run.argtypes = [P, C.c_int32, P, dp]
    lib.matex_tr_run.restype = C.c_int
    lib.matex_measure_fp64_peak.argtypes = [C.c_int32, dp, dp]
    lib.matex_measure_fp64_peak.restype = C.c_int
    return lib


_lib = _load()


def lib():
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def _check(ctx, status, allow=(MATEX_OK,)):
    if status not in allow:
        msg = _lib.matex_last_error(ctx)
        raise MatexError(status, msg.decode() if msg else "")
    return status


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def matex_default_opts():
    o = MatexOpts()
    _lib.matex_default_opts(C.byref(o))
    return o


def matex_setup(n, c, g_rowptr, g_col, g_val, dc_inject, src_node, pwl_off, pwl_t, pwl_v,
                src_group, n_groups, gamma, tol, m_max, t_end, dt_out, opts=None, stream=None):
    """matex_setup of the C ABI; arrays are host numpy arrays (copied)."""
    keep = []

    def arr(x, dt):
        a = np.ascontiguousarray(np.asarray(x, dtype=dt))
        keep.append(a)
        return a

    c_ = arr(c, np.float64)
    rp = arr(g_rowptr, np.int64)
    gc = arr(g_col, np.int32)
    gv = arr(g_val, np.float64)
    dc = arr(dc_inject, np.float64) if dc_inject is not None else None
    sn = arr(src_node, np.int32)
    po = arr(pwl_off, np.int32)
    pt = arr(pwl_t, np.float64)
    pv = arr(pwl_v, np.float64)
    sg = arr(src_group, np.int32)
    o = opts if opts is not None else matex_default_opts()
    ctx = C.c_void_p()
    st = _lib.matex_setup(C.byref(ctx), int(n), _ptr(c_, C.c_double), _ptr(rp, C.c_int64),
                          _ptr(gc, C.c_int32), _ptr(gv, C.c_double),
                          _ptr(dc, C.c_double) if dc is not None else None, int(sn.shape[0]),
                          _ptr(sn, C.c_int32), _ptr(po, C.c_int32), _ptr(pt, C.c_double),
                          _ptr(pv, C.c_double), _ptr(sg, C.c_int32), int(n_groups), float(gamma),
                          float(tol), int(m_max), float(t_end), float(dt_out), C.byref(o),
                          _stream_handle(stream))
    if st != MATEX_OK:
        msg = _lib.matex_last_error(None)
        raise MatexError(st, msg.decode() if msg else "")
    return ctx


def matex_run(ctx, x_out_ptr, strict_ok=True):
    s = MatexStats()
    st = _lib.matex_run(ctx, C.c_void_p(x_out_ptr), C.byref(s))
    _check(ctx, st, allow=(MATEX_OK, MATEX_ERR_NOCONV) if strict_ok else (MATEX_OK,))
    return s


def matex_run_host(ctx, pwl_v_host, x_out_host):
    s = MatexStats()
    st = _lib.matex_run_host(ctx, _ptr(pwl_v_host, C.c_double) if pwl_v_host is not None else None,
                             _ptr(x_out_host, C.c_double), C.byref(s))
    _check(ctx, st, allow=(MATEX_OK, MATEX_ERR_NOCONV))
    return s


def matex_set_sources(ctx, pwl_v_host):
    a = np.ascontiguousarray(pwl_v_host, dtype=np.float64)
    _check(ctx, _lib.matex_set_sources(ctx, _ptr(a, C.c_double)))


def matex_solve(ctx, which, ncols, b_ptr, x_ptr):
    _check(ctx, _lib.matex_solve(ctx, int(which), int(ncols), C.c_void_p(b_ptr), C.c_void_p(x_ptr)))


def matex_solve_resident(ctx, which, ncols, b_ptr, x_ptr):
    """matex_solve through the one-CTA substitution of the resident rounds."""
    _check(ctx, _lib.matex_solve_resident(ctx, int(which), int(ncols), C.c_void_p(b_ptr),
                                          C.c_void_p(x_ptr)))


def matex_solve_noalloc(ctx, which, ncols, b_ptr, x_ptr):
    """matex_solve without any allocation (static device scratch; see matex.h)."""
    _check(ctx, _lib.matex_solve_noalloc(ctx, int(which), int(ncols), C.c_void_p(b_ptr),
                                         C.c_void_p(x_ptr)))


def matex_expm(ctx, batch, m, a_ptr, h_ptr, e_ptr):
    _check(ctx, _lib.matex_expm(ctx, int(batch), int(m), C.c_void_p(a_ptr), C.c_void_p(h_ptr),
                                C.c_void_p(e_ptr)))


def matex_get_m(ctx):
    cnt = C.c_int64()
    _check(ctx, _lib.matex_get_m(ctx, None, 0, C.byref(cnt)))
    out = np.zeros(max(cnt.value, 1), np.int32)
    _check(ctx, _lib.matex_get_m(ctx, _ptr(out, C.c_int32), cnt.value, C.byref(cnt)))
    return out[: cnt.value]


def matex_get_sizes(ctx):
    nt, nr, ns = C.c_int32(), C.c_int32(), C.c_int64()
    _check(ctx, _lib.matex_get_sizes(ctx, C.byref(nt), C.byref(nr), C.byref(ns)))
    return nt.value, nr.value, ns.value


def matex_get_setup_stats(ctx):
    s = MatexStats()
    _check(ctx, _lib.matex_get_setup_stats(ctx, C.byref(s)))
    return s


def matex_get_autotune(ctx):
    cnt = C.c_int32()
    _check(ctx, _lib.matex_get_autotune(ctx, None, None, None, 0, C.byref(cnt)))
    k = cnt.value
    nc = np.zeros(max(k, 1), np.int32)
    md = np.zeros(max(k, 1), np.int32)
    ms = np.zeros(max(2 * k, 2), np.float32)
    _check(ctx, _lib.matex_get_autotune(ctx, _ptr(nc, C.c_int32), _ptr(md, C.c_int32),
                                        ms.ctypes.data_as(C.POINTER(C.c_float)), k, C.byref(cnt)))
    return [dict(ncols=int(nc[i]), mode=int(md[i]), persistent_ms=float(ms[2 * i]),
                 level_ms=float(ms[2 * i + 1])) for i in range(k)]


def matex_set_caps(ctx, c_host):
    a = np.ascontiguousarray(c_host, dtype=np.float64)
    _check(ctx, _lib.matex_set_caps(ctx, _ptr(a, C.c_double)))


def matex_grad(ctx, xbar_ptr, dc_ptr, damp_ptr):
    _check(ctx, _lib.matex_grad(ctx, C.c_void_p(xbar_ptr), C.c_void_p(dc_ptr), C.c_void_p(damp_ptr)))


def matex_debug_inject_wait(ctx, on):
    _check(ctx, _lib.matex_debug_inject_wait(ctx, int(bool(on))))


def matex_set_batching(ctx, one_group_at_a_time):
    _check(ctx, _lib.matex_set_batching(ctx, int(bool(one_group_at_a_time))))


def matex_set_profiling(ctx, on):
    _check(ctx, _lib.matex_set_profiling(ctx, int(bool(on))))


def matex_get_profile(ctx):
    p = MatexProfile()
    _check(ctx, _lib.matex_get_profile(ctx, C.byref(p)))
    return p


def matex_destroy(ctx):
    if ctx:
        _lib.matex_destroy(ctx)


class Sim:
    """Owner of one context built from a problem-like object (attributes n, c,
    g_rowptr, g_col, g_val, dc_inject, src_node, pwl_off, pwl_t, pwl_v,
    src_group, n_groups, gamma, tol, m_max, t_end, dt_out)."""

    def __init__(self, p, col_block=0, group_select=-1, include_dc=True, rows=None,
                 replay_m=None, max_width=0, strict=False, stream=None, solve_mode=2,
                 tape=False, graph=True, krylov="R", tail_eps=0.0, tape_window=0, tape_block=0,
                 recombine="auto", decompose="groups", resident="auto", tc_solve="auto",
                 tc_min_width=0, single_column="auto", **overrides):
        o = matex_default_opts()
        o.graph = int(bool(graph))
        o.tail_eps = float(tail_eps)
        o.krylov = {"R": 0, "I": 1, "S": 2}[krylov]
        o.col_block = col_block
        o.group_select = group_select
        o.include_dc = int(bool(include_dc))
        if max_width:
            o.max_width = max_width
        o.strict = int(bool(strict))
        o.solve_mode = int(solve_mode)
        o.tape = {False: 0, True: 1, 0: 0, 1: 1, 2: 2, "full": 1, "checkpoint": 2}[tape]
        o.recombine = {"auto": 0, "tensor": 0, "fp64": 1}[recombine]
        o.decompose = {"groups": 0, "ramps": 1}[decompose]
        o.resident = {"auto": 0, "off": 1, "on": 2, "on_inline_inputs": 3, 0: 0, 1: 1, 2: 2,
                      3: 3}[resident]
        o.tc_solve = {"auto": 0, "off": 1, "on": 2, 0: 0, 1: 1, 2: 2}[tc_solve]
        o.tc_min_width = int(tc_min_width)
        o.single_column = {"auto": 0, "off": 1, "on": 2, 0: 0, 1: 1, 2: 2}[single_column]
        o.tape_window = int(tape_window)
        o.tape_block = int(tape_block)
        self._keep = []
        if rows is not None:
            r = np.ascontiguousarray(rows, dtype=np.int32)
            self._keep.append(r)
            o.n_rows = int(r.shape[0])
            o.rows = _ptr(r, C.c_int32)
        if replay_m is not None:
            rm = np.ascontiguousarray(replay_m, dtype=np.int32)
            self._keep.append(rm)
            o.replay_m = _ptr(rm, C.c_int32)
            o.n_replay = int(rm.shape[0])
        g = dict(gamma=p.gamma, tol=p.tol, m_max=p.m_max, t_end=p.t_end, dt_out=p.dt_out)
        g.update(overrides)
        self.ctx = matex_setup(p.n, p.c, p.g_rowptr, p.g_col, p.g_val, p.dc_inject, p.src_node,
                               p.pwl_off, p.pwl_t, p.pwl_v, p.src_group, p.n_groups, g["gamma"],
                               g["tol"], g["m_max"], g["t_end"], g["dt_out"], opts=o, stream=stream)
        self.n = int(p.n)
        self.n_times, self.n_rows, self.n_segments = matex_get_sizes(self.ctx)
        self.pwl_len = int(np.asarray(p.pwl_v).shape[0])
        self.n_src = int(np.asarray(p.src_node).shape[0])

    def run(self, out=None):
        import torch
        if out is None:
            out = torch.empty((self.n_times, self.n_rows), dtype=torch.float64, device="cuda")
        self.stats = matex_run(self.ctx, out.data_ptr())
        return out

    def run_host(self, pwl_v=None, out=None):
        if out is None:
            out = np.empty((self.n_times, self.n_rows), np.float64)
        pv = None if pwl_v is None else np.ascontiguousarray(pwl_v, dtype=np.float64)
        self.stats = matex_run_host(self.ctx, pv, out)
        return out

    def tr_run(self, substeps=1, out=None):
        """Fixed-step trapezoidal integration with h = dt_out / substeps on the
        same solves (matex_tr_run); returns (voltages, device ms)."""
        import torch
        if out is None:
            out = torch.empty((self.n_times, self.n_rows), dtype=torch.float64, device="cuda")
        ms = C.c_double()
        _check(self.ctx, _lib.matex_tr_run(self.ctx, int(substeps), C.c_void_p(out.data_ptr()),
                                           C.byref(ms)))
        return out, ms.value

    def set_caps(self, c):
        matex_set_caps(self.ctx, c)

    def set_sources(self, pwl_v):
        matex_set_sources(self.ctx, pwl_v)

    def grad(self, xbar):
        """(dL/dc, dL/d amp_scale) for dL/dX_out = xbar ([N+1][n_rows] cuda float64)."""
        import torch
        xbar = xbar.contiguous()
        dc = torch.empty(self.n, dtype=torch.float64, device="cuda")
        da = torch.empty(self.n_src, dtype=torch.float64, device="cuda")
        matex_grad(self.ctx, xbar.data_ptr(), dc.data_ptr(), da.data_ptr())
        return dc, da

    def m_sequence(self):
        return matex_get_m(self.ctx)

    def solve(self, which, b):
        import torch
        b = b.contiguous()
        x = torch.empty_like(b)
        ncols = 1 if b.dim() == 1 else b.shape[0]
        matex_solve(self.ctx, which, ncols, b.data_ptr(), x.data_ptr())
        torch.cuda.synchronize()
        return x

    def time_solve(self, which, ncols, reps=10):
        """(best ms, mean ms) of the bare batched solve pair with ncols
        right-hand sides (matex_time_solve)."""
        best, mean = C.c_float(), C.c_float()
        _check(self.ctx, _lib.matex_time_solve(self.ctx, int(which), int(ncols), int(reps),
                                               C.byref(best), C.byref(mean)))
        return best.value, mean.value

    def level_blocks(self):
        """Per tree level: the column blocks of the forward and backward level
        launches and their tuned times (matex_get_level_blocks)."""
        n = C.c_int32()
        _check(self.ctx, _lib.matex_get_level_blocks(self.ctx, None, None, None, 0, C.byref(n)))
        L = n.value
        f = np.zeros(L, np.int32)
        b = np.zeros(L, np.int32)
        ms = np.zeros(2 * L, np.float32)
        _check(self.ctx, _lib.matex_get_level_blocks(
            self.ctx, f.ctypes.data_as(C.POINTER(C.c_int32)), b.ctypes.data_as(C.POINTER(C.c_int32)),
            ms.ctypes.data_as(C.POINTER(C.c_float)), L, C.byref(n)))
        return [{"level": l, "kb_fwd": int(f[l]), "kb_bwd": int(b[l]),
                 "fwd_ms": float(ms[2 * l]), "bwd_ms": float(ms[2 * l + 1])} for l in range(L)]

    def one_group_at_a_time(self, on=True):
        matex_set_batching(self.ctx, on)

    def autotune(self):
        return matex_get_autotune(self.ctx)

    def profile(self, on=None):
        if on is not None:
            matex_set_profiling(self.ctx, on)
        return matex_get_profile(self.ctx).as_dict()

    def setup_stats(self):
        return matex_get_setup_stats(self.ctx).as_dict()

    def close(self):
        if getattr(self, "ctx", None):
            matex_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_fp64_peak(reps=5):
    """(TFLOP/s, ms) of the FP64 FMA probe on the current device."""
    tf, ms = C.c_double(), C.c_double()
    st = _lib.matex_measure_fp64_peak(int(reps), C.byref(tf), C.byref(ms))
    if st != MATEX_OK:
        raise MatexError(st, "FP64 probe failed")
    return tf.value, ms.value


class Batch:
    """Several Sims (independent grids) run as one CUDA graph launch
    (matex_batch_create / matex_batch_run).  The Sims must outlive the batch."""

    def __init__(self, sims):
        self.sims = list(sims)
        arr = (C.c_void_p * len(self.sims))(*[s.ctx.value for s in self.sims])
        b = C.c_void_p()
        st = _lib.matex_batch_create(C.byref(b), arr, len(self.sims))
        if st != MATEX_OK:
            msg = _lib.matex_last_error(None)
            raise MatexError(st, msg.decode() if msg else "")
        self.b = b

    def run(self, outs=None):
        """Returns (outputs, per-grid ms from the batch start to the end of each
        grid's branch); per-Sim statistics land in each Sim's ``stats``."""
        import torch
        if outs is None:
            outs = [torch.empty((s.n_times, s.n_rows), dtype=torch.float64, device="cuda")
                    for s in self.sims]
        k = len(self.sims)
        ptrs = (C.c_void_p * k)(*[o.data_ptr() for o in outs])
        stats = (MatexStats * k)()
        ms = (C.c_float * k)()
        st = _lib.matex_batch_run(self.b, ptrs, stats, ms)
        if st not in (MATEX_OK, MATEX_ERR_NOCONV):
            msg = _lib.matex_batch_last_error(self.b)
            raise MatexError(st, msg.decode() if msg else "")
        for s, x in zip(self.sims, stats):
            s.stats = x
        return outs, np.array(list(ms), dtype=np.float64)

    def close(self):
        if getattr(self, "b", None):
            _lib.matex_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def expm(sim, A, h):
    """Batched e^{h A} through matex_expm (A: [batch, m, m] cuda float64)."""
    import torch
    A = A.contiguous()
    h = h.contiguous()
    E = torch.empty_like(A)
    matex_expm(sim.ctx, A.shape[0], A.shape[1], A.data_ptr(), h.data_ptr(), E.data_ptr())
    return E
