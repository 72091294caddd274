"""ctypes binding of include/cfc_gb300.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "lib", "libcfc_gb300.so")

(LAP_OK, LAP_EINVAL, LAP_ENOTCONN, LAP_ENOMEM, LAP_ENOCONV, LAP_ECUDA, LAP_EBUDGET, LAP_ENOTIMPL,
 LAP_EPENDING) = range(9)
LAP_FP64, LAP_FP32_REFINED, LAP_FP32_BF16COARSE_REFINED = 0, 1, 2
LAP_SMOOTH_JACOBI, LAP_SMOOTH_CHEBYSHEV = 0, 1
LAP_AGG_STRENGTH, LAP_AGG_AFFINITY = 0, 1
KERNEL_FAMILIES = ["spmv_fine", "smooth_fine", "restrict_fine", "blas1", "coarse_levels", "resid64", "setup",
                   "cfc"]

SYMBOLS = [
    "lap_default_hier_opts", "lap_default_solve_opts", "lap_build_hierarchy", "lap_hierarchy_destroy",
    "lap_hierarchy_info", "lap_solve_multi", "cfc_jl_rhs", "cfc_farness_jl", "cfc_farness_jl_rows",
    "cfc_farness_from_solution",
    "cfc_farness_from_solution_noalloc", "cfc_sample_pivots",
    "cfc_farness_sampled", "cfc_exact_small", "lap_status_string", "lap_last_error", "lap_stats_reset",
    "lap_stats_set_timing", "lap_stats_read", "lap_stats_set_log", "lap_stats_read_log",
    "cfc_server_default_opts", "cfc_server_create", "cfc_server_add_graph", "cfc_server_submit",
    "cfc_server_poll", "cfc_server_stats", "cfc_server_reset_stats", "cfc_server_destroy",
    "lap_tune_save", "lap_tune_load", "lap_tune_entries",
]


class HierOpts(C.Structure):
    _fields_ = [("coarse_max", C.c_int32), ("max_levels", C.c_int32), ("agg_passes", C.c_int32),
                ("match_rounds", C.c_int32), ("eager", C.c_int32), ("eliminate", C.c_int32),
                ("reorder", C.c_int32), ("aggregation", C.c_int32), ("chunking", C.c_int32),
                ("hub_factor", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("tol", C.c_double), ("max_outer", C.c_int32),
                ("max_inner", C.c_int32), ("inner_tol", C.c_double), ("k_tile", C.c_int32),
                ("smoother", C.c_int32), ("nu_pre", C.c_int32), ("nu_post", C.c_int32),
                ("check_every", C.c_int32), ("levels_used", C.c_int32), ("nu_coarse", C.c_int32),
                ("cycle", C.c_int32), ("coarse_scale", C.c_double), ("w_levels", C.c_int32),
                ("graphs", C.c_int32), ("first_residual_ff", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("outer_iters", C.c_int32), ("inner_iters", C.c_int32), ("max_rel_residual", C.c_double),
                ("k_tile", C.c_int32), ("levels_used", C.c_int32), ("nu_coarse", C.c_int32), ("cycle", C.c_int32),
                ("coarse_scale", C.c_double), ("w_levels", C.c_int32), ("first_residual_ff", C.c_int32)]


class HierInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("levels", C.c_int32), ("coarse_n", C.c_int32),
                ("level_n", C.c_int64 * 32), ("level_nnz", C.c_int64 * 32), ("setup_ms", C.c_double),
                ("weight_exp", C.c_int32), ("level_row_order", C.c_int32 * 32), ("fingerprint", C.c_uint64),
                ("elim_levels", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("launches_total", C.c_uint64), ("launches", C.c_uint64 * 8), ("ms", C.c_double * 8),
                ("bytes", C.c_double * 8)]


class ServerOpts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("hbm_budget", C.c_int64), ("solve", SolveOpts),
                ("resident_pivots", C.c_int32), ("pivot_seed", C.c_uint64), ("batch_columns", C.c_int32)]


class RequestInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("graph_id", C.c_int32), ("q", C.c_int32), ("n_pivots", C.c_int32),
                ("device_bytes", C.c_int64), ("queue_ms", C.c_double), ("run_ms", C.c_double),
                ("latency_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("pending", C.c_int64),
                ("in_flight", C.c_int64), ("max_in_flight", C.c_int32), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("max_ms", C.c_double),
                ("queries_per_s", C.c_double), ("rhs_per_s", C.c_double), ("graph_bytes", C.c_int64),
                ("budget_bytes", C.c_int64), ("peak_in_flight_bytes", C.c_int64), ("max_batch", C.c_int32)]


class LapError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {lap_status_string(status)}" + (f" ({detail})" if detail else ""))


_lib = None


def lib():
    """Load libcfc_gb300.so.  Raises RuntimeError when it has not been built:
    there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(lib_path):
        raise RuntimeError(f"{lib_path} is missing: build it with "
                           "paper_1607_02955_gb300.build_ext.build() (needs nvcc)")
    L = C.CDLL(lib_path)
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    L.lap_default_hier_opts.argtypes = [C.POINTER(HierOpts)]
    L.lap_default_hier_opts.restype = None
    L.lap_default_solve_opts.argtypes = [C.POINTER(SolveOpts)]
    L.lap_default_solve_opts.restype = None
    L.lap_build_hierarchy.argtypes = [i64, i64, vp, vp, vp, C.POINTER(HierOpts), vp, C.POINTER(vp)]
    L.lap_build_hierarchy.restype = C.c_int
    L.lap_hierarchy_destroy.argtypes = [vp]
    L.lap_hierarchy_destroy.restype = None
    L.lap_hierarchy_info.argtypes = [vp, C.POINTER(HierInfo)]
    L.lap_hierarchy_info.restype = C.c_int
    L.lap_solve_multi.argtypes = [vp, i32, vp, vp, C.POINTER(SolveOpts), vp, C.POINTER(SolveInfo)]
    L.lap_solve_multi.restype = C.c_int
    L.cfc_jl_rhs.argtypes = [vp, i32, u64, vp, vp]
    L.cfc_jl_rhs.restype = C.c_int
    L.cfc_farness_jl.argtypes = [vp, i32, dbl, u64, i32, vp, vp, C.POINTER(SolveOpts), vp]
    L.cfc_farness_jl.restype = C.c_int
    L.cfc_farness_jl_rows.argtypes = [vp, i32, i32, i32, u64, i32, vp, vp, C.POINTER(SolveOpts), vp]
    L.cfc_farness_jl_rows.restype = C.c_int
    L.cfc_farness_from_solution.argtypes = [i64, i32, vp, i32, vp, vp, vp]
    L.cfc_farness_from_solution.restype = C.c_int
    L.cfc_farness_from_solution_noalloc.argtypes = [i64, i32, vp, i32, vp, vp, vp]
    L.cfc_farness_from_solution_noalloc.restype = C.c_int
    L.cfc_sample_pivots.argtypes = [vp, i32, u64, vp, vp]
    L.cfc_sample_pivots.restype = C.c_int
    L.cfc_farness_sampled.argtypes = [vp, i32, u64, i32, vp, vp, C.POINTER(SolveOpts), vp]
    L.cfc_farness_sampled.restype = C.c_int
    L.cfc_exact_small.argtypes = [i64, i64, vp, vp, vp, vp, vp, vp]
    L.cfc_exact_small.restype = C.c_int
    L.lap_status_string.argtypes = [C.c_int]
    L.lap_status_string.restype = C.c_char_p
    L.lap_last_error.argtypes = []
    L.lap_last_error.restype = C.c_char_p
    L.lap_stats_reset.argtypes = []
    L.lap_stats_reset.restype = None
    L.lap_stats_set_timing.argtypes = [i32]
    L.lap_stats_set_timing.restype = None
    L.lap_stats_read.argtypes = [C.POINTER(Stats)]
    L.lap_stats_read.restype = C.c_int
    L.cfc_server_default_opts.argtypes = [C.POINTER(ServerOpts)]
    L.cfc_server_default_opts.restype = None
    L.cfc_server_create.argtypes = [C.POINTER(ServerOpts), C.POINTER(vp)]
    L.cfc_server_create.restype = C.c_int
    L.cfc_server_add_graph.argtypes = [vp, i64, i64, vp, vp, vp, C.POINTER(i32)]
    L.cfc_server_add_graph.restype = C.c_int
    L.cfc_server_submit.argtypes = [vp, i32, i32, vp, i32, u64, C.POINTER(i64)]
    L.cfc_server_submit.restype = C.c_int
    L.cfc_server_poll.argtypes = [vp, i64, i32, vp, C.POINTER(RequestInfo)]
    L.cfc_server_poll.restype = C.c_int
    L.cfc_server_stats.argtypes = [vp, C.POINTER(ServerStats)]
    L.cfc_server_stats.restype = C.c_int
    L.cfc_server_reset_stats.argtypes = [vp]
    L.cfc_server_reset_stats.restype = None
    L.cfc_server_destroy.argtypes = [vp]
    L.cfc_server_destroy.restype = None
    L.lap_tune_save.argtypes = [C.c_char_p]
    L.lap_tune_save.restype = C.c_int
    L.lap_tune_load.argtypes = [C.c_char_p, C.POINTER(C.c_int64)]
    L.lap_tune_load.restype = C.c_int
    L.lap_tune_entries.argtypes = []
    L.lap_tune_entries.restype = C.c_int64
    L.lap_stats_set_log.argtypes = [i32]
    L.lap_stats_set_log.restype = None
    L.lap_stats_read_log.argtypes = [vp, i64, C.POINTER(C.c_int64)]
    L.lap_stats_read_log.restype = C.c_int
    _lib = L
    return L


def exported_symbols():
    L = lib()
    return [s for s in SYMBOLS if hasattr(L, s)]


# ------------------------------------------------------------------ marshalling
def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return C.c_void_p(0)


def _ptr(x, dtype):
    """Pointer of a torch tensor (any device) or numpy array of the given
    numpy dtype; None -> NULL.  Returns (pointer, keep-alive object)."""
    if x is None:
        return C.c_void_p(0), None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            want = {np.int32: torch.int32, np.float64: torch.float64}[dtype]
            if x.dtype != want or not x.is_contiguous():
                raise TypeError(f"expected a contiguous {want} tensor")
            return C.c_void_p(x.data_ptr()), x
    except ImportError:
        pass
    a = np.ascontiguousarray(x, dtype=dtype)
    return C.c_void_p(a.ctypes.data), a


def _check(st, where, allow=()):
    if st != LAP_OK and st not in allow:
        detail = lib().lap_last_error().decode(errors="replace")
        raise LapError(st, where, detail)
    return st


def lap_status_string(status: int) -> str:
    return lib().lap_status_string(int(status)).decode()


def lap_last_error() -> str:
    return lib().lap_last_error().decode(errors="replace")


def lap_default_hier_opts(**kw) -> HierOpts:
    o = HierOpts()
    lib().lap_default_hier_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def lap_default_solve_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().lap_default_solve_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Hierarchy:
    """Owns a lap_hierarchy_t; destroyed with the object or by destroy()."""

    def __init__(self, handle: int, n: int):
        self.handle = C.c_void_p(handle)
        self.n = n

    def destroy(self):
        if self.handle and self.handle.value:
            lib().lap_hierarchy_destroy(self.handle)
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def lap_build_hierarchy(n, src, dst, w=None, opts: HierOpts | None = None, stream=None) -> Hierarchy:
    ps, ks = _ptr(src, np.int32)
    pd, kd = _ptr(dst, np.int32)
    pw, kw = _ptr(w, np.float64)
    m = len(src) if not hasattr(src, "numel") else src.numel()
    out = C.c_void_p(0)
    st = lib().lap_build_hierarchy(int(n), int(m), ps, pd, pw, C.byref(opts) if opts is not None else None,
                                   _stream(stream), C.byref(out))
    _check(st, "lap_build_hierarchy")
    return Hierarchy(out.value, int(n))


def lap_hierarchy_destroy(h: Hierarchy):
    h.destroy()


def lap_hierarchy_info(h: Hierarchy) -> dict:
    info = HierInfo()
    _check(lib().lap_hierarchy_info(h.handle, C.byref(info)), "lap_hierarchy_info")
    L = info.levels
    return {"n": info.n, "m": info.m, "levels": L, "coarse_n": info.coarse_n,
            "level_n": list(info.level_n[:L]), "level_nnz": list(info.level_nnz[:L]), "setup_ms": info.setup_ms,
            "weight_exp": info.weight_exp, "level_row_order": list(info.level_row_order[:L]),
            "fingerprint": int(info.fingerprint), "elim_levels": info.elim_levels}


def lap_solve_multi(h: Hierarchy, B, X, opts: SolveOpts | None = None, stream=None, allow_noconv=False) -> dict:
    """B, X: contiguous FP64 CUDA tensors of shape (n, k)."""
    k = 1 if B.dim() == 1 else B.shape[1]
    pb, kb = _ptr(B, np.float64)
    px, kx = _ptr(X, np.float64)
    info = SolveInfo()
    st = lib().lap_solve_multi(h.handle, int(k), pb, px, C.byref(opts) if opts is not None else None,
                               _stream(stream), C.byref(info))
    _check(st, "lap_solve_multi", allow=(LAP_ENOCONV,) if allow_noconv else ())
    return {"status": st, "outer_iters": info.outer_iters, "inner_iters": info.inner_iters,
            "max_rel_residual": info.max_rel_residual, "k_tile": info.k_tile, "levels_used": info.levels_used,
            "nu_coarse": info.nu_coarse, "cycle": info.cycle, "coarse_scale": info.coarse_scale,
            "w_levels": info.w_levels, "first_residual_ff": info.first_residual_ff}


def cfc_jl_rhs(h: Hierarchy, k: int, seed: int, Y, stream=None):
    py, ky = _ptr(Y, np.float64)
    _check(lib().cfc_jl_rhs(h.handle, int(k), int(seed), py, _stream(stream)), "cfc_jl_rhs")
    return Y


def _out_f64(out, q):
    return np.empty(q, np.float64) if out is None else out


def cfc_farness_jl(h: Hierarchy, k: int, seed: int, nodes, eps: float = 0.0, opts: SolveOpts | None = None,
                   out=None, stream=None):
    q = len(nodes)
    pn, kn = _ptr(nodes, np.int32)
    out = _out_f64(out, q)
    po, ko = _ptr(out, np.float64)
    st = lib().cfc_farness_jl(h.handle, int(k), float(eps), int(seed), int(q), pn, po,
                              C.byref(opts) if opts is not None else None, _stream(stream))
    _check(st, "cfc_farness_jl")
    return out


def cfc_farness_jl_rows(h: Hierarchy, k_total: int, row_begin: int, row_count: int, seed: int, nodes,
                        opts: SolveOpts | None = None, out=None, stream=None):
    q = len(nodes)
    pn, kn = _ptr(nodes, np.int32)
    out = _out_f64(out, q)
    po, ko = _ptr(out, np.float64)
    st = lib().cfc_farness_jl_rows(h.handle, int(k_total), int(row_begin), int(row_count), int(seed), int(q), pn,
                                   po, C.byref(opts) if opts is not None else None, _stream(stream))
    _check(st, "cfc_farness_jl_rows")
    return out


def cfc_farness_from_solution(Z, nodes, out=None, stream=None):
    """Z: contiguous FP64 CUDA tensor (n, k); returns the farness of each node."""
    n, k = Z.shape
    q = len(nodes)
    pz, kz = _ptr(Z, np.float64)
    pn, kn = _ptr(nodes, np.int32)
    out = _out_f64(out, q)
    po, ko = _ptr(out, np.float64)
    _check(lib().cfc_farness_from_solution(int(n), int(k), pz, int(q), pn, po, _stream(stream)),
           "cfc_farness_from_solution")
    return out


def cfc_farness_from_solution_noalloc(Z, nodes, out, stream=None):
    """Allocation-free variant: Z (n, k) FP64, nodes int32 and out FP64 must
    all be CUDA tensors; returns after enqueuing the work on the stream."""
    n, k = Z.shape
    q = nodes.numel()
    pz, kz = _ptr(Z, np.float64)
    pn, kn = _ptr(nodes, np.int32)
    po, ko = _ptr(out, np.float64)
    _check(lib().cfc_farness_from_solution_noalloc(int(n), int(k), pz, int(q), pn, po, _stream(stream)),
           "cfc_farness_from_solution_noalloc")
    return out


def cfc_sample_pivots(h: Hierarchy, n_pivots: int, seed: int, out=None, stream=None):
    out = np.empty(n_pivots, np.int32) if out is None else out
    po, ko = _ptr(out, np.int32)
    _check(lib().cfc_sample_pivots(h.handle, int(n_pivots), int(seed), po, _stream(stream)), "cfc_sample_pivots")
    return out


def cfc_farness_sampled(h: Hierarchy, n_pivots: int, seed: int, nodes, opts: SolveOpts | None = None, out=None,
                        stream=None):
    q = len(nodes)
    pn, kn = _ptr(nodes, np.int32)
    out = _out_f64(out, q)
    po, ko = _ptr(out, np.float64)
    st = lib().cfc_farness_sampled(h.handle, int(n_pivots), int(seed), int(q), pn, po,
                                   C.byref(opts) if opts is not None else None, _stream(stream))
    _check(st, "cfc_farness_sampled")
    return out


def cfc_exact_small(n, src, dst, w=None, stream=None):
    """Returns (farness, closeness) as numpy arrays."""
    ps, ks = _ptr(src, np.int32)
    pd, kd = _ptr(dst, np.int32)
    pw, kw = _ptr(w, np.float64)
    m = len(src)
    f = np.empty(n, np.float64)
    c = np.empty(n, np.float64)
    st = lib().cfc_exact_small(int(n), int(m), ps, pd, pw, C.c_void_p(f.ctypes.data), C.c_void_p(c.ctypes.data),
                               _stream(stream))
    _check(st, "cfc_exact_small")
    return f, c


def lap_stats_reset():
    lib().lap_stats_reset()


def lap_stats_set_timing(on: bool):
    lib().lap_stats_set_timing(1 if on else 0)


def lap_stats_read() -> dict:
    s = Stats()
    _check(lib().lap_stats_read(C.byref(s)), "lap_stats_read")
    return {"launches_total": int(s.launches_total),
            "families": {name: {"launches": int(s.launches[i]), "ms": s.ms[i], "bytes": s.bytes[i]}
                         for i, name in enumerate(KERNEL_FAMILIES)}}


def lap_stats_set_log(on: bool):
    lib().lap_stats_set_log(1 if on else 0)


def lap_stats_read_log() -> list:
    """Families (names of KERNEL_FAMILIES) of the logged launches, in launch order."""
    cnt = C.c_int64(0)
    _check(lib().lap_stats_read_log(None, 0, C.byref(cnt)), "lap_stats_read_log")
    buf = (C.c_int32 * max(cnt.value, 1))()
    _check(lib().lap_stats_read_log(C.cast(buf, C.c_void_p), cnt.value, C.byref(cnt)), "lap_stats_read_log")
    return [KERNEL_FAMILIES[buf[i]] for i in range(cnt.value)]


def lap_tune_save(path: str):
    _check(lib().lap_tune_save(os.fsencode(path)), "lap_tune_save")


def lap_tune_load(path: str) -> int:
    added = C.c_int64(0)
    _check(lib().lap_tune_load(os.fsencode(path), C.byref(added)), "lap_tune_load")
    return added.value


def lap_tune_entries() -> int:
    return int(lib().lap_tune_entries())


# ------------------------------------------------------------------ serving
def cfc_server_default_opts(**kw) -> ServerOpts:
    o = ServerOpts()
    lib().cfc_server_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "solve":
            o.solve = v
        else:
            setattr(o, k, v)
    return o


class Server:
    """Owner of a cfc_server_t handle (freed by destroy() or on collection)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)

    def destroy(self):
        if self.handle:
            lib().cfc_server_destroy(self.handle)
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def cfc_server_create(opts: ServerOpts | None = None) -> Server:
    out = C.c_void_p(0)
    _check(lib().cfc_server_create(C.byref(opts if opts is not None else cfc_server_default_opts()),
                                   C.byref(out)), "cfc_server_create")
    return Server(out.value)


def cfc_server_add_graph(sv: Server, n, src, dst, w=None) -> int:
    """Host numpy edge arrays (copied); returns the graph id."""
    ps, ks = _ptr(np.ascontiguousarray(src, np.int32), np.int32)
    pd, kd = _ptr(np.ascontiguousarray(dst, np.int32), np.int32)
    pw, kw = _ptr(None if w is None else np.ascontiguousarray(w, np.float64), np.float64)
    gid = C.c_int32(-1)
    _check(lib().cfc_server_add_graph(sv.handle, int(n), int(len(src)), ps, pd, pw, C.byref(gid)),
           "cfc_server_add_graph")
    return gid.value


def cfc_server_submit(sv: Server, graph_id: int, nodes, n_pivots: int, seed: int = 0) -> int:
    """n_pivots = 0: use the graph's resident pivot set (see ServerOpts.resident_pivots)."""
    nd = np.ascontiguousarray(nodes, np.int32)
    rid = C.c_int64(0)
    _check(lib().cfc_server_submit(sv.handle, int(graph_id), int(nd.size), nd.ctypes.data_as(C.c_void_p),
                                   int(n_pivots), C.c_uint64(seed), C.byref(rid)), "cfc_server_submit")
    return rid.value


def cfc_server_poll(sv: Server, request_id: int, wait_ms: int = -1, q: int | None = None):
    """Returns (farness numpy array, info dict) when done, None while pending."""
    info = RequestInfo()
    buf = np.zeros(4096, np.float64) if q is None else np.zeros(q, np.float64)
    st = lib().cfc_server_poll(sv.handle, int(request_id), int(wait_ms), buf.ctypes.data_as(C.c_void_p),
                               C.byref(info))
    if st == LAP_EPENDING:
        return None
    _check(st, "cfc_server_poll")
    d = {f: getattr(info, f) for f, _ in RequestInfo._fields_}
    return buf[:info.q].copy(), d


def cfc_server_stats(sv: Server) -> dict:
    st = ServerStats()
    _check(lib().cfc_server_stats(sv.handle, C.byref(st)), "cfc_server_stats")
    return {f: getattr(st, f) for f, _ in ServerStats._fields_}


def cfc_server_reset_stats(sv: Server):
    lib().cfc_server_reset_stats(sv.handle)


def cfc_server_destroy(sv: Server):
    sv.destroy()
