"""Python binding of libcfc_gb300 (include/cfc_gb300.h), the GB300 Laplacian
solver behind the current-flow closeness estimators of Bergamini et al.
(arXiv:1607.02955).

The binding only marshals arguments: every step of the computation runs in
the native library's CUDA kernels.  Functions carry the C names.  Device
buffers are torch CUDA tensors (FP64, contiguous); host buffers are numpy
arrays.  The library must be built (``build_ext.build()``); importing works
without it, but every call raises ``RuntimeError`` when it is missing.
"""
from __future__ import annotations

from ._binding import (  # noqa: F401
    LapError,
    Hierarchy,
    HierOpts,
    SolveOpts,
    LAP_OK,
    LAP_EINVAL,
    LAP_ENOTCONN,
    LAP_ENOMEM,
    LAP_ENOCONV,
    LAP_ECUDA,
    LAP_EBUDGET,
    LAP_ENOTIMPL,
    LAP_EPENDING,
    LAP_FP64,
    LAP_FP32_REFINED,
    LAP_FP32_BF16COARSE_REFINED,
    LAP_SMOOTH_JACOBI,
    LAP_SMOOTH_CHEBYSHEV,
    LAP_AGG_STRENGTH,
    LAP_AGG_AFFINITY,
    KERNEL_FAMILIES,
    lib,
    lib_path,
    exported_symbols,
    lap_default_hier_opts,
    lap_default_solve_opts,
    lap_build_hierarchy,
    lap_hierarchy_destroy,
    lap_hierarchy_info,
    lap_solve_multi,
    cfc_jl_rhs,
    cfc_farness_jl,
    cfc_farness_jl_rows,
    cfc_farness_from_solution,
    cfc_farness_from_solution_noalloc,
    cfc_sample_pivots,
    cfc_farness_sampled,
    cfc_exact_small,
    lap_status_string,
    lap_last_error,
    lap_stats_reset,
    lap_stats_set_timing,
    lap_stats_read,
    lap_stats_set_log,
    lap_stats_read_log,
    lap_tune_entries,
    lap_tune_load,
    lap_tune_save,
    Server,
    ServerOpts,
    cfc_server_default_opts,
    cfc_server_create,
    cfc_server_add_graph,
    cfc_server_submit,
    cfc_server_poll,
    cfc_server_stats,
    cfc_server_reset_stats,
    cfc_server_destroy,
)
