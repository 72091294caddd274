/*
 * cfc_gb300.h -- C ABI of the GB300 Laplacian-solver / current-flow
 * closeness library.
 *
 * Method: Bergamini, Wegner, Lukarski, Meyerhenke, "Estimating Current-Flow
 * Closeness Centrality with a Multigrid Laplacian Solver" (arXiv:1607.02955).
 * Notation follows the paper: G = (V, E, w) connected, undirected, weighted
 * (Sec. 2); L = D - A its Laplacian (Sec. 2); supplies b with sum 0 and
 * potentials L p = b (Eq. system); effective resistance
 * d_ER(u, v) = p_uv(u) - p_uv(v) (Sec. 4); electrical farness
 * f(v) = sum_{w != v} d_ER(v, w) and current-flow closeness
 * c_ER(v) = (n - 1) / f(v) (Eq. closeness2).
 *
 * Conventions shared by every call
 *  - Every call returns a lap_status_t; none aborts, prints or throws.
 *    lap_status_string() names a status.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All device work of a call is ordered on it.  Calls that write
 *    host memory synchronise the stream before returning; calls that only
 *    write device memory return without synchronising.
 *  - Pointers documented "host or device" may be either; the library asks
 *    the CUDA driver which one (cudaPointerGetAttributes).  Device pointers
 *    must be on the current device.
 *  - Inputs are read, never kept: the caller keeps ownership of every array
 *    it passes.  A lap_hierarchy_t is owned by the library until
 *    lap_hierarchy_destroy().
 *  - Dense n x k blocks are row-major with the k columns of a row
 *    contiguous (element (i, j) at [i * k + j]).
 *  - Sizes: 2 <= n < 2^31 and 2 * m < 2^31 (32-bit row pointers).
 *  - Solves on one hierarchy may run at the same time on different streams
 *    (and from different host threads): each stream gets its own solve
 *    workspace, and a call that grows the hierarchy (lazy coarse levels,
 *    BF16 copies, autotuning) holds it exclusively while it does.  Calls on
 *    one stream run in stream order.  lap_hierarchy_destroy must not overlap
 *    any call on the same hierarchy.
 *  - A device reset (cudaDeviceReset) frees the library's device state
 *    along with everything else: hierarchies and servers made before it must
 *    not be used after it.
 */
#ifndef CFC_GB300_H
#define CFC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LAP_OK = 0,
    LAP_EINVAL = 1,    /* bad argument: size, index range, weight outside [1e-150, 1e150], NULL */
    LAP_ENOTCONN = 2,  /* the graph is not connected (Sec. 2 assumes connected G) */
    LAP_ENOMEM = 3,    /* a device allocation failed; nothing leaked */
    LAP_ENOCONV = 4,   /* a solve hit its iteration cap, or its residual became non-finite
                          (NaN or infinite, e.g. from FP32 overflow); outputs hold the last
                          iterate and lap_solve_info_t.max_rel_residual the (possibly NaN)
                          residual.  cfc_exact_small: its dense FP64 factorization lost
                          positive definiteness (weights too far apart) */
    LAP_ECUDA = 5,     /* a CUDA runtime error (the text is kept, see lap_last_error) */
    LAP_EBUDGET = 6,   /* request exceeds a documented maximum */
    LAP_ENOTIMPL = 7,
    LAP_EPENDING = 8   /* a served request has not finished yet (cfc_server_poll) */
} lap_status_t;

/* Arithmetic of a solve. */
enum {
    LAP_FP64 = 0,                     /* FP64 PCG + FP64 V-cycle */
    LAP_FP32_REFINED = 1,             /* FP32 PCG + V-cycle inside FP64 iterative refinement */
    LAP_FP32_BF16COARSE_REFINED = 2   /* as 1, with BF16 edge weights on levels >= 1 (Sec. 3.1
                                         solver, reduced-precision coarse operators): each
                                         coarse weight rounded to BF16, the coarse degrees
                                         recomputed from the rounded weights so every coarse
                                         operator is still a Laplacian; FP32 accumulation.
                                         Changes the preconditioner only: the FP64 outer
                                         residual and stopping test are those of mode 1. */
};

/* Smoother of the V-cycle. */
enum { LAP_SMOOTH_JACOBI = 0, LAP_SMOOTH_CHEBYSHEV = 1 };

/* How the pairwise matching of the aggregation ranks a neighbour j of node i
 * (Sec. 3.1 names LAMG's affinity-based aggregation without a formula):
 * LAP_AGG_STRENGTH  w_ij / max(D_ii, D_jj);
 * LAP_AGG_AFFINITY  (x_i . x_j)^2 / ((x_i . x_i)(x_j . x_j)) over 8 test vectors
 *                   relaxed by 4 damped Jacobi sweeps on L x = 0 of that graph. */
enum { LAP_AGG_STRENGTH = 0, LAP_AGG_AFFINITY = 1 };

typedef struct {
    int32_t coarse_max;   /* stop coarsening at n_l <= coarse_max (values above 2048 act as 2048);
                             the coarsest level (at most 2048 nodes) is solved with a dense
                             inverse, FP64 in LAP_FP64 and an FP32 copy in the FP32 modes.
                             0 (default): automatic, n_top / 4096 clamped to [256, 1024] with
                             n_top the size of the level the PCG runs on (the dense inverse is
                             built in every setup, so small graphs keep it small) */
    int32_t max_levels;   /* cap on levels incl. the finest (default 24); 1 = no coarsening */
    int32_t agg_passes;   /* pairwise-matching passes per level (default 2: aggregates of ~4) */
    int32_t match_rounds; /* handshake rounds per pass (default 4) */
    int32_t eager;        /* 1: build every level now; 0 (default): build the coarse
                             levels on the first solve that uses them */
    int32_t eliminate;    /* 1 (default): LAMG's low-degree elimination (Sec. 3.1): an
                             independent set of the nodes with one or two neighbours is
                             eliminated exactly before the multigrid levels, when that
                             removes at least 5% of the nodes; the PCG and the cycle then
                             run on the Schur complement (a Laplacian), the FP64 residual
                             of the refinement on G itself.  0: no elimination */
    int32_t reorder;      /* processing order of each level's rows by the row kernels (the
                             nodes keep their labels): 0 (default) longest rows first on
                             levels whose row lengths are very uneven, natural order
                             elsewhere; 1 natural order; 2 longest first everywhere */
    int32_t aggregation;  /* LAP_AGG_STRENGTH (default) | LAP_AGG_AFFINITY */
    int32_t chunking;     /* how the row kernels split long rows (the hubs): 1 rows longer
                             than 32 entries in chunks of 16 (many small work units: best on
                             small levels, whose short sweeps a long chunk would dominate), 2
                             rows longer than 128 in chunks of 128 (fewer partial sums through
                             DRAM: best on large levels); 0 (default): 1 for levels (and the
                             elimination's pull lists) of at most 2^22 entries, 2 above */
    int32_t hub_factor;   /* > 0: a node with more than hub_factor x the mean row length of
                             its level neither joins nor absorbs an aggregate (it stays a
                             singleton); 0 (default): no hub rule.  At most 1000000 */
} lap_hier_opts_t;

typedef struct {
    int32_t precision;    /* LAP_FP64 | LAP_FP32_REFINED | LAP_FP32_BF16COARSE_REFINED */
    double tol;           /* per-column ||b - L x||_2 / ||b||_2 target (default 1e-8) */
    int32_t max_outer;    /* refinement steps (default 8) */
    int32_t max_inner;    /* PCG iterations per refinement step (default 200) */
    double inner_tol;     /* inner PCG relative residual (default 1e-4) */
    int32_t k_tile;       /* columns per tile: 0 = autotune, else 16, 32, 64 or 128 */
    int32_t smoother;     /* LAP_SMOOTH_JACOBI | LAP_SMOOTH_CHEBYSHEV (default Chebyshev) */
    int32_t nu_pre;       /* smoothing steps before the coarse correction (default 2) */
    int32_t nu_post;      /* smoothing steps after (default 2) */
    int32_t check_every;  /* inner iterations between host convergence reads (default 4) */
    int32_t levels_used;  /* levels of the hierarchy the cycle uses: > 0 that many
                             (at most), -1 every level, 0 (default) autotuned: the
                             first solve for a graph size and configuration times
                             complete solves (smoother alone, 2, 3, 4 and all levels,
                             coarse scales, W-cycles, column tiles; each candidate
                             stopped once it runs twice as long as the best) and the
                             fastest converged one is kept for the process; the choice
                             is reported in lap_solve_info_t */
    int32_t nu_coarse;    /* smoothing steps (Chebyshev degree) at a coarsest level that has
                             no dense solve, e.g. the one-level smoother-only
                             preconditioner; 0 (default): max(nu_pre, 4), or autotuned
                             together with levels_used */
    int32_t cycle;        /* 1: V-cycle, 2: W-cycle (two coarse corrections per level);
                             0 (default): V, or autotuned together with levels_used */
    double coarse_scale;  /* factor on each coarse correction (> 0; 0 = 1.0, or autotuned) */
    int32_t w_levels;     /* with cycle 2: the levels, from the finest, that take two coarse
                             corrections (V below them); 0 (default): every level, or
                             autotuned together with the cycle */
    int32_t graphs;       /* 1 (default): a multilevel cycle is captured once per solve as
                             a CUDA graph and replayed at every preconditioner application
                             (one launch instead of one per kernel); 0: plain launches.
                             Plain launches are also used while lap_stats timing or the
                             launch log is on, so that those see every kernel */
    int32_t first_residual_ff; /* 1 (default): the first refinement step's residual is formed
                             in two FP32 words where that is exact enough (FP32 modes, FP32
                             weights exactly 2^-e w; see lap_solve_info_t); 0: every residual
                             in FP64.  The stopping test uses an FP64 residual either way */
} lap_solve_opts_t;

typedef struct {
    int32_t outer_iters;
    int32_t inner_iters;        /* total over all refinement steps */
    double max_rel_residual;    /* max over columns of the final FP64 ||b - Lx|| / ||b||;
                                   NaN when some column's residual is NaN */
    /* the configuration the solve ran with (the autotuner's choice where the
       options left it open); passing these back as options repeats the solve
       bit for bit without tuning */
    int32_t k_tile, levels_used, nu_coarse, cycle;
    double coarse_scale;
    int32_t w_levels;
    int32_t first_residual_ff;  /* 1 when the first refinement step's residual (x = the first
                                   correction) was formed in two FP32 words from exact FP32
                                   weights (about 48 bits) instead of FP64; it only feeds the
                                   next inner solve, and the stopping test always uses an FP64
                                   residual.  0 otherwise (FP64 mode, weights not exact in
                                   FP32, max_outer <= 1, or no second step) */
} lap_solve_info_t;

typedef struct {
    int64_t n, m;               /* nodes, undirected edges after merging duplicates */
    int32_t levels;
    int32_t coarse_n;           /* size of the dense coarsest level (0 if none) */
    int64_t level_n[32];
    int64_t level_nnz[32];      /* off-diagonal entries of each level's CSR */
    double setup_ms;            /* device time of lap_build_hierarchy */
    int32_t weight_exp;         /* e with 2^e <= largest weight < 2^(e+1): the FP32 and BF16
                                   sweeps run on the exactly scaled operator 2^-e L, so that
                                   weights far from 1 stay inside FP32's range */
    int32_t level_row_order[32];/* 1: the row kernels take the level's rows longest first (the
                                   level's row lengths are very uneven); 0: natural order */
    uint64_t fingerprint;       /* order-free 64-bit hash of the merged graph (its edges and
                                   weights): the key of the autotuner's choices */
    int32_t elim_levels;        /* leading levels made by low-degree elimination (0 or 1): the
                                   PCG and the multigrid cycle start at level elim_levels */
} lap_hier_info_t;

typedef struct lap_hierarchy lap_hierarchy_t;

/* Fill defaults into an options struct. */
void lap_default_hier_opts(lap_hier_opts_t *o);
void lap_default_solve_opts(lap_solve_opts_t *o);

/*
 * lap_build_hierarchy -- ingest G and build the multigrid hierarchy.
 * Sec. 2 (graph model, L = D - A), Sec. 3.1 and Sec. 6.1 (an algebraic
 * multigrid Laplacian solver; the paper's LAMG coarsens by elimination and
 * affinity-based aggregation -- this library eliminates nodes with one or two
 * neighbours and aggregates by pairwise matching, see lap_hier_opts_t).
 *   n           number of nodes, 2 <= n < 2^31
 *   m           number of input edges (m >= 1)
 *   src, dst    int32[m], host or device: edge endpoints in [0, n).
 *               Self-loops are dropped; edge direction is ignored;
 *               repeated pairs are merged with their weights summed
 *               (parallel conductances) (Sec. 6.3).  Page-locked host
 *               buffers (cudaHostAlloc, cudaHostRegister) are read in place
 *               by the first kernels, other host buffers are copied first;
 *               either way they are not read after the call returns.
 *   w           double[m], host or device, or NULL for unit weights; each
 *               weight a conductance (Sec. 2) with 1e-150 <= w <= 1e150, a
 *               range in which the FP64 sums and products of the solver
 *               cannot overflow.
 *   opts        NULL = defaults.
 *   out         receives the hierarchy on LAP_OK, NULL otherwise.
 * Errors: LAP_EINVAL (sizes, NULL, endpoint out of range, weight outside the range);
 * LAP_ENOTCONN (G not connected, Sec. 2); LAP_ENOMEM; LAP_ECUDA.
 * Synchronises `stream`.
 */
lap_status_t lap_build_hierarchy(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                 const double *w, const lap_hier_opts_t *opts, void *stream,
                                 lap_hierarchy_t **out);

/* Release every device and host resource of h (NULL is a no-op). */
void lap_hierarchy_destroy(lap_hierarchy_t *h);

/* Sizes of h's levels. */
lap_status_t lap_hierarchy_info(const lap_hierarchy_t *h, lap_hier_info_t *info);

/*
 * lap_solve_multi -- solve L X = B for k right-hand sides at once (Eq.
 * system; Sec. 3.1: iterate until the relative residual is below tol).
 * Each column is an independent system (its own CG step lengths): results
 * do not depend on k, the tile width or the other columns.
 *   k    number of columns, 1 <= k <= 4096
 *   B    device double[n * k] row-major.  Each column is projected onto
 *        range(L) = 1-perp first (the null space span{1} of L, Sec. 2).
 *   X    device double[n * k] row-major, output: the zero-mean solution
 *        L^+ B of every column.  May not alias B.
 *   o    NULL = defaults.  info may be NULL.
 * A column is converged once its FP64 relative residual is <= tol; a NaN or
 * infinite residual never is.  The FP32 modes scale each column's residual
 * by a power of two before demoting it to FP32 (and the operator by
 * 2^-weight_exp), so the inner solves see no overflow or underflow.
 * Errors: LAP_EINVAL (also when a column of B has a non-finite 2-norm: NaN or
 * infinite entries, or entries too large to square; X is then not written);
 * LAP_ENOCONV (some column above tol after max_outer refinement steps, or a
 * residual that became non-finite; X holds the last iterate, info the
 * residual); LAP_ENOMEM; LAP_ECUDA.  Synchronises `stream` (convergence is
 * read on the host).
 */
lap_status_t lap_solve_multi(lap_hierarchy_t *h, int32_t k, const double *B, double *X,
                             const lap_solve_opts_t *o, void *stream, lap_solve_info_t *info);

/*
 * cfc_jl_rhs -- Algorithm 1, steps 1-2: Y = Q W^{1/2} B with Q a k x m
 * matrix of +-1/sqrt(k) entries drawn from Philox4x64-10 (Sec. 5.2).
 * Edge e = {u < v} (ids: lexicographic rank of (u, v) after merging) has
 * B(e, u) = +1, B(e, v) = -1.  Sign of Q[i, e]: bit (i % 64) of word
 * (i % 256) / 64 of Philox4x64-10(counter = (e, i / 256, 0, 0),
 * key = (seed, 0x4A4C)); bit 0 -> +1/sqrt(k), 1 -> -1/sqrt(k).
 *   Y    device double[n * k], row-major: Y[u * k + i] = (Q W^{1/2} B)_{i,u},
 *        i.e. column i of this block is row i of the paper's k x n Y.
 */
lap_status_t cfc_jl_rhs(lap_hierarchy_t *h, int32_t k, uint64_t seed, double *Y, void *stream);

/*
 * cfc_farness_jl -- the projection estimator of Sec. 5.2 / Algorithm 1:
 * build Y (cfc_jl_rhs), solve L z_i = Y_i for the k rows (lap_solve_multi),
 * and return f~(v) = sum_{w != v} ||Z_{.,v} - Z_{.,w}||^2 for each query node,
 * evaluated in O(nk) as sum_i [n Z_iv^2 - 2 Z_iv S_i + T_i] with
 * S_i = sum_w Z_iw, T_i = sum_w Z_iw^2 (FP64).  The closeness estimate is
 * (n - 1) / f~(v).
 *   k        JL dimension; k <= 0 means k = ceil(ln(n) / eps^2) (Sec. 6.4)
 *   eps      used only when k <= 0
 *   q        number of query nodes, 1 <= q <= n
 *   nodes    int32[q], host or device
 *   farness  double[q], host or device, output
 * Errors: as lap_solve_multi; LAP_EINVAL for a node out of range.
 */
lap_status_t cfc_farness_jl(lap_hierarchy_t *h, int32_t k, double eps, uint64_t seed, int32_t q,
                            const int32_t *nodes, double *farness, const lap_solve_opts_t *o,
                            void *stream);

/*
 * cfc_farness_jl_rows -- the terms of cfc_farness_jl contributed by rows
 * row_begin .. row_begin + row_count - 1 of the k_total-row Q (Algorithm 1:
 * the rows are independent solves, and f~(v) is a sum over rows), scaled by
 * 1/sqrt(k_total).  Summing the outputs over a partition of [0, k_total)
 * gives cfc_farness_jl(h, k_total, ...) up to the order of the FP64 sums:
 * the unit of work that several GPUs split, each summing its own rows, with
 * one reduction of q doubles at the end (no counterpart in the paper, which
 * runs on one machine).
 *   row_begin  multiple of 32, 0 <= row_begin;  row_count >= 1, <= 4096,
 *              row_begin + row_count <= k_total
 *   q, nodes, farness as cfc_farness_jl (farness receives the partial sums)
 */
lap_status_t cfc_farness_jl_rows(lap_hierarchy_t *h, int32_t k_total, int32_t row_begin, int32_t row_count,
                                 uint64_t seed, int32_t q, const int32_t *nodes, double *farness,
                                 const lap_solve_opts_t *o, void *stream);

/*
 * cfc_farness_from_solution -- Algorithm 1, step 4 and the closing formula of
 * Sec. 5.2 on a solution block the caller already has: for each query node v,
 * f~(v) = sum_{w != v} ||Z_{.,v} - Z_{.,w}||^2, evaluated in O(nk) as
 * sum_i [n Z_vi^2 - 2 Z_vi S_i + T_i] with S_i = sum_w Z_wi, T_i = sum_w Z_wi^2,
 * all sums in FP64 in a fixed order (bitwise reproducible).
 *   n        number of nodes, n >= 2
 *   k        columns of Z, 1 <= k <= 4096
 *   Z        device double[n * k] row-major: Z[u * k + i] = z_i(u), the i-th
 *            solution of Algorithm 1 evaluated at node u
 *   q, nodes, farness as cfc_farness_jl (host or device)
 * Errors: LAP_EINVAL (sizes, NULL, Z not on the device, node out of range),
 * LAP_ENOMEM, LAP_ECUDA.  Synchronises `stream`.
 */
lap_status_t cfc_farness_from_solution(int64_t n, int32_t k, const double *Z, int32_t q,
                                       const int32_t *nodes, double *farness, void *stream);

/*
 * cfc_farness_from_solution_noalloc -- cfc_farness_from_solution for callers
 * that cannot allocate device memory when they need the result: code running
 * inside an allocator or out-of-memory handler, a process held to a hard
 * device-memory cap, or work on a stream that must not wait on the
 * allocator.  The paper has no counterpart: this is a deployment variant.
 * It allocates nothing (no cudaMalloc, cudaFree or allocating library call);
 * its scratch is a fixed 2 MiB + 4 KiB array in the library, reserved on
 * every GPU that loads the library until the process exits.
 *   n, k, Z    as cfc_farness_from_solution, with k <= 256
 *   q >= 1, nodes  device int32[q]; a node outside [0, n) gets NaN
 *   farness    device double[q], output
 * The scratch address is looked up once per device, by the first call on
 * that device of this function, cfc_farness_from_solution or
 * lap_build_hierarchy, with the device current; under CUDA's lazy module
 * loading that first call also loads the library's device code, which
 * allocates.  So make one such call on each device before memory runs short
 * and before capturing the stream into a CUDA graph.
 * Results equal those of cfc_farness_from_solution.  All calls share the one
 * scratch array: calls whose work overlaps on the same GPU race, so order
 * them on one stream (or synchronise between them).  The call only enqueues
 * work on `stream` and returns without synchronising.
 * Errors: LAP_EBUDGET (k > 256), LAP_EINVAL (sizes, NULL, a pointer that is
 * not device memory), LAP_ECUDA.
 */
lap_status_t cfc_farness_from_solution_noalloc(int64_t n, int32_t k, const double *Z, int32_t q,
                                               const int32_t *nodes, double *farness, void *stream);

/*
 * cfc_sample_pivots -- the pivot set S of Sec. 5.1: a uniform n_pivots-subset
 * of V without replacement (all of V: a query node may be a pivot), drawn on
 * the device by Floyd's algorithm; Floyd step s (s = 0..n_pivots-1, range
 * [0, n - n_pivots + s]) draws floor(u * range / 2^64) with u = word 0 of
 * Philox4x64-10(counter = (s, 0, 0, 0), key = (seed, 0x534D50)).
 *   pivots  int32[n_pivots], host or device, output, ascending.
 */
lap_status_t cfc_sample_pivots(lap_hierarchy_t *h, int32_t n_pivots, uint64_t seed, int32_t *pivots,
                               void *stream);

/*
 * cfc_farness_sampled -- the sampling estimator of Sec. 5.1: with S from
 * cfc_sample_pivots, f^(v) = (n / |S|) sum_{s in S} d_ER(v, s), the unbiased
 * farness estimate of Proposition 1.  d_ER(v, s) is evaluated from column
 * solves x_u = L^+ (e_u - 1/n) for u in S and the query nodes:
 * d_ER(v, s) = x_v(v) - x_v(s) - x_s(v) + x_s(s), algebraically the
 * potential difference of the pair system L p = e_v - e_s (Eq. system).
 * Closeness: (n - 1) / f^(v) (equal to (k/n)(n-1)/f~(v, S) of Sec. 5.1).
 *   n_pivots 1 <= n_pivots <= n;  q, nodes, farness as cfc_farness_jl.
 */
lap_status_t cfc_farness_sampled(lap_hierarchy_t *h, int32_t n_pivots, uint64_t seed, int32_t q,
                                 const int32_t *nodes, double *farness, const lap_solve_opts_t *o,
                                 void *stream);

/*
 * cfc_exact_small -- exact electrical farness and current-flow closeness of
 * every node of a small graph (Sec. 4, Eq. closeness2), in FP64 on the
 * device, from the dense pseudoinverse L^+ = (L + J/n)^{-1} - J/n:
 * f(v) = n L^+_vv + tr(L^+) (equal to sum_w [L^+_vv - 2 L^+_vw + L^+_ww]
 * since L^+ 1 = 0), c(v) = (n - 1) / f(v).
 *   n <= 16384 (the dense n x n FP64 matrix is held on the device);
 *   src, dst, w as lap_build_hierarchy;
 *   farness   double[n], host or device, output
 *   closeness double[n], host or device, output, or NULL
 * Errors: LAP_EINVAL, LAP_EBUDGET (n too large), LAP_ENOTCONN, LAP_ENOCONV
 * (the FP64 factorization lost definiteness: weights too far apart),
 * LAP_ENOMEM, LAP_ECUDA.  Synchronises `stream`.
 */
lap_status_t cfc_exact_small(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                             const double *w, double *farness, double *closeness, void *stream);

/*
 * Autotuner table (no counterpart in the paper).  A solve whose options leave
 * the configuration open (levels_used = 0) is tuned once per graph (keyed by
 * lap_hier_info_t.fingerprint, so graphs of equal size but different
 * structure are tuned separately) and per solve configuration (k, precision
 * and the fields the caller fixed); the choice is kept for the process.  The
 * choice depends on timings, so two processes may choose differently; a
 * process that loads the table another one saved repeats its choices, and
 * with them the bits of every solve, without timing candidates again.
 *   lap_tune_save   writes the whole table to `path` as JSON (through a
 *                   temporary file renamed into place)
 *   lap_tune_load   adds the entries of such a file (keys already present
 *                   keep their choice); *added (nullable) receives how many
 *   lap_tune_entries  number of entries in the table
 * With the environment variable LAP_TUNE_CACHE set to a path, that file is
 * loaded before the process's first tuning and rewritten after each new
 * choice.  Errors: LAP_EINVAL (NULL or empty path, a file that cannot be
 * read or written, a malformed entry).
 */
lap_status_t lap_tune_save(const char *path);
lap_status_t lap_tune_load(const char *path, int64_t *added);
int64_t lap_tune_entries(void);

/* Human-readable name of a status. */
const char *lap_status_string(lap_status_t s);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char *lap_last_error(void);

/*
 * Instrumentation (no counterpart in the paper).  Counts every kernel this
 * library launches; when timing is on, brackets each launch of the kernel
 * families below with CUDA events on the launching stream and accumulates
 * the device time and the algorithmic bytes (each operand read once,
 * each result written once) of those launches.
 */
enum {
    LAP_KF_SPMV_FINE = 0,     /* FP32 L*p of the PCG at the finest level */
    LAP_KF_SMOOTH_FINE = 1,   /* FP32 smoother steps at the finest level */
    LAP_KF_RESTRICT_FINE = 2, /* residual + restriction at the finest level */
    LAP_KF_BLAS1 = 3,         /* PCG vector updates and dot products (finest level) */
    LAP_KF_COARSE_LEVELS = 4, /* every V-cycle kernel below the finest level */
    LAP_KF_RESID64 = 5,       /* FP64 outer residual */
    LAP_KF_SETUP = 6,         /* ingest + hierarchy */
    LAP_KF_CFC = 7,           /* RHS generation and farness reductions */
    LAP_KF_COUNT = 8
};

typedef struct {
    uint64_t launches_total;          /* every kernel launch since the last reset */
    uint64_t launches[LAP_KF_COUNT];
    double ms[LAP_KF_COUNT];          /* event-timed device ms (timing on only) */
    double bytes[LAP_KF_COUNT];       /* algorithmic bytes of the timed launches */
} lap_stats_t;

void lap_stats_reset(void);
void lap_stats_set_timing(int32_t on);
/* Synchronises the pending timing events, then copies the counters. */
lap_status_t lap_stats_read(lap_stats_t *out);

/*
 * Launch log (no counterpart in the paper): while on, the family (LAP_KF_*)
 * of every kernel launch is appended, in launch order, to a host-side log
 * that lap_stats_reset clears.  A profiler's per-launch list of the same
 * region lines up with it one to one, which attributes per-launch hardware
 * counters to families.  lap_stats_read_log copies min(count, capacity)
 * entries to the host array `families` and stores the full count in *count;
 * LAP_EINVAL if `count` is NULL or `families` is NULL with capacity > 0.
 */
void lap_stats_set_log(int32_t on);
lap_status_t lap_stats_read_log(int32_t *families, int64_t capacity, int64_t *count);

/*
 * Serving (no counterpart in the paper, which times one query at a time):
 * a request loop over resident graphs for the sampling estimator of Sec. 5.1
 * (cfc_farness_sampled), with continuous batching.  Each request is the
 * farness of q query nodes from one pivot set of n_pivots nodes (n_pivots + q
 * column solves).  `slots` worker threads, each with its own CUDA stream,
 * take requests in arrival order as soon as a slot is free and the request's
 * device memory fits the HBM budget next to the resident graphs and the
 * requests in flight, so requests that arrive while others run are admitted
 * while those are still on the GPU and their solves overlap on the device.
 * A slot that takes the head of the queue also takes the queued requests on
 * the same graph that fit (batch_columns) and solves their columns as one
 * block.
 *
 * A graph's hierarchy is built completely when it is added, and the solver
 * configuration for its requests is autotuned once then and pinned, so a
 * request's result does not depend on what else is in flight (the kernels'
 * reductions have a fixed order): the same bits alone and in a mix.
 *
 * Ownership: the server owns the hierarchies it builds and the request
 * results until they are polled.  Inputs are copied.  Calls are thread-safe.
 */
typedef struct cfc_server cfc_server_t;

typedef struct {
    int32_t slots;          /* concurrent requests on the device, 1..64 (default 4) */
    int64_t hbm_budget;     /* bytes for resident graphs + requests in flight; 0 (default):
                               80% of the device memory free at creation */
    lap_solve_opts_t solve; /* solve options (precision, tol, ...); tuned fields left 0 are
                               autotuned per graph when it is added */
    int32_t resident_pivots; /* > 0: every added graph also gets a pivot set of this many
                                nodes (drawn as cfc_sample_pivots with seed pivot_seed +
                                graph id) whose solutions stay on the device (n x count FP64,
                                charged to the budget); requests with n_pivots = 0 then solve
                                only their q nodes' columns against it.  0 (default): none */
    uint64_t pivot_seed;
    int32_t batch_columns;  /* continuous batching: when a slot takes the head of the queue it
                               also takes the queued requests on the same graph and of the same
                               kind (drawn pivots, or the resident set) that fit, and solves all
                               their columns as one block, up to this many columns (default
                               1024; at most 4096 and 64 tiles of the graph's pinned tile
                               width); 1: one request per solve.  A request's result is the
                               same alone and in a batch (columns are independent systems) */
} cfc_server_opts_t;

typedef struct {
    int32_t status;         /* the request's lap_status_t */
    int32_t graph_id, q, n_pivots;
    int64_t device_bytes;   /* the memory it was admitted with (estimate, charged to the budget) */
    double queue_ms;        /* submit -> admitted to a slot */
    double run_ms;          /* admitted -> result on the host */
    double latency_ms;      /* submit -> result on the host */
} cfc_request_info_t;

typedef struct {
    int64_t submitted, completed, pending, in_flight;
    int32_t max_in_flight;  /* most requests seen on the device at once */
    double p50_ms, p99_ms, mean_ms, max_ms;  /* latency of the completed requests (nearest rank) */
    double queries_per_s;   /* completed requests / (last completion - first submission) */
    double rhs_per_s;       /* their column solves per second over the same span */
    int64_t graph_bytes, budget_bytes, peak_in_flight_bytes;
    int32_t max_batch;      /* most requests solved together in one block */
} cfc_server_stats_t;

void cfc_server_default_opts(cfc_server_opts_t *o);
/* LAP_EINVAL on bad options; LAP_ECUDA if the streams cannot be made. */
lap_status_t cfc_server_create(const cfc_server_opts_t *o, cfc_server_t **out);
/* Builds the graph's hierarchy (as lap_build_hierarchy, every level) and
 * tunes its solves; *graph_id receives its index.  LAP_EBUDGET if it does not
 * fit the budget next to the graphs already resident. */
lap_status_t cfc_server_add_graph(cfc_server_t *sv, int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                  const double *w, int32_t *graph_id);
/* Queues a request (host `nodes`, copied) and returns at once with its id.
 * n_pivots > 0: a fresh pivot set of that size drawn with `seed` (n_pivots + q
 * column solves); n_pivots = 0: the graph's resident pivot set (q column
 * solves; `seed` unused).  The estimate is unbiased either way (Proposition
 * 1); requests sharing the resident set are correlated with each other.
 * LAP_EINVAL for a bad graph id, node or count, or n_pivots = 0 on a graph
 * without a resident set; LAP_EBUDGET if the request alone exceeds what the
 * budget leaves beside the resident graphs. */
lap_status_t cfc_server_submit(cfc_server_t *sv, int32_t graph_id, int32_t q, const int32_t *nodes,
                               int32_t n_pivots, uint64_t seed, int64_t *request_id);
/* Waits up to wait_ms (0: no wait, < 0: until done) for the request.  Done:
 * copies its q farness values to the host array `farness` (may be NULL),
 * fills *info (may be NULL), forgets the request and returns its status.
 * Not done: LAP_EPENDING.  Unknown (or already polled) id: LAP_EINVAL. */
lap_status_t cfc_server_poll(cfc_server_t *sv, int64_t request_id, int32_t wait_ms, double *farness,
                             cfc_request_info_t *info);
lap_status_t cfc_server_stats(cfc_server_t *sv, cfc_server_stats_t *out);
/* Drops the latency record (the counters of completed requests) and the
 * throughput span, e.g. after a warm-up. */
void cfc_server_reset_stats(cfc_server_t *sv);
/* Finishes the requests in flight, drops the queued ones, frees everything. */
void cfc_server_destroy(cfc_server_t *sv);

#ifdef __cplusplus
}
#endif
#endif /* CFC_GB300_H */
