// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (include/cfc_gb300.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <new>
#include <string>
#include <deque>
#include <map>
#include <mutex>
#include <shared_mutex>
#include <vector>

#include "../../include/cfc_gb300.h"

struct lap_hierarchy;

namespace cfc {

// ------------------------------------------------------------------ errors
struct Error {
    lap_status_t status;
    std::string what;
};

void set_last_error(const std::string &s);
void clear_last_error();

// Runs f and turns what it throws into a status (the text kept for
// lap_last_error): no C entry point lets an exception through.
template <class F>
lap_status_t guard(F &&f) {
    try {
        clear_last_error();
        return f();
    } catch (const Error &e) {
        set_last_error(e.what);
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return LAP_ENOMEM;
    } catch (...) {
        set_last_error("unknown error");
        return LAP_ECUDA;
    }
}

#define CFC_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            if (e_ == cudaErrorMemoryAllocation) {                                             \
                cudaGetLastError();                                                            \
                throw ::cfc::Error{LAP_ENOMEM, "out of device memory"};                        \
            }                                                                                  \
            throw ::cfc::Error{LAP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
        }                                                                                      \
    } while (0)

#define CFC_REQUIRE(cond, st, msg)                  \
    do {                                            \
        if (!(cond)) throw ::cfc::Error{(st), (msg)}; \
    } while (0)

// ------------------------------------------------------------------ launches
// Every kernel launch goes through a LaunchScope so the library
// can count its launches and, when timing is on, time the families of
// include/cfc_gb300.h with CUDA events on the launching stream.
struct LaunchScope {
    int family;
    cudaStream_t stream;
    double bytes;
    cudaEvent_t start = nullptr;
    LaunchScope(int family, cudaStream_t s, double algorithmic_bytes);
    ~LaunchScope();
};
// for graph replays: whether timing or the launch log is on (graphs are then
// not used), the per-family launch counters, and adding a graph's launches
bool stats_detailed();
void stats_launches(int64_t out[LAP_KF_COUNT]);
void stats_add_launches(const int64_t delta[LAP_KF_COUNT], int64_t times);

#define CFC_LAUNCH(family, stream, bytes, kernel, grid, block, smem, ...)       \
    do {                                                                       \
        ::cfc::LaunchScope scope_((family), (stream), (bytes));                \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);            \
        CFC_CUDA(cudaGetLastError());                                          \
    } while (0)

// ------------------------------------------------------------------ memory
// The library's own stream-ordered memory pool (one per device), with a
// release threshold high enough that freed blocks stay reserved for reuse:
// repeated builds and solves then allocate without reaching the driver.
cudaMemPool_t library_pool();

// Device buffers owned by the library.  All allocations are stream-ordered
// (cudaMallocAsync) and freed the same way.
template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    bool async = false;
    DBuf() = default;
    DBuf(size_t count, cudaStream_t stream) { alloc(count, stream); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), s(o.s), async(o.async) { o.p = nullptr; o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; s = o.s; async = o.async;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    // stream-ordered temporary, freed on the same stream
    void alloc(size_t count, cudaStream_t stream) {
        release();
        s = stream;
        n = count;
        async = true;
        if (count) CFC_CUDA(cudaMallocFromPoolAsync((void **)&p, count * sizeof(T) + 16, library_pool(), stream));
    }
    // long-lived buffer (hierarchy data, workspace): taken from the pool on
    // the legacy default stream and returned there when released
    void alloc_persistent(size_t count) {
        release();
        n = count;
        async = true;
        s = nullptr;
        if (count) CFC_CUDA(cudaMallocFromPoolAsync((void **)&p, count * sizeof(T) + 16, library_pool(), nullptr));
    }
    void zero(cudaStream_t stream) const {
        if (n) CFC_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), stream));
    }
    void release() noexcept {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        n = 0;
    }
    ~DBuf() { release(); }
    T *get() const { return p; }
};

bool is_device_pointer(const void *p);
// The device address of a page-locked host buffer (read in place by kernels
// over the host link), or nullptr for any other pointer.
const void *mapped_host_pointer(const void *p);

// ------------------------------------------------------------------ graph levels
// One level of the multigrid hierarchy: the Laplacian L = D - A of a graph in
// CSR form holding only the off-diagonal adjacency weights w_ij > 0 (the
// matrix entries are -w_ij) plus the degree vector D_ii = sum_j w_ij.
struct Level {
    int32_t n = 0;
    int64_t nnz = 0;
    DBuf<int32_t> rowptr, col;
    DBuf<double> w64, deg64, dinv64;
    DBuf<float> w32, deg32, dinv32;
    // BF16 copy of the weights (bit patterns) and the FP32 degrees of the
    // rounded weights, made on first use by a solve in the BF16-coarse mode
    DBuf<uint16_t> wbf;
    DBuf<float> degbf, dinvbf;
    // rows longer than long_row nonzeros are split into chunks of `chunk`
    // (chunk_params: short chunks on levels with few entries)
    int32_t long_row = 0, chunk = 0;
    int32_t n_long = 0, n_chunks = 0;
    DBuf<int32_t> chunk_row;     // [n_chunks] row of each chunk
    DBuf<int32_t> chunk_begin;   // [n_chunks] first nonzero of the chunk
    DBuf<int32_t> chunk_long;    // [n_chunks] index of the chunk's long row
    DBuf<int32_t> long_first;    // [n_long + 1] first chunk of each long row
    DBuf<int32_t> long_of_row;   // [n] index of the row among the long rows, -1 if short
    // [n_chunks] processing order of the chunks: ascending first column, so
    // that the chunks in flight together gather from a narrow range of
    // columns (the long rows' columns are sorted) and the gathered rows are
    // reused from L2; each chunk's partial sum stays at its own index
    DBuf<int32_t> chunk_order;
    DBuf<int32_t> order;         // [n] processing order of the rows (longest first), or empty: natural
    // map to the next coarser level (empty at the coarsest)
    DBuf<int32_t> agg;           // [n] aggregate (coarse node) of each node
    DBuf<int32_t> mem_ptr, mem;  // members of each coarse node, ascending
    // Elimination to the next level (LAMG's low-degree elimination, Sec. 3.1):
    // an independent set of this level's nodes with one or two neighbours is
    // eliminated exactly, and the next level is the Schur complement, itself
    // a Laplacian (a leaf disappears; a node between a and b becomes the
    // series edge w_a w_b / (w_a + w_b)).  With b on this level:
    //   restriction   b'(I) = b(keep_node[I]) + sum over the eliminated
    //                 neighbours u of keep_node[I] of (w_u,I / d_u) b(u)
    //   back-substitution  x(u) = b(u) / d_u + sum_m (w_um / d_u) x'(nb_m(u))
    bool w32_exact = false;      // every FP32 weight is exactly 2^-wexp times the FP64 one
    bool elim = false;
    int32_t n_elim = 0;
    DBuf<int32_t> row_of;        // [nnz] row of each entry, level 0 during setup only
    DBuf<int32_t> keep_id;       // [n] id at the next level, or -(j + 1) for eliminated node j
    DBuf<int32_t> keep_node;     // [n_next] the node of this level each next-level node is
    DBuf<int32_t> e_node;        // [n_elim] the eliminated nodes, ascending
    DBuf<int32_t> e_nb;          // [2 n_elim] their neighbours, as next-level ids (-1: none)
    DBuf<double> e_c64;          // [2 n_elim] w_um / d_u
    DBuf<float> e_c32;
    DBuf<double> e_dinv64;       // [n_elim] 1 / d_u
    DBuf<float> e_dinv32;        //          2^wexp / d_u (the FP32 operators are 2^-wexp L)
    DBuf<int32_t> pull_ptr;      // [n_next + 1] eliminated neighbours of each next-level node,
    DBuf<int32_t> pull_e;        //   as slots 2 j + m of e_nb / e_c (ascending j),
    DBuf<int32_t> pull_u;        //   the eliminated node of each slot,
    DBuf<double> pull_c64;       //   and its coefficient w_um / d_u
    DBuf<float> pull_c32;
    // level 0 only: the JL right-hand sides' own split of the rows (cfc.cu),
    // rows longer than kJlRow in chunks of kJlChunk (one thread sums a chunk)
    int32_t jl_n_chunks = 0, jl_n_long = 0;
    DBuf<int32_t> jl_chunk_row, jl_chunk_begin, jl_long_first;
    // pull lists longer than pull_long_row split into chunks of pull_chunk, as the rows of a level
    int32_t pull_long_row = 0, pull_chunk = 0;
    int32_t pull_n_chunks = 0, pull_n_long = 0;
    DBuf<int32_t> pull_chunk_row, pull_chunk_begin, pull_chunk_long, pull_long_first, pull_long_of_row;
};

constexpr int kDenseMax = 2048;  // largest coarsest level solved by a dense inverse
// Long rows are split into chunks, per level (or per set of pull lists): one
// with at most kBigLevelEntries entries splits rows longer than 32 into
// chunks of 16: its sweeps take tens of microseconds, and a 128-entry chunk
// (32 rounds of gathers by one row group) would be their critical path.  A
// larger one splits rows longer than 128 into chunks of 128, which cuts the
// chunk partials that go through DRAM.  Measured: BA 100k (1M entries) 18.9k
// RHS/s with the short chunks against 16.1k with the long ones; R-MAT 20's
// PCG level (15.6M entries) SpMV 7.0 against 13.0 ms per step, R-MAT 24's 118
// against 186.  mode (the hierarchy option `chunking`): 0 by size, 1 short,
// 2 long.
constexpr int kLongRowSmall = 32, kChunkSmall = 16;
constexpr int kLongRowBig = 128, kChunkBig = 128;
constexpr int64_t kBigLevelEntries = int64_t(1) << 22;
inline void chunk_params(int64_t entries, int mode, int32_t *long_row, int32_t *chunk) {
    const bool big = mode == 2 || (mode == 0 && entries > kBigLevelEntries);
    *long_row = big ? kLongRowBig : kLongRowSmall;
    *chunk = big ? kChunkBig : kChunkSmall;
}
constexpr int kJlRow = 32;       // the JL right-hand sides: rows with more entries are split
constexpr int kJlChunk = 32;     //   into chunks of this many (one thread each)
constexpr int kMaxTiles = 64;    // column tiles per launch (k <= 64 * 64)
constexpr int kBlock = 256;

// Device view of a level passed by value to kernels.
struct LevelView {
    int32_t n;
    const int32_t *rowptr, *col;
    const float *w32, *deg32, *dinv32;
    const uint16_t *wbf;  // BF16 weights, read by the kernels instantiated for them
    const double *w64, *deg64, *dinv64;
    int32_t n_chunks, n_long;
    int32_t long_row, chunk;  // rows longer than long_row are split into chunks of `chunk`
    const int32_t *chunk_row, *chunk_begin, *chunk_long, *long_first, *long_of_row, *order, *chunk_order;
    uint32_t *long_count;  // [n_long * kMaxTiles] arrival counters of the launching solve
};
LevelView view(const Level &L);
// The same level with BF16 weights (and the degrees of the rounded weights)
// in place of the FP32 ones; ensure_bf16 must have run on it.
LevelView view_bf16(const Level &L);
// The pull lists of an elimination level as the rows of a level (n = next
// level's size, columns = eliminated nodes of G, weights = coefficients), so
// that the restriction runs on the row kernels with their long-row chunks.
LevelView pull_view(const Level &E);

// ------------------------------------------------------------------ primitives (prims.cu)
// Exclusive prefix sum of n int32 or int64 values; returns the total.
int64_t scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
int64_t scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
// The same scan without the total: nothing waits for the device.
void scan_exclusive_i32_async(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
// The same scan with its total written to *d_total (device); nothing waits.
void scan_exclusive_i32_total(const int32_t *in, int32_t *out, int64_t n, int64_t *d_total, cudaStream_t s);
// Copies `count` int64 device values to the host with one synchronisation.
void read_totals(const int64_t *d_totals, int count, int64_t *host, cudaStream_t s);
int64_t *pinned_small();  // per-thread pinned host buffer of 64 int64
// Stable LSD radix sort of (key, value) pairs on the low `bits` key bits.
// keys/vals are sorted in place (scratch is allocated internally).
void radix_sort_pairs(uint64_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s);

// ------------------------------------------------------------------ ingest (graph.cu)
struct Csr64 {
    int32_t n = 0;
    int64_t nnz = 0;
    DBuf<int32_t> rowptr, col, eid;   // eid: undirected edge id of each entry
    DBuf<int32_t> row_of;             // row of each entry (setup only: released after the elimination)
    DBuf<double> w, deg;
    int64_t m = 0;                    // undirected edges after merging
};
// Edge list (host or device) -> symmetric CSR, merged, loop-free, with the
// connectivity check.  Throws Error on invalid input / disconnected graph.
void ingest(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const double *w,
            cudaStream_t s, Csr64 &out);

// ------------------------------------------------------------------ hierarchy (amg.cu)
void init_levels(lap_hierarchy &h, Csr64 &fine, const lap_hier_opts_t &o, cudaStream_t s);
void grow_levels(lap_hierarchy &h, int target, cudaStream_t s);  // target 0: all
int64_t build_jl_chunks(Level &L, cudaStream_t s);  // Level::jl_* of level 0; returns its rows of length 1 or 2
int effective_coarse_max(const lap_hierarchy &h);                 // the option, or its automatic value
// Makes L.wbf / degbf / dinvbf (no-op when present): each weight rounded to
// FP32 and then to BF16 (nearest, ties to even); the degrees are the FP64
// row sums of the rounded weights, rounded to FP32, so the level stays an
// exact Laplacian (null space = constants) of the rounded weights.
// wexp: the hierarchy's weight exponent; the FP32 and BF16 copies hold
// w * 2^-wexp (see lap_hierarchy::wexp)
void ensure_bf16(Level &L, int wexp, cudaStream_t s);
// FP32 copies, inverse degrees, long-row split, row order (reorder as lap_hier_opts_t)
void finish_level(Level &L, int wexp, int reorder, int chunking, cudaStream_t s);
// Exponent of the largest of n positive FP64 values (device array): the e with
// 2^e <= max < 2^(e+1).  Synchronises s.
int max_exponent(const double *v, int64_t n, cudaStream_t s);
// Order-free 64-bit fingerprint of level 0's graph (its CSR entries and
// weights: equal graphs give equal values) and max_exponent of its weights,
// in one pass (needs L.row_of) and one synchronisation of s
void fingerprint_and_exponent(const Level &L, uint64_t *fp, int *wexp, cudaStream_t s);

// dense SPD inverse (in place, FP64, row-major n x n) for the coarsest level
// and cfc_exact_small: one block in shared memory for n <= 160, else blocked
// Gauss-Jordan in one cooperative launch.  *d_flag is set (and A left
// partly updated) when a pivot is not positive.
void dense_spd_inverse_small(double *A, int n, int *d_flag, cudaStream_t s);
void dense_spd_inverse_large(double *A, int n, int *d_flag, cudaStream_t s);

}  // namespace cfc

// ------------------------------------------------------------------ handle
struct lap_hierarchy {
    int device = 0;
    int64_t n = 0, m = 0;
    std::deque<cfc::Level> lv;        // appending a level leaves the others in place
    cfc::DBuf<int32_t> eid;           // level-0 undirected edge id of each CSR entry
    lap_hier_opts_t hopts{};
    bool complete = false;            // coarsening finished (no further levels)
    std::vector<double> level_ms;     // device time to build each level (level 0: ingest)
    int32_t coarse_n = 0;             // dense coarsest size (0: none)
    cfc::DBuf<double> coarse_inv;     // (L_c + 2^wexp J/n_c)^{-1}, row-major
    cfc::DBuf<float> coarse_inv32;    // 2^wexp times it in FP32 (the FP32 modes' coarse solve)
    // Weight exponent: the largest level-0 weight lies in [2^wexp, 2^(wexp+1)).
    // The FP32 (and BF16) operators of every level are those of 2^-wexp L, an
    // exact power-of-two scaling, so that weights far from 1 (conductances of
    // any magnitude, Sec. 2) neither overflow nor fall below FP32's normal
    // range; the FP64 copies are unscaled.  0 for weights in [1, 2).
    int32_t wexp = 0;
    // fingerprint of the level-0 graph: the autotuner's choices are kept per graph
    uint64_t fingerprint = 0;
    // elimination levels in front of the cycle (lv[0 .. p0-1] have elim set):
    // the PCG and the multigrid cycle run from lv[p0]; the FP64 residual of
    // the outer refinement stays on lv[0]
    int32_t p0 = 0;
    double setup_ms = 0;
    // One solve workspace per stream, grown on demand and reused (stream
    // order keeps consecutive solves on one stream apart), so solves on
    // different streams can run on one hierarchy at the same time.
    struct Workspace {
        cfc::DBuf<char> buf;
        size_t bytes = 0;
        size_t zero_bytes = 0;  // leading bytes known to be zero (arrival counters)
    };
    std::mutex ws_mu;
    std::map<cudaStream_t, Workspace> ws;
    // exclusive while a call grows the hierarchy (lazy levels, BF16 copies) or
    // autotunes on it; shared while a solve runs on it
    mutable std::shared_mutex mu;
    cudaEvent_t grown = nullptr;  // recorded after the latest growth, on the stream that grew it
    ~lap_hierarchy() {
        if (grown) cudaEventDestroy(grown);
    }
};

namespace cfc {
// solve.cu
lap_status_t solve_multi(lap_hierarchy *h, int32_t k, const double *B, double *X,
                         const lap_solve_opts_t &o, cudaStream_t s, lap_solve_info_t *info);
lap_status_t tune_save(const char *path);
lap_status_t tune_load(const char *path, int64_t *added);
int64_t tune_entries();
lap_status_t solve_multi_direct(lap_hierarchy *h, int32_t k, const double *B, double *X, const lap_solve_opts_t &o,
                                cudaStream_t s, lap_solve_info_t *info);
int solve_ld(int32_t k, const lap_solve_opts_t &o);  // padded column count of the solver's blocks
int num_sms_public();
int32_t *pinned_scratch();  // per-thread pinned host buffer of 8192 int32
// Frees the solve workspace a hierarchy keeps for stream s (stream-ordered).
void release_workspace(lap_hierarchy *h, cudaStream_t s);
// Device bytes held by a hierarchy (levels, dense coarsest inverse), workspaces excluded.
int64_t hierarchy_bytes(const lap_hierarchy *h);
// amg.cu
// M = L + alpha J/n (dense, row-major): (L + alpha J/n)^{-1} = L^+ + J/(alpha n)
// for a connected graph; alpha of the order of the weights keeps M well scaled
void build_dense(const int32_t *rowptr, const int32_t *col, const double *w, const double *deg, int32_t n,
                 double alpha, double *M, cudaStream_t s);
// cfc.cu
// rows row0 .. row0 + k - 1 of the k_total-row Q (row0 a multiple of 32)
void jl_rhs(lap_hierarchy *h, int k_total, int row0, int k, int ld, uint64_t seed, double *Y, cudaStream_t s);
lap_status_t farness_jl(lap_hierarchy *h, int32_t k, double eps, uint64_t seed, int32_t q, const int32_t *nodes,
                        double *farness, const lap_solve_opts_t &o, cudaStream_t s);
lap_status_t farness_jl_rows(lap_hierarchy *h, int32_t k_total, int32_t row0, int32_t k, uint64_t seed, int32_t q,
                             const int32_t *nodes, double *farness, const lap_solve_opts_t &o, cudaStream_t s);
lap_status_t farness_from_solution(int64_t n, int32_t k, const double *Z, int32_t q, const int32_t *nodes,
                                   double *farness, cudaStream_t s);
// Looks up (once per device, with the device current) the address of the
// fixed scratch array of farness_from_solution_noalloc.
void noalloc_prepare();
lap_status_t farness_from_solution_noalloc(int64_t n, int32_t k, const double *Z, int32_t q, const int32_t *nodes,
                                           double *farness, cudaStream_t s);
lap_status_t pivots_api(lap_hierarchy *h, int32_t kk, uint64_t seed, int32_t *pivots, cudaStream_t s);
lap_status_t farness_sampled(lap_hierarchy *h, int32_t kk, uint64_t seed, int32_t q, const int32_t *nodes,
                             double *farness, const lap_solve_opts_t &o, cudaStream_t s, lap_solve_info_t *info = nullptr);
// A pivot set kept on the device: the kk pivots drawn as cfc_sample_pivots and
// their solutions x_s = L^+ (e_s - 1/n) (n x kk, row-major); and the sampling
// estimate of q nodes that solves only the nodes' columns against such a set.
lap_status_t pivot_solutions(lap_hierarchy *h, int32_t kk, uint64_t seed, double *XS, int32_t *piv,
                             const lap_solve_opts_t &o, cudaStream_t s, lap_solve_info_t *info);
lap_status_t farness_sampled_resident(lap_hierarchy *h, const double *XS, const int32_t *piv, int32_t kk, int32_t q,
                                      const int32_t *nodes, double *farness, const lap_solve_opts_t &o,
                                      cudaStream_t s);
// Several sampling queries as one block solve (the serving loop's batches):
// all with drawn pivots (kk > 0, kp = 0), or all on the resident pivot set
// (kk = 0; XS n x kp, piv_res).  Host nodes and outputs.
struct SampledQuery {
    int32_t kk;
    uint64_t seed;
    int32_t q;
    const int32_t *nodes;
    double *farness;
};
lap_status_t farness_sampled_batch(lap_hierarchy *h, const SampledQuery *qs, int nq, const double *XS,
                                   const int32_t *piv_res, int32_t kp, const lap_solve_opts_t &o, cudaStream_t s);
lap_status_t exact_small(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const double *w,
                         double *farness, double *closeness, cudaStream_t s);
}  // namespace cfc
