// Multigrid hierarchy of aggregation type (Sec. 3.1, Sec. 6.1: the paper's
// LAMG coarsens by elimination of low-degree nodes and by aggregation driven
// by an affinity measure; this file aggregates by parallel pairwise
// matching on the edge strength s_ij = w_ij / max(D_ii, D_jj)).
//
// Per level: a few handshake rounds of locally-dominant-edge matching (each
// unmatched node proposes its strongest unmatched neighbour; mutual
// proposals pair up), leftover nodes join the aggregate of their strongest
// matched neighbour, and `agg_passes` such passes are composed (two passes:
// aggregates of about four nodes).  With the piecewise-constant
// prolongation P of an aggregation, P^T L P is exactly the Laplacian of the
// quotient graph (edge weights between aggregates summed, edges inside an
// aggregate dropped), so the Galerkin operator is built by a sort-and-merge
// of the aggregated edge list.  The coarsest level (n_c <= coarse_max) is
// solved by the dense FP64 inverse of L_c + alpha J/n_c (alpha = 2^wexp, of
// the order of the weights), which equals L_c^+ on zero-sum vectors.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "internal.h"

struct lap_hierarchy;

namespace cfc {

namespace {

int grid_for(int64_t work, int threads = kBlock) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

int bits_for(int64_t n) {
    int b = 1;
    while ((int64_t(1) << b) < n) ++b;
    return b;
}

#define GRID_LOOP(i, count) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (count); i += (int64_t)gridDim.x * blockDim.x)

// Tie-break hash of an edge: the 64-bit finaliser of MurmurHash3 (fmix64,
// Appleby; public domain) applied to the ordered pair.
__device__ __forceinline__ uint32_t edge_hash(uint32_t a, uint32_t b) {
    // symmetric in (a, b): the same edge gets the same tie-break from both ends
    uint32_t lo = min(a, b), hi = max(a, b);
    uint64_t x = ((uint64_t)lo << 32) | hi;
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return (uint32_t)x;
}

// priority of edge (i, j): strength first, then the hash, then the smaller j
struct Cand {
    float s;
    uint32_t h;
    int32_t j;
};
__device__ __forceinline__ bool better(const Cand &a, const Cand &b) {
    if (a.j < 0) return false;
    if (b.j < 0) return true;
    if (a.s != b.s) return a.s > b.s;
    if (a.h != b.h) return a.h > b.h;
    return a.j < b.j;
}
__device__ __forceinline__ Cand warp_best(Cand c) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        Cand o{__shfl_down_sync(0xffffffffu, c.s, d), __shfl_down_sync(0xffffffffu, c.h, d),
               __shfl_down_sync(0xffffffffu, c.j, d)};
        if (better(o, c)) c = o;
    }
    return c;
}

#define WARP_ROW_LOOP(i, count)                                                              \
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < (count);       \
         i += ((int64_t)gridDim.x * blockDim.x) >> 5)

// How the pairwise matching ranks a neighbour j of node i.
//  - X null: the strength w_ij / max(D_ii, D_jj);
//  - X set: LAMG's affinity (Sec. 3.1, affinity-based aggregation) of the
//    relaxed test vectors, (X_i . X_j)^2 / ((X_i . X_i)(X_j . X_j)), in [0, 1];
//  - hub_len > 0: a node with more than hub_len neighbours stays a singleton
//    (it neither proposes, nor is proposed to, nor takes in a leftover).
constexpr int kTestVecs = 8;
struct Strength {
    const float *X;   // [n][kTestVecs], or null
    int32_t hub_len;  // 0: no hub rule
};
__device__ __forceinline__ bool is_hub(const int32_t *rowptr, int32_t i, const Strength &st) {
    return st.hub_len > 0 && rowptr[i + 1] - rowptr[i] > st.hub_len;
}
__device__ __forceinline__ float affinity(const float *X, int32_t i, int32_t j) {
    float xy = 0.f, xx = 0.f, yy = 0.f;
#pragma unroll
    for (int t = 0; t < kTestVecs; ++t) {
        const float a = __ldg(X + (size_t)i * kTestVecs + t), b = __ldg(X + (size_t)j * kTestVecs + t);
        xy = fmaf(a, b, xy);
        xx = fmaf(a, a, xx);
        yy = fmaf(b, b, yy);
    }
    return (xx > 0.f && yy > 0.f) ? (xy * xy) / (xx * yy) : 0.f;
}

// strongest neighbour of row i among those with (match[j] < 0) == want_unmatched;
// one warp per row, lanes stride over the row
__device__ __forceinline__ Cand best_neighbour(const int32_t *rowptr, const int32_t *col, const double *w,
                                               const double *deg, const int32_t *match, int32_t i,
                                               bool want_unmatched, const Strength &st) {
    const int lane = threadIdx.x & 31;
    const double di = deg[i];
    Cand b{-1.f, 0u, -1};
    for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
        const int32_t j = col[e];
        if ((match[j] < 0) != want_unmatched || is_hub(rowptr, j, st)) continue;
        const float sv = st.X ? affinity(st.X, i, j) : (float)(w[e] / fmax(di, deg[j]));
        Cand c{sv, edge_hash((uint32_t)i, (uint32_t)j), j};
        if (better(c, b)) b = c;
    }
    return warp_best(b);
}

__global__ void k_propose(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                          const double *__restrict__ w, const double *__restrict__ deg, int32_t n,
                          const int32_t *__restrict__ match, int32_t *__restrict__ prop, Strength st) {
    WARP_ROW_LOOP(i, n) {
        if (match[i] >= 0 || is_hub(rowptr, (int32_t)i, st)) {
            if ((threadIdx.x & 31) == 0) prop[i] = -1;
            continue;
        }
        const Cand b = best_neighbour(rowptr, col, w, deg, match, (int32_t)i, true, st);
        if ((threadIdx.x & 31) == 0) prop[i] = b.j;
    }
}

// Test vectors of the affinity: kTestVecs vectors with entries from a hash of
// (node, vector) in [-1, 1), then damped Jacobi sweeps on L x = 0
// (x <- (1 - omega) x + omega D^{-1} A x), which leave mostly the smooth
// components the coarse levels must represent.
__global__ void k_tv_init(int32_t n, float *__restrict__ X) {
    GRID_LOOP(t, (int64_t)n * kTestVecs) {
        uint32_t h = (uint32_t)t * 0x9E3779B1u + 0x7F4A7C15u;
        h ^= h >> 16;
        h *= 0x85ebca6bu;
        h ^= h >> 13;
        h *= 0xc2b2ae35u;
        h ^= h >> 16;
        X[t] = (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;
    }
}

// one warp per row: lanes over the neighbours, a fixed shuffle tree per vector
__global__ void k_tv_relax(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                          const double *__restrict__ w, const double *__restrict__ deg, int32_t n,
                          const float *__restrict__ X, float *__restrict__ Xn, float omega) {
    const int lane = threadIdx.x & 31;
    WARP_ROW_LOOP(i, n) {
        float acc[kTestVecs];
#pragma unroll
        for (int t = 0; t < kTestVecs; ++t) acc[t] = 0.f;
        for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
            const float we = (float)w[e];
            const int32_t j = col[e];
#pragma unroll
            for (int t = 0; t < kTestVecs; ++t) acc[t] = fmaf(we, X[(size_t)j * kTestVecs + t], acc[t]);
        }
#pragma unroll
        for (int t = 0; t < kTestVecs; ++t)
            for (int o = 16; o > 0; o >>= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
        if (lane < kTestVecs) {
            float a = acc[0];
#pragma unroll
            for (int t = 1; t < kTestVecs; ++t)
                if (lane == t) a = acc[t];
            const float di = (float)(1.0 / deg[i]);
            Xn[(size_t)i * kTestVecs + lane] = (1.f - omega) * X[(size_t)i * kTestVecs + lane] + omega * di * a;
        }
    }
}

__global__ void k_accept(const int32_t *__restrict__ prop, int32_t n, int32_t *__restrict__ match) {
    GRID_LOOP(i, n) {
        const int32_t j = prop[i];
        if (j >= 0 && prop[j] == (int32_t)i) match[i] = j;
    }
}

// leader of each node's aggregate: min of a matched pair; a leftover joins
// its strongest matched neighbour's pair; otherwise it stays alone
__global__ void k_leaders(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                          const double *__restrict__ w, const double *__restrict__ deg, int32_t n,
                          const int32_t *__restrict__ match, int32_t *__restrict__ leader,
                          int32_t *__restrict__ is_leader, Strength st) {
    WARP_ROW_LOOP(i, n) {
        const int32_t mi = match[i];
        int32_t l;
        if (mi >= 0) {
            l = min((int32_t)i, mi);
        } else if (is_hub(rowptr, (int32_t)i, st)) {
            l = (int32_t)i;  // a hub stays a singleton
        } else {
            const Cand b = best_neighbour(rowptr, col, w, deg, match, (int32_t)i, false, st);
            l = b.j >= 0 ? min(b.j, match[b.j]) : (int32_t)i;
        }
        if ((threadIdx.x & 31) == 0) {
            leader[i] = l;
            is_leader[i] = (l == (int32_t)i) ? 1 : 0;
        }
    }
}

__global__ void k_assign(const int32_t *__restrict__ leader, const int32_t *__restrict__ lid, int32_t n,
                         int32_t *__restrict__ agg) {
    GRID_LOOP(i, n) agg[i] = lid[leader[i]];
}

__global__ void k_compose(int32_t *__restrict__ agg, const int32_t *__restrict__ agg2, int32_t n) {
    GRID_LOOP(i, n) agg[i] = agg2[agg[i]];
}

// Galerkin: flags of fine entries that cross aggregates
__global__ void k_cross_flags(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, int32_t n,
                              const int32_t *__restrict__ agg, int32_t *__restrict__ flag) {
    const int lane = threadIdx.x & 31;
    WARP_ROW_LOOP(i, n) {
        const int32_t I = agg[i];
        for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) flag[e] = (agg[col[e]] != I) ? 1 : 0;
    }
}

__global__ void k_cross_emit(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, int32_t n,
                             const int32_t *__restrict__ agg, const int32_t *__restrict__ flag,
                             const int32_t *__restrict__ pos, int b, uint64_t *__restrict__ keys,
                             uint32_t *__restrict__ vals) {
    const int lane = threadIdx.x & 31;
    WARP_ROW_LOOP(i, n) {
        const uint64_t I = (uint32_t)agg[i];
        for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
            if (!flag[e]) continue;
            keys[pos[e]] = (I << b) | (uint32_t)agg[col[e]];
            vals[pos[e]] = (uint32_t)e;
        }
    }
}

__global__ void k_heads(const uint64_t *__restrict__ keys, int64_t len, int32_t *__restrict__ head) {
    GRID_LOOP(i, len) head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_merge(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                        const int32_t *__restrict__ head, const int32_t *__restrict__ hpos, int64_t len, int b,
                        const double *__restrict__ w, int32_t *__restrict__ col, double *__restrict__ wout,
                        int32_t *__restrict__ rowcnt) {
    GRID_LOOP(i, len) {
        if (!head[i]) continue;
        const uint64_t key = keys[i];
        double s = 0.0;
        for (int64_t j = i; j < len && keys[j] == key; ++j) s += w[vals[j]];
        const int32_t o = hpos[i];
        col[o] = (int32_t)(key & ((uint64_t(1) << b) - 1));
        wout[o] = s;
        atomicAdd(&rowcnt[key >> b], 1);
    }
}

__global__ void k_set_last(int32_t *p, int32_t idx, int32_t v) {
    if (blockIdx.x == 0 && threadIdx.x == 0) p[idx] = v;
}

// D_ii = sum_j w_ij in CSR order: one thread per row of at most 32 entries
// (most rows), one warp per longer row (lane-strided sums + a fixed tree);
// both orders are fixed, so the sums are reproducible
__global__ void k_row_sums_short(const int32_t *__restrict__ rowptr, const double *__restrict__ w, int32_t n,
                                 double *__restrict__ deg) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int e0 = rowptr[r], e1 = rowptr[r + 1];
        if (e1 - e0 > 32) continue;
        double s = 0.0;
        for (int e = e0; e < e1; ++e) s += w[e];
        deg[r] = s;
    }
}
__global__ void k_row_sums_long(const int32_t *__restrict__ rowptr, const double *__restrict__ w, int32_t n,
                                double *__restrict__ deg) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int e0 = rowptr[r], e1 = rowptr[r + 1];
        if (e1 - e0 <= 32) continue;
        double s = 0.0;
        for (int e = e0 + lane; e < e1; e += 32) s += w[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) deg[r] = s;
    }
}

__global__ void k_iota_keys(const int32_t *__restrict__ agg, int32_t n, uint64_t *__restrict__ keys,
                            uint32_t *__restrict__ vals, int32_t *__restrict__ cnt) {
    GRID_LOOP(i, n) {
        keys[i] = (uint32_t)agg[i];
        vals[i] = (uint32_t)i;
        atomicAdd(&cnt[agg[i]], 1);
    }
}

__global__ void k_u32_to_i32(const uint32_t *__restrict__ a, int32_t *__restrict__ b, int32_t n) {
    GRID_LOOP(i, n) b[i] = (int32_t)a[i];
}

// FP32 copies of 2^-wexp times the weights and degrees (an exact power-of-two
// scaling, see lap_hierarchy::wexp), inverse degrees, long-row flags.  An
// inverse degree beyond FP32's range (a degree that underflows after the
// scaling) is stored as 0: the smoother then leaves that node alone instead
// of producing infinities.
__global__ void k_finish(const int32_t *__restrict__ rowptr, const double *__restrict__ w64,
                         const double *__restrict__ deg64, int32_t n, int64_t nnz, double sc,
                         float *__restrict__ w32, float *__restrict__ deg32, float *__restrict__ dinv32,
                         double *__restrict__ dinv64, int32_t *__restrict__ nchunk,
                         unsigned long long *__restrict__ inexact, int long_row, int chunk) {
    // inexact: set when some FP32 weight is not exactly the scaled FP64 one
    bool bad = false;
    GRID_LOOP(e, nnz) {
        const double x = w64[e] * sc;
        const float f = (float)x;
        w32[e] = f;
        bad = bad || ((double)f != x);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(inexact, 1ull);
    GRID_LOOP(i, n) {
        const double d = deg64[i];
        const double ds = d * sc;
        deg32[i] = (float)ds;
        const double di = 1.0 / ds;
        dinv32[i] = (deg32[i] > 0.f && di <= 3.0e38) ? (float)di : 0.f;
        dinv64[i] = 1.0 / d;
        const int len = rowptr[i + 1] - rowptr[i];
        nchunk[i] = len > long_row ? (len + chunk - 1) / chunk : 0;
    }
}

// Order-free fingerprint of a level's graph: the sum (mod 2^64) over its CSR
// entries of the MurmurHash3 finaliser (fmix64) of (row, column) mixed with
// the weight's bit pattern.  Integer sums commute, so the value does not
// depend on scheduling.
__device__ __forceinline__ unsigned long long fmix64(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// The fingerprint's sum and the largest weight's bit pattern in one pass over
// the entries, one thread each (the row of each entry from row_of)
__global__ void k_fingerprint_flat(const int32_t *__restrict__ row_of, const int32_t *__restrict__ col,
                                   const double *__restrict__ w, int64_t nnz, unsigned long long *__restrict__ out) {
    unsigned long long acc = 0, m = 0;
    GRID_LOOP(e, nnz) {
        const unsigned long long wb = (unsigned long long)__double_as_longlong(w[e]);
        const unsigned long long rc = ((unsigned long long)(uint32_t)row_of[e] << 32) | (uint32_t)col[e];
        acc += fmix64(rc ^ fmix64(wb));
        m = wb > m ? wb : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_down_sync(0xffffffffu, acc, o);
        const unsigned long long t = __shfl_down_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0) {
        if (acc) atomicAdd(out, acc);
        if (m) atomicMax(out + 1, m);
    }
}

// largest of n positive doubles: positive doubles order like their bit
// patterns read as unsigned integers
__global__ void k_max_bits(const double *__restrict__ v, int64_t n, unsigned long long *__restrict__ out) {
    unsigned long long m = 0;
    GRID_LOOP(i, n) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v[i]);
        m = b > m ? b : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_down_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// thread per row: round the row's weights to BF16 (via FP32) and sum the
// rounded values in FP64, in CSR order
__global__ void k_bf16_level(const int32_t *__restrict__ rowptr, const double *__restrict__ w64, int32_t n,
                             double sc, uint16_t *__restrict__ wbf, float *__restrict__ degbf,
                             float *__restrict__ dinvbf) {
    GRID_LOOP(i, n) {
        double d = 0.0;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const uint16_t b = __bfloat16_as_ushort(__float2bfloat16_rn((float)(w64[e] * sc)));
            wbf[e] = b;
            d += (double)__uint_as_float((uint32_t)b << 16);
        }
        const float df = (float)d;
        degbf[i] = df;
        dinvbf[i] = (df > 0.f && 1.0 / d <= 3.0e38) ? 1.0f / df : 0.f;
    }
}

// gather rounds of the row kernels (4 neighbours per round, rows up to
// long_row) in the natural order, four rows sharing a warp: [0] the sum over
// warps of their longest row's rounds, [1] the sum over rows of their rounds
__global__ void k_order_stats(const int32_t *__restrict__ rowptr, int32_t n, int long_row,
                              unsigned long long *__restrict__ out) {
    unsigned long long wmax = 0, rsum = 0;
    GRID_LOOP(w, ((int64_t)n + 3) / 4) {
        unsigned long long m = 0;
        for (int j = 0; j < 4; ++j) {
            const int64_t i = 4 * w + j;
            if (i >= n) break;
            const int len = min(rowptr[i + 1] - rowptr[i], long_row + 1);
            const unsigned long long rounds = (unsigned long long)((len + 3) / 4);
            m = rounds > m ? rounds : m;
            rsum += rounds;
        }
        wmax += m;
    }
    for (int o = 16; o > 0; o >>= 1) {  // one atomic per warp, not per thread
        wmax += __shfl_down_sync(0xffffffffu, wmax, o);
        rsum += __shfl_down_sync(0xffffffffu, rsum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, wmax);
        atomicAdd(out + 1, rsum);
    }
}

// sort key of a row for the processing order: shorter rows later, rows longer
// than long_row first, equal lengths in row order
__global__ void k_order_keys(const int32_t *__restrict__ rowptr, int32_t n, int long_row,
                             uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    GRID_LOOP(i, n) {
        const int len = rowptr[i + 1] - rowptr[i];
        keys[i] = (uint64_t)(long_row + 1 - min(len, long_row + 1));
        vals[i] = (uint32_t)i;
    }
}

// sort key of a chunk for its processing order: the column of its first entry
__global__ void k_chunk_keys(const int32_t *__restrict__ col, const int32_t *__restrict__ chunk_begin, int32_t n_chunks,
                             uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    GRID_LOOP(c, n_chunks) {
        keys[c] = (uint32_t)col[chunk_begin[c]];
        vals[c] = (uint32_t)c;
    }
}

// chunks of each row of (rowptr, n): rows longer than long_row take ceil(len / chunk)
__global__ void k_nchunk(const int32_t *__restrict__ rowptr, int32_t n, int long_row, int chunk,
                         int32_t *__restrict__ nchunk) {
    GRID_LOOP(i, n) {
        const int len = rowptr[i + 1] - rowptr[i];
        nchunk[i] = len > long_row ? (len + chunk - 1) / chunk : 0;
    }
}

// the JL split of level 0's rows: chunks per row, then each chunk's row and
// start; also counts the rows with one or two entries (the candidates of the
// low-degree elimination) into *low
__global__ void k_jl_nchunk(const int32_t *__restrict__ rowptr, int32_t n, int32_t *__restrict__ nchunk,
                            unsigned long long *__restrict__ low) {
    unsigned long long c = 0;
    GRID_LOOP(i, n) {
        const int len = rowptr[i + 1] - rowptr[i];
        nchunk[i] = len > kJlRow ? (len + kJlChunk - 1) / kJlChunk : 0;
        c += (len >= 1 && len <= 2) ? 1ull : 0ull;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(low, c);
}
__global__ void k_jl_fill(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ nchunk,
                          const int32_t *__restrict__ cfirst, const int32_t *__restrict__ lidx, int32_t n,
                          int32_t *__restrict__ chunk_row, int32_t *__restrict__ chunk_begin,
                          int32_t *__restrict__ long_first) {
    GRID_LOOP(i, n) {
        const int c = nchunk[i];
        if (!c) continue;
        const int f = cfirst[i];
        long_first[lidx[i]] = f;
        for (int t = 0; t < c; ++t) {
            chunk_row[f + t] = (int32_t)i;
            chunk_begin[f + t] = rowptr[i] + t * kJlChunk;
        }
    }
}

__global__ void k_long_index(const int32_t *__restrict__ nchunk, int32_t n, int32_t *__restrict__ is_long) {
    GRID_LOOP(i, n) is_long[i] = nchunk[i] > 0 ? 1 : 0;
}

__global__ void k_fill_chunks(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ nchunk,
                              const int32_t *__restrict__ cfirst, const int32_t *__restrict__ lidx, int32_t n,
                              int chunk,
                              int32_t *__restrict__ chunk_row, int32_t *__restrict__ chunk_begin,
                              int32_t *__restrict__ chunk_long, int32_t *__restrict__ long_first,
                              int32_t *__restrict__ long_of_row) {
    GRID_LOOP(i, n) {
        const int c = nchunk[i];
        long_of_row[i] = c ? lidx[i] : -1;
        if (!c) continue;
        const int f = cfirst[i], l = lidx[i];
        long_first[l] = f;
        for (int t = 0; t < c; ++t) {
            chunk_row[f + t] = (int32_t)i;
            chunk_begin[f + t] = rowptr[i] + t * chunk;
            chunk_long[f + t] = l;
        }
    }
}

// FP32 copy of 2^e times an FP64 array (the scaled coarse inverse)
__global__ void k_scaled_f32(const double *__restrict__ src, int64_t count, int e, float *__restrict__ dst) {
    GRID_LOOP(t, count) dst[t] = (float)ldexp(src[t], e);
}

// dense M = L_c + J/n_c
__global__ void k_fill(double *__restrict__ M, int64_t count, double v) {
    GRID_LOOP(t, count) M[t] = v;
}

__global__ void k_dense_scatter(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                const double *__restrict__ w, const double *__restrict__ deg, int32_t n,
                                double *__restrict__ M) {
    GRID_LOOP(i, n) {
        M[i * (int64_t)n + i] += deg[i];
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) M[i * (int64_t)n + col[e]] -= w[e];
    }
}

// In-place Gauss-Jordan inversion of an SPD matrix (no pivoting needed),
// whole matrix in shared memory, one CTA.  Step k: scale row k by 1/a_kk
// with the identity column stored in place, then eliminate column k from
// every other row.  A pivot <= 0 flags a singular (disconnected) matrix.
__global__ void __launch_bounds__(1024) k_gj_smem(double *__restrict__ A, int n, int *__restrict__ flag) {
    extern __shared__ double sm[];
    double *a = sm;           // n*n
    double *fc = sm + n * n;  // column k saved
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) a[t] = A[t];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const double akk = a[k * n + k];
        if (!(akk > 0.0)) {
            if (threadIdx.x == 0) atomicOr(flag, 1);
            return;
        }
        const double piv = 1.0 / akk;
        for (int i = threadIdx.x; i < n; i += blockDim.x) fc[i] = a[i * n + k];
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) a[k * n + j] = (j == k ? 1.0 : a[k * n + j]) * piv;
        __syncthreads();
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int i = t / n, j = t - (t / n) * n;
            if (i == k) continue;
            const double cur = (j == k) ? 0.0 : a[t];
            a[t] = cur - fc[i] * a[k * n + j];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[t] = a[t];
}

// Blocked Gauss-Jordan in global memory, one cooperative launch.  The
// pivots are taken kGjB at a time; with K the block's index range, P = A[K,K],
// C = A[:,K] (before the step) and R = P^-1 A[K,:], one block step sets
//   A[K,K] = P^-1,  A[K,J] = R[:,J],  A[I,K] = -C[I,:] P^-1,
//   A[I,J] -= C[I,:] R[:,J]                      (I, J outside K),
// which is kGjB single-pivot Gauss-Jordan steps at once.  Each step has three
// phases separated by grid barriers: (A) one warp inverts P in registers
// while all blocks copy C; (B) R; (C) the update in 64 x 64 tiles.  The
// matrix is SPD, so every pivot is positive in exact arithmetic; a pivot that
// is not (lost definiteness in floating point, or NaN) sets *flag, and every
// block reads the flag after the next barrier and returns with the others.
constexpr int kGjB = 32;
constexpr int kGjTile = 64;
static_assert(kBlock == 256, "k_gj_blocked maps 256 threads to 16 x 16 groups of 4 x 4 outputs");

__global__ void __launch_bounds__(256) k_gj_blocked(double *__restrict__ A, int n, double *__restrict__ Pinv,
                                                    double *__restrict__ Cold, double *__restrict__ Rnew,
                                                    int *__restrict__ flag) {
    namespace cg = cooperative_groups;
    cg::grid_group g = cg::this_grid();
    __shared__ double Cs[kGjTile][kGjB + 1];
    __shared__ double Rs[kGjB][kGjTile];
    double(*Ps)[kGjB + 1] = Cs;  // phase B reuses the tile buffer for P^-1
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t gt = (int64_t)g.thread_rank(), gn = (int64_t)g.size();
    const int nb = (n + kGjB - 1) / kGjB;
    const int td = (n + kGjTile - 1) / kGjTile;
    for (int kb = 0; kb < nb; ++kb) {
        const int k0 = kb * kGjB, bk = min(kGjB, n - k0);
        // ---- A: P^-1 by warp 0 of block 0 (lane j holds column j; P padded with
        // the identity beyond bk), and C = A[:, K] by everyone
        if (blockIdx.x == 0 && tid < 32) {
            double p[kGjB];
#pragma unroll
            for (int i = 0; i < kGjB; ++i)
                p[i] = (i < bk && lane < bk) ? A[(size_t)(k0 + i) * n + k0 + lane] : (i == lane ? 1.0 : 0.0);
            bool ok = true;
#pragma unroll
            for (int q = 0; q < kGjB; ++q) {
                const double akk = __shfl_sync(0xffffffffu, p[q], q);
                ok = ok && (akk > 0.0);
                const double inv = 1.0 / akk;
                const double rowq = (lane == q ? 1.0 : p[q]) * inv;
#pragma unroll
                for (int i = 0; i < kGjB; ++i) {
                    if (i == q) continue;
                    const double ciq = __shfl_sync(0xffffffffu, p[i], q);
                    p[i] = (lane == q ? 0.0 : p[i]) - ciq * rowq;
                }
                p[q] = rowq;
            }
            if (!ok) {
                if (lane == 0) atomicOr(flag, 1);
            } else {
#pragma unroll
                for (int i = 0; i < kGjB; ++i) Pinv[i * kGjB + lane] = p[i];
            }
        }
        for (int64_t t = gt; t < (int64_t)n * kGjB; t += gn) {
            const int64_t i = t / kGjB;
            const int b = (int)(t - i * kGjB);
            Cold[t] = b < bk ? A[(size_t)i * n + k0 + b] : 0.0;
        }
        g.sync();
        if (*(volatile int *)flag) return;  // the same value in every block
        // ---- B: R = P^-1 A[K, :] (on K's own columns: P^-1 itself)
        for (int t = tid; t < kGjB * kGjB; t += blockDim.x) Ps[t / kGjB][t % kGjB] = Pinv[t];
        __syncthreads();
        for (int64_t j = gt; j < n; j += gn) {
            if (j >= k0 && j < k0 + bk) {
#pragma unroll 4
                for (int b = 0; b < kGjB; ++b) Rnew[(size_t)b * n + j] = Ps[b][j - k0];
            } else {
                double a[kGjB];
#pragma unroll
                for (int c = 0; c < kGjB; ++c) a[c] = c < bk ? A[(size_t)(k0 + c) * n + j] : 0.0;
#pragma unroll 4
                for (int b = 0; b < kGjB; ++b) {
                    double v = 0.0;
#pragma unroll
                    for (int c = 0; c < kGjB; ++c) v = fma(Ps[b][c], a[c], v);
                    Rnew[(size_t)b * n + j] = v;
                }
            }
        }
        g.sync();
        // ---- C: the update, 64 x 64 tiles, 4 x 4 outputs per thread
        const int ty = tid / 16, tx = tid % 16;
        for (int tile = blockIdx.x; tile < td * td; tile += gridDim.x) {
            const int i0 = (tile / td) * kGjTile, j0 = (tile % td) * kGjTile;
            __syncthreads();
            for (int t = tid; t < kGjTile * kGjB; t += blockDim.x) {
                const int r = t / kGjB, b = t % kGjB;
                Cs[r][b] = i0 + r < n ? Cold[(size_t)(i0 + r) * kGjB + b] : 0.0;
            }
            for (int t = tid; t < kGjB * kGjTile; t += blockDim.x) {
                const int b = t / kGjTile, c = t % kGjTile;
                Rs[b][c] = j0 + c < n ? Rnew[(size_t)b * n + j0 + c] : 0.0;
            }
            __syncthreads();
            double acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
#pragma unroll 8
            for (int b = 0; b < kGjB; ++b) {
                double cv[4], rv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) cv[u] = Cs[ty + 16 * u][b];
#pragma unroll
                for (int v = 0; v < 4; ++v) rv[v] = Rs[b][tx + 16 * v];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fma(cv[u], rv[v], acc[u][v]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + ty + 16 * u;
                if (i >= n) continue;
                const bool iK = i >= k0 && i < k0 + bk;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int j = j0 + tx + 16 * v;
                    if (j >= n) continue;
                    double *aij = A + (size_t)i * n + j;
                    if (iK) {
                        *aij = Rs[i - k0][tx + 16 * v];
                    } else {
                        const bool jK = j >= k0 && j < k0 + bk;
                        *aij = (jK ? 0.0 : *aij) - acc[u][v];
                    }
                }
            }
        }
        g.sync();
    }
}

struct Graph64 {
    int32_t n = 0;
    int64_t nnz = 0;
    DBuf<int32_t> rowptr, col;
    DBuf<double> w, deg;
};

// kTestVecs relaxed test vectors of the graph (rowptr, col, w, deg): hashed
// start, kTvSweeps damped Jacobi sweeps with omega = 0.7
constexpr int kTvSweeps = 4;
DBuf<float> test_vectors(const int32_t *rowptr, const int32_t *col, const double *w, const double *deg, int32_t n,
                         cudaStream_t s) {
    DBuf<float> X((size_t)n * kTestVecs, s), Y((size_t)n * kTestVecs, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_tv_init, grid_for((int64_t)n * kTestVecs), kBlock, 0, n, X.get());
    for (int t = 0; t < kTvSweeps; ++t) {
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_tv_relax, grid_for(32 * (int64_t)n), kBlock, 0, rowptr, col, w, deg, n,
                   X.get(), Y.get(), 0.7f);
        std::swap(X, Y);
    }
    return X;
}

// one pairwise-matching pass: agg[n], returns the number of aggregates.
// aggregation: LAP_AGG_STRENGTH or LAP_AGG_AFFINITY; hub_factor > 0: nodes
// with more than hub_factor x the mean row length stay singletons.
int32_t pairwise_pass(const int32_t *rowptr, const int32_t *col, const double *w, const double *deg, int32_t n,
                      int64_t nnz, int rounds, int aggregation, int hub_factor, int32_t *agg, cudaStream_t s) {
    DBuf<int32_t> match(n, s), prop(n, s), leader(n, s), isl(n, s), lid(n, s);
    DBuf<float> X;
    Strength st{nullptr, 0};
    if (hub_factor > 0 && n > 0) {
        const double len = (double)hub_factor * (double)nnz / (double)n;
        st.hub_len = (int32_t)std::min<double>(std::max(1.0, std::ceil(len)), 2e9);
    }
    if (aggregation == LAP_AGG_AFFINITY && n > 0) {
        X = test_vectors(rowptr, col, w, deg, n, s);
        st.X = X.get();
    }
    CFC_CUDA(cudaMemsetAsync(match.get(), 0xff, n * sizeof(int32_t), s));
    for (int r = 0; r < rounds; ++r) {
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_propose, grid_for(32 * (int64_t)n), kBlock, 0, rowptr, col, w, deg, n,
                   match.get(), prop.get(), st);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_accept, grid_for(n), kBlock, 0, prop.get(), n, match.get());
    }
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_leaders, grid_for(32 * (int64_t)n), kBlock, 0, rowptr, col, w, deg, n,
               match.get(), leader.get(), isl.get(), st);
    const int64_t nc = scan_exclusive_i32(isl.get(), lid.get(), n, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_assign, grid_for(n), kBlock, 0, leader.get(), lid.get(), n, agg);
    return (int32_t)nc;
}

// quotient graph of (rowptr, col, w) under agg (nc aggregates)
void contract(const int32_t *rowptr, const int32_t *col, const double *w, int32_t n, int64_t nnz,
              const int32_t *agg, int32_t nc, bool persistent, Graph64 &out, cudaStream_t s) {
    DBuf<int32_t> flag(nnz, s), pos(nnz, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_cross_flags, grid_for(32 * (int64_t)n), kBlock, 0, rowptr, col, n, agg,
               flag.get());
    const int64_t len = scan_exclusive_i32(flag.get(), pos.get(), nnz, s);
    const int b = bits_for(nc);
    out.n = nc;
    auto alloc_i = [&](DBuf<int32_t> &d, size_t c) { persistent ? d.alloc_persistent(c) : d.alloc(c, s); };
    auto alloc_d = [&](DBuf<double> &d, size_t c) { persistent ? d.alloc_persistent(c) : d.alloc(c, s); };
    alloc_i(out.rowptr, nc + 1);
    alloc_d(out.deg, nc);
    DBuf<int32_t> rowcnt(nc + 1, s);
    rowcnt.zero(s);
    if (len == 0) {
        out.nnz = 0;
        alloc_i(out.col, 1);
        alloc_d(out.w, 1);
        CFC_CUDA(cudaMemsetAsync(out.rowptr.get(), 0, (nc + 1) * sizeof(int32_t), s));
        CFC_CUDA(cudaMemsetAsync(out.deg.get(), 0, nc * sizeof(double), s));
        return;
    }
    DBuf<uint64_t> keys(len, s);
    DBuf<uint32_t> vals(len, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_cross_emit, grid_for(32 * (int64_t)n), kBlock, 0, rowptr, col, n, agg,
               flag.get(), pos.get(), b, keys.get(), vals.get());
    flag.release();
    pos.release();
    radix_sort_pairs(keys.get(), vals.get(), len, 2 * b, s);
    DBuf<int32_t> head(len, s), hpos(len, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_heads, grid_for(len), kBlock, 0, keys.get(), len, head.get());
    const int64_t cnnz = scan_exclusive_i32(head.get(), hpos.get(), len, s);
    out.nnz = cnnz;
    alloc_i(out.col, cnnz);
    alloc_d(out.w, cnnz);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_merge, grid_for(len), kBlock, 0, keys.get(), vals.get(), head.get(),
               hpos.get(), len, b, w, out.col.get(), out.w.get(), rowcnt.get());
    scan_exclusive_i32(rowcnt.get(), out.rowptr.get(), nc, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_set_last, 1, 1, 0, out.rowptr.get(), nc, (int32_t)cnnz);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_row_sums_short, grid_for(nc), kBlock, 0,
               out.rowptr.get(), out.w.get(), nc, out.deg.get());
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_row_sums_long, grid_for(32 * (int64_t)nc), kBlock, 0,
               out.rowptr.get(), out.w.get(), nc, out.deg.get());
}

// ---------------------------------------------------------------- low-degree elimination
// Candidates are the nodes with one or two neighbours; they are picked in an
// independent set by Luby-style rounds on the key (neighbour count, fmix32 of
// the id) -- MurmurHash3's 32-bit finaliser, a bijection, so the tie-break
// is unrelated to the labelling and never ties.  State: 0 undecided
// candidate, 1 eliminated, 2 kept.  A round eliminates every undecided
// candidate with no undecided neighbour of smaller key and keeps every
// undecided candidate next to an eliminated node; nodes still undecided after
// the last round are kept.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
__device__ __forceinline__ uint64_t elim_key(const int32_t *rowptr, int32_t i) {
    return ((uint64_t)(rowptr[i + 1] - rowptr[i]) << 32) | fmix32((uint32_t)i);
}

__global__ void k_elim_init(const int32_t *__restrict__ rowptr, int32_t n, int32_t *__restrict__ state) {
    GRID_LOOP(i, n) {
        const int c = rowptr[i + 1] - rowptr[i];
        state[i] = (c >= 1 && c <= 2) ? 0 : 2;
    }
}

__global__ void k_elim_round(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, int32_t n,
                             const int32_t *__restrict__ st, int32_t *__restrict__ st_next) {
    GRID_LOOP(i, n) {
        int v = st[i];
        if (v == 0) {
            const uint64_t ki = elim_key(rowptr, (int32_t)i);
            bool blocked = false, smaller = false;
            for (int t = rowptr[i]; t < rowptr[i + 1]; ++t) {
                const int j = col[t];
                const int sj = st[j];
                blocked |= (sj == 1);
                smaller |= (sj == 0 && elim_key(rowptr, j) < ki);
            }
            v = blocked ? 2 : (smaller ? 0 : 1);
        }
        st_next[i] = v;
    }
}

__global__ void k_elim_flags(const int32_t *__restrict__ st, int32_t n, int32_t *__restrict__ elim,
                             int32_t *__restrict__ keep) {
    GRID_LOOP(i, n) {
        const int e = st[i] == 1 ? 1 : 0;
        elim[i] = e;
        keep[i] = 1 - e;
    }
}

// ids at the next level, the eliminated nodes' neighbours and coefficients,
// and the series weight w_a w_b / d_u of each eliminated node with two
// neighbours (its fill edge)
__global__ void k_elim_tables(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                              const double *__restrict__ w, const double *__restrict__ deg, int32_t n,
                              const int32_t *__restrict__ elim, const int32_t *__restrict__ eidx,
                              const int32_t *__restrict__ kidx, double sc, int32_t *__restrict__ keep_id,
                              int32_t *__restrict__ keep_node, int32_t *__restrict__ e_node,
                              int32_t *__restrict__ e_nb, double *__restrict__ e_c64, float *__restrict__ e_c32,
                              double *__restrict__ e_dinv64, float *__restrict__ e_dinv32,
                              int32_t *__restrict__ fill_cnt, int32_t *__restrict__ pull_cnt,
                              double *__restrict__ fill_w) {
    GRID_LOOP(i, n) {
        if (!elim[i]) {
            keep_id[i] = kidx[i];
            keep_node[kidx[i]] = (int32_t)i;
            continue;
        }
        const int j = eidx[i];
        keep_id[i] = -(j + 1);
        e_node[j] = (int32_t)i;
        const double d = deg[i];
        const int e0 = rowptr[i], cnt = rowptr[i + 1] - e0;
        for (int m = 0; m < 2; ++m) {
            const bool has = m < cnt;
            e_nb[2 * j + m] = has ? kidx[col[e0 + m]] : -1;  // neighbours are kept (independent set)
            e_c64[2 * j + m] = has ? w[e0 + m] / d : 0.0;
            e_c32[2 * j + m] = has ? (float)(w[e0 + m] / d) : 0.f;
        }
        e_dinv64[j] = 1.0 / d;
        const double di = 1.0 / (d * sc);
        e_dinv32[j] = di <= 3.0e38 ? (float)di : 0.f;
        fill_cnt[j] = cnt == 2 ? 2 : 0;
        pull_cnt[j] = cnt;
        fill_w[j] = cnt == 2 ? w[e0] * w[e0 + 1] / d : 0.0;
    }
}

// entries of the next level between two kept nodes: a flag per entry, and
// the entry's column at the next level (keep_id is read once per entry)
// per entry of G (one thread each): kept at the next level when both ends are
// kept, and its column's next-level id
__global__ void k_keep_flags(const int32_t *__restrict__ row_of, const int32_t *__restrict__ col, int64_t nnz,
                             const int32_t *__restrict__ keep_id, int32_t *__restrict__ flag,
                             int32_t *__restrict__ newcol) {
    GRID_LOOP(e, nnz) {
        const int32_t c = keep_id[col[e]];
        flag[e] = (keep_id[row_of[e]] >= 0 && c >= 0) ? 1 : 0;
        newcol[e] = c;
    }
}

// both directions of each fill edge as (row << b | col) keys at base + fpos[j],
// their weights in wv
__global__ void k_elim_emit_fill(const int32_t *__restrict__ e_nb, const int32_t *__restrict__ fill_cnt,
                                 const int32_t *__restrict__ fpos, const double *__restrict__ fill_w, int32_t n_elim,
                                 int64_t base, int b, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                 double *__restrict__ wv) {
    GRID_LOOP(j, n_elim) {
        if (!fill_cnt[j]) continue;
        const uint64_t a = (uint32_t)e_nb[2 * j], c = (uint32_t)e_nb[2 * j + 1];
        const int64_t p = base + fpos[j];
        keys[p] = (a << b) | c;
        keys[p + 1] = (c << b) | a;
        vals[p] = (uint32_t)p;
        vals[p + 1] = (uint32_t)(p + 1);
        wv[p] = fill_w[j];
        wv[p + 1] = fill_w[j];
    }
}

// The next level's rows without a global sort.  Old-to-new ids are
// monotone, so the entries between two kept nodes, taken in CSR order, are
// already sorted by (new row, new column): they are compacted (kcol, kw) and
// each new row's run starts at kstart.  The fill edges (few) are sorted on
// their own and merged with equal fills summed (ucol, uw, rows at fptr); then
// each row's fills are merged into its kept run: a fill whose column the row
// already has adds its weight there, the others are inserted in order.
__global__ void k_elim_compact(const int32_t *__restrict__ row_of, const double *__restrict__ w, int64_t nnz,
                               const int32_t *__restrict__ kidx, const int32_t *__restrict__ flag,
                               const int32_t *__restrict__ pos, const int32_t *__restrict__ newcol,
                               int32_t *__restrict__ kcol, double *__restrict__ kw, int32_t *__restrict__ krow) {
    GRID_LOOP(e, nnz) {
        if (!flag[e]) continue;
        const int32_t p = pos[e];
        kcol[p] = newcol[e];
        kw[p] = w[e];
        krow[p] = kidx[row_of[e]];
    }
}

// where each next-level row's kept entries start (every row of G has an entry)
__global__ void k_elim_kstart(const int32_t *__restrict__ rowptr, int32_t n, const int32_t *__restrict__ elim,
                              const int32_t *__restrict__ kidx, const int32_t *__restrict__ pos,
                              int32_t *__restrict__ kstart) {
    GRID_LOOP(i, n) {
        if (!elim[i]) kstart[kidx[i]] = pos[rowptr[i]];
    }
}

// first index in a[lo, hi) with a[idx] >= x
__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int lo, int hi, int32_t x) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// per fill: 1 when its column is not among the row's kept entries (inserted)
__global__ void k_elim_fill_new(const int32_t *__restrict__ kcol, const int32_t *__restrict__ kstart,
                                const int32_t *__restrict__ ucol, const int32_t *__restrict__ fptr, int32_t nk,
                                int32_t *__restrict__ fnew) {
    const int lane = threadIdx.x & 31;
    WARP_ROW_LOOP(I, nk) {
        const int k0 = kstart[I], k1 = kstart[I + 1];
        for (int f = fptr[I] + lane; f < fptr[I + 1]; f += 32) {
            const int p = lower_bound_i32(kcol, k0, k1, ucol[f]);
            fnew[f] = (p < k1 && kcol[p] == ucol[f]) ? 0 : 1;
        }
    }
}

// row lengths of the next level: kept entries plus inserted fills
__global__ void k_elim_row_len(const int32_t *__restrict__ kstart, const int32_t *__restrict__ fptr,
                               const int32_t *__restrict__ fnew_pref, int32_t nk, int32_t *__restrict__ len) {
    GRID_LOOP(I, nk) len[I] = (kstart[I + 1] - kstart[I]) + (fnew_pref[fptr[I + 1]] - fnew_pref[fptr[I]]);
}

// the kept entries at their place in the next level's rows (one thread each):
// after the row's inserted fills with a smaller column, with the weights of
// equal fills added
__global__ void k_elim_write_kept(const int32_t *__restrict__ kcol, const double *__restrict__ kw,
                                  const int32_t *__restrict__ krow, int64_t nkept,
                                  const int32_t *__restrict__ kstart, const int32_t *__restrict__ ucol,
                                  const double *__restrict__ uw, const int32_t *__restrict__ fptr,
                                  const int32_t *__restrict__ fnew_pref, const int32_t *__restrict__ rowptr_n,
                                  int32_t *__restrict__ col_n, double *__restrict__ w_n) {
    GRID_LOOP(t, nkept) {
        const int32_t I = krow[t];
        const int f0 = fptr[I], f1 = fptr[I + 1];
        const int32_t c = kcol[t];
        double wt = kw[t];
        int ins = 0;
        if (f0 < f1) {
            const int p = lower_bound_i32(ucol, f0, f1, c);  // fills with a smaller column
            if (p < f1 && ucol[p] == c) wt += uw[p];         // the kept weight, then the fills' sum
            ins = fnew_pref[p] - fnew_pref[f0];
        }
        const int64_t o = (int64_t)rowptr_n[I] + (t - kstart[I]) + ins;
        col_n[o] = c;
        w_n[o] = wt;
    }
}

// the inserted fills (one warp per next-level row; rows without fills skip)
__global__ void k_elim_write_fills(const int32_t *__restrict__ kcol, const int32_t *__restrict__ kstart,
                                   const int32_t *__restrict__ ucol, const double *__restrict__ uw,
                                   const int32_t *__restrict__ fptr, const int32_t *__restrict__ fnew,
                                   const int32_t *__restrict__ fnew_pref, const int32_t *__restrict__ rowptr_n,
                                   int32_t nk, int32_t *__restrict__ col_n, double *__restrict__ w_n) {
    const int lane = threadIdx.x & 31;
    WARP_ROW_LOOP(I, nk) {
        const int f0 = fptr[I], f1 = fptr[I + 1];
        if (f0 == f1) continue;
        const int k0 = kstart[I], k1 = kstart[I + 1];
        const int base = rowptr_n[I];
        for (int f = f0 + lane; f < f1; f += 32) {
            if (!fnew[f]) continue;
            const int q = lower_bound_i32(kcol, k0, k1, ucol[f]) - k0;  // kept entries with a smaller column
            col_n[base + q + (fnew_pref[f] - fnew_pref[f0])] = ucol[f];
            w_n[base + q + (fnew_pref[f] - fnew_pref[f0])] = uw[f];
        }
    }
}

// the restriction's operands per pull entry, read directly by the solve
__global__ void k_elim_pull_direct(const int32_t *__restrict__ pull_e, int64_t npull, const int32_t *__restrict__ e_node,
                                   const double *__restrict__ e_c64, const float *__restrict__ e_c32,
                                   int32_t *__restrict__ pull_u, double *__restrict__ pull_c64,
                                   float *__restrict__ pull_c32) {
    GRID_LOOP(t, npull) {
        const int slot = pull_e[t];
        pull_u[t] = e_node[slot / 2];
        pull_c64[t] = e_c64[slot];
        pull_c32[t] = e_c32[slot];
    }
}

// pull lists: (next-level node, slot 2 j + m) pairs, sorted by node (stable:
// ascending j within a node)
__global__ void k_elim_emit_pull(const int32_t *__restrict__ e_nb, const int32_t *__restrict__ pull_cnt,
                                 const int32_t *__restrict__ ppos, int32_t n_elim, uint64_t *__restrict__ keys,
                                 uint32_t *__restrict__ vals, int32_t *__restrict__ cnt) {
    GRID_LOOP(j, n_elim) {
        for (int m = 0; m < pull_cnt[j]; ++m) {
            const int64_t p = ppos[j] + m;
            keys[p] = (uint32_t)e_nb[2 * j + m];
            vals[p] = (uint32_t)(2 * j + m);
            atomicAdd(&cnt[e_nb[2 * j + m]], 1);
        }
    }
}

}  // namespace

void fingerprint_and_exponent(const Level &L, uint64_t *fp, int *wexp, cudaStream_t s) {
    DBuf<int64_t> f(2, s);
    f.zero(s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_fingerprint_flat, grid_for(L.nnz), kBlock, 0, L.row_of.get(), L.col.get(),
               L.w64.get(), L.nnz, reinterpret_cast<unsigned long long *>(f.get()));
    int64_t h[2] = {0, 0};
    read_totals(f.get(), 2, h, s);
    *fp = (uint64_t)h[0];
    double mx = 0.0;
    std::memcpy(&mx, &h[1], sizeof(mx));
    *wexp = mx > 0.0 ? std::ilogb(mx) : 0;
}

int max_exponent(const double *v, int64_t n, cudaStream_t s) {
    DBuf<int64_t> m(1, s);
    m.zero(s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_max_bits, grid_for(n), kBlock, 0, v, n,
               reinterpret_cast<unsigned long long *>(m.get()));
    int64_t h = 0;
    read_totals(m.get(), 1, &h, s);
    double mx = 0.0;
    std::memcpy(&mx, &h, sizeof(mx));
    return mx > 0.0 ? std::ilogb(mx) : 0;
}

void finish_level(Level &L, int wexp, int reorder, int chunking, cudaStream_t s) {
    const int32_t n = L.n;
    const int64_t nnz = L.nnz;
    chunk_params(nnz, chunking, &L.long_row, &L.chunk);
    L.w32.alloc_persistent(std::max<int64_t>(nnz, 1));
    L.deg32.alloc_persistent(n);
    L.dinv32.alloc_persistent(n);
    L.dinv64.alloc_persistent(n);
    DBuf<int32_t> nchunk(n, s), cfirst(n, s), isl(n, s), lidx(n, s);
    // the counts, the round statistics and the FP32 weights' exactness come
    // back with one synchronisation
    DBuf<int64_t> tot(5, s);
    tot.zero(s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_finish, grid_for(std::max<int64_t>(nnz, n)), kBlock, 0, L.rowptr.get(),
               L.w64.get(), L.deg64.get(), n, nnz, std::ldexp(1.0, -wexp), L.w32.get(), L.deg32.get(),
               L.dinv32.get(), L.dinv64.get(), nchunk.get(), reinterpret_cast<unsigned long long *>(tot.get() + 4),
               L.long_row, L.chunk);
    scan_exclusive_i32_total(nchunk.get(), cfirst.get(), n, tot.get(), s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_long_index, grid_for(n), kBlock, 0, nchunk.get(), n, isl.get());
    scan_exclusive_i32_total(isl.get(), lidx.get(), n, tot.get() + 1, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_order_stats, grid_for((n + 3) / 4), kBlock, 0, L.rowptr.get(), n, L.long_row,
               reinterpret_cast<unsigned long long *>(tot.get() + 2));
    int64_t h[5];
    read_totals(tot.get(), 5, h, s);
    L.n_chunks = (int32_t)h[0];
    L.n_long = (int32_t)h[1];
    L.w32_exact = h[4] == 0;
    // When the row lengths are very uneven (power-law degrees), the row
    // kernels take the rows longest first (a stable sort by length), so that
    // the row groups of a warp get rows of about the same length and the
    // blocks start on the long rows.  Measured with the sorted order on every
    // level: R-MAT 20 SpMV -12 % (this statistic 2.1); BA 100k row kernels
    // -4 % but setup +70 us, a net loss (1.19); grid 1024^2 fine level +8 %
    // from the extra indirection (1.0).  Sorting only within 32-row windows
    // lost the gain.
    L.order.release();
    // reorder 0: when warps spend 50 % more rounds than balanced rows would
    const bool uneven = (double)h[2] > 1.5 * (double)h[3] / 4.0;
    if (reorder == 2 || (reorder == 0 && uneven)) {
        DBuf<uint64_t> keys(n, s);
        L.order.alloc_persistent(n);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_order_keys, grid_for(n), kBlock, 0, L.rowptr.get(), n, L.long_row,
                   keys.get(), reinterpret_cast<uint32_t *>(L.order.get()));
        // keys in [0, long_row + 1]
        radix_sort_pairs(keys.get(), reinterpret_cast<uint32_t *>(L.order.get()), n, bits_for(L.long_row + 2), s);
    }
    if (L.n_chunks == 0) return;
    L.chunk_row.alloc_persistent(L.n_chunks);
    L.chunk_begin.alloc_persistent(L.n_chunks);
    L.chunk_long.alloc_persistent(L.n_chunks);
    L.long_first.alloc_persistent(L.n_long + 1);
    L.long_of_row.alloc_persistent(n);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_fill_chunks, grid_for(n), kBlock, 0, L.rowptr.get(), nchunk.get(),
               cfirst.get(), lidx.get(), n, L.chunk, L.chunk_row.get(), L.chunk_begin.get(), L.chunk_long.get(),
               L.long_first.get(), L.long_of_row.get());
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_set_last, 1, 1, 0, L.long_first.get(), L.n_long, L.n_chunks);
    // chunks in ascending order of their first column (stable: row order among equals)
    {
        DBuf<uint64_t> keys(L.n_chunks, s);
        L.chunk_order.alloc_persistent(L.n_chunks);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_chunk_keys, grid_for(L.n_chunks), kBlock, 0, L.col.get(),
                   L.chunk_begin.get(), L.n_chunks, keys.get(), reinterpret_cast<uint32_t *>(L.chunk_order.get()));
        radix_sort_pairs(keys.get(), reinterpret_cast<uint32_t *>(L.chunk_order.get()), L.n_chunks, bits_for(n), s);
    }
}

// LAMG's low-degree elimination (Sec. 3.1) from the last level of h: an
// independent set of nodes with one or two neighbours is eliminated exactly,
// and the Schur complement becomes the next level.  Returns false (and builds
// nothing) when fewer than min_frac of the nodes would go, or fewer than 64
// would stay.
bool eliminate_level(lap_hierarchy &h, double min_frac, cudaStream_t s) {
    Level &F = h.lv.back();
    const int32_t n = F.n;
    DBuf<int32_t> elim(n, s), keep(n, s), eidx(n, s), kidx(n, s);
    {
        DBuf<int32_t> st0(n, s), st1(n, s);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_init, grid_for(n), kBlock, 0, F.rowptr.get(), n, st0.get());
        for (int r = 0; r < 4; ++r) {
            CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_round, grid_for(n), kBlock, 0, F.rowptr.get(), F.col.get(), n,
                       st0.get(), st1.get());
            std::swap(st0, st1);
        }
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_flags, grid_for(n), kBlock, 0, st0.get(), n, elim.get(), keep.get());
    }
    DBuf<int64_t> tot(2, s);
    tot.zero(s);
    scan_exclusive_i32_total(elim.get(), eidx.get(), n, tot.get(), s);
    scan_exclusive_i32_total(keep.get(), kidx.get(), n, tot.get() + 1, s);
    int64_t ht[2];
    read_totals(tot.get(), 2, ht, s);
    const int32_t ne = (int32_t)ht[0], nk = (int32_t)ht[1];
    if (ne < min_frac * n || nk < 64) return false;
    F.elim = true;
    F.n_elim = ne;
    F.keep_id.alloc_persistent(n);
    F.keep_node.alloc_persistent(nk);
    F.e_node.alloc_persistent(ne);
    F.e_nb.alloc_persistent(2 * (size_t)ne);
    F.e_c64.alloc_persistent(2 * (size_t)ne);
    F.e_c32.alloc_persistent(2 * (size_t)ne);
    F.e_dinv64.alloc_persistent(ne);
    F.e_dinv32.alloc_persistent(ne);
    DBuf<int32_t> fill_cnt(ne, s), pull_cnt(ne, s), fpos(ne, s), ppos(ne, s);
    DBuf<double> fill_w(ne, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_tables, grid_for(n), kBlock, 0, F.rowptr.get(), F.col.get(),
               F.w64.get(), F.deg64.get(), n, elim.get(), eidx.get(), kidx.get(), std::ldexp(1.0, -h.wexp),
               F.keep_id.get(), F.keep_node.get(), F.e_node.get(), F.e_nb.get(), F.e_c64.get(), F.e_c32.get(),
               F.e_dinv64.get(), F.e_dinv32.get(), fill_cnt.get(), pull_cnt.get(), fill_w.get());
    // next-level entries: the kept ones (already in order), merged row by row
    // with the fill edges (sorted and summed on their own)
    DBuf<int32_t> flag(F.nnz, s), pos(F.nnz, s), newcol(F.nnz, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_keep_flags, grid_for(F.nnz), kBlock, 0, F.row_of.get(), F.col.get(), F.nnz,
               F.keep_id.get(), flag.get(), newcol.get());
    DBuf<int64_t> tot2(3, s);
    tot2.zero(s);
    scan_exclusive_i32_total(flag.get(), pos.get(), F.nnz, tot2.get(), s);
    scan_exclusive_i32_total(fill_cnt.get(), fpos.get(), ne, tot2.get() + 1, s);
    scan_exclusive_i32_total(pull_cnt.get(), ppos.get(), ne, tot2.get() + 2, s);
    int64_t h3[3];
    read_totals(tot2.get(), 3, h3, s);
    const int64_t nkept = h3[0], nfill = h3[1], npull = h3[2];
    const int b = bits_for(nk);
    Graph64 C;
    C.n = nk;
    C.rowptr.alloc_persistent(nk + 1);
    C.deg.alloc_persistent(nk);
    {
        DBuf<int32_t> kcol(std::max<int64_t>(nkept, 1), s), krow(std::max<int64_t>(nkept, 1), s), kstart(nk + 1, s);
        DBuf<double> kw(std::max<int64_t>(nkept, 1), s);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_compact, grid_for(F.nnz), kBlock, 0, F.row_of.get(), F.w64.get(),
                   F.nnz, kidx.get(), flag.get(), pos.get(), newcol.get(), kcol.get(), kw.get(), krow.get());
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_kstart, grid_for(n), kBlock, 0, F.rowptr.get(), n, elim.get(),
                   kidx.get(), pos.get(), kstart.get());
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_set_last, 1, 1, 0, kstart.get(), nk, (int32_t)nkept);
        flag.release();
        pos.release();
        newcol.release();
        // fill edges: sort, sum equal pairs, count per row
        DBuf<int32_t> ucol(std::max<int64_t>(nfill, 1), s), fptr(nk + 1, s), fcnt(nk + 1, s);
        DBuf<double> uw(std::max<int64_t>(nfill, 1), s);
        fcnt.zero(s);
        int64_t nu = 0;
        if (nfill > 0) {
            DBuf<uint64_t> keys(nfill, s);
            DBuf<uint32_t> vals(nfill, s);
            DBuf<double> wv(nfill, s);
            CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_emit_fill, grid_for(ne), kBlock, 0, F.e_nb.get(), fill_cnt.get(),
                       fpos.get(), fill_w.get(), ne, (int64_t)0, b, keys.get(), vals.get(), wv.get());
            radix_sort_pairs(keys.get(), vals.get(), nfill, 2 * b, s);
            DBuf<int32_t> head(nfill, s), hpos(nfill, s);
            CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_heads, grid_for(nfill), kBlock, 0, keys.get(), nfill, head.get());
            nu = scan_exclusive_i32(head.get(), hpos.get(), nfill, s);
            CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_merge, grid_for(nfill), kBlock, 0, keys.get(), vals.get(), head.get(),
                       hpos.get(), nfill, b, wv.get(), ucol.get(), uw.get(), fcnt.get());
        }
        scan_exclusive_i32(fcnt.get(), fptr.get(), nk, s);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_set_last, 1, 1, 0, fptr.get(), nk, (int32_t)nu);
        // which fills are new entries, the row lengths, and the merge
        DBuf<int32_t> fnew(std::max<int64_t>(nu, 1), s), fnew_pref(nu + 1, s), rlen(nk, s);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_fill_new, grid_for(32 * (int64_t)nk), kBlock, 0, kcol.get(),
                   kstart.get(), ucol.get(), fptr.get(), nk, fnew.get());
        const int64_t nnew = nu > 0 ? scan_exclusive_i32(fnew.get(), fnew_pref.get(), nu, s) : 0;
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_set_last, 1, 1, 0, fnew_pref.get(), (int32_t)nu, (int32_t)nnew);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_row_len, grid_for(nk), kBlock, 0, kstart.get(), fptr.get(),
                   fnew_pref.get(), nk, rlen.get());
        const int64_t cnnz = scan_exclusive_i32(rlen.get(), C.rowptr.get(), nk, s);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_set_last, 1, 1, 0, C.rowptr.get(), nk, (int32_t)cnnz);
        C.nnz = cnnz;
        C.col.alloc_persistent(std::max<int64_t>(cnnz, 1));
        C.w.alloc_persistent(std::max<int64_t>(cnnz, 1));
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_write_kept, grid_for(nkept), kBlock, 0, kcol.get(), kw.get(),
                   krow.get(), nkept, kstart.get(), ucol.get(), uw.get(), fptr.get(), fnew_pref.get(),
                   C.rowptr.get(), C.col.get(), C.w.get());
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_write_fills, grid_for(32 * (int64_t)nk), kBlock, 0, kcol.get(),
                   kstart.get(), ucol.get(), uw.get(), fptr.get(), fnew.get(), fnew_pref.get(), C.rowptr.get(), nk,
                   C.col.get(), C.w.get());
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_row_sums_short, grid_for(nk), kBlock, 0,
                   C.rowptr.get(), C.w.get(), nk, C.deg.get());
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_row_sums_long, grid_for(32 * (int64_t)nk), kBlock, 0,
                   C.rowptr.get(), C.w.get(), nk, C.deg.get());
    }
    // pull lists of the restriction, in ascending order of the eliminated node
    {
        DBuf<uint64_t> keys(std::max<int64_t>(npull, 1), s);
        DBuf<uint32_t> vals(std::max<int64_t>(npull, 1), s);
        DBuf<int32_t> cnt(nk + 1, s);
        cnt.zero(s);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_emit_pull, grid_for(ne), kBlock, 0, F.e_nb.get(), pull_cnt.get(),
                   ppos.get(), ne, keys.get(), vals.get(), cnt.get());
        radix_sort_pairs(keys.get(), vals.get(), npull, bits_for(nk), s);
        F.pull_ptr.alloc_persistent(nk + 1);
        F.pull_e.alloc_persistent(std::max<int64_t>(npull, 1));
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_u32_to_i32, grid_for(npull), kBlock, 0, vals.get(), F.pull_e.get(),
                   (int32_t)npull);
        scan_exclusive_i32(cnt.get(), F.pull_ptr.get(), nk, s);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_set_last, 1, 1, 0, F.pull_ptr.get(), nk, (int32_t)npull);
        F.pull_u.alloc_persistent(std::max<int64_t>(npull, 1));
        F.pull_c64.alloc_persistent(std::max<int64_t>(npull, 1));
        F.pull_c32.alloc_persistent(std::max<int64_t>(npull, 1));
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_elim_pull_direct, grid_for(npull), kBlock, 0, F.pull_e.get(), npull,
                   F.e_node.get(), F.e_c64.get(), F.e_c32.get(), F.pull_u.get(), F.pull_c64.get(),
                   F.pull_c32.get());
        // long pull lists (hubs with many eliminated neighbours) in chunks, like long rows
        DBuf<int32_t> nchunk(nk, s), cfirst(nk, s), isl(nk, s), lidx(nk, s);
        DBuf<int64_t> ct(2, s);
        ct.zero(s);
        chunk_params(npull, h.hopts.chunking, &F.pull_long_row, &F.pull_chunk);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_nchunk, grid_for(nk), kBlock, 0, F.pull_ptr.get(), nk, F.pull_long_row,
                   F.pull_chunk, nchunk.get());
        scan_exclusive_i32_total(nchunk.get(), cfirst.get(), nk, ct.get(), s);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_long_index, grid_for(nk), kBlock, 0, nchunk.get(), nk, isl.get());
        scan_exclusive_i32_total(isl.get(), lidx.get(), nk, ct.get() + 1, s);
        int64_t hc[2];
        read_totals(ct.get(), 2, hc, s);
        F.pull_n_chunks = (int32_t)hc[0];
        F.pull_n_long = (int32_t)hc[1];
        if (F.pull_n_chunks > 0) {
            F.pull_chunk_row.alloc_persistent(F.pull_n_chunks);
            F.pull_chunk_begin.alloc_persistent(F.pull_n_chunks);
            F.pull_chunk_long.alloc_persistent(F.pull_n_chunks);
            F.pull_long_first.alloc_persistent(F.pull_n_long + 1);
            F.pull_long_of_row.alloc_persistent(nk);
            CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_fill_chunks, grid_for(nk), kBlock, 0, F.pull_ptr.get(), nchunk.get(),
                       cfirst.get(), lidx.get(), nk, F.pull_chunk, F.pull_chunk_row.get(), F.pull_chunk_begin.get(),
                       F.pull_chunk_long.get(), F.pull_long_first.get(), F.pull_long_of_row.get());
            CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_set_last, 1, 1, 0, F.pull_long_first.get(), F.pull_n_long,
                       F.pull_n_chunks);
        }
    }
    Level Cl;
    Cl.n = nk;
    Cl.nnz = C.nnz;
    Cl.rowptr = std::move(C.rowptr);
    Cl.col = std::move(C.col);
    Cl.w64 = std::move(C.w);
    Cl.deg64 = std::move(C.deg);
    h.lv.push_back(std::move(Cl));
    finish_level(h.lv.back(), h.wexp, h.hopts.reorder, h.hopts.chunking, s);
    return true;
}

void ensure_bf16(Level &L, int wexp, cudaStream_t s) {
    if (L.wbf.get()) return;
    L.wbf.alloc_persistent(std::max<int64_t>(L.nnz, 1));
    L.degbf.alloc_persistent(L.n);
    L.dinvbf.alloc_persistent(L.n);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_bf16_level, grid_for(L.n), kBlock, 0, L.rowptr.get(), L.w64.get(), L.n,
               std::ldexp(1.0, -wexp), L.wbf.get(), L.degbf.get(), L.dinvbf.get());
}

void dense_spd_inverse_small(double *A, int n, int *d_flag, cudaStream_t s) {
    const size_t smem = (size_t)(n * n + n) * sizeof(double);
    CFC_CUDA(cudaFuncSetAttribute(k_gj_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_gj_smem, 1, 1024, smem, A, n, d_flag);
}

void dense_spd_inverse_large(double *A, int n, int *d_flag, cudaStream_t s) {
    DBuf<double> pinv((size_t)kGjB * kGjB, s), cold((size_t)n * kGjB, s), rnew((size_t)kGjB * n, s);
    int per_sm = 0;
    CFC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_blocked, kBlock, 0));
    int dev = 0, sms = 0;
    CFC_CUDA(cudaGetDevice(&dev));
    CFC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t td = (n + kGjTile - 1) / kGjTile;
    // every block must be resident (grid barriers): at most the co-resident count
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(1, per_sm) * sms, td * td));
    double *a = A, *pi = pinv.get(), *co = cold.get(), *rn = rnew.get();
    int nn = n, *f = d_flag;
    void *args[] = {&a, &nn, &pi, &co, &rn, &f};
    ::cfc::LaunchScope scope_(LAP_KF_SETUP, s, 0.0);
    CFC_CUDA(cudaLaunchCooperativeKernel((const void *)k_gj_blocked, blocks, kBlock, args, 0, s));
}

void build_dense(const int32_t *rowptr, const int32_t *col, const double *w, const double *deg, int32_t n,
                 double alpha, double *M, cudaStream_t s) {
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_fill, grid_for((int64_t)n * n), kBlock, 0, M, (int64_t)n * n, alpha / n);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_dense_scatter, grid_for(n), kBlock, 0, rowptr, col, w, deg, n, M);
}

// Level 0 from the ingested graph; coarser levels are added by grow_levels.
void init_levels(lap_hierarchy &h, Csr64 &fine, const lap_hier_opts_t &o, cudaStream_t s) {
    h.lv.clear();
    h.lv.emplace_back();
    Level &L0 = h.lv.back();
    L0.n = fine.n;
    L0.nnz = fine.nnz;
    L0.rowptr = std::move(fine.rowptr);
    L0.col = std::move(fine.col);
    L0.w64 = std::move(fine.w);
    L0.deg64 = std::move(fine.deg);
    L0.row_of = std::move(fine.row_of);
    h.hopts = o;
    h.complete = false;
    h.coarse_n = 0;
    // the graph's fingerprint and the largest weight's exponent, with one pass and one synchronisation
    fingerprint_and_exponent(L0, &h.fingerprint, &h.wexp, s);
    finish_level(L0, h.wexp, o.reorder, o.chunking, s);
    const int64_t low = build_jl_chunks(L0, s);
    h.p0 = 0;
    // low-degree elimination when it removes at least 5 % of the nodes (the
    // nodes with one or two neighbours bound what it can remove)
    if (o.eliminate && L0.n > 256 && low >= 0.05 * L0.n && eliminate_level(h, 0.05, s)) h.p0 = 1;
    h.lv[0].row_of.release();
    const Level &T = h.lv.back();
    if (T.n <= effective_coarse_max(h) || o.max_levels <= 1) grow_levels(h, 0, s);
}

int64_t build_jl_chunks(Level &L, cudaStream_t s) {
    const int32_t n = L.n;
    DBuf<int32_t> nchunk(n, s), cfirst(n, s), isl(n, s), lidx(n, s);
    DBuf<int64_t> ct(3, s);
    ct.zero(s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_jl_nchunk, grid_for(n), kBlock, 0, L.rowptr.get(), n, nchunk.get(),
               reinterpret_cast<unsigned long long *>(ct.get() + 2));
    scan_exclusive_i32_total(nchunk.get(), cfirst.get(), n, ct.get(), s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_long_index, grid_for(n), kBlock, 0, nchunk.get(), n, isl.get());
    scan_exclusive_i32_total(isl.get(), lidx.get(), n, ct.get() + 1, s);
    int64_t hc[3];
    read_totals(ct.get(), 3, hc, s);
    L.jl_n_chunks = (int32_t)hc[0];
    L.jl_n_long = (int32_t)hc[1];
    if (L.jl_n_chunks == 0) return hc[2];
    L.jl_chunk_row.alloc_persistent(L.jl_n_chunks);
    L.jl_chunk_begin.alloc_persistent(L.jl_n_chunks);
    L.jl_long_first.alloc_persistent(L.jl_n_long + 1);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_jl_fill, grid_for(n), kBlock, 0, L.rowptr.get(), nchunk.get(), cfirst.get(),
               lidx.get(), n, L.jl_chunk_row.get(), L.jl_chunk_begin.get(), L.jl_long_first.get());
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_set_last, 1, 1, 0, L.jl_long_first.get(), L.jl_n_long, L.jl_n_chunks);
    return hc[2];
}

// coarse_max in effect: the option, or (0) n_top / 4096 clamped to [256, 1024]
// with n_top the PCG level's size; at most kDenseMax
int effective_coarse_max(const lap_hierarchy &h) {
    const int o = h.hopts.coarse_max;
    int c = o;
    if (o <= 0) {
        const int64_t ntop = h.lv[h.p0].n;
        c = (int)std::min<int64_t>(1024, std::max<int64_t>(256, ntop / 4096));
    }
    return std::min(kDenseMax, std::max(2, c));
}

// Coarsen until the hierarchy has `target` levels (0: until coarsening stops:
// n_l <= coarse_max, the level cap, or a stall).  On completion the coarsest
// level gets its dense inverse when it is small enough.
void grow_levels(lap_hierarchy &h, int target, cudaStream_t s) {
    if (h.complete) return;
    const lap_hier_opts_t &o = h.hopts;
    const int coarse_max = effective_coarse_max(h);
    const int max_levels = std::max(1, std::min(32, o.max_levels));
    bool stalled = false;
    cudaEvent_t ev0, ev1;
    CFC_CUDA(cudaEventCreate(&ev0));
    CFC_CUDA(cudaEventCreate(&ev1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evg{ev0, ev1};
    // levels of the cycle: those from lv[p0] on (the elimination levels in front are not counted)
    auto cycle_levels = [&]() { return (int)h.lv.size() - h.p0; };
    while (cycle_levels() < max_levels && h.lv.back().n > coarse_max && (target <= 0 || cycle_levels() < target)) {
        CFC_CUDA(cudaEventRecord(ev0, s));
        Level &F = h.lv.back();
        const int32_t n = F.n;
        DBuf<int32_t> agg;
        agg.alloc_persistent(n);
        int32_t nc = pairwise_pass(F.rowptr.get(), F.col.get(), F.w64.get(), F.deg64.get(), n, F.nnz,
                                   std::max(1, o.match_rounds), o.aggregation, o.hub_factor, agg.get(), s);
        for (int p = 1; p < o.agg_passes && nc > coarse_max; ++p) {
            Graph64 mid;
            contract(F.rowptr.get(), F.col.get(), F.w64.get(), n, F.nnz, agg.get(), nc, false, mid, s);
            DBuf<int32_t> agg2(nc, s);
            const int32_t nc2 = pairwise_pass(mid.rowptr.get(), mid.col.get(), mid.w.get(), mid.deg.get(), nc,
                                              mid.nnz, std::max(1, o.match_rounds), o.aggregation, o.hub_factor,
                                              agg2.get(), s);
            CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_compose, grid_for(n), kBlock, 0, agg.get(), agg2.get(), n);
            nc = nc2;
        }
        if (nc >= n || (double)nc > 0.9 * n) {  // coarsening stalled
            stalled = true;
            break;
        }
        Graph64 C;
        contract(F.rowptr.get(), F.col.get(), F.w64.get(), n, F.nnz, agg.get(), nc, true, C, s);
        // members of each aggregate in ascending node order (stable sort by aggregate)
        {
            DBuf<uint64_t> keys(n, s);
            DBuf<uint32_t> vals(n, s);
            DBuf<int32_t> cnt(nc + 1, s);
            cnt.zero(s);
            CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_iota_keys, grid_for(n), kBlock, 0, agg.get(), n, keys.get(),
                       vals.get(), cnt.get());
            radix_sort_pairs(keys.get(), vals.get(), n, bits_for(nc), s);
            F.mem.alloc_persistent(n);
            F.mem_ptr.alloc_persistent(nc + 1);
            CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_u32_to_i32, grid_for(n), kBlock, 0, vals.get(), F.mem.get(), n);
            scan_exclusive_i32(cnt.get(), F.mem_ptr.get(), nc, s);
            CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_set_last, 1, 1, 0, F.mem_ptr.get(), nc, n);
        }
        F.agg = std::move(agg);
        Level Cl;
        Cl.n = nc;
        Cl.nnz = C.nnz;
        Cl.rowptr = std::move(C.rowptr);
        Cl.col = std::move(C.col);
        Cl.w64 = std::move(C.w);
        Cl.deg64 = std::move(C.deg);
        h.lv.push_back(std::move(Cl));
        finish_level(h.lv.back(), h.wexp, o.reorder, o.chunking, s);
        CFC_CUDA(cudaEventRecord(ev1, s));
        CFC_CUDA(cudaEventSynchronize(ev1));
        float ms = 0.f;
        CFC_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
        h.level_ms.resize(h.lv.size(), 0.0);
        h.level_ms[h.lv.size() - 1] = ms;
    }
    const bool done = stalled || cycle_levels() >= max_levels || h.lv.back().n <= coarse_max;
    if (!done) return;
    h.complete = true;
    // dense coarsest solve
    Level &Lc = h.lv.back();
    h.coarse_n = 0;
    CFC_CUDA(cudaEventRecord(ev0, s));
    if (Lc.n <= kDenseMax) {
        const int nc = Lc.n;
        h.coarse_inv.alloc_persistent((size_t)nc * nc);
        // the constant mode gets eigenvalue 2^wexp, of the order of the weights
        build_dense(Lc.rowptr.get(), Lc.col.get(), Lc.w64.get(), Lc.deg64.get(), nc, std::ldexp(1.0, h.wexp),
                    h.coarse_inv.get(), s);
        DBuf<int> flag(1, s);
        flag.zero(s);
        if (nc <= 160) dense_spd_inverse_small(h.coarse_inv.get(), nc, flag.get(), s);
        else dense_spd_inverse_large(h.coarse_inv.get(), nc, flag.get(), s);
        int hf = 0;
        CFC_CUDA(cudaMemcpyAsync(&hf, flag.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
        CFC_CUDA(cudaStreamSynchronize(s));
        // The graph is connected (checked at ingest), so a non-positive pivot
        // means FP64 lost the matrix's definiteness (weights many orders of
        // magnitude apart): the coarsest level is then smoothed instead of
        // solved densely, which keeps the cycle a valid preconditioner.
        if (hf == 0) {
            h.coarse_n = nc;
            h.coarse_inv32.alloc_persistent((size_t)nc * nc);
            CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_scaled_f32, grid_for((int64_t)nc * nc), kBlock, 0, h.coarse_inv.get(),
                       (int64_t)nc * nc, h.wexp, h.coarse_inv32.get());
        } else {
            h.coarse_inv.release();
        }
        CFC_CUDA(cudaEventRecord(ev1, s));
        CFC_CUDA(cudaEventSynchronize(ev1));
        float ms = 0.f;
        CFC_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
        h.level_ms.resize(h.lv.size(), 0.0);
        h.level_ms.back() += ms;
    }
}

}  // namespace cfc
