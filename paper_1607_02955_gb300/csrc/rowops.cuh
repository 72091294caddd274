// Generic kernels over the rows of a level's Laplacian, applied to a tile of
// KT right-hand-side columns of row-major n x ld blocks.
//
// Layout: a group of G = KT / VW lanes owns one row; each lane owns VW
// consecutive columns (float4 for FP32, double2 for FP64), so a gathered
// neighbour row of the tile is one coalesced KT*sizeof(T)-byte load.
// Rows with more than kLongRow nonzeros are split into chunks processed by
// separate groups; the chunk sums go to a scratch buffer and the group that
// finishes a row's last chunk (arrival counter) adds them up in chunk order
// and runs the row's epilogue, so results are independent of scheduling.
//
// Per-column reductions (dot products, norms, sums) are accumulated in FP64:
// per thread over its rows, per block over its groups in a fixed order,
// then across blocks by the last block to arrive, again in a fixed order.
// The grid size depends only on the problem and the device's SM count, so
// every reduction is bitwise reproducible.
#pragma once

#include "internal.h"

namespace cfc {

template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using V = float4;
    static constexpr int W = 4;
};
template <>
struct Vec<double> {
    using V = double2;
    static constexpr int W = 2;
};

template <typename V>
__device__ __forceinline__ V vzero();
template <>
__device__ __forceinline__ float4 vzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <>
__device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }

template <typename T>
__device__ __forceinline__ typename Vec<T>::V vld(const T *p) {
    return *reinterpret_cast<const typename Vec<T>::V *>(p);
}
template <typename T>
__device__ __forceinline__ typename Vec<T>::V vldg(const T *p) {  // read-only path
    return __ldg(reinterpret_cast<const typename Vec<T>::V *>(p));
}
template <typename T>
__device__ __forceinline__ typename Vec<T>::V vldcg(const T *p) {  // L2, coherent across blocks
    return __ldcg(reinterpret_cast<const typename Vec<T>::V *>(p));
}
template <typename T>
__device__ __forceinline__ void vst(T *p, typename Vec<T>::V v) {
    *reinterpret_cast<typename Vec<T>::V *>(p) = v;
}

// element access
__device__ __forceinline__ float &vel(float4 &v, int i) { return (&v.x)[i]; }
__device__ __forceinline__ double &vel(double2 &v, int i) { return (&v.x)[i]; }
__device__ __forceinline__ float vel(const float4 &v, int i) { return (&v.x)[i]; }
__device__ __forceinline__ double vel(const double2 &v, int i) { return (&v.x)[i]; }

// s += a * x
__device__ __forceinline__ void vfma(float4 &s, float a, const float4 &x) {
    s.x = fmaf(a, x.x, s.x);
    s.y = fmaf(a, x.y, s.y);
    s.z = fmaf(a, x.z, s.z);
    s.w = fmaf(a, x.w, s.w);
}
__device__ __forceinline__ void vfma(double2 &s, double a, const double2 &x) {
    s.x = fma(a, x.x, s.x);
    s.y = fma(a, x.y, s.y);
}
__device__ __forceinline__ float4 vadd(const float4 &a, const float4 &b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ double2 vadd(const double2 &a, const double2 &b) { return make_double2(a.x + b.x, a.y + b.y); }

template <typename T>
__device__ __forceinline__ T lw(const LevelView &A, int e);
template <>
__device__ __forceinline__ float lw<float>(const LevelView &A, int e) { return __ldg(A.w32 + e); }
template <>
__device__ __forceinline__ double lw<double>(const LevelView &A, int e) { return __ldg(A.w64 + e); }
template <typename T>
__device__ __forceinline__ T ldeg(const LevelView &A, int i);
template <>
__device__ __forceinline__ float ldeg<float>(const LevelView &A, int i) { return __ldg(A.deg32 + i); }
template <>
__device__ __forceinline__ double ldeg<double>(const LevelView &A, int i) { return __ldg(A.deg64 + i); }
template <typename T>
__device__ __forceinline__ T ldinv(const LevelView &A, int i);
template <>
__device__ __forceinline__ float ldinv<float>(const LevelView &A, int i) { return __ldg(A.dinv32 + i); }
template <>
__device__ __forceinline__ double ldinv<double>(const LevelView &A, int i) { return __ldg(A.dinv64 + i); }

// ------------------------------------------------------------------ reductions
// Two-level, fixed-order cross-block reduction.  Blocks are grouped in teams
// of kTeam consecutive blocks; the last block of a team to arrive sums the
// team's partials (in block order), and the last team to arrive sums the
// team partials (in team order) and runs the per-column finalisation.  No
// block waits for another, and the order of every sum is fixed.
constexpr int kTeam = 32;
constexpr int kMaxTeams = 128;

struct RedBuf {
    double *part;            // [ntiles][NR*KT][P]
    double *team_part;       // [ntiles][NR*KT][kMaxTeams]
    uint32_t *counter;       // [kMaxTiles], zero between launches
    uint32_t *team_counter;  // [kMaxTiles][kMaxTeams], zero between launches
};

// acc holds this thread's partial sums in the kernel's arithmetic type (FP32
// partials over a few rows: FP64 per element would run on GB300's narrow
// FP64 pipe); the block, team and final stages add in FP64.
template <int KT, int NR, int VW, int RPB, typename TA, class Op>
__device__ __forceinline__ void block_reduce_finalize(TA (&acc)[NR][VW], int lane, int grp, RedBuf rb,
                                                      Op &op) {
    constexpr int NO = NR * KT;
    __shared__ double sm[RPB][NO];
    __shared__ double fin[NO];
    __shared__ int is_last;
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int v = 0; v < VW; ++v) sm[grp][r * KT + lane * VW + v] = (double)acc[r][v];
    __syncthreads();
    const int tile = blockIdx.y;
    const int P = gridDim.x;
    for (int o = threadIdx.x; o < NO; o += blockDim.x) {
        double s = 0.0;
        for (int g = 0; g < RPB; ++g) s += sm[g][o];
        rb.part[((size_t)tile * NO + o) * P + blockIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    const int team = blockIdx.x / kTeam;
    const int team_size = min(kTeam, P - team * kTeam);
    const int nteams = (P + kTeam - 1) / kTeam;
    if (threadIdx.x == 0) {
        const uint32_t t = atomicAdd(rb.team_counter + tile * kMaxTeams + team, 1u);
        is_last = (t == (uint32_t)team_size - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // team stage: one thread per output, the team's partials loaded together
    for (int o = threadIdx.x; o < NO; o += blockDim.x) {
        const double *src = rb.part + ((size_t)tile * NO + o) * P + team * kTeam;
        double v[kTeam];
#pragma unroll
        for (int i = 0; i < kTeam; ++i) v[i] = (i < team_size) ? __ldcg(src + i) : 0.0;
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < kTeam; ++i) t += v[i];
        rb.team_part[((size_t)tile * NO + o) * kMaxTeams + team] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        rb.team_counter[tile * kMaxTeams + team] = 0;
        const uint32_t t = atomicAdd(rb.counter + tile, 1u);
        is_last = (t == (uint32_t)nteams - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int o = threadIdx.x; o < NO; o += blockDim.x) {
        const double *src = rb.team_part + ((size_t)tile * NO + o) * kMaxTeams;
        double t = 0.0;
        for (int t0 = 0; t0 < nteams; t0 += kTeam) {
            double v[kTeam];
#pragma unroll
            for (int i = 0; i < kTeam; ++i) v[i] = (t0 + i < nteams) ? __ldcg(src + t0 + i) : 0.0;
#pragma unroll
            for (int i = 0; i < kTeam; ++i) t += v[i];
        }
        fin[o] = t;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < KT; c += blockDim.x) {
        double sums[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) sums[r] = fin[r * KT + c];
        op.fin(tile * KT + c, sums);
    }
    if (threadIdx.x == 0) rb.counter[tile] = 0;
}

// sum_{e in [e0, e1)} w_e x_{col(e)} for this lane's columns; eight gathers
// in flight per lane
template <typename T, class Op>
__device__ __forceinline__ typename Vec<T>::V row_sum(const LevelView &A, const Op &op, int e0, int e1, int c0) {
    using V = typename Vec<T>::V;
    V s0 = vzero<V>(), s1 = vzero<V>();
    int e = e0;
    for (; e + 7 < e1; e += 8) {
        int j[8];
        T w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            j[u] = __ldg(A.col + e + u);
            w[u] = lw<T>(A, e + u);
        }
        V x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = op.gather(j[u], c0);
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            vfma(s0, w[u], x[u]);
            vfma(s1, w[u + 1], x[u + 1]);
        }
    }
    if (e + 3 < e1) {
        int j[4];
        T w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            j[u] = __ldg(A.col + e + u);
            w[u] = lw<T>(A, e + u);
        }
        V x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = op.gather(j[u], c0);
        vfma(s0, w[0], x[0]);
        vfma(s1, w[1], x[1]);
        vfma(s0, w[2], x[2]);
        vfma(s1, w[3], x[3]);
        e += 4;
    }
    for (; e < e1; ++e) vfma(s0, lw<T>(A, e), op.gather(__ldg(A.col + e), c0));
    return vadd(s0, s1);
}

// ------------------------------------------------------------------ SpMM-like row operator
// Op provides:
//   V gather(int j, int c0) const             operand of node j, this lane's columns
//   void epi(int i, int c0, V s, double acc[NR][VW])   row i given s = sum_j w_ij x_j
//   void fin(int c, const double *sums)        per-column finalisation (NR > 0)
template <typename T, int KT, int NR, class Op>
__global__ void __launch_bounds__(kBlock) k_rowop(LevelView A, Op op, int nvb_short, int nvb_total,
                                                  T *chunk_part, int ld_part, RedBuf rb) {
    using V = typename Vec<T>::V;
    constexpr int VW = Vec<T>::W;
    constexpr int G = KT / VW;
    constexpr int RPB = kBlock / G;
    constexpr int NRA = NR > 0 ? NR : 1;
    __shared__ int s_last[RPB];
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int tile = blockIdx.y;
    const int c0 = tile * KT + lane * VW;
    T acc[NRA][VW];
#pragma unroll
    for (int r = 0; r < NRA; ++r)
#pragma unroll
        for (int v = 0; v < VW; ++v) acc[r][v] = T(0);

    for (int vb = blockIdx.x; vb < nvb_total; vb += gridDim.x) {
        if (vb < nvb_short) {
            const int i = vb * RPB + grp;
            if (i < A.n) {
                const int e0 = __ldg(A.rowptr + i), e1 = __ldg(A.rowptr + i + 1);
                if (e1 - e0 <= kLongRow) {
                    const V s = row_sum<T>(A, op, e0, e1, c0);
                    op.epi(i, c0, s, acc);
                }
            }
        } else {
            const int ch = (vb - nvb_short) * RPB + grp;
            const bool has = ch < A.n_chunks;
            int i = 0;
            if (has) {
                i = __ldg(A.chunk_row + ch);
                const int e0 = __ldg(A.chunk_begin + ch);
                const int e1 = min(e0 + kLongRow, __ldg(A.rowptr + i + 1));
                const V s = row_sum<T>(A, op, e0, e1, c0);
                vst<T>(chunk_part + (size_t)ch * ld_part + c0, s);
                __threadfence();
            }
            __syncwarp();
            if (has && lane == 0) {
                const int li = __ldg(A.chunk_long + ch);
                const uint32_t nch = (uint32_t)(__ldg(A.long_first + li + 1) - __ldg(A.long_first + li));
                const uint32_t t = atomicAdd(A.long_count + (size_t)li * kMaxTiles + tile, 1u);
                s_last[grp] = (t == nch - 1) ? 1 : 0;
            }
            __syncwarp();
            if (has && s_last[grp]) {
                __threadfence();
                const int li = __ldg(A.chunk_long + ch);
                const int f0 = __ldg(A.long_first + li), f1 = __ldg(A.long_first + li + 1);
                V s = vzero<V>();
                for (int f = f0; f < f1; ++f) s = vadd(s, vldcg<T>(chunk_part + (size_t)f * ld_part + c0));
                op.epi(i, c0, s, acc);
                if (lane == 0) A.long_count[(size_t)li * kMaxTiles + tile] = 0;
            }
            __syncwarp();
        }
    }
    if constexpr (NR > 0) block_reduce_finalize<KT, NR, VW, RPB, T>(acc, lane, grp, rb, op);
}

// ------------------------------------------------------------------ row-local kernels (no gathers)
// Op provides: void row(int i, int c0, double acc[NR][VW]) and fin (NR > 0).
template <typename T, int KT, int NR, class Op>
__global__ void __launch_bounds__(kBlock) k_rows(int n, Op op, RedBuf rb) {
    constexpr int VW = Vec<T>::W;
    constexpr int G = KT / VW;
    constexpr int RPB = kBlock / G;
    constexpr int NRA = NR > 0 ? NR : 1;
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int c0 = blockIdx.y * KT + lane * VW;
    T acc[NRA][VW];
#pragma unroll
    for (int r = 0; r < NRA; ++r)
#pragma unroll
        for (int v = 0; v < VW; ++v) acc[r][v] = T(0);
    for (int i = blockIdx.x * RPB + grp; i < n; i += gridDim.x * RPB) op.row(i, c0, acc);
    if constexpr (NR > 0) block_reduce_finalize<KT, NR, VW, RPB, T>(acc, lane, grp, rb, op);
}

}  // namespace cfc
