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
struct RedBuf {
    double *part;       // [ntiles][NR*KT][P]
    uint32_t *counter;  // [ntiles], zero between launches
};

template <int KT, int NR, int VW, int RPB, class Op>
__device__ __forceinline__ void block_reduce_finalize(double (&acc)[NR][VW], int lane, int grp, RedBuf rb,
                                                      Op &op) {
    constexpr int NO = NR * KT;
    __shared__ double sm[RPB][NO];
    __shared__ double fin[NO];
    __shared__ int is_last;
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int v = 0; v < VW; ++v) sm[grp][r * KT + lane * VW + v] = acc[r][v];
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
    if (threadIdx.x == 0) {
        const uint32_t t = atomicAdd(rb.counter + tile, 1u);
        is_last = (t == (uint32_t)P - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const int wl = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = wid; o < NO; o += nw) {
        const double *src = rb.part + ((size_t)tile * NO + o) * P;
        double s = 0.0;
        for (int p = wl; p < P; p += 32) s += __ldcg(src + p);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
        if (wl == 0) fin[o] = s;
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
    double acc[NRA][VW];
#pragma unroll
    for (int r = 0; r < NRA; ++r)
#pragma unroll
        for (int v = 0; v < VW; ++v) acc[r][v] = 0.0;

    for (int vb = blockIdx.x; vb < nvb_total; vb += gridDim.x) {
        if (vb < nvb_short) {
            const int i = vb * RPB + grp;
            if (i < A.n) {
                const int e0 = __ldg(A.rowptr + i), e1 = __ldg(A.rowptr + i + 1);
                if (e1 - e0 <= kLongRow) {
                    V s = vzero<V>();
                    int e = e0;
                    for (; e + 3 < e1; e += 4) {
                        const int j0 = __ldg(A.col + e), j1 = __ldg(A.col + e + 1);
                        const int j2 = __ldg(A.col + e + 2), j3 = __ldg(A.col + e + 3);
                        const T w0 = lw<T>(A, e), w1 = lw<T>(A, e + 1), w2 = lw<T>(A, e + 2), w3 = lw<T>(A, e + 3);
                        const V x0 = op.gather(j0, c0), x1 = op.gather(j1, c0);
                        const V x2 = op.gather(j2, c0), x3 = op.gather(j3, c0);
                        vfma(s, w0, x0);
                        vfma(s, w1, x1);
                        vfma(s, w2, x2);
                        vfma(s, w3, x3);
                    }
                    for (; e < e1; ++e) vfma(s, lw<T>(A, e), op.gather(__ldg(A.col + e), c0));
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
                V s = vzero<V>();
                for (int e = e0; e < e1; ++e) vfma(s, lw<T>(A, e), op.gather(__ldg(A.col + e), c0));
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
    if constexpr (NR > 0) block_reduce_finalize<KT, NR, VW, RPB>(acc, lane, grp, rb, op);
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
    double acc[NRA][VW];
#pragma unroll
    for (int r = 0; r < NRA; ++r)
#pragma unroll
        for (int v = 0; v < VW; ++v) acc[r][v] = 0.0;
    for (int i = blockIdx.x * RPB + grp; i < n; i += gridDim.x * RPB) op.row(i, c0, acc);
    if constexpr (NR > 0) block_reduce_finalize<KT, NR, VW, RPB>(acc, lane, grp, rb, op);
}

}  // namespace cfc
