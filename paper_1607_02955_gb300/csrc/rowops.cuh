// Generic kernels over the rows of a level's Laplacian, applied to a tile of
// KT right-hand-side columns of row-major n x ld blocks.
//
// Layout: a group of G = KT / VW lanes owns one row; each lane owns VW
// consecutive columns (8 floats or 4 doubles, 32 bytes, one 256-bit access),
// so a gathered neighbour row of the tile is one contiguous KT*sizeof(T)-byte
// run read with one instruction per lane.  Blocks walk row blocks
// grid-stride; on levels with very uneven row lengths the rows are taken in a
// fixed longest-first order (LevelView::order).
//
// Rows with more than A.long_row nonzeros are split into chunks of A.chunk.
// Without reductions the group that finishes a row's last chunk (arrival
// counter) adds the chunk sums in chunk order and runs the row's epilogue;
// with reductions the chunk sums come from a k_chunk_sums launch just before
// and the row's own group finishes it.  Either way results do not depend on
// scheduling.
//
// Per-column reductions (dot products, norms, sums) keep thread partials in
// the kernel's arithmetic type over the rows a thread handles, add them
// across a warp by a fixed shuffle tree and across warps in order, and then
// in FP64 across blocks, by teams of blocks and by the last team to arrive,
// each in a fixed order.  The grid size depends only on the problem and the
// device's SM count, so every reduction is bitwise reproducible.
#pragma once

#include <type_traits>

#include "internal.h"

namespace cfc {

// A lane owns VW consecutive columns: 8 floats or 4 doubles, 32 bytes, moved
// by one 256-bit load or store (sm_100 and later).  A row group of KT/VW
// lanes thus reads a neighbour's tile row as one contiguous run with one
// instruction per lane: two 16-byte accesses per lane would touch every
// 32-byte sector of the run twice, in two instructions.  Every block of
// vectors is 32-byte aligned (checked on the host before a solve).
struct f8 {
    float4 a, b;
};
struct d4 {
    double2 a, b;
};

template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using V = f8;
    static constexpr int W = 8;
};
template <>
struct Vec<double> {
    using V = d4;
    static constexpr int W = 4;
};

template <typename V>
__device__ __forceinline__ V vzero();
template <>
__device__ __forceinline__ f8 vzero<f8>() {
    return f8{make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
}
template <>
__device__ __forceinline__ d4 vzero<d4>() {
    return d4{make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
}

#define CFC_V8F_OUT(v) "=f"(v.a.x), "=f"(v.a.y), "=f"(v.a.z), "=f"(v.a.w), "=f"(v.b.x), "=f"(v.b.y), "=f"(v.b.z), "=f"(v.b.w)
#define CFC_V4D_OUT(v) "=d"(v.a.x), "=d"(v.a.y), "=d"(v.b.x), "=d"(v.b.y)

// plain load (data this kernel may also write)
template <typename T>
__device__ __forceinline__ typename Vec<T>::V vld(const T *p);
template <>
__device__ __forceinline__ f8 vld<float>(const float *p) {
    f8 v;
    asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];" : CFC_V8F_OUT(v) : "l"(p) : "memory");
    return v;
}
template <>
__device__ __forceinline__ d4 vld<double>(const double *p) {
    d4 v;
    asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];" : CFC_V4D_OUT(v) : "l"(p) : "memory");
    return v;
}
// read-only path (data no thread of the kernel writes)
template <typename T>
__device__ __forceinline__ typename Vec<T>::V vldg(const T *p);
template <>
__device__ __forceinline__ f8 vldg<float>(const float *p) {
    f8 v;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];" : CFC_V8F_OUT(v) : "l"(p));
    return v;
}
template <>
__device__ __forceinline__ d4 vldg<double>(const double *p) {
    d4 v;
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : CFC_V4D_OUT(v) : "l"(p));
    return v;
}
// L2 only, coherent across blocks (data other blocks of this kernel wrote)
template <typename T>
__device__ __forceinline__ typename Vec<T>::V vldcg(const T *p);
template <>
__device__ __forceinline__ f8 vldcg<float>(const float *p) {
    f8 v;
    asm volatile("ld.global.cg.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];" : CFC_V8F_OUT(v) : "l"(p) : "memory");
    return v;
}
template <>
__device__ __forceinline__ d4 vldcg<double>(const double *p) {
    d4 v;
    asm volatile("ld.global.cg.v4.f64 {%0, %1, %2, %3}, [%4];" : CFC_V4D_OUT(v) : "l"(p) : "memory");
    return v;
}
#undef CFC_V8F_OUT
#undef CFC_V4D_OUT
__device__ __forceinline__ void vst_(float *p, const f8 &v) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v.a.x), "f"(v.a.y),
                 "f"(v.a.z), "f"(v.a.w), "f"(v.b.x), "f"(v.b.y), "f"(v.b.z), "f"(v.b.w)
                 : "memory");
}
__device__ __forceinline__ void vst_(double *p, const d4 &v) {
    asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(v.a.x), "d"(v.a.y), "d"(v.b.x), "d"(v.b.y)
                 : "memory");
}
template <typename T>
__device__ __forceinline__ void vst(T *p, const typename Vec<T>::V &v) {
    vst_(p, v);
}

// element access
__device__ __forceinline__ float &vel(f8 &v, int i) { return i < 4 ? (&v.a.x)[i] : (&v.b.x)[i - 4]; }
__device__ __forceinline__ double &vel(d4 &v, int i) { return i < 2 ? (&v.a.x)[i] : (&v.b.x)[i - 2]; }
__device__ __forceinline__ float vel(const f8 &v, int i) { return i < 4 ? (&v.a.x)[i] : (&v.b.x)[i - 4]; }
__device__ __forceinline__ double vel(const d4 &v, int i) { return i < 2 ? (&v.a.x)[i] : (&v.b.x)[i - 2]; }

// s += a * x
__device__ __forceinline__ void vfma(f8 &s, float a, const f8 &x) {
    s.a.x = fmaf(a, x.a.x, s.a.x);
    s.a.y = fmaf(a, x.a.y, s.a.y);
    s.a.z = fmaf(a, x.a.z, s.a.z);
    s.a.w = fmaf(a, x.a.w, s.a.w);
    s.b.x = fmaf(a, x.b.x, s.b.x);
    s.b.y = fmaf(a, x.b.y, s.b.y);
    s.b.z = fmaf(a, x.b.z, s.b.z);
    s.b.w = fmaf(a, x.b.w, s.b.w);
}
__device__ __forceinline__ void vfma(d4 &s, double a, const d4 &x) {
    s.a.x = fma(a, x.a.x, s.a.x);
    s.a.y = fma(a, x.a.y, s.a.y);
    s.b.x = fma(a, x.b.x, s.b.x);
    s.b.y = fma(a, x.b.y, s.b.y);
}
__device__ __forceinline__ f8 vadd(const f8 &x, const f8 &y) {
    return f8{make_float4(x.a.x + y.a.x, x.a.y + y.a.y, x.a.z + y.a.z, x.a.w + y.a.w),
              make_float4(x.b.x + y.b.x, x.b.y + y.b.y, x.b.z + y.b.z, x.b.w + y.b.w)};
}
__device__ __forceinline__ d4 vadd(const d4 &x, const d4 &y) {
    return d4{make_double2(x.a.x + y.a.x, x.a.y + y.a.y), make_double2(x.b.x + y.b.x, x.b.y + y.b.y)};
}

// FP32 <-> FP64 conversions with integer instructions (GB300 runs the
// hardware conversions on its narrow FP64 pipe).  Widening is exact; narrowing
// rounds to nearest, ties to even; zeros, subnormals, infinities, NaNs and
// out-of-range values take the hardware conversion.
__device__ __forceinline__ double f2d(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    return __longlong_as_double((long long)(((uint64_t)(u >> 31) << 63) | ((uint64_t)(e + 896u) << 52) |
                                            ((uint64_t)(u & 0x7fffffu) << 29)));
}
__device__ __forceinline__ float d2f(double d) {
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const int E = (int)((b >> 52) & 0x7ffu) - 1023;
    if (E < -126 || E > 127) return (float)d;
    uint32_t m = (uint32_t)((b >> 29) & 0x7fffffu);
    const uint32_t rem = (uint32_t)(b & 0x1fffffffu);
    uint32_t ex = (uint32_t)(E + 127);
    if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) {
        if (++m == 0x800000u) {
            m = 0u;
            if (++ex == 255u) return (float)d;
        }
    }
    return __uint_as_float(((uint32_t)(b >> 63) << 31) | (ex << 23) | m);
}
// x * 2^e by an integer add on the exponent field where the result stays a
// normal number (exact either way); zeros, subnormals, infinities, NaNs and
// results outside the normal range take ldexp.
__device__ __forceinline__ double scale2(double x, int e) {
    if (e == 0) return x;
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0 || ex == 0x7ff || ex + e <= 0 || ex + e >= 0x7ff) return ldexp(x, e);
    return __longlong_as_double(b + ((long long)e << 52));
}

template <typename T>
__device__ __forceinline__ T from_double(double d);
template <>
__device__ __forceinline__ float from_double<float>(double d) { return d2f(d); }
template <>
__device__ __forceinline__ double from_double<double>(double d) { return d; }
template <typename T>
__device__ __forceinline__ double to_double(T x);
template <>
__device__ __forceinline__ double to_double<float>(float x) { return f2d(x); }
template <>
__device__ __forceinline__ double to_double<double>(double x) { return x; }

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
// Per-column partial sums of this lane's columns, in registers:
// acc.add(r, v, x) adds x to reduction r of the lane's column v.
template <typename TA, int NR, int VW>
struct RAcc {
    TA a[NR > 0 ? NR : 1][VW];
    __device__ __forceinline__ void add(int r, int v, TA x) { a[r][v] += x; }
};

// Two-level, fixed-order cross-block reduction.  Blocks are grouped in teams
// of kTeam consecutive blocks; the last block of a team to arrive sums the
// team's partials (in block order), and the last team to arrive sums the
// team partials (in team order) and runs the per-column finalisation.  No
// block waits for another, and the order of every sum is fixed.
constexpr int kTeam = 32;
constexpr int kMaxTeams = 1024;  // P <= kTeam * kMaxTeams blocks per tile

struct RedBuf {
    double *part;            // [ntiles][P][NR*KT]
    double *team_part;       // [ntiles][kMaxTeams][NR*KT]
    uint32_t *counter;       // [kMaxTiles], zero between launches
    uint32_t *team_counter;  // [kMaxTiles][kMaxTeams], zero between launches
};

// acc holds this thread's partial sums in the kernel's arithmetic type (FP32
// partials over a few rows: FP64 per element would run on GB300's narrow
// FP64 pipe); the block, team and final stages add in FP64.
template <int KT, int NR, int VW, int G, typename TA, class Op>
__device__ __forceinline__ void block_reduce_finalize(RAcc<TA, NR, VW> &acc, RedBuf rb, Op &op) {
    constexpr int NO = NR * KT;
    constexpr int NWARP = kBlock / 32;
    __shared__ TA sm[NWARP][NO];
    __shared__ double fin[NO];
    __shared__ int is_last;
    // warp stage: the row groups of a warp own the same columns; add them up
    // with a fixed xor-shuffle tree, then group 0 of each warp stores them
    const int wl = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int v = 0; v < VW; ++v) {
            TA x = acc.a[r][v];
#pragma unroll
            for (int d = G; d < 32; d <<= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
            acc.a[r][v] = x;
        }
    if (wl < G) {
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int v = 0; v < VW; ++v) sm[wid][r * KT + wl * VW + v] = acc.a[r][v];
    }
    __syncthreads();
    const int tile = blockIdx.y;
    const int P = gridDim.x;
    // block stage: partial of this block, stored contiguously ([tile][block][output])
    for (int o = threadIdx.x; o < NO; o += blockDim.x) {
        TA s = TA(0);
#pragma unroll
        for (int g = 0; g < NWARP; ++g) s += sm[g][o];
        rb.part[((size_t)tile * P + blockIdx.x) * NO + o] = (double)s;
    }
    const int team = blockIdx.x / kTeam;
    const int team_size = min(kTeam, P - team * kTeam);
    const int nteams = (P + kTeam - 1) / kTeam;
    // one release per block: barrier, then a device-scope fence and the ticket
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t t = atomicAdd(rb.team_counter + tile * kMaxTeams + team, 1u);
        is_last = (t == (uint32_t)team_size - 1);
        if (is_last) __threadfence();
    }
    __syncthreads();
    if (!is_last) return;
    // team stage: one thread per output, the team's partials loaded together
    for (int o = threadIdx.x; o < NO; o += blockDim.x) {
        const double *src = rb.part + ((size_t)tile * P + team * kTeam) * NO + o;
        double v[kTeam];
#pragma unroll
        for (int i = 0; i < kTeam; ++i) v[i] = (i < team_size) ? __ldcg(src + (size_t)i * NO) : 0.0;
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < kTeam; ++i) t += v[i];
        rb.team_part[((size_t)tile * kMaxTeams + team) * NO + o] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        rb.team_counter[tile * kMaxTeams + team] = 0;
        __threadfence();
        const uint32_t t = atomicAdd(rb.counter + tile, 1u);
        is_last = (t == (uint32_t)nteams - 1);
        if (is_last) __threadfence();
    }
    __syncthreads();
    if (!is_last) return;
    for (int o = threadIdx.x; o < NO; o += blockDim.x) {
        const double *src = rb.team_part + (size_t)tile * kMaxTeams * NO + o;
        double t = 0.0;
        for (int t0 = 0; t0 < nteams; t0 += kTeam) {
            double v[kTeam];
#pragma unroll
            for (int i = 0; i < kTeam; ++i) v[i] = (t0 + i < nteams) ? __ldcg(src + (size_t)(t0 + i) * NO) : 0.0;
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

// edge weight in the kernel's arithmetic type; BF = true reads the BF16 copy
// (FP32 kernels only), which widens exactly (its 16 bits are the top half of
// the FP32 pattern)
template <typename T, bool BF>
__device__ __forceinline__ T lwk(const LevelView &A, int e) {
    if constexpr (BF) {
        static_assert(std::is_same<T, float>::value, "BF16 weights feed FP32 kernels");
        return __uint_as_float((uint32_t)__ldg(A.wbf + e) << 16);
    } else {
        return lw<T>(A, e);
    }
}

// sum_{e in [e0, e1)} w_e x_{col(e)} for this lane's columns.  Every round
// puts four neighbours (eight 16-byte gathers) in flight per lane, the last
// round of a row masked, so a row of length d costs ceil(d / 4) gather
// latencies.  In the FP64 kernels (16-lane groups at 64 columns) the G lanes
// of a row group first load up to G column indices and weights of the row in
// one coalesced access (lane l takes entry e + l) and hand them out by
// shuffles: measured 4-10 % faster there, and slower for the FP32 kernels,
// whose index loads are not what limits them.
template <typename T, bool BF, int G, class Op>
__device__ __forceinline__ typename Vec<T>::V row_sum(const LevelView &A, const Op &op, int e0, int e1, int c0,
                                                     int lane) {
    using V = typename Vec<T>::V;
    V s0 = vzero<V>(), s1 = vzero<V>();
    if constexpr (G >= 4 && std::is_same<T, double>::value) {
        // the group's lanes within the warp (G divides 32)
        const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << ((threadIdx.x & 31) & ~(G - 1));
        for (int eb = e0; eb < e1; eb += G) {
            const int my = eb + lane;
            const int jj = my < e1 ? __ldg(A.col + my) : -1;
            const T ww = my < e1 ? lwk<T, BF>(A, my) : T(0);
            const int cnt = min(G, e1 - eb);
            for (int u = 0; u < cnt; u += 4) {
                int j[4];
                T w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    j[q] = __shfl_sync(gmask, jj, u + q, G);  // u + q < G: cnt <= G and G % 4 == 0
                    w[q] = __shfl_sync(gmask, ww, u + q, G);
                }
                V x[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) x[q] = j[q] >= 0 ? op.gather(j[q], c0) : vzero<V>();
#pragma unroll
                for (int q = 0; q < 4; ++q) vfma(s0, w[q], x[q]);  // one accumulator: registers are the limit
            }
        }
        return s0;
    } else {
        for (int e = e0; e < e1; e += 4) {
            int j[4];
            T w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = e + u < e1;
                j[u] = ok ? __ldg(A.col + e + u) : -1;
                w[u] = ok ? lwk<T, BF>(A, e + u) : T(0);
            }
            V x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = j[u] >= 0 ? op.gather(j[u], c0) : vzero<V>();
            vfma(s0, w[0], x[0]);
            vfma(s1, w[1], x[1]);
            vfma(s0, w[2], x[2]);
            vfma(s1, w[3], x[3]);
        }
    }
    return vadd(s0, s1);
}

// An Op with a member `custom_sum(A, e0, e1, c0, lane)` computes the sum
// sum_{e in [e0, e1)} w_e x_{col(e)} itself (another arithmetic or operand
// layout); every other Op takes row_sum.
template <class Op, class = void>
struct has_custom_sum : std::false_type {};
template <class Op>
struct has_custom_sum<Op, std::void_t<decltype(&Op::custom_sum)>> : std::true_type {};

template <typename T, bool BF, int G, class Op>
__device__ __forceinline__ typename Vec<T>::V row_sum_of(const LevelView &A, const Op &op, int e0, int e1, int c0,
                                                        int lane) {
    if constexpr (has_custom_sum<Op>::value) return op.custom_sum(A, e0, e1, c0, lane);
    else return row_sum<T, BF, G>(A, op, e0, e1, c0, lane);
}

// ------------------------------------------------------------------ SpMM-like row operator
// Op provides:
//   V gather(int j, int c0) const              operand of node j, this lane's columns
//   Pre pre(int i, int c0) const               row i's own operands (loaded before the gathers)
//   void epi(int i, int c0, V s, Pre, RAcc &acc)  row i given s = sum_j w_ij x_j
//   void fin(int c, const double *sums)        per-column finalisation (NR > 0)
// With NR > 0 the per-column sums must not depend on which block finishes a
// long row, so long rows take their chunk sums from k_chunk_sums (launched
// just before) and are finished by the group that owns the row, like short
// rows (PRE = true).  Without reductions the last chunk to arrive finishes
// the row in the same launch (PRE = false).
template <typename T, int KT, class Op, bool BF = false>
__global__ void __launch_bounds__(kBlock, 4) k_chunk_sums(LevelView A, Op op, T *chunk_part, int ld_part) {
    constexpr int VW = Vec<T>::W;
    constexpr int G = KT / VW;
    constexpr int RPB = kBlock / G;
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int c0 = blockIdx.y * KT + lane * VW;
    const int slot = blockIdx.x * RPB + grp;
    if (slot >= A.n_chunks) return;
    const int ch = A.chunk_order ? __ldg(A.chunk_order + slot) : slot;
    const int i = __ldg(A.chunk_row + ch);
    const int e0 = __ldg(A.chunk_begin + ch);
    const int e1 = min(e0 + A.chunk, __ldg(A.rowptr + i + 1));
    vst<T>(chunk_part + (size_t)ch * ld_part + c0, row_sum_of<T, BF, G>(A, op, e0, e1, c0, lane));
}

// How rows longer than A.long_row are handled:
//   kLongLast  chunks are spread over groups; the group finishing a row's last
//              chunk (arrival counter) adds the chunk sums and finishes the row
//   kLongPre   chunk sums come from k_chunk_sums, launched just before, and the
//              row's own group finishes it, so per-column reductions do not
//              depend on scheduling
constexpr int kLongLast = 0, kLongPre = 1;

template <typename T, int KT, int NR, class Op, int MODE = kLongLast, bool BF = false>
__global__ void __launch_bounds__(kBlock, (NR >= 3 ? 3 : 4)) k_rowop(LevelView A, Op op, int nvb_short, int nvb_total,
                                                  T *chunk_part, int ld_part, RedBuf rb) {
    constexpr bool PRE = (MODE == kLongPre);
    using V = typename Vec<T>::V;
    constexpr int VW = Vec<T>::W;
    constexpr int G = KT / VW;
    constexpr int RPB = kBlock / G;
    constexpr int NRA = NR > 0 ? NR : 1;
    __shared__ int s_last[RPB];
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int tile = blockIdx.y;
    const int c0 = tile * KT + lane * VW;
    RAcc<T, NR, VW> acc;
#pragma unroll
    for (int r = 0; r < NRA; ++r)
#pragma unroll
        for (int v = 0; v < VW; ++v) acc.a[r][v] = T(0);

    const int nvb_long = nvb_total - nvb_short;  // chunk blocks come first: they start early
    for (int vb0 = blockIdx.x; vb0 < nvb_total; vb0 += gridDim.x) {
        const int vb = PRE ? vb0 : (vb0 < nvb_long ? nvb_short + vb0 : vb0 - nvb_long);
        if (vb < nvb_short) {
            const int slot = vb * RPB + grp;
            if (slot < A.n) {
                const int i = A.order ? __ldg(A.order + slot) : slot;
                const int e0 = __ldg(A.rowptr + i), e1 = __ldg(A.rowptr + i + 1);
                if (e1 - e0 <= A.long_row) {
                    const auto pr = op.pre(i, c0);  // own-row operands, in flight with the gathers
                    const V s = row_sum_of<T, BF, G>(A, op, e0, e1, c0, lane);
                    op.epi(i, c0, s, pr, acc);
                } else if (PRE) {
                    const auto pr = op.pre(i, c0);
                    const int li = __ldg(A.long_of_row + i);
                    const int f0 = __ldg(A.long_first + li), f1 = __ldg(A.long_first + li + 1);
                    V s = vzero<V>();
                    for (int f = f0; f < f1; ++f) s = vadd(s, vld<T>(chunk_part + (size_t)f * ld_part + c0));
                    op.epi(i, c0, s, pr, acc);
                }
            }
        } else {
            const int cslot = (vb - nvb_short) * RPB + grp;
            const bool has = cslot < A.n_chunks;
            const int ch = has ? (A.chunk_order ? __ldg(A.chunk_order + cslot) : cslot) : 0;
            int i = 0;
            if (has) {
                i = __ldg(A.chunk_row + ch);
                const int e0 = __ldg(A.chunk_begin + ch);
                const int e1 = min(e0 + A.chunk, __ldg(A.rowptr + i + 1));
                const V s = row_sum_of<T, BF, G>(A, op, e0, e1, c0, lane);
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
                op.epi(i, c0, s, op.pre(i, c0), acc);
                if (lane == 0) A.long_count[(size_t)li * kMaxTiles + tile] = 0;
            }
            __syncwarp();
        }
    }
    if constexpr (NR > 0) block_reduce_finalize<KT, NR, VW, G, T>(acc, rb, op);
}

// ------------------------------------------------------------------ row-local kernels (no gathers)
// Op provides: void row(int i, int c0, RAcc &acc) and fin (NR > 0).
template <typename T, int KT, int NR, class Op>
__global__ void __launch_bounds__(kBlock, 4) k_rows(int n, Op op, RedBuf rb) {
    constexpr int VW = Vec<T>::W;
    constexpr int G = KT / VW;
    constexpr int RPB = kBlock / G;
    constexpr int NRA = NR > 0 ? NR : 1;
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int c0 = blockIdx.y * KT + lane * VW;
    RAcc<T, NR, VW> acc;
#pragma unroll
    for (int r = 0; r < NRA; ++r)
#pragma unroll
        for (int v = 0; v < VW; ++v) acc.a[r][v] = T(0);
    for (int i = blockIdx.x * RPB + grp; i < n; i += gridDim.x * RPB) op.row(i, c0, acc);
    if constexpr (NR > 0) block_reduce_finalize<KT, NR, VW, G, T>(acc, rb, op);
}

}  // namespace cfc
