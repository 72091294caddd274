// Current-flow closeness estimators on top of the block solver:
//  * projection / JL estimator (Sec. 5.2, Algorithm 1): right-hand sides
//    Y = Q W^{1/2} B generated on the device, k solves, farness reduction;
//  * sampling estimator (Sec. 5.1): pivots by Floyd's algorithm on the
//    device, column solves, unbiased farness (n/k) sum_s d_ER(v, s);
//  * exact farness of small graphs from the dense pseudoinverse (Sec. 4).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace cfc {

namespace {

constexpr uint64_t kTagJL = 0x4A4C;
constexpr uint64_t kTagSample = 0x534D50;

// Philox4x64-10 (Salmon et al., SC'11): 10 rounds of two 64x64->128-bit
// multiplications, xor with the round key and a word permutation; the key
// advances by the Weyl constants after each round.
struct U64x4 {
    uint64_t v[4];
};
__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                               uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    return U64x4{{c0, c1, c2, c3}};
}

#define GRID_LOOP(i, count) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (count); i += (int64_t)gridDim.x * blockDim.x)

int grid_for(int64_t work, int threads = kBlock) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

// 32 sign bits of Q for rows cb*32 .. cb*32+31 of edge id e: row i uses bit
// (i % 64) of word (i % 256) / 64 of Philox(counter (e, i / 256, 0, 0), key (seed, JL))
__device__ __forceinline__ uint32_t jl_bits32(uint64_t e, int cb, uint64_t seed) {
    const int i0 = cb * 32;
    const U64x4 r = philox4x64_10(e, (uint64_t)(i0 / 256), 0, 0, seed, kTagJL);
    const uint64_t word = r.v[(i0 % 256) / 64];
    return (uint32_t)(word >> (i0 % 64));
}

// JL right-hand sides in exact fixed point.  Row u's terms
// sgn * sqrt(w_e) / sqrt(k) (sgn = +1 if u < v else -1, the orientation of B)
// are held as integers in units of 2^-S_u, with S_u chosen from the
// Cauchy-Schwarz bound
//   sum_e sqrt(w_e) / sqrt(k) <= sqrt(len_u * D_uu / k) < 2^(61 - S_u),
// so every column sum is an exact int64 addition (order-free: split rows
// combine without ordering concerns) and is rounded to FP64 once, by
// integer instructions.  Each term is rounded to 2^-(S_u + 1).
__device__ __forceinline__ int jl_row_shift(const int32_t *rowptr, const double *deg, int u, double inv_k) {
    const double x = (double)(rowptr[u + 1] - rowptr[u]) * deg[u] * inv_k;
    int ex = 0;
    frexp(isfinite(x) ? x : 1e300, &ex);  // x < 2^ex, so sqrt(x) < 2^ceil(ex / 2)
    const int half = ex >= 0 ? (ex + 1) / 2 : -((-ex) / 2);
    return 61 - half;
}
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// a * 2^e2 rounded to the nearest FP64 (ties to even) with integer
// instructions only; the result must be a normal number
__device__ __forceinline__ double i64_scaled_to_double(long long a, int e2) {
    if (a == 0) return 0.0;
    const unsigned long long sign = a < 0 ? (1ull << 63) : 0ull;
    unsigned long long m = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
    const int lz = __clzll((long long)m);
    int ex = 63 - lz + e2;  // exponent of the leading bit
    m <<= lz;               // leading bit at position 63
    unsigned long long mant = m >> 11;  // 53 bits
    const unsigned long long rem = m & 0x7FFull;
    if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
        mant += 1ull;
        if (mant >> 53) {
            mant >>= 1;
            ex += 1;
        }
    }
    return __longlong_as_double((long long)(sign | ((unsigned long long)(ex + 1023) << 52) |
                                            (mant & ((1ull << 52) - 1))));
}

// Row u's fixed-point scale 2^S_u / sqrt(k) and its unit term round(2^S_u / sqrt(k)).
struct JlRow {
    double sc;
    long long t1;
};
__device__ __forceinline__ JlRow jl_row(const int32_t *rowptr, const double *deg, int u, double inv_k,
                                        double inv_sqrt_k) {
    const double sc = pow2(jl_row_shift(rowptr, deg, u, inv_k)) * inv_sqrt_k;
    return JlRow{sc, llrint(sc)};
}

// The JL sums of 32 units per warp, a unit being a row of at most kJlRow
// entries (k_jl_short) or a kJlChunk-entry chunk of a longer row
// (k_jl_chunks); lane l owns unit l.  The warp first stages the units'
// entries in shared memory, one unit at a time with the lanes over its
// entries (coalesced loads of the edge ids, columns and weights), as the
// fixed-point terms a_e = sgn * round(sqrt(w_e) * 2^S_u / sqrt(k)) (a unit
// weight skips the square root: sqrt(1) = 1 exactly).  Then every lane sums
// its own unit, for each 32-row block of Q in turn:
//   acc_q = sum_e (bit q of the block's Philox word for e) ? -a_e : a_e.
constexpr int kJlWarps = 2;  // warps per block
struct JlStage {
    int32_t id[32][33];
    long long t[32][33];
};

template <class Emit>
__device__ __forceinline__ void jl_warp_units(const int32_t *eid, const int32_t *col, const double *w, int u,
                                              const JlRow &jr, int e0, int len, int ncb, int cb_off, uint64_t seed,
                                              JlStage &st, Emit emit) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < 32; ++r) {
        const int e0r = __shfl_sync(0xffffffffu, e0, r), lr = __shfl_sync(0xffffffffu, len, r);
        const int ur = __shfl_sync(0xffffffffu, u, r);
        const double scr = __shfl_sync(0xffffffffu, jr.sc, r);
        const long long t1r = __shfl_sync(0xffffffffu, jr.t1, r);
        if (lane < lr) {
            const int e = e0r + lane;
            const double we = __ldg(w + e);
            long long t = we == 1.0 ? t1r : llrint(sqrt(we) * scr);
            if (ur > __ldg(col + e)) t = -t;
            st.id[lane][r] = __ldg(eid + e);
            st.t[lane][r] = t;
        }
    }
    __syncwarp();
    for (int cb = 0; cb < ncb; ++cb) {
        long long acc[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = 0;
        for (int j = 0; j < len; ++j) {
            const long long t = st.t[j][lane];
            const uint32_t bits = jl_bits32((uint64_t)(uint32_t)st.id[j][lane], cb_off + cb, seed);
#pragma unroll
            for (int q = 0; q < 32; ++q) acc[q] += ((bits >> q) & 1u) ? -t : t;
        }
        emit(cb, acc);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(32 * kJlWarps) k_jl_short(const int32_t *__restrict__ rowptr,
                                                           const int32_t *__restrict__ eid,
                                                           const int32_t *__restrict__ col,
                                                           const double *__restrict__ w,
                                                           const double *__restrict__ deg, int32_t n, int k, int ld,
                                                           int cb_off, uint64_t seed, double inv_k,
                                                           double inv_sqrt_k, double *__restrict__ Y) {
    __shared__ JlStage stage[kJlWarps];
    JlStage &st = stage[threadIdx.x >> 5];
    const int ncb = (ld + 31) / 32;
    const int64_t nwarp = (n + 31) / 32;
    for (int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wg < nwarp;
         wg += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int u = (int)(wg * 32 + (threadIdx.x & 31));
        int e0 = 0, len = 0;
        JlRow jr{0.0, 0};
        if (u < n) {
            e0 = rowptr[u];
            len = rowptr[u + 1] - e0;
            if (len > kJlRow) len = 0;  // split rows: k_jl_chunks
            jr = jl_row(rowptr, deg, u, inv_k, inv_sqrt_k);
        }
        const bool mine = u < n && rowptr[u + 1] - e0 <= kJlRow;
        const int sh = mine ? -jl_row_shift(rowptr, deg, u, inv_k) : 0;
        jl_warp_units(eid, col, w, u, jr, e0, len, ncb, cb_off, seed, st,
                      [&](int cb, const long long(&acc)[32]) {
                          if (!mine) return;
#pragma unroll
                          for (int q = 0; q < 32; ++q) {
                              const int c = cb * 32 + q;
                              if (c < ld) Y[(size_t)u * ld + c] = c < k ? i64_scaled_to_double(acc[q], sh) : 0.0;
                          }
                      });
    }
}

__global__ void __launch_bounds__(32 * kJlWarps) k_jl_chunks(const int32_t *__restrict__ rowptr,
                                                            const int32_t *__restrict__ eid,
                                                            const int32_t *__restrict__ col,
                                                            const double *__restrict__ w,
                                                            const double *__restrict__ deg,
                                                            const int32_t *__restrict__ chunk_row,
                                                            const int32_t *__restrict__ chunk_begin,
                                                            int32_t n_chunks, int ld, int cb_off, uint64_t seed,
                                                            double inv_k, double inv_sqrt_k,
                                                            long long *__restrict__ part) {
    __shared__ JlStage stage[kJlWarps];
    JlStage &st = stage[threadIdx.x >> 5];
    const int ncb = (ld + 31) / 32;
    const int64_t nwarp = (n_chunks + 31) / 32;
    for (int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wg < nwarp;
         wg += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int ch = (int)(wg * 32 + (threadIdx.x & 31));
        int u = 0, e0 = 0, len = 0;
        JlRow jr{0.0, 0};
        if (ch < n_chunks) {
            u = chunk_row[ch];
            e0 = chunk_begin[ch];
            len = min(kJlChunk, rowptr[u + 1] - e0);
            jr = jl_row(rowptr, deg, u, inv_k, inv_sqrt_k);
        }
        jl_warp_units(eid, col, w, u, jr, e0, len, ncb, cb_off, seed, st,
                      [&](int cb, const long long(&acc)[32]) {
                          if (ch >= n_chunks) return;
#pragma unroll
                          for (int q = 0; q < 32; ++q) part[((size_t)ch * ncb + cb) * 32 + q] = acc[q];
                      });
    }
}

// one thread per (long row, column): exact sum of the row's chunk partials
__global__ void k_jl_long(const int32_t *__restrict__ rowptr, const double *__restrict__ deg,
                          const int32_t *__restrict__ chunk_row, const int32_t *__restrict__ long_first,
                          int32_t n_long, int k, int ld, double inv_k, const long long *__restrict__ part,
                          double *__restrict__ Y) {
    const int ncb = (ld + 31) / 32;
    GRID_LOOP(t, (int64_t)n_long * ld) {
        const int li = (int)(t / ld), c = (int)(t - (int64_t)li * ld);
        const int f0 = long_first[li], f1 = long_first[li + 1];
        const int u = chunk_row[f0];
        long long acc = 0;
        for (int f = f0; f < f1; ++f) acc += part[((size_t)f * ncb + c / 32) * 32 + (c & 31)];
        Y[(size_t)u * ld + c] = c < k ? i64_scaled_to_double(acc, -jl_row_shift(rowptr, deg, u, inv_k)) : 0.0;
    }
}

// per-column sums S_i = sum_w Z_wi and T_i = sum_w Z_wi^2 (FP64, fixed order):
// block partials, then one warp per column
constexpr int kRedRows = 8;
__global__ void k_colsum2_part(const double *__restrict__ Z, int64_t n, int k, int ld, double *__restrict__ part) {
    // blockDim = (32, kRedRows); grid = (P, ceil(k/32))
    const int c = blockIdx.y * 32 + threadIdx.x;
    double s = 0.0, t = 0.0;
    if (c < k) {
        for (int64_t i = (int64_t)blockIdx.x * kRedRows + threadIdx.y; i < n; i += (int64_t)gridDim.x * kRedRows) {
            const double z = Z[i * ld + c];
            s += z;
            t += z * z;
        }
    }
    __shared__ double ss[kRedRows][32], tt[kRedRows][32];
    ss[threadIdx.y][threadIdx.x] = s;
    tt[threadIdx.y][threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.y == 0 && c < k) {
        double a = 0.0, b = 0.0;
        for (int r = 0; r < kRedRows; ++r) {
            a += ss[r][threadIdx.x];
            b += tt[r][threadIdx.x];
        }
        part[((size_t)c * gridDim.x + blockIdx.x) * 2 + 0] = a;
        part[((size_t)c * gridDim.x + blockIdx.x) * 2 + 1] = b;
    }
}

__global__ void k_colsum2_final(const double *__restrict__ part, int P, int k, double *__restrict__ S,
                                double *__restrict__ T) {
    const int c = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (c >= k) return;
    double a = 0.0, b = 0.0;
    for (int p = lane; p < P; p += 32) {
        a += part[((size_t)c * P + p) * 2 + 0];
        b += part[((size_t)c * P + p) * 2 + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        S[c] = a;
        T[c] = b;
    }
}

// f(v) = sum_i [n Z_vi^2 - 2 Z_vi S_i + T_i]: one warp per query node
__global__ void k_jl_farness(const double *__restrict__ Z, int64_t n, int k, int ld, const double *__restrict__ S,
                             const double *__restrict__ T, const int32_t *__restrict__ nodes, int q,
                             double *__restrict__ f) {
    const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (t >= q) return;
    const int64_t v = nodes[t];
    double a = 0.0;
    for (int i = lane; i < k; i += 32) {
        const double z = Z[v * ld + i];
        a += (double)n * z * z - 2.0 * z * S[i] + T[i];
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) f[t] = a;
}

__global__ void k_check_nodes(const int32_t *__restrict__ nodes, int q, int32_t n, int32_t *__restrict__ bad) {
    GRID_LOOP(t, q) {
        if (nodes[t] < 0 || nodes[t] >= n) atomicOr(bad, 1);
    }
}

// Floyd's algorithm (Bentley & Floyd 1987), one warp: step s draws
// t uniform in [0, n - kk + s] and inserts t unless present, else the top
// value n - kk + s.  Membership is tested by all lanes in parallel.
__global__ void k_floyd(int64_t n, int kk, uint64_t seed, int32_t *__restrict__ out) {
    extern __shared__ int32_t S[];
    const int lane = threadIdx.x;
    for (int s = 0; s < kk; ++s) {
        const uint64_t j = (uint64_t)(n - kk + s);
        int32_t tval = 0;
        if (lane == 0) {
            const U64x4 r = philox4x64_10((uint64_t)s, 0, 0, 0, seed, kTagSample);
            tval = (int32_t)__umul64hi(r.v[0], j + 1);
        }
        tval = __shfl_sync(0xffffffffu, tval, 0);
        bool found = false;
        for (int u = lane; u < s; u += 32) found |= (S[u] == tval);
        found = __any_sync(0xffffffffu, found);
        if (lane == 0) S[s] = found ? (int32_t)j : tval;
        __syncwarp();
    }
    // ascending order: rank of each element (values are distinct)
    for (int a = lane; a < kk; a += 32) {
        const int32_t x = S[a];
        int rank = 0;
        for (int b = 0; b < kk; ++b) rank += (S[b] < x) ? 1 : 0;
        out[rank] = x;
    }
}

// column c of B is e_{U_c}, U = [pivots..., query nodes...]
__global__ void k_unit_columns(const int32_t *__restrict__ piv, int kk, const int32_t *__restrict__ nodes, int q,
                               int ld, double *__restrict__ B) {
    GRID_LOOP(c, kk + q) {
        const int u = c < kk ? piv[c] : nodes[c - kk];
        B[(size_t)u * ld + c] = 1.0;
    }
}

// f^(v) = (n/k) sum_s [x_v(v) - x_v(s) - x_s(v) + x_s(s)]: one warp per query node
// (n / kk) sum_s d(v, s), d(v, s) = x_v(v) - x_v(s) - x_s(v) + x_s(s) (Proposition 1,
// with pair solves written as single-node solves): the pivot solutions are
// columns cs0 + i of XS (leading dimension ldS), the query nodes' columns
// cv0 + t of XV (ldV); a warp per query node, its lanes over the pivots
__global__ void k_sample_farness(const double *__restrict__ XS, int ldS, int cs0, const double *__restrict__ XV,
                                 int ldV, int cv0, int64_t n, const int32_t *__restrict__ piv, int kk,
                                 const int32_t *__restrict__ nodes, int q, double *__restrict__ f) {
    const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (t >= q) return;
    const int64_t v = nodes[t];
    const int cv = cv0 + t;
    const double xvv = XV[v * ldV + cv];
    double a = 0.0;
    for (int i = lane; i < kk; i += 32) {
        const int64_t sv = piv[i];
        if (sv == v) continue;  // d_ER(v, v) = 0
        a += xvv - XV[sv * ldV + cv] - XS[v * ldS + cs0 + i] + XS[sv * ldS + cs0 + i];
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) f[t] = a * ((double)n / kk);
}

// exact: f(v) = n L+_vv + tr L+ with L+ = M^{-1} - J/(alpha n), M = L + alpha J/n
__global__ void k_trace(const double *__restrict__ Minv, int n, double *__restrict__ tr) {
    __shared__ double sm[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += Minv[(size_t)i * n + i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) tr[0] = sm[0];
}

__global__ void k_exact_farness(const double *__restrict__ Minv, int n, double alpha, const double *__restrict__ tr,
                                double *__restrict__ f, double *__restrict__ c) {
    GRID_LOOP(v, n) {
        const double lpv = Minv[(size_t)v * n + v] - 1.0 / (alpha * n);
        const double trl = tr[0] - 1.0 / alpha;
        const double fv = (double)n * lpv + trl;
        f[v] = fv;
        if (c) c[v] = (double)(n - 1) / fv;
    }
}

void copy_out(double *dst, const double *dsrc, size_t count, cudaStream_t s) {
    const cudaMemcpyKind kind = is_device_pointer(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CFC_CUDA(cudaMemcpyAsync(dst, dsrc, count * sizeof(double), kind, s));
}

void copy_out_i32(int32_t *dst, const int32_t *dsrc, size_t count, cudaStream_t s) {
    const cudaMemcpyKind kind = is_device_pointer(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CFC_CUDA(cudaMemcpyAsync(dst, dsrc, count * sizeof(int32_t), kind, s));
}

const int32_t *nodes_to_device(const int32_t *nodes, int q, int32_t n, DBuf<int32_t> &tmp, cudaStream_t s) {
    CFC_REQUIRE(nodes, LAP_EINVAL, "nodes must not be NULL");
    const int32_t *d = nodes;
    if (!is_device_pointer(nodes)) {
        tmp.alloc(q, s);
        CFC_CUDA(cudaMemcpyAsync(tmp.get(), nodes, q * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        d = tmp.get();
    }
    DBuf<int32_t> bad(1, s);
    bad.zero(s);
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_check_nodes, grid_for(q), kBlock, 0, d, q, n, bad.get());
    int32_t hb = 0;
    CFC_CUDA(cudaMemcpyAsync(&hb, bad.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CFC_CUDA(cudaStreamSynchronize(s));
    CFC_REQUIRE(hb == 0, LAP_EINVAL, "query node out of range");
    return d;
}

}  // namespace

void jl_rhs(lap_hierarchy *h, int k_total, int row0, int k, int ld, uint64_t seed, double *Y, cudaStream_t s) {
    const Level &L = h->lv[0];
    const int n = L.n;
    const int ncb = (ld + 31) / 32;
    // the scale (and the fixed-point bound) are those of the full k_total-row Q
    const double inv_sqrt_k = 1.0 / std::sqrt((double)k_total), inv_k = 1.0 / k_total;
    const int cb_off = row0 / 32;
    // entries: eid, col, weight (16 B); rows: rowptr, degree; the block of Y
    const double bytes = (double)L.nnz * 16 + (double)n * 12 + (double)n * ld * 8;
    CFC_LAUNCH(LAP_KF_CFC, s, bytes, k_jl_short, grid_for((int64_t)n, 32 * kJlWarps), 32 * kJlWarps, 0, L.rowptr.get(),
               h->eid.get(), L.col.get(), L.w64.get(), L.deg64.get(), n, k, ld, cb_off, seed, inv_k, inv_sqrt_k, Y);
    if (L.jl_n_chunks > 0) {  // rows longer than kJlRow: chunk partials, then exact sums per row
        DBuf<long long> part((size_t)L.jl_n_chunks * ncb * 32, s);
        CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_jl_chunks, grid_for((int64_t)L.jl_n_chunks, 32 * kJlWarps), 32 * kJlWarps, 0,
                   L.rowptr.get(), h->eid.get(), L.col.get(), L.w64.get(), L.deg64.get(), L.jl_chunk_row.get(),
                   L.jl_chunk_begin.get(), L.jl_n_chunks, ld, cb_off, seed, inv_k, inv_sqrt_k, part.get());
        CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_jl_long, grid_for((int64_t)L.jl_n_long * ld, 128), 128, 0,
                   L.rowptr.get(), L.deg64.get(), L.jl_chunk_row.get(), L.jl_long_first.get(), L.jl_n_long, k, ld,
                   inv_k, part.get(), Y);
    }
}

lap_status_t farness_jl(lap_hierarchy *h, int32_t k, double eps, uint64_t seed, int32_t q, const int32_t *nodes,
                        double *farness, const lap_solve_opts_t &o, cudaStream_t s) {
    const int64_t n = h->lv[0].n;
    if (k <= 0) {
        CFC_REQUIRE(eps > 0 && std::isfinite(eps), LAP_EINVAL, "k <= 0 needs eps > 0");
        k = (int32_t)std::ceil(std::log((double)n) / (eps * eps));
    }
    CFC_REQUIRE(k >= 1 && k <= 4096, LAP_EINVAL, "need 1 <= k <= 4096");
    return farness_jl_rows(h, k, 0, k, seed, q, nodes, farness, o, s);
}

lap_status_t farness_jl_rows(lap_hierarchy *h, int32_t k_total, int32_t row0, int32_t k, uint64_t seed, int32_t q,
                             const int32_t *nodes, double *farness, const lap_solve_opts_t &o, cudaStream_t s) {
    const int64_t n = h->lv[0].n;
    CFC_REQUIRE(k_total >= 1, LAP_EINVAL, "need k_total >= 1");
    CFC_REQUIRE(row0 >= 0 && row0 % 32 == 0, LAP_EINVAL, "row_begin must be a multiple of 32");
    CFC_REQUIRE(k >= 1 && k <= 4096 && (int64_t)row0 + k <= k_total, LAP_EINVAL,
                "need 1 <= row_count <= 4096 and row_begin + row_count <= k_total");
    CFC_REQUIRE(q >= 1 && q <= n, LAP_EINVAL, "need 1 <= q <= n");
    CFC_REQUIRE(farness, LAP_EINVAL, "farness must not be NULL");
    DBuf<int32_t> ntmp;
    const int32_t *dn = nodes_to_device(nodes, q, (int32_t)n, ntmp, s);
    // Y is generated straight into the solver's padded layout; its columns sum
    // to zero (B 1 = 0), and the farness sums are unchanged by a constant
    // added to a column of Z, so the solve skips both mean projections
    const int ld = solve_ld(k, o);
    DBuf<double> Y((size_t)n * ld, s), Z((size_t)n * ld, s);
    jl_rhs(h, k_total, row0, k, ld, seed, Y.get(), s);
    lap_status_t st = solve_multi_direct(h, k, Y.get(), Z.get(), o, s, nullptr);
    if (st != LAP_OK && st != LAP_ENOCONV) return st;
    const int P = std::min<int64_t>(2 * num_sms_public(), (n + kRedRows - 1) / kRedRows);
    DBuf<double> part((size_t)k * P * 2, s), S(k, s), T(k, s), f(q, s);
    dim3 g1(P, (k + 31) / 32), b1(32, kRedRows);
    CFC_LAUNCH(LAP_KF_CFC, s, (double)n * k * 8, k_colsum2_part, g1, b1, 0, Z.get(), n, k, ld, part.get());
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_colsum2_final, (k + 7) / 8, 256, 0, part.get(), P, k, S.get(), T.get());
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_jl_farness, (q + 7) / 8, 256, 0, Z.get(), n, k, ld, S.get(), T.get(), dn, q,
               f.get());
    copy_out(farness, f.get(), q, s);
    CFC_CUDA(cudaStreamSynchronize(s));
    return st;
}

// Algorithm 1 step 4 on a given block Z (n x k, row-major, device)
lap_status_t farness_from_solution(int64_t n, int32_t k, const double *Z, int32_t q, const int32_t *nodes,
                                   double *farness, cudaStream_t s) {
    CFC_REQUIRE(n >= 2 && n < (int64_t(1) << 31), LAP_EINVAL, "need 2 <= n < 2^31");
    CFC_REQUIRE(k >= 1 && k <= 4096, LAP_EINVAL, "need 1 <= k <= 4096");
    CFC_REQUIRE(q >= 1 && q <= n, LAP_EINVAL, "need 1 <= q <= n");
    CFC_REQUIRE(Z && farness, LAP_EINVAL, "Z and farness must not be NULL");
    CFC_REQUIRE(is_device_pointer(Z), LAP_EINVAL, "Z must be a device pointer");
    noalloc_prepare();  // the allocation-free variant's scratch, on this device
    DBuf<int32_t> ntmp;
    const int32_t *dn = nodes_to_device(nodes, q, (int32_t)n, ntmp, s);
    const int P = (int)std::min<int64_t>(2 * num_sms_public(), (n + kRedRows - 1) / kRedRows);
    DBuf<double> part((size_t)k * P * 2, s), S(k, s), T(k, s), f(q, s);
    dim3 g1(P, (k + 31) / 32), b1(32, kRedRows);
    CFC_LAUNCH(LAP_KF_CFC, s, (double)n * k * 8, k_colsum2_part, g1, b1, 0, Z, n, k, k, part.get());
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_colsum2_final, (k + 7) / 8, 256, 0, part.get(), P, k, S.get(), T.get());
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_jl_farness, (q + 7) / 8, 256, 0, Z, n, k, k, S.get(), T.get(), dn, q, f.get());
    copy_out(farness, f.get(), q, s);
    CFC_CUDA(cudaStreamSynchronize(s));
    return LAP_OK;
}

// ---------------------------------------------------------------- allocation-free variant
// Some callers cannot allocate device memory at the point where they need a
// farness (code running inside an allocator or out-of-memory handler, a
// process under a hard device-memory cap, or a stream that must not
// synchronise with the allocator).  cfc_farness_from_solution_noalloc serves
// them: its scratch is the array below, reserved on every GPU that loads this
// library until the process exits.  It holds the per-block column partials
// (at most kNoAllocMaxP blocks of kNoAllocMaxK columns) and the column sums
// S, T: 2 MiB + 4 KiB.  Every call overwrites what it uses before reading it;
// calls that overlap on one GPU share the array and race.
constexpr int kNoAllocMaxK = 256;
constexpr int kNoAllocMaxP = 512;
constexpr size_t kNoAllocDoubles = (size_t)kNoAllocMaxP * kNoAllocMaxK * 2 + 2 * kNoAllocMaxK;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

namespace {
// The host cannot use g_noalloc_scratch's name as a device address: the
// address is looked up once per device, with that device current.
double *noalloc_scratch() {
    static std::mutex mu;
    static double *ptr[128] = {};
    int dev = 0;
    CFC_CUDA(cudaGetDevice(&dev));
    CFC_REQUIRE(dev >= 0 && dev < 128, LAP_ECUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!ptr[dev]) {
        void *p = nullptr;
        CFC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        ptr[dev] = static_cast<double *>(p);
    }
    return ptr[dev];
}

}  // namespace

void noalloc_prepare() { noalloc_scratch(); }

namespace {
// k_jl_farness with a range check: a node outside [0, n) gets NaN
__global__ void k_jl_farness_checked(const double *__restrict__ Z, int64_t n, int k, const double *__restrict__ S,
                                     const double *__restrict__ T, const int32_t *__restrict__ nodes, int q,
                                     double *__restrict__ f) {
    const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (t >= q) return;
    const int64_t v = nodes[t];
    if (v < 0 || v >= n) {
        if (lane == 0) f[t] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    double a = 0.0;
    for (int i = lane; i < k; i += 32) {
        const double z = Z[v * k + i];
        a += (double)n * z * z - 2.0 * z * S[i] + T[i];
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) f[t] = a;
}
}  // namespace

lap_status_t farness_from_solution_noalloc(int64_t n, int32_t k, const double *Z, int32_t q, const int32_t *nodes,
                                           double *farness, cudaStream_t s) {
    CFC_REQUIRE(n >= 2 && n < (int64_t(1) << 31), LAP_EINVAL, "need 2 <= n < 2^31");
    CFC_REQUIRE(k >= 1, LAP_EINVAL, "need k >= 1");
    CFC_REQUIRE(k <= kNoAllocMaxK, LAP_EBUDGET,
                "cfc_farness_from_solution_noalloc: k exceeds its fixed scratch (at most 256 columns)");
    CFC_REQUIRE(q >= 1, LAP_EINVAL, "need q >= 1");
    CFC_REQUIRE(Z && nodes && farness, LAP_EINVAL, "Z, nodes and farness must not be NULL");
    CFC_REQUIRE(is_device_pointer(Z) && is_device_pointer(nodes) && is_device_pointer(farness), LAP_EINVAL,
                "Z, nodes and farness must be device pointers");
    double *scr = noalloc_scratch();
    double *part = scr;
    double *S = scr + (size_t)kNoAllocMaxP * kNoAllocMaxK * 2;
    double *T = S + kNoAllocMaxK;
    const int P = (int)std::min<int64_t>(std::min(2 * num_sms_public(), kNoAllocMaxP), (n + kRedRows - 1) / kRedRows);
    dim3 g1(P, (k + 31) / 32), b1(32, kRedRows);
    CFC_LAUNCH(LAP_KF_CFC, s, (double)n * k * 8, k_colsum2_part, g1, b1, 0, Z, n, k, k, part);
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_colsum2_final, (k + 7) / 8, 256, 0, part, P, k, S, T);
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_jl_farness_checked, (q + 7) / 8, 256, 0, Z, n, k, S, T, nodes, q, farness);
    return LAP_OK;
}

void sample_pivots(int64_t n, int32_t kk, uint64_t seed, int32_t *dpiv, cudaStream_t s) {
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_floyd, 1, 32, (size_t)kk * sizeof(int32_t), n, kk, seed, dpiv);
}

lap_status_t pivots_api(lap_hierarchy *h, int32_t kk, uint64_t seed, int32_t *pivots, cudaStream_t s) {
    const int64_t n = h->lv[0].n;
    CFC_REQUIRE(kk >= 1 && kk <= n && kk <= 8192, LAP_EINVAL, "need 1 <= n_pivots <= min(n, 8192)");
    CFC_REQUIRE(pivots, LAP_EINVAL, "pivots must not be NULL");
    DBuf<int32_t> d(kk, s);
    sample_pivots(n, kk, seed, d.get(), s);
    copy_out_i32(pivots, d.get(), kk, s);
    CFC_CUDA(cudaStreamSynchronize(s));
    return LAP_OK;
}

lap_status_t farness_sampled(lap_hierarchy *h, int32_t kk, uint64_t seed, int32_t q, const int32_t *nodes,
                             double *farness, const lap_solve_opts_t &o, cudaStream_t s, lap_solve_info_t *info) {
    const int64_t n = h->lv[0].n;
    CFC_REQUIRE(kk >= 1 && kk <= n, LAP_EINVAL, "need 1 <= n_pivots <= n");
    CFC_REQUIRE(q >= 1 && q <= n, LAP_EINVAL, "need 1 <= q <= n");
    CFC_REQUIRE(kk + q <= 4096, LAP_EBUDGET, "n_pivots + q must be <= 4096 columns");
    CFC_REQUIRE(farness, LAP_EINVAL, "farness must not be NULL");
    DBuf<int32_t> ntmp;
    const int32_t *dn = nodes_to_device(nodes, q, (int32_t)n, ntmp, s);
    const int kc = kk + q;
    DBuf<int32_t> piv(kk, s);
    sample_pivots(n, kk, seed, piv.get(), s);
    DBuf<double> B((size_t)n * kc, s), X((size_t)n * kc, s), f(q, s);
    B.zero(s);
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_unit_columns, grid_for(kc), kBlock, 0, piv.get(), kk, dn, q, kc, B.get());
    lap_status_t st = solve_multi(h, kc, B.get(), X.get(), o, s, info);
    if (st != LAP_OK && st != LAP_ENOCONV) return st;
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_sample_farness, (q + 7) / 8, 256, 0, X.get(), kc, 0, X.get(), kc, kk, n,
               piv.get(), kk, dn, q, f.get());
    copy_out(farness, f.get(), q, s);
    CFC_CUDA(cudaStreamSynchronize(s));
    return st;
}

lap_status_t pivot_solutions(lap_hierarchy *h, int32_t kk, uint64_t seed, double *XS, int32_t *piv,
                             const lap_solve_opts_t &o, cudaStream_t s, lap_solve_info_t *info) {
    const int64_t n = h->lv[0].n;
    CFC_REQUIRE(kk >= 1 && kk <= n && kk <= 4096, LAP_EINVAL, "need 1 <= n_pivots <= min(n, 4096)");
    sample_pivots(n, kk, seed, piv, s);
    DBuf<double> B((size_t)n * kk, s);
    B.zero(s);
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_unit_columns, grid_for(kk), kBlock, 0, piv, kk, (const int32_t *)nullptr, 0,
               kk, B.get());
    const lap_status_t st = solve_multi(h, kk, B.get(), XS, o, s, info);
    CFC_CUDA(cudaStreamSynchronize(s));
    return st;
}

lap_status_t farness_sampled_resident(lap_hierarchy *h, const double *XS, const int32_t *piv, int32_t kk, int32_t q,
                                      const int32_t *nodes, double *farness, const lap_solve_opts_t &o,
                                      cudaStream_t s) {
    const int64_t n = h->lv[0].n;
    CFC_REQUIRE(q >= 1 && q <= n && q <= 4096, LAP_EINVAL, "need 1 <= q <= min(n, 4096)");
    CFC_REQUIRE(farness, LAP_EINVAL, "farness must not be NULL");
    DBuf<int32_t> ntmp;
    const int32_t *dn = nodes_to_device(nodes, q, (int32_t)n, ntmp, s);
    DBuf<double> B((size_t)n * q, s), X((size_t)n * q, s), f(q, s);
    B.zero(s);
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_unit_columns, grid_for(q), kBlock, 0, (const int32_t *)nullptr, 0, dn, q, q,
               B.get());
    lap_status_t st = solve_multi(h, q, B.get(), X.get(), o, s, nullptr);
    if (st != LAP_OK && st != LAP_ENOCONV) return st;
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_sample_farness, (q + 7) / 8, 256, 0, XS, kk, 0, X.get(), q, 0, n, piv, kk,
               dn, q, f.get());
    copy_out(farness, f.get(), q, s);
    CFC_CUDA(cudaStreamSynchronize(s));
    return st;
}

// Several sampling queries on one hierarchy as one block solve: each query's
// pivot columns (drawn with its own seed) and node columns sit side by side,
// one solve covers them all, and each query's farness comes from its own
// columns (Sec. 5.1, Proposition 1).  A column's solution does not depend on
// the other columns of the block (per-column PCG scalars and stopping tests,
// reductions in a fixed order per column), so at the same tile width a query
// gets the same bits alone and in a batch.  With kp > 0 every query uses the
// resident pivot set (XS, piv_res) and contributes only its node columns.
lap_status_t farness_sampled_batch(lap_hierarchy *h, const SampledQuery *qs, int nq, const double *XS,
                                   const int32_t *piv_res, int32_t kp, const lap_solve_opts_t &o, cudaStream_t s) {
    const int64_t n = h->lv[0].n;
    CFC_REQUIRE(nq >= 1, LAP_EINVAL, "empty batch");
    std::vector<int64_t> cbase(nq), pbase(nq), qbase(nq);
    int64_t cols = 0, npiv = 0, nnodes = 0;
    for (int i = 0; i < nq; ++i) {
        CFC_REQUIRE((kp > 0) == (qs[i].kk == 0) && qs[i].q >= 1, LAP_EINVAL, "mixed batch");
        cbase[i] = cols;
        pbase[i] = npiv;
        qbase[i] = nnodes;
        cols += qs[i].kk + qs[i].q;
        npiv += qs[i].kk;
        nnodes += qs[i].q;
    }
    CFC_REQUIRE(cols <= 4096, LAP_EBUDGET, "a batch holds at most 4096 columns");
    std::vector<int32_t> hn(nnodes);
    for (int i = 0; i < nq; ++i) std::memcpy(hn.data() + qbase[i], qs[i].nodes, qs[i].q * sizeof(int32_t));
    DBuf<int32_t> dn(nnodes, s), piv(std::max<int64_t>(npiv, 1), s);
    CFC_CUDA(cudaMemcpyAsync(dn.get(), hn.data(), nnodes * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DBuf<double> B((size_t)n * cols, s), X((size_t)n * cols, s), f(nnodes, s);
    B.zero(s);
    for (int i = 0; i < nq; ++i) {
        if (qs[i].kk > 0) sample_pivots(n, qs[i].kk, qs[i].seed, piv.get() + pbase[i], s);
        CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_unit_columns, grid_for(qs[i].kk + qs[i].q), kBlock, 0, piv.get() + pbase[i],
                   qs[i].kk, dn.get() + qbase[i], qs[i].q, (int)cols, B.get() + cbase[i]);
    }
    const lap_status_t st = solve_multi(h, (int32_t)cols, B.get(), X.get(), o, s, nullptr);
    if (st != LAP_OK && st != LAP_ENOCONV) return st;
    for (int i = 0; i < nq; ++i) {
        const int q = qs[i].q;
        if (kp > 0)
            CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_sample_farness, (q + 7) / 8, 256, 0, XS, kp, 0, X.get(), (int)cols,
                       (int)cbase[i], n, piv_res, kp, dn.get() + qbase[i], q, f.get() + qbase[i]);
        else
            CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_sample_farness, (q + 7) / 8, 256, 0, X.get(), (int)cols, (int)cbase[i],
                       X.get(), (int)cols, (int)(cbase[i] + qs[i].kk), n, piv.get() + pbase[i], qs[i].kk,
                       dn.get() + qbase[i], q, f.get() + qbase[i]);
    }
    std::vector<double> hf(nnodes);
    CFC_CUDA(cudaMemcpyAsync(hf.data(), f.get(), nnodes * sizeof(double), cudaMemcpyDeviceToHost, s));
    CFC_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < nq; ++i) std::memcpy(qs[i].farness, hf.data() + qbase[i], qs[i].q * sizeof(double));
    return st;
}

lap_status_t exact_small(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const double *w,
                         double *farness, double *closeness, cudaStream_t s) {
    CFC_REQUIRE(n >= 2, LAP_EINVAL, "need n >= 2");
    CFC_REQUIRE(n <= 16384, LAP_EBUDGET, "cfc_exact_small holds n x n doubles: n <= 16384");
    CFC_REQUIRE(farness, LAP_EINVAL, "farness must not be NULL");
    Csr64 g;
    ingest(n, m, src, dst, w, s, g);
    DBuf<double> M((size_t)n * n, s), tr(1, s), f(n, s), c(n, s);
    // the constant mode of M gets an eigenvalue of the order of the weights
    const double alpha = std::ldexp(1.0, max_exponent(g.w.get(), std::max<int64_t>(g.nnz, 1), s));
    build_dense(g.rowptr.get(), g.col.get(), g.w.get(), g.deg.get(), (int32_t)n, alpha, M.get(), s);
    DBuf<int> flag(1, s);
    flag.zero(s);
    if (n <= 160) dense_spd_inverse_small(M.get(), (int)n, flag.get(), s);
    else dense_spd_inverse_large(M.get(), (int)n, flag.get(), s);
    int hf = 0;
    CFC_CUDA(cudaMemcpyAsync(&hf, flag.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    CFC_CUDA(cudaStreamSynchronize(s));
    // connectivity was checked at ingest: a non-positive pivot is FP64 losing definiteness
    CFC_REQUIRE(hf == 0, LAP_ENOCONV,
                "the dense FP64 factorization of L + alpha J/n lost positive definiteness (weights too far apart)");
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_trace, 1, 1024, 0, M.get(), (int)n, tr.get());
    CFC_LAUNCH(LAP_KF_CFC, s, 0.0, k_exact_farness, grid_for(n), kBlock, 0, M.get(), (int)n, alpha, tr.get(),
               f.get(), closeness ? c.get() : nullptr);
    copy_out(farness, f.get(), n, s);
    if (closeness) copy_out(closeness, c.get(), n, s);
    CFC_CUDA(cudaStreamSynchronize(s));
    return LAP_OK;
}

}  // namespace cfc
