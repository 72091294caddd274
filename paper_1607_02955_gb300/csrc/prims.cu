// Device primitives: exclusive prefix sums and a stable LSD radix sort of
// (key, value) pairs.  Used by graph ingest (CSR construction, merging of
// repeated edges) and by the Galerkin contraction of the hierarchy.
#include "internal.h"

namespace cfc {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread; returns the block total.
template <typename T>
__device__ T block_exclusive_scan(T v, T *warp_tot, T &excl) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T t = lane < (kScanThreads / 32) ? warp_tot[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < (kScanThreads / 32)) warp_tot[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    T base = wid ? warp_tot[wid - 1] : T(0);
    T total = warp_tot[kScanThreads / 32 - 1];
    excl = base + x - v;
    __syncthreads();
    return total;
}

template <typename T>
__global__ void k_scan_tile(const T *in, T *out, T *sums, int64_t n) {  // in may alias out
    __shared__ T warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : T(0);
        s += v[i];
    }
    T excl;
    T total = block_exclusive_scan<T>(s, warp_tot, excl);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = excl;
        excl += v[i];
    }
    if (threadIdx.x == 0 && sums) sums[blockIdx.x] = total;
}

template <typename T>
__global__ void k_scan_add(T *out, const T *offs, int64_t n) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const T o = offs[blockIdx.x];
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t j = base + i;
        if (j < n) out[j] += o;
    }
}

// in-place capable recursive scan; returns nothing (total computed by caller)
template <typename T>
void scan_rec(const T *in, T *out, int64_t n, cudaStream_t s) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb <= 1) {
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_scan_tile<T>, 1, kScanThreads, 0, in, out, (T *)nullptr, n);
        return;
    }
    DBuf<T> sums(nb, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_scan_tile<T>, (unsigned)nb, kScanThreads, 0, in, out, sums.get(), n);
    scan_rec<T>(sums.get(), sums.get(), nb, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_scan_add<T>, (unsigned)nb, kScanThreads, 0, out, sums.get(), n);
}

template <typename T>
int64_t scan_impl(const T *in, T *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return 0;
    T last_in = 0, last_out = 0;
    CFC_CUDA(cudaMemcpyAsync(&last_in, in + n - 1, sizeof(T), cudaMemcpyDeviceToHost, s));
    CFC_CUDA(cudaStreamSynchronize(s));
    scan_rec<T>(in, out, n, s);
    CFC_CUDA(cudaMemcpyAsync(&last_out, out + n - 1, sizeof(T), cudaMemcpyDeviceToHost, s));
    CFC_CUDA(cudaStreamSynchronize(s));
    return (int64_t)last_out + (int64_t)last_in;
}

// ------------------------------------------------------------------ radix sort
constexpr int kRsThreads = 256;
constexpr int kRsRounds = 16;
constexpr int kRsTile = kRsThreads * kRsRounds;
constexpr int kRsWarps = kRsThreads / 32;

__global__ void k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, int32_t *__restrict__ hist,
                          int nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsRounds; ++r) {
        int64_t i = base + r * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = (int32_t)h[threadIdx.x];
}

// Stable scatter: the tile is consumed in rounds of 256 consecutive keys;
// within a round a key's rank is (keys of its digit in earlier warps) +
// (lower lanes of its warp with the same digit).
__global__ void k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
                             const int32_t *__restrict__ offs, int nblocks) {
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[kRsWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    run[tid] = (uint32_t)offs[(int64_t)tid * nblocks + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = 0; r < kRsRounds; ++r) {
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const int64_t i = base + r * kRsThreads + tid;
        const bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0;
        uint32_t val = valid ? vin[i] : 0;
        const uint32_t digit = valid ? (uint32_t)((key >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, digit);
        const uint32_t rank = __popc(peers & lt);
        if (valid && lane == (__ffs(peers) - 1)) wcnt[wid][digit] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = run[digit] + rank;
            for (int w = 0; w < wid; ++w) pos += wcnt[w][digit];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        uint32_t add = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) add += wcnt[w][tid];
        run[tid] += add;
        __syncthreads();
    }
}

}  // namespace

int64_t scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, s);
}
int64_t scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, s);
}

void radix_sort_pairs(uint64_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return;
    CFC_REQUIRE(n < (int64_t(1) << 31), LAP_EBUDGET, "sort too large");
    const int nblocks = (int)((n + kRsTile - 1) / kRsTile);
    DBuf<uint64_t> k2(n, s);
    DBuf<uint32_t> v2(n, s);
    DBuf<int32_t> hist((size_t)256 * nblocks, s);
    uint64_t *ka = keys, *kb = k2.get();
    uint32_t *va = vals, *vb = v2.get();
    const int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_rs_hist, nblocks, kRsThreads, 0, ka, n, shift, hist.get(), nblocks);
        scan_rec<int32_t>(hist.get(), hist.get(), (int64_t)256 * nblocks, s);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_rs_scatter, nblocks, kRsThreads, 0, ka, va, kb, vb, n, shift,
                   hist.get(), nblocks);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        CFC_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        CFC_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

}  // namespace cfc
