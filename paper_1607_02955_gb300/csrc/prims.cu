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

// One block of 1024 threads scans up to kSingleMax values: each thread sums a
// contiguous run, the run totals are scanned across the block, and each
// thread writes its run's prefix (in may alias out).  One launch instead of
// the three of the tiled scan, for inputs small enough that one SM reading
// them beats three launches (measured: at 2^17 values it is several times
// slower than the tiled scan).
constexpr int kSingleThreads = 1024;
constexpr int64_t kSingleMax = int64_t(1) << 14;

template <typename T>
__global__ void __launch_bounds__(kSingleThreads) k_scan_single(const T *in, T *out, int64_t n) {
    __shared__ T warp_tot[kSingleThreads / 32];
    const int64_t per = (n + kSingleThreads - 1) / kSingleThreads;
    const int64_t b = (int64_t)threadIdx.x * per, e = min(n, b + per);
    T s = 0;
    for (int64_t i = b; i < e; ++i) s += in[i];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    T run = (wid ? warp_tot[wid - 1] : T(0)) + x - s;
    for (int64_t i = b; i < e; ++i) {
        const T v = in[i];
        out[i] = run;
        run += v;
    }
}

// Second pass of a two-launch scan: block b adds the sum of the tile totals
// before it (read and reduced by the block itself, in a fixed order: at most
// kPrefixMaxTiles of them) to its tile's local scan.
constexpr int64_t kPrefixMaxTiles = 4096;
template <typename T>
__global__ void k_scan_add_prefix(T *out, const T *sums, int64_t n) {
    __shared__ T warp_tot[kScanThreads / 32];
    const int b = blockIdx.x;
    T part = 0;
    for (int j = threadIdx.x; j < b; j += kScanThreads) part += sums[j];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) warp_tot[wid] = part;
    __syncthreads();
    T off = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) off += warp_tot[w];
    const int64_t base = (int64_t)b * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        const int64_t j = base + i;
        if (j < n) out[j] += off;
    }
}

// in-place capable recursive scan; returns nothing (total computed by caller)
template <typename T>
void scan_rec(const T *in, T *out, int64_t n, cudaStream_t s) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (n > kScanTile && n <= kSingleMax) {
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_scan_single<T>, 1, kSingleThreads, 0, in, out, n);
        return;
    }
    if (nb <= 1) {
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_scan_tile<T>, 1, kScanThreads, 0, in, out, (T *)nullptr, n);
        return;
    }
    DBuf<T> sums(nb, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_scan_tile<T>, (unsigned)nb, kScanThreads, 0, in, out, sums.get(), n);
    if (nb <= kPrefixMaxTiles) {  // two launches: each tile sums the totals before it
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_scan_add_prefix<T>, (unsigned)nb, kScanThreads, 0, out, sums.get(), n);
        return;
    }
    scan_rec<T>(sums.get(), sums.get(), nb, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_scan_add<T>, (unsigned)nb, kScanThreads, 0, out, sums.get(), n);
}

// total = last input + last output, read back with one synchronisation (the
// last input is saved on the device first: the scan may run in place)
template <typename T>
int64_t scan_impl(const T *in, T *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return 0;
    DBuf<T> last(2, s);
    CFC_CUDA(cudaMemcpyAsync(last.get(), in + n - 1, sizeof(T), cudaMemcpyDeviceToDevice, s));
    scan_rec<T>(in, out, n, s);
    CFC_CUDA(cudaMemcpyAsync(last.get() + 1, out + n - 1, sizeof(T), cudaMemcpyDeviceToDevice, s));
    T h[2] = {0, 0};
    CFC_CUDA(cudaMemcpyAsync(h, last.get(), 2 * sizeof(T), cudaMemcpyDeviceToHost, s));
    CFC_CUDA(cudaStreamSynchronize(s));
    return (int64_t)h[0] + (int64_t)h[1];
}

// ------------------------------------------------------------------ radix sort
constexpr int kRsThreads = 256;
constexpr int kRsRounds = 16;
constexpr int kRsTile = kRsThreads * kRsRounds;
constexpr int kRsWarps = kRsThreads / 32;

template <int RB>
__global__ void k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, int32_t *__restrict__ hist,
                          int nblocks) {
    constexpr int NB = 1 << RB;
    __shared__ uint32_t h[NB];
    for (int d = threadIdx.x; d < NB; d += kRsThreads) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsRounds; ++r) {
        int64_t i = base + r * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (NB - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < NB; d += kRsThreads) hist[(int64_t)d * nblocks + blockIdx.x] = (int32_t)h[d];
}

// Stable scatter of RB-bit digits: the tile is consumed in rounds of 256
// consecutive keys; within a round a key's rank is (keys of its digit in
// earlier warps) + (lower lanes of its warp with the same digit).  Each
// warp's leader of a digit group records the group's size, advances the
// digit's running offset and clears its record, so the work per round
// follows the keys, not the number of digits.
template <int RB>
__global__ void k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
                             const int32_t *__restrict__ offs, int nblocks) {
    constexpr int NB = 1 << RB;
    __shared__ uint32_t run[NB];
    __shared__ uint32_t wcnt[kRsWarps][NB];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int d = tid; d < NB; d += kRsThreads) {
        run[d] = (uint32_t)offs[(int64_t)d * nblocks + blockIdx.x];
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) wcnt[w][d] = 0;
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = 0; r < kRsRounds; ++r) {
        const int64_t i = base + r * kRsThreads + tid;
        const bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0;
        uint32_t val = valid ? vin[i] : 0;
        const uint32_t digit = valid ? (uint32_t)((key >> shift) & (NB - 1)) : (uint32_t)NB;
        const uint32_t peers = __match_any_sync(0xffffffffu, digit);
        const uint32_t rank = __popc(peers & lt);
        const bool leader = valid && lane == (__ffs(peers) - 1);
        if (leader) wcnt[wid][digit] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = run[digit] + rank;
            for (int w = 0; w < wid; ++w) pos += wcnt[w][digit];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        if (leader) {
            atomicAdd(&run[digit], (uint32_t)__popc(peers));
            wcnt[wid][digit] = 0;
        }
        __syncthreads();
    }
}

template <int RB>
void radix_passes(uint64_t *&ka, uint32_t *&va, uint64_t *&kb, uint32_t *&vb, int32_t *hist, int64_t n,
                  int nblocks, int bits, cudaStream_t s) {
    const int passes = (bits + RB - 1) / RB;
    for (int p = 0; p < passes; ++p) {
        const int shift = RB * p;
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_rs_hist<RB>, nblocks, kRsThreads, 0, ka, n, shift, hist, nblocks);
        scan_rec<int32_t>(hist, hist, ((int64_t)1 << RB) * nblocks, s);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_rs_scatter<RB>, nblocks, kRsThreads, 0, ka, va, kb, vb, n, shift, hist,
                   nblocks);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
}

__global__ void k_save_last(const int32_t *last_in, int64_t *total) { *total = *last_in; }
__global__ void k_add_last(const int32_t *last_out, int64_t *total) { *total += *last_out; }

}  // namespace

void scan_exclusive_i32_total(const int32_t *in, int32_t *out, int64_t n, int64_t *d_total, cudaStream_t s) {
    if (n <= 0) {
        CFC_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int64_t), s));
        return;
    }
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_save_last, 1, 1, 0, in + n - 1, d_total);
    scan_rec<int32_t>(in, out, n, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_add_last, 1, 1, 0, out + n - 1, d_total);
}

int64_t *pinned_small() {
    thread_local int64_t *buf = nullptr;
    if (!buf) CFC_CUDA(cudaMallocHost((void **)&buf, 64 * sizeof(int64_t)));
    return buf;
}

void read_totals(const int64_t *d_totals, int count, int64_t *host, cudaStream_t s) {
    int64_t *pin = pinned_small();
    CFC_CUDA(cudaMemcpyAsync(pin, d_totals, count * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CFC_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i) host[i] = pin[i];
}

int64_t scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, s);
}
void scan_exclusive_i32_async(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    if (n > 0) scan_rec<int32_t>(in, out, n, s);
}
int64_t scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, s);
}

void radix_sort_pairs(uint64_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return;
    CFC_REQUIRE(n < (int64_t(1) << 31), LAP_EBUDGET, "sort too large");
    const int nblocks = (int)((n + kRsTile - 1) / kRsTile);
    // digit width 8..10 bits: the fewest passes, then the smallest histogram
    int rb = 8;
    for (int c = 9; c <= 10; ++c)
        if ((bits + c - 1) / c < (bits + rb - 1) / rb) rb = c;
    DBuf<uint64_t> k2(n, s);
    DBuf<uint32_t> v2(n, s);
    DBuf<int32_t> hist(((size_t)1 << rb) * nblocks, s);
    uint64_t *ka = keys, *kb = k2.get();
    uint32_t *va = vals, *vb = v2.get();
    if (rb == 8)
        radix_passes<8>(ka, va, kb, vb, hist.get(), n, nblocks, bits, s);
    else if (rb == 9)
        radix_passes<9>(ka, va, kb, vb, hist.get(), n, nblocks, bits, s);
    else
        radix_passes<10>(ka, va, kb, vb, hist.get(), n, nblocks, bits, s);
    if (ka != keys) {
        CFC_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        CFC_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

}  // namespace cfc
