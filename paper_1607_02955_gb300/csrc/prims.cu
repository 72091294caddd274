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
// LSD radix sort of (64-bit key, 32-bit value) pairs, 8-bit digits.  A block
// owns a tile of consecutive pairs (16384, or 4096 for small sorts).  Its
// scatter stages the tile in shared memory in digit order (stable) and then
// writes each digit's run to its place in one pass over the staged tile, so
// the global writes come in runs (64 pairs per digit on average for the large
// tile) instead of single 8-byte stores.
constexpr int kRsBits = 8;
constexpr int kRsDigits = 1 << kRsBits;
constexpr int kRsThreads = 1024;
constexpr int kRsWarps = kRsThreads / 32;
// R rounds of 32 pairs per warp: a tile of 32 x 32 x R pairs (16 384 at R = 16
// for large sorts, 4 096 at R = 4 when the large tiles would not fill the GPU)
template <int R>
__host__ __device__ constexpr int rs_tile() { return kRsWarps * 32 * R; }
template <int R>
constexpr size_t rs_smem() {
    return (size_t)rs_tile<R>() * 12                    // staged keys and values
           + (size_t)kRsWarps * kRsDigits * 2           // per-warp digit counts, then offsets (u16)
           + (size_t)3 * kRsDigits * 4;                 // tile offsets, global starts, totals
}

template <int R>
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                                                        int32_t *__restrict__ hist, int nblocks) {
    constexpr int kRsTile = rs_tile<R>();
    __shared__ uint32_t h[kRsDigits];
    for (int d = threadIdx.x; d < kRsDigits; d += kRsThreads) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < kRsTile / kRsThreads; ++r) {
        const int64_t i = base + r * kRsThreads + threadIdx.x;
        const uint32_t digit = i < n ? (uint32_t)((keys[i] >> shift) & (kRsDigits - 1)) : (uint32_t)kRsDigits;
        // one shared-memory atomic per distinct digit of the warp (few digits on the high passes)
        const uint32_t peers = __match_any_sync(0xffffffffu, digit);
        if (digit < kRsDigits && lane == __ffs(peers) - 1) atomicAdd(&h[digit], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRsDigits; d += kRsThreads)
        hist[(int64_t)d * nblocks + blockIdx.x] = (int32_t)h[d];
}

// offs[d * nblocks + b]: exclusive scan of the histograms in digit-major
// order, i.e. where block b's run of digit d starts in the output.
template <int R>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t *__restrict__ kin,
                                                           const uint32_t *__restrict__ vin,
                                                           uint64_t *__restrict__ kout,
                                                           uint32_t *__restrict__ vout, int64_t n, int shift,
                                                           const int32_t *__restrict__ offs, int nblocks) {
    constexpr int kRsTile = rs_tile<R>();
    constexpr int kRsRounds = R;
    constexpr int kRsSub = 32 * R;
    extern __shared__ __align__(16) unsigned char rs_smem_raw[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(rs_smem_raw);            // [kRsTile]
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kRsTile);           // [kRsTile]
    uint16_t *wpos = reinterpret_cast<uint16_t *>(sv + kRsTile);         // [kRsWarps][kRsDigits]
    uint32_t *loc = reinterpret_cast<uint32_t *>(wpos + kRsWarps * kRsDigits);  // [kRsDigits]
    uint32_t *gst = loc + kRsDigits;                                     // [kRsDigits]
    uint32_t *tot = gst + kRsDigits;                                     // [kRsDigits]
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    const int cnt = (int)((n - base) < (int64_t)kRsTile ? (n - base) : (int64_t)kRsTile);
    for (int t = tid; t < kRsWarps * kRsDigits; t += kRsThreads) wpos[t] = 0;
    for (int d = tid; d < kRsDigits; d += kRsThreads) gst[d] = (uint32_t)offs[(int64_t)d * nblocks + blockIdx.x];
    __syncthreads();

    // A: each warp ranks its sub-tile: rank = earlier pairs of the same digit
    // in this sub-tile (rounds in order, lanes in order)
    uint16_t *wc = wpos + wid * kRsDigits;
    const int sub = wid * kRsSub;
    // only the ranks stay in registers; the keys are read again (from L2) when staged
    uint32_t rank2[kRsRounds / 2];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int li = sub + r * 32 + lane;
        const bool valid = li < cnt;
        const uint64_t key = valid ? kin[base + li] : 0ull;
        const uint32_t digit = valid ? (uint32_t)((key >> shift) & (kRsDigits - 1)) : (uint32_t)kRsDigits;
        const uint32_t peers = __match_any_sync(0xffffffffu, digit);
        const uint32_t before = valid ? (uint32_t)wc[digit] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wc[digit] = (uint16_t)(before + __popc(peers));
        __syncwarp();
        const uint32_t rk = before + __popc(peers & lt);
        if (r & 1) rank2[r >> 1] |= rk << 16;
        else rank2[r >> 1] = rk;
    }
    __syncthreads();

    // B: per digit, the counts of the warps become offsets within the tile
    for (int d = tid; d < kRsDigits; d += kRsThreads) {
        uint32_t run = 0;
        for (int w = 0; w < kRsWarps; ++w) {
            const uint32_t c = wpos[w * kRsDigits + d];
            wpos[w * kRsDigits + d] = (uint16_t)run;
            run += c;
        }
        tot[d] = run;
    }
    __syncthreads();
    if (tid < 32) {  // exclusive scan of the 256 digit totals by one warp
        uint32_t v[kRsDigits / 32], sum = 0;
#pragma unroll
        for (int q = 0; q < kRsDigits / 32; ++q) {
            v[q] = tot[lane * (kRsDigits / 32) + q];
            sum += v[q];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        uint32_t run = inc - sum;
#pragma unroll
        for (int q = 0; q < kRsDigits / 32; ++q) {
            loc[lane * (kRsDigits / 32) + q] = run;
            run += v[q];
        }
    }
    __syncthreads();

    // C: stage the pairs in digit order
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int li = sub + r * 32 + lane;
        if (li < cnt) {
            const uint64_t key = kin[base + li];
            const uint32_t digit = (uint32_t)((key >> shift) & (kRsDigits - 1));
            const uint32_t rk = (r & 1) ? (rank2[r >> 1] >> 16) : (rank2[r >> 1] & 0xffffu);
            const uint32_t L = loc[digit] + wpos[wid * kRsDigits + digit] + rk;
            sk[L] = key;
            sv[L] = vin[base + li];
        }
    }
    __syncthreads();

    // D: write out; consecutive staged pairs of one digit go to consecutive places
    for (int L = tid; L < cnt; L += kRsThreads) {
        const uint64_t k = sk[L];
        const uint32_t digit = (uint32_t)((k >> shift) & (kRsDigits - 1));
        const int64_t g = (int64_t)gst[digit] + (L - (int)loc[digit]);
        kout[g] = k;
        vout[g] = sv[L];
    }
}

template <int R>
void radix_passes(uint64_t *&ka, uint32_t *&va, uint64_t *&kb, uint32_t *&vb, int32_t *hist, int64_t n,
                  int nblocks, int bits, cudaStream_t s) {
    // the staged tile needs more than the default 48 KB of shared memory (set on the current device)
    CFC_CUDA(cudaFuncSetAttribute(k_rs_scatter<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs_smem<R>()));
    const int passes = (bits + kRsBits - 1) / kRsBits;
    for (int p = 0; p < passes; ++p) {
        const int shift = kRsBits * p;
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_rs_hist<R>, nblocks, kRsThreads, 0, ka, n, shift, hist, nblocks);
        scan_rec<int32_t>(hist, hist, (int64_t)kRsDigits * nblocks, s);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_rs_scatter<R>, nblocks, kRsThreads, rs_smem<R>(), ka, va, kb, vb, n, shift,
                   hist, nblocks);
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
    // large tiles once they give every SM two blocks, small ones below
    const bool big = (n + rs_tile<16>() - 1) / rs_tile<16>() >= 2 * num_sms_public();
    const int tile = big ? rs_tile<16>() : rs_tile<4>();
    const int nblocks = (int)((n + tile - 1) / tile);
    DBuf<uint64_t> k2(n, s);
    DBuf<uint32_t> v2(n, s);
    DBuf<int32_t> hist((size_t)kRsDigits * nblocks, s);
    uint64_t *ka = keys, *kb = k2.get();
    uint32_t *va = vals, *vb = v2.get();
    if (big) radix_passes<16>(ka, va, kb, vb, hist.get(), n, nblocks, bits, s);
    else radix_passes<4>(ka, va, kb, vb, hist.get(), n, nblocks, bits, s);
    if (ka != keys) {
        CFC_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        CFC_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

}  // namespace cfc
