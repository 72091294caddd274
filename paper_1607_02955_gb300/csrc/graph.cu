// Graph ingest (Sec. 2, Sec. 6.3): edge list -> symmetric CSR of the
// adjacency weights of G, with self-loops dropped, edge directions ignored
// and repeated pairs merged (weights summed: parallel conductances), the
// degree vector D_ii = sum_j w_ij, the undirected edge id of each CSR entry
// (lexicographic rank of (min, max), the orientation used for the incidence
// matrix B of Sec. 5.2) and the connectivity check (Sec. 2 assumes G
// connected).
#include "internal.h"

namespace cfc {

namespace {

// One pass over the input edges: validation, and two CSR candidates per
// kept edge, (u, v) and (v, u) with key = row * 2^b + col, at slots 2e and
// 2e + 1.  A dropped edge (self-loop or invalid) gets the key 2^(2b) - 1 in
// both slots, above every real key (a real key is at most
// (n-1) 2^b + (n-2) < 2^(2b) - 1), so it sorts to the end.  The kept count
// and an invalid-edge flag come back in out[0..1].
__global__ void k_validate_emit(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                                const double *__restrict__ w, int64_t m, int32_t n, int b,
                                uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                unsigned long long *__restrict__ out) {
    const uint64_t drop = (uint64_t(1) << (2 * b)) - 1;
    unsigned long long kept = 0;
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e], v = dst[e];
        bool ok = u >= 0 && v >= 0 && u < n && v < n;
        if (w) {  // conductances (Sec. 2), in a range whose sums and products FP64 holds
            const double x = w[e];
            ok = ok && x >= 1e-150 && x <= 1e150;
        }
        bad = bad || !ok;
        const bool keep = ok && u != v;
        kept += keep ? 1ull : 0ull;
        keys[2 * e] = keep ? ((uint64_t)(uint32_t)u << b) | (uint32_t)v : drop;
        keys[2 * e + 1] = keep ? ((uint64_t)(uint32_t)v << b) | (uint32_t)u : drop;
        vals[2 * e] = (uint32_t)e;
        vals[2 * e + 1] = (uint32_t)e;
    }
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_down_sync(0xffffffffu, kept, o);
    const bool anybad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        if (kept) atomicAdd(out + 1, kept);
        if (anybad) atomicOr(out, 1ull);
    }
}

__global__ void k_heads(const uint64_t *__restrict__ keys, int64_t len, int32_t *__restrict__ head) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// one thread per merged entry: sums the weights of its run of equal keys in
// sorted (stable) order.  The sort is stable and both directions of an input
// edge carry its index, so the runs of (u, v) and (v, u) start with the same
// input edge e: src_edge[o] = e for every merged entry, and tab[e] = o for
// the upper one (row < col), which gives each lower entry its mirror.
__global__ void k_merge(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                        const int32_t *__restrict__ head, const int32_t *__restrict__ hpos, int64_t len, int b,
                        const double *__restrict__ w, int32_t *__restrict__ col, double *__restrict__ wout,
                        int32_t *__restrict__ rowcnt, int32_t *__restrict__ row_of, int32_t *__restrict__ src_edge,
                        int32_t *__restrict__ tab) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        if (!head[i]) continue;
        const uint64_t key = keys[i];
        double s = 0.0;
        for (int64_t j = i; j < len && keys[j] == key; ++j) s += w ? w[vals[j]] : 1.0;
        const int32_t o = hpos[i];
        const int32_t r = (int32_t)(key >> b);
        const int32_t c = (int32_t)(key & ((uint64_t(1) << b) - 1));
        col[o] = c;
        row_of[o] = r;
        wout[o] = s;
        src_edge[o] = (int32_t)vals[i];
        if (r < c) tab[vals[i]] = o;
        atomicAdd(&rowcnt[r], 1);
    }
}

__global__ void k_finish_rowptr(int32_t *rowptr, int32_t n, int32_t nnz) {
    if (blockIdx.x == 0 && threadIdx.x == 0) rowptr[n] = nnz;
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

__global__ void k_upper_flags(const int32_t *__restrict__ row_of, const int32_t *__restrict__ col, int64_t nnz,
                              int32_t *__restrict__ up) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x)
        up[i] = row_of[i] < col[i] ? 1 : 0;
}

// the lower entry (r, c), r > c, takes the id of its mirror (c, r): the upper
// entry that k_merge recorded for the same input edge
__global__ void k_mirror_eid(const int32_t *__restrict__ row_of, const int32_t *__restrict__ col,
                             const int32_t *__restrict__ src_edge, const int32_t *__restrict__ tab, int64_t nnz,
                             int32_t *__restrict__ eid) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x)
        if (row_of[i] > col[i]) eid[i] = eid[tab[src_edge[i]]];
}

// ---------------------------------------------------------------- connectivity
// Lock-free union-find with hooking of the larger root under the smaller by
// compare-and-swap and path halving (the scheme of Jaiganesh & Burtscher's
// ECL-CC).  Parent pointers only ever point to smaller ids, so every find
// terminates.
__device__ __forceinline__ int32_t uf_find(int32_t *par, int32_t x) {
    while (true) {
        const int32_t p = __ldcg(par + x);
        if (p == x) return x;
        const int32_t gp = __ldcg(par + p);
        if (gp != p) __stcg(par + x, gp);
        x = gp;
    }
}

// start from a forest: every node points to its smallest neighbour when
// that is smaller than itself (rows are sorted, so it is the first entry)
__global__ void k_uf_init(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, int32_t *par,
                          int32_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e0 = rowptr[i];
        const int32_t j = (e0 < rowptr[i + 1]) ? col[e0] : (int32_t)i;
        par[i] = j < (int32_t)i ? j : (int32_t)i;
    }
}

// Afforest's order (Sutton, Ben-Nun, Bar-Barak, IPDPS 2018): first hook every
// node to its first `rounds` neighbours, then let the rest of the entries
// only of nodes outside the largest tree so far hook.  Correct whichever tree
// is skipped: the entries are symmetric, so an edge between the skipped tree
// and another one is seen from the other side.
__device__ __forceinline__ void uf_hook(int32_t *par, int32_t u, int32_t v) {
    int32_t ru = uf_find(par, u), rv = uf_find(par, v);
    while (ru != rv) {
        if (ru < rv) {
            const int32_t t = ru;
            ru = rv;
            rv = t;
        }
        const int32_t old = atomicCAS(par + ru, ru, rv);
        if (old == ru) break;
        ru = uf_find(par, ru);
        rv = uf_find(par, rv);
    }
}

__global__ void k_uf_sample(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, int32_t n,
                            int r, int32_t *par) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = rowptr[i] + r;
        if (e < rowptr[i + 1]) uf_hook(par, (int32_t)i, col[e]);
    }
}

__global__ void k_uf_compress(int32_t *par, int32_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        __stcg(par + i, uf_find(par, (int32_t)i));
}

// the most frequent root among 32 evenly spaced nodes (one warp)
__global__ void k_uf_giant(const int32_t *par, int32_t n, int32_t *giant) {
    const int lane = threadIdx.x & 31;
    const int32_t r = uf_find(const_cast<int32_t *>(par), (int32_t)(((int64_t)n * lane) / 32));
    const uint32_t peers = __match_any_sync(0xffffffffu, r);
    int c = __popc(peers), best = r;
    for (int o = 16; o > 0; o >>= 1) {
        const int oc = __shfl_xor_sync(0xffffffffu, c, o), ob = __shfl_xor_sync(0xffffffffu, best, o);
        if (oc > c || (oc == c && ob < best)) {
            c = oc;
            best = ob;
        }
    }
    if (lane == 0) *giant = best;
}

// giant == nullptr: every upper entry (row < column) hooks, no sampling before
__global__ void k_uf_rest(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ row_of,
                          const int32_t *__restrict__ col, int64_t nnz, int r0, const int32_t *__restrict__ giant,
                          int32_t *par) {
    const int32_t g = giant ? *giant : -1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = row_of[e];
        if (!giant) {
            const int32_t v = col[e];
            if (u < v) uf_hook(par, u, v);
            continue;
        }
        if (e < (int64_t)rowptr[u] + r0) continue;  // hooked in the sampling rounds
        if (uf_find(par, u) == g) continue;
        uf_hook(par, u, col[e]);
    }
}

__global__ void k_uf_count_roots(const int32_t *par, int32_t n, int32_t *count) {
    int32_t c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += (__ldcg(par + i) == (int32_t)i) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

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

template <typename T>
const T *to_device(const T *p, int64_t count, DBuf<T> &tmp, cudaStream_t s) {
    if (!p || is_device_pointer(p)) return p;
    tmp.alloc(count, s);
    CFC_CUDA(cudaMemcpyAsync(tmp.get(), p, count * sizeof(T), cudaMemcpyHostToDevice, s));
    return tmp.get();
}

}  // namespace

void ingest(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const double *w, cudaStream_t s,
            Csr64 &out) {
    CFC_REQUIRE(src && dst, LAP_EINVAL, "src/dst must not be NULL");
    CFC_REQUIRE(n >= 2 && n < (int64_t(1) << 31) - 1, LAP_EINVAL, "need 2 <= n < 2^31");
    CFC_REQUIRE(m >= 1 && 2 * m < (int64_t(1) << 31) - 1, LAP_EINVAL, "need 1 <= m and 2m < 2^31");
    DBuf<int32_t> ts, td;
    DBuf<double> tw;
    // endpoints in page-locked host memory are read in place, once, by the
    // validation and pair emission: no staging copy
    const void *ms = mapped_host_pointer(src), *md = mapped_host_pointer(dst);
    const int32_t *ds = ms ? static_cast<const int32_t *>(ms) : to_device(src, m, ts, s);
    const int32_t *dd = md ? static_cast<const int32_t *>(md) : to_device(dst, m, td, s);
    const double *dw = to_device(w, m, tw, s);

    // device scalars read back in batches: [0] invalid-edge flag, [1] kept
    // edges, [2] merged entries, [3] union-find roots
    DBuf<int64_t> tot(4, s);
    tot.zero(s);
    const int b = bits_for(n);
    DBuf<uint64_t> keys(2 * m, s);
    DBuf<uint32_t> vals(2 * m, s);
    const double eb = (double)m * (8.0 + (w ? 8.0 : 0.0) + 24.0);
    // dropped edges sort behind the 2 kept candidates of every kept edge
    CFC_LAUNCH(LAP_KF_SETUP, s, eb, k_validate_emit, grid_for(m), kBlock, 0, ds, dd, dw, m, (int32_t)n, b,
               keys.get(), vals.get(), reinterpret_cast<unsigned long long *>(tot.get()));
    int64_t h[4];
    read_totals(tot.get(), 2, h, s);
    CFC_REQUIRE(h[0] == 0, LAP_EINVAL, "edge endpoint out of range or weight outside [1e-150, 1e150]");
    const int64_t kept = h[1];
    CFC_REQUIRE(kept > 0, LAP_ENOTCONN, "graph has no edges besides self-loops");
    const int64_t len = 2 * kept;
    // the dropped edges' slots have the largest key: the sort moves them past len
    radix_sort_pairs(keys.get(), vals.get(), 2 * m, 2 * b, s);

    DBuf<int32_t> head(len, s), hpos(len, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_heads, grid_for(len), kBlock, 0, keys.get(), len, head.get());
    scan_exclusive_i32_total(head.get(), hpos.get(), len, tot.get() + 2, s);
    read_totals(tot.get() + 2, 1, h + 2, s);
    const int64_t nnz = h[2];

    out.n = (int32_t)n;
    out.nnz = nnz;
    out.m = nnz / 2;
    out.rowptr.alloc_persistent(n + 1);
    out.col.alloc_persistent(nnz);
    out.w.alloc_persistent(nnz);
    out.deg.alloc_persistent(n);
    out.eid.alloc_persistent(nnz);
    DBuf<int32_t> rowcnt(n + 1, s), src_edge(nnz, s), tab(m, s);
    out.row_of.alloc(nnz, s);
    int32_t *row_of = out.row_of.get();
    rowcnt.zero(s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_merge, grid_for(len), kBlock, 0, keys.get(), vals.get(), head.get(),
               hpos.get(), len, b, dw, out.col.get(), out.w.get(), rowcnt.get(), row_of, src_edge.get(),
               tab.get());
    keys.release();
    vals.release();
    head.release();
    hpos.release();
    scan_exclusive_i32_async(rowcnt.get(), out.rowptr.get(), n, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_finish_rowptr, 1, 1, 0, out.rowptr.get(), (int32_t)n, (int32_t)nnz);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_row_sums_short, grid_for(n), kBlock, 0,
               out.rowptr.get(), out.w.get(), (int32_t)n, out.deg.get());
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_row_sums_long, grid_for(32 * (int64_t)n), kBlock, 0,
               out.rowptr.get(), out.w.get(), (int32_t)n, out.deg.get());

    // edge ids: lexicographic rank among the upper entries (row < col)
    DBuf<int32_t> up(nnz, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_upper_flags, grid_for(nnz), kBlock, 0, row_of, out.col.get(), nnz,
               up.get());
    scan_exclusive_i32_async(up.get(), out.eid.get(), nnz, s);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_mirror_eid, grid_for(nnz), kBlock, 0, row_of, out.col.get(),
               src_edge.get(), tab.get(), nnz, out.eid.get());
    src_edge.release();
    tab.release();

    // connectivity
    DBuf<int32_t> par(n, s);
    int32_t *roots = reinterpret_cast<int32_t *>(tot.get() + 3);
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_uf_init, grid_for(n), kBlock, 0, out.rowptr.get(), out.col.get(), par.get(),
               (int32_t)n);
    if (nnz < (int64_t(1) << 24)) {
        // small graphs: one pass over the upper entries (the sampling rounds
        // contend on the hubs' roots when ids follow arrival order, as in BA)
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_uf_rest, grid_for(nnz), kBlock, 0, out.rowptr.get(), row_of,
                   out.col.get(), nnz, 0, (const int32_t *)nullptr, par.get());
    } else {
        constexpr int kSample = 2;
        for (int r = 0; r < kSample; ++r)
            CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_uf_sample, grid_for(n), kBlock, 0, out.rowptr.get(), out.col.get(),
                       (int32_t)n, r, par.get());
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_uf_compress, grid_for(n), kBlock, 0, par.get(), (int32_t)n);
        DBuf<int32_t> giant(1, s);
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_uf_giant, 1, 32, 0, par.get(), (int32_t)n, giant.get());
        CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_uf_rest, grid_for(nnz), kBlock, 0, out.rowptr.get(), row_of,
                   out.col.get(), nnz, kSample, giant.get(), par.get());
    }
    CFC_LAUNCH(LAP_KF_SETUP, s, 0.0, k_uf_count_roots, grid_for(n), kBlock, 0, par.get(), (int32_t)n, roots);
    read_totals(tot.get() + 3, 1, h + 3, s);
    CFC_REQUIRE(h[3] == 1, LAP_ENOTCONN, "graph is not connected");
}

}  // namespace cfc
