// Block solve of L X = B (Eq. system) for k right-hand sides: FP64 iterative
// refinement around a column-independent preconditioned CG (Sec. 3.1: CG,
// relative-residual stopping rule) whose preconditioner is one multigrid
// cycle of the aggregation hierarchy built in amg.cu.
//
//   outer (FP64):  r = b - L x ;  stop when ||r_j|| <= tol ||b_j|| for all j
//                  d = PCG(L, r) in Tin (FP32, or FP64 in LAP_FP64 mode)
//                  x += d
//   inner PCG:     per column j its own alpha_j, beta_j (columns never mix)
//   cycle:         Chebyshev (or damped Jacobi) smoothing with D^{-1},
//                  residual, restriction (sum over each aggregate),
//                  recursion (once: V-cycle, twice on the top levels:
//                  W-cycle), dense FP64 coarsest solve, prolongation scaled
//                  by the coarse-correction factor, the same smoothing again
//                  (a symmetric preconditioner).  Levels below the finest may
//                  run on BF16 weights (LAP_FP32_BF16COARSE_REFINED).  A
//                  multilevel cycle is captured once per solve as a CUDA graph
//                  and replayed at every application.
//
// L is singular with null space span{1} (Sec. 2): b is projected to zero
// mean once, the search directions are projected every iteration, and the
// result is returned with zero mean.  The first solve of a graph size and
// configuration autotunes what the options leave open (depth, smoother
// degree, cycle, coarse scale, column tile).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "rowops.cuh"

namespace cfc {

namespace {

// ====================================================================== ops
// q = L p ; sum p.q ; alpha = rz / pq
template <typename T>
struct OpSpmvDot {
    using V = typename Vec<T>::V;
    static constexpr int VW = Vec<T>::W;
    LevelView A;
    const T *p;
    T *q;
    int ld;
    const double *rz;
    double *alpha;
    T *alpha_t;
    const int32_t *active;
    __device__ V gather(int j, int c0) const { return vldg<T>(p + (size_t)j * ld + c0); }
    struct Pre {
        T d;
    };
    __device__ Pre pre(int i, int) const { return Pre{ldeg<T>(A, i)}; }
    template <class Acc>
    __device__ void epi(int i, int c0, V s, const Pre &pr, Acc &acc) const {
        const V x = gather(i, c0);
        const T d = pr.d;
        V y;
#pragma unroll
        for (int v = 0; v < VW; ++v) {
            vel(y, v) = d * vel(x, v) - vel(s, v);
            acc.add(0, v, vel(x, v) * vel(y, v));
        }
        vst<T>(q + (size_t)i * ld + c0, y);
    }
    __device__ void fin(int c, const double *sums) const {
        const double pq = sums[0];
        alpha[c] = (active[c] && pq > 0.0) ? rz[c] / pq : 0.0;
        alpha_t[c] = (T)alpha[c];
    }
};

// FP64 outer residual r = b - L x, written in the inner type scaled by
// 2^rexp_j (a per-column power of two, so that the FP32 copy and its squares
// stay inside FP32's normal range whatever the residual's size); sum r^2;
// relres_j = ||r_j|| / ||b_j||.  A column stays active until relres_j <= tol
// holds, so a NaN residual never counts as converged.  With scaling on, fin
// also predicts the exponent of the next refinement step's residual (this
// one reduced by the inner tolerance), used by the next residual pass.
template <typename Tin>
struct OpResid64 {
    using V = typename Vec<double>::V;
    static constexpr int VW = Vec<double>::W;
    LevelView A;
    const double *x;
    const double *b;
    Tin *r;
    int ld;
    const double *bnorm;
    double *relres;
    int32_t *active;
    double tol;
    const int32_t *rexp;      // exponent of this pass's scaling
    int32_t *rexp_next;       // predicted exponent for the next pass (null: no scaling)
    double pred;              // inner tolerance / sqrt(n): predicted RMS of the next residual per unit norm
    __device__ V gather(int j, int c0) const { return vldg<double>(x + (size_t)j * ld + c0); }
    struct Pre {
        double d;
    };
    __device__ Pre pre(int i, int) const { return Pre{ldeg<double>(A, i)}; }
    template <class Acc>
    __device__ void epi(int i, int c0, V s, const Pre &pr, Acc &acc) const {
        const V xi = gather(i, c0);
        const V bi = vldg<double>(b + (size_t)i * ld + c0);
#pragma unroll
        for (int v = 0; v < VW; ++v) {
            const double rv = (vel(bi, v) + vel(s, v)) - pr.d * vel(xi, v);
            acc.add(0, v, rv * rv);
            r[(size_t)i * ld + c0 + v] = from_double<Tin>(scale2(rv, __ldg(rexp + c0 + v)));
        }
    }
    __device__ void fin(int c, const double *sums) const {
        const double bn = bnorm[c];
        const double rn = sqrt(sums[0]);
        const double rr = bn > 0.0 ? rn / bn : 0.0;
        relres[c] = rr;
        active[c] = (bn > 0.0 && !(rr <= tol)) ? 1 : 0;
        if (rexp_next) rexp_next[c] = (rn * pred > 0.0 && isfinite(rn)) ? -ilogb(rn * pred) : rexp[c];
    }
};

// hi + lo += w * x with error-free transformations in FP32 (the product by
// an FMA, the sum by Knuth's two-sum); explicit roundings keep the compiler
// from contracting them
__device__ __forceinline__ void ff_acc(float &hi, float &lo, float w, float x) {
    const float p = __fmul_rn(w, x);
    const float pe = __fmaf_rn(w, x, -p);  // w x = p + pe exactly
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));  // hi + p = s + err
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, pe));
}

// The residual of the first refinement step, when x is still the first
// correction alone: x = 2^-(wexp + rexp0) d with d the FP32 inner solution on
// G.  With FP32 weights that are exactly 2^-wexp w (Level::w32_exact) every
// product w_ij d_j is exact in two FP32 words, and the row sums are carried
// in two FP32 words (about 48 bits), then finished in FP64:
//   r = b - 2^-rexp0 (2^-wexp D d - sum_j w32_ij d_j).
// The gathers move FP32 rows (half of the FP64 residual's bytes) and the
// arithmetic runs on the FP32 pipes, not on GB300's narrow FP64 one.  This
// residual only feeds the second inner solve: a column is never declared
// converged here; the step that can converge uses OpResid64.
template <typename Tin>
struct OpResidFirst {
    using V = typename Vec<double>::V;
    static constexpr int VW = Vec<double>::W;
    LevelView A;
    const float *d;
    const double *b;
    Tin *r;
    int ld;
    const double *bnorm;
    double *relres;
    int32_t *active;
    int wexp;
    const int32_t *rexp0;  // exponent of the step that produced d
    const int32_t *rexp;   // exponent of this residual's scaled copy
    int32_t *rexp_next;
    double pred;
    __device__ float4 drow(int j, int c0) const {
        return __ldg(reinterpret_cast<const float4 *>(d + (size_t)j * ld + c0));
    }
    __device__ V custom_sum(const LevelView &Av, int e0, int e1, int c0, int) const {
        float hi[VW] = {0.f, 0.f, 0.f, 0.f}, lo[VW] = {0.f, 0.f, 0.f, 0.f};
        for (int e = e0; e < e1; e += 4) {
            int j[4];
            float w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = e + u < e1;
                j[u] = ok ? __ldg(Av.col + e + u) : -1;
                w[u] = ok ? __ldg(Av.w32 + e + u) : 0.f;
            }
            float4 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = j[u] >= 0 ? drow(j[u], c0) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                ff_acc(hi[0], lo[0], w[u], x[u].x);
                ff_acc(hi[1], lo[1], w[u], x[u].y);
                ff_acc(hi[2], lo[2], w[u], x[u].z);
                ff_acc(hi[3], lo[3], w[u], x[u].w);
            }
        }
        V out;
#pragma unroll
        for (int v = 0; v < VW; ++v) vel(out, v) = (double)hi[v] + (double)lo[v];
        return out;
    }
    __device__ V gather(int j, int c0) const {  // d as FP64 (the generic sum is not used)
        const float4 x = drow(j, c0);
        V o;
        vel(o, 0) = x.x;
        vel(o, 1) = x.y;
        vel(o, 2) = x.z;
        vel(o, 3) = x.w;
        return o;
    }
    struct Pre {
        double ds;  // 2^-wexp D_ii
    };
    __device__ Pre pre(int i, int) const { return Pre{scale2(ldeg<double>(A, i), -wexp)}; }
    template <class Acc>
    __device__ void epi(int i, int c0, V s, const Pre &pr, Acc &acc) const {
        const V di = gather(i, c0);
        const V bi = vldg<double>(b + (size_t)i * ld + c0);
#pragma unroll
        for (int v = 0; v < VW; ++v) {
            const double q = pr.ds * vel(di, v) - vel(s, v);  // (2^-wexp L d)_i
            const double rv = vel(bi, v) - scale2(q, -__ldg(rexp0 + c0 + v));
            acc.add(0, v, rv * rv);
            r[(size_t)i * ld + c0 + v] = from_double<Tin>(scale2(rv, __ldg(rexp + c0 + v)));
        }
    }
    __device__ void fin(int c, const double *sums) const {
        const double bn = bnorm[c];
        const double rn = sqrt(sums[0]);
        relres[c] = bn > 0.0 ? rn / bn : 0.0;
        active[c] = bn > 0.0 ? 1 : 0;  // never converged here
        rexp_next[c] = (rn * pred > 0.0 && isfinite(rn)) ? -ilogb(rn * pred) : rexp[c];
    }
};

// PCG scalars from the sums r.z, sum z, sum r (and r.r at the start):
// mu = mean(z) (the projection of z onto 1-perp), rz = r.(z - mu),
// beta = rz / rz_old; Init also records rr0 = r.r and the active columns.
template <typename T>
struct DotState {
    double inv_n;
    double *rz, *beta, *mu, *rr0;
    T *beta_t, *mu_t;
    int32_t *active;
    const int32_t *active_out;
    template <bool Init>
    __device__ void fin(int c, const double *s) const {
        const double m = s[1] * inv_n;
        const double rzn = s[0] - m * s[2];
        mu[c] = m;
        if constexpr (Init) {
            rr0[c] = s[3];
            active[c] = (active_out[c] && s[3] > 0.0) ? 1 : 0;
            beta[c] = 0.0;
        } else {
            beta[c] = (active[c] && rz[c] != 0.0) ? rzn / rz[c] : 0.0;
        }
        rz[c] = rzn;
        mu_t[c] = (T)m;
        beta_t[c] = (T)beta[c];
    }
};

// Chebyshev / Jacobi step: out = x + c (x - xp) + e D^{-1} (b - L x), in place
// on xp.  With NR = 3 (4 when Init) the step also accumulates b.out, sum out,
// sum b (and b.b) for the PCG scalars (b is the PCG residual at level 0).
template <typename T, int NR = 0, bool Init = false>
struct OpSmooth {
    using V = typename Vec<T>::V;
    static constexpr int VW = Vec<T>::W;
    LevelView A;
    const T *x;
    T *xp;
    const T *b;
    int ld;
    T c, e;
    bool xp_zero;  // the previous iterate is the zero initial guess
    DotState<T> ds;
    __device__ V gather(int j, int c0) const { return vldg<T>(x + (size_t)j * ld + c0); }
    struct Pre {
        T d, di;
    };
    __device__ Pre pre(int i, int) const { return Pre{ldeg<T>(A, i), ldinv<T>(A, i)}; }
    template <class Acc>
    __device__ void epi(int i, int c0, V s, const Pre &pr, Acc &acc) const {
        const V xi = gather(i, c0);
        const V bi = vld<T>(b + (size_t)i * ld + c0);
        const T d = pr.d, di = pr.di;
        V out;
        if (c != T(0)) {
            const V pi = xp_zero ? vzero<V>() : vld<T>(xp + (size_t)i * ld + c0);
#pragma unroll
            for (int v = 0; v < VW; ++v)
                vel(out, v) = vel(xi, v) + c * (vel(xi, v) - vel(pi, v)) +
                              e * di * (vel(bi, v) - (d * vel(xi, v) - vel(s, v)));
        } else {
#pragma unroll
            for (int v = 0; v < VW; ++v)
                vel(out, v) = vel(xi, v) + e * di * (vel(bi, v) - (d * vel(xi, v) - vel(s, v)));
        }
        vst<T>(xp + (size_t)i * ld + c0, out);
        if constexpr (NR > 0) {
#pragma unroll
            for (int v = 0; v < VW; ++v) {
                acc.add(0, v, vel(bi, v) * vel(out, v));
                acc.add(1, v, vel(out, v));
                acc.add(2, v, vel(bi, v));
                if constexpr (Init) acc.add(NR - 1, v, vel(bi, v) * vel(bi, v));
            }
        }
    }
    __device__ void fin(int c, const double *sums) const {
        if constexpr (NR > 0) ds.template fin<Init>(c, sums);
    }
};

// r = b - L x
template <typename T>
struct OpResid {
    using V = typename Vec<T>::V;
    static constexpr int VW = Vec<T>::W;
    LevelView A;
    const T *x;
    const T *b;
    T *r;
    int ld;
    __device__ V gather(int j, int c0) const { return vldg<T>(x + (size_t)j * ld + c0); }
    struct Pre {
        T d;
    };
    __device__ Pre pre(int i, int) const { return Pre{ldeg<T>(A, i)}; }
    template <class Acc>
    __device__ void epi(int i, int c0, V s, const Pre &pr, Acc &) const {
        const V xi = gather(i, c0);
        const V bi = vld<T>(b + (size_t)i * ld + c0);
        V out;
#pragma unroll
        for (int v = 0; v < VW; ++v) vel(out, v) = vel(bi, v) - (pr.d * vel(xi, v) - vel(s, v));
        vst<T>(r + (size_t)i * ld + c0, out);
    }
    __device__ void fin(int, const double *) const {}
};

// ---------------------------------------------------------------- row-local ops
// x = e D^{-1} b  (first smoothing step from a zero guess)
template <typename T>
struct OpJacobiZero {
    using V = typename Vec<T>::V;
    static constexpr int VW = Vec<T>::W;
    LevelView A;
    const T *b;
    T *x;
    int ld;
    T e;
    template <class Acc>
    __device__ void row(int i, int c0, Acc &) const {
        const V bi = vld<T>(b + (size_t)i * ld + c0);
        const T di = e * ldinv<T>(A, i);
        V out;
#pragma unroll
        for (int v = 0; v < VW; ++v) vel(out, v) = di * vel(bi, v);
        vst<T>(x + (size_t)i * ld + c0, out);
    }
    __device__ void fin(int, const double *) const {}
};

// coarse b_c[I] = sum over the members i of aggregate I of r[i]
template <typename T>
struct OpRestrict {
    using V = typename Vec<T>::V;
    const int32_t *mem_ptr, *mem;
    const T *r;
    T *bc;
    int ld;
    template <class Acc>
    __device__ void row(int I, int c0, Acc &) const {
        V s = vzero<V>();
        for (int t = __ldg(mem_ptr + I); t < __ldg(mem_ptr + I + 1); ++t)
            s = vadd(s, vld<T>(r + (size_t)__ldg(mem + t) * ld + c0));
        vst<T>(bc + (size_t)I * ld + c0, s);
    }
    __device__ void fin(int, const double *) const {}
};

// x[i] += gamma * xc[agg[i]]
template <typename T>
struct OpProlong {
    using V = typename Vec<T>::V;
    static constexpr int VW = Vec<T>::W;
    const int32_t *agg;
    const T *xc;
    T *x;
    int ld;
    T gamma;
    template <class Acc>
    __device__ void row(int i, int c0, Acc &) const {
        const V c = vld<T>(xc + (size_t)__ldg(agg + i) * ld + c0);
        V xi = vld<T>(x + (size_t)i * ld + c0);
#pragma unroll
        for (int v = 0; v < VW; ++v) vel(xi, v) += gamma * vel(c, v);
        vst<T>(x + (size_t)i * ld + c0, xi);
    }
    __device__ void fin(int, const double *) const {}
};

// x += alpha p ; r -= alpha q ; sum r^2 -> inner convergence flags; when z1
// is set, also the preconditioner's first smoothing step z1 = e D^{-1} r
template <typename T>
struct OpUpdateXR {
    using V = typename Vec<T>::V;
    static constexpr int VW = Vec<T>::W;
    T *x, *r;
    const T *p, *q;
    T *z1;
    LevelView A;
    T e0;
    int ld;
    const T *alpha_t;
    int32_t *active;
    const double *rr0;
    double tol2;
    template <class Acc>
    __device__ void row(int i, int c0, Acc &acc) const {
        const size_t o = (size_t)i * ld + c0;
        V xi = vld<T>(x + o), ri = vld<T>(r + o);
        const V pi = vld<T>(p + o), qi = vld<T>(q + o);
        const V a = vld<T>(alpha_t + c0);
#pragma unroll
        for (int v = 0; v < VW; ++v) {
            vel(xi, v) += vel(a, v) * vel(pi, v);
            vel(ri, v) -= vel(a, v) * vel(qi, v);
            acc.add(0, v, vel(ri, v) * vel(ri, v));
        }
        vst<T>(x + o, xi);
        vst<T>(r + o, ri);
        if (z1) {
            const T di = e0 * ldinv<T>(A, i);
            V zi;
#pragma unroll
            for (int v = 0; v < VW; ++v) vel(zi, v) = di * vel(ri, v);
            vst<T>(z1 + o, zi);
        }
    }
    __device__ void fin(int c, const double *sums) const {
        if (active[c] && !(sums[0] > tol2 * rr0[c])) active[c] = 0;
    }
};

// The Jacobi preconditioner (a one-level cycle of a single smoothing step,
// z = e0 D^{-1} r) fused into the PCG updates, so that z is never stored:
//   x += alpha p ; r -= alpha q ; z formed in registers ; sums r^2 (inner
//   convergence), r.z, sum z, sum r (the PCG scalars) -- then
//   p = (z - mu) + beta p with z formed again from r.
// The values, and the order of every sum, are those of OpUpdateXR with z1,
// OpDotRZ and OpUpdateP, so the results are the same bits.
// a * b rounded once, never contracted into an FMA with a later add: the
// fused ops must round z exactly as the stored z was rounded
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename T>
struct OpUpdateXRJacobi {
    using V = typename Vec<T>::V;
    static constexpr int VW = Vec<T>::W;
    T *x, *r;
    const T *p, *q;
    LevelView A;
    T e0;
    int ld;
    const T *alpha_t;
    int32_t *active;
    const double *rr0;
    double tol2;
    DotState<T> ds;
    template <class Acc>
    __device__ void row(int i, int c0, Acc &acc) const {
        const size_t o = (size_t)i * ld + c0;
        V xi = vld<T>(x + o), ri = vld<T>(r + o);
        const V pi = vld<T>(p + o), qi = vld<T>(q + o);
        const V a = vld<T>(alpha_t + c0);
        const T di = e0 * ldinv<T>(A, i);
#pragma unroll
        for (int v = 0; v < VW; ++v) {
            vel(xi, v) += vel(a, v) * vel(pi, v);
            vel(ri, v) -= vel(a, v) * vel(qi, v);
            const T rv = vel(ri, v), zv = mul_rn(di, rv);
            acc.add(0, v, rv * rv);
            acc.add(1, v, rv * zv);
            acc.add(2, v, zv);
            acc.add(3, v, rv);
        }
        vst<T>(x + o, xi);
        vst<T>(r + o, ri);
    }
    __device__ void fin(int c, const double *sums) const {
        if (active[c] && !(sums[0] > tol2 * rr0[c])) active[c] = 0;
        ds.template fin<false>(c, sums + 1);
    }
};

template <typename T>
struct OpUpdatePJacobi {
    using V = typename Vec<T>::V;
    static constexpr int VW = Vec<T>::W;
    const T *r;
    T *p;
    LevelView A;
    T e0;
    int ld;
    const T *mu_t, *beta_t;
    template <class Acc>
    __device__ void row(int i, int c0, Acc &) const {
        const size_t o = (size_t)i * ld + c0;
        const V ri = vld<T>(r + o);
        const V m = vld<T>(mu_t + c0), bt = vld<T>(beta_t + c0);
        V pi = vld<T>(p + o);
        const T di = e0 * ldinv<T>(A, i);
#pragma unroll
        for (int v = 0; v < VW; ++v) vel(pi, v) = (mul_rn(di, vel(ri, v)) - vel(m, v)) + vel(bt, v) * vel(pi, v);
        vst<T>(p + o, pi);
    }
    __device__ void fin(int, const double *) const {}
};

// sums r.z, z, r (and r.r when Init) -> the PCG scalars (DotState)
template <typename T, bool Init>
struct OpDotRZ {
    using V = typename Vec<T>::V;
    static constexpr int VW = Vec<T>::W;
    const T *r, *z;
    int ld;
    DotState<T> ds;
    template <class Acc>
    __device__ void row(int i, int c0, Acc &acc) const {
        const size_t o = (size_t)i * ld + c0;
        const V ri = vld<T>(r + o), zi = vld<T>(z + o);
#pragma unroll
        for (int v = 0; v < VW; ++v) {
            const T a = vel(ri, v), b = vel(zi, v);
            acc.add(0, v, a * b);
            acc.add(1, v, b);
            acc.add(2, v, a);
            if constexpr (Init) acc.add(3, v, a * a);
        }
    }
    __device__ void fin(int c, const double *s) const { ds.template fin<Init>(c, s); }
};

// p = (z - mu) + beta p   (First: p = z - mu; the old p is not read)
template <typename T, bool First>
struct OpUpdateP {
    using V = typename Vec<T>::V;
    static constexpr int VW = Vec<T>::W;
    const T *z;
    T *p;
    int ld;
    const T *mu_t, *beta_t;
    template <class Acc>
    __device__ void row(int i, int c0, Acc &) const {
        const size_t o = (size_t)i * ld + c0;
        const V zi = vld<T>(z + o);
        const V m = vld<T>(mu_t + c0);
        V pi;
        if constexpr (First) {
#pragma unroll
            for (int v = 0; v < VW; ++v) vel(pi, v) = vel(zi, v) - vel(m, v);
        } else {
            const V bt = vld<T>(beta_t + c0);
            pi = vld<T>(p + o);
#pragma unroll
            for (int v = 0; v < VW; ++v) vel(pi, v) = (vel(zi, v) - vel(m, v)) + vel(bt, v) * vel(pi, v);
        }
        vst<T>(p + o, pi);
    }
    __device__ void fin(int, const double *) const {}
};

// first outer step (x = 0): r = b in the inner type, scaled by 2^rexp
template <typename Tin>
struct OpCastB {
    using V = typename Vec<double>::V;
    static constexpr int VW = Vec<double>::W;
    const double *b;
    Tin *r;
    int ld;
    const int32_t *rexp;
    template <class Acc>
    __device__ void row(int i, int c0, Acc &) const {
        const size_t o = (size_t)i * ld + c0;
        const V bi = vld<double>(b + o);
#pragma unroll
        for (int v = 0; v < VW; ++v) r[o + v] = from_double<Tin>(scale2(vel(bi, v), __ldg(rexp + c0 + v)));
    }
    __device__ void fin(int, const double *) const {}
};

// Column state of the first outer step from ||b_j|| (FP64): relres = 1 and
// active for a nonzero column, and (with scaling on) the exponents that
// scale b to unit RMS and the next residual to its predicted RMS.
__device__ __forceinline__ void init_column(int c, double bn, double inv_sqrt_n, double pred, double *relres,
                                            int32_t *active, int32_t *rexp0, int32_t *rexp1) {
    relres[c] = bn > 0.0 ? 1.0 : 0.0;
    active[c] = bn > 0.0 ? 1 : 0;
    if (rexp0) {
        const bool ok = bn > 0.0 && isfinite(bn);
        rexp0[c] = ok ? -ilogb(bn * inv_sqrt_n) : 0;
        rexp1[c] = ok ? -ilogb(bn * pred) : 0;
    }
}

// ||b_j|| in FP64 (direct solves: B is the caller's padded block)
struct OpColNorm64 {
    using V = typename Vec<double>::V;
    static constexpr int VW = Vec<double>::W;
    const double *b;
    int ld;
    double *bnorm, *relres;
    int32_t *active, *rexp0, *rexp1;
    double inv_sqrt_n, pred;
    template <class Acc>
    __device__ void row(int i, int c0, Acc &acc) const {
        const V bi = vld<double>(b + (size_t)i * ld + c0);
#pragma unroll
        for (int v = 0; v < VW; ++v) acc.add(0, v, vel(bi, v) * vel(bi, v));
    }
    __device__ void fin(int c, const double *s) const {
        const double bn = sqrt(s[0]);
        bnorm[c] = bn;
        init_column(c, bn, inv_sqrt_n, pred, relres, active, rexp0, rexp1);
    }
};

__global__ void k_init_cols(const double *__restrict__ bnorm, double *__restrict__ relres,
                            int32_t *__restrict__ active, int32_t *__restrict__ rexp0, int32_t *__restrict__ rexp1,
                            double inv_sqrt_n, double pred, int ld) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ld; c += gridDim.x * blockDim.x)
        init_column(c, bnorm[c], inv_sqrt_n, pred, relres, active, rexp0, rexp1);
}

// x64 += d 2^-(wexp + rexp_j) (active columns only): the inner solve ran on
// the operator 2^-wexp L and the right-hand side 2^rexp_j r
template <typename Tin>
struct OpAddCorr {
    using V = typename Vec<double>::V;
    static constexpr int VW = Vec<double>::W;
    double *x;
    const Tin *d;
    int ld;
    const int32_t *active;
    const int32_t *rexp;
    int wexp;
    template <class Acc>
    __device__ void row(int i, int c0, Acc &) const {
        const size_t o = (size_t)i * ld + c0;
        V xi = vld<double>(x + o);
#pragma unroll
        for (int v = 0; v < VW; ++v)
            if (active[c0 + v]) vel(xi, v) += scale2(to_double<Tin>(d[o + v]), -(wexp + __ldg(rexp + c0 + v)));
        vst<double>(x + o, xi);
    }
    __device__ void fin(int, const double *) const {}
};

// column sums of an FP64 block -> mean
struct OpColMean64 {
    using V = typename Vec<double>::V;
    static constexpr int VW = Vec<double>::W;
    const double *a;
    int ld;
    double inv_n;
    double *mean;
    template <class Acc>
    __device__ void row(int i, int c0, Acc &acc) const {
        const V ai = vld<double>(a + (size_t)i * ld + c0);
#pragma unroll
        for (int v = 0; v < VW; ++v) acc.add(0, v, vel(ai, v));
    }
    __device__ void fin(int c, const double *s) const { mean[c] = s[0] * inv_n; }
};

// out = a - mean (in place allowed), sum out^2 -> norm
struct OpSubMean64 {
    using V = typename Vec<double>::V;
    static constexpr int VW = Vec<double>::W;
    const double *a;
    double *out;
    int ld;
    const double *mean;
    double *norm;  // may be null
    template <class Acc>
    __device__ void row(int i, int c0, Acc &acc) const {
        const size_t o = (size_t)i * ld + c0;
        V ai = vld<double>(a + o);
#pragma unroll
        for (int v = 0; v < VW; ++v) {
            vel(ai, v) -= mean[c0 + v];
            acc.add(0, v, vel(ai, v) * vel(ai, v));
        }
        vst<double>(out + o, ai);
    }
    __device__ void fin(int c, const double *s) const {
        if (norm) norm[c] = sqrt(s[0]);
    }
};

// ---------------------------------------------------------------- elimination transfers
// Restriction through an elimination level (Level::elim): the next level's
// right-hand side b'(I) = b(keep_node[I]) + sum of (w_uI / d_u) b(u) over the
// eliminated neighbours u of keep_node[I] (ascending u, in the fixed order of
// the row kernels).  It runs on the row kernels over pull_view, so that a
// hub's long list of eliminated leaves is cut into chunks summed in parallel.
template <typename T>
struct OpRestrictPull {
    using V = typename Vec<T>::V;
    static constexpr int VW = Vec<T>::W;
    const int32_t *keep_node;
    const T *b;
    T *bn;
    int ld;
    __device__ V gather(int j, int c0) const { return vldg<T>(b + (size_t)j * ld + c0); }
    struct Pre {
        int32_t u;
    };
    __device__ Pre pre(int I, int) const { return Pre{__ldg(keep_node + I)}; }
    template <class Acc>
    __device__ void epi(int I, int c0, V s, const Pre &pr, Acc &) const {
        vst<T>(bn + (size_t)I * ld + c0, vadd(gather(pr.u, c0), s));
    }
    __device__ void fin(int, const double *) const {}
};

// Back-substitution through an elimination level: a kept node takes its
// next-level value; eliminated node u = e_node[j] gets
// x(u) = b(u) / d_u + sum_m (w_um / d_u) x'(nb_m(u)) (dinv already carries the
// operator's power-of-two scale in the FP32 sweeps).
template <typename T>
struct OpElimBack {
    using V = typename Vec<T>::V;
    static constexpr int VW = Vec<T>::W;
    const int32_t *keep_id, *e_nb;
    const T *coef, *dinv;
    const T *b, *xn;
    T *x;
    int ld;
    template <class Acc>
    __device__ void row(int i, int c0, Acc &) const {
        const int kid = __ldg(keep_id + i);
        V out;
        if (kid >= 0) {
            out = vld<T>(xn + (size_t)kid * ld + c0);
        } else {
            const int j = -kid - 1;
            const T di = __ldg(dinv + j);
            const V bi = vld<T>(b + (size_t)i * ld + c0);
#pragma unroll
            for (int v = 0; v < VW; ++v) vel(out, v) = di * vel(bi, v);
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int a = __ldg(e_nb + 2 * j + m);
                if (a >= 0) vfma(out, __ldg(coef + 2 * j + m), vld<T>(xn + (size_t)a * ld + c0));
            }
        }
        vst<T>(x + (size_t)i * ld + c0, out);
    }
    __device__ void fin(int, const double *) const {}
};

// ---------------------------------------------------------------- plain kernels
__global__ void k_copy_pad(const double *__restrict__ src, int k, double *__restrict__ dst, int ld, int64_t n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * ld; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / ld;
        const int c = (int)(t - i * ld);
        dst[t] = c < k ? src[i * k + c] : 0.0;
    }
}

__global__ void k_copy_unpad(const double *__restrict__ src, int ld, double *__restrict__ dst, int k, int64_t n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * k; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k;
        const int c = (int)(t - i * k);
        dst[t] = src[i * ld + c];
    }
}

// x_c = 2^e M^{-1} b_c with the dense FP64 inverse (coarsest level), FP64
// sums; e = wexp when the cycle runs on the operator 2^-wexp L (FP32), else 0
template <typename T>
__global__ void k_coarse_dense(const double *__restrict__ Minv, int nc, const T *__restrict__ b, T *__restrict__ x,
                               int ld, int k, int e) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nc * k; t += gridDim.x * blockDim.x) {
        const int I = t / k, c = t - (t / k) * k;
        const double *row = Minv + (size_t)I * nc;
        double s = 0.0;
        for (int J = 0; J < nc; ++J) s += row[J] * (double)b[(size_t)J * ld + c];
        x[(size_t)I * ld + c] = (T)scale2(s, e);
    }
}

// The same in FP32 (the FP32 modes): x_c = (2^wexp M^{-1}) b_c with the FP32
// copy of the scaled inverse (entries of order one whatever the weights) and
// FP32 sums in a fixed order (GB300's FP64 rate would make the FP64 product
// the cost of the whole coarse solve at n_c in the thousands).  One warp per
// coarse row I, a lane per column of a 32-column chunk; the row of the
// inverse is read once per warp and broadcast.
__global__ void __launch_bounds__(256) k_coarse_dense32(const float *__restrict__ Minv, int nc,
                                                        const float *__restrict__ b, float *__restrict__ x, int ld,
                                                        int k) {
    const int lane = threadIdx.x & 31;
    const int chunks = (k + 31) / 32;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nc * chunks; w += (gridDim.x * blockDim.x) >> 5) {
        const int I = w / chunks, c = (w - I * chunks) * 32 + lane;
        const float *row = Minv + (size_t)I * nc;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        if (c < k) {
            int J = 0;
            for (; J + 4 <= nc; J += 4) {
                s0 = fmaf(__ldg(row + J), __ldg(b + (size_t)J * ld + c), s0);
                s1 = fmaf(__ldg(row + J + 1), __ldg(b + (size_t)(J + 1) * ld + c), s1);
                s2 = fmaf(__ldg(row + J + 2), __ldg(b + (size_t)(J + 2) * ld + c), s2);
                s3 = fmaf(__ldg(row + J + 3), __ldg(b + (size_t)(J + 3) * ld + c), s3);
            }
            for (; J < nc; ++J) s0 = fmaf(__ldg(row + J), __ldg(b + (size_t)J * ld + c), s0);
            x[(size_t)I * ld + c] = (s0 + s1) + (s2 + s3);
        }
    }
}

constexpr int kRedMaxBlocks = 32768;  // = kTeam * kMaxTeams

int g_num_sms = 0;
int num_sms() {
    if (!g_num_sms) {
        int dev = 0;
        CFC_CUDA(cudaGetDevice(&dev));
        CFC_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

// ====================================================================== solver
// Deadline of an autotuning trial on this thread (steady clock, seconds; 0 =
// none), checked at the solve's host synchronisations, so that a slow
// candidate is abandoned early.
thread_local double t_trial_deadline = 0.0;
double steady_seconds() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
bool past_trial_deadline() { return t_trial_deadline > 0.0 && steady_seconds() > t_trial_deadline; }

struct ColState {
    double *bnorm, *relres, *alpha, *beta, *rz, *rr0, *mu;
    void *alpha_t, *beta_t, *mu_t;  // the same scalars in the inner arithmetic type
    int32_t *active_out, *active_in;
    int32_t *rexp[2];  // residual exponents of even and odd refinement steps
};

template <typename Tin, int KT>
struct Solver {
    static constexpr int K64 = KT > 64 ? 64 : KT;  // FP64 tile: at most 16 lanes of 4 doubles
    static constexpr int G64 = K64 / Vec<double>::W;
    static constexpr int RPB64 = kBlock / G64;

    lap_hierarchy *h;
    cudaStream_t s;
    int ld, ntiles, ntiles64, nlev, k;
    const lap_solve_opts_t &o;
    // workspace
    double *b64, *x64;
    std::vector<Tin *> lb, lx, lt;  // per cycle level: rhs, iterate, scratch
    Tin *r, *z, *p, *q, *t0;        // PCG vectors at the top cycle level (+ lb[0] = r, lx[0] = z)
    // with an elimination level in front: the FP32 residual and correction on G itself
    Tin *r0 = nullptr, *d0 = nullptr;
    // Cycle level c is hierarchy level p0 + c: levels lv[0 .. p0-1] are
    // eliminations, which only the outer refinement passes through.
    int p0 = 0;
    const Level &lvl(int c) const { return h->lv[p0 + c]; }
    Tin *chunk_part;
    double *chunk_part64;
    RedBuf rb;
    ColState cs;
    int32_t *h_active;  // pinned
    std::vector<double> cheb_c, cheb_e;
    double gamma = 1.0;  // coarse-correction scale
    int cycle = 1;       // 1: V-cycle, 2: W-cycle
    int w_levels = 0;    // W-cycle: levels 0 .. w_levels-1 correct twice (0: all)
    int nu_pre, nu_post, nu_coarse;
    bool bf16 = false;  // BF16 weights below the finest level
    int hsize = 0;      // levels of the hierarchy and its dense coarsest size, as the solve began
    int32_t coarse_n = 0;

    // the finest level always runs on FP32 weights; coarser ones on BF16 in that mode
    std::vector<uint32_t *> long_cnt;  // per level: this solve's long-row arrival counters

    LevelView lv_view(const Level &L) const {
        LevelView v = (bf16 && &L != &lvl(0)) ? view_bf16(L) : view(L);
        v.long_count = nullptr;
        for (size_t l = 0; l < long_cnt.size(); ++l)
            if (&lvl((int)l) == &L) v.long_count = long_cnt[l];
        return v;
    }

    Solver(lap_hierarchy *h_, cudaStream_t s_, int k_, int ld_, const lap_solve_opts_t &o_)
        : h(h_), s(s_), ld(ld_), ntiles(ld_ / KT), ntiles64(ld_ / K64), k(k_), o(o_) {
        p0 = h->p0;
        nlev = (int)h->lv.size() - p0;
        if (o.levels_used > 0) nlev = std::min(nlev, o.levels_used);
        nu_pre = std::max(1, o.nu_pre);
        nu_post = std::max(1, o.nu_post);
        nu_coarse = o.nu_coarse > 0 ? o.nu_coarse : std::max(nu_pre, 4);
        cycle = o.cycle == 2 ? 2 : 1;
        w_levels = std::max(0, o.w_levels);
        gamma = o.coarse_scale > 0.0 ? o.coarse_scale : 1.0;
        bf16 = std::is_same<Tin, float>::value && o.precision == LAP_FP32_BF16COARSE_REFINED;
        hsize = (int)h->lv.size() - p0;
        coarse_n = h->coarse_n;
        // a one-level preconditioner is two or three kernels: nothing to gain
        use_graphs = o.graphs != 0 && nlev >= 2 && !stats_detailed();
        setup_smoother();
    }

    void setup_smoother() {
        // D^{-1} L of a Laplacian has its spectrum in [0, 2] (Gershgorin).
        const int nu = std::max(std::max(nu_pre, nu_post), nu_coarse);
        cheb_c.assign(nu, 0.0);
        cheb_e.assign(nu, 0.0);
        if (o.smoother == LAP_SMOOTH_JACOBI) {
            for (int t = 0; t < nu; ++t) cheb_e[t] = 2.0 / 3.0;
            return;
        }
        const double hi = 2.0, lo = hi / 4.0;  // smooth the upper part of the spectrum
        const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
        double rho = 1.0 / sigma;
        cheb_e[0] = 1.0 / theta;
        cheb_c[0] = 0.0;
        for (int t = 1; t < nu; ++t) {
            const double rn = 1.0 / (2.0 * sigma - rho);
            cheb_c[t] = rn * rho;
            cheb_e[t] = 2.0 * rn / delta;
            rho = rn;
        }
    }

    // about one and a half waves of resident blocks, each walking its row
    // blocks grid-stride: measured faster than one block per row block (fewer
    // block launches and block-level reductions), while the half wave of spare
    // blocks evens out the blocks that drew long rows
    int red_grid(int nvb) const { return std::max(1, std::min({nvb, 6 * num_sms(), kRedMaxBlocks})); }
    int plain_grid(int nvb) const { return red_grid(nvb); }

    // bytes of one edge weight as the sweeps of level L read it
    int wbytes(const Level &L) const { return (bf16 && &L != &lvl(0)) ? 2 : (int)sizeof(Tin); }
    static double vec_bytes(int64_t n, int ld, int nvec, int elem) { return (double)n * ld * elem * nvec; }
    static double mat_bytes(const Level &L, int wb) {
        return (double)L.nnz * (4.0 + wb) + (double)L.n * (4.0 + 2.0 * wb);
    }

    // ---------------- generic launches
    template <typename T, int NR, class Op>
    void rowop(int fam, const Level &L, const Op &op, T *cpart, double bytes) {
        constexpr int G = KT / Vec<T>::W;
        constexpr int RPB = kBlock / G;
        const int nvb_short = (L.n + RPB - 1) / RPB;
        const int nvb_long = (L.n_chunks + RPB - 1) / RPB;
        if (bf16 && &L != &lvl(0)) {
            // below the top cycle level only reduction-free sweeps run (smoothing, residual)
            CFC_REQUIRE(NR == 0, LAP_ECUDA, "internal: reduction sweep on a BF16 level");
            if constexpr (NR == 0 && std::is_same<T, float>::value) {
                const int nvb = nvb_short + nvb_long;
                dim3 grid(plain_grid(nvb), ntiles);
                CFC_LAUNCH(fam, s, bytes, (k_rowop<T, KT, 0, Op, kLongLast, true>), grid, kBlock, 0, lv_view(L), op,
                           nvb_short, nvb, cpart, ld, rb);
            }
            return;
        }
        if (NR > 0 && L.n_chunks > 0) {
            // deterministic reductions: chunk sums first, rows finished by their own group
            CFC_LAUNCH(fam, s, 0.0, (k_chunk_sums<T, KT, Op>), dim3(nvb_long, ntiles), kBlock, 0, lv_view(L), op, cpart,
                       ld);
            dim3 grid(red_grid(nvb_short), ntiles);
            CFC_LAUNCH(fam, s, bytes, (k_rowop<T, KT, NR, Op, kLongPre>), grid, kBlock, 0, lv_view(L), op, nvb_short,
                       nvb_short, cpart, ld, rb);
            return;
        }
        const int nvb = nvb_short + nvb_long;
        const int gx = NR > 0 ? red_grid(nvb) : plain_grid(nvb);
        dim3 grid(gx, ntiles);
        CFC_LAUNCH(fam, s, bytes, (k_rowop<T, KT, NR, Op>), grid, kBlock, 0, lv_view(L), op, nvb_short, nvb, cpart, ld,
                   rb);
    }
    template <typename T, int NR, class Op>
    void rows(int fam, int64_t n, const Op &op, double bytes) {
        constexpr int G = KT / Vec<T>::W;
        constexpr int RPB = kBlock / G;
        const int nvb = (int)((n + RPB - 1) / RPB);
        const int gx = NR > 0 ? red_grid(nvb) : plain_grid(nvb);
        dim3 grid(gx, ntiles);
        CFC_LAUNCH(fam, s, bytes, (k_rows<T, KT, NR, Op>), grid, kBlock, 0, (int)n, op, rb);
    }

    int fam_level(int l, int fine_fam) const { return l == 0 ? fine_fam : LAP_KF_COARSE_LEVELS; }

    // one smoothing step at level l (cur -> oth, swapped); at level 0 the
    // step may also produce the PCG dot products (dot = 1: update, 2: init)
    void smooth_step(int l, Tin *&cur, Tin *&oth, int t, bool xp_zero, int dot) {
        const Level &L = lvl(l);
        const int et = (int)sizeof(Tin);
        const int ti = std::min(t, (int)cheb_c.size() - 1);
        const double bytes = mat_bytes(L, wbytes(L)) + vec_bytes(L.n, ld, xp_zero || cheb_c[ti] == 0.0 ? 3 : 4, et);
        const Tin c = (Tin)cheb_c[ti], e = (Tin)cheb_e[ti];
        const int fam = fam_level(l, LAP_KF_SMOOTH_FINE);
        if (dot == 0) {
            rowop<Tin, 0>(fam, L, OpSmooth<Tin>{lv_view(L), cur, oth, lb[l], ld, c, e, xp_zero, {}}, chunk_part, bytes);
        } else if (dot == 1) {
            rowop<Tin, 3>(fam, L, OpSmooth<Tin, 3, false>{lv_view(L), cur, oth, lb[l], ld, c, e, xp_zero, dstate()},
                          chunk_part, bytes);
        } else {
            rowop<Tin, 4>(fam, L, OpSmooth<Tin, 4, true>{lv_view(L), cur, oth, lb[l], ld, c, e, xp_zero, dstate()},
                          chunk_part, bytes);
        }
        std::swap(cur, oth);
    }

    DotState<Tin> dstate() const {
        return DotState<Tin>{1.0 / lvl(0).n, cs.rz, cs.beta, cs.mu, cs.rr0, (Tin *)cs.beta_t, (Tin *)cs.mu_t,
                             cs.active_in, cs.active_out};
    }

    bool level0_is_dense() const { return nlev == 1 && coarse_n == lvl(0).n && hsize == 1; }

    // The FP32 sweeps run on 2^-wexp L and on residuals scaled per column by
    // powers of two (exact: FP32 results are those of the unscaled problem
    // wherever that stays in range); FP64 sweeps are unscaled.
    static constexpr bool kScaled = std::is_same<Tin, float>::value;
    int op_wexp() const { return kScaled ? h->wexp : 0; }

    // ---------------- V-cycle on level l: b = lb[l] -> x = lx[l].
    // first_done: x already holds the first smoothing step e D^{-1} b (fused
    // into the PCG update); dot: the level-0 final step also computes the PCG
    // dot products (1: update, 2: init).  Returns true when it did.
    bool vcycle(int l, bool first_done = false, int dot = 0) {
        const Level &L = lvl(l);
        const int et = (int)sizeof(Tin);
        const int wb = wbytes(L);
        const bool coarsest = (l == nlev - 1);
        if (coarsest && coarse_n == L.n && l == hsize - 1) {
            const int nc = L.n;
            const double bytes = (double)nc * nc * (kScaled ? 4 : 8) + 2.0 * nc * ld * et;
            if constexpr (kScaled) {
                const int chunks = (ld + 31) / 32;
                const int blocks = std::max(1, std::min((nc * chunks + 7) / 8, 8 * num_sms()));
                CFC_LAUNCH(LAP_KF_COARSE_LEVELS, s, bytes, k_coarse_dense32, blocks, 256, 0, h->coarse_inv32.get(), nc,
                           (const float *)lb[l], (float *)lx[l], ld, ld);
            } else {
                const int threads = 128;
                const int blocks = std::max(1, std::min((nc * ld + threads - 1) / threads, 8 * num_sms()));
                CFC_LAUNCH(LAP_KF_COARSE_LEVELS, s, bytes, k_coarse_dense<Tin>, blocks, threads, 0, h->coarse_inv.get(),
                           nc, lb[l], lx[l], ld, ld, op_wexp());
            }
            return false;
        }
        // pre-smoothing from zero
        Tin *cur = lx[l], *oth = lt[l];
        if (!first_done)
            rows<Tin, 0>(fam_level(l, LAP_KF_SMOOTH_FINE), L.n,
                         OpJacobiZero<Tin>{lv_view(L), lb[l], cur, ld, (Tin)cheb_e[0]},
                         vec_bytes(L.n, ld, 2, et) + L.n * (double)wb);
        const int npre = coarsest ? nu_coarse : nu_pre;
        bool dotted = false;
        for (int t = 1; t < npre; ++t) {
            const int d = (coarsest && t == npre - 1) ? dot : 0;
            smooth_step(l, cur, oth, t, t == 1, d);
            dotted = dotted || d;
        }
        if (coarsest) {
            lx[l] = cur;
            lt[l] = oth;
            return dotted;
        }
        // coarse corrections: residual into oth, restrict to level l+1, recurse,
        // prolong; a W-cycle does this twice (the same operator twice keeps
        // the preconditioner symmetric); the coarse level's dense solve is
        // exact, so one correction suffices just above it
        const Level &C = lvl(l + 1);
        const bool next_dense = (l + 1 == nlev - 1) && coarse_n == C.n && l + 1 == hsize - 1;
        const int ncorr = (cycle == 2 && !next_dense && (w_levels == 0 || l < w_levels)) ? 2 : 1;
        for (int cc = 0; cc < ncorr; ++cc) {
            rowop<Tin, 0>(fam_level(l, LAP_KF_RESTRICT_FINE), L, OpResid<Tin>{lv_view(L), cur, lb[l], oth, ld},
                          chunk_part, mat_bytes(L, wb) + vec_bytes(L.n, ld, 3, et));
            rows<Tin, 0>(fam_level(l, LAP_KF_RESTRICT_FINE), C.n,
                         OpRestrict<Tin>{L.mem_ptr.get(), L.mem.get(), oth, lb[l + 1], ld},
                         vec_bytes(L.n, ld, 1, et) + vec_bytes(C.n, ld, 1, et) + 4.0 * (L.n + C.n));
            vcycle(l + 1);
            rows<Tin, 0>(LAP_KF_COARSE_LEVELS, L.n, OpProlong<Tin>{L.agg.get(), lx[l + 1], cur, ld, (Tin)gamma},
                         vec_bytes(L.n, ld, 2, et) + vec_bytes(C.n, ld, 1, et) + 4.0 * L.n);
        }
        // post-smoothing (the same polynomial: symmetric V-cycle)
        for (int t = 0; t < nu_post; ++t) {
            const int d = (t == nu_post - 1) ? dot : 0;
            smooth_step(l, cur, oth, t, false, d);
            dotted = dotted || d;
        }
        lx[l] = cur;
        lt[l] = oth;
        return dotted;
    }

    // z = M^{-1} r  (the result may land in either of the two finest-level
    // buffers; z and t0 are swapped accordingly).  Returns true when the PCG
    // dot products were computed on the way.
    bool precond_eager(bool first_done, int dot) {
        lb[0] = r;
        lx[0] = z;
        lt[0] = t0;
        const bool dotted = vcycle(0, first_done, dot);
        z = lx[0];
        t0 = lt[0];
        return dotted;
    }

    // A multilevel cycle is a fixed sequence of kernels for a given entry
    // state (variant, and which of the two level-0 buffers holds z): the
    // first application in each state is captured as a CUDA graph (on a
    // private stream: capture cannot run on the legacy stream) and every
    // application replays it with one launch on the solve's stream.  The
    // smoothing ping-pongs buffers, so the state after the cycle is recorded
    // with the graph and restored on replay.  Coarse-level buffers are
    // scratch within a cycle, so their assignment at capture is kept.
    struct CycleGraph {
        cudaGraphExec_t exec = nullptr;
        bool dotted = false;
        Tin *z_after = nullptr, *t0_after = nullptr;
        int64_t launches[LAP_KF_COUNT] = {};
    };
    std::map<std::tuple<bool, int, Tin *, Tin *>, CycleGraph> graphs;
    cudaStream_t cap_stream = nullptr;
    bool use_graphs = false;

    ~Solver() {
        for (auto &g : graphs)
            if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }

    bool precond(bool first_done, int dot) {
        if (!use_graphs) return precond_eager(first_done, dot);
        const auto key = std::make_tuple(first_done, dot, z, t0);
        auto it = graphs.find(key);
        if (it == graphs.end()) {
            CycleGraph g;
            if (!cap_stream) CFC_CUDA(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
            int64_t before[LAP_KF_COUNT], after[LAP_KF_COUNT];
            stats_launches(before);
            const cudaStream_t run_stream = s;
            s = cap_stream;
            cudaGraph_t graph = nullptr;
            CFC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            try {
                g.dotted = precond_eager(first_done, dot);
            } catch (...) {
                cudaStreamEndCapture(s, &graph);
                if (graph) cudaGraphDestroy(graph);
                s = run_stream;
                throw;
            }
            CFC_CUDA(cudaStreamEndCapture(s, &graph));
            s = run_stream;
            const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
            cudaGraphDestroy(graph);
            CFC_CUDA(ie);
            stats_launches(after);
            for (int f = 0; f < LAP_KF_COUNT; ++f) g.launches[f] = after[f] - before[f];
            stats_add_launches(g.launches, -1);  // captured, not run: counted per replay below
            g.z_after = z;
            g.t0_after = t0;
            it = graphs.emplace(key, g).first;
        }
        CFC_CUDA(cudaGraphLaunch(it->second.exec, s));
        stats_add_launches(it->second.launches, 1);
        z = it->second.z_after;
        t0 = it->second.t0_after;
        return it->second.dotted;
    }

    // inner PCG on the finest level: solves L d = r; returns iterations
    int inner_pcg(Tin *d, int max_inner, double inner_tol) {
        const Level &L0 = lvl(0);
        const int et = (int)sizeof(Tin);
        const int64_t n = L0.n;
        const double vb1 = vec_bytes(n, ld, 1, et);
        CFC_CUDA(cudaMemsetAsync(d, 0, (size_t)n * ld * et, s));
        Tin *alpha_t = (Tin *)cs.alpha_t, *beta_t = (Tin *)cs.beta_t, *mu_t = (Tin *)cs.mu_t;
        if (!precond(false, 2))
            rows<Tin, 4>(LAP_KF_BLAS1, n, OpDotRZ<Tin, true>{r, z, ld, dstate()}, 2 * vb1);
        rows<Tin, 0>(LAP_KF_BLAS1, n, OpUpdateP<Tin, true>{z, p, ld, mu_t, beta_t}, 2 * vb1);
        const bool fuse_first = !level0_is_dense();
        // one level, one smoothing step: the preconditioner is z = e0 D^{-1} r
        const bool jacobi = fuse_first && nlev == 1 && nu_coarse <= 1;
        const Tin e0 = (Tin)cheb_e[0];
        const int check = std::max(1, o.check_every);
        int it = 0;
        for (it = 1; it <= max_inner; ++it) {
            rowop<Tin, 1>(LAP_KF_SPMV_FINE, L0,
                          OpSpmvDot<Tin>{lv_view(L0), p, q, ld, cs.rz, cs.alpha, alpha_t, cs.active_in}, chunk_part,
                          mat_bytes(L0, et) + 2 * vb1);
            if (jacobi)
                rows<Tin, 4>(LAP_KF_BLAS1, n,
                             OpUpdateXRJacobi<Tin>{d, r, p, q, lv_view(L0), e0, ld, alpha_t, cs.active_in, cs.rr0,
                                                   inner_tol * inner_tol, dstate()},
                             6 * vb1 + (double)n * et);
            else
                rows<Tin, 1>(LAP_KF_BLAS1, n,
                             OpUpdateXR<Tin>{d, r, p, q, fuse_first ? z : nullptr, lv_view(L0), e0, ld, alpha_t,
                                             cs.active_in, cs.rr0, inner_tol * inner_tol},
                             (fuse_first ? 7 : 6) * vb1);
            if (it % check == 0 || it == max_inner) {
                CFC_CUDA(cudaMemcpyAsync(h_active, cs.active_in, ld * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                CFC_CUDA(cudaStreamSynchronize(s));
                int na = 0;
                for (int c = 0; c < ld; ++c) na += h_active[c] ? 1 : 0;
                if (na == 0) break;
                if (it == max_inner || past_trial_deadline()) break;
            }
            if (jacobi) {
                rows<Tin, 0>(LAP_KF_BLAS1, n, OpUpdatePJacobi<Tin>{r, p, lv_view(L0), e0, ld, mu_t, beta_t},
                             3 * vb1 + (double)n * et);
                continue;
            }
            if (!precond(fuse_first, 1))
                rows<Tin, 3>(LAP_KF_BLAS1, n, OpDotRZ<Tin, false>{r, z, ld, dstate()}, 2 * vb1);
            rows<Tin, 0>(LAP_KF_BLAS1, n, OpUpdateP<Tin, false>{z, p, ld, mu_t, beta_t}, 3 * vb1);
        }
        return std::min(it, max_inner);
    }

    // through the elimination level (p0 == 1): r0 on G -> r on the top cycle
    // level, and the inner solution dbuf -> d0 on G
    template <typename T>
    static const T *coef_of(const Level &E) {
        if constexpr (std::is_same<T, float>::value) return E.e_c32.get();
        else return E.e_c64.get();
    }
    template <typename T>
    static const T *dinv_of(const Level &E) {
        if constexpr (std::is_same<T, float>::value) return E.e_dinv32.get();
        else return E.e_dinv64.get();
    }
    void elim_restrict() {
        const Level &E = h->lv[0];
        const int et = (int)sizeof(Tin);
        const double bytes = vec_bytes(E.n, ld, 1, et) + vec_bytes(lvl(0).n, ld, 1, et);
        const LevelView pv = pull_view(E);
        const OpRestrictPull<Tin> op{E.keep_node.get(), r0, r, ld};
        constexpr int G = KT / Vec<Tin>::W;
        constexpr int RPB = kBlock / G;
        const int nvb_short = (pv.n + RPB - 1) / RPB;
        if (pv.n_chunks > 0) {  // chunk sums first, then every row finished by its own group
            const int nvb_long = (pv.n_chunks + RPB - 1) / RPB;
            CFC_LAUNCH(LAP_KF_BLAS1, s, 0.0, (k_chunk_sums<Tin, KT, OpRestrictPull<Tin>>), dim3(nvb_long, ntiles),
                       kBlock, 0, pv, op, chunk_part, ld);
            CFC_LAUNCH(LAP_KF_BLAS1, s, bytes, (k_rowop<Tin, KT, 0, OpRestrictPull<Tin>, kLongPre>),
                       dim3(plain_grid(nvb_short), ntiles), kBlock, 0, pv, op, nvb_short, nvb_short, chunk_part, ld,
                       rb);
        } else {
            CFC_LAUNCH(LAP_KF_BLAS1, s, bytes, (k_rowop<Tin, KT, 0, OpRestrictPull<Tin>>),
                       dim3(plain_grid(nvb_short), ntiles), kBlock, 0, pv, op, nvb_short, nvb_short, chunk_part, ld,
                       rb);
        }
    }
    void elim_back() {
        const Level &E = h->lv[0];
        const int et = (int)sizeof(Tin);
        rows<Tin, 0>(LAP_KF_BLAS1, E.n,
                     OpElimBack<Tin>{E.keep_id.get(), E.e_nb.get(), coef_of<Tin>(E), dinv_of<Tin>(E), r0, dbuf, d0,
                                     ld},
                     vec_bytes(lvl(0).n, ld, 1, et) + vec_bytes(E.n, ld, 1, et) + vec_bytes(E.n_elim, ld, 1, et));
    }

    lap_status_t run(const double *B, double *X, lap_solve_info_t *info) {
        const Level &L0 = h->lv[0];
        const int64_t n = L0.n;
        const double v64 = vec_bytes(n, ld, 1, 8);
        const double inv_sqrt_n = 1.0 / std::sqrt((double)n);
        // predicted RMS of the next refinement step's residual per unit of this
        // one's norm: the inner solve reduces it by about its tolerance
        const double itol = (o.precision == LAP_FP64) ? std::max(o.tol * 0.5, 1e-15) : o.inner_tol;
        const double pred = std::max(itol, 1e-7) * inv_sqrt_n;
        int32_t *rx0 = kScaled ? cs.rexp[0] : nullptr, *rx1 = kScaled ? cs.rexp[1] : nullptr;
        // the FP32 residual on G itself: the PCG's right-hand side, or (with an
        // elimination level in front) the input of the restriction
        Tin *rfine = p0 ? r0 : r;
        // b64 = B (padded), projected to zero mean; bnorm (direct: B is used in
        // place and its norm comes with the first step below)
        if (!direct) {
            const int64_t tot = n * ld;
            const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 8 * num_sms());
            CFC_LAUNCH(LAP_KF_BLAS1, s, v64 * 2, k_copy_pad, blocks, 256, 0, B, k, b64, ld, n);
            rowsd<1>(n, OpColMean64{b64, ld, 1.0 / n, cs.mu}, v64);
            rowsd<1>(n, OpSubMean64{b64, b64, ld, cs.mu, cs.bnorm}, 2 * v64);
        }
        CFC_CUDA(cudaMemsetAsync(x64, 0, (size_t)n * ld * 8, s));

        int outer = 0, inner_total = 0;
        bool converged = false, used_ff = false;
        double maxrel = 0.0;
        std::vector<double> hrel(ld), hbn(ld);
        for (outer = 0;; ++outer) {
            // step j's residual is written scaled by 2^rexp[j % 2]; its pass
            // predicts rexp[(j + 1) % 2] for the next step
            const int32_t *rx_cur = cs.rexp[outer & 1];
            // FP64 residual, written to r in the inner type (x = 0 at the first step: r = b)
            if (outer == 0 && direct) {
                rowsd<1>(n, OpColNorm64{b64, ld, cs.bnorm, cs.relres, cs.active_out, rx0, rx1, inv_sqrt_n, pred}, v64);
                rowsd<0>(n, OpCastB<Tin>{b64, rfine, ld, rx_cur}, v64 + vec_bytes(n, ld, 1, sizeof(Tin)));
            } else if (outer == 0) {
                CFC_LAUNCH(LAP_KF_BLAS1, s, 0.0, k_init_cols, (ld + 255) / 256, 256, 0, cs.bnorm, cs.relres,
                           cs.active_out, rx0, rx1, inv_sqrt_n, pred, ld);
                rowsd<0>(n, OpCastB<Tin>{b64, rfine, ld, rx_cur}, v64 + vec_bytes(n, ld, 1, sizeof(Tin)));
            } else {
                constexpr int RPB = RPB64;
                const int nvb_short = (L0.n + RPB - 1) / RPB;
                const int nvb_long = (L0.n_chunks + RPB - 1) / RPB;
                const int nvb = nvb_short + nvb_long;
                dim3 grid(red_grid(nvb), ntiles64);
                LevelView v0 = view(L0);
                v0.long_count = nullptr;  // FP64 sweeps finish long rows from chunk sums: no counters
                // x is still the first correction alone: its residual in two FP32 words
                const bool first_ff =
                    kScaled && outer == 1 && L0.w32_exact && o.max_outer > 1 && o.first_residual_ff != 0;
                auto launch = [&](const auto &op, double bytes) {
                    using Op = std::decay_t<decltype(op)>;
                    if (L0.n_chunks > 0) {
                        CFC_LAUNCH(LAP_KF_RESID64, s, 0.0, (k_chunk_sums<double, K64, Op>),
                                   dim3(nvb_long, ntiles64), kBlock, 0, v0, op, chunk_part64, ld);
                        CFC_LAUNCH(LAP_KF_RESID64, s, bytes, (k_rowop<double, K64, 1, Op, kLongPre>),
                                   dim3(red_grid(nvb_short), ntiles64), kBlock, 0, v0, op, nvb_short, nvb_short,
                                   chunk_part64, ld, rb);
                    } else {
                        CFC_LAUNCH(LAP_KF_RESID64, s, bytes, (k_rowop<double, K64, 1, Op>), grid, kBlock, 0, v0, op,
                                   nvb_short, nvb, chunk_part64, ld, rb);
                    }
                };
                used_ff = used_ff || first_ff;
                if constexpr (kScaled) {
                    if (first_ff) {
                        launch(OpResidFirst<Tin>{v0, p0 ? d0 : dbuf, b64, rfine, ld, cs.bnorm, cs.relres,
                                                 cs.active_out, h->wexp, cs.rexp[0], rx_cur, cs.rexp[0], pred},
                               mat_bytes(L0, 4) + v64 + 2 * vec_bytes(n, ld, 1, sizeof(Tin)));
                    }
                }
                if (!first_ff)
                    launch(OpResid64<Tin>{v0, x64, b64, rfine, ld, cs.bnorm, cs.relres, cs.active_out, o.tol, rx_cur,
                                          kScaled ? cs.rexp[(outer + 1) & 1] : nullptr, pred},
                           mat_bytes(L0, 8) + 2 * v64 + vec_bytes(n, ld, 1, sizeof(Tin)));
            }
            if (p0) elim_restrict();
            CFC_CUDA(cudaMemcpyAsync(h_active, cs.active_out, ld * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            CFC_CUDA(cudaMemcpyAsync(hrel.data(), cs.relres, ld * sizeof(double), cudaMemcpyDeviceToHost, s));
            if (outer == 0)
                CFC_CUDA(cudaMemcpyAsync(hbn.data(), cs.bnorm, ld * sizeof(double), cudaMemcpyDeviceToHost, s));
            CFC_CUDA(cudaStreamSynchronize(s));
            if (outer == 0)
                for (int c = 0; c < ld; ++c)
                    CFC_REQUIRE(std::isfinite(hbn[c]), LAP_EINVAL,
                                "a column of B has a non-finite 2-norm (NaN or infinite entries, or entries too "
                                "large to square)");
            int na = 0;
            bool finite = true;
            maxrel = 0.0;
            for (int c = 0; c < ld; ++c) {
                na += h_active[c] ? 1 : 0;
                if (!std::isfinite(hrel[c])) finite = false;
                if (std::isnan(hrel[c]) || hrel[c] > maxrel) maxrel = hrel[c];  // a NaN is kept
                if (std::isnan(maxrel)) break;
            }
            if (na == 0 && finite) {
                converged = true;
                break;
            }
            // a non-finite residual cannot recover: stop with LAP_ENOCONV
            if (!finite || outer >= o.max_outer || past_trial_deadline()) break;
            // inner solve of L d = r; d lives in lt-independent buffer `dbuf`
            inner_total += inner_pcg(dbuf, o.max_inner, itol);
            if (p0) elim_back();
            rowsd<0>(n, OpAddCorr<Tin>{x64, p0 ? d0 : dbuf, ld, cs.active_out, rx_cur, op_wexp()},
                     2 * v64 + vec_bytes(n, ld, 1, sizeof(Tin)));
        }
        // zero-mean result, copied out unpadded (direct: left as is)
        if (!direct) {
            rowsd<1>(n, OpColMean64{x64, ld, 1.0 / n, cs.mu}, v64);
            rowsd<1>(n, OpSubMean64{x64, x64, ld, cs.mu, nullptr}, 2 * v64);
            const int64_t tot = n * k;
            const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 8 * num_sms());
            CFC_LAUNCH(LAP_KF_BLAS1, s, v64 * 2, k_copy_unpad, blocks, 256, 0, x64, ld, X, k, n);
        }
        CFC_CUDA(cudaStreamSynchronize(s));
        if (info) {
            info->outer_iters = outer;
            info->inner_iters = inner_total;
            info->max_rel_residual = maxrel;
            info->k_tile = KT;
            info->levels_used = nlev;
            info->nu_coarse = nu_coarse;
            info->cycle = cycle;
            info->coarse_scale = gamma;
            info->w_levels = cycle == 2 ? w_levels : 0;
            info->first_residual_ff = used_ff ? 1 : 0;
        }
        return converged ? LAP_OK : LAP_ENOCONV;
    }

    template <int NR, class Op>
    void rowsd(int64_t n, const Op &op, double bytes) {
        const int nvb = (int)((n + RPB64 - 1) / RPB64);
        const int gx = NR > 0 ? red_grid(nvb) : plain_grid(nvb);
        dim3 grid(gx, ntiles64);
        CFC_LAUNCH(LAP_KF_BLAS1, s, bytes, (k_rows<double, K64, NR, Op>), grid, kBlock, 0, (int)n, op, rb);
    }

    Tin *dbuf = nullptr;
    bool direct = false;
};

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

template <typename Tin, int KT>
lap_status_t run_solver(lap_hierarchy *h, int32_t k, const double *B, double *X, const lap_solve_opts_t &o,
                        cudaStream_t s, lap_solve_info_t *info, bool direct) {
    const int ld = ((k + KT - 1) / KT) * KT;
    const int ntiles = ld / KT;
    CFC_REQUIRE(ntiles <= kMaxTiles, LAP_EBUDGET, "too many column tiles");
    Solver<Tin, KT> S(h, s, k, ld, o);
    const int nlev = S.nlev;
    // workspace layout: G itself (level 0: FP64 residual and, with an
    // elimination level, the FP32 residual and correction), then the cycle
    // levels p0 .. p0 + nlev - 1
    const int p0 = S.p0;
    const int64_t n0 = h->lv[0].n, ntop = h->lv[p0].n;
    int64_t max_chunks = std::max<int64_t>(h->lv[0].n_chunks, h->lv[0].pull_n_chunks);
    for (int l = 0; l < nlev; ++l) max_chunks = std::max<int64_t>(max_chunks, h->lv[p0 + l].n_chunks);
    std::vector<size_t> sizes;
    int64_t n_long_total = 0;
    for (int l = 0; l < nlev; ++l) n_long_total += h->lv[p0 + l].n_long;
    // arrival counters first: reduction tickets, then the long-row counters
    // of every level; zero at allocation, and every launch leaves them zero
    const size_t counter_bytes = align_up(kMaxTiles * 4 + kMaxTiles * kMaxTeams * 4 + n_long_total * kMaxTiles * 4);
    sizes.push_back(counter_bytes);
    sizes.push_back(direct ? 0 : align_up(n0 * ld * 8));  // b64 (direct: the caller's block)
    sizes.push_back(direct ? 0 : align_up(n0 * ld * 8));  // x64 (direct: the caller's block)
    sizes.push_back(align_up(ntop * ld * sizeof(Tin)));  // r
    sizes.push_back(align_up(ntop * ld * sizeof(Tin)));  // z
    sizes.push_back(align_up(ntop * ld * sizeof(Tin)));  // p
    sizes.push_back(align_up(ntop * ld * sizeof(Tin)));  // q
    sizes.push_back(align_up(ntop * ld * sizeof(Tin)));  // d
    sizes.push_back(align_up(ntop * ld * sizeof(Tin)));  // t0
    sizes.push_back(p0 ? align_up(n0 * ld * sizeof(Tin)) : 0);  // r0 (FP32 residual on G)
    sizes.push_back(p0 ? align_up(n0 * ld * sizeof(Tin)) : 0);  // d0 (correction on G)
    for (int l = 1; l < nlev; ++l)
        for (int v = 0; v < 3; ++v) sizes.push_back(align_up((size_t)h->lv[p0 + l].n * ld * sizeof(Tin)));
    sizes.push_back(align_up(std::max<int64_t>(max_chunks, 1) * ld * 8));  // chunk partials (FP64 size)
    // blocks of any launch: at most ceil(n/8) row blocks (8 = fewest rows per
    // block) plus one block per long row or one per 8 chunks
    int64_t max_blocks = 1;
    for (int l = -1; l < nlev; ++l) {
        const Level &Ll = l < 0 ? h->lv[0] : h->lv[p0 + l];
        max_blocks = std::max<int64_t>(
            max_blocks, (Ll.n + 7) / 8 + std::max<int64_t>(Ll.n_long, (Ll.n_chunks + 7) / 8) + 1);
    }
    const int P = (int)std::min<int64_t>(kRedMaxBlocks, max_blocks);
    sizes.push_back(align_up((size_t)ntiles * 4 * KT * P * 8));          // reduction partials
    sizes.push_back(align_up((size_t)ntiles * 4 * KT * kMaxTeams * 8));  // team partials
    sizes.push_back(align_up(ld * 8) * 10);                       // column scalars
    sizes.push_back(align_up(ld * 4) * 4);                        // column flags, residual exponents
    size_t total = 0;
    for (size_t z : sizes) total += z;
    char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(h->ws_mu);
        lap_hierarchy::Workspace &w = h->ws[s];
        if (w.bytes < total) {
            w.buf.release();  // stream-ordered: after this stream's earlier solves
            w.buf.alloc(total, s);
            w.bytes = total;
            w.zero_bytes = 0;
        }
        // after a solve exactly its counter region is known to be zero; a
        // larger region (more levels) also covers former data
        if (counter_bytes > w.zero_bytes)
            CFC_CUDA(cudaMemsetAsync(w.buf.get() + w.zero_bytes, 0, counter_bytes - w.zero_bytes, s));
        w.zero_bytes = counter_bytes;
        base = w.buf.get();
    }
    // the row kernels move 32-byte vectors: every block must start 32-byte
    // aligned (pool blocks are; the workspace is carved in 256-byte steps)
    CFC_REQUIRE(((uintptr_t)base & 255) == 0, LAP_ECUDA, "internal: solve workspace not 256-byte aligned");
    CFC_REQUIRE(!direct || (((uintptr_t)B & 31) == 0 && ((uintptr_t)X & 31) == 0), LAP_ECUDA,
                "internal: padded blocks not 32-byte aligned");
    size_t off = 0;
    auto take = [&](size_t i) {
        char *p = base + off;
        off += sizes[i];
        if (off > total) throw Error{LAP_ECUDA, "internal: workspace layout overflow"};
        return p;
    };
    size_t idx = 0;
    S.rb.counter = (uint32_t *)take(idx++);
    S.rb.team_counter = S.rb.counter + kMaxTiles;
    {
        uint32_t *c = S.rb.team_counter + (size_t)kMaxTiles * kMaxTeams;
        S.long_cnt.assign(nlev, nullptr);
        for (int l = 0; l < nlev; ++l) {
            S.long_cnt[l] = c;
            c += (size_t)h->lv[p0 + l].n_long * kMaxTiles;
        }
    }
    S.b64 = (double *)take(idx++);
    S.x64 = (double *)take(idx++);
    S.direct = direct;
    if (direct) {  // caller's padded blocks are used in place
        S.b64 = const_cast<double *>(B);
        S.x64 = X;
    }
    S.r = (Tin *)take(idx++);
    S.z = (Tin *)take(idx++);
    S.p = (Tin *)take(idx++);
    S.q = (Tin *)take(idx++);
    S.dbuf = (Tin *)take(idx++);
    S.t0 = (Tin *)take(idx++);
    S.r0 = p0 ? (Tin *)take(idx) : nullptr;
    ++idx;
    S.d0 = p0 ? (Tin *)take(idx) : nullptr;
    ++idx;
    Tin *t0 = S.t0;
    S.lb.assign(nlev, nullptr);
    S.lx.assign(nlev, nullptr);
    S.lt.assign(nlev, nullptr);
    S.lb[0] = S.r;
    S.lx[0] = S.z;
    S.lt[0] = t0;
    for (int l = 1; l < nlev; ++l) {
        S.lb[l] = (Tin *)take(idx++);
        S.lx[l] = (Tin *)take(idx++);
        S.lt[l] = (Tin *)take(idx++);
    }
    {
        char *cp = take(idx++);  // one buffer, viewed in the inner type or FP64
        S.chunk_part = (Tin *)cp;
        S.chunk_part64 = (double *)cp;
    }
    S.rb.part = (double *)take(idx++);
    S.rb.team_part = (double *)take(idx++);
    {
        char *cd = take(idx++);
        const size_t st = align_up(ld * 8);
        S.cs.bnorm = (double *)(cd + 0 * st);
        S.cs.relres = (double *)(cd + 1 * st);
        S.cs.alpha = (double *)(cd + 2 * st);
        S.cs.beta = (double *)(cd + 3 * st);
        S.cs.rz = (double *)(cd + 4 * st);
        S.cs.rr0 = (double *)(cd + 5 * st);
        S.cs.mu = (double *)(cd + 6 * st);
        S.cs.alpha_t = (void *)(cd + 7 * st);
        S.cs.beta_t = (void *)(cd + 8 * st);
        S.cs.mu_t = (void *)(cd + 9 * st);
        char *cf = take(idx++);
        S.cs.active_out = (int32_t *)cf;
        S.cs.active_in = (int32_t *)(cf + align_up(ld * 4));
        S.cs.rexp[0] = (int32_t *)(cf + 2 * align_up(ld * 4));
        S.cs.rexp[1] = (int32_t *)(cf + 3 * align_up(ld * 4));
    }
    // arrival counters must start at zero (every kernel leaves them at zero)
    CFC_CUDA(cudaMemsetAsync(S.rb.counter, 0, kMaxTiles * 4 + kMaxTiles * kMaxTeams * 4, s));
    CFC_CUDA(cudaMemsetAsync(S.cs.active_in, 0, ld * 4, s));
    // residual exponents stay 0 in FP64 solves (no scaling)
    CFC_CUDA(cudaMemsetAsync(S.cs.rexp[0], 0, 2 * align_up(ld * 4), s));
    S.h_active = pinned_scratch();
    return S.run(B, X, info);
}

}  // namespace

int num_sms_public() { return num_sms(); }

int32_t *pinned_scratch() {
    thread_local int32_t *buf = nullptr;
    if (!buf) CFC_CUDA(cudaMallocHost((void **)&buf, 8192 * sizeof(int32_t)));
    return buf;
}

namespace {

lap_status_t dispatch(lap_hierarchy *h, int32_t k, const double *B, double *X, const lap_solve_opts_t &o,
                      cudaStream_t s, lap_solve_info_t *info, int kt, bool direct) {
    const bool fp64 = (o.precision == LAP_FP64);
    if (fp64) {
        switch (kt) {
            case 16: return run_solver<double, 16>(h, k, B, X, o, s, info, direct);
            case 32: return run_solver<double, 32>(h, k, B, X, o, s, info, direct);
            default: return run_solver<double, 64>(h, k, B, X, o, s, info, direct);
        }
    }
    switch (kt) {
        case 16: return run_solver<float, 16>(h, k, B, X, o, s, info, direct);
        case 32: return run_solver<float, 32>(h, k, B, X, o, s, info, direct);
        case 64: return run_solver<float, 64>(h, k, B, X, o, s, info, direct);
        default: return run_solver<float, 128>(h, k, B, X, o, s, info, direct);
    }
}

// Autotuned configuration, per graph and solve configuration: the first
// solve with a new key times complete solves (depths, smoother degrees,
// cycles, coarse scales, column tiles) and keeps the fastest that converged
// (a one-time cost, like a library picking kernels by timing them).  The key
// holds the graph's fingerprint (its CSR entries and weights), so two graphs
// of equal size but different structure get their own choices.  The table
// can be written to and read from a JSON file (lap_tune_save / lap_tune_load,
// or the file named by LAP_TUNE_CACHE), so that a later process repeats a
// choice, and with it the bits of every solve, instead of timing again.
struct TuneKey {
    uint64_t fp;
    int64_t n, nnz;
    int k, precision, kt, smoother, nu_pre, nu_post, nu_coarse, cycle;
    double scale;
    int w_levels;
    bool operator<(const TuneKey &o) const {
        return std::tie(fp, n, nnz, k, precision, kt, smoother, nu_pre, nu_post, nu_coarse, cycle, scale, w_levels) <
               std::tie(o.fp, o.n, o.nnz, o.k, o.precision, o.kt, o.smoother, o.nu_pre, o.nu_post, o.nu_coarse,
                        o.cycle, o.scale, o.w_levels);
    }
};
struct TuneChoice {
    int kt, levels, nu_coarse, cycle;
    double scale;
    int w_levels = 0;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune;

// one entry per line: {"key": [fp, n, nnz, k, precision, kt, smoother, nu_pre,
// nu_post, nu_coarse, cycle, scale, w_levels], "choice": [kt, levels,
// nu_coarse, cycle, scale, w_levels]}; fp in hexadecimal, doubles with 17
// significant digits (exact round trip).  Caller holds g_tune_mu.
void tune_write_locked(const char *path) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    CFC_REQUIRE(f, LAP_EINVAL, std::string("cannot write ") + tmp);
    std::fprintf(f, "{\"format\": \"lap_tune_v1\", \"entries\": [\n");
    size_t i = 0;
    for (const auto &e : g_tune) {
        const TuneKey &k = e.first;
        const TuneChoice &c = e.second;
        std::fprintf(f,
                     "{\"key\": [\"%016llx\", %lld, %lld, %d, %d, %d, %d, %d, %d, %d, %d, %.17g, %d], "
                     "\"choice\": [%d, %d, %d, %d, %.17g, %d]}%s\n",
                     (unsigned long long)k.fp, (long long)k.n, (long long)k.nnz, k.k, k.precision, k.kt, k.smoother,
                     k.nu_pre, k.nu_post, k.nu_coarse, k.cycle, k.scale, k.w_levels, c.kt, c.levels, c.nu_coarse,
                     c.cycle, c.scale, c.w_levels, ++i < g_tune.size() ? "," : "");
    }
    std::fprintf(f, "]}\n");
    const bool ok = std::fclose(f) == 0;
    CFC_REQUIRE(ok && std::rename(tmp.c_str(), path) == 0, LAP_EINVAL, std::string("cannot write ") + path);
}

// reads the entries written by tune_write_locked; returns how many it added
int tune_read_locked(const char *path) {
    FILE *f = std::fopen(path, "r");
    CFC_REQUIRE(f, LAP_EINVAL, std::string("cannot read ") + path);
    char line[1024];
    int added = 0;
    while (std::fgets(line, sizeof line, f)) {
        const char *p = std::strstr(line, "\"key\": [\"");
        if (!p) continue;
        unsigned long long fp = 0;
        long long n = 0, nnz = 0;
        TuneKey k{};
        TuneChoice c{};
        const int got = std::sscanf(p, "\"key\": [\"%llx\", %lld, %lld, %d, %d, %d, %d, %d, %d, %d, %d, %lf, %d], "
                                       "\"choice\": [%d, %d, %d, %d, %lf, %d]",
                                    &fp, &n, &nnz, &k.k, &k.precision, &k.kt, &k.smoother, &k.nu_pre, &k.nu_post,
                                    &k.nu_coarse, &k.cycle, &k.scale, &k.w_levels, &c.kt, &c.levels, &c.nu_coarse,
                                    &c.cycle, &c.scale, &c.w_levels);
        if (got != 19) {
            std::fclose(f);
            throw Error{LAP_EINVAL, std::string("malformed tuning entry in ") + path};
        }
        k.fp = fp;
        k.n = n;
        k.nnz = nnz;
        added += g_tune.emplace(k, c).second ? 1 : 0;
    }
    std::fclose(f);
    return added;
}

// LAP_TUNE_CACHE: read once per process before the first tuning; written
// after every new choice
const char *tune_cache_path() {
    static const char *p = std::getenv("LAP_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}
void tune_cache_load_once_locked() {
    static bool done = false;
    if (done) return;
    done = true;
    const char *p = tune_cache_path();
    if (!p) return;
    if (FILE *f = std::fopen(p, "r")) {
        std::fclose(f);
        tune_read_locked(p);
    }
}

}  // namespace

int solve_tile(int32_t k, const lap_solve_opts_t &o) {
    int kt = o.k_tile;
    const bool fp64 = (o.precision == LAP_FP64);
    if (kt == 0) kt = (k >= 64) ? 64 : (k > 16 ? 32 : 16);
    if (fp64 && kt > 64) kt = 64;
    while ((k + kt - 1) / kt > kMaxTiles) kt *= 2;
    return kt;
}

int solve_ld(int32_t k, const lap_solve_opts_t &o) {
    const int kt = solve_tile(k, o);
    return ((k + kt - 1) / kt) * kt;
}

namespace {
// Autotuned configuration (caller holds the hierarchy exclusively): tile
// width (when not given), depth, smoother degree, cycle shape and coarse
// scale (those not given), chosen by timing complete solves the first time a
// graph size and configuration is seen.  Leaves the choice in o and returns
// its tile width.
template <class PrepareBf16>
int tune(lap_hierarchy *h, int32_t k, const double *B, double *X, lap_solve_opts_t &o, cudaStream_t s,
         lap_solve_info_t *info, int kt, bool direct, PrepareBf16 &&prepare_bf16) {
    const TuneKey key{h->fingerprint, h->lv[0].n, h->lv[0].nnz, k,         o.precision, o.k_tile,
                      o.smoother,     o.nu_pre,   o.nu_post,    o.nu_coarse, o.cycle, o.coarse_scale, o.w_levels};
    auto apply = [&](const TuneChoice &c, lap_solve_opts_t &oo) {
        oo.levels_used = c.levels;
        oo.nu_coarse = c.nu_coarse;
        oo.cycle = c.cycle;
        oo.coarse_scale = c.scale;
        oo.w_levels = c.w_levels;
    };
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache_load_once_locked();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            apply(it->second, o);
            grow_levels(*h, o.levels_used, s);
            return it->second.kt;
        }
    }
    grow_levels(*h, 0, s);
    const int L = (int)h->lv.size() - h->p0;  // levels of the cycle
    prepare_bf16(L);
    const int nc_default = o.nu_coarse > 0 ? o.nu_coarse : std::max(std::max(1, o.nu_pre), 4);
    const int cyc_default = o.cycle > 0 ? o.cycle : 1;
    const double sc_default = o.coarse_scale > 0.0 ? o.coarse_scale : 1.0;
    cudaEvent_t e0, e1;
    CFC_CUDA(cudaEventCreate(&e0));
    CFC_CUDA(cudaEventCreate(&e1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evg{e0, e1};
    const bool verbose = std::getenv("LAP_TUNE_VERBOSE") != nullptr;
    lap_solve_opts_t trial_o = o;
    trial_o.max_outer = std::min(o.max_outer, 4);  // a failing candidate should not run long
    float best_cost = 0.f;
    int best = -1;
    std::vector<TuneChoice> tried;
    // a candidate's cost: its solve plus building its coarse levels (every new
    // hierarchy of this graph pays that again)
    // returns the candidate's cost, or -1 when it did not converge within the trial cap
    // A candidate is abandoned once it has run twice as long as the best one
    // so far (checked at the solve's host synchronisations).
    struct TrialLimits {
        ~TrialLimits() { t_trial_deadline = 0.0; }
    } limits_guard;
    auto trial = [&](const TuneChoice &c) -> float {
        lap_solve_opts_t oo = trial_o;
        apply(c, oo);
        // the solve's own check interval: checking more often would add host
        // synchronisations to every candidate's cost and favour fewer, dearer iterations
        t_trial_deadline = best >= 0 ? steady_seconds() + 2.0 * best_cost * 1e-3 : 0.0;
        CFC_CUDA(cudaEventRecord(e0, s));
        const lap_status_t st = dispatch(h, k, B, X, oo, s, info, c.kt, direct);
        t_trial_deadline = 0.0;
        CFC_CUDA(cudaEventRecord(e1, s));
        CFC_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        CFC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        double build = 0.0;
        for (int l = 1; l < c.levels && h->p0 + l < (int)h->level_ms.size(); ++l) build += h->level_ms[h->p0 + l];
        const float cost = ms + (float)build;
        if (verbose)
            std::fprintf(stderr,
                         "lap autotune n=%lld k=%d kt=%d levels=%d nu_coarse=%d cycle=%d w_levels=%d scale=%.2f "
                         "solve=%.3f ms build=%.3f ms status=%d\n",
                         (long long)h->lv[0].n, k, c.kt, c.levels, c.nu_coarse, c.cycle, c.w_levels, c.scale, ms,
                         build, (int)st);
        tried.push_back(c);
        if (st == LAP_OK && (best < 0 || cost < best_cost)) {
            best_cost = cost;
            best = (int)tried.size() - 1;
        }
        return st == LAP_OK ? cost : -1.f;
    };
    // untimed warm-up: first launches load kernels and size the workspace
    {
        lap_solve_opts_t oo = trial_o;
        apply({kt, 1, 1, 1, 1.0}, oo);
        oo.max_outer = 1;  // a couple of iterations is all this needs
        oo.max_inner = 2;
        dispatch(h, k, B, X, oo, s, info, kt, direct);
    }
    // stage 1: preconditioner, at the default tile width.  First a baseline
    // that converges on every graph family seen (the full-depth V-cycle), so
    // that every later candidate runs under a deadline.
    const double sc_base = o.coarse_scale > 0.0 ? o.coarse_scale : 1.5;
    const float base_cost = L >= 3 ? trial({kt, L, nc_default, cyc_default, sc_base}) : -1.f;
    if (o.nu_coarse > 0) {
        trial({kt, 1, o.nu_coarse, cyc_default, sc_default});
    } else {
        for (int d : {1, 2, 3, 4, 6, 8}) {
            const float cost = trial({kt, 1, d, cyc_default, sc_default});
            if (cost < 0 && d >= 2) break;  // smoothing alone does not reach the tolerance
        }
    }
    std::vector<int> depths;
    for (int l = 2; l <= L && l <= 4; ++l) depths.push_back(l);
    if (L > 4) depths.push_back(L);
    for (int l : depths) trial({kt, l, nc_default, cyc_default, sc_default});
    if (L >= 3) {
        // unsmoothed aggregation under-corrects; scaling the coarse correction helps
        double sc_best = sc_base;
        if (o.coarse_scale <= 0.0) {
            float sc_cost = base_cost;
            for (double sc : {1.8, 2.0}) {
                const float cost = trial({kt, L, nc_default, cyc_default, sc});
                if (cost >= 0 && (sc_cost < 0 || cost < sc_cost)) {
                    sc_best = sc;
                    sc_cost = cost;
                }
            }
        }
        // W-cycles, when the hierarchy pays at all: two coarse corrections on
        // the top 1, 2 or 3 levels or on all of them (each extra level doubles
        // the visits below it); two corrections at scale 2 overshoot, so at
        // most 1.5
        if (o.cycle == 0 && best >= 0 && tried[best].levels > 1)
            for (int w : {1, 2, 3, 0})
                if (w < L - 1) trial({kt, L, nc_default, 2, std::min(sc_best, 1.5), w});
    }
    // stage 2: the tile width, with the best preconditioner
    if (best >= 0 && o.k_tile == 0) {
        const TuneChoice b0 = tried[best];
        const bool fp64 = (o.precision == LAP_FP64);
        const int ld0 = ((k + kt - 1) / kt) * kt;
        for (int t : {16, 32, 64, 128}) {
            if (t == kt || (fp64 && t > 64) || (k + t - 1) / t > kMaxTiles) continue;
            if (((k + t - 1) / t) * t > ld0) continue;  // no more padding than the default
            TuneChoice c = b0;
            c.kt = t;
            trial(c);
        }
    }
    if (best < 0) {  // nothing converged within the trial cap: one full-length attempt at full depth
        apply({kt, L, nc_default, cyc_default, sc_default}, o);
        return kt;
    }
    const TuneChoice choice = tried[best];
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = choice;
        if (const char *p = tune_cache_path()) tune_write_locked(p);
    }
    apply(choice, o);
    return choice.kt;
}

lap_status_t solve_impl(lap_hierarchy *h, int32_t k, const double *B, double *X, const lap_solve_opts_t &o_in,
                        cudaStream_t s, lap_solve_info_t *info, bool direct) {
    CFC_REQUIRE(k >= 1 && k <= 4096, LAP_EINVAL, "need 1 <= k <= 4096");
    CFC_REQUIRE(B && X && B != X, LAP_EINVAL, "B and X must be distinct device buffers");
    CFC_REQUIRE(is_device_pointer(B) && is_device_pointer(X), LAP_EINVAL, "B and X must be device pointers");
    CFC_REQUIRE(o_in.tol > 0 && o_in.max_outer >= 0 && o_in.max_inner >= 1, LAP_EINVAL, "bad solve options");
    CFC_REQUIRE(o_in.precision == LAP_FP64 || o_in.precision == LAP_FP32_REFINED ||
                    o_in.precision == LAP_FP32_BF16COARSE_REFINED,
                LAP_EINVAL, "unknown precision mode");
    lap_solve_opts_t o = o_in;
    const bool fp64 = (o.precision == LAP_FP64);
    const int kt = solve_tile(k, o);
    CFC_REQUIRE(kt == 16 || kt == 32 || kt == 64 || (kt == 128 && !fp64), LAP_EINVAL, "k_tile must be 16/32/64/128");
    int kt_run = kt;
    {
        // phase 1, exclusive: settle the configuration and build what it needs
        // (lazy levels, BF16 copies, autotuning trials), all on this stream
        std::unique_lock<std::shared_mutex> ex(h->mu);
        const size_t levels_before = h->lv.size();
        int bf16_made = 0;
        auto prepare_bf16 = [&](int upto) {
            if (o.precision != LAP_FP32_BF16COARSE_REFINED) return;
            for (int l = h->p0 + 1; l < h->p0 + upto && l < (int)h->lv.size(); ++l)
                if (!h->lv[l].wbf.get()) {
                    ensure_bf16(h->lv[l], h->wexp, s);
                    ++bf16_made;
                }
        };
        if (o.levels_used > 0) {
            grow_levels(*h, o.levels_used, s);
        } else if (o.levels_used < 0) {  // every level
            grow_levels(*h, 0, s);
            o.levels_used = 0;
        } else {
            kt_run = tune(h, k, B, X, o, s, info, kt, direct, prepare_bf16);
        }
        prepare_bf16(o.levels_used > 0 ? o.levels_used : (int)h->lv.size() - h->p0);
        if (h->lv.size() != levels_before || bf16_made > 0) {
            // solves on other streams wait for what this call built
            if (!h->grown) CFC_CUDA(cudaEventCreateWithFlags(&h->grown, cudaEventDisableTiming));
            CFC_CUDA(cudaEventRecord(h->grown, s));
        }
    }
    // phase 2, shared: the solve itself (solves on other streams may run alongside)
    std::shared_lock<std::shared_mutex> sh(h->mu);
    if (h->grown) CFC_CUDA(cudaStreamWaitEvent(s, h->grown, 0));
    return dispatch(h, k, B, X, o, s, info, kt_run, direct);
}

}  // namespace

lap_status_t tune_save(const char *path) {
    CFC_REQUIRE(path && *path, LAP_EINVAL, "path must not be NULL or empty");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_write_locked(path);
    return LAP_OK;
}

lap_status_t tune_load(const char *path, int64_t *added) {
    CFC_REQUIRE(path && *path, LAP_EINVAL, "path must not be NULL or empty");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int a = tune_read_locked(path);
    if (added) *added = a;
    return LAP_OK;
}

int64_t tune_entries() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (int64_t)g_tune.size();
}

lap_status_t solve_multi(lap_hierarchy *h, int32_t k, const double *B, double *X, const lap_solve_opts_t &o,
                         cudaStream_t s, lap_solve_info_t *info) {
    return solve_impl(h, k, B, X, o, s, info, false);
}

// B and X already n x solve_ld(k) with zero padding columns, B's columns
// summing to zero up to rounding; X is returned without the mean removal
lap_status_t solve_multi_direct(lap_hierarchy *h, int32_t k, const double *B, double *X, const lap_solve_opts_t &o,
                                cudaStream_t s, lap_solve_info_t *info) {
    return solve_impl(h, k, B, X, o, s, info, true);
}

}  // namespace cfc
