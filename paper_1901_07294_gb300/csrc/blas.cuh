// BLAS-1 on device fields with deterministic FP64 reductions.
//
// One thread per site (grid-stride).  A site's 24 reals are combined in the
// compute type of the field (FP32 for the 16/32-bit formats), each site's
// contribution is added in FP64, then FP64 warp shuffles, a fixed-order sum
// over the warps of the block, per-block partials in scratch memory, and the
// last block to finish (atomic ticket) sums the partials the same way (thread
// t takes partials t, t+256, ...), so the order is fixed.  The
// grid size depends only on the field size, the SM count and the kernel, so
// repeated calls give bitwise identical results.
#pragma once

#include "wd_device.cuh"

namespace wd {

constexpr int BLAS_THREADS = 256;
constexpr int MAX_RED_BLOCKS = 2048;
constexpr int MAX_NR = 4;

// Scratch used by one reduction: MAX_RED_BLOCKS*MAX_NR partials + a ticket.
struct RedScratch {
    double *partials;
    unsigned *ticket;
};

// A field seen as `nhalf` consecutive half fields of vh sites each.
template <int P> struct FieldRef {
    char *p;
    size_t half_bytes;
    int vh;
    __device__ __forceinline__ void load(int j, typename Prec<P>::real (&v)[24]) const
    {
        const int h = j >= vh;
        Spinor<P>::load(p + h * half_bytes, vh, j - h * vh, v);
    }
    __device__ __forceinline__ void store(int j, const typename Prec<P>::real (&v)[24]) const
    {
        const int h = j >= vh;
        Spinor<P>::store(p + h * half_bytes, vh, j - h * vh, v);
    }
};

// The site loop and the deterministic reduction of one BLAS operation over a
// grid of blocks along x (shared by blas_kernel and the per-member kernels of
// a request group, which run one operation per blockIdx.y).
template <typename Op> __device__ __forceinline__ void blas_body(const Op &op, const int nsite, const RedScratch &rs)
{
    constexpr int NR = Op::NR;
    double acc[NR > 0 ? NR : 1];
#pragma unroll
    for (int k = 0; k < (NR > 0 ? NR : 1); ++k) acc[k] = 0.0;
    // two sites per pass where the loop runs twice or more: the second site's
    // loads can then be in flight with the first's
    const int stride = gridDim.x * blockDim.x;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    for (; j + stride < nsite; j += 2 * stride) {
        op.site(j, acc);
        op.site(j + stride, acc);
    }
    if (j < nsite) op.site(j, acc);
    if constexpr (NR > 0) {
        __shared__ double sm[BLAS_THREADS / 32][NR];
        __shared__ bool last;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < NR; ++k)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], off);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < NR; ++k) sm[warp][k] = acc[k];
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                double s = 0.0;
                for (int w = 0; w < BLAS_THREADS / 32; ++w) s += sm[w][k];
                rs.partials[blockIdx.x * NR + k] = s;
            }
            __threadfence();
            const unsigned t = atomicAdd(rs.ticket, 1u);
            last = (t == gridDim.x - 1);
        }
        __syncthreads();
        if (last) {   // block-uniform: the whole last block sums the partials
            __threadfence();
            double s[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) s[k] = 0.0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += BLAS_THREADS)
#pragma unroll
                for (int k = 0; k < NR; ++k) s[k] += __ldcg(rs.partials + b * NR + k);
#pragma unroll
            for (int k = 0; k < NR; ++k)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], off);
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < NR; ++k) sm[warp][k] = s[k];
            __syncthreads();
            if (threadIdx.x == 0) {
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    s[k] = 0.0;
                    for (int w = 0; w < BLAS_THREADS / 32; ++w) s[k] += sm[w][k];
                }
                op.finish(s);
                *rs.ticket = 0u;   // ready for the next reduction
            }
        }
    }
}

template <typename Op>
__global__ void __launch_bounds__(BLAS_THREADS) blas_kernel(const Op op, const int nsite, const RedScratch rs)
{
    grid_dependency_enter();
    blas_body(op, nsite, rs);
}

// ---- operations -----------------------------------------------------------
// |x|^2
template <int P> struct OpNorm2 {
    static constexpr int NR = 1;
    FieldRef<P> x;
    double *out;
    __device__ __forceinline__ void site(int j, double (&a)[1]) const
    {
        typename Prec<P>::real v[24];
        x.load(j, v);
        typename Prec<P>::real s = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) s = fma(v[k], v[k], s);
        a[0] += (double)s;
    }
    __device__ __forceinline__ void finish(const double (&s)[1]) const { out[0] = s[0]; }
};

// <a, b> = sum conj(a) b  (re, im)
template <int PA, int PB> struct OpDot {
    static constexpr int NR = 2;
    FieldRef<PA> a;
    FieldRef<PB> b;
    double *out;
    __device__ __forceinline__ void site(int j, double (&acc)[2]) const
    {
        using T = typename Prec<PA>::real;
        T u[24];
        typename Prec<PB>::real w[24];
        a.load(j, u);
        b.load(j, w);
        T re = 0, im = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            re = fma(u[2 * k], to_real<T>(w[2 * k]), re);
            re = fma(u[2 * k + 1], to_real<T>(w[2 * k + 1]), re);
            im = fma(u[2 * k], to_real<T>(w[2 * k + 1]), im);
            im = fma(-u[2 * k + 1], to_real<T>(w[2 * k]), im);
        }
        acc[0] += (double)re;
        acc[1] += (double)im;
    }
    __device__ __forceinline__ void finish(const double (&s)[2]) const { out[0] = s[0]; out[1] = s[1]; }
};

// Re <p, q>; also alpha = num / Re<p,q> (CG step length) into out[1].
template <int P> struct OpDotReAlpha {
    static constexpr int NR = 1;
    FieldRef<P> p, q;
    double num;
    double *out;   // out[0] = Re<p,q>, out[1] = num / out[0]
    __device__ __forceinline__ void site(int j, double (&acc)[1]) const
    {
        typename Prec<P>::real u[24], w[24];
        p.load(j, u);
        q.load(j, w);
        typename Prec<P>::real s = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) s = fma(u[k], w[k], s);
        acc[0] += (double)s;
    }
    __device__ __forceinline__ void finish(const double (&s)[1]) const
    {
        out[0] = s[0];
        out[1] = num / s[0];
    }
};

// CG update with alpha read from device memory:
//   r -= alpha * Ap;  x += alpha * p;  returns |r|^2.   x may have another precision.
template <int PX, int PR> struct OpCgUpdate {
    static constexpr int NR = 1;
    FieldRef<PX> x;
    FieldRef<PR> r, p, ap;
    const double *alpha;
    double *out;
    __device__ __forceinline__ void site(int j, double (&acc)[1]) const
    {
        using T = typename Prec<PR>::real;
        using TX = typename Prec<PX>::real;
        const double al = *alpha;
        T rv[24], pv[24], av[24];
        TX xv[24];
        r.load(j, rv);
        ap.load(j, av);
        const T a = (T)al;
        T s = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            rv[k] = fma(-a, av[k], rv[k]);
            s = fma(rv[k], rv[k], s);
        }
        r.store(j, rv);
        p.load(j, pv);
        x.load(j, xv);
        const TX ax = (TX)al;
#pragma unroll
        for (int k = 0; k < 24; ++k) xv[k] = fma(ax, to_real<TX>(pv[k]), xv[k]);
        x.store(j, xv);
        acc[0] += (double)s;
    }
    __device__ __forceinline__ void finish(const double (&s)[1]) const { out[0] = s[0]; }
};

// r = b - y; returns |r|^2 (used for the true residual, FP64; y may be a
// double-word field, widened exactly to FP64 first).
template <int P, int PY = P> struct OpXmyNorm {
    static constexpr int NR = 1;
    FieldRef<P> b;
    FieldRef<PY> y;
    FieldRef<P> r;
    double *out;
    __device__ __forceinline__ void site(int j, double (&acc)[1]) const
    {
        using T = typename Prec<P>::real;
        T bv[24];
        typename Prec<PY>::real yv[24];
        b.load(j, bv);
        y.load(j, yv);
        T s = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            bv[k] -= to_real<T>(yv[k]);
            s = fma(bv[k], bv[k], s);
        }
        r.store(j, bv);
        acc[0] += (double)s;
    }
    __device__ __forceinline__ void finish(const double (&s)[1]) const { out[0] = s[0]; }
};

// ---- CG steps whose scalars live in device memory (replayable in a graph) ----
// Scalar slots: s[0] = |r|^2 now, s[1] = pAp, s[2] = alpha, s[4] = |r|^2 of
// the previous step, s[5] = beta for the next direction update, s[6] =
// breakdown flag.

// pAp = Re<p, Ap>;  alpha = s[0] / pAp  (alpha = 0 and the flag set on breakdown)
template <int P> struct OpDotAlphaDev {
    static constexpr int NR = 1;
    FieldRef<P> p, q;
    double *s;
    __device__ __forceinline__ void site(int j, double (&acc)[1]) const
    {
        typename Prec<P>::real u[24], w[24];
        p.load(j, u);
        q.load(j, w);
        typename Prec<P>::real t = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) t = fma(u[k], w[k], t);
        acc[0] += (double)t;
    }
    __device__ __forceinline__ void finish(const double (&r)[1]) const
    {
        s[1] = r[0];
        const bool ok = r[0] > 0.0 && r[0] < 1e300;
        s[2] = ok ? s[0] / r[0] : 0.0;
        if (!ok) s[6] = 1.0;
    }
};

// r -= alpha Ap; x += alpha p (alpha = s[2]); then s[4] = s[0], s[0] = |r|^2.
template <int PX, int PR> struct OpCgUpdateDev {
    static constexpr int NR = 1;
    OpCgUpdate<PX, PR> u;
    double *s;
    __device__ __forceinline__ void site(int j, double (&acc)[1]) const { u.site(j, acc); }
    __device__ __forceinline__ void finish(const double (&r)[1]) const
    {
        s[4] = s[0];
        s[0] = r[0];
    }
};

// p = r + beta p with beta = s[5] (= s[0] / s[4], set once per iteration by the
// solve's control step, or by the host after a reliable update)
template <int P> struct OpXpayDev {
    static constexpr int NR = 0;
    FieldRef<P> r, p;
    const double *s;
    __device__ __forceinline__ void site(int j, double (&)[1]) const
    {
        using T = typename Prec<P>::real;
        const T beta = (T)s[5];
        T rv[24], pv[24];
        r.load(j, rv);
        p.load(j, pv);
#pragma unroll
        for (int k = 0; k < 24; ++k) pv[k] = fma(beta, pv[k], rv[k]);
        p.store(j, pv);
    }
    __device__ __forceinline__ void finish(const double (&)[1]) const {}
};

// y = a x + b y   (no reduction)
template <int PX, int PY> struct OpAxpby {
    static constexpr int NR = 0;
    FieldRef<PX> x;
    FieldRef<PY> y;
    double a, b;
    __device__ __forceinline__ void site(int j, double (&)[1]) const
    {
        using T = typename Prec<PY>::real;
        typename Prec<PX>::real xv[24];
        T yv[24];
        x.load(j, xv);
        y.load(j, yv);
        const T ta = (T)a, tb = (T)b;
        if (b == 1.0) {   // y += a x (a reliable update's x += x_lo): one operation a real
#pragma unroll
            for (int k = 0; k < 24; ++k) yv[k] = fma(ta, to_real<T>(xv[k]), yv[k]);
        } else {
#pragma unroll
            for (int k = 0; k < 24; ++k) yv[k] = fma(ta, to_real<T>(xv[k]), tb * yv[k]);
        }
        y.store(j, yv);
    }
    __device__ __forceinline__ void finish(const double (&)[1]) const {}
};

// dst = src with a change of storage precision (no reduction)
template <int PD, int PS> struct OpConvert {
    static constexpr int NR = 0;
    FieldRef<PD> dst;
    FieldRef<PS> src;
    __device__ __forceinline__ void site(int j, double (&)[1]) const
    {
        typename Prec<PS>::real sv[24];
        typename Prec<PD>::real dv[24];
        src.load(j, sv);
#pragma unroll
        for (int k = 0; k < 24; ++k) dv[k] = to_real<typename Prec<PD>::real>(sv[k]);
        dst.store(j, dv);
    }
    __device__ __forceinline__ void finish(const double (&)[1]) const {}
};

} // namespace wd
