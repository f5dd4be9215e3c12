// BiCGStab steps on device fields (van der Vorst 1992), with the complex
// scalars kept in device memory: each reduction's finish() derives the next
// scalar (alpha, omega, rho and beta), so one iteration needs no host round
// trip until its residual norm is read.
//
// Iteration on Mhat x = b (shadow residual r^ fixed since the last restart):
//   p = r + beta (p - omega v)         beta = (rho / rho_prev)(alpha / omega)
//   v = Mhat p;  alpha = rho / <r^, v>
//   s = r - alpha v
//   t = Mhat s;  omega = <t, s> / <t, t>
//   x += alpha p + omega s;  r = s - omega t;  rho_prev = rho, rho = <r^, r>
// A zero or non-finite <r^, v>, omega or rho sets the breakdown flag; the
// driver then recomputes the true residual and restarts.
#pragma once

#include "blas.cuh"

namespace wd {

// Scalar slots of a BiCGStab solve in the context's scalar array (complex
// values as re, im).  The CG steps use slots below 16.
constexpr int BS_RHO = 16, BS_RHO_PREV = 18, BS_ALPHA = 20, BS_OMEGA = 22, BS_BETA = 24, BS_R2 = 26,
              BS_RV = 28, BS_TS = 30, BS_TT = 32, BS_FLAG = 33, BS_S2 = 34;

struct zd {
    double re, im;
};
__device__ __forceinline__ zd zget(const double *s, int k) { return {s[k], s[k + 1]}; }
__device__ __forceinline__ void zput(double *s, int k, zd z)
{
    s[k] = z.re;
    s[k + 1] = z.im;
}
__device__ __forceinline__ zd zmul(zd a, zd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ zd zdiv(zd a, zd b)
{
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
// nonzero and finite
__device__ __forceinline__ bool zok(zd z)
{
    const double m = fabs(z.re) + fabs(z.im);
    return m > 0.0 && m < 1e300;
}

// y += c x over the 12 complex components of a site (c = cr + i ci)
template <typename T, typename TX>
__device__ __forceinline__ void site_zaxpy(T (&y)[24], T cr, T ci, const TX (&x)[24])
{
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const T xr = (T)x[2 * k], xi = (T)x[2 * k + 1];
        const T yr = y[2 * k], yi = y[2 * k + 1];
        y[2 * k] = fma(cr, xr, fma(-ci, xi, yr));
        y[2 * k + 1] = fma(cr, xi, fma(ci, xr, yi));
    }
}

// <a, b> = sum conj(a) b over a site, accumulated into (re, im)
template <typename T>
__device__ __forceinline__ void site_zdot(const T (&a)[24], const T (&b)[24], T &re, T &im)
{
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        re = fma(a[2 * k], b[2 * k], fma(a[2 * k + 1], b[2 * k + 1], re));
        im = fma(a[2 * k], b[2 * k + 1], fma(-a[2 * k + 1], b[2 * k], im));
    }
}

// p = r + beta p - (beta omega) v
template <int P> struct OpBicgP {
    static constexpr int NR = 0;
    FieldRef<P> r, p, v;
    const double *s;
    __device__ __forceinline__ void site(int j, double (&)[1]) const
    {
        using T = typename Prec<P>::real;
        const zd beta = zget(s, BS_BETA), bw = zmul(beta, zget(s, BS_OMEGA));
        T rv[24], pv[24], vv[24];
        r.load(j, rv);
        p.load(j, pv);
        v.load(j, vv);
        T o[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) o[k] = rv[k];
        site_zaxpy(o, (T)beta.re, (T)beta.im, pv);
        site_zaxpy(o, (T)-bw.re, (T)-bw.im, vv);
        p.store(j, o);
    }
    __device__ __forceinline__ void finish(const double (&)[1]) const {}
};

// <r^, v>;  alpha = rho / <r^, v>
template <int P> struct OpBicgAlpha {
    static constexpr int NR = 2;
    FieldRef<P> rh, v;
    double *s;
    __device__ __forceinline__ void site(int j, double (&acc)[2]) const
    {
        using T = typename Prec<P>::real;
        T a[24], b[24];
        rh.load(j, a);
        v.load(j, b);
        T re = 0, im = 0;
        site_zdot(a, b, re, im);
        acc[0] += (double)re;
        acc[1] += (double)im;
    }
    __device__ __forceinline__ void finish(const double (&d)[2]) const
    {
        const zd rv{d[0], d[1]};
        zput(s, BS_RV, rv);
        if (zok(rv)) {
            zput(s, BS_ALPHA, zdiv(zget(s, BS_RHO), rv));
        } else {
            zput(s, BS_ALPHA, zd{0.0, 0.0});
            s[BS_FLAG] = 1.0;
        }
    }
};

// s = r - alpha v;  |s|^2
template <int P> struct OpBicgS {
    static constexpr int NR = 1;
    FieldRef<P> r, v, out;
    double *s;
    __device__ __forceinline__ void site(int j, double (&acc)[1]) const
    {
        using T = typename Prec<P>::real;
        const zd al = zget(s, BS_ALPHA);
        T rv[24], vv[24];
        r.load(j, rv);
        v.load(j, vv);
        site_zaxpy(rv, (T)-al.re, (T)-al.im, vv);
        T n = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) n = fma(rv[k], rv[k], n);
        out.store(j, rv);
        acc[0] += (double)n;
    }
    __device__ __forceinline__ void finish(const double (&d)[1]) const { s[BS_S2] = d[0]; }
};

// <t, s> and |t|^2;  omega = <t, s> / |t|^2
template <int P> struct OpBicgOmega {
    static constexpr int NR = 3;
    FieldRef<P> t, sv;
    double *s;
    __device__ __forceinline__ void site(int j, double (&acc)[3]) const
    {
        using T = typename Prec<P>::real;
        T a[24], b[24];
        t.load(j, a);
        sv.load(j, b);
        T re = 0, im = 0, tt = 0;
        site_zdot(a, b, re, im);
#pragma unroll
        for (int k = 0; k < 24; ++k) tt = fma(a[k], a[k], tt);
        acc[0] += (double)re;
        acc[1] += (double)im;
        acc[2] += (double)tt;
    }
    __device__ __forceinline__ void finish(const double (&d)[3]) const
    {
        zput(s, BS_TS, zd{d[0], d[1]});
        s[BS_TT] = d[2];
        const bool ok = d[2] > 0.0 && d[2] < 1e300;
        const zd om = ok ? zd{d[0] / d[2], d[1] / d[2]} : zd{0.0, 0.0};
        zput(s, BS_OMEGA, om);
        if (!zok(om)) s[BS_FLAG] = 1.0;
    }
};

// x += alpha p + omega s;  r = s - omega t;  |r|^2 and rho = <r^, r>;
// beta = (rho / rho_prev)(alpha / omega).  x may have another precision.
template <int PX, int P> struct OpBicgUpdate {
    static constexpr int NR = 3;
    FieldRef<PX> x;
    FieldRef<P> p, sv, t, rh, r;
    double *s;
    __device__ __forceinline__ void site(int j, double (&acc)[3]) const
    {
        using T = typename Prec<P>::real;
        using TX = typename Prec<PX>::real;
        const zd al = zget(s, BS_ALPHA), om = zget(s, BS_OMEGA);
        T pv[24], svv[24];
        TX xv[24];
        p.load(j, pv);
        sv.load(j, svv);
        x.load(j, xv);
        site_zaxpy(xv, (TX)al.re, (TX)al.im, pv);
        site_zaxpy(xv, (TX)om.re, (TX)om.im, svv);
        x.store(j, xv);
        T tv[24], hv[24];
        t.load(j, tv);
        rh.load(j, hv);
        site_zaxpy(svv, (T)-om.re, (T)-om.im, tv);   // svv = r_new
        T n = 0, re = 0, im = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) n = fma(svv[k], svv[k], n);
        site_zdot(hv, svv, re, im);
        r.store(j, svv);
        acc[0] += (double)n;
        acc[1] += (double)re;
        acc[2] += (double)im;
    }
    __device__ __forceinline__ void finish(const double (&d)[3]) const
    {
        s[BS_R2] = d[0];
        const zd rho_old = zget(s, BS_RHO), rho{d[1], d[2]};
        zput(s, BS_RHO_PREV, rho_old);
        zput(s, BS_RHO, rho);
        const zd al = zget(s, BS_ALPHA), om = zget(s, BS_OMEGA);
        if (zok(rho) && zok(rho_old) && zok(om)) {
            zput(s, BS_BETA, zmul(zdiv(rho, rho_old), zdiv(al, om)));
        } else {
            zput(s, BS_BETA, zd{0.0, 0.0});
            s[BS_FLAG] = 1.0;
        }
    }
};

// After the residual was replaced by the true one: rho = <r^, r> and beta again.
template <int P> struct OpBicgRho {
    static constexpr int NR = 2;
    FieldRef<P> rh, r;
    double *s;
    __device__ __forceinline__ void site(int j, double (&acc)[2]) const
    {
        using T = typename Prec<P>::real;
        T a[24], b[24];
        rh.load(j, a);
        r.load(j, b);
        T re = 0, im = 0;
        site_zdot(a, b, re, im);
        acc[0] += (double)re;
        acc[1] += (double)im;
    }
    __device__ __forceinline__ void finish(const double (&d)[2]) const
    {
        const zd rho{d[0], d[1]}, rho_old = zget(s, BS_RHO_PREV);
        zput(s, BS_RHO, rho);
        const zd al = zget(s, BS_ALPHA), om = zget(s, BS_OMEGA);
        if (zok(rho) && zok(rho_old) && zok(om)) {
            zput(s, BS_BETA, zmul(zdiv(rho, rho_old), zdiv(al, om)));
        } else {
            zput(s, BS_BETA, zd{0.0, 0.0});
            s[BS_FLAG] = 1.0;
        }
    }
};

// Restart: r^ = r, rho = |r|^2, rho_prev = alpha = omega = 1, beta = rho, flag
// cleared (with p = v = 0 the next step gives p = r).
template <int P> struct OpBicgRestart {
    static constexpr int NR = 1;
    FieldRef<P> r, rh;
    double *s;
    __device__ __forceinline__ void site(int j, double (&acc)[1]) const
    {
        using T = typename Prec<P>::real;
        T rv[24];
        r.load(j, rv);
        rh.store(j, rv);
        T n = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) n = fma(rv[k], rv[k], n);
        acc[0] += (double)n;
    }
    __device__ __forceinline__ void finish(const double (&d)[1]) const
    {
        zput(s, BS_RHO, zd{d[0], 0.0});
        zput(s, BS_RHO_PREV, zd{1.0, 0.0});
        zput(s, BS_ALPHA, zd{1.0, 0.0});
        zput(s, BS_OMEGA, zd{1.0, 0.0});
        zput(s, BS_BETA, zd{d[0], 0.0});
        s[BS_R2] = d[0];
        s[BS_FLAG] = 0.0;
    }
};

} // namespace wd
