// Wilson hopping kernel: one thread per output site of one parity.
//
// For output parity p and checkerboard site i the kernel computes
//     acc = sum_mu (1 + s_f gamma_mu) U_mu(x) psi(x+mu)
//         +        (1 + s_b gamma_mu) U_mu(x-mu)^dagger psi(x-mu)
// with s_f = -1, s_b = +1 (the library's H; Sec. II-A, Eq. (1) up to the
// gamma5 similarity) or the swapped signs for gamma5 H gamma5 (DAG), and
// stores out = a*x + b*acc.  Each direction: load the 24-real neighbour
// spinor (16-byte plane loads), project to two spin components (12 reals),
// load the link (reconstructing row 3 when 12 reals are stored), multiply
// the two colour vectors by U or U^dagger, and rebuild the two lower spin
// components from the upper ones.  1320 flops per output site.
#pragma once

#include "launch.cuh"
#include "wd_device.cuh"

namespace wd {

struct HopArgs {
    const char *in[2];    // neighbour source for output parity p (a half field of parity 1-p)
    const char *x[2];     // axpy term of parity p (NULL if unused)
    char *out[2];         // output half field of parity p
    const char *gauge[2]; // links at sites of parity p: 4 mu blocks of `link_blk` bytes
    size_t link_blk;
    size_t rhs_stride;    // bytes between consecutive right-hand sides
    int L[4];
    int vh;
    int nparity;          // 2: blocks alternate parity (full operator); 1: parity0 only
    int parity0;
    int tneg;             // 1: antiperiodic in t (hops across the t boundary change sign)
    int topen;            // 1: open t boundary (a sub-domain): no hop crosses it (selects the TOPEN kernel)
    unsigned div_m[3];    // n / d for d = L[0]/2, L[1], L[2] as (n * m) >> s (set by hop_setup)
    int div_s[3];
    int *status;          // device status word for asynchronous errors (bounded waits); may be NULL
    double a, b;
};

// Division by an invariant integer (Granlund and Montgomery, 1994): for
// 0 <= n < 2^31, m = ceil(2^s / d) and s = 31 + ceil(log2 d) give
// floor(n m / 2^s) = floor(n / d) exactly (n (m d - 2^s) / (d 2^s) < 1/d).
__host__ __device__ __forceinline__ int div_inv(int n, unsigned m, int s)
{
    return (int)(((unsigned long long)(unsigned)n * m) >> s);
}
inline void div_magic(unsigned d, unsigned &m, int &s)
{
    int l = 0;
    while ((1ull << l) < d) ++l;
    s = 31 + l;
    m = (unsigned)((((unsigned long long)1 << s) + d - 1) / d);
}

// h0, h1 = upper two spin components of (1 + S gamma_MU) psi, chiral basis.
template <int MU, int S, typename T>
__device__ __forceinline__ void project(const T (&v)[24], cpx<T> (&h0)[3], cpx<T> (&h1)[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cpx<T> p0{v[2 * c], v[2 * c + 1]}, p1{v[6 + 2 * c], v[7 + 2 * c]};
        const cpx<T> p2{v[12 + 2 * c], v[13 + 2 * c]}, p3{v[18 + 2 * c], v[19 + 2 * c]};
        if constexpr (MU == 0) {        // h0 = p0 + S i p3, h1 = p1 + S i p2
            h0[c] = {p0.re - S * p3.im, p0.im + S * p3.re};
            h1[c] = {p1.re - S * p2.im, p1.im + S * p2.re};
        } else if constexpr (MU == 1) { // h0 = p0 - S p3, h1 = p1 + S p2
            h0[c] = {p0.re - S * p3.re, p0.im - S * p3.im};
            h1[c] = {p1.re + S * p2.re, p1.im + S * p2.im};
        } else if constexpr (MU == 2) { // h0 = p0 + S i p2, h1 = p1 - S i p3
            h0[c] = {p0.re - S * p2.im, p0.im + S * p2.re};
            h1[c] = {p1.re + S * p3.im, p1.im - S * p3.re};
        } else {                        // h0 = p0 + S p2, h1 = p1 + S p3
            h0[c] = {p0.re + S * p2.re, p0.im + S * p2.im};
            h1[c] = {p1.re + S * p3.re, p1.im + S * p3.im};
        }
    }
}

// acc += (1 + S gamma_MU) applied in the projected form: spins 0,1 get w0,w1
// and spins 2,3 are the fixed multiples of w0,w1 that the projector implies.
// FIRST: the first direction of a site, whose terms are assigned instead of
// added to zeros (the same values, without 24 additions).
// NC: colours held (3; 1 where a thread owns one colour row of the site).
template <int MU, int S, bool FIRST = false, typename T, int NC>
__device__ __forceinline__ void accumulate(cpx<T> (&acc)[4][NC], const cpx<T> (&w0)[NC], const cpx<T> (&w1)[NC])
{
    if constexpr (FIRST) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            acc[0][c] = w0[c];
            acc[1][c] = w1[c];
            if constexpr (MU == 0) {        // spin2 = -S i w1, spin3 = -S i w0
                acc[2][c] = {S * w1[c].im, -S * w1[c].re};
                acc[3][c] = {S * w0[c].im, -S * w0[c].re};
            } else if constexpr (MU == 1) { // spin2 = S w1, spin3 = -S w0
                acc[2][c] = {S * w1[c].re, S * w1[c].im};
                acc[3][c] = {-S * w0[c].re, -S * w0[c].im};
            } else if constexpr (MU == 2) { // spin2 = -S i w0, spin3 = S i w1
                acc[2][c] = {S * w0[c].im, -S * w0[c].re};
                acc[3][c] = {-S * w1[c].im, S * w1[c].re};
            } else {                        // spin2 = S w0, spin3 = S w1
                acc[2][c] = {S * w0[c].re, S * w0[c].im};
                acc[3][c] = {S * w1[c].re, S * w1[c].im};
            }
        }
        return;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        acc[0][c].re += w0[c].re; acc[0][c].im += w0[c].im;
        acc[1][c].re += w1[c].re; acc[1][c].im += w1[c].im;
        if constexpr (MU == 0) {        // spin2 += -S i w1, spin3 += -S i w0
            acc[2][c].re += S * w1[c].im; acc[2][c].im -= S * w1[c].re;
            acc[3][c].re += S * w0[c].im; acc[3][c].im -= S * w0[c].re;
        } else if constexpr (MU == 1) { // spin2 += S w1, spin3 += -S w0
            acc[2][c].re += S * w1[c].re; acc[2][c].im += S * w1[c].im;
            acc[3][c].re -= S * w0[c].re; acc[3][c].im -= S * w0[c].im;
        } else if constexpr (MU == 2) { // spin2 += -S i w0, spin3 += S i w1
            acc[2][c].re += S * w0[c].im; acc[2][c].im -= S * w0[c].re;
            acc[3][c].re -= S * w1[c].im; acc[3][c].im += S * w1[c].re;
        } else {                        // spin2 += S w0, spin3 += S w1
            acc[2][c].re += S * w0[c].re; acc[2][c].im += S * w0[c].im;
            acc[3][c].re += S * w1[c].re; acc[3][c].im += S * w1[c].im;
        }
    }
}

// project for 16-bit storage, from the twelve storage words: each of the 12
// outputs is one stored value plus or minus another, widened and added in
// one rounding (the result of project on the widened values, bit for bit).
template <int P, int MU, int S>
__device__ __forceinline__ void project_words(const unsigned (&u)[12], cpx<float> (&h0)[3], cpx<float> (&h1)[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const unsigned p0 = u[c], p1 = u[3 + c], p2 = u[6 + c], p3 = u[9 + c];
        if constexpr (MU == 0) {        // h0 = p0 + S i p3, h1 = p1 + S i p2
            h0[c] = {h16_pm<P, 0, 1, -S>(p0, p3), h16_pm<P, 1, 0, S>(p0, p3)};
            h1[c] = {h16_pm<P, 0, 1, -S>(p1, p2), h16_pm<P, 1, 0, S>(p1, p2)};
        } else if constexpr (MU == 1) { // h0 = p0 - S p3, h1 = p1 + S p2
            h0[c] = {h16_pm<P, 0, 0, -S>(p0, p3), h16_pm<P, 1, 1, -S>(p0, p3)};
            h1[c] = {h16_pm<P, 0, 0, S>(p1, p2), h16_pm<P, 1, 1, S>(p1, p2)};
        } else if constexpr (MU == 2) { // h0 = p0 + S i p2, h1 = p1 - S i p3
            h0[c] = {h16_pm<P, 0, 1, -S>(p0, p2), h16_pm<P, 1, 0, S>(p0, p2)};
            h1[c] = {h16_pm<P, 0, 1, S>(p1, p3), h16_pm<P, 1, 0, -S>(p1, p3)};
        } else {                        // h0 = p0 + S p2, h1 = p1 + S p3
            h0[c] = {h16_pm<P, 0, 0, S>(p0, p2), h16_pm<P, 1, 1, S>(p0, p2)};
            h1[c] = {h16_pm<P, 0, 0, S>(p1, p3), h16_pm<P, 1, 1, S>(p1, p3)};
        }
    }
}

// accumulate with every term weighted by f (the neighbour's scale times the
// hop coefficient): the weight rides on the additions as FMAs instead of
// costing 12 multiplications of U h per direction and 24 of the sum.
template <int MU, int S, bool FIRST = false>
__device__ __forceinline__ void accumulate_f(cpx<float> (&acc)[4][3], const cpx<float> (&w0)[3], const cpx<float> (&w1)[3],
                                             const float f)
{
    const float g = S * f;
    if constexpr (FIRST) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            acc[0][c] = {f * w0[c].re, f * w0[c].im};
            acc[1][c] = {f * w1[c].re, f * w1[c].im};
            if constexpr (MU == 0) {        // spin2 = -S i w1, spin3 = -S i w0
                acc[2][c] = {g * w1[c].im, -g * w1[c].re};
                acc[3][c] = {g * w0[c].im, -g * w0[c].re};
            } else if constexpr (MU == 1) { // spin2 = S w1, spin3 = -S w0
                acc[2][c] = {g * w1[c].re, g * w1[c].im};
                acc[3][c] = {-g * w0[c].re, -g * w0[c].im};
            } else if constexpr (MU == 2) { // spin2 = -S i w0, spin3 = S i w1
                acc[2][c] = {g * w0[c].im, -g * w0[c].re};
                acc[3][c] = {-g * w1[c].im, g * w1[c].re};
            } else {                        // spin2 = S w0, spin3 = S w1
                acc[2][c] = {g * w0[c].re, g * w0[c].im};
                acc[3][c] = {g * w1[c].re, g * w1[c].im};
            }
        }
        return;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[0][c].re = fmaf(f, w0[c].re, acc[0][c].re); acc[0][c].im = fmaf(f, w0[c].im, acc[0][c].im);
        acc[1][c].re = fmaf(f, w1[c].re, acc[1][c].re); acc[1][c].im = fmaf(f, w1[c].im, acc[1][c].im);
        if constexpr (MU == 0) {
            acc[2][c].re = fmaf(g, w1[c].im, acc[2][c].re); acc[2][c].im = fmaf(-g, w1[c].re, acc[2][c].im);
            acc[3][c].re = fmaf(g, w0[c].im, acc[3][c].re); acc[3][c].im = fmaf(-g, w0[c].re, acc[3][c].im);
        } else if constexpr (MU == 1) {
            acc[2][c].re = fmaf(g, w1[c].re, acc[2][c].re); acc[2][c].im = fmaf(g, w1[c].im, acc[2][c].im);
            acc[3][c].re = fmaf(-g, w0[c].re, acc[3][c].re); acc[3][c].im = fmaf(-g, w0[c].im, acc[3][c].im);
        } else if constexpr (MU == 2) {
            acc[2][c].re = fmaf(g, w0[c].im, acc[2][c].re); acc[2][c].im = fmaf(-g, w0[c].re, acc[2][c].im);
            acc[3][c].re = fmaf(-g, w1[c].im, acc[3][c].re); acc[3][c].im = fmaf(g, w1[c].re, acc[3][c].im);
        } else {
            acc[2][c].re = fmaf(g, w0[c].re, acc[2][c].re); acc[2][c].im = fmaf(g, w0[c].im, acc[2][c].im);
            acc[3][c].re = fmaf(g, w1[c].re, acc[3][c].re); acc[3][c].im = fmaf(g, w1[c].im, acc[3][c].im);
        }
    }
}

// w = U h (FWD) or U^dagger h.
template <bool FWD, typename T>
__device__ __forceinline__ void su3_mul(const cpx<T> (&U)[3][3], const cpx<T> (&h)[3], cpx<T> (&w)[3])
{
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        if constexpr (FWD) {
            cpx<T> s = cmul(U[r][0], h[0]);
            s = cfma(U[r][1], h[1], s);
            w[r] = cfma(U[r][2], h[2], s);
        } else {
            cpx<T> s = cmul_conj(U[0][r], h[0]);
            s = cfma_conj(U[1][r], h[1], s);
            w[r] = cfma_conj(U[2][r], h[2], s);
        }
    }
}

// One direction.  For 16-bit storage the projection reads the stored words,
// and the neighbour's per-site scale times wt (the hop coefficient, applied
// here instead of to the sum) weights the accumulated terms: the operation is
// linear, so neither the 24 stored reals nor the 12 of U h are scaled on
// their own.  neg: the hop crosses an antiperiodic boundary, U h changes sign
// (done here rather than in the stored links, whose 12-real form rebuilds
// row 3 assuming det U = 1).
template <int P, int RECON, int MU, int S, bool FWD, bool LNA = false, bool FIRST = false>
__device__ __forceinline__ void hop_dir(const char *in, const char *lblk, int vh, int nb, int li, bool neg,
                                        cpx<typename Prec<P>::real> (&acc)[4][3], const float wt = 1.0f)
{
    using T = typename Prec<P>::real;
    if constexpr (Prec<P>::scaled) {
        unsigned u[12];
        const float sc = Spinor<P>::load_words(in, vh, nb, u);
        cpx<float> h0[3], h1[3];
        project_words<P, MU, S>(u, h0, h1);
        cpx<float> U[3][3];
        Link<link_prec(P), RECON>::template load<LNA>(lblk, vh, li, U);
        cpx<float> w0[3], w1[3];
        su3_mul<FWD>(U, h0, w0);
        su3_mul<FWD>(U, h1, w1);
        accumulate_f<MU, S, FIRST>(acc, w0, w1, (neg ? -sc : sc) * wt);
        return;
    }
    T psi[24];
    Spinor<P>::load(in, vh, nb, psi);
    cpx<T> h0[3], h1[3];
    project<MU, S>(psi, h0, h1);
    cpx<T> U[3][3];
    Link<link_prec(P), RECON>::template load<LNA>(lblk, vh, li, U);
    cpx<T> w0[3], w1[3];
    su3_mul<FWD>(U, h0, w0);
    su3_mul<FWD>(U, h1, w1);
    if (neg) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            w0[c].re = -w0[c].re; w0[c].im = -w0[c].im;
            w1[c].re = -w1[c].re; w1[c].im = -w1[c].im;
        }
    }
    accumulate<MU, S, FIRST>(acc, w0, w1);
}

// 16-bit storage: out = a x + acc at site i, with acc the sum already
// weighted by the hop coefficient (hop_dir's wt); x is read as stored and its
// per-site scale folded into a.
template <int P, bool HAS_X>
__device__ __forceinline__ void store_weighted(const char *x, char *out, int vh, int i, float a,
                                               const cpx<float> (&acc)[4][3])
{
    float o[24];
    if constexpr (HAS_X) {
        unsigned u[12];
        const float ax = a * Spinor<P>::load_words(x, vh, i, u);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o[6 * s + 2 * c] = fmaf(ax, h16_f32<P, 0>(u[3 * s + c]), acc[s][c].re);
                o[6 * s + 2 * c + 1] = fmaf(ax, h16_f32<P, 1>(u[3 * s + c]), acc[s][c].im);
            }
    } else {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o[6 * s + 2 * c] = acc[s][c].re;
                o[6 * s + 2 * c + 1] = acc[s][c].im;
            }
    }
    Spinor<P>::store(out, vh, i, o);
}

// PF selects the memory schedule (chosen per problem by the autotuner):
//   0: directions in the order x+, x-, y+, y-, ..., no prefetch;
//   1: backward directions first (their data is mostly already in L2), the
//      forward links and the t-forward neighbour (the first touches of new
//      data) prefetched into L2 at thread start;
//   2: as 1, and the backward links prefetched too (even-odd blocks touch
//      every link once, so all of them come from DRAM).
// One output site: checkerboard index i < A.vh of parity p, right-hand side
// at byte offset roff.  Shared by hop_kernel and the persistent solver.
// TOPEN: the t boundary is open (a sub-domain of a decomposed lattice): the
// hops across it are skipped; their halo terms are added separately.
template <int P, int RECON, bool DAG, bool HAS_X, int PF, bool TOPEN = false, bool LNA = false>
__device__ __forceinline__ void hop_site(const HopArgs &A, const int p, const int i, const size_t roff)
{
    using T = typename Prec<P>::real;
    const int vh = A.vh;
    // parity-dependent pointers chosen by select: a runtime index into the
    // parameter struct would force a copy of it into local memory
    const char *in = (p ? A.in[1] : A.in[0]) + roff;
    const char *gf = p ? A.gauge[1] : A.gauge[0];
    const char *gb = p ? A.gauge[0] : A.gauge[1];

    // checkerboard index -> coordinates; x-parity bit from the site parity
    const int Lx = A.L[0], Ly = A.L[1], Lz = A.L[2], Lt = A.L[3];
    const int lxh = Lx >> 1;
    const int r = div_inv(i, A.div_m[0], A.div_s[0]);
    const int xh = i - r * lxh;
    const int r2 = div_inv(r, A.div_m[1], A.div_s[1]);
    const int y = r - r2 * Ly;
    const int t = div_inv(r2, A.div_m[2], A.div_s[2]);
    const int z = r2 - t * Lz;
    const int x = 2 * xh + ((p + y + z + t) & 1);
    const int sy = lxh, sz = lxh * Ly, st = sz * Lz;
    const int row = i - xh;
    const int xf = row + ((x + 1 == Lx ? 0 : x + 1) >> 1);
    const int xb = row + ((x == 0 ? Lx - 1 : x - 1) >> 1);
    const int yf = (y == Ly - 1) ? i - (Ly - 1) * sy : i + sy;
    const int yb = (y == 0) ? i + (Ly - 1) * sy : i - sy;
    const int zf = (z == Lz - 1) ? i - (Lz - 1) * sz : i + sz;
    const int zb = (z == 0) ? i + (Lz - 1) * sz : i - sz;
    const int tf = (t == Lt - 1) ? i - (Lt - 1) * st : i + st;
    const int tb = (t == 0) ? i + (Lt - 1) * st : i - st;
    const bool ntf = A.tneg && t == Lt - 1, ntb = A.tneg && t == 0;
    const bool dtf = !TOPEN || t != Lt - 1, dtb = !TOPEN || t != 0;   // t hops taken here

    constexpr int SF = DAG ? +1 : -1;   // forward projector 1 + SF gamma
    constexpr int SB = -SF;             // backward projector
    const size_t lb = A.link_blk;

    cpx<T> acc[4][3];   // set by the first direction (x, taken in every pass)
    // 16-bit storage: the hop coefficient b weights the accumulated terms
    const float wt = Prec<P>::scaled ? (float)A.b : 1.0f;

    using LK = Link<link_prec(P), RECON>;
    if constexpr (PF == 0 || PF == 5) {
        hop_dir<P, RECON, 0, SF, true, LNA, true>(in, gf + 0 * lb, vh, xf, i, false, acc, wt);
        hop_dir<P, RECON, 0, SB, false, LNA>(in, gb + 0 * lb, vh, xb, xb, false, acc, wt);
        hop_dir<P, RECON, 1, SF, true, LNA>(in, gf + 1 * lb, vh, yf, i, false, acc, wt);
        hop_dir<P, RECON, 1, SB, false, LNA>(in, gb + 1 * lb, vh, yb, yb, false, acc, wt);
        hop_dir<P, RECON, 2, SF, true, LNA>(in, gf + 2 * lb, vh, zf, i, false, acc, wt);
        hop_dir<P, RECON, 2, SB, false, LNA>(in, gb + 2 * lb, vh, zb, zb, false, acc, wt);
        if (dtf) hop_dir<P, RECON, 3, SF, true, LNA>(in, gf + 3 * lb, vh, tf, i, ntf, acc, wt);
        if (dtb) hop_dir<P, RECON, 3, SB, false, LNA>(in, gb + 3 * lb, vh, tb, tb, ntb, acc, wt);
    } else {
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) LK::prefetch(gf + mu * lb, vh, i);
        Spinor<P>::prefetch(in, vh, tf);
        if constexpr (PF == 2) {
            LK::prefetch(gb + 0 * lb, vh, xb);
            LK::prefetch(gb + 1 * lb, vh, yb);
            LK::prefetch(gb + 2 * lb, vh, zb);
            LK::prefetch(gb + 3 * lb, vh, tb);
        }
        hop_dir<P, RECON, 0, SB, false, LNA, true>(in, gb + 0 * lb, vh, xb, xb, false, acc, wt);
        hop_dir<P, RECON, 1, SB, false, LNA>(in, gb + 1 * lb, vh, yb, yb, false, acc, wt);
        hop_dir<P, RECON, 2, SB, false, LNA>(in, gb + 2 * lb, vh, zb, zb, false, acc, wt);
        if (dtb) hop_dir<P, RECON, 3, SB, false, LNA>(in, gb + 3 * lb, vh, tb, tb, ntb, acc, wt);
        hop_dir<P, RECON, 0, SF, true, LNA>(in, gf + 0 * lb, vh, xf, i, false, acc, wt);
        hop_dir<P, RECON, 1, SF, true, LNA>(in, gf + 1 * lb, vh, yf, i, false, acc, wt);
        hop_dir<P, RECON, 2, SF, true, LNA>(in, gf + 2 * lb, vh, zf, i, false, acc, wt);
        if (dtf) hop_dir<P, RECON, 3, SF, true, LNA>(in, gf + 3 * lb, vh, tf, i, ntf, acc, wt);
    }

    const T a = (T)A.a, b = (T)A.b;
    T o[24];
    if constexpr (Prec<P>::scaled) {   // acc already carries b
        store_weighted<P, HAS_X>(HAS_X ? (p ? A.x[1] : A.x[0]) + roff : nullptr, (p ? A.out[1] : A.out[0]) + roff,
                                 vh, i, (float)A.a, acc);
        return;
    } else if constexpr (HAS_X) {
        Spinor<P>::load((p ? A.x[1] : A.x[0]) + roff, vh, i, o);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o[6 * s + 2 * c] = a * o[6 * s + 2 * c] + b * acc[s][c].re;
                o[6 * s + 2 * c + 1] = a * o[6 * s + 2 * c + 1] + b * acc[s][c].im;
            }
    } else if (A.b == 1.0) {   // the bare hopping term: no scaling
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o[6 * s + 2 * c] = acc[s][c].re;
                o[6 * s + 2 * c + 1] = acc[s][c].im;
            }
    } else {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o[6 * s + 2 * c] = b * acc[s][c].re;
                o[6 * s + 2 * c + 1] = b * acc[s][c].im;
            }
    }
    Spinor<P>::store((p ? A.out[1] : A.out[0]) + roff, vh, i, o);
}

// PF 4 is schedule 1 compiled for 3 resident blocks of 256 threads per SM
// (at most 85 registers): more warps to hide latency, at the price of
// registers the compiler would otherwise use to hoist loads.  PF 5 is
// schedule 0 compiled for one block of 256 per SM: the FP64 kernel, bound by
// the FP64 pipe rather than by latency, then needs no spill stores (at the
// 128-register cap of two blocks it spills 200-550 bytes per thread).  PF 6
// is schedule 1 compiled the same way (double-word FP32, whose values take
// two registers like FP64 ones).
template <int P, int RECON, bool DAG, bool HAS_X, int PF, bool TOPEN = false, bool LNA = false>
__global__ void __launch_bounds__(256, PF == 4 ? 3 : (PF == 5 || PF == 6) ? 1 : 2) hop_kernel(const HopArgs A)
{
    grid_dependency_enter();
    int p, blk;
    if (A.nparity == 2) { p = blockIdx.x & 1; blk = blockIdx.x >> 1; }
    else { p = A.parity0; blk = blockIdx.x; }
    const int i = blk * blockDim.x + threadIdx.x;
    if (i >= A.vh) return;
    hop_site<P, RECON, DAG, HAS_X, PF, TOPEN, LNA>(A, p, i, (size_t)blockIdx.y * A.rhs_stride);
}

// lna: links loaded without L1 allocation (schedules 0 and 1 only).
template <int P, int RECON, bool DAG, bool HX>
cudaError_t launch_hop_pf(const HopArgs &A, dim3 grid, int threads, int pf, bool lna, cudaStream_t s)
{
    if (A.topen)   // sub-domain interior pass: schedule 1 with the open t boundary
        return wd_launch(hop_kernel<P, RECON, DAG, HX, 1, true>, grid, dim3(threads), 0, s, A);
    if (lna && pf == 0) return wd_launch(hop_kernel<P, RECON, DAG, HX, 0, false, true>, grid, dim3(threads), 0, s, A);
    if (lna && pf == 1) return wd_launch(hop_kernel<P, RECON, DAG, HX, 1, false, true>, grid, dim3(threads), 0, s, A);
    switch (pf) {
    case 0: return wd_launch(hop_kernel<P, RECON, DAG, HX, 0>, grid, dim3(threads), 0, s, A);
    case 1: return wd_launch(hop_kernel<P, RECON, DAG, HX, 1>, grid, dim3(threads), 0, s, A);
    case 2: return wd_launch(hop_kernel<P, RECON, DAG, HX, 2>, grid, dim3(threads), 0, s, A);
    case 5:
        if constexpr (P == PREC_F64) return wd_launch(hop_kernel<P, RECON, DAG, HX, 5>, grid, dim3(threads), 0, s, A);
        else return wd_launch(hop_kernel<P, RECON, DAG, HX, 0>, grid, dim3(threads), 0, s, A);
    default: return wd_launch(hop_kernel<P, RECON, DAG, HX, 4>, grid, dim3(threads), 0, s, A);
    }
}

// Double-word FP32 hop: schedule 0 (pf 5) or 1 (pf 6), one block of 256 per
// SM; no open-boundary pass.
template <int RECON, bool DAG, bool HX>
cudaError_t launch_hop_df(const HopArgs &A, dim3 grid, int threads, int pf, cudaStream_t s)
{
    if (pf == 6) return wd_launch(hop_kernel<PREC_DF, RECON, DAG, HX, 6>, grid, dim3(threads), 0, s, A);
    return wd_launch(hop_kernel<PREC_DF, RECON, DAG, HX, 5>, grid, dim3(threads), 0, s, A);
}

} // namespace wd
