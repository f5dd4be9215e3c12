// Paired FP32 arithmetic for the 16-bit storage formats.
//
// Blackwell executes add, mul and fma on a pair of FP32 values held in two
// adjacent registers as one instruction (the f32x2 forms): half the issue
// slots of two scalar instructions, the same FMA-pipe time.  The 16-bit hop
// kernels issue about 1650 instructions per site with the issue slots about
// 70 % busy, so fewer instructions at unchanged occupancy make them faster.
// One thread still computes one site; the pairs are the two spin components
// that the projected form carries through each direction:
//   (h0, h1)          the projected half spinor, from (psi_0, psi_1) and
//                     (psi_3, psi_2) or (psi_2, psi_3), which the
//                     half-to-float conversion writes straight into lanes;
//   (U h0, U h1)      the SU(3) product, with each link entry converted once
//                     and copied into both lanes;
//   (acc_0, acc_1), (acc_3, acc_2), (acc_2, acc_3)
//                     accumulators: directions x, y add into the first lower
//                     pair, z, t into the second (the projector pairs the
//                     spins crosswise there), summed once at the end.
// Per direction that is 60 paired operations in place of 120 scalar ones.
// The FP32 format would need register moves to form the pairs (its loads
// fill four consecutive registers of one site) and gains nothing; FP64 has no
// paired form: both use the scalar kernels.
#pragma once

#include "dslash_impl.cuh"

namespace wd {

using f2 = float2;
struct c2 {   // a pair of complex numbers: lanes x and y
    f2 re, im;
};

__device__ __forceinline__ f2 p_add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 p_neg(f2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ f2 p_sub(f2 a, f2 b) { return __fadd2_rn(a, p_neg(b)); }
__device__ __forceinline__ f2 p_mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 p_fma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a + S b for S = +1 or -1
template <int S> __device__ __forceinline__ f2 p_adds(f2 a, f2 b) { return S > 0 ? p_add(a, b) : p_sub(a, b); }
// a + (SX, SY) b lane-wise, SX, SY = +1 or -1
template <int SX, int SY> __device__ __forceinline__ f2 p_addss(f2 a, f2 b)
{
    if constexpr (SX == SY) return p_adds<SX>(a, b);
    else return p_fma(make_float2((float)SX, (float)SY), b, a);
}
__device__ __forceinline__ f2 p_bcast(float v) { return make_float2(v, v); }

// ---- 16-bit spinor words to spin pairs ---------------------------------
// A 16-bit spinor holds complex number 3 s + c (spin s, colour c) as one
// 32-bit word (re in the low half, im in the high half).
template <int P> __device__ __forceinline__ float lo16(unsigned w);
template <int P> __device__ __forceinline__ float hi16(unsigned w);
template <> __device__ __forceinline__ float lo16<PREC_F16>(unsigned w)
{
    return __low2float(*reinterpret_cast<const __half2 *>(&w));
}
template <> __device__ __forceinline__ float hi16<PREC_F16>(unsigned w)
{
    return __high2float(*reinterpret_cast<const __half2 *>(&w));
}
// a bfloat16 is the upper half of the float with the same value
template <> __device__ __forceinline__ float lo16<PREC_BF16>(unsigned w) { return __uint_as_float(w << 16); }
template <> __device__ __forceinline__ float hi16<PREC_BF16>(unsigned w) { return __uint_as_float(w & 0xffff0000u); }

// (spin a, spin b) of colour c from the 12 words of a site
template <int P> __device__ __forceinline__ c2 spin_pair(const unsigned (&w)[12], int sa, int sb, int c)
{
    const unsigned a = w[3 * sa + c], b = w[3 * sb + c];
    return c2{make_float2(lo16<P>(a), lo16<P>(b)), make_float2(hi16<P>(a), hi16<P>(b))};
}

// (h0, h1) = upper spin components of (1 + S gamma_MU) psi (chiral basis),
// from the unscaled 16-bit words of psi.
template <int P, int MU, int S>
__device__ __forceinline__ void sp_project(const unsigned (&w)[12], c2 (&h)[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const c2 u = spin_pair<P>(w, 0, 1, c);
        if constexpr (MU == 0) {        // h0 = p0 + S i p3, h1 = p1 + S i p2
            const c2 l = spin_pair<P>(w, 3, 2, c);
            h[c] = {p_adds<-S>(u.re, l.im), p_adds<S>(u.im, l.re)};
        } else if constexpr (MU == 1) { // h0 = p0 - S p3, h1 = p1 + S p2
            const c2 l = spin_pair<P>(w, 3, 2, c);
            h[c] = {p_addss<-S, S>(u.re, l.re), p_addss<-S, S>(u.im, l.im)};
        } else if constexpr (MU == 2) { // h0 = p0 + S i p2, h1 = p1 - S i p3
            const c2 l = spin_pair<P>(w, 2, 3, c);
            h[c] = {p_addss<-S, S>(u.re, l.im), p_addss<S, -S>(u.im, l.re)};
        } else {                        // h0 = p0 + S p2, h1 = p1 + S p3
            const c2 l = spin_pair<P>(w, 2, 3, c);
            h[c] = {p_adds<S>(u.re, l.re), p_adds<S>(u.im, l.im)};
        }
    }
}

// (w0, w1)[r] = (U h0, U h1)[r] (FWD) or with U^dagger; U in both lanes.
template <bool FWD>
__device__ __forceinline__ void sp_su3(const cpx<float> (&U)[3][3], const c2 (&h)[3], c2 (&w)[3])
{
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        f2 re, im;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cpx<float> u = FWD ? U[r][c] : U[c][r];
            const f2 ur = p_bcast(u.re), ui = p_bcast(FWD ? u.im : -u.im);   // conj for U^dagger
            if (c == 0) {
                re = p_mul(ur, h[0].re);
                im = p_mul(ur, h[0].im);
            } else {
                re = p_fma(ur, h[c].re, re);
                im = p_fma(ur, h[c].im, im);
            }
            re = p_fma(p_neg(ui), h[c].im, re);
            im = p_fma(ui, h[c].re, im);
        }
        w[r] = {re, im};
    }
}

// Accumulators of the spin-paired kernel.
struct SpAcc {
    c2 up[3];   // (acc_0, acc_1)
    c2 l32[3];  // (acc_3, acc_2), from the x and y directions
    c2 l23[3];  // (acc_2, acc_3), from the z and t directions
};

// acc += (1 + S gamma_MU) applied in the projected form, w = (U h0, U h1).
template <int MU, int S>
__device__ __forceinline__ void sp_accumulate(SpAcc &a, const c2 (&w)[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a.up[c].re = p_add(a.up[c].re, w[c].re);
        a.up[c].im = p_add(a.up[c].im, w[c].im);
        if constexpr (MU == 0) {        // spin3 += -S i w0, spin2 += -S i w1
            a.l32[c].re = p_adds<S>(a.l32[c].re, w[c].im);
            a.l32[c].im = p_adds<-S>(a.l32[c].im, w[c].re);
        } else if constexpr (MU == 1) { // spin3 += -S w0, spin2 += S w1
            a.l32[c].re = p_addss<-S, S>(a.l32[c].re, w[c].re);
            a.l32[c].im = p_addss<-S, S>(a.l32[c].im, w[c].im);
        } else if constexpr (MU == 2) { // spin2 += -S i w0, spin3 += S i w1
            a.l23[c].re = p_addss<S, -S>(a.l23[c].re, w[c].im);
            a.l23[c].im = p_addss<-S, S>(a.l23[c].im, w[c].re);
        } else {                        // spin2 += S w0, spin3 += S w1
            a.l23[c].re = p_adds<S>(a.l23[c].re, w[c].re);
            a.l23[c].im = p_adds<S>(a.l23[c].im, w[c].im);
        }
    }
}

// One direction: neighbour nb, link of site li; neg: the hop crosses an
// antiperiodic boundary.  The neighbour's 16-bit scale multiplies U h.
template <int P, int RECON, int MU, int S, bool FWD, bool LNA>
__device__ __forceinline__ void sp_dir(const char *in, const char *lblk, int vh, int nb, int li, bool neg, SpAcc &acc)
{
    constexpr int NP = Spinor<P>::nplane;
    unsigned w[12];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const uint4 v = ldg16(in + ((size_t)k * vh + nb) * 16);
        w[4 * k] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
    }
    const float sc = __ldg(reinterpret_cast<const float *>(in + (size_t)NP * vh * 16) + nb);
    c2 h[3];
    sp_project<P, MU, S>(w, h);
    cpx<float> U[3][3];
    Link<link_prec(P), RECON>::template load<LNA>(lblk, vh, li, U);
    c2 r[3];
    sp_su3<FWD>(U, h, r);
    const f2 f = p_bcast(neg ? -sc : sc);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        r[c].re = p_mul(r[c].re, f);
        r[c].im = p_mul(r[c].im, f);
    }
    sp_accumulate<MU, S>(acc, r);
}

// One output site with the spin-paired arithmetic.  PF 1: memory schedule 1
// of hop_site (backward directions first, forward links and t-forward
// neighbour prefetched into L2); PF 0: schedule 0 (natural order, no
// prefetch).  LNA: links loaded without L1 allocation.
template <int P, int RECON, bool DAG, bool HAS_X, int PF, bool LNA>
__device__ __forceinline__ void sp_site(const HopArgs &A, const int p, const int i, const size_t roff)
{
    const int vh = A.vh;
    const char *in = (p ? A.in[1] : A.in[0]) + roff;
    const char *gf = p ? A.gauge[1] : A.gauge[0];
    const char *gb = p ? A.gauge[0] : A.gauge[1];
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
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    const size_t lb = A.link_blk;

    SpAcc acc;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc.up[c] = acc.l32[c] = acc.l23[c] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    }
    if constexpr (PF == 0) {
        sp_dir<P, RECON, 0, SF, true, LNA>(in, gf + 0 * lb, vh, xf, i, false, acc);
        sp_dir<P, RECON, 0, SB, false, LNA>(in, gb + 0 * lb, vh, xb, xb, false, acc);
        sp_dir<P, RECON, 1, SF, true, LNA>(in, gf + 1 * lb, vh, yf, i, false, acc);
        sp_dir<P, RECON, 1, SB, false, LNA>(in, gb + 1 * lb, vh, yb, yb, false, acc);
        sp_dir<P, RECON, 2, SF, true, LNA>(in, gf + 2 * lb, vh, zf, i, false, acc);
        sp_dir<P, RECON, 2, SB, false, LNA>(in, gb + 2 * lb, vh, zb, zb, false, acc);
        sp_dir<P, RECON, 3, SF, true, LNA>(in, gf + 3 * lb, vh, tf, i, ntf, acc);
        sp_dir<P, RECON, 3, SB, false, LNA>(in, gb + 3 * lb, vh, tb, tb, ntb, acc);
    } else {
        using LK = Link<link_prec(P), RECON>;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) LK::prefetch(gf + mu * lb, vh, i);
        Spinor<P>::prefetch(in, vh, tf);
        sp_dir<P, RECON, 0, SB, false, LNA>(in, gb + 0 * lb, vh, xb, xb, false, acc);
        sp_dir<P, RECON, 1, SB, false, LNA>(in, gb + 1 * lb, vh, yb, yb, false, acc);
        sp_dir<P, RECON, 2, SB, false, LNA>(in, gb + 2 * lb, vh, zb, zb, false, acc);
        sp_dir<P, RECON, 3, SB, false, LNA>(in, gb + 3 * lb, vh, tb, tb, ntb, acc);
        sp_dir<P, RECON, 0, SF, true, LNA>(in, gf + 0 * lb, vh, xf, i, false, acc);
        sp_dir<P, RECON, 1, SF, true, LNA>(in, gf + 1 * lb, vh, yf, i, false, acc);
        sp_dir<P, RECON, 2, SF, true, LNA>(in, gf + 2 * lb, vh, zf, i, false, acc);
        sp_dir<P, RECON, 3, SF, true, LNA>(in, gf + 3 * lb, vh, tf, i, ntf, acc);
    }

    // the four spins: 0, 1 from the upper pair, 2 and 3 from both lower pairs
    const float a = (float)A.a, b = (float)A.b;
    float o[24];
    if constexpr (HAS_X) Spinor<P>::load((p ? A.x[1] : A.x[0]) + roff, vh, i, o);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float sre[4] = {acc.up[c].re.x, acc.up[c].re.y, acc.l23[c].re.x + acc.l32[c].re.y,
                              acc.l23[c].re.y + acc.l32[c].re.x};
        const float sim[4] = {acc.up[c].im.x, acc.up[c].im.y, acc.l23[c].im.x + acc.l32[c].im.y,
                              acc.l23[c].im.y + acc.l32[c].im.x};
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
            if constexpr (HAS_X) {
                o[6 * sp + 2 * c] = fmaf(b, sre[sp], a * o[6 * sp + 2 * c]);
                o[6 * sp + 2 * c + 1] = fmaf(b, sim[sp], a * o[6 * sp + 2 * c + 1]);
            } else {
                o[6 * sp + 2 * c] = b * sre[sp];
                o[6 * sp + 2 * c + 1] = b * sim[sp];
            }
        }
    }
    Spinor<P>::store((p ? A.out[1] : A.out[0]) + roff, vh, i, o);
}

template <int P, int RECON, bool DAG, bool HAS_X, int PF, bool LNA>
__global__ void __launch_bounds__(256, 2) hop_sp_kernel(const HopArgs A)
{
    int p, blk;
    if (A.nparity == 2) { p = blockIdx.x & 1; blk = blockIdx.x >> 1; }
    else { p = A.parity0; blk = blockIdx.x; }
    const int i = blk * blockDim.x + threadIdx.x;
    if (i >= A.vh) return;
    sp_site<P, RECON, DAG, HAS_X, PF, LNA>(A, p, i, (size_t)blockIdx.y * A.rhs_stride);
}

// pf 1: schedule 1 with L1-allocating link loads; pf 0: schedule 0 with
// links loaded without L1 allocation (the even-odd hops' choice).
template <int P, int RECON, bool DAG, bool HX>
cudaError_t launch_hop_sp(const HopArgs &A, dim3 grid, int threads, int pf, cudaStream_t s)
{
    if (pf == 1) return wd_launch(hop_sp_kernel<P, RECON, DAG, HX, 1, false>, grid, dim3(threads), 0, s, A);
    return wd_launch(hop_sp_kernel<P, RECON, DAG, HX, 0, true>, grid, dim3(threads), 0, s, A);
}

} // namespace wd
