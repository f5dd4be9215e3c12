// Paired FP32 arithmetic for the 16-bit storage formats.
//
// Blackwell executes add, mul and fma on a pair of FP32 values held in two
// adjacent registers as one instruction (the f32x2 forms): half the issue
// slots of two scalar instructions, the same FMA-pipe time.  The 16-bit hop
// kernels issue about 1650 instructions per site with the issue slots about
// 70 % busy, so fewer instructions at unchanged occupancy make them faster.
// One thread still computes one site; the pairs are the two spin components
// that the projected form carries through each direction:
//   (h0, h1)          the projected half spinor, each lane one sum of two
//                     stored values with one of them taken as stored
//                     (project_words);
//   (U h0, U h1)      the SU(3) product, with each link entry converted once
//                     and copied into both lanes;
//   (acc_0, acc_1), (acc_3, acc_2), (acc_2, acc_3)
//                     accumulators: directions x, y add into the first lower
//                     pair, z, t into the second (the projector pairs the
//                     spins crosswise there), summed once at the end; each
//                     term weighted in a paired FMA by the neighbour's scale
//                     times the hop coefficient.
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

// (h0, h1) paired from project_words: each sum takes one operand as stored
// (sm_100's FP32 addition with a 16-bit operand), written into its lane.
template <int P, int MU, int S>
__device__ __forceinline__ void sp_project_words(const unsigned (&w)[12], c2 (&h)[3])
{
    cpx<float> h0[3], h1[3];
    project_words<P, MU, S>(w, h0, h1);
#pragma unroll
    for (int c = 0; c < 3; ++c) h[c] = {make_float2(h0[c].re, h1[c].re), make_float2(h0[c].im, h1[c].im)};
}

// Accumulators of the spin-paired kernel.
struct SpAcc {
    c2 up[3];   // (acc_0, acc_1)
    c2 l32[3];  // (acc_3, acc_2), from the x and y directions
    c2 l23[3];  // (acc_2, acc_3), from the z and t directions
};

// acc += f (1 + S gamma_MU) applied in the projected form, w = (U h0, U h1):
// the weight f (the neighbour's scale times the hop coefficient) rides on the
// paired FMAs, lane signs in the weight pair.
template <int SX, int SY> __device__ __forceinline__ f2 p_w(float f) { return make_float2(SX * f, SY * f); }

template <int MU, int S>
__device__ __forceinline__ void sp_accumulate(SpAcc &a, const c2 (&w)[3], const float f)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a.up[c].re = p_fma(p_w<1, 1>(f), w[c].re, a.up[c].re);
        a.up[c].im = p_fma(p_w<1, 1>(f), w[c].im, a.up[c].im);
        if constexpr (MU == 0) {        // spin3 += -S i w0, spin2 += -S i w1
            a.l32[c].re = p_fma(p_w<S, S>(f), w[c].im, a.l32[c].re);
            a.l32[c].im = p_fma(p_w<-S, -S>(f), w[c].re, a.l32[c].im);
        } else if constexpr (MU == 1) { // spin3 += -S w0, spin2 += S w1
            a.l32[c].re = p_fma(p_w<-S, S>(f), w[c].re, a.l32[c].re);
            a.l32[c].im = p_fma(p_w<-S, S>(f), w[c].im, a.l32[c].im);
        } else if constexpr (MU == 2) { // spin2 += -S i w0, spin3 += S i w1
            a.l23[c].re = p_fma(p_w<S, -S>(f), w[c].im, a.l23[c].re);
            a.l23[c].im = p_fma(p_w<-S, S>(f), w[c].re, a.l23[c].im);
        } else {                        // spin2 += S w0, spin3 += S w1
            a.l23[c].re = p_fma(p_w<S, S>(f), w[c].re, a.l23[c].re);
            a.l23[c].im = p_fma(p_w<S, S>(f), w[c].im, a.l23[c].im);
        }
    }
}

// One direction: neighbour nb, link of site li; neg: the hop crosses an
// antiperiodic boundary.  The neighbour's 16-bit scale times wt (the hop
// coefficient) weights the accumulated terms.
template <int P, int RECON, int MU, int S, bool FWD, bool LNA>
__device__ __forceinline__ void sp_dir(const char *in, const char *lblk, int vh, int nb, int li, bool neg, SpAcc &acc,
                                       const float wt)
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
    sp_project_words<P, MU, S>(w, h);
    cpx<float> U[3][3];
    Link<link_prec(P), RECON>::template load<LNA>(lblk, vh, li, U);
    c2 r[3];
    sp_su3<FWD>(U, h, r);
    sp_accumulate<MU, S>(acc, r, (neg ? -sc : sc) * wt);
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

    const float wt = (float)A.b;   // the hop coefficient weights the accumulated terms
    SpAcc acc;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc.up[c] = acc.l32[c] = acc.l23[c] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    }
    if constexpr (PF == 0) {
        sp_dir<P, RECON, 0, SF, true, LNA>(in, gf + 0 * lb, vh, xf, i, false, acc, wt);
        sp_dir<P, RECON, 0, SB, false, LNA>(in, gb + 0 * lb, vh, xb, xb, false, acc, wt);
        sp_dir<P, RECON, 1, SF, true, LNA>(in, gf + 1 * lb, vh, yf, i, false, acc, wt);
        sp_dir<P, RECON, 1, SB, false, LNA>(in, gb + 1 * lb, vh, yb, yb, false, acc, wt);
        sp_dir<P, RECON, 2, SF, true, LNA>(in, gf + 2 * lb, vh, zf, i, false, acc, wt);
        sp_dir<P, RECON, 2, SB, false, LNA>(in, gb + 2 * lb, vh, zb, zb, false, acc, wt);
        sp_dir<P, RECON, 3, SF, true, LNA>(in, gf + 3 * lb, vh, tf, i, ntf, acc, wt);
        sp_dir<P, RECON, 3, SB, false, LNA>(in, gb + 3 * lb, vh, tb, tb, ntb, acc, wt);
    } else {
        using LK = Link<link_prec(P), RECON>;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) LK::prefetch(gf + mu * lb, vh, i);
        Spinor<P>::prefetch(in, vh, tf);
        sp_dir<P, RECON, 0, SB, false, LNA>(in, gb + 0 * lb, vh, xb, xb, false, acc, wt);
        sp_dir<P, RECON, 1, SB, false, LNA>(in, gb + 1 * lb, vh, yb, yb, false, acc, wt);
        sp_dir<P, RECON, 2, SB, false, LNA>(in, gb + 2 * lb, vh, zb, zb, false, acc, wt);
        sp_dir<P, RECON, 3, SB, false, LNA>(in, gb + 3 * lb, vh, tb, tb, ntb, acc, wt);
        sp_dir<P, RECON, 0, SF, true, LNA>(in, gf + 0 * lb, vh, xf, i, false, acc, wt);
        sp_dir<P, RECON, 1, SF, true, LNA>(in, gf + 1 * lb, vh, yf, i, false, acc, wt);
        sp_dir<P, RECON, 2, SF, true, LNA>(in, gf + 2 * lb, vh, zf, i, false, acc, wt);
        sp_dir<P, RECON, 3, SF, true, LNA>(in, gf + 3 * lb, vh, tf, i, ntf, acc, wt);
    }

    // the four spins: 0, 1 from the upper pair, 2 and 3 from both lower pairs
    cpx<float> v[4][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[0][c] = {acc.up[c].re.x, acc.up[c].im.x};
        v[1][c] = {acc.up[c].re.y, acc.up[c].im.y};
        v[2][c] = {acc.l23[c].re.x + acc.l32[c].re.y, acc.l23[c].im.x + acc.l32[c].im.y};
        v[3][c] = {acc.l23[c].re.y + acc.l32[c].re.x, acc.l23[c].im.y + acc.l32[c].im.x};
    }
    store_weighted<P, HAS_X>(HAS_X ? (p ? A.x[1] : A.x[0]) + roff : nullptr, (p ? A.out[1] : A.out[0]) + roff, vh, i,
                             (float)A.a, v);
}

template <int P, int RECON, bool DAG, bool HAS_X, int PF, bool LNA>
__global__ void __launch_bounds__(256, 2) hop_sp_kernel(const HopArgs A)
{
    grid_dependency_enter();
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
