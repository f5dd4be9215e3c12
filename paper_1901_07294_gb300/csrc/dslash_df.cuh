// Double-word FP32 hop with three threads per site.
//
// The per-site kernel in double-word arithmetic needs about 250 registers a
// thread (a value is two FP32 registers, and its error terms add more), so only
// 8 warps fit on an SM, too few to hide the dependent chains of the error-free
// transformations.  Here warp r of a 96-thread block computes colour row r of
// the output for 32 consecutive checkerboard sites.  For each direction warp r
// loads the neighbours' colour-r spin components and projects them, the block
// exchanges the projected half spinors through shared memory, and each thread
// multiplies them by row r of U (column r for U^dagger) and accumulates the four
// spin components of colour r.  That is about a third of the per-site state,
// so more warps fit.  With 12-real links each warp also rebuilds one entry of
// the link's third row and shares it through the same tile.
#pragma once

#include "dslash_impl.cuh"
#include "dslash_mrhs.cuh"

namespace wd {

constexpr int DF_ROW_THREADS = 96;
constexpr int DF_ROW_BLOCKS = 8;   // resident blocks per SM the register budget is set for (80 registers)

// (h0, h1) = upper two spin components of (1 + S gamma_MU) psi for one colour,
// from its four spin components p[s] (the table of project).
template <int MU, int S>
__device__ __forceinline__ void project_colour(const cpx<df> (&p)[4], cpx<df> &h0, cpx<df> &h1)
{
    if constexpr (MU == 0) {        // h0 = p0 + S i p3, h1 = p1 + S i p2
        h0 = {p[0].re - S * p[3].im, p[0].im + S * p[3].re};
        h1 = {p[1].re - S * p[2].im, p[1].im + S * p[2].re};
    } else if constexpr (MU == 1) { // h0 = p0 - S p3, h1 = p1 + S p2
        h0 = {p[0].re - S * p[3].re, p[0].im - S * p[3].im};
        h1 = {p[1].re + S * p[2].re, p[1].im + S * p[2].im};
    } else if constexpr (MU == 2) { // h0 = p0 + S i p2, h1 = p1 - S i p3
        h0 = {p[0].re - S * p[2].im, p[0].im + S * p[2].re};
        h1 = {p[1].re + S * p[3].im, p[1].im - S * p[3].re};
    } else {                        // h0 = p0 + S p2, h1 = p1 + S p3
        h0 = {p[0].re + S * p[2].re, p[0].im + S * p[2].im};
        h1 = {p[1].re + S * p[3].re, p[1].im + S * p[3].im};
    }
}

// a += s x (s = +1 or -1) without renormalising: the running sum of a
// compensated dot product, normalised once before it is used as a product
// operand (a lo part that grew past hi would lose accuracy there).
template <int SG> __device__ __forceinline__ void lazy_acc(df &a, df x)
{
    const float xh = SG > 0 ? x.hi : -x.hi, xl = SG > 0 ? x.lo : -x.lo;
    const df t = df_two_sum(a.hi, xh);
    a = {t.hi, __fadd_rn(t.lo, __fadd_rn(a.lo, xl))};
}

// accumulate for colour row r only, with lazy sums (FIRST assigns)
template <int MU, int S, bool FIRST>
__device__ __forceinline__ void df_accumulate(cpx<df> (&acc)[4], const cpx<df> &w0, const cpx<df> &w1)
{
    // spins 2, 3 = (a + i b) style multiples of w0, w1 fixed by the projector:
    // each entry is (source, component taken, sign) for re and im
    if constexpr (FIRST) {
        acc[0] = w0;
        acc[1] = w1;
        if constexpr (MU == 0) {        // spin2 = -S i w1, spin3 = -S i w0
            acc[2] = {S * w1.im, -S * w1.re};
            acc[3] = {S * w0.im, -S * w0.re};
        } else if constexpr (MU == 1) { // spin2 = S w1, spin3 = -S w0
            acc[2] = {S * w1.re, S * w1.im};
            acc[3] = {-S * w0.re, -S * w0.im};
        } else if constexpr (MU == 2) { // spin2 = -S i w0, spin3 = S i w1
            acc[2] = {S * w0.im, -S * w0.re};
            acc[3] = {-S * w1.im, S * w1.re};
        } else {                        // spin2 = S w0, spin3 = S w1
            acc[2] = {S * w0.re, S * w0.im};
            acc[3] = {S * w1.re, S * w1.im};
        }
        return;
    }
    lazy_acc<1>(acc[0].re, w0.re); lazy_acc<1>(acc[0].im, w0.im);
    lazy_acc<1>(acc[1].re, w1.re); lazy_acc<1>(acc[1].im, w1.im);
    if constexpr (MU == 0) {
        lazy_acc<S>(acc[2].re, w1.im); lazy_acc<-S>(acc[2].im, w1.re);
        lazy_acc<S>(acc[3].re, w0.im); lazy_acc<-S>(acc[3].im, w0.re);
    } else if constexpr (MU == 1) {
        lazy_acc<S>(acc[2].re, w1.re); lazy_acc<S>(acc[2].im, w1.im);
        lazy_acc<-S>(acc[3].re, w0.re); lazy_acc<-S>(acc[3].im, w0.im);
    } else if constexpr (MU == 2) {
        lazy_acc<S>(acc[2].re, w0.im); lazy_acc<-S>(acc[2].im, w0.re);
        lazy_acc<-S>(acc[3].re, w1.im); lazy_acc<S>(acc[3].im, w1.re);
    } else {
        lazy_acc<S>(acc[2].re, w0.re); lazy_acc<S>(acc[2].im, w0.im);
        lazy_acc<S>(acc[3].re, w1.re); lazy_acc<S>(acc[3].im, w1.im);
    }
}

// The projected half spinors of the block's 32 sites for one direction:
// warp c writes colour c, every warp then reads all three.  [colour][h0 re,
// h0 im, h1 re, h1 im as (hi, lo) pairs: two float4][site].  With 12-real
// links, rec[c] holds entry (2, c) of the direction's link, rebuilt by warp c.
template <int RECON> struct DfHalfTile {
    float4 v[3][2][32];
    float4 rec[RECON == 12 ? 3 : 1][32];
};

// Entry (2, C) of a 12-real link from its stored rows 0 and 1:
// conj(U0a U1b - U0b U1a) with a = C+1, b = C+2 (mod 3), one four-term
// compensated chain per part as in Link::load, normalised for use as a
// product operand.
template <int C>
__device__ __forceinline__ cpx<df> df_row3_entry(const cpx<df> (&e0)[3], const cpx<df> (&e1)[3])
{
    constexpr int a = (C + 1) % 3, b = (C + 2) % 3;
    const cpx<df> x = e0[a], y = e1[b], z = e0[b], w = e1[a];
    df re = x.re * y.re;
    re = fma(-x.im, y.im, re);
    re = fma(-z.re, w.re, re);
    re = fma(z.im, w.im, re);
    df im = -(x.re * y.im);
    im = fma(-x.im, y.re, im);
    im = fma(z.re, w.im, im);
    im = fma(z.im, w.re, im);
    return {df_normalize(re), df_normalize(im)};
}

// One direction for colour row r: acc[s] += the (s, r) component of
// (1 + S gamma_MU) U psi (FWD) or (1 + S gamma_MU) U^dagger psi.  Warp r loads
// the neighbour's colour-r spin components only and projects them; the block
// exchanges the projections through `tile` (one barrier; the tile of a
// direction is rewritten two directions later, after the next barrier).
// With 12-real links every warp loads the two stored rows and rebuilds entry
// (2, r); a forward hop's row 2 is then the three warps' entries, read from
// the tile after the same barrier.
template <int MU, int S, bool FWD, int RECON, bool FIRST = false>
__device__ __forceinline__ void df_row_dir(const char *in, const char *lblk, int vh, int nb, int li, bool neg, int r,
                                           int lane, DfHalfTile<RECON> &tile, cpx<df> (&acc)[4])
{
    cpx<df> p[4];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {   // plane 3 sp + r holds (spin sp, colour r)
        df v[2];
        unpack16<PREC_DF>(ldg16(in + ((size_t)(3 * sp + r) * vh + nb) * 16), v, 1.0f);
        p[sp] = {v[0], v[1]};
    }
    cpx<df> u[3];   // U[r][c] (FWD) or U[c][r]
    auto entry = [&](int k) {   // plane k = 3 row + column holds one complex number
        df v[2];
        unpack16<PREC_DF>(ldg16(lblk + ((size_t)k * vh + li) * 16), v, 1.0f);
        return cpx<df>{v[0], v[1]};
    };
    if constexpr (RECON == 18) {
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = entry(FWD ? 3 * r + c : 3 * c + r);
    } else {
        cpx<df> e0[3], e1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            e0[c] = entry(c);
            e1[c] = entry(3 + c);
        }
        const cpx<df> rec = r == 0 ? df_row3_entry<0>(e0, e1) : r == 1 ? df_row3_entry<1>(e0, e1)
                                                                       : df_row3_entry<2>(e0, e1);
        tile.rec[r][lane] = make_float4(rec.re.hi, rec.re.lo, rec.im.hi, rec.im.lo);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if constexpr (FWD) u[c] = r == 0 ? e0[c] : e1[c];   // row 2: from the tile below
            else u[c] = c == 2 ? rec : (r == 0 ? (c == 0 ? e0[0] : e1[0]) : r == 1 ? (c == 0 ? e0[1] : e1[1])
                                                                             : (c == 0 ? e0[2] : e1[2]));
        }
    }
    cpx<df> g0, g1;
    project_colour<MU, S>(p, g0, g1);
    tile.v[r][0][lane] = make_float4(g0.re.hi, g0.re.lo, g0.im.hi, g0.im.lo);
    tile.v[r][1][lane] = make_float4(g1.re.hi, g1.re.lo, g1.im.hi, g1.im.lo);
    __syncthreads();
    if constexpr (RECON == 12 && FWD) {
        if (r == 2)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float4 q = tile.rec[c][lane];
                u[c] = {df(q.x, q.y), df(q.z, q.w)};
            }
    }
    cpx<df> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float4 a = tile.v[c][0][lane], b = tile.v[c][1][lane];
        h0[c] = {df(a.x, a.y), df(a.z, a.w)};
        h1[c] = {df(b.x, b.y), df(b.z, b.w)};
    }
    cpx<df> w0, w1;
    if constexpr (FWD) {
        w0 = cfma(u[2], h0[2], cfma(u[1], h0[1], cmul(u[0], h0[0])));
        w1 = cfma(u[2], h1[2], cfma(u[1], h1[1], cmul(u[0], h1[0])));
    } else {
        w0 = cfma_conj(u[2], h0[2], cfma_conj(u[1], h0[1], cmul_conj(u[0], h0[0])));
        w1 = cfma_conj(u[2], h1[2], cfma_conj(u[1], h1[1], cmul_conj(u[0], h1[0])));
    }
    if (neg) {
        w0 = {-w0.re, -w0.im};
        w1 = {-w1.re, -w1.im};
    }
    df_accumulate<MU, S, FIRST>(acc, w0, w1);
}

// 18- or 12-real links; blocks alternate parity for the full operator as in
// hop_kernel; out = a x + b acc.  Every thread of a block takes part in the
// barriers: threads past the last site compute the last site and store nothing.
template <int RECON, bool DAG, bool HAS_X>
__global__ void __launch_bounds__(DF_ROW_THREADS, DF_ROW_BLOCKS) hop_df_row_kernel(const HopArgs A)
{
    grid_dependency_enter();
    __shared__ DfHalfTile<RECON> tile[2];
    int p, blk;
    if (A.nparity == 2) { p = blockIdx.x & 1; blk = blockIdx.x >> 1; }
    else { p = A.parity0; blk = blockIdx.x; }
    const int r = threadIdx.x >> 5;   // warp-uniform
    const int lane = threadIdx.x & 31;
    const int vh = A.vh;
    const int i0 = blk * 32 + lane;
    const bool active = i0 < vh;
    const int i = active ? i0 : vh - 1;
    const size_t roff = (size_t)blockIdx.y * A.rhs_stride, lb = A.link_blk;
    const char *in = (p ? A.in[1] : A.in[0]) + roff;
    const char *gf = p ? A.gauge[1] : A.gauge[0];
    const char *gb = p ? A.gauge[0] : A.gauge[1];
    int nb[8];
    site_neighbours(A, p, i, nb);
    // a t hop wraps exactly when the neighbour's index falls below (forward) or above (backward) i
    const bool ntf = A.tneg && nb[3] < i, ntb = A.tneg && nb[7] > i;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    cpx<df> acc[4];
    df_row_dir<0, SB, false, RECON, true>(in, gb + 0 * lb, vh, nb[4], nb[4], false, r, lane, tile[0], acc);
    df_row_dir<1, SB, false, RECON>(in, gb + 1 * lb, vh, nb[5], nb[5], false, r, lane, tile[1], acc);
    df_row_dir<2, SB, false, RECON>(in, gb + 2 * lb, vh, nb[6], nb[6], false, r, lane, tile[0], acc);
    df_row_dir<3, SB, false, RECON>(in, gb + 3 * lb, vh, nb[7], nb[7], ntb, r, lane, tile[1], acc);
    df_row_dir<0, SF, true, RECON>(in, gf + 0 * lb, vh, nb[0], i, false, r, lane, tile[0], acc);
    df_row_dir<1, SF, true, RECON>(in, gf + 1 * lb, vh, nb[1], i, false, r, lane, tile[1], acc);
    df_row_dir<2, SF, true, RECON>(in, gf + 2 * lb, vh, nb[2], i, false, r, lane, tile[0], acc);
    df_row_dir<3, SF, true, RECON>(in, gf + 3 * lb, vh, nb[3], i, ntf, r, lane, tile[1], acc);
    if (!active) return;

    const df a = (df)A.a, b = (df)A.b;
    char *out = (p ? A.out[1] : A.out[0]) + roff;
    const char *x = HAS_X ? (p ? A.x[1] : A.x[0]) + roff : nullptr;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const size_t off = ((size_t)(3 * s + r) * vh + i) * 16;   // plane of (spin s, colour r)
        const cpx<df> v = {df_normalize(acc[s].re), df_normalize(acc[s].im)};
        df o[2];
        if constexpr (HAS_X) {
            df xv[2];
            unpack16<PREC_DF>(ldg16(x + off), xv, 1.0f);
            o[0] = a * xv[0] + b * v.re;
            o[1] = a * xv[1] + b * v.im;
        } else if (A.b == 1.0) {
            o[0] = v.re;
            o[1] = v.im;
        } else {
            o[0] = b * v.re;
            o[1] = b * v.im;
        }
        stg16(out + off, pack16<PREC_DF>(o, 1.0f));
    }
}

template <int RECON, bool DAG, bool HX>
cudaError_t launch_hop_df_row(const HopArgs &A, int nrhs, cudaStream_t s)
{
    const int per = (A.vh + 31) / 32;
    return wd_launch(hop_df_row_kernel<RECON, DAG, HX>, dim3((unsigned)(per * A.nparity), (unsigned)nrhs),
                     dim3(DF_ROW_THREADS), 0, s, A);
}

} // namespace wd
