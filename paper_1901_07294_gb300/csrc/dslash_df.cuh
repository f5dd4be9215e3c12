// Double-word FP32 hop with three threads per site.
//
// The per-site kernel in double-word arithmetic needs about 250 registers a
// thread (a value is two FP32 registers, and its error terms add more), so only
// 8 warps fit on an SM, too few to hide the dependent chains of the error-free
// transformations.  Here warp r of a 96-thread block computes colour row r of
// the output for 32 consecutive checkerboard sites: each thread projects the
// whole neighbour spinor (the three warps read the same lines, the second and
// third from L1), multiplies by row r of U (column r of U for U^dagger), and
// accumulates the four spin components of colour r.  That is about a third of
// the per-site state, so more warps fit, for a threefold projection.
#pragma once

#include "dslash_impl.cuh"
#include "dslash_mrhs.cuh"

namespace wd {

constexpr int DF_ROW_THREADS = 96;
constexpr int DF_ROW_BLOCKS = 6;   // resident blocks per SM the register budget is set for

// One direction for colour row r: acc[s] += the (s, r) component of
// (1 + S gamma_MU) U psi (FWD) or (1 + S gamma_MU) U^dagger psi.
template <int MU, int S, bool FWD, bool FIRST = false>
__device__ __forceinline__ void df_row_dir(const char *in, const char *lblk, int vh, int nb, int li, bool neg, int r,
                                           cpx<df> (&acc)[4][1])
{
    df psi[24];
    Spinor<PREC_DF>::load(in, vh, nb, psi);
    cpx<df> h0[3], h1[3];
    project<MU, S>(psi, h0, h1);
    cpx<df> u[3];   // U[r][c] (FWD) or U[c][r]
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int k = FWD ? 3 * r + c : 3 * c + r;   // plane of the entry (one complex number per plane)
        df v[2];
        unpack16<PREC_DF>(ldg16(lblk + ((size_t)k * vh + li) * 16), v, 1.0f);
        u[c] = {v[0], v[1]};
    }
    cpx<df> w0[1], w1[1];
    if constexpr (FWD) {
        w0[0] = cfma(u[2], h0[2], cfma(u[1], h0[1], cmul(u[0], h0[0])));
        w1[0] = cfma(u[2], h1[2], cfma(u[1], h1[1], cmul(u[0], h1[0])));
    } else {
        w0[0] = cfma_conj(u[2], h0[2], cfma_conj(u[1], h0[1], cmul_conj(u[0], h0[0])));
        w1[0] = cfma_conj(u[2], h1[2], cfma_conj(u[1], h1[1], cmul_conj(u[0], h1[0])));
    }
    if (neg) {
        w0[0] = {-w0[0].re, -w0[0].im};
        w1[0] = {-w1[0].re, -w1[0].im};
    }
    accumulate<MU, S, FIRST>(acc, w0, w1);
}

// 18-real links; blocks alternate parity for the full operator as in
// hop_kernel; out = a x + b acc.
template <bool DAG, bool HAS_X>
__global__ void __launch_bounds__(DF_ROW_THREADS, DF_ROW_BLOCKS) hop_df_row_kernel(const HopArgs A)
{
    int p, blk;
    if (A.nparity == 2) { p = blockIdx.x & 1; blk = blockIdx.x >> 1; }
    else { p = A.parity0; blk = blockIdx.x; }
    const int r = threadIdx.x >> 5;   // warp-uniform
    const int i = blk * 32 + (threadIdx.x & 31);
    if (i >= A.vh) return;
    const int vh = A.vh;
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
    cpx<df> acc[4][1];
    df_row_dir<0, SB, false, true>(in, gb + 0 * lb, vh, nb[4], nb[4], false, r, acc);
    df_row_dir<1, SB, false>(in, gb + 1 * lb, vh, nb[5], nb[5], false, r, acc);
    df_row_dir<2, SB, false>(in, gb + 2 * lb, vh, nb[6], nb[6], false, r, acc);
    df_row_dir<3, SB, false>(in, gb + 3 * lb, vh, nb[7], nb[7], ntb, r, acc);
    df_row_dir<0, SF, true>(in, gf + 0 * lb, vh, nb[0], i, false, r, acc);
    df_row_dir<1, SF, true>(in, gf + 1 * lb, vh, nb[1], i, false, r, acc);
    df_row_dir<2, SF, true>(in, gf + 2 * lb, vh, nb[2], i, false, r, acc);
    df_row_dir<3, SF, true>(in, gf + 3 * lb, vh, nb[3], i, ntf, r, acc);

    const df a = (df)A.a, b = (df)A.b;
    char *out = (p ? A.out[1] : A.out[0]) + roff;
    const char *x = HAS_X ? (p ? A.x[1] : A.x[0]) + roff : nullptr;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const size_t off = ((size_t)(3 * s + r) * vh + i) * 16;   // plane of (spin s, colour r)
        df o[2];
        if constexpr (HAS_X) {
            df xv[2];
            unpack16<PREC_DF>(ldg16(x + off), xv, 1.0f);
            o[0] = a * xv[0] + b * acc[s][0].re;
            o[1] = a * xv[1] + b * acc[s][0].im;
        } else if (A.b == 1.0) {
            o[0] = acc[s][0].re;
            o[1] = acc[s][0].im;
        } else {
            o[0] = b * acc[s][0].re;
            o[1] = b * acc[s][0].im;
        }
        stg16(out + off, pack16<PREC_DF>(o, 1.0f));
    }
}

template <bool DAG, bool HX>
cudaError_t launch_hop_df_row(const HopArgs &A, int nrhs, cudaStream_t s)
{
    const int per = (A.vh + 31) / 32;
    return wd_launch(hop_df_row_kernel<DAG, HX>, dim3((unsigned)(per * A.nparity), (unsigned)nrhs),
                     dim3(DF_ROW_THREADS), 0, s, A);
}

} // namespace wd
