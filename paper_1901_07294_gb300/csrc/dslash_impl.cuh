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
    double a, b;
};

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
template <int MU, int S, typename T>
__device__ __forceinline__ void accumulate(cpx<T> (&acc)[4][3], const cpx<T> (&w0)[3], const cpx<T> (&w1)[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
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

// One direction.  For 16-bit storage the neighbour's per-site scale is applied
// to the 12 reals of U h (the operation is linear) rather than to its 24
// stored reals.
template <int P, int RECON, int MU, int S, bool FWD>
__device__ __forceinline__ void hop_dir(const char *in, const char *lblk, int vh, int nb, int li,
                                        cpx<typename Prec<P>::real> (&acc)[4][3])
{
    using T = typename Prec<P>::real;
    T psi[24];
    const float sc = Spinor<P>::load_unscaled(in, vh, nb, psi);
    cpx<T> h0[3], h1[3];
    project<MU, S>(psi, h0, h1);
    cpx<T> U[3][3];
    Link<link_prec(P), RECON>::load(lblk, vh, li, U);
    cpx<T> w0[3], w1[3];
    su3_mul<FWD>(U, h0, w0);
    su3_mul<FWD>(U, h1, w1);
    if constexpr (Prec<P>::scaled) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            w0[c].re *= sc; w0[c].im *= sc;
            w1[c].re *= sc; w1[c].im *= sc;
        }
    }
    accumulate<MU, S>(acc, w0, w1);
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
template <int P, int RECON, bool DAG, bool HAS_X, int PF>
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
    int r = i / lxh;
    const int xh = i - r * lxh;
    const int y = r % Ly;
    r /= Ly;
    const int z = r % Lz;
    const int t = r / Lz;
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

    constexpr int SF = DAG ? +1 : -1;   // forward projector 1 + SF gamma
    constexpr int SB = -SF;             // backward projector
    const size_t lb = A.link_blk;

    cpx<T> acc[4][3];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[s][c] = {T(0), T(0)};

    using LK = Link<link_prec(P), RECON>;
    if constexpr (PF == 0) {
        hop_dir<P, RECON, 0, SF, true>(in, gf + 0 * lb, vh, xf, i, acc);
        hop_dir<P, RECON, 0, SB, false>(in, gb + 0 * lb, vh, xb, xb, acc);
        hop_dir<P, RECON, 1, SF, true>(in, gf + 1 * lb, vh, yf, i, acc);
        hop_dir<P, RECON, 1, SB, false>(in, gb + 1 * lb, vh, yb, yb, acc);
        hop_dir<P, RECON, 2, SF, true>(in, gf + 2 * lb, vh, zf, i, acc);
        hop_dir<P, RECON, 2, SB, false>(in, gb + 2 * lb, vh, zb, zb, acc);
        hop_dir<P, RECON, 3, SF, true>(in, gf + 3 * lb, vh, tf, i, acc);
        hop_dir<P, RECON, 3, SB, false>(in, gb + 3 * lb, vh, tb, tb, acc);
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
        hop_dir<P, RECON, 0, SB, false>(in, gb + 0 * lb, vh, xb, xb, acc);
        hop_dir<P, RECON, 1, SB, false>(in, gb + 1 * lb, vh, yb, yb, acc);
        hop_dir<P, RECON, 2, SB, false>(in, gb + 2 * lb, vh, zb, zb, acc);
        hop_dir<P, RECON, 3, SB, false>(in, gb + 3 * lb, vh, tb, tb, acc);
        hop_dir<P, RECON, 0, SF, true>(in, gf + 0 * lb, vh, xf, i, acc);
        hop_dir<P, RECON, 1, SF, true>(in, gf + 1 * lb, vh, yf, i, acc);
        hop_dir<P, RECON, 2, SF, true>(in, gf + 2 * lb, vh, zf, i, acc);
        hop_dir<P, RECON, 3, SF, true>(in, gf + 3 * lb, vh, tf, i, acc);
    }

    const T a = (T)A.a, b = (T)A.b;
    T o[24];
    if constexpr (HAS_X) {
        Spinor<P>::load((p ? A.x[1] : A.x[0]) + roff, vh, i, o);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o[6 * s + 2 * c] = a * o[6 * s + 2 * c] + b * acc[s][c].re;
                o[6 * s + 2 * c + 1] = a * o[6 * s + 2 * c + 1] + b * acc[s][c].im;
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
// registers the compiler would otherwise use to hoist loads.
template <int P, int RECON, bool DAG, bool HAS_X, int PF>
__global__ void __launch_bounds__(256, PF == 4 ? 3 : 2) hop_kernel(const HopArgs A)
{
    int p, blk;
    if (A.nparity == 2) { p = blockIdx.x & 1; blk = blockIdx.x >> 1; }
    else { p = A.parity0; blk = blockIdx.x; }
    const int i = blk * blockDim.x + threadIdx.x;
    if (i >= A.vh) return;
    hop_site<P, RECON, DAG, HAS_X, PF>(A, p, i, (size_t)blockIdx.y * A.rhs_stride);
}

// Neighbour checkerboard indices of site i of parity p, order
// x+, y+, z+, t+, x-, y-, z-, t- (same arithmetic as in hop_kernel).
__device__ __forceinline__ void site_neighbours(const HopArgs &A, int p, int i, int (&nb)[8])
{
    const int Lx = A.L[0], Ly = A.L[1], Lz = A.L[2], Lt = A.L[3];
    const int lxh = Lx >> 1;
    int r = i / lxh;
    const int xh = i - r * lxh;
    const int y = r % Ly;
    r /= Ly;
    const int z = r % Lz;
    const int t = r / Lz;
    const int x = 2 * xh + ((p + y + z + t) & 1);
    const int sy = lxh, sz = lxh * Ly, st = sz * Lz;
    const int row = i - xh;
    nb[0] = row + ((x + 1 == Lx ? 0 : x + 1) >> 1);
    nb[4] = row + ((x == 0 ? Lx - 1 : x - 1) >> 1);
    nb[1] = (y == Ly - 1) ? i - (Ly - 1) * sy : i + sy;
    nb[5] = (y == 0) ? i + (Ly - 1) * sy : i - sy;
    nb[2] = (z == Lz - 1) ? i - (Lz - 1) * sz : i + sz;
    nb[6] = (z == 0) ? i + (Lz - 1) * sz : i - sz;
    nb[3] = (t == Lt - 1) ? i - (Lt - 1) * st : i + st;
    nb[7] = (t == 0) ? i + (Lt - 1) * st : i - st;
}

// A link of the multi-RHS shared tile: its 18 reals (row-major, re/im
// interleaved) in NV 16-byte vectors, vector k of site s at [k][s] so that a
// warp reads 32 consecutive vectors (FP32: 5 float4, the last two reals
// padding; FP64: 9 double2).
template <typename T> struct LinkTile;
template <> struct LinkTile<float> { using V = float4; static constexpr int NV = 5; };
template <> struct LinkTile<double> { using V = double2; static constexpr int NV = 9; };

template <typename T>
__device__ __forceinline__ void tile_put(typename LinkTile<T>::V *lk, const cpx<T> (&U)[3][3])
{
    using LT = LinkTile<T>;
    alignas(16) T r[16 / sizeof(T) * LT::NV];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            r[6 * a + 2 * c] = U[a][c].re;
            r[6 * a + 2 * c + 1] = U[a][c].im;
        }
#pragma unroll
    for (int k = 18; k < (int)(sizeof(r) / sizeof(T)); ++k) r[k] = T(0);
#pragma unroll
    for (int k = 0; k < LT::NV; ++k) lk[k * 32] = reinterpret_cast<const typename LT::V *>(r)[k];
}

template <typename T>
__device__ __forceinline__ void tile_get(const typename LinkTile<T>::V *lk, cpx<T> (&U)[3][3])
{
    using LT = LinkTile<T>;
    typename LT::V v[LT::NV];
#pragma unroll
    for (int k = 0; k < LT::NV; ++k) v[k] = lk[k * 32];
    const T *r = reinterpret_cast<const T *>(v);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) U[a][c] = {r[6 * a + 2 * c], r[6 * a + 2 * c + 1]};
}

template <int P, int MU, int S, bool FWD>
__device__ __forceinline__ void hop_dir_smem(const char *in, int vh, int nb,
                                             const typename LinkTile<typename Prec<P>::real>::V *lk,
                                             cpx<typename Prec<P>::real> (&acc)[4][3])
{
    using T = typename Prec<P>::real;
    T psi[24];
    Spinor<P>::load(in, vh, nb, psi);
    cpx<T> h0[3], h1[3];
    project<MU, S>(psi, h0, h1);
    cpx<T> U[3][3];
    tile_get<T>(lk, U);
    cpx<T> w0[3], w1[3];
    su3_mul<FWD>(U, h0, w0);
    su3_mul<FWD>(U, h1, w1);
    accumulate<MU, S>(acc, w0, w1);
}

// Multi right-hand-side hop: a block owns 32 consecutive checkerboard sites
// and all nrhs fields.  The 8 links of each site are loaded once (row 3
// rebuilt once for 12-real storage) into shared memory, then warp y of the
// block computes right-hand sides y, y + blockDim.y, ... from them, so links
// cost 1/nrhs of their single-field traffic.  Spinors are read per field as in
// hop_kernel.  blockDim = (32, RY).  Reduced precisions are compiled for 3
// resident blocks of 256 threads per SM (at most 80 registers, no spills);
// FP64 needs twice the registers per complex number and is left unbounded.
//
// Site order.  With zs = 0 block b takes checkerboard sites 32b .. 32b+31, so
// the (z, t) slices of the lattice are visited t-major and a source spinor read
// as the t+ neighbour of slice (z, t-1) is read again as the t- neighbour of
// slice (z, t+1) 2*Lz slices later: with all nrhs fields per block that span
// (inputs, outputs and links of 2*Lz slices) can exceed what L2 keeps.  With
// 0 < zs < Lz the slices are visited in z-strips of width zs, t
// outer and z inner within a strip, which brings that distance down to 2*zs
// slices at the price of re-reading the two z-planes at each strip boundary.
// The last strip is narrower when zs does not divide Lz.  j -> site is a
// bijection of [0, vh) that keeps the order within a slice.
__device__ __forceinline__ int mrhs_site(const HopArgs &A, int j, int zs)
{
    if (zs == 0) return j;
    const int sxy = (A.L[0] >> 1) * A.L[1];
    const int q = j / sxy;
    const int off = j - q * sxy;
    const int per_strip = zs * A.L[3];
    const int k = q / per_strip;
    const int w = min(zs, A.L[2] - k * zs);
    const int l = q - k * per_strip;
    const int t = l / w;
    const int z = k * zs + (l - t * w);
    return off + sxy * (z + A.L[2] * t);
}

template <int P, int RECON, bool DAG, bool HAS_X>
__global__ void __launch_bounds__(256, P == PREC_F64 ? 1 : 3) hop_mrhs_kernel(const HopArgs A, const int nrhs, const int zs)
{
    using T = typename Prec<P>::real;
    using LT = LinkTile<T>;
    __shared__ typename LT::V lk[8][LT::NV][32];
    __shared__ int nbs[9][32];   // rows 0..7: neighbours, row 8: the site itself (-1: none)
    int p, blk;
    if (A.nparity == 2) { p = blockIdx.x & 1; blk = blockIdx.x >> 1; }
    else { p = A.parity0; blk = blockIdx.x; }
    const int vh = A.vh;
    const int s = threadIdx.x;
    const int j = blk * 32 + s;
    const bool active = j < vh;
    const int i = active ? mrhs_site(A, j, zs) : -1;
    const char *gf = p ? A.gauge[1] : A.gauge[0];
    const char *gb = p ? A.gauge[0] : A.gauge[1];
    const size_t lb = A.link_blk;
    using LK = Link<link_prec(P), RECON>;
    if (threadIdx.y == 0) {
        nbs[8][s] = i;
        if (active) {
            int nb[8];
            site_neighbours(A, p, i, nb);
#pragma unroll
            for (int d = 0; d < 8; ++d) nbs[d][s] = nb[d];
        }
    }
    __syncthreads();
    // stage the 8 links of the 32 sites: pair (direction d, site ss)
    const int tid = threadIdx.y * 32 + threadIdx.x, nthr = 32 * blockDim.y;
    for (int pr = tid; pr < 256; pr += nthr) {
        const int d = pr >> 5, ss = pr & 31;
        const int is = nbs[8][ss];
        if (is < 0) continue;
        const int mu = d & 3;
        const char *lblk = d < 4 ? gf + mu * lb : gb + mu * lb;
        const int li = d < 4 ? is : nbs[d][ss];
        cpx<T> U[3][3];
        LK::load(lblk, vh, li, U);
        tile_put<T>(&lk[d][0][ss], U);
    }
    __syncthreads();
    if (!active) return;
    int nb[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) nb[d] = nbs[d][s];
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    const T a = (T)A.a, b = (T)A.b;
    for (int rhs = threadIdx.y; rhs < nrhs; rhs += blockDim.y) {
        const size_t roff = (size_t)rhs * A.rhs_stride;
        const char *in = (p ? A.in[1] : A.in[0]) + roff;
        cpx<T> acc[4][3];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[sp][c] = {T(0), T(0)};
        hop_dir_smem<P, 0, SB, false>(in, vh, nb[4], &lk[4][0][s], acc);
        hop_dir_smem<P, 1, SB, false>(in, vh, nb[5], &lk[5][0][s], acc);
        hop_dir_smem<P, 2, SB, false>(in, vh, nb[6], &lk[6][0][s], acc);
        hop_dir_smem<P, 3, SB, false>(in, vh, nb[7], &lk[7][0][s], acc);
        hop_dir_smem<P, 0, SF, true>(in, vh, nb[0], &lk[0][0][s], acc);
        hop_dir_smem<P, 1, SF, true>(in, vh, nb[1], &lk[1][0][s], acc);
        hop_dir_smem<P, 2, SF, true>(in, vh, nb[2], &lk[2][0][s], acc);
        hop_dir_smem<P, 3, SF, true>(in, vh, nb[3], &lk[3][0][s], acc);
        T o[24];
        if constexpr (HAS_X) {
            Spinor<P>::load((p ? A.x[1] : A.x[0]) + roff, vh, i, o);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    o[6 * sp + 2 * c] = a * o[6 * sp + 2 * c] + b * acc[sp][c].re;
                    o[6 * sp + 2 * c + 1] = a * o[6 * sp + 2 * c + 1] + b * acc[sp][c].im;
                }
        } else {
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    o[6 * sp + 2 * c] = b * acc[sp][c].re;
                    o[6 * sp + 2 * c + 1] = b * acc[sp][c].im;
                }
        }
        Spinor<P>::store((p ? A.out[1] : A.out[0]) + roff, vh, i, o);
    }
}

constexpr int HOP_VARIANTS = 3;       // memory schedules 0..2 (one site per thread, linear blocks)
constexpr int HOP_MRHS_VARIANT = 3;   // variant index of the shared-link multi-RHS kernel
constexpr int HOP_OCC_VARIANT = 4;    // schedule 1 compiled for 3 blocks of 256 threads per SM
constexpr int HOP_MAX_VARIANT = 7;    // 5, 6, 7: the multi-RHS kernel in z-strips of 16, 8, 4

// Multi-RHS variants and their z-strip width (0: natural order); -1 if v is not one.
__host__ __device__ constexpr int hop_mrhs_strip(int v)
{
    return v == HOP_MRHS_VARIANT ? 0 : v == 5 ? 16 : v == 6 ? 8 : v == 7 ? 4 : -1;
}

template <int P, int RECON, bool DAG, bool HX>
void launch_hop_pf(const HopArgs &A, dim3 grid, int threads, int pf, cudaStream_t s)
{
    switch (pf) {
    case 0: wd_launch(hop_kernel<P, RECON, DAG, HX, 0>, grid, dim3(threads), 0, s, A); break;
    case 1: wd_launch(hop_kernel<P, RECON, DAG, HX, 1>, grid, dim3(threads), 0, s, A); break;
    case 2: wd_launch(hop_kernel<P, RECON, DAG, HX, 2>, grid, dim3(threads), 0, s, A); break;
    default: wd_launch(hop_kernel<P, RECON, DAG, HX, 4>, grid, dim3(threads), 0, s, A); break;
    }
}

template <int P, int RECON, bool DAG, bool HX>
void launch_hop_mrhs(const HopArgs &A, int nrhs, int threads, int zs, cudaStream_t s)
{
    const int ry = threads / 32;
    const int per = (A.vh + 31) / 32;
    if (zs <= 0 || zs >= A.L[2]) zs = 0;
    wd_launch(hop_mrhs_kernel<P, RECON, DAG, HX>, dim3((unsigned)(per * A.nparity)), dim3(32, ry), 0, s, A, nrhs, zs);
}

// Launches the hop kernel of precision P for the runtime (recon, dagger,
// has_x) with `threads` per block (at most 256) and memory schedule `pf`
// (pf = HOP_MRHS_VARIANT and 5..7: the shared-link multi-RHS kernel, threads/32
// fields at a time, in the site order hop_mrhs_strip(pf) names).
template <int P>
cudaError_t launch_hop(const HopArgs &A, int recon, int dagger, int nrhs, int threads, int pf, cudaStream_t s)
{
    const int zs = hop_mrhs_strip(pf);
    if (zs >= 0) {
        const bool hx = A.x[0] != nullptr || A.x[1] != nullptr;
        const int key = (recon == 12 ? 4 : 0) + (dagger ? 2 : 0) + (hx ? 1 : 0);
        switch (key) {
        case 0: launch_hop_mrhs<P, 18, false, false>(A, nrhs, threads, zs, s); break;
        case 1: launch_hop_mrhs<P, 18, false, true>(A, nrhs, threads, zs, s); break;
        case 2: launch_hop_mrhs<P, 18, true, false>(A, nrhs, threads, zs, s); break;
        case 3: launch_hop_mrhs<P, 18, true, true>(A, nrhs, threads, zs, s); break;
        case 4: launch_hop_mrhs<P, 12, false, false>(A, nrhs, threads, zs, s); break;
        case 5: launch_hop_mrhs<P, 12, false, true>(A, nrhs, threads, zs, s); break;
        case 6: launch_hop_mrhs<P, 12, true, false>(A, nrhs, threads, zs, s); break;
        case 7: launch_hop_mrhs<P, 12, true, true>(A, nrhs, threads, zs, s); break;
        }
        return cudaGetLastError();
    }
    const HopArgs &B = A;
    const int per = (A.vh + threads - 1) / threads;
    const dim3 grid((unsigned)(per * A.nparity), (unsigned)nrhs);
    const bool hx = A.x[0] != nullptr || A.x[1] != nullptr;
    const int key = (recon == 12 ? 4 : 0) + (dagger ? 2 : 0) + (hx ? 1 : 0);
    switch (key) {
    case 0: launch_hop_pf<P, 18, false, false>(B, grid, threads, pf, s); break;
    case 1: launch_hop_pf<P, 18, false, true>(B, grid, threads, pf, s); break;
    case 2: launch_hop_pf<P, 18, true, false>(B, grid, threads, pf, s); break;
    case 3: launch_hop_pf<P, 18, true, true>(B, grid, threads, pf, s); break;
    case 4: launch_hop_pf<P, 12, false, false>(B, grid, threads, pf, s); break;
    case 5: launch_hop_pf<P, 12, false, true>(B, grid, threads, pf, s); break;
    case 6: launch_hop_pf<P, 12, true, false>(B, grid, threads, pf, s); break;
    case 7: launch_hop_pf<P, 12, true, true>(B, grid, threads, pf, s); break;
    }
    return cudaGetLastError();
}

} // namespace wd
