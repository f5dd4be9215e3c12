// Multi right-hand-side Wilson hop: the links of 32 sites are staged once in
// shared memory and applied to all fields of the launch (variants
// HOP_MRHS_VARIANT and 5..7 of the hop launch).
#pragma once

#include "dslash_impl.cuh"

namespace wd {

// Neighbour checkerboard indices of site i of parity p, order
// x+, y+, z+, t+, x-, y-, z-, t- (same arithmetic as in hop_kernel).
__device__ __forceinline__ void site_neighbours(const HopArgs &A, int p, int i, int (&nb)[8])
{
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

// hop_dir with the link from the shared-memory tile; for 16-bit storage the
// terms are weighted by the neighbour's scale times wt, as in hop_dir.
template <int P, int MU, int S, bool FWD>
__device__ __forceinline__ void hop_dir_smem(const char *in, int vh, int nb,
                                             const typename LinkTile<typename Prec<P>::real>::V *lk, bool neg,
                                             cpx<typename Prec<P>::real> (&acc)[4][3], const float wt = 1.0f)
{
    using T = typename Prec<P>::real;
    if constexpr (Prec<P>::scaled) {
        unsigned u[12];
        const float sc = Spinor<P>::load_words(in, vh, nb, u);
        cpx<float> h0[3], h1[3];
        project_words<P, MU, S>(u, h0, h1);
        cpx<float> U[3][3];
        tile_get<float>(lk, U);
        cpx<float> w0[3], w1[3];
        su3_mul<FWD>(U, h0, w0);
        su3_mul<FWD>(U, h1, w1);
        accumulate_f<MU, S>(acc, w0, w1, (neg ? -sc : sc) * wt);
        return;
    }
    T psi[24];
    Spinor<P>::load(in, vh, nb, psi);
    cpx<T> h0[3], h1[3];
    project<MU, S>(psi, h0, h1);
    cpx<T> U[3][3];
    tile_get<T>(lk, U);
    cpx<T> w0[3], w1[3];
    su3_mul<FWD>(U, h0, w0);
    su3_mul<FWD>(U, h1, w1);
    if (neg) {   // hop across an antiperiodic boundary
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            w0[c].re = -w0[c].re; w0[c].im = -w0[c].im;
            w1[c].re = -w1[c].re; w1[c].im = -w1[c].im;
        }
    }
    accumulate<MU, S>(acc, w0, w1);
}

// out = a x + b acc at site i of parity p for the field at byte offset roff
template <int P, bool HAS_X>
__device__ __forceinline__ void mrhs_store(const HopArgs &A, int p, int i, size_t roff,
                                           const cpx<typename Prec<P>::real> (&acc)[4][3])
{
    using T = typename Prec<P>::real;
    if constexpr (Prec<P>::scaled) {   // acc already carries b
        store_weighted<P, HAS_X>(HAS_X ? (p ? A.x[1] : A.x[0]) + roff : nullptr, (p ? A.out[1] : A.out[0]) + roff,
                                 A.vh, i, (float)A.a, acc);
        return;
    }
    const T a = (T)A.a, b = (T)A.b;
    T o[24];
    if constexpr (HAS_X) {
        Spinor<P>::load((p ? A.x[1] : A.x[0]) + roff, A.vh, i, o);
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
    Spinor<P>::store((p ? A.out[1] : A.out[0]) + roff, A.vh, i, o);
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
    grid_dependency_enter();
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
        LK::template load<true>(lblk, vh, li, U);   // each link is staged once: no L1 allocation
        tile_put<T>(&lk[d][0][ss], U);
    }
    __syncthreads();
    if (!active) return;
    // the neighbour indices stay in shared memory and are read where used,
    // which keeps eight registers free across the field loop
    const int *nb = &nbs[0][s];   // nb[32 d] = neighbour in direction d; a t hop wraps
                                  // (t = Lt-1 forward, t = 0 backward) exactly when that
                                  // neighbour's checkerboard index falls below / above i
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    for (int rhs = threadIdx.y; rhs < nrhs; rhs += blockDim.y) {
        const size_t roff = (size_t)rhs * A.rhs_stride;
        const char *in = (p ? A.in[1] : A.in[0]) + roff;
        const float wt = Prec<P>::scaled ? (float)A.b : 1.0f;   // 16-bit: b weights the terms
        cpx<T> acc[4][3];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[sp][c] = {T(0), T(0)};
        hop_dir_smem<P, 0, SB, false>(in, vh, nb[128], &lk[4][0][s], false, acc, wt);
        hop_dir_smem<P, 1, SB, false>(in, vh, nb[160], &lk[5][0][s], false, acc, wt);
        hop_dir_smem<P, 2, SB, false>(in, vh, nb[192], &lk[6][0][s], false, acc, wt);
        hop_dir_smem<P, 3, SB, false>(in, vh, nb[224], &lk[7][0][s], A.tneg && nb[224] > i, acc, wt);
        hop_dir_smem<P, 0, SF, true>(in, vh, nb[0], &lk[0][0][s], false, acc, wt);
        hop_dir_smem<P, 1, SF, true>(in, vh, nb[32], &lk[1][0][s], false, acc, wt);
        hop_dir_smem<P, 2, SF, true>(in, vh, nb[64], &lk[2][0][s], false, acc, wt);
        hop_dir_smem<P, 3, SF, true>(in, vh, nb[96], &lk[3][0][s], A.tneg && nb[96] < i, acc, wt);
        mrhs_store<P, HAS_X>(A, p, i, roff, acc);
    }
}

template <int P, int RECON, bool DAG, bool HX>
cudaError_t launch_hop_mrhs(const HopArgs &A, int nrhs, int threads, int zs, cudaStream_t s)
{
    const int ry = threads / 32;
    const int per = (A.vh + 31) / 32;
    if (zs <= 0 || zs >= A.L[2]) zs = 0;
    return wd_launch(hop_mrhs_kernel<P, RECON, DAG, HX>, dim3((unsigned)(per * A.nparity)), dim3(32, ry), 0, s, A, nrhs, zs);
}

} // namespace wd
