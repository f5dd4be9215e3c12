// Autotuner candidate HOP_BULK_VARIANT: memory schedule 1 with the block's
// contiguous data staged in shared memory by the bulk-copy (TMA) engine.
//
// A block of B threads takes the checkerboard sites [i0, i0 + B) of parity p,
// all in one t-slice (the launch requires B to divide the slice).  Three kinds
// of data it reads are then contiguous ranges of 16-byte planes:
//   - the forward links U_mu(x) of its sites, planes [i0, i0 + B) of the four
//     (p, mu) link blocks;
//   - the t-forward neighbours, planes [j0, j0 + B) of the source field, with
//     j0 = i0 + (one t-slice), or the first slice for the last one;
//   - the axpy term x at its own sites.
// These are the data a block touches first (the backward links and the x, y,
// z neighbours have mostly been brought into L2 by neighbouring blocks).  One
// warp issues a cp.async.bulk per plane at block start, completing on one
// mbarrier; the threads meanwhile run the four backward directions from
// global memory, then wait on the mbarrier and run the forward directions
// with their links, the t neighbour and x read from shared memory.  The
// copies take no registers and no load instructions of the computing warps.
//
// The wait is bounded (one second of clock cycles by default,
// WD_BULK_TIMEOUT_S); on expiry the block writes WD_ETIMEOUT to the context's
// status word, waits once more (bounded) for its copies, and returns without
// writing its output.  Tests make the wait run out with a host-side switch
// (WD_FAULT=bulk_tx) that makes the barrier expect 16 bytes more than are
// copied.
#pragma once

#include <cstdlib>
#include <cstring>

#include "dslash_impl.cuh"
#include "wdirac.h"

namespace wd {

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned phase)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Waits for phase `phase` of the barrier for at most `limit` clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned phase, long long limit)
{
    if (mbar_try_wait(bar, phase)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Global -> shared bulk copy of `bytes` (a multiple of 16; both addresses
// 16-byte aligned) completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}


// Shared-memory image of the staged data for B sites: per mu the link planes
// (main planes, then the tail plane) of the forward links, then the t-forward
// neighbour's spinor planes (+ scales), then those of x.  Every piece starts
// on a 16-byte boundary when B is a multiple of 4.
template <int P, int RECON> struct BulkTile {
    static constexpr int LP = link_prec(P);
    using LK = Link<LP, RECON>;
    static constexpr int lmain = LK::nmain;
    static constexpr int ltail = LK::ntail * Prec<LP>::bytes;   // tail bytes per site
    static constexpr int lsite = RECON * Prec<LP>::bytes;       // link bytes per site and mu
    static constexpr int splanes = Spinor<P>::nplane;
    static constexpr int sscale = Prec<P>::scaled ? 4 : 0;
    static constexpr int ssite = splanes * 16 + sscale;          // spinor bytes per site
    static constexpr int lcopies = lmain + (ltail ? 1 : 0);      // bulk copies per mu
    static constexpr int scopies = splanes + (sscale ? 1 : 0);   // bulk copies per spinor range
    __host__ __device__ static constexpr size_t bytes(int b, bool hx)
    {
        return (size_t)b * (4 * lsite + ssite * (hx ? 2 : 1));
    }
};

// Link of site s from its staged planes (`tile` = the mu block of B sites).
template <int P, int RECON>
__device__ __forceinline__ void tile_link(const unsigned char *tile, int b, int s,
                                          cpx<typename Prec<P>::real> (&U)[3][3])
{
    using BT = BulkTile<P, RECON>;
    constexpr int LP = BT::LP;
    using real = typename Prec<LP>::real;   // storage-side real (FP32 for the 16-bit formats)
    real u[18];
#pragma unroll
    for (int k = 0; k < BT::lmain; ++k)
        unpack16<LP>(*reinterpret_cast<const uint4 *>(tile + ((size_t)k * b + s) * 16), u + k * Prec<LP>::per16,
                     1.0f);
    if constexpr (BT::ltail > 0) {
        const unsigned char *tp = tile + (size_t)BT::lmain * b * 16 + (size_t)s * BT::ltail;
        constexpr int o = BT::lmain * Prec<LP>::per16;
        if constexpr (LP == PREC_F32) {
            const float2 t = *reinterpret_cast<const float2 *>(tp);
            u[o] = t.x; u[o + 1] = t.y;
        } else if constexpr (BT::ltail == 4) {
            const __half2 t = *reinterpret_cast<const __half2 *>(tp);
            const float2 f = __half22float2(t);
            u[o] = f.x; u[o + 1] = f.y;
        } else {
            const uint2 t = *reinterpret_cast<const uint2 *>(tp);
            const float2 f0 = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
            const float2 f1 = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
            u[o] = f0.x; u[o + 1] = f0.y; u[o + 2] = f1.x; u[o + 3] = f1.y;
        }
    }
#pragma unroll
    for (int r = 0; r < (RECON == 18 ? 3 : 2); ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) { U[r][c].re = u[6 * r + 2 * c]; U[r][c].im = u[6 * r + 2 * c + 1]; }
    if constexpr (RECON == 12) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int a = (c + 1) % 3, d = (c + 2) % 3;
            const cpx<real> t = cmul(U[0][a], U[1][d]);
            const cpx<real> q = cmul(U[0][d], U[1][a]);
            U[2][c].re = t.re - q.re;
            U[2][c].im = -(t.im - q.im);
        }
    }
}

// Spinor of site s from its staged planes; returns the per-site scale (1 for
// FP64/FP32), the 24 reals left unscaled.
template <int P>
__device__ __forceinline__ float tile_spinor(const unsigned char *tile, int b, int s, typename Prec<P>::real (&v)[24])
{
    using BT = BulkTile<P, 18>;
#pragma unroll
    for (int k = 0; k < BT::splanes; ++k)
        unpack16<P>(*reinterpret_cast<const uint4 *>(tile + ((size_t)k * b + s) * 16), v + k * Prec<P>::per16, 1.0f);
    if constexpr (Prec<P>::scaled) return reinterpret_cast<const float *>(tile + (size_t)BT::splanes * b * 16)[s];
    return 1.0f;
}

// One direction from an already loaded neighbour (unscaled reals + scale) and link.
template <int P, int MU, int S, bool FWD>
__device__ __forceinline__ void hop_dir_loaded(const typename Prec<P>::real (&psi)[24], float sc,
                                               const cpx<typename Prec<P>::real> (&U)[3][3], bool neg,
                                               cpx<typename Prec<P>::real> (&acc)[4][3])
{
    using T = typename Prec<P>::real;
    cpx<T> h0[3], h1[3];
    project<MU, S>(psi, h0, h1);
    cpx<T> w0[3], w1[3];
    su3_mul<FWD>(U, h0, w0);
    su3_mul<FWD>(U, h1, w1);
    T f = T(1);
    if constexpr (Prec<P>::scaled) f = sc;
    if (neg) f = -f;
    if (Prec<P>::scaled || neg) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            w0[c].re *= f; w0[c].im *= f;
            w1[c].re *= f; w1[c].im *= f;
        }
    }
    accumulate<MU, S>(acc, w0, w1);
}

// Issues the block's bulk copies (called by all 32 lanes of one warp).
template <int P, int RECON, bool HAS_X>
__device__ __forceinline__ void bulk_issue(unsigned char *tile, int b, const char *gf, size_t lb, int vh, int i0,
                                           const char *in, int j0, const char *x, unsigned long long *bar, int lane,
                                           unsigned extra_tx)
{
    using BT = BulkTile<P, RECON>;
    constexpr int nl = 4 * BT::lcopies;
    constexpr int nc = nl + BT::scopies * (HAS_X ? 2 : 1);
    if (lane == 0) mbar_arrive_expect_tx(bar, (unsigned)BT::bytes(b, HAS_X) + extra_tx);
    __syncwarp();
    for (int c = lane; c < nc; c += 32) {
        unsigned char *dst;
        const char *src;
        unsigned n;
        if (c < nl) {   // link plane k of direction mu
            const int mu = c / BT::lcopies, k = c - mu * BT::lcopies;
            const char *blk = gf + mu * lb;
            unsigned char *t = tile + (size_t)mu * b * BT::lsite;
            if (k < BT::lmain) {
                dst = t + (size_t)k * b * 16;
                src = blk + ((size_t)k * vh + i0) * 16;
                n = (unsigned)b * 16u;
            } else {
                dst = t + (size_t)BT::lmain * b * 16;
                src = blk + (size_t)BT::lmain * vh * 16 + (size_t)i0 * BT::ltail;
                n = (unsigned)b * (unsigned)BT::ltail;
            }
        } else {        // spinor plane k of the t neighbour (q = 0) or of x (q = 1)
            const int q = (c - nl) / BT::scopies, k = (c - nl) - q * BT::scopies;
            const char *f = q ? x : in;
            const int j = q ? i0 : j0;
            unsigned char *t = tile + (size_t)b * (4 * BT::lsite + q * BT::ssite);
            if (k < BT::splanes) {
                dst = t + (size_t)k * b * 16;
                src = f + ((size_t)k * vh + j) * 16;
                n = (unsigned)b * 16u;
            } else {
                dst = t + (size_t)BT::splanes * b * 16;
                src = f + (size_t)BT::splanes * vh * 16 + (size_t)j * 4;
                n = (unsigned)b * 4u;
            }
        }
        bulk_g2s(dst, src, n, bar);
    }
}

template <int P, int RECON, bool DAG, bool HAS_X>
__global__ void __launch_bounds__(256, P == PREC_F64 ? 1 : 2) hop_bulk_kernel(const HopArgs A, const unsigned extra_tx,
                                                                            const long long limit)
{
    using T = typename Prec<P>::real;
    using BT = BulkTile<P, RECON>;
    extern __shared__ __align__(16) unsigned char bulk_smem[];
    __shared__ __align__(8) unsigned long long bar;
    int p, blk;
    if (A.nparity == 2) { p = blockIdx.x & 1; blk = blockIdx.x >> 1; }
    else { p = A.parity0; blk = blockIdx.x; }
    const int b = blockDim.x, s = threadIdx.x;
    const int i0 = blk * b, i = i0 + s;     // every block is full (launch condition)
    const int vh = A.vh;
    const size_t roff = (size_t)blockIdx.y * A.rhs_stride;
    const char *in = (p ? A.in[1] : A.in[0]) + roff;
    const char *gf = p ? A.gauge[1] : A.gauge[0];
    const char *gb = p ? A.gauge[0] : A.gauge[1];
    const size_t lb = A.link_blk;

    const int Lx = A.L[0], Ly = A.L[1], Lz = A.L[2], Lt = A.L[3];
    const int lxh = Lx >> 1;
    const int sy = lxh, sz = lxh * Ly, st = sz * Lz;
    const int t = i0 / st;                  // the block's t-slice
    const int j0 = (t == Lt - 1) ? i0 - (Lt - 1) * st : i0 + st;

    if (s == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (s < 32)
        bulk_issue<P, RECON, HAS_X>(bulk_smem, b, gf, lb, vh, i0, in, j0,
                                    HAS_X ? (p ? A.x[1] : A.x[0]) + roff : nullptr, &bar, s, extra_tx);

    // site coordinates (as in hop_site)
    const int r = div_inv(i, A.div_m[0], A.div_s[0]);
    const int xh = i - r * lxh;
    const int r2 = div_inv(r, A.div_m[1], A.div_s[1]);
    const int y = r - r2 * Ly;
    const int z = r2 - t * Lz;
    const int xc = 2 * xh + ((p + y + z + t) & 1);
    const int row = i - xh;
    const int xf = row + ((xc + 1 == Lx ? 0 : xc + 1) >> 1);
    const int xb = row + ((xc == 0 ? Lx - 1 : xc - 1) >> 1);
    const int yf = (y == Ly - 1) ? i - (Ly - 1) * sy : i + sy;
    const int yb = (y == 0) ? i + (Ly - 1) * sy : i - sy;
    const int zf = (z == Lz - 1) ? i - (Lz - 1) * sz : i + sz;
    const int zb = (z == 0) ? i + (Lz - 1) * sz : i - sz;
    const int tb = (t == 0) ? i + (Lt - 1) * st : i - st;
    const bool ntf = A.tneg && t == Lt - 1, ntb = A.tneg && t == 0;

    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    cpx<T> acc[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[a][c] = {T(0), T(0)};

    // backward directions from global memory while the copies are in flight
    hop_dir<P, RECON, 0, SB, false>(in, gb + 0 * lb, vh, xb, xb, false, acc);
    hop_dir<P, RECON, 1, SB, false>(in, gb + 1 * lb, vh, yb, yb, false, acc);
    hop_dir<P, RECON, 2, SB, false>(in, gb + 2 * lb, vh, zb, zb, false, acc);
    hop_dir<P, RECON, 3, SB, false>(in, gb + 3 * lb, vh, tb, tb, ntb, acc);

    if (!mbar_wait_bounded(&bar, 0, limit)) {
        if (A.status) atomicExch(A.status, WD_ETIMEOUT);
        mbar_wait_bounded(&bar, 0, limit);   // let the copies land before the block exits
        return;
    }
    const unsigned char *lt = bulk_smem;
    const unsigned char *tn = bulk_smem + (size_t)b * 4 * BT::lsite;
    {
        T psi[24];
        cpx<T> U[3][3];
        float sc = Spinor<P>::load_unscaled(in, vh, xf, psi);
        tile_link<P, RECON>(lt + 0 * (size_t)b * BT::lsite, b, s, U);
        hop_dir_loaded<P, 0, SF, true>(psi, sc, U, false, acc);
        sc = Spinor<P>::load_unscaled(in, vh, yf, psi);
        tile_link<P, RECON>(lt + 1 * (size_t)b * BT::lsite, b, s, U);
        hop_dir_loaded<P, 1, SF, true>(psi, sc, U, false, acc);
        sc = Spinor<P>::load_unscaled(in, vh, zf, psi);
        tile_link<P, RECON>(lt + 2 * (size_t)b * BT::lsite, b, s, U);
        hop_dir_loaded<P, 2, SF, true>(psi, sc, U, false, acc);
        sc = tile_spinor<P>(tn, b, s, psi);
        tile_link<P, RECON>(lt + 3 * (size_t)b * BT::lsite, b, s, U);
        hop_dir_loaded<P, 3, SF, true>(psi, sc, U, ntf, acc);
    }

    const T bb = (T)A.b;
    T o[24];
    if constexpr (HAS_X) {
        T a = (T)A.a;
        const float xs = tile_spinor<P>(tn + (size_t)b * BT::ssite, b, s, o);
        if constexpr (Prec<P>::scaled) a *= xs;
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o[6 * sp + 2 * c] = a * o[6 * sp + 2 * c] + bb * acc[sp][c].re;
                o[6 * sp + 2 * c + 1] = a * o[6 * sp + 2 * c + 1] + bb * acc[sp][c].im;
            }
    } else {
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o[6 * sp + 2 * c] = bb * acc[sp][c].re;
                o[6 * sp + 2 * c + 1] = bb * acc[sp][c].im;
            }
    }
    Spinor<P>::store((p ? A.out[1] : A.out[0]) + roff, vh, i, o);
}

// Launches the staged kernel if the problem allows it (every block inside one
// t-slice, all bases and plane offsets 16-byte aligned, no open boundary);
// returns false otherwise and the caller uses schedule 1.
template <int P, int RECON, bool DAG, bool HX>
bool launch_hop_bulk(const HopArgs &A, dim3 grid, int threads, cudaStream_t s, cudaError_t &err)
{
    using BT = BulkTile<P, RECON>;
    const int st = (A.L[0] >> 1) * A.L[1] * A.L[2];
    auto al = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
    if (A.topen || st % threads != 0 || (threads & 3)) return false;
    if (!al(A.gauge[0]) || !al(A.gauge[1]) || (A.link_blk & 15) || (A.rhs_stride & 15)) return false;
    for (int q = 0; q < 2; ++q)
        if (!al(A.in[q]) || (HX && !al(A.x[q]))) return false;
    const size_t smem = BT::bytes(threads, HX);
    if (smem > 200 * 1024) return false;
    // dynamic shared memory beyond 48 KB minus the static barrier word needs the opt-in
    if (smem > 47 * 1024 &&
        cudaFuncSetAttribute(hop_bulk_kernel<P, RECON, DAG, HX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // host-side fault injection for tests (WD_FAULT=bulk_tx) and the wait limit
    const char *fault = std::getenv("WD_FAULT");
    const unsigned extra_tx = (fault && std::strstr(fault, "bulk_tx")) ? 16u : 0u;
    double limit_s = 1.0;
    if (const char *ls = std::getenv("WD_BULK_TIMEOUT_S")) limit_s = std::atof(ls);
    const long long limit = (long long)(limit_s * device_clock_khz() * 1e3);
    err = wd_launch(hop_bulk_kernel<P, RECON, DAG, HX>, grid, dim3(threads), smem, s, A, extra_tx, limit);
    return true;
}

} // namespace wd
