// Autotuner candidates beside the memory schedules of hop_kernel: a kernel
// that stages the neighbour window in shared memory (HOP_TILE_VARIANT) and one
// that gives every thread two sites (HOP_2SITE_VARIANT).
//
// Shared-memory window:
// A block of B threads takes the checkerboard sites [i0, i0 + B) of parity p.
// Their x and y neighbours (and any other neighbour that happens to be close)
// have checkerboard indices in [i0 - Lx/2, i0 + B + Lx/2) of the other
// parity's field.  The block copies that window, all its 16-byte planes, into
// shared memory with coalesced loads that are all in flight together, then
// reads each neighbour from shared memory if it falls inside the window and
// from global memory otherwise (z, t, and y across the lattice boundary).
// About a third of the spinor traffic through L1/L2 is replaced by one window
// load per block; the price is a block-wide wait for that load before any
// arithmetic.  Links, the direction order and the L2 prefetches are those of
// memory schedule 1 (hop_site).
#pragma once

#include "dslash_impl.cuh"

namespace wd {

template <int P> struct SpinorWindow {
    const uint4 *v;      // Spinor<P>::nplane planes of `stride` vectors each
    const float *scale;  // 16-bit types: per-site scales
    int lo, n, stride;   // window [lo, lo + n) of the neighbour field
};

template <int P>
__device__ __forceinline__ float window_load_unscaled(const char *in, int vh, int nb, const SpinorWindow<P> &w,
                                                      typename Prec<P>::real (&v)[24])
{
    const unsigned li = (unsigned)(nb - w.lo);
    if (li < (unsigned)w.n) {
        float s = 1.0f;
        if constexpr (Prec<P>::scaled) s = w.scale[li];
#pragma unroll
        for (int k = 0; k < Spinor<P>::nplane; ++k) unpack16<P>(w.v[k * w.stride + li], v + k * Prec<P>::per16, 1.0f);
        return s;
    }
    return Spinor<P>::load_unscaled(in, vh, nb, v);
}

// hop_dir with the neighbour spinor read through the window
template <int P, int RECON, int MU, int S, bool FWD>
__device__ __forceinline__ void hop_dir_window(const char *in, const char *lblk, int vh, int nb, int li, bool neg,
                                               const SpinorWindow<P> &w, cpx<typename Prec<P>::real> (&acc)[4][3])
{
    using T = typename Prec<P>::real;
    T psi[24];
    const float sc = window_load_unscaled<P>(in, vh, nb, w, psi);
    cpx<T> h0[3], h1[3];
    project<MU, S>(psi, h0, h1);
    cpx<T> U[3][3];
    Link<link_prec(P), RECON>::load(lblk, vh, li, U);
    cpx<T> w0[3], w1[3];
    su3_mul<FWD>(U, h0, w0);
    su3_mul<FWD>(U, h1, w1);
    if constexpr (Prec<P>::scaled) {
        const T f = neg ? -sc : sc;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            w0[c].re *= f; w0[c].im *= f;
            w1[c].re *= f; w1[c].im *= f;
        }
    } else {
        if (neg) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                w0[c].re = -w0[c].re; w0[c].im = -w0[c].im;
                w1[c].re = -w1[c].re; w1[c].im = -w1[c].im;
            }
        }
    }
    accumulate<MU, S>(acc, w0, w1);
}

// Shared memory of one block: nplane x (B + Lx) vectors, plus the scales.
template <int P> __host__ __device__ constexpr size_t window_bytes(int threads, int lxh)
{
    return (size_t)Spinor<P>::nplane * (threads + 2 * lxh) * 16 + (Prec<P>::scaled ? (size_t)(threads + 2 * lxh) * 4 : 0);
}

template <int P, int RECON, bool DAG, bool HAS_X>
__global__ void __launch_bounds__(256, 2) hop_window_kernel(const HopArgs A)
{
    grid_dependency_enter();
    using T = typename Prec<P>::real;
    extern __shared__ uint4 window_mem[];
    int p, blk;
    if (A.nparity == 2) { p = blockIdx.x & 1; blk = blockIdx.x >> 1; }
    else { p = A.parity0; blk = blockIdx.x; }
    const int vh = A.vh;
    const int lxh = A.L[0] >> 1;
    const int i0 = blk * blockDim.x;
    const int i = i0 + threadIdx.x;
    const size_t roff = (size_t)blockIdx.y * A.rhs_stride;
    const char *in = (p ? A.in[1] : A.in[0]) + roff;

    // stage the window [lo, hi) of the neighbour field (every thread of the block)
    constexpr int NP = Spinor<P>::nplane;
    const int lo = max(0, i0 - lxh), hi = min(vh, i0 + (int)blockDim.x + lxh);
    const int n = hi - lo;
    const int stride = (int)blockDim.x + 2 * lxh;
    for (int e = threadIdx.x; e < NP * n; e += blockDim.x) {
        const int k = e / n, s = e - k * n;
        window_mem[k * stride + s] = ldg16(in + ((size_t)k * vh + lo + s) * 16);
    }
    float *wscale = reinterpret_cast<float *>(window_mem + NP * stride);
    if constexpr (Prec<P>::scaled)
        for (int s = threadIdx.x; s < n; s += blockDim.x)
            wscale[s] = __ldg(reinterpret_cast<const float *>(in + (size_t)NP * vh * 16) + lo + s);
    __syncthreads();
    if (i >= vh) return;
    const SpinorWindow<P> w{window_mem, wscale, lo, n, stride};

    const char *gf = p ? A.gauge[1] : A.gauge[0];
    const char *gb = p ? A.gauge[0] : A.gauge[1];
    const int Lx = A.L[0], Ly = A.L[1], Lz = A.L[2], Lt = A.L[3];
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
    using LK = Link<link_prec(P), RECON>;

    cpx<T> acc[4][3];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[s][c] = {T(0), T(0)};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) LK::prefetch(gf + mu * lb, vh, i);
    Spinor<P>::prefetch(in, vh, tf);
    hop_dir_window<P, RECON, 0, SB, false>(in, gb + 0 * lb, vh, xb, xb, false, w, acc);
    hop_dir_window<P, RECON, 1, SB, false>(in, gb + 1 * lb, vh, yb, yb, false, w, acc);
    hop_dir_window<P, RECON, 2, SB, false>(in, gb + 2 * lb, vh, zb, zb, false, w, acc);
    hop_dir_window<P, RECON, 3, SB, false>(in, gb + 3 * lb, vh, tb, tb, ntb, w, acc);
    hop_dir_window<P, RECON, 0, SF, true>(in, gf + 0 * lb, vh, xf, i, false, w, acc);
    hop_dir_window<P, RECON, 1, SF, true>(in, gf + 1 * lb, vh, yf, i, false, w, acc);
    hop_dir_window<P, RECON, 2, SF, true>(in, gf + 2 * lb, vh, zf, i, false, w, acc);
    hop_dir_window<P, RECON, 3, SF, true>(in, gf + 3 * lb, vh, tf, i, ntf, w, acc);

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

// Launches the windowed kernel; false (nothing launched) if its shared memory
// would exceed the default 48 KB per block.
template <int P, int RECON, bool DAG, bool HX>
bool launch_hop_window(const HopArgs &A, dim3 grid, int threads, cudaStream_t s, cudaError_t &err)
{
    const size_t smem = window_bytes<P>(threads, A.L[0] >> 1);
    if (smem > 48 * 1024) return false;
    err = wd_launch(hop_window_kernel<P, RECON, DAG, HX>, grid, dim3(threads), smem, s, A);
    return true;
}

// Two sites per thread: sites i and i + B of a block's 2B, schedule 1 for
// each.  The unrolled pair lets the compiler overlap one site's loads with
// the other's arithmetic, at the cost of registers.
template <int P, int RECON, bool DAG, bool HAS_X>
__global__ void __launch_bounds__(256, 2) hop_2site_kernel(const HopArgs A)
{
    grid_dependency_enter();
    int p, blk;
    if (A.nparity == 2) { p = blockIdx.x & 1; blk = blockIdx.x >> 1; }
    else { p = A.parity0; blk = blockIdx.x; }
    const int i = blk * 2 * (int)blockDim.x + threadIdx.x;
    const size_t roff = (size_t)blockIdx.y * A.rhs_stride;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int ik = i + k * (int)blockDim.x;
        if (ik < A.vh) hop_site<P, RECON, DAG, HAS_X, 1>(A, p, ik, roff);
    }
}

template <int P, int RECON, bool DAG, bool HX>
cudaError_t launch_hop_2site(const HopArgs &A, int nrhs, int threads, cudaStream_t s)
{
    const int per = (A.vh + 2 * threads - 1) / (2 * threads);
    return wd_launch(hop_2site_kernel<P, RECON, DAG, HX>, dim3((unsigned)(per * A.nparity), (unsigned)nrhs), dim3(threads),
              0, s, A);
}

} // namespace wd
