// Dispatch of a hop launch (precision, link format, dagger, axpy term and
// variant) to the single-field kernel or the multi right-hand-side kernel.
#pragma once

#include "dslash_df.cuh"
#include "dslash_impl.cuh"
#include "dslash_mrhs.cuh"
#include "dslash_pair.cuh"
#include "dslash_variants.cuh"

namespace wd {

constexpr int HOP_VARIANTS = 3;       // memory schedules 0..2 (one site per thread, linear blocks)
constexpr int HOP_MRHS_VARIANT = 3;   // variant index of the shared-link multi-RHS kernel
constexpr int HOP_OCC_VARIANT = 4;    // schedule 1 compiled for 3 blocks of 256 threads per SM
constexpr int HOP_TILE_VARIANT = 8;   // schedule 1 with the neighbour window staged in shared memory
constexpr int HOP_2SITE_VARIANT = 9;  // schedule 1 with two sites per thread
constexpr int HOP_RETIRED_VARIANT = 10;  // unused (a bulk-copy staged kernel, measured slower and removed): schedule 1
constexpr int HOP_NA0_VARIANT = 11;   // schedule 0 with the links loaded without L1 allocation
constexpr int HOP_NA1_VARIANT = 12;   // schedule 1 with the links loaded without L1 allocation
constexpr int HOP_SP1_VARIANT = 13;   // 16-bit formats: schedule 1 with spin-paired FP32 arithmetic
constexpr int HOP_SP0_VARIANT = 14;   // 16-bit formats: schedule 0, spin-paired, links without L1 allocation
constexpr int HOP_F64_1B_VARIANT = 15;// FP64: schedule 0 built for one block of 256 per SM (no spills); else schedule 0
constexpr int HOP_MAX_VARIANT = 15;   // 5, 6, 7: the multi-RHS kernel in z-strips of 16, 8, 4

// Multi-RHS variants and their z-strip width (0: natural order); -1 if v is not one.
__host__ __device__ constexpr int hop_mrhs_strip(int v)
{
    return v == HOP_MRHS_VARIANT ? 0 : v == 5 ? 16 : v == 6 ? 8 : v == 7 ? 4 : -1;
}

// Launches the hop kernel of precision P (FP64, FP32, FP16, BF16) for the
// runtime link format, dagger and axpy term (`key`, as in launch_hop) with
// `threads` per block (at most 256) and memory schedule `pf`
// (pf = HOP_MRHS_VARIANT and 5..7: the shared-link multi-RHS kernel, threads/32
// fields at a time, in the site order hop_mrhs_strip(pf) names;
// HOP_TILE_VARIANT and HOP_2SITE_VARIANT: the kernels of dslash_variants.cuh;
// HOP_NA0_VARIANT and HOP_NA1_VARIANT: schedules 0 and 1 with the links
// loaded without L1 allocation, for even-odd hops, which read every link
// exactly once; HOP_SP1_VARIANT and HOP_SP0_VARIANT: the spin-paired kernel
// of dslash_pair.cuh for FP16 and BF16 storage, schedules 1 and 0 for FP32,
// FP64 and open-boundary passes).
template <int P>
cudaError_t launch_hop_std(const HopArgs &A, int nrhs, int threads, int pf, int key, cudaStream_t s)
{
    const int zs = A.topen ? -1 : hop_mrhs_strip(pf);   // open-boundary passes use the single-field kernel
    if (zs >= 0) {
        switch (key) {
        case 0: return launch_hop_mrhs<P, 18, false, false>(A, nrhs, threads, zs, s);
        case 1: return launch_hop_mrhs<P, 18, false, true>(A, nrhs, threads, zs, s);
        case 2: return launch_hop_mrhs<P, 18, true, false>(A, nrhs, threads, zs, s);
        case 3: return launch_hop_mrhs<P, 18, true, true>(A, nrhs, threads, zs, s);
        case 4: return launch_hop_mrhs<P, 12, false, false>(A, nrhs, threads, zs, s);
        case 5: return launch_hop_mrhs<P, 12, false, true>(A, nrhs, threads, zs, s);
        case 6: return launch_hop_mrhs<P, 12, true, false>(A, nrhs, threads, zs, s);
        default: return launch_hop_mrhs<P, 12, true, true>(A, nrhs, threads, zs, s);
        }
    }
    const HopArgs &B = A;
    const int per = (A.vh + threads - 1) / threads;
    const dim3 grid((unsigned)(per * A.nparity), (unsigned)nrhs);
    if (pf == HOP_2SITE_VARIANT && !A.topen) {
        switch (key) {
        case 0: return launch_hop_2site<P, 18, false, false>(B, nrhs, threads, s);
        case 1: return launch_hop_2site<P, 18, false, true>(B, nrhs, threads, s);
        case 2: return launch_hop_2site<P, 18, true, false>(B, nrhs, threads, s);
        case 3: return launch_hop_2site<P, 18, true, true>(B, nrhs, threads, s);
        case 4: return launch_hop_2site<P, 12, false, false>(B, nrhs, threads, s);
        case 5: return launch_hop_2site<P, 12, false, true>(B, nrhs, threads, s);
        case 6: return launch_hop_2site<P, 12, true, false>(B, nrhs, threads, s);
        default: return launch_hop_2site<P, 12, true, true>(B, nrhs, threads, s);
        }
    }
    if constexpr (Prec<P>::scaled) {
        if ((pf == HOP_SP1_VARIANT || pf == HOP_SP0_VARIANT) && !A.topen) {
            const int spf = pf == HOP_SP1_VARIANT ? 1 : 0;
            switch (key) {
            case 0: return launch_hop_sp<P, 18, false, false>(B, grid, threads, spf, s);
            case 1: return launch_hop_sp<P, 18, false, true>(B, grid, threads, spf, s);
            case 2: return launch_hop_sp<P, 18, true, false>(B, grid, threads, spf, s);
            case 3: return launch_hop_sp<P, 18, true, true>(B, grid, threads, spf, s);
            case 4: return launch_hop_sp<P, 12, false, false>(B, grid, threads, spf, s);
            case 5: return launch_hop_sp<P, 12, false, true>(B, grid, threads, spf, s);
            case 6: return launch_hop_sp<P, 12, true, false>(B, grid, threads, spf, s);
            default: return launch_hop_sp<P, 12, true, true>(B, grid, threads, spf, s);
            }
        }
    }
    if (pf == HOP_SP1_VARIANT) pf = 1;   // FP32, FP64, or an open-boundary pass
    if (pf == HOP_SP0_VARIANT) pf = 0;
    if (pf == HOP_F64_1B_VARIANT) pf = 5;   // launch_hop_pf: schedule 0 outside FP64
    cudaError_t e = cudaSuccess;
    if (pf == HOP_RETIRED_VARIANT) pf = 1;
    if (pf == HOP_TILE_VARIANT) {
        bool ok = false;
        if (!A.topen) {
            switch (key) {
            case 0: ok = launch_hop_window<P, 18, false, false>(B, grid, threads, s, e); break;
            case 1: ok = launch_hop_window<P, 18, false, true>(B, grid, threads, s, e); break;
            case 2: ok = launch_hop_window<P, 18, true, false>(B, grid, threads, s, e); break;
            case 3: ok = launch_hop_window<P, 18, true, true>(B, grid, threads, s, e); break;
            case 4: ok = launch_hop_window<P, 12, false, false>(B, grid, threads, s, e); break;
            case 5: ok = launch_hop_window<P, 12, false, true>(B, grid, threads, s, e); break;
            case 6: ok = launch_hop_window<P, 12, true, false>(B, grid, threads, s, e); break;
            case 7: ok = launch_hop_window<P, 12, true, true>(B, grid, threads, s, e); break;
            }
        }
        if (ok) return e;
        pf = 1;   // window larger than 48 KB, or an open-boundary pass: schedule 1
    }
    if (pf == HOP_2SITE_VARIANT) pf = 1;   // open-boundary pass
    const bool lna = pf == HOP_NA0_VARIANT || pf == HOP_NA1_VARIANT;
    if (lna) pf = pf == HOP_NA0_VARIANT ? 0 : 1;
    switch (key) {
    case 0: return launch_hop_pf<P, 18, false, false>(B, grid, threads, pf, lna, s);
    case 1: return launch_hop_pf<P, 18, false, true>(B, grid, threads, pf, lna, s);
    case 2: return launch_hop_pf<P, 18, true, false>(B, grid, threads, pf, lna, s);
    case 3: return launch_hop_pf<P, 18, true, true>(B, grid, threads, pf, lna, s);
    case 4: return launch_hop_pf<P, 12, false, false>(B, grid, threads, pf, lna, s);
    case 5: return launch_hop_pf<P, 12, false, true>(B, grid, threads, pf, lna, s);
    case 6: return launch_hop_pf<P, 12, true, false>(B, grid, threads, pf, lna, s);
    default: return launch_hop_pf<P, 12, true, true>(B, grid, threads, pf, lna, s);
    }
}

// Launches the hop kernel of precision P for the runtime (recon, dagger,
// has_x); double-word FP32 has kernels of its own (launch_hop_df).
template <int P>
cudaError_t launch_hop(const HopArgs &A, int recon, int dagger, int nrhs, int threads, int pf, cudaStream_t s)
{
    const bool hx = A.x[0] != nullptr || A.x[1] != nullptr;
    const int key = (recon == 12 ? 4 : 0) + (dagger ? 2 : 0) + (hx ? 1 : 0);
    if constexpr (P == PREC_DF) {
        // double-word FP32: variant HOP_F64_1B_VARIANT is the
        // three-threads-per-site kernel (dslash_df.cuh); otherwise one site
        // per thread, one block of 256 per SM, schedule 1 for variants 1 and 12
        // and schedule 0 for the rest
        if (A.topen) return cudaErrorInvalidValue;
        if (pf == HOP_F64_1B_VARIANT) {
            switch (key) {
            case 0: return launch_hop_df_row<18, false, false>(A, nrhs, s);
            case 1: return launch_hop_df_row<18, false, true>(A, nrhs, s);
            case 2: return launch_hop_df_row<18, true, false>(A, nrhs, s);
            case 3: return launch_hop_df_row<18, true, true>(A, nrhs, s);
            case 4: return launch_hop_df_row<12, false, false>(A, nrhs, s);
            case 5: return launch_hop_df_row<12, false, true>(A, nrhs, s);
            case 6: return launch_hop_df_row<12, true, false>(A, nrhs, s);
            default: return launch_hop_df_row<12, true, true>(A, nrhs, s);
            }
        }
        const int per = (A.vh + threads - 1) / threads;
        const dim3 grid((unsigned)(per * A.nparity), (unsigned)nrhs);
        const int dpf = (pf == 1 || pf == HOP_NA1_VARIANT) ? 6 : 5;
        switch (key) {
        case 0: return launch_hop_df<18, false, false>(A, grid, threads, dpf, s);
        case 1: return launch_hop_df<18, false, true>(A, grid, threads, dpf, s);
        case 2: return launch_hop_df<18, true, false>(A, grid, threads, dpf, s);
        case 3: return launch_hop_df<18, true, true>(A, grid, threads, dpf, s);
        case 4: return launch_hop_df<12, false, false>(A, grid, threads, dpf, s);
        case 5: return launch_hop_df<12, false, true>(A, grid, threads, dpf, s);
        case 6: return launch_hop_df<12, true, false>(A, grid, threads, dpf, s);
        default: return launch_hop_df<12, true, true>(A, grid, threads, dpf, s);
        }
    } else {
        return launch_hop_std<P>(A, nrhs, threads, pf, key, s);
    }
}

} // namespace wd
