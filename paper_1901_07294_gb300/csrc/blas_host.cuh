// Host-side launcher of the BLAS-1 kernels (shared by the BLAS entry points and the solvers).
#pragma once

#include "blas.cuh"
#include "launch.cuh"
#include "wd_internal.h"

namespace wd {

// Mixed-precision CG: iterations after which a reliable update is forced
// even if the low-precision residual has not yet dropped by delta.
constexpr int RELIABLE_MAX_GAP = 128;

template <int P> inline FieldRef<P> field_ref(const void *p, int vh)
{
    return FieldRef<P>{(char *)p, half_field_bytes(vh, P), vh};
}

// One site per thread up to 8 blocks of 256 threads per SM (the BLAS kernels
// use at most 78 registers, most of them 32-48, so a full SM holds 4-8 blocks):
// short fields finish in one wave and long ones loop with as many loads in
// flight as the SM allows.
inline int blas_grid(const wd_ctx *ctx, int nsite)
{
    int want = (nsite + BLAS_THREADS - 1) / BLAS_THREADS;
    int cap = 8 * (ctx->num_sms > 0 ? ctx->num_sms : 132);
    if (cap > MAX_RED_BLOCKS) cap = MAX_RED_BLOCKS;
    return want < cap ? (want > 0 ? want : 1) : cap;
}

template <typename Op> int run_blas(const wd_ctx *ctx, const Op &op, int nsite, cudaStream_t s)
{
    RedScratch rs{ctx->d_partials, ctx->d_ticket};
    cudaError_t e = wd_launch(blas_kernel<Op>, dim3(blas_grid(ctx, nsite)), dim3(BLAS_THREADS), 0, s, op, nsite, rs);
    if (e != cudaSuccess) return set_error(WD_ECUDA, "BLAS kernel launch failed: %s", cudaGetErrorString(e));
    return WD_OK;
}

} // namespace wd
