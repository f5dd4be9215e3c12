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

// Blocks of blas_kernel<Op> that fit on one SM at once (queried once per
// operation type).
template <typename Op> inline int blas_resident_blocks()
{
    static const int n = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, blas_kernel<Op>, BLAS_THREADS, 0) != cudaSuccess || b < 1) {
            cudaGetLastError();
            b = 1;
        }
        return b;
    }();
    return n;
}

// Grid of blas_kernel<Op>.  A reduction runs as a single wave: one site per
// thread up to the blocks that fit on the device at once, longer fields
// looping within it (a partial second wave, as with a fixed 8 blocks per SM
// for a kernel that fits 6, leaves the last blocks' partial sums, and so the
// final sum, waiting on its stragglers).  Operations without a reduction keep
// blas_grid.  Fixed by the field size, the SM count and the kernel, so the
// reduction order is too.
template <typename Op> inline int blas_grid_for(const wd_ctx *ctx, int nsite)
{
    if constexpr (Op::NR == 0) return blas_grid(ctx, nsite);
    const int want = (nsite + BLAS_THREADS - 1) / BLAS_THREADS;
    int cap = blas_resident_blocks<Op>() * (ctx->num_sms > 0 ? ctx->num_sms : 132);
    if (cap > MAX_RED_BLOCKS) cap = MAX_RED_BLOCKS;
    return want < cap ? (want > 0 ? want : 1) : cap;
}

template <typename Op> int run_blas(const wd_ctx *ctx, const Op &op, int nsite, cudaStream_t s)
{
    RedScratch rs{ctx->d_partials, ctx->d_ticket};
    cudaError_t e = wd_launch(blas_kernel<Op>, dim3(blas_grid_for<Op>(ctx, nsite)), dim3(BLAS_THREADS), 0, s, op, nsite, rs);
    if (e != cudaSuccess) return set_error(WD_ECUDA, "BLAS kernel launch failed: %s", cudaGetErrorString(e));
    return WD_OK;
}

// Arithmetic of the operator that recomputes the true residual at a reliable
// update: double-word FP32 when a mixed-precision solve asks for it
// (outer_prec = WD_DF), else FP64.  The solution, source, residual and norms
// stay FP64 either way.
inline int outer_prec_of(const wd_cg_opts &o)
{
    return (o.inner_prec != WD_F64 && o.outer_prec == WD_DF) ? WD_DF : WD_F64;
}

// r = b - A x and |r|^2 -> *out for FP64 even half fields x, b, r; ax is
// scratch for A x.  apply(prec, in, out) applies A in precision prec;
// blas(op) launches a BLAS operation on the caller's stream and scratch.  In
// double-word arithmetic x is first converted into r's buffer (r is written
// only by the last step), and A x is widened exactly to FP64 in the difference.
template <typename Apply, typename Blas>
int true_residual(int op, int vh, const char *x, const char *b, char *r, char *ax, double *out, Apply &&apply,
                  Blas &&blas)
{
    const FieldRef<PREC_F64> fb = field_ref<PREC_F64>(b, vh), fr = field_ref<PREC_F64>(r, vh);
    if (op == WD_DF) {
        WD_TRY(blas(OpConvert<PREC_DF, PREC_F64>{field_ref<PREC_DF>(r, vh), field_ref<PREC_F64>(x, vh)}));
        WD_TRY(apply(WD_DF, (const char *)r, ax));
        return blas(OpXmyNorm<PREC_F64, PREC_DF>{fb, field_ref<PREC_DF>(ax, vh), fr, out});
    }
    WD_TRY(apply(WD_F64, x, ax));
    return blas(OpXmyNorm<PREC_F64>{fb, field_ref<PREC_F64>(ax, vh), fr, out});
}

} // namespace wd
