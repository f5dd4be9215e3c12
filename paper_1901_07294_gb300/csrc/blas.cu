// BLAS-1 entry points: norm, inner product, axpby and precision conversion of
// device fields, with deterministic FP64 reductions.
#include "blas_host.cuh"

namespace wd {

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Number of sites covered by a field of `sites` (2*Vh for a full field).
static int blas_sites(const int dims[4], int sites, Geometry &g)
{
    WD_TRY(make_geometry(dims, g));
    if (sites == WD_SITES_FULL) return 2 * g.Vh;
    if (sites == WD_SITES_EVEN || sites == WD_SITES_ODD) return g.Vh;
    return set_error(WD_EINVAL, "sites = %d is not a wd_sites value", sites);
}

#define WD_PREC_SWITCH(prec, ...)                           \
    switch (prec) {                                         \
    case WD_F64: { constexpr int P = PREC_F64; __VA_ARGS__; } break; \
    case WD_F32: { constexpr int P = PREC_F32; __VA_ARGS__; } break; \
    case WD_F16: { constexpr int P = PREC_F16; __VA_ARGS__; } break; \
    case WD_BF16: { constexpr int P = PREC_BF16; __VA_ARGS__; } break; \
    case WD_DF: { constexpr int P = PREC_DF; __VA_ARGS__; } break; \
    default: return set_error(WD_EINVAL, "bad precision %d", prec); \
    }

} // namespace wd

using namespace wd;

extern "C" {

int wd_norm2(wd_ctx *ctx, const int dims[4], int sites, int prec, const void *x, double *result, void *stream)
{
    clear_error();
    if (!ctx || !x || !result) return set_error(WD_EINVAL, "NULL argument");
    if (!aligned16(x) || ((uintptr_t)result & 7u)) return set_error(WD_EINVAL, "misaligned pointer");
    Geometry g;
    const int n = blas_sites(dims, sites, g);
    if (n < 0) return n;
    WD_PREC_SWITCH(prec, {
        OpNorm2<P> op{field_ref<P>(x, g.Vh), result};
        return run_blas(ctx, op, n, (cudaStream_t)stream);
    });
    return WD_OK;
}

int wd_dot(wd_ctx *ctx, const int dims[4], int sites, int prec, const void *a, const void *b, double *result,
           void *stream)
{
    clear_error();
    if (!ctx || !a || !b || !result) return set_error(WD_EINVAL, "NULL argument");
    if (!aligned16(a) || !aligned16(b) || ((uintptr_t)result & 7u)) return set_error(WD_EINVAL, "misaligned pointer");
    Geometry g;
    const int n = blas_sites(dims, sites, g);
    if (n < 0) return n;
    WD_PREC_SWITCH(prec, {
        OpDot<P, P> op{field_ref<P>(a, g.Vh), field_ref<P>(b, g.Vh), result};
        return run_blas(ctx, op, n, (cudaStream_t)stream);
    });
    return WD_OK;
}

int wd_axpby(wd_ctx *ctx, const int dims[4], int sites, int prec, double a, const void *x, double b, void *y,
             void *stream)
{
    clear_error();
    if (!ctx || !x || !y) return set_error(WD_EINVAL, "NULL argument");
    if (!aligned16(x) || !aligned16(y)) return set_error(WD_EINVAL, "misaligned pointer");
    Geometry g;
    const int n = blas_sites(dims, sites, g);
    if (n < 0) return n;
    WD_PREC_SWITCH(prec, {
        OpAxpby<P, P> op{field_ref<P>(x, g.Vh), field_ref<P>(y, g.Vh), a, b};
        return run_blas(ctx, op, n, (cudaStream_t)stream);
    });
    return WD_OK;
}

int wd_convert(wd_ctx *ctx, const int dims[4], int sites, int prec_out, void *out, int prec_in, const void *in,
               void *stream)
{
    clear_error();
    if (!ctx || !out || !in) return set_error(WD_EINVAL, "NULL argument");
    if (!aligned16(out) || !aligned16(in)) return set_error(WD_EINVAL, "misaligned pointer");
    if (out == in) return set_error(WD_EINVAL, "out must not alias in");
    Geometry g;
    const int n = blas_sites(dims, sites, g);
    if (n < 0) return n;
    if (!valid_field_prec(prec_in)) return set_error(WD_EINVAL, "bad precision %d", prec_in);
    WD_PREC_SWITCH(prec_out, {
        constexpr int PD = P;
        WD_PREC_SWITCH(prec_in, {
            OpConvert<PD, P> op{field_ref<PD>(out, g.Vh), field_ref<P>(in, g.Vh)};
            return run_blas(ctx, op, n, (cudaStream_t)stream);
        });
    });
    return WD_OK;
}

} // extern "C"
