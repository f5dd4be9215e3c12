// Element-wise products of Sec. IV (z_i = x_i y_i on double and on complex
// double arrays) and the complex multiply-add forms of Sec. III-D
// (z += x y, z += conj(x) y: the FCMLA rotation pairs), as HBM stream kernels.
//
// On SVE the complex forms map onto FCMLA.  Here one complex number is one
// 16-byte double2 and its product four FP64 instructions (two multiplies and
// two FMAs; four FMAs for the multiply-add forms).  On this part that is
// close to balanced: at full HBM bandwidth the complex kernels need about 90%
// of the FP64 FMA rate, so they are bounded by whichever of the two the
// measured peaks make slower.  Each thread loads STREAM_UNROLL vectors of
// each input before any arithmetic (all loads in flight together), with
// streaming (evict-first) loads and stores; the grid is a multiple of the SM
// count and strides over the arrays.
#include <cstdint>

#include "wd_internal.h"

namespace wd {

namespace {

constexpr int STREAM_THREADS = 256;
constexpr int STREAM_UNROLL = 4;

template <int KIND>
__device__ __forceinline__ double2 stream_op(double2 a, double2 b, double2 c)
{
    if constexpr (KIND == WD_STREAM_REAL_MUL) {
        return make_double2(a.x * b.x, a.y * b.y);
    } else {
        const double ai = (KIND == WD_STREAM_CPLX_CONJ_MUL || KIND == WD_STREAM_CPLX_CONJ_MADD) ? -a.y : a.y;
        if constexpr (KIND == WD_STREAM_CPLX_MADD || KIND == WD_STREAM_CPLX_CONJ_MADD) {
            return make_double2(fma(a.x, b.x, fma(-ai, b.y, c.x)), fma(a.x, b.y, fma(ai, b.x, c.y)));
        } else {
            return make_double2(fma(a.x, b.x, -ai * b.y), fma(a.x, b.y, ai * b.x));
        }
    }
}

// n2 16-byte vectors; z may equal x or y (every element is read before it is
// written, by the same thread).
template <int KIND>
__global__ void __launch_bounds__(STREAM_THREADS) stream_kernel(const double2 *x, const double2 *y, double2 *z,
                                                                size_t n2)
{
    constexpr bool MADD = KIND == WD_STREAM_CPLX_MADD || KIND == WD_STREAM_CPLX_CONJ_MADD;
    const size_t step = (size_t)STREAM_THREADS * STREAM_UNROLL;
    for (size_t base = (size_t)blockIdx.x * step + threadIdx.x; base < n2; base += (size_t)gridDim.x * step) {
        double2 a[STREAM_UNROLL], b[STREAM_UNROLL], c[STREAM_UNROLL];
#pragma unroll
        for (int u = 0; u < STREAM_UNROLL; ++u) {
            const size_t k = base + (size_t)u * STREAM_THREADS;
            if (k < n2) {
                a[u] = __ldcs(x + k);
                b[u] = __ldcs(y + k);
                c[u] = MADD ? __ldcs(z + k) : make_double2(0.0, 0.0);
            }
        }
#pragma unroll
        for (int u = 0; u < STREAM_UNROLL; ++u) {
            const size_t k = base + (size_t)u * STREAM_THREADS;
            if (k < n2) __stcs(z + k, stream_op<KIND>(a[u], b[u], c[u]));
        }
    }
}

// the last element of an odd-length real array
__global__ void stream_real_tail(const double *x, const double *y, double *z, size_t i) { z[i] = x[i] * y[i]; }

template <int KIND>
cudaError_t launch_stream(const wd_ctx *ctx, const double *x, const double *y, double *z, size_t n2, cudaStream_t s)
{
    if (n2 == 0) return cudaSuccess;
    const size_t step = (size_t)STREAM_THREADS * STREAM_UNROLL;
    const size_t want = (n2 + step - 1) / step;
    const size_t cap = (size_t)8 * (ctx->num_sms > 0 ? ctx->num_sms : 132);
    const unsigned blocks = (unsigned)(want < cap ? want : cap);
    stream_kernel<KIND><<<blocks, STREAM_THREADS, 0, s>>>((const double2 *)x, (const double2 *)y, (double2 *)z, n2);
    return cudaGetLastError();
}

} // namespace

} // namespace wd

using namespace wd;

extern "C" {

int wd_stream_mul(wd_ctx *ctx, int kind, size_t n, const double *x, const double *y, double *z, void *stream)
{
    clear_error();
    if (!ctx) return set_error(WD_EINVAL, "ctx is NULL");
    if (kind < WD_STREAM_REAL_MUL || kind > WD_STREAM_CPLX_CONJ_MADD)
        return set_error(WD_EINVAL, "kind = %d is not a wd_stream_kind value", kind);
    if (n == 0) return WD_OK;
    if (!x || !y || !z) return set_error(WD_EINVAL, "NULL array pointer");
    if (((uintptr_t)x | (uintptr_t)y | (uintptr_t)z) & 15u)
        return set_error(WD_EINVAL, "arrays must be 16-byte aligned");
    if (n > ((size_t)1 << 40)) return set_error(WD_EINVAL, "n = %zu is too large", n);
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    switch (kind) {
    case WD_STREAM_REAL_MUL:
        e = launch_stream<WD_STREAM_REAL_MUL>(ctx, x, y, z, n / 2, s);
        if (e == cudaSuccess && (n & 1)) {
            stream_real_tail<<<1, 1, 0, s>>>(x, y, z, n - 1);
            e = cudaGetLastError();
        }
        break;
    case WD_STREAM_CPLX_MUL: e = launch_stream<WD_STREAM_CPLX_MUL>(ctx, x, y, z, n, s); break;
    case WD_STREAM_CPLX_CONJ_MUL: e = launch_stream<WD_STREAM_CPLX_CONJ_MUL>(ctx, x, y, z, n, s); break;
    case WD_STREAM_CPLX_MADD: e = launch_stream<WD_STREAM_CPLX_MADD>(ctx, x, y, z, n, s); break;
    default: e = launch_stream<WD_STREAM_CPLX_CONJ_MADD>(ctx, x, y, z, n, s); break;
    }
    if (e != cudaSuccess) return set_error(WD_ECUDA, "stream kernel launch failed: %s", cudaGetErrorString(e));
    return WD_OK;
}

} // extern "C"
