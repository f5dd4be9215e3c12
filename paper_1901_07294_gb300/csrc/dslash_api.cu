// C entry points of the Wilson-Dirac operator: dslash_apply (full lattice)
// and dslash_eo_apply (even-odd block with fused axpby).
#include <cstdio>
#include <string>

#include "dslash_launch.cuh"
#include "wd_internal.h"

namespace wd {
extern template cudaError_t launch_hop<PREC_F64>(const HopArgs &, int, int, int, int, int, cudaStream_t);
extern template cudaError_t launch_hop<PREC_F32>(const HopArgs &, int, int, int, int, int, cudaStream_t);
extern template cudaError_t launch_hop<PREC_F16>(const HopArgs &, int, int, int, int, int, cudaStream_t);
extern template cudaError_t launch_hop<PREC_BF16>(const HopArgs &, int, int, int, int, int, cudaStream_t);
extern template cudaError_t launch_hop<PREC_DF>(const HopArgs &, int, int, int, int, int, cudaStream_t);

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Key of a hop launch in the tuning cache (dagger shares its configuration).
std::string hop_key(const wd_ctx *ctx, const HopArgs &A, int prec, int recon, int nrhs)
{
    const bool hx = A.x[0] != nullptr || A.x[1] != nullptr;
    char buf[160];
    snprintf(buf, sizeof(buf), "hop sm%d p%d r%d np%d x%d n%d L%dx%dx%dx%d", ctx->num_sms, prec, recon, A.nparity,
             hx ? 1 : 0, nrhs, A.L[0], A.L[1], A.L[2], A.L[3]);
    return buf;
}

// Untuned defaults, from tuning runs on GB300 (32^4, 24^3x48, 16^3x32): the
// FP32/FP16/BF16 kernels are fastest with 64-thread blocks and memory
// schedule 1; even-odd hops (each link read once) load the links without L1
// allocation, FP32 ones with schedule 0 (24^3x48: 40.1 against 43.3 us for
// schedule 1; 32^4: 62.6 against 63.8 us) and the 16-bit ones with the
// spin-paired kernel (schedule 0); the FP64 kernel (FP64-ALU bound) with 128
// threads, schedule 0.
static std::pair<int, int> hop_default(int prec, int nrhs, int nparity)
{
    if (prec == WD_DF) return {96, HOP_F64_1B_VARIANT};   // double-word: three threads per site
    if (nrhs > 1) return {128, HOP_MRHS_VARIANT};   // shared-link kernel, 4 fields at a time
    if (prec == WD_F64) return {128, 0};
    if (nparity == 1 && (prec == WD_F16 || prec == WD_BF16)) return {64, HOP_SP0_VARIANT};
    return {64, nparity == 1 ? HOP_NA0_VARIANT : 1};
}

int hop_launch_cfg(const HopArgs &A, int prec, int recon, int dagger, int nrhs, int threads, int variant,
                   cudaStream_t s)
{
    if (threads < 32 || threads > 256 || (threads & 31) || variant < 0 || variant > HOP_MAX_VARIANT)
        return set_error(WD_EINVAL, "bad hop launch configuration (%d threads, variant %d)", threads, variant);
    cudaError_t e = cudaSuccess;
    switch (prec) {
    case WD_F64: e = launch_hop<PREC_F64>(A, recon, dagger, nrhs, threads, variant, s); break;
    case WD_F32: e = launch_hop<PREC_F32>(A, recon, dagger, nrhs, threads, variant, s); break;
    case WD_F16: e = launch_hop<PREC_F16>(A, recon, dagger, nrhs, threads, variant, s); break;
    case WD_BF16: e = launch_hop<PREC_BF16>(A, recon, dagger, nrhs, threads, variant, s); break;
    case WD_DF: e = launch_hop<PREC_DF>(A, recon, dagger, nrhs, threads, variant, s); break;
    }
    if (e != cudaSuccess) return set_error(WD_ECUDA, "hop kernel launch failed: %s", cudaGetErrorString(e));
    return WD_OK;
}

int hop_launch(wd_ctx *ctx, const HopArgs &A, int prec, int recon, int dagger, int nrhs, cudaStream_t s)
{
    auto cfg = tuned_config(ctx, hop_key(ctx, A, prec, recon, nrhs), hop_default(prec, nrhs, A.nparity));
    return hop_launch_cfg(A, prec, recon, dagger, nrhs, cfg.first, cfg.second, s);
}

// Fills the geometry and gauge parts of HopArgs.
int hop_setup(const wd_gauge *g, int prec, int recon, HopArgs &A)
{
    if (!g) return set_error(WD_EINVAL, "gauge is NULL");
    if (!valid_field_prec(prec)) return set_error(WD_EINVAL, "bad precision %d", prec);
    if (!valid_recon(recon)) return set_error(WD_EINVAL, "bad reconstruction %d", recon);
    const char *base = nullptr;
    WD_TRY(gauge_layout(g, prec, recon, &base));
    const int vh = g->geo.Vh;
    A.link_blk = link_block_bytes(vh, link_prec(prec), recon);
    A.gauge[0] = base;
    A.gauge[1] = base + 4 * A.link_blk;
    for (int mu = 0; mu < 4; ++mu) A.L[mu] = g->geo.L[mu];
    A.vh = vh;
    A.tneg = g->t_sign < 0 ? 1 : 0;
    A.status = ctx_status_word(g->ctx);
    div_magic((unsigned)(A.L[0] >> 1), A.div_m[0], A.div_s[0]);
    div_magic((unsigned)A.L[1], A.div_m[1], A.div_s[1]);
    div_magic((unsigned)A.L[2], A.div_m[2], A.div_s[2]);
    return WD_OK;
}

int eo_hop(const wd_gauge *g, int prec, int recon, void *out, const void *in, const void *x, int p, double a,
           double b, int dagger, cudaStream_t s)
{
    HopArgs A{};
    WD_TRY(hop_setup(g, prec, recon, A));
    A.in[0] = A.in[1] = (const char *)in;
    A.x[0] = A.x[1] = (const char *)x;
    A.out[0] = A.out[1] = (char *)out;
    A.rhs_stride = half_field_bytes(A.vh, prec);
    A.nparity = 1;
    A.parity0 = p;
    A.a = a;
    A.b = b;
    return hop_launch(g->ctx, A, prec, recon, dagger ? 1 : 0, 1, s);
}

int full_hop(const wd_gauge *g, int prec, int recon, void *out, const void *in, double a, double b, cudaStream_t s)
{
    HopArgs A{};
    WD_TRY(hop_setup(g, prec, recon, A));
    const size_t half = half_field_bytes(A.vh, prec);
    for (int p = 0; p < 2; ++p) {
        A.in[p] = (const char *)in + (size_t)(1 - p) * half;
        A.x[p] = (const char *)in + (size_t)p * half;
        A.out[p] = (char *)out + (size_t)p * half;
    }
    A.rhs_stride = 2 * half;
    A.nparity = 2;
    A.parity0 = 0;
    A.a = a;
    A.b = b;
    return hop_launch(g->ctx, A, prec, recon, 0, 1, s);
}

} // namespace wd

using namespace wd;

extern "C" {

static int full_apply(wd_ctx *ctx, const wd_gauge *g, void *out, const void *in, double mass, int dagger, int nrhs,
                      int prec, int recon, void *stream)
{
    clear_error();
    if (!ctx) return set_error(WD_EINVAL, "ctx is NULL");
    if (!out || !in) return set_error(WD_EINVAL, "NULL field pointer");
    if (!aligned16(out) || !aligned16(in)) return set_error(WD_EINVAL, "field pointers must be 16-byte aligned");
    if (out == in) return set_error(WD_EINVAL, "out must not alias in");
    if (nrhs < 1) return set_error(WD_EINVAL, "nrhs = %d must be >= 1", nrhs);
    HopArgs A{};
    WD_TRY(hop_setup(g, prec, recon, A));
    const size_t half = half_field_bytes(A.vh, prec);
    const char *src = (const char *)in;
    char *dst = (char *)out;
    for (int p = 0; p < 2; ++p) {
        A.in[p] = src + (size_t)(1 - p) * half;
        A.x[p] = src + (size_t)p * half;
        A.out[p] = dst + (size_t)p * half;
    }
    A.rhs_stride = 2 * half;
    A.nparity = 2;
    A.parity0 = 0;
    A.a = mass + 4.0;
    A.b = -0.5;
    return hop_launch(ctx, A, prec, recon, dagger, nrhs, (cudaStream_t)stream);
}

int dslash_apply(wd_ctx *ctx, const wd_gauge *g, void *out, const void *in, double mass, int nrhs, int prec,
                 int recon, void *stream)
{
    return full_apply(ctx, g, out, in, mass, 0, nrhs, prec, recon, stream);
}

int dslash_apply_dagger(wd_ctx *ctx, const wd_gauge *g, void *out, const void *in, double mass, int nrhs, int prec,
                        int recon, void *stream)
{
    return full_apply(ctx, g, out, in, mass, 1, nrhs, prec, recon, stream);
}

int dslash_eo_apply(wd_ctx *ctx, const wd_gauge *g, void *out, const void *in, const void *x, int out_parity,
                    double a, double b, int dagger, int nrhs, int prec, int recon, void *stream)
{
    clear_error();
    if (!ctx) return set_error(WD_EINVAL, "ctx is NULL");
    if (!out || !in) return set_error(WD_EINVAL, "NULL field pointer");
    if (!aligned16(out) || !aligned16(in) || (x && !aligned16(x)))
        return set_error(WD_EINVAL, "field pointers must be 16-byte aligned");
    if (out == in) return set_error(WD_EINVAL, "out must not alias in");
    if (out_parity != WD_EVEN && out_parity != WD_ODD) return set_error(WD_EINVAL, "out_parity must be 0 or 1");
    if (nrhs < 1) return set_error(WD_EINVAL, "nrhs = %d must be >= 1", nrhs);
    HopArgs A{};
    WD_TRY(hop_setup(g, prec, recon, A));
    const int p = out_parity;
    A.in[p] = A.in[1 - p] = (const char *)in;
    A.x[p] = A.x[1 - p] = (const char *)x;
    A.out[p] = A.out[1 - p] = (char *)out;
    A.rhs_stride = half_field_bytes(A.vh, prec);
    A.nparity = 1;
    A.parity0 = p;
    A.a = a;
    A.b = b;
    return hop_launch(ctx, A, prec, recon, dagger ? 1 : 0, nrhs, (cudaStream_t)stream);
}

} // extern "C"
