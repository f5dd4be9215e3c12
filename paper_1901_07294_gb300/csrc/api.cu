// Context, errors, geometry, layout conversion (pack/unpack) and gauge objects.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "blas.cuh"
#include "launch.cuh"
#include "wd_device.cuh"
#include "wd_internal.h"

namespace wd {

static thread_local char g_err[512] = "";

int set_error(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}

void clear_error()
{
    g_err[0] = 0;
    cudaGetLastError();   // drop a runtime error left by an unrelated earlier call
}

bool valid_prec(int prec) { return prec >= WD_F64 && prec <= WD_BF16; }
bool valid_field_prec(int prec) { return valid_prec(prec) || prec == WD_DF; }
bool valid_recon(int recon) { return recon == WD_RECON_18 || recon == WD_RECON_12; }

static int storage_bytes(int prec) { return (prec == WD_F64 || prec == WD_DF) ? 8 : prec == WD_F32 ? 4 : 2; }

size_t half_field_bytes(int vh, int prec)
{
    size_t per_site = 24 * (size_t)storage_bytes(prec) + ((prec == WD_F16 || prec == WD_BF16) ? 4 : 0);
    return per_site * (size_t)vh;
}

size_t link_block_bytes(int vh, int prec, int recon)
{
    return (size_t)recon * storage_bytes(prec) * (size_t)vh;
}

int make_geometry(const int dims[4], Geometry &g)
{
    if (!dims) return set_error(WD_EINVAL, "dims is NULL");
    int64_t v = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2 || (dims[mu] & 1))
            return set_error(WD_EINVAL, "lattice extent L[%d] = %d must be even and >= 2", mu, dims[mu]);
        g.L[mu] = dims[mu];
        v *= dims[mu];
    }
    if (v / 2 >= (int64_t)1 << 31) return set_error(WD_EINVAL, "volume %lld too large (V/2 must be < 2^31)", (long long)v);
    g.V = v;
    g.Vh = (int)(v / 2);
    return WD_OK;
}

// ---- spinor pack / unpack ------------------------------------------------
struct SiteMap {
    int Lx, Ly, Lz, vh, p0, np;
    size_t half_bytes;
    // (parity slot, checkerboard index) -> lexicographic site
    __device__ __forceinline__ int64_t lex(int p, int i) const
    {
        const int lxh = Lx >> 1;
        int r = i / lxh;
        const int xh = i - r * lxh;
        const int y = r % Ly;
        const int r2 = r / Ly;
        const int z = r2 % Lz;
        const int t = r2 / Lz;
        const int bit = (p + y + z + t) & 1;
        return (int64_t)r * Lx + 2 * xh + bit;
    }
};

// Canonical spinor arrays hold 24 reals per site of type CT (double or
// float): CT2 is a complex pair, NC the site's 16-byte chunks.
template <typename CT> struct Canon;
template <> struct Canon<double> { using CT2 = double2; static constexpr int NC = 12; };
template <> struct Canon<float> { using CT2 = float2; static constexpr int NC = 6; };

template <int P, typename CT>
__global__ void pack_spinor_kernel(const CT *__restrict__ aos, char *__restrict__ field, SiteMap m)
{
    grid_dependency_enter();
    using CT2 = typename Canon<CT>::CT2;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)m.np * m.vh) return;
    const int slot = (int)(gid / m.vh);
    const int i = (int)(gid - (int64_t)slot * m.vh);
    const int64_t s = m.lex(m.p0 + slot, i);
    typename Prec<P>::real v[24];
    const CT2 *src = reinterpret_cast<const CT2 *>(aos + s * 24);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const CT2 d = src[k];
        v[2 * k] = (typename Prec<P>::real)d.x;
        v[2 * k + 1] = (typename Prec<P>::real)d.y;
    }
    Spinor<P>::store(field + slot * m.half_bytes, m.vh, i, v);
}

template <int P, typename CT>
__global__ void unpack_spinor_kernel(const char *__restrict__ field, CT *__restrict__ aos, SiteMap m)
{
    grid_dependency_enter();
    using CT2 = typename Canon<CT>::CT2;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)m.np * m.vh) return;
    const int slot = (int)(gid / m.vh);
    const int i = (int)(gid - (int64_t)slot * m.vh);
    const int64_t s = m.lex(m.p0 + slot, i);
    typename Prec<P>::real v[24];
    Spinor<P>::load(field + slot * m.half_bytes, m.vh, i, v);
    CT2 *dst = reinterpret_cast<CT2 *>(aos + s * 24);
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[k] = CT2{(CT)v[2 * k], (CT)v[2 * k + 1]};
}

// Full-lattice fields (both parities) in lexicographic order: block b takes
// sites [LEX_TILE*b, LEX_TILE*b + LEX_TILE), so the canonical array moves as
// contiguous 16-byte chunks staged in shared memory (a site's NC chunks at a
// padded stride of NC + 1, an odd number of chunks, which keeps the 16-byte
// shared accesses conflict-free), while the field side is read or written per
// site from its parity's planes.  (In checkerboard order the canonical side is
// touched at a 2-site stride, so each cache line is filled in two passes that
// lie a half field apart.)
constexpr int LEX_TILE = 128;

__device__ __forceinline__ void lex_to_cb(const SiteMap &m, int64_t s, int &p, int &i)
{
    const int64_t r = s / m.Lx;
    const int x = (int)(s - r * m.Lx);
    const int y = (int)(r % m.Ly);
    const int64_t r2 = r / m.Ly;
    const int z = (int)(r2 % m.Lz);
    const int t = (int)(r2 / m.Lz);
    p = (x + y + z + t) & 1;
    i = (int)(r * (m.Lx >> 1) + (x >> 1));
}

template <int P, typename CT>
__global__ void __launch_bounds__(LEX_TILE) pack_lex_kernel(const CT *__restrict__ aos, char *__restrict__ field,
                                                            SiteMap m, int64_t V)
{
    grid_dependency_enter();
    constexpr int NC = Canon<CT>::NC, PAD = NC + 1;
    __shared__ uint4 sh[LEX_TILE * PAD];
    const int64_t s0 = (int64_t)blockIdx.x * LEX_TILE;
    const int n = (int)min((int64_t)LEX_TILE, V - s0);
    const uint4 *src = reinterpret_cast<const uint4 *>(aos + s0 * 24);
    for (int c = threadIdx.x; c < n * NC; c += LEX_TILE) sh[(c / NC) * PAD + c % NC] = src[c];
    __syncthreads();
    if ((int)threadIdx.x >= n) return;
    int p, i;
    lex_to_cb(m, s0 + threadIdx.x, p, i);
    const CT *site = reinterpret_cast<const CT *>(&sh[threadIdx.x * PAD]);
    typename Prec<P>::real v[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = (typename Prec<P>::real)site[k];
    Spinor<P>::store(field + p * m.half_bytes, m.vh, i, v);
}

template <int P, typename CT>
__global__ void __launch_bounds__(LEX_TILE) unpack_lex_kernel(const char *__restrict__ field, CT *__restrict__ aos,
                                                              SiteMap m, int64_t V)
{
    grid_dependency_enter();
    constexpr int NC = Canon<CT>::NC, PAD = NC + 1;
    __shared__ uint4 sh[LEX_TILE * PAD];
    const int64_t s0 = (int64_t)blockIdx.x * LEX_TILE;
    const int n = (int)min((int64_t)LEX_TILE, V - s0);
    if ((int)threadIdx.x < n) {
        int p, i;
        lex_to_cb(m, s0 + threadIdx.x, p, i);
        typename Prec<P>::real v[24];
        Spinor<P>::load(field + p * m.half_bytes, m.vh, i, v);
        CT *site = reinterpret_cast<CT *>(&sh[threadIdx.x * PAD]);
#pragma unroll
        for (int k = 0; k < 24; ++k) site[k] = (CT)v[k];
    }
    __syncthreads();
    uint4 *dst = reinterpret_cast<uint4 *>(aos + s0 * 24);
    for (int c = threadIdx.x; c < n * NC; c += LEX_TILE) dst[c] = sh[(c / NC) * PAD + c % NC];
}

// ---- link pack -----------------------------------------------------------
template <int P, int RECON>
__global__ void pack_links_kernel(const double *__restrict__ links, char *__restrict__ out, SiteMap m, size_t blk)
{
    using real = typename Prec<P>::real;
    using L = Link<P, RECON>;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)2 * m.vh) return;
    const int p = (int)(gid / m.vh);
    const int i = (int)(gid - (int64_t)p * m.vh);
    const int64_t s = m.lex(p, i);
    for (int mu = 0; mu < 4; ++mu) {
        real u[18];
        const double *src = links + (s * 4 + mu) * 18;
#pragma unroll
        for (int k = 0; k < 18; ++k) u[k] = (real)src[k];
        char *b = out + (size_t)(p * 4 + mu) * blk;
#pragma unroll
        for (int k = 0; k < L::nmain; ++k) stg16(b + ((size_t)k * m.vh + i) * 16, pack16<P>(u + k * L::per16, 1.0f));
        if constexpr (L::ntail > 0) {
            char *tp = b + (size_t)L::nmain * m.vh * 16;
            const int o = L::nmain * L::per16;
            if constexpr (P == PREC_F32) {
                reinterpret_cast<float2 *>(tp)[i] = make_float2(u[o], u[o + 1]);
            } else if constexpr (P == PREC_F16) {
                __half2 h0 = __floats2half2_rn(u[o], u[o + 1]);
                if constexpr (L::ntail == 2) {
                    reinterpret_cast<__half2 *>(tp)[i] = h0;
                } else {
                    __half2 h1 = __floats2half2_rn(u[o + 2], u[o + 3]);
                    uint2 w;
                    w.x = *reinterpret_cast<unsigned *>(&h0);
                    w.y = *reinterpret_cast<unsigned *>(&h1);
                    reinterpret_cast<uint2 *>(tp)[i] = w;
                }
            } else {
                __nv_bfloat162 h0 = __floats2bfloat162_rn(u[o], u[o + 1]);
                if constexpr (L::ntail == 2) {
                    reinterpret_cast<__nv_bfloat162 *>(tp)[i] = h0;
                } else {
                    __nv_bfloat162 h1 = __floats2bfloat162_rn(u[o + 2], u[o + 3]);
                    uint2 w;
                    w.x = *reinterpret_cast<unsigned *>(&h0);
                    w.y = *reinterpret_cast<unsigned *>(&h1);
                    reinterpret_cast<uint2 *>(tp)[i] = w;
                }
            }
        }
    }
}

static int sites_to_map(const Geometry &g, int sites, int prec, SiteMap &m)
{
    m.Lx = g.L[0]; m.Ly = g.L[1]; m.Lz = g.L[2]; m.vh = g.Vh;
    m.half_bytes = half_field_bytes(g.Vh, prec);
    switch (sites) {
    case WD_SITES_FULL: m.p0 = 0; m.np = 2; break;
    case WD_SITES_EVEN: m.p0 = 0; m.np = 1; break;
    case WD_SITES_ODD: m.p0 = 1; m.np = 1; break;
    default: return set_error(WD_EINVAL, "sites = %d is not a wd_sites value", sites);
    }
    return WD_OK;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

GraphSink *&graph_sink()
{
    static thread_local GraphSink *sink = nullptr;
    return sink;
}

// Copies and clears on a private stream, so that set-up calls never
// synchronise the whole device.
static cudaError_t copy_private(void *dst, const void *src, size_t n, cudaMemcpyKind kind)
{
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(dst, src, n, kind, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    return e;
}

static bool zero_device(void *p, size_t n)
{
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return false;
    cudaError_t e = cudaMemsetAsync(p, 0, n, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    return e == cudaSuccess;
}

int ctx_workspace(wd_ctx *ctx, size_t bytes, char **out)
{
    if (ctx->work_bytes < bytes) {
        DeviceGuard dg(ctx->device);
        if (ctx->d_work) {   // solves using it are synchronous, so it is idle here
            cudaFree(ctx->d_work);
            ctx->d_work = nullptr;
            ctx->work_bytes = 0;
        }
        if (cudaMalloc(&ctx->d_work, bytes) != cudaSuccess) {
            cudaGetLastError();
            return set_error(WD_ENOMEM, "cudaMalloc of %zu bytes of solver workspace failed", bytes);
        }
        ctx->work_bytes = bytes;
    }
    *out = ctx->d_work;
    return WD_OK;
}

int ctx_aux_workspace(wd_ctx *ctx, size_t bytes, char **out)
{
    if (ctx->aux_bytes < bytes) {
        DeviceGuard dg(ctx->device);
        if (ctx->d_aux) {   // its users are synchronous, so it is idle here
            cudaFree(ctx->d_aux);
            ctx->d_aux = nullptr;
            ctx->aux_bytes = 0;
        }
        if (cudaMalloc(&ctx->d_aux, bytes) != cudaSuccess) {
            cudaGetLastError();
            return set_error(WD_ENOMEM, "cudaMalloc of %zu bytes of solver workspace failed", bytes);
        }
        ctx->aux_bytes = bytes;
    }
    *out = ctx->d_aux;
    return WD_OK;
}

int gauge_layout(const wd_gauge *gc, int prec, int recon, const char **out)
{
    wd_gauge *g = const_cast<wd_gauge *>(gc);
    if (!valid_field_prec(prec)) return set_error(WD_EINVAL, "bad precision %d", prec);
    if (!valid_recon(recon)) return set_error(WD_EINVAL, "bad reconstruction %d (use 18 or 12)", recon);
    prec = link_prec(prec);   // BF16 fields use FP16 links
    std::lock_guard<std::mutex> lk(g->mu);
    auto key = std::make_pair(prec, recon);
    auto it = g->layouts.find(key);
    if (it != g->layouts.end()) {
        *out = it->second;
        return WD_OK;
    }
    DeviceGuard dg(g->device);
    const size_t blk = link_block_bytes(g->geo.Vh, prec, recon);
    char *buf = nullptr;
    if (cudaMalloc(&buf, 8 * blk) != cudaSuccess) {
        cudaGetLastError();
        return set_error(WD_ENOMEM, "cudaMalloc of %zu bytes for a gauge layout failed", 8 * blk);
    }
    SiteMap m;
    sites_to_map(g->geo, WD_SITES_FULL, prec, m);
    const int threads = 256;
    const int blocks = (int)((2 * (int64_t)g->geo.Vh + threads - 1) / threads);
    // a private stream: no device-wide synchronisation, which would disturb
    // other threads (for example one building a graph)
    cudaStream_t ps = nullptr;
    if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(buf);
        return set_error(WD_ECUDA, "stream creation failed");
    }
#define WD_PACK_LINKS(P, R) pack_links_kernel<P, R><<<blocks, threads, 0, ps>>>(g->canonical, buf, m, blk)
    switch (prec * 100 + recon) {
    case WD_F64 * 100 + 18: WD_PACK_LINKS(PREC_F64, 18); break;
    case WD_F64 * 100 + 12: WD_PACK_LINKS(PREC_F64, 12); break;
    case WD_F32 * 100 + 18: WD_PACK_LINKS(PREC_F32, 18); break;
    case WD_F32 * 100 + 12: WD_PACK_LINKS(PREC_F32, 12); break;
    case WD_F16 * 100 + 18: WD_PACK_LINKS(PREC_F16, 18); break;
    case WD_F16 * 100 + 12: WD_PACK_LINKS(PREC_F16, 12); break;
    case WD_DF * 100 + 18: WD_PACK_LINKS(PREC_DF, 18); break;
    case WD_DF * 100 + 12: WD_PACK_LINKS(PREC_DF, 12); break;
    }
#undef WD_PACK_LINKS
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
    cudaStreamDestroy(ps);
    if (e != cudaSuccess) {
        cudaFree(buf);
        return set_error(WD_ECUDA, "link packing failed: %s", cudaGetErrorString(e));
    }
    g->layouts[key] = buf;
    *out = buf;
    return WD_OK;
}

} // namespace wd

using namespace wd;

extern "C" {

int wd_version(void) { return 100; }

const char *wd_last_error(void) { return wd::g_err; }

int wd_ctx_create(int device, wd_ctx **out)
{
    clear_error();
    if (!out) return set_error(WD_EINVAL, "out is NULL");
    *out = nullptr;
    int n = 0;
    WD_CUDA_TRY(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return set_error(WD_EINVAL, "device %d out of range (%d devices)", device, n);
    wd_ctx *c = new (std::nothrow) wd_ctx();
    if (!c) return set_error(WD_ENOMEM, "host allocation failed");
    c->device = device;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete c;
        return set_error(WD_ECUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    }
    c->num_sms = prop.multiProcessorCount;
    c->cc_major = prop.major;
    c->cc_minor = prop.minor;
    {
        DeviceGuard dg(device);
        const size_t pbytes = (size_t)MAX_RED_BLOCKS * MAX_NR * sizeof(double);
        if (cudaMalloc(&c->d_partials, pbytes) != cudaSuccess || cudaMalloc(&c->d_ticket, 256) != cudaSuccess ||
            cudaMalloc(&c->d_scal, NSCAL * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&c->h_scal, NSCAL * sizeof(double)) != cudaSuccess ||
            !zero_device(c->d_ticket, 256) || !zero_device(c->d_scal, NSCAL * sizeof(double))) {
            cudaGetLastError();
            wd_ctx_destroy(c);
            return set_error(WD_ENOMEM, "allocating the context scratch failed");
        }
    }
    load_tune_file(c);
    *out = c;
    return WD_OK;
}

int wd_ctx_destroy(wd_ctx *ctx)
{
    clear_error();
    if (!ctx) return WD_OK;
    {
        DeviceGuard dg(ctx->device);
        cudaFree(ctx->d_partials);
        cudaFree(ctx->d_ticket);
        cudaFree(ctx->d_scal);
        cudaFree(ctx->d_work);
        cudaFree(ctx->d_aux);
        if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
    }
    delete ctx;
    return WD_OK;
}

int wd_field_bytes(const int dims[4], int sites, int prec, int nrhs, size_t *out)
{
    clear_error();
    Geometry g;
    WD_TRY(make_geometry(dims, g));
    if (!valid_field_prec(prec)) return set_error(WD_EINVAL, "bad precision %d", prec);
    if (nrhs < 1) return set_error(WD_EINVAL, "nrhs = %d must be >= 1", nrhs);
    if (!out) return set_error(WD_EINVAL, "out is NULL");
    size_t half = half_field_bytes(g.Vh, prec);
    size_t one;
    switch (sites) {
    case WD_SITES_FULL: one = 2 * half; break;
    case WD_SITES_EVEN:
    case WD_SITES_ODD: one = half; break;
    default: return set_error(WD_EINVAL, "sites = %d is not a wd_sites value", sites);
    }
    *out = one * (size_t)nrhs;
    return WD_OK;
}

// The address through which this context's kernels reach the canonical
// array p: device memory of the context's GPU and managed memory as they are;
// page-locked host memory through its device mapping (the kernel then reads
// or writes host memory directly over the host link); pageable host memory
// only where the device can access it (address translation, as on Grace
// systems).  nullptr if the device cannot dereference p.
static void *device_view(const wd_ctx *ctx, const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    switch (at.type) {
    case cudaMemoryTypeDevice: return at.device == ctx->device ? const_cast<void *>(p) : nullptr;
    case cudaMemoryTypeManaged: return const_cast<void *>(p);
    case cudaMemoryTypeHost: return at.devicePointer;
    default: {
        int pageable = 0;
        if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, ctx->device) != cudaSuccess) {
            cudaGetLastError();
            pageable = 0;
        }
        return pageable ? const_cast<void *>(p) : nullptr;
    }
    }
}

static int pack_common(wd_ctx *ctx, const int dims[4], int sites, int prec, const void *a, const void *b,
                       Geometry &g, SiteMap &m)
{
    if (!ctx) return set_error(WD_EINVAL, "ctx is NULL");
    WD_TRY(make_geometry(dims, g));
    if (!valid_field_prec(prec)) return set_error(WD_EINVAL, "bad precision %d", prec);
    if (!a || !b) return set_error(WD_EINVAL, "NULL field pointer");
    if (!aligned16(a) || !aligned16(b)) return set_error(WD_EINVAL, "field pointers must be 16-byte aligned");
    return sites_to_map(g, sites, prec, m);
}

} // extern "C"

namespace wd {

template <typename CT>
static int pack_impl(wd_ctx *ctx, const int dims[4], int sites, int prec, const CT *aos, void *field, void *stream)
{
    clear_error();
    Geometry g;
    SiteMap m;
    WD_TRY(pack_common(ctx, dims, sites, prec, aos, field, g, m));
    aos = (const CT *)device_view(ctx, aos);
    if (!aos) return set_error(WD_EINVAL, "the canonical array is not accessible from the context's device");
    cudaStream_t s = (cudaStream_t)stream;
    char *f = (char *)field;
    if (m.np == 2) {
        const int64_t V = 2 * (int64_t)m.vh;
        const int blocks = (int)((V + LEX_TILE - 1) / LEX_TILE);
        switch (prec) {
        case WD_F64: wd_launch(pack_lex_kernel<PREC_F64, CT>, dim3(blocks), dim3(LEX_TILE), 0, s, aos, f, m, V); break;
        case WD_F32: wd_launch(pack_lex_kernel<PREC_F32, CT>, dim3(blocks), dim3(LEX_TILE), 0, s, aos, f, m, V); break;
        case WD_F16: wd_launch(pack_lex_kernel<PREC_F16, CT>, dim3(blocks), dim3(LEX_TILE), 0, s, aos, f, m, V); break;
        case WD_BF16: wd_launch(pack_lex_kernel<PREC_BF16, CT>, dim3(blocks), dim3(LEX_TILE), 0, s, aos, f, m, V); break;
        case WD_DF: wd_launch(pack_lex_kernel<PREC_DF, CT>, dim3(blocks), dim3(LEX_TILE), 0, s, aos, f, m, V); break;
        }
        WD_CUDA_TRY(cudaGetLastError());
        return WD_OK;
    }
    const int threads = 256;
    const int blocks = (int)(((int64_t)m.np * m.vh + threads - 1) / threads);
    switch (prec) {
    case WD_F64: wd_launch(pack_spinor_kernel<PREC_F64, CT>, dim3(blocks), dim3(threads), 0, s, aos, f, m); break;
    case WD_F32: wd_launch(pack_spinor_kernel<PREC_F32, CT>, dim3(blocks), dim3(threads), 0, s, aos, f, m); break;
    case WD_F16: wd_launch(pack_spinor_kernel<PREC_F16, CT>, dim3(blocks), dim3(threads), 0, s, aos, f, m); break;
    case WD_BF16: wd_launch(pack_spinor_kernel<PREC_BF16, CT>, dim3(blocks), dim3(threads), 0, s, aos, f, m); break;
    case WD_DF: wd_launch(pack_spinor_kernel<PREC_DF, CT>, dim3(blocks), dim3(threads), 0, s, aos, f, m); break;
    }
    WD_CUDA_TRY(cudaGetLastError());
    return WD_OK;
}

template <typename CT>
static int unpack_impl(wd_ctx *ctx, const int dims[4], int sites, int prec, const void *field, CT *aos, void *stream)
{
    clear_error();
    Geometry g;
    SiteMap m;
    WD_TRY(pack_common(ctx, dims, sites, prec, field, aos, g, m));
    aos = (CT *)device_view(ctx, aos);
    if (!aos) return set_error(WD_EINVAL, "the canonical array is not accessible from the context's device");
    cudaStream_t s = (cudaStream_t)stream;
    const char *f = (const char *)field;
    if (m.np == 2) {
        const int64_t V = 2 * (int64_t)m.vh;
        const int blocks = (int)((V + LEX_TILE - 1) / LEX_TILE);
        switch (prec) {
        case WD_F64: wd_launch(unpack_lex_kernel<PREC_F64, CT>, dim3(blocks), dim3(LEX_TILE), 0, s, f, aos, m, V); break;
        case WD_F32: wd_launch(unpack_lex_kernel<PREC_F32, CT>, dim3(blocks), dim3(LEX_TILE), 0, s, f, aos, m, V); break;
        case WD_F16: wd_launch(unpack_lex_kernel<PREC_F16, CT>, dim3(blocks), dim3(LEX_TILE), 0, s, f, aos, m, V); break;
        case WD_BF16: wd_launch(unpack_lex_kernel<PREC_BF16, CT>, dim3(blocks), dim3(LEX_TILE), 0, s, f, aos, m, V); break;
        case WD_DF: wd_launch(unpack_lex_kernel<PREC_DF, CT>, dim3(blocks), dim3(LEX_TILE), 0, s, f, aos, m, V); break;
        }
        WD_CUDA_TRY(cudaGetLastError());
        return WD_OK;
    }
    const int threads = 256;
    const int blocks = (int)(((int64_t)m.np * m.vh + threads - 1) / threads);
    switch (prec) {
    case WD_F64: wd_launch(unpack_spinor_kernel<PREC_F64, CT>, dim3(blocks), dim3(threads), 0, s, f, aos, m); break;
    case WD_F32: wd_launch(unpack_spinor_kernel<PREC_F32, CT>, dim3(blocks), dim3(threads), 0, s, f, aos, m); break;
    case WD_F16: wd_launch(unpack_spinor_kernel<PREC_F16, CT>, dim3(blocks), dim3(threads), 0, s, f, aos, m); break;
    case WD_BF16: wd_launch(unpack_spinor_kernel<PREC_BF16, CT>, dim3(blocks), dim3(threads), 0, s, f, aos, m); break;
    case WD_DF: wd_launch(unpack_spinor_kernel<PREC_DF, CT>, dim3(blocks), dim3(threads), 0, s, f, aos, m); break;
    }
    WD_CUDA_TRY(cudaGetLastError());
    return WD_OK;
}

} // namespace wd

extern "C" {

int wd_pack(wd_ctx *ctx, const int dims[4], int sites, int prec, const double *aos, void *field, void *stream)
{
    return pack_impl<double>(ctx, dims, sites, prec, aos, field, stream);
}

int wd_unpack(wd_ctx *ctx, const int dims[4], int sites, int prec, const void *field, double *aos, void *stream)
{
    return unpack_impl<double>(ctx, dims, sites, prec, field, aos, stream);
}

int wd_pack_f32(wd_ctx *ctx, const int dims[4], int sites, int prec, const float *aos, void *field, void *stream)
{
    return pack_impl<float>(ctx, dims, sites, prec, aos, field, stream);
}

int wd_unpack_f32(wd_ctx *ctx, const int dims[4], int sites, int prec, const void *field, float *aos, void *stream)
{
    return unpack_impl<float>(ctx, dims, sites, prec, field, aos, stream);
}

int wd_gauge_create(wd_ctx *ctx, const int dims[4], const double *links, int links_on_host, wd_gauge **out)
{
    clear_error();
    if (!ctx || !links || !out) return set_error(WD_EINVAL, "NULL argument");
    *out = nullptr;
    Geometry geo;
    WD_TRY(make_geometry(dims, geo));
    DeviceGuard dg(ctx->device);
    wd_gauge *g = new (std::nothrow) wd_gauge();
    if (!g) return set_error(WD_ENOMEM, "host allocation failed");
    g->ctx = ctx;
    g->device = ctx->device;
    g->geo = geo;
    const size_t nb = (size_t)geo.V * 4 * 18 * sizeof(double);
    if (cudaMalloc(&g->canonical, nb) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return set_error(WD_ENOMEM, "cudaMalloc of %zu bytes for the gauge field failed", nb);
    }
    cudaError_t e = copy_private(g->canonical, links, nb, links_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
        cudaFree(g->canonical);
        delete g;
        return set_error(WD_ECUDA, "copying the gauge field failed: %s", cudaGetErrorString(e));
    }
    *out = g;
    return WD_OK;
}

int wd_gauge_set_boundary(wd_gauge *g, int t_sign)
{
    clear_error();
    if (!g) return set_error(WD_EINVAL, "gauge is NULL");
    if (t_sign != 1 && t_sign != -1) return set_error(WD_EINVAL, "t_sign = %d must be +1 or -1", t_sign);
    g->t_sign = t_sign;
    return WD_OK;
}

int wd_gauge_prepare(wd_gauge *g, int prec, int recon)
{
    clear_error();
    if (!g) return set_error(WD_EINVAL, "gauge is NULL");
    const char *p;
    return gauge_layout(g, prec, recon, &p);
}

int wd_gauge_bytes(const wd_gauge *g, int prec, int recon, size_t *out)
{
    clear_error();
    if (!g || !out) return set_error(WD_EINVAL, "NULL argument");
    if (!valid_field_prec(prec) || !valid_recon(recon)) return set_error(WD_EINVAL, "bad precision or reconstruction");
    *out = 8 * link_block_bytes(g->geo.Vh, link_prec(prec), recon);
    return WD_OK;
}

int wd_gauge_destroy(wd_gauge *g)
{
    clear_error();
    if (!g) return WD_OK;
    DeviceGuard dg(g->device);
    for (auto &kv : g->layouts) cudaFree(kv.second);
    cudaFree(g->canonical);
    delete g;
    return WD_OK;
}

} // extern "C"
