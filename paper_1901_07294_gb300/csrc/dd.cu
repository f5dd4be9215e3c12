// Domain decomposition of the lattice along t with a halo exchange.
//
// Sec. II-A parallelises the hopping term by decomposing the lattice into
// sub-lattices, one per process, each exchanging its boundary with its
// neighbours; Sec. V keeps 16-bit floats only for compressing that exchanged
// data.  Here the sub-lattices are slabs of L_t / nsub time slices.  Each has
// its own gauge object (its slice of the links: with t slowest in the
// canonical order, slab k is a contiguous range) and its own fields, exactly
// as one process per slab would hold them.  This library keeps all slabs on
// one GPU: the exchange is a device-to-device copy into the receiver's own
// halo buffer, the step a multi-GPU build does with NCCL send/recv.
//
// One application of D = (m+4) - H/2 on all slabs:
//   side stream: gather the two faces of every slab into its send buffers
//     forward face (sites at local t = 0): h = (1 - gamma_t) psi projected to
//       12 reals, for the lower neighbour's forward hop (it owns the link);
//     backward face (sites at local t = T-1): w = U_t(x)^dagger (1 + gamma_t) psi
//       projected and multiplied by the sender's own link, for the upper
//       neighbour's backward hop;
//   then copy send buffers into the neighbours' halo buffers;
//   caller stream, concurrently: the interior pass, the ordinary hop kernel
//     with the t boundary open (hops across it are skipped);
//   caller stream, after both: the boundary pass adds b * (reconstructed halo
//     term) at the sites of local t = T-1 (forward hop: U_t(x) h with the
//     receiver's link) and t = 0 (backward hop: w as received).
// Halos are FP64, FP32 or FP16 with a per-site scale (12 reals per face site).
// Antiperiodic t: the sign is applied to the faces that cross the global
// boundary (slab 0's forward face, slab nsub-1's backward face).
#include <cstdint>
#include <new>
#include <vector>

#include <cuda_fp16.h>

#include "dslash_launch.cuh"
#include "wd_internal.h"

namespace wd {

int hop_setup(const wd_gauge *g, int prec, int recon, HopArgs &A);
int hop_launch(wd_ctx *ctx, const HopArgs &A, int prec, int recon, int dagger, int nrhs, cudaStream_t s);

namespace {

// ---- halo storage: 12 reals per face site, plane-major ---------------------
template <int HP> struct Halo;
template <> struct Halo<PREC_F64> {   // 6 planes of double2
    static size_t bytes(int nf) { return (size_t)nf * 96; }
    template <typename T> __device__ static void store(char *b, int nf, int j, const T (&v)[12])
    {
#pragma unroll
        for (int k = 0; k < 6; ++k)
            reinterpret_cast<double2 *>(b)[(size_t)k * nf + j] = make_double2((double)v[2 * k], (double)v[2 * k + 1]);
    }
    template <typename T> __device__ static void load(const char *b, int nf, int j, T (&v)[12])
    {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double2 d = reinterpret_cast<const double2 *>(b)[(size_t)k * nf + j];
            v[2 * k] = (T)d.x;
            v[2 * k + 1] = (T)d.y;
        }
    }
};
template <> struct Halo<PREC_F32> {   // 3 planes of float4
    static size_t bytes(int nf) { return (size_t)nf * 48; }
    template <typename T> __device__ static void store(char *b, int nf, int j, const T (&v)[12])
    {
#pragma unroll
        for (int k = 0; k < 3; ++k)
            reinterpret_cast<float4 *>(b)[(size_t)k * nf + j] =
                make_float4((float)v[4 * k], (float)v[4 * k + 1], (float)v[4 * k + 2], (float)v[4 * k + 3]);
    }
    template <typename T> __device__ static void load(const char *b, int nf, int j, T (&v)[12])
    {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 f = reinterpret_cast<const float4 *>(b)[(size_t)k * nf + j];
            v[4 * k] = (T)f.x;
            v[4 * k + 1] = (T)f.y;
            v[4 * k + 2] = (T)f.z;
            v[4 * k + 3] = (T)f.w;
        }
    }
};
template <> struct Halo<PREC_F16> {   // 3 planes of 4 halves (8 B) + an FP32 scale plane
    static size_t bytes(int nf) { return (size_t)nf * 28; }
    template <typename T> __device__ static void store(char *b, int nf, int j, const T (&v)[12])
    {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmaxf(m, fabsf((float)v[k]));
        const float inv = m > 0.f ? 1.0f / m : 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            __half2 lo = __floats2half2_rn((float)v[4 * k] * inv, (float)v[4 * k + 1] * inv);
            __half2 hi = __floats2half2_rn((float)v[4 * k + 2] * inv, (float)v[4 * k + 3] * inv);
            uint2 w;
            w.x = *reinterpret_cast<unsigned *>(&lo);
            w.y = *reinterpret_cast<unsigned *>(&hi);
            reinterpret_cast<uint2 *>(b)[(size_t)k * nf + j] = w;
        }
        reinterpret_cast<float *>(b + (size_t)nf * 24)[j] = m;
    }
    template <typename T> __device__ static void load(const char *b, int nf, int j, T (&v)[12])
    {
        const float m = reinterpret_cast<const float *>(b + (size_t)nf * 24)[j];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint2 w = reinterpret_cast<const uint2 *>(b)[(size_t)k * nf + j];
            const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&w.x));
            const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&w.y));
            v[4 * k] = (T)(lo.x * m);
            v[4 * k + 1] = (T)(lo.y * m);
            v[4 * k + 2] = (T)(hi.x * m);
            v[4 * k + 3] = (T)(hi.y * m);
        }
    }
};

// bytes of one (parity) face buffer, rounded for alignment
size_t face_bytes(int hp, int nf)
{
    const size_t b = hp == WD_F64 ? Halo<PREC_F64>::bytes(nf) : hp == WD_F32 ? Halo<PREC_F32>::bytes(nf)
                                                                             : Halo<PREC_F16>::bytes(nf);
    return (b + 255) & ~size_t(255);
}

struct FaceArgs {
    const char *field;     // local full field (parity 0 half, then parity 1)
    size_t half_bytes;
    const char *gauge[2];  // local links per parity (4 mu blocks of link_blk)
    size_t link_blk;
    char *buf[2];          // send (gather) or halo (boundary pass) buffers for faces [fwd, bwd], both parities
    char *out;             // boundary pass: local full output field
    size_t face_bytes;     // one parity's face buffer
    int vh, nf, lt;
    int neg_f, neg_b;      // gather: the face crosses the global antiperiodic boundary
    double b;              // boundary pass: coefficient of the hopping term
};

template <typename T> __device__ __forceinline__ void neg12(cpx<T> (&w0)[3], cpx<T> (&w1)[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        w0[c].re = -w0[c].re; w0[c].im = -w0[c].im;
        w1[c].re = -w1[c].re; w1[c].im = -w1[c].im;
    }
}

template <typename T> __device__ __forceinline__ void to12(const cpx<T> (&a)[3], const cpx<T> (&b)[3], T (&v)[12])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[2 * c] = a[c].re; v[2 * c + 1] = a[c].im;
        v[6 + 2 * c] = b[c].re; v[7 + 2 * c] = b[c].im;
    }
}

template <typename T> __device__ __forceinline__ void from12(const T (&v)[12], cpx<T> (&a)[3], cpx<T> (&b)[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a[c] = {v[2 * c], v[2 * c + 1]};
        b[c] = {v[6 + 2 * c], v[7 + 2 * c]};
    }
}

// Gather both faces of one slab: thread g < 2 nf takes face index j of parity s
// (the parity of the sending site).
template <int P, int HP, int RECON>
__global__ void __launch_bounds__(128) dd_gather_kernel(const FaceArgs A)
{
    grid_dependency_enter();
    using T = typename Prec<P>::real;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 2 * A.nf) return;
    const int s = g >= A.nf ? 1 : 0;
    const int j = g - s * A.nf;
    const char *f = A.field + (size_t)s * A.half_bytes;
    T psi[24];
    cpx<T> h0[3], h1[3];
    T v[12];
    // forward face: site at t = 0, projector of the forward hop (1 - gamma_t)
    Spinor<P>::load(f, A.vh, j, psi);
    project<3, -1>(psi, h0, h1);
    if (A.neg_f) neg12(h0, h1);
    to12(h0, h1, v);
    Halo<HP>::store(A.buf[0] + (size_t)s * A.face_bytes, A.nf, j, v);
    // backward face: site at t = T-1, (1 + gamma_t) projected, times its own U_t^dagger
    const int i1 = j + (A.lt - 1) * A.nf;
    Spinor<P>::load(f, A.vh, i1, psi);
    project<3, +1>(psi, h0, h1);
    cpx<T> U[3][3];
    Link<link_prec(P), RECON>::load(A.gauge[s] + 3 * A.link_blk, A.vh, i1, U);
    cpx<T> w0[3], w1[3];
    su3_mul<false>(U, h0, w0);
    su3_mul<false>(U, h1, w1);
    if (A.neg_b) neg12(w0, w1);
    to12(w0, w1, v);
    Halo<HP>::store(A.buf[1] + (size_t)s * A.face_bytes, A.nf, j, v);
}

// Boundary pass of one slab: thread g < 2 nf takes face index j of parity p
// (the receiving site); the sender had parity 1 - p.
template <int P, int HP, int RECON>
__global__ void __launch_bounds__(128) dd_boundary_kernel(const FaceArgs A)
{
    grid_dependency_enter();
    using T = typename Prec<P>::real;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 2 * A.nf) return;
    const int p = g >= A.nf ? 1 : 0;
    const int j = g - p * A.nf;
    char *o = A.out + (size_t)p * A.half_bytes;
    const T b = (T)A.b;
    T v[12];
    cpx<T> h0[3], h1[3], w0[3], w1[3];
    // site at t = T-1: forward hop with the received h and this slab's U_t(x)
    {
        const int i1 = j + (A.lt - 1) * A.nf;
        Halo<HP>::load(A.buf[0] + (size_t)(1 - p) * A.face_bytes, A.nf, j, v);
        from12(v, h0, h1);
        cpx<T> U[3][3];
        Link<link_prec(P), RECON>::load(A.gauge[p] + 3 * A.link_blk, A.vh, i1, U);
        su3_mul<true>(U, h0, w0);
        su3_mul<true>(U, h1, w1);
        cpx<T> acc[4][3];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[sp][c] = {T(0), T(0)};
        accumulate<3, -1>(acc, w0, w1);
        T out[24];
        Spinor<P>::load(o, A.vh, i1, out);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                out[6 * sp + 2 * c] += b * acc[sp][c].re;
                out[6 * sp + 2 * c + 1] += b * acc[sp][c].im;
            }
        Spinor<P>::store(o, A.vh, i1, out);
    }
    // site at t = 0: backward hop, already multiplied by the sender's link
    {
        Halo<HP>::load(A.buf[1] + (size_t)(1 - p) * A.face_bytes, A.nf, j, v);
        from12(v, w0, w1);
        cpx<T> acc[4][3];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[sp][c] = {T(0), T(0)};
        accumulate<3, +1>(acc, w0, w1);
        T out[24];
        Spinor<P>::load(o, A.vh, j, out);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                out[6 * sp + 2 * c] += b * acc[sp][c].re;
                out[6 * sp + 2 * c + 1] += b * acc[sp][c].im;
            }
        Spinor<P>::store(o, A.vh, j, out);
    }
}

template <int P, int HP>
cudaError_t launch_faces(bool gather, int recon, const FaceArgs &A, cudaStream_t s)
{
    const int threads = 128;
    const int blocks = (2 * A.nf + threads - 1) / threads;
    if (gather) {
        if (recon == 12) wd_launch(dd_gather_kernel<P, HP, 12>, dim3(blocks), dim3(threads), 0, s, A);
        else wd_launch(dd_gather_kernel<P, HP, 18>, dim3(blocks), dim3(threads), 0, s, A);
    } else {
        if (recon == 12) wd_launch(dd_boundary_kernel<P, HP, 12>, dim3(blocks), dim3(threads), 0, s, A);
        else wd_launch(dd_boundary_kernel<P, HP, 18>, dim3(blocks), dim3(threads), 0, s, A);
    }
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_faces_p(bool gather, int recon, int hp, const FaceArgs &A, cudaStream_t s)
{
    switch (hp) {
    case WD_F64: return launch_faces<P, PREC_F64>(gather, recon, A, s);
    case WD_F32: return launch_faces<P, PREC_F32>(gather, recon, A, s);
    default: return launch_faces<P, PREC_F16>(gather, recon, A, s);
    }
}

cudaError_t launch_face_kernels(bool gather, int prec, int recon, int hp, const FaceArgs &A, cudaStream_t s)
{
    switch (prec) {
    case WD_F64: return launch_faces_p<PREC_F64>(gather, recon, hp, A, s);
    case WD_F32: return launch_faces_p<PREC_F32>(gather, recon, hp, A, s);
    case WD_F16: return launch_faces_p<PREC_F16>(gather, recon, hp, A, s);
    default: return launch_faces_p<PREC_BF16>(gather, recon, hp, A, s);
    }
}

} // namespace

} // namespace wd

struct wd_dd {
    wd_ctx *ctx = nullptr;
    int device = 0;
    int nsub = 0;
    int Lg[4] = {0, 0, 0, 0}, Ll[4] = {0, 0, 0, 0};
    int nf = 0, vh = 0;   // face sites per parity, local half volume
    int t_sign = 1;
    std::vector<wd_gauge *> sub;
    char *buf = nullptr;   // [send | halo] x nsub x [fwd | bwd] x 2 parities, F64-sized faces
    size_t slot = 0;       // bytes of one (slab, direction) pair of parity buffers at F64 size
    cudaStream_t side = nullptr;
    cudaEvent_t ev_in = nullptr, ev_halo = nullptr;
};

using namespace wd;

namespace {

char *dd_slot(wd_dd *d, int which, int k, int dir)   // which: 0 send, 1 halo
{
    return d->buf + ((size_t)(which * d->nsub + k) * 2 + dir) * d->slot;
}

void dd_free(wd_dd *d)
{
    DeviceGuard dg(d->device);
    for (wd_gauge *g : d->sub)
        if (g) wd_gauge_destroy(g);
    cudaFree(d->buf);
    if (d->side) cudaStreamDestroy(d->side);
    if (d->ev_in) cudaEventDestroy(d->ev_in);
    if (d->ev_halo) cudaEventDestroy(d->ev_halo);
    delete d;
}

} // namespace

extern "C" {

int wd_dd_create(wd_ctx *ctx, const int dims[4], int nsub, const double *links, int links_on_host, wd_dd **out)
{
    clear_error();
    if (!ctx || !dims || !links || !out) return set_error(WD_EINVAL, "NULL argument");
    *out = nullptr;
    Geometry geo;
    WD_TRY(make_geometry(dims, geo));
    if (nsub < 1 || dims[3] % nsub != 0)
        return set_error(WD_EINVAL, "nsub = %d must divide L_t = %d", nsub, dims[3]);
    const int lt = dims[3] / nsub;
    if (lt < 2 || (lt & 1)) return set_error(WD_EINVAL, "local L_t = %d must be even and >= 2", lt);
    DeviceGuard dg(ctx->device);
    wd_dd *d = new (std::nothrow) wd_dd();
    if (!d) return set_error(WD_ENOMEM, "host allocation failed");
    d->ctx = ctx;
    d->device = ctx->device;
    d->nsub = nsub;
    for (int mu = 0; mu < 4; ++mu) d->Lg[mu] = d->Ll[mu] = dims[mu];
    d->Ll[3] = lt;
    d->nf = dims[0] * dims[1] * dims[2] / 2;
    d->vh = d->nf * lt;
    const size_t vloc = (size_t)dims[0] * dims[1] * dims[2] * lt;
    for (int k = 0; k < nsub; ++k) {
        wd_gauge *g = nullptr;
        const int rc = wd_gauge_create(ctx, d->Ll, links + (size_t)k * vloc * 72, links_on_host, &g);
        if (rc != WD_OK) {
            dd_free(d);
            return rc;
        }
        d->sub.push_back(g);
    }
    d->slot = 2 * face_bytes(WD_F64, d->nf);
    if (cudaMalloc(&d->buf, (size_t)2 * nsub * 2 * d->slot) != cudaSuccess ||
        cudaStreamCreateWithFlags(&d->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&d->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&d->ev_halo, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        dd_free(d);
        return set_error(WD_ENOMEM, "allocation of the halo buffers failed");
    }
    *out = d;
    return WD_OK;
}

int wd_dd_destroy(wd_dd *d)
{
    clear_error();
    if (!d) return WD_OK;
    dd_free(d);
    return WD_OK;
}

int wd_dd_local_dims(const wd_dd *d, int dims_out[4])
{
    clear_error();
    if (!d || !dims_out) return set_error(WD_EINVAL, "NULL argument");
    for (int mu = 0; mu < 4; ++mu) dims_out[mu] = d->Ll[mu];
    return WD_OK;
}

int wd_dd_set_boundary(wd_dd *d, int t_sign)
{
    clear_error();
    if (!d) return set_error(WD_EINVAL, "NULL argument");
    if (t_sign != 1 && t_sign != -1) return set_error(WD_EINVAL, "t_sign = %d must be +1 or -1", t_sign);
    d->t_sign = t_sign;
    return WD_OK;
}

int wd_dd_halo_bytes(const wd_dd *d, int halo_prec, size_t *out)
{
    clear_error();
    if (!d || !out) return set_error(WD_EINVAL, "NULL argument");
    if (halo_prec != WD_F64 && halo_prec != WD_F32 && halo_prec != WD_F16)
        return set_error(WD_EINVAL, "halo precision must be WD_F64, WD_F32 or WD_F16");
    const size_t per = halo_prec == WD_F64 ? 96 : halo_prec == WD_F32 ? 48 : 28;
    *out = (size_t)d->nsub * 2 * 2 * d->nf * per;
    return WD_OK;
}

int wd_dd_dslash(wd_dd *d, void *const *out, const void *const *in, double mass, int prec, int recon, int halo_prec,
                 void *stream)
{
    clear_error();
    if (!d || !out || !in) return set_error(WD_EINVAL, "NULL argument");
    if (!valid_prec(prec)) return set_error(WD_EINVAL, "bad precision %d", prec);
    if (!valid_recon(recon)) return set_error(WD_EINVAL, "bad reconstruction %d", recon);
    if (halo_prec != WD_F64 && halo_prec != WD_F32 && halo_prec != WD_F16)
        return set_error(WD_EINVAL, "halo precision must be WD_F64, WD_F32 or WD_F16");
    for (int k = 0; k < d->nsub; ++k) {
        if (!out[k] || !in[k]) return set_error(WD_EINVAL, "NULL field pointer for slab %d", k);
        if (((uintptr_t)out[k] | (uintptr_t)in[k]) & 15u) return set_error(WD_EINVAL, "fields must be 16-byte aligned");
        if (out[k] == in[k]) return set_error(WD_EINVAL, "out must not alias in");
    }
    DeviceGuard dg(d->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int n = d->nsub;
    const size_t half = half_field_bytes(d->vh, prec);
    const size_t fb = face_bytes(halo_prec, d->nf);
    std::vector<HopArgs> H(n);
    std::vector<FaceArgs> F(n);
    for (int k = 0; k < n; ++k) {
        HopArgs &A = H[k];
        A = HopArgs{};
        WD_TRY(hop_setup(d->sub[k], prec, recon, A));
        const char *src = (const char *)in[k];
        char *dst = (char *)out[k];
        for (int p = 0; p < 2; ++p) {
            A.in[p] = src + (size_t)(1 - p) * half;
            A.x[p] = src + (size_t)p * half;
            A.out[p] = dst + (size_t)p * half;
        }
        A.rhs_stride = 2 * half;
        A.nparity = 2;
        A.parity0 = 0;
        A.topen = 1;
        A.a = mass + 4.0;
        A.b = -0.5;
        FaceArgs &f = F[k];
        f = FaceArgs{};
        f.field = src;
        f.out = dst;
        f.half_bytes = half;
        f.gauge[0] = A.gauge[0];
        f.gauge[1] = A.gauge[1];
        f.link_blk = A.link_blk;
        f.face_bytes = fb;
        f.vh = d->vh;
        f.nf = d->nf;
        f.lt = d->Ll[3];
        f.b = -0.5;
    }
    // faces and exchange on the side stream, after whatever the caller queued before
    WD_CUDA_TRY(cudaEventRecord(d->ev_in, s));
    WD_CUDA_TRY(cudaStreamWaitEvent(d->side, d->ev_in, 0));
    for (int k = 0; k < n; ++k) {
        FaceArgs g = F[k];
        g.buf[0] = dd_slot(d, 0, k, 0);
        g.buf[1] = dd_slot(d, 0, k, 1);
        g.neg_f = (d->t_sign < 0 && k == 0) ? 1 : 0;
        g.neg_b = (d->t_sign < 0 && k == n - 1) ? 1 : 0;
        cudaError_t e = launch_face_kernels(true, prec, recon, halo_prec, g, d->side);
        if (e != cudaSuccess) return set_error(WD_ECUDA, "face gather launch failed: %s", cudaGetErrorString(e));
    }
    for (int k = 0; k < n; ++k) {
        // slab k's forward face goes to slab k-1, its backward face to slab k+1
        WD_CUDA_TRY(cudaMemcpyAsync(dd_slot(d, 1, (k + n - 1) % n, 0), dd_slot(d, 0, k, 0), 2 * fb,
                                    cudaMemcpyDeviceToDevice, d->side));
        WD_CUDA_TRY(cudaMemcpyAsync(dd_slot(d, 1, (k + 1) % n, 1), dd_slot(d, 0, k, 1), 2 * fb,
                                    cudaMemcpyDeviceToDevice, d->side));
    }
    WD_CUDA_TRY(cudaEventRecord(d->ev_halo, d->side));
    // interior passes on the caller's stream, overlapping the exchange
    for (int k = 0; k < n; ++k) WD_TRY(hop_launch(d->ctx, H[k], prec, recon, 0, 1, s));
    WD_CUDA_TRY(cudaStreamWaitEvent(s, d->ev_halo, 0));
    for (int k = 0; k < n; ++k) {
        FaceArgs g = F[k];
        g.buf[0] = dd_slot(d, 1, k, 0);
        g.buf[1] = dd_slot(d, 1, k, 1);
        cudaError_t e = launch_face_kernels(false, prec, recon, halo_prec, g, s);
        if (e != cudaSuccess) return set_error(WD_ECUDA, "boundary pass launch failed: %s", cudaGetErrorString(e));
    }
    return WD_OK;
}

} // extern "C"

// ---- one slab per process --------------------------------------------------
// The same three steps for a lattice whose slabs live in different processes
// (Sec. II-A: one sub-lattice per process): each process holds one wd_slab
// and its own fields, gathers its two faces into buffers it owns, sends them
// to its neighbours by whatever transport it uses (NCCL send/recv into the
// receiver's own buffers), runs the interior pass meanwhile and adds the
// received halos in the boundary pass.
struct wd_slab {
    wd_ctx *ctx = nullptr;
    int device = 0;
    int nsub = 0, k = 0;
    int Ll[4] = {0, 0, 0, 0};
    int nf = 0, vh = 0;
    int t_sign = 1;
    wd_gauge *g = nullptr;
};

namespace {

int slab_face_args(const wd_slab *sl, const void *field, void *out, int prec, int recon, int halo_prec, FaceArgs &f,
                   HopArgs &A)
{
    A = HopArgs{};
    WD_TRY(hop_setup(sl->g, prec, recon, A));
    f = FaceArgs{};
    f.field = (const char *)field;
    f.out = (char *)out;
    f.half_bytes = half_field_bytes(sl->vh, prec);
    f.gauge[0] = A.gauge[0];
    f.gauge[1] = A.gauge[1];
    f.link_blk = A.link_blk;
    f.face_bytes = face_bytes(halo_prec, sl->nf);
    f.vh = sl->vh;
    f.nf = sl->nf;
    f.lt = sl->Ll[3];
    f.b = -0.5;
    return WD_OK;
}

int slab_check(const wd_slab *sl, int prec, int recon, int halo_prec)
{
    if (!sl) return set_error(WD_EINVAL, "NULL slab");
    if (!valid_prec(prec)) return set_error(WD_EINVAL, "bad precision %d", prec);
    if (!valid_recon(recon)) return set_error(WD_EINVAL, "bad reconstruction %d", recon);
    if (halo_prec != WD_F64 && halo_prec != WD_F32 && halo_prec != WD_F16)
        return set_error(WD_EINVAL, "halo precision must be WD_F64, WD_F32 or WD_F16");
    return WD_OK;
}

bool misaligned(const void *p) { return ((uintptr_t)p & 15u) != 0; }

} // namespace

extern "C" {

int wd_slab_create(wd_ctx *ctx, const int dims[4], int nsub, int k, const double *links, int links_on_host,
                   wd_slab **out)
{
    clear_error();
    if (!ctx || !dims || !links || !out) return set_error(WD_EINVAL, "NULL argument");
    *out = nullptr;
    Geometry geo;
    WD_TRY(make_geometry(dims, geo));
    if (nsub < 1 || dims[3] % nsub != 0)
        return set_error(WD_EINVAL, "nsub = %d must divide L_t = %d", nsub, dims[3]);
    if (k < 0 || k >= nsub) return set_error(WD_EINVAL, "slab index %d out of range [0, %d)", k, nsub);
    const int lt = dims[3] / nsub;
    if (lt < 2 || (lt & 1)) return set_error(WD_EINVAL, "local L_t = %d must be even and >= 2", lt);
    DeviceGuard dg(ctx->device);
    wd_slab *sl = new (std::nothrow) wd_slab();
    if (!sl) return set_error(WD_ENOMEM, "host allocation failed");
    sl->ctx = ctx;
    sl->device = ctx->device;
    sl->nsub = nsub;
    sl->k = k;
    for (int mu = 0; mu < 4; ++mu) sl->Ll[mu] = dims[mu];
    sl->Ll[3] = lt;
    sl->nf = dims[0] * dims[1] * dims[2] / 2;
    sl->vh = sl->nf * lt;
    const int rc = wd_gauge_create(ctx, sl->Ll, links, links_on_host, &sl->g);
    if (rc != WD_OK) {
        delete sl;
        return rc;
    }
    *out = sl;
    return WD_OK;
}

int wd_slab_destroy(wd_slab *sl)
{
    clear_error();
    if (!sl) return WD_OK;
    {
        DeviceGuard dg(sl->device);
        if (sl->g) wd_gauge_destroy(sl->g);
    }
    delete sl;
    return WD_OK;
}

int wd_slab_local_dims(const wd_slab *sl, int dims_out[4])
{
    clear_error();
    if (!sl || !dims_out) return set_error(WD_EINVAL, "NULL argument");
    for (int mu = 0; mu < 4; ++mu) dims_out[mu] = sl->Ll[mu];
    return WD_OK;
}

int wd_slab_set_boundary(wd_slab *sl, int t_sign)
{
    clear_error();
    if (!sl) return set_error(WD_EINVAL, "NULL argument");
    if (t_sign != 1 && t_sign != -1) return set_error(WD_EINVAL, "t_sign = %d must be +1 or -1", t_sign);
    sl->t_sign = t_sign;
    return WD_OK;
}

int wd_slab_face_bytes(const wd_slab *sl, int halo_prec, size_t *out)
{
    clear_error();
    if (!sl || !out) return set_error(WD_EINVAL, "NULL argument");
    if (halo_prec != WD_F64 && halo_prec != WD_F32 && halo_prec != WD_F16)
        return set_error(WD_EINVAL, "halo precision must be WD_F64, WD_F32 or WD_F16");
    *out = 2 * face_bytes(halo_prec, sl->nf);
    return WD_OK;
}

int wd_slab_gather(wd_slab *sl, const void *in, int prec, int recon, int halo_prec, void *send_fwd, void *send_bwd,
                   void *stream)
{
    clear_error();
    WD_TRY(slab_check(sl, prec, recon, halo_prec));
    if (!in || !send_fwd || !send_bwd) return set_error(WD_EINVAL, "NULL argument");
    if (misaligned(in) || misaligned(send_fwd) || misaligned(send_bwd))
        return set_error(WD_EINVAL, "fields and face buffers must be 16-byte aligned");
    DeviceGuard dg(sl->device);
    FaceArgs f;
    HopArgs A;
    WD_TRY(slab_face_args(sl, in, nullptr, prec, recon, halo_prec, f, A));
    f.buf[0] = (char *)send_fwd;
    f.buf[1] = (char *)send_bwd;
    f.neg_f = (sl->t_sign < 0 && sl->k == 0) ? 1 : 0;
    f.neg_b = (sl->t_sign < 0 && sl->k == sl->nsub - 1) ? 1 : 0;
    cudaError_t e = launch_face_kernels(true, prec, recon, halo_prec, f, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(WD_ECUDA, "face gather launch failed: %s", cudaGetErrorString(e));
    return WD_OK;
}

int wd_slab_interior(wd_slab *sl, void *out, const void *in, double mass, int prec, int recon, void *stream)
{
    clear_error();
    WD_TRY(slab_check(sl, prec, recon, WD_F64));
    if (!in || !out) return set_error(WD_EINVAL, "NULL argument");
    if (misaligned(in) || misaligned(out)) return set_error(WD_EINVAL, "fields must be 16-byte aligned");
    if (in == out) return set_error(WD_EINVAL, "out must not alias in");
    DeviceGuard dg(sl->device);
    HopArgs A{};
    WD_TRY(hop_setup(sl->g, prec, recon, A));
    const size_t half = half_field_bytes(sl->vh, prec);
    for (int p = 0; p < 2; ++p) {
        A.in[p] = (const char *)in + (size_t)(1 - p) * half;
        A.x[p] = (const char *)in + (size_t)p * half;
        A.out[p] = (char *)out + (size_t)p * half;
    }
    A.rhs_stride = 2 * half;
    A.nparity = 2;
    A.topen = 1;
    A.a = mass + 4.0;
    A.b = -0.5;
    return hop_launch(sl->ctx, A, prec, recon, 0, 1, (cudaStream_t)stream);
}

int wd_slab_boundary(wd_slab *sl, void *out, const void *recv_fwd, const void *recv_bwd, int prec, int recon,
                     int halo_prec, void *stream)
{
    clear_error();
    WD_TRY(slab_check(sl, prec, recon, halo_prec));
    if (!out || !recv_fwd || !recv_bwd) return set_error(WD_EINVAL, "NULL argument");
    if (misaligned(out) || misaligned(recv_fwd) || misaligned(recv_bwd))
        return set_error(WD_EINVAL, "fields and face buffers must be 16-byte aligned");
    DeviceGuard dg(sl->device);
    FaceArgs f;
    HopArgs A;
    WD_TRY(slab_face_args(sl, nullptr, out, prec, recon, halo_prec, f, A));
    f.buf[0] = (char *)recv_fwd;
    f.buf[1] = (char *)recv_bwd;
    cudaError_t e = launch_face_kernels(false, prec, recon, halo_prec, f, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(WD_ECUDA, "boundary pass launch failed: %s", cudaGetErrorString(e));
    return WD_OK;
}

} // extern "C"
