// |x|^2 of a device field without allocating anything.
//
// wd_norm2 keeps its partial sums in scratch that wd_ctx_create allocates.
// Some callers cannot do that: plug-ins whose host framework owns all device
// memory through a pooling allocator and forbids raw cudaMalloc, and
// latency-critical loops that cannot afford cudaMalloc's implicit device
// synchronisation.  For them, wd_norm2_noalloc runs the same reduction kernel
// with its scratch in the fixed array below, which every GPU that loads this
// library holds until the process exits.
#include <mutex>

#include "blas.cuh"
#include "wd_internal.h"

namespace wd {
namespace {

// One partial sum per block of BLAS_THREADS sites, plus 256 bytes for the
// ticket counter of the last-block reduction.
constexpr int NOALLOC_MAX_BLOCKS = 8192;   // => at most 8192 * 256 = 2,097,152 sites
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_BLOCKS + 32];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
// Per device: the scratch array's device address and the unique ID of the CUDA
// context it was looked up in.  A device reset destroys that context (and the
// module holding the array); the next call sees a new ID and looks it up again.
double *g_noalloc_addr[NOALLOC_MAX_DEVICES];
unsigned long long g_noalloc_ctx_id[NOALLOC_MAX_DEVICES];

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current;
CtxGetIdFn g_ctx_get_id;

// The unique ID of the current thread's CUDA context (driver entry points found
// through the runtime, so the library needs no link against libcuda).
int current_ctx_id(unsigned long long *id)
{
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return set_error(WD_ECUDA, "driver entry points cuCtxGetCurrent/cuCtxGetId not found");
        g_ctx_get_current = (CtxGetCurrentFn)f1;
        g_ctx_get_id = (CtxGetIdFn)f2;
    }
    void *c = nullptr;
    if (g_ctx_get_current(&c) != 0 || !c) return set_error(WD_ECUDA, "no current CUDA context");
    if (g_ctx_get_id(c, id) != 0) return set_error(WD_ECUDA, "cuCtxGetId failed");
    return WD_OK;
}

// Device address of the scratch array on device `dev` (which must be the
// current device); looked up once per device and context.  In host code the
// array's name is only a host-side stand-in, so the kernel must be given this
// address.
int noalloc_scratch(int dev, double **out)
{
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return set_error(WD_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    unsigned long long id = 0;
    if (!g_noalloc_addr[dev] || current_ctx_id(&id) != WD_OK || id != g_noalloc_ctx_id[dev]) {
        void *p = nullptr;
        // also makes the device's primary context current if it is not yet
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return set_error(WD_ECUDA, "cudaGetSymbolAddress of the fixed scratch failed: %s", cudaGetErrorString(e));
        WD_TRY(current_ctx_id(&id));
        g_noalloc_addr[dev] = (double *)p;
        g_noalloc_ctx_id[dev] = id;
    }
    *out = g_noalloc_addr[dev];
    return WD_OK;
}

template <int P> int noalloc_norm2(const void *x, int vh, int nsite, double *result, cudaStream_t s)
{
    int dev = -1;
    WD_CUDA_TRY(cudaGetDevice(&dev));
    double *scratch = nullptr;
    WD_TRY(noalloc_scratch(dev, &scratch));
    unsigned *ticket = reinterpret_cast<unsigned *>(scratch + NOALLOC_MAX_BLOCKS);
    // the ticket must start at zero; a completed reduction leaves it at zero,
    // but clear it so that an interrupted earlier call cannot leave it stale
    WD_CUDA_TRY(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s));
    const int blocks = (nsite + BLAS_THREADS - 1) / BLAS_THREADS;
    OpNorm2<P> op{FieldRef<P>{(char *)x, half_field_bytes(vh, P), vh}, result};
    blas_kernel<OpNorm2<P>><<<blocks, BLAS_THREADS, 0, s>>>(op, nsite, RedScratch{scratch, ticket});
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(WD_ECUDA, "reduction launch failed: %s", cudaGetErrorString(e));
    return WD_OK;
}

} // namespace
} // namespace wd

using namespace wd;

extern "C" int wd_norm2_noalloc(const int dims[4], int sites, int prec, const void *x, double *result,
                                void *stream)
{
    clear_error();
    if (!x || !result) return set_error(WD_EINVAL, "NULL argument");
    if (((uintptr_t)x & 15u) || ((uintptr_t)result & 7u)) return set_error(WD_EINVAL, "misaligned pointer");
    Geometry g;
    WD_TRY(make_geometry(dims, g));
    int64_t nsite;
    if (sites == WD_SITES_FULL) nsite = 2 * (int64_t)g.Vh;
    else if (sites == WD_SITES_EVEN || sites == WD_SITES_ODD) nsite = g.Vh;
    else return set_error(WD_EINVAL, "sites = %d is not a wd_sites value", sites);
    if (nsite > (int64_t)NOALLOC_MAX_BLOCKS * BLAS_THREADS)
        return set_error(WD_EINVAL,
                         "field of %lld sites is larger than the fixed scratch allows (at most %d sites); "
                         "use wd_norm2 with a context instead",
                         (long long)nsite, NOALLOC_MAX_BLOCKS * BLAS_THREADS);
    cudaStream_t s = (cudaStream_t)stream;
    switch (prec) {
    case WD_F64: return noalloc_norm2<PREC_F64>(x, g.Vh, (int)nsite, result, s);
    case WD_F32: return noalloc_norm2<PREC_F32>(x, g.Vh, (int)nsite, result, s);
    case WD_F16: return noalloc_norm2<PREC_F16>(x, g.Vh, (int)nsite, result, s);
    case WD_BF16: return noalloc_norm2<PREC_BF16>(x, g.Vh, (int)nsite, result, s);
    case WD_DF: return noalloc_norm2<PREC_DF>(x, g.Vh, (int)nsite, result, s);
    default: return set_error(WD_EINVAL, "bad precision %d", prec);
    }
}
