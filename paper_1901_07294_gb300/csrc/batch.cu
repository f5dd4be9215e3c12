// Many CG solves at once (different lattices, masses, tolerances).
//
// Three ways to run a batch of Mhat^dagger Mhat x = b solves, all with the
// reliable-update scheme of cg.cu (low-precision iterated residual, FP64
// solution, true residual and inner products):
//   WD_BATCH_SEQUENTIAL  one cg_solve after another;
//   WD_BATCH_GRAPH       the solves of one gauge run as a request group of
//                        the serving queue: one CUDA graph per group whose
//                        device-side WHILE loop runs their iterations with
//                        one shared-link launch per hop for all of them (4 hop
//                        launches and 3 BLAS kernels, scalars in device
//                        memory) until one needs its reliable update, which
//                        the host enqueues on that solve's own stream while
//                        the group goes on;
//   WD_BATCH_PERSISTENT  one cooperative launch (all solves with the same
//                        inner precision): each solve owns a group of
//                        thread blocks (sized in proportion to its volume)
//                        that runs the whole solve, separated by group-local
//                        barriers and deterministic group reductions.  Every
//                        barrier wait is bounded (about a second of clock
//                        cycles); on timeout the kernel sets an error word and
//                        returns, and the call reports WD_ETIMEOUT.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "blas_host.cuh"
#include "dslash_impl.cuh"
#include "gsolve.cuh"

namespace wd {

int hop_setup(const wd_gauge *g, int prec, int recon, HopArgs &A);

namespace {

// ---------------------------------------------------------------------------
// persistent kernel
// ---------------------------------------------------------------------------
struct PSolve {
    HopArgs hs;            // inner-precision geometry and links
    HopArgs hd;            // FP64 geometry and links
    const char *b;         // FP64 even half fields
    char *x, *r, *ax, *to64, *te64;
    char *rs, *ps, *aps, *tso, *tse;   // inner-precision even/odd half fields
    char *xs;              // FP32 solution increment since the last reliable update
    double mass, tol, delta;
    int maxiter;
    int block0, nblocks;
    int barrier_target;    // blocks that must arrive at each barrier
    unsigned *bar;         // [0] arrivals, [32] generation (separate lines)
    double *part;          // 2 buffers x nchunk x 8 warps x 2 partial sums
    int nchunk;            // 256-site chunks of a half field: ceil(vh / 256)
    int *out_int;          // [0] status, [1] iterations, [2] reliable updates
    double *out_rel;       // true relative residual
};

struct GroupCtx {
    const PSolve *S;
    int gb, G;             // block index in the group, group size
    unsigned gen;          // barrier generation seen by this block
    int red;               // reduction counter (selects the partial-sum buffer)
    long long limit;       // clock cycles a barrier may wait
    int *err;              // grid-wide error word
};

// Group barrier: all blocks of the group (S->barrier_target of them) arrive
// before any leaves.  Returns false if the wait ran out or another block
// reported an error; the caller then returns.
__device__ bool group_sync(GroupCtx &g)
{
    __shared__ int s_fail;
    __syncthreads();
    if (threadIdx.x == 0) {
        int fail = 0;
        unsigned *cnt = g.S->bar;
        unsigned *gen = g.S->bar + 32;
        __threadfence();
        if (atomicAdd(cnt, 1u) == (unsigned)g.S->barrier_target - 1u) {
            atomicExch(cnt, 0u);
            __threadfence();
            atomicExch(gen, g.gen + 1u);
        } else {
            const long long t0 = clock64();
            while (atomicAdd(gen, 0u) == g.gen) {
                if (*(volatile int *)g.err != 0) { fail = 1; break; }
                if (clock64() - t0 > g.limit) {
                    atomicExch(g.err, WD_ETIMEOUT);
                    fail = 1;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_fail = fail;
    }
    __syncthreads();
    g.gen += 1u;
    return s_fail == 0;
}

// Group reductions whose result does not depend on the group size: a half
// field is cut into chunks of 256 sites (chunk c = sites 256c .. 256c+255, one
// block-sized pass of the group's loops); each warp's 32 per-site values of a
// chunk are summed by a fixed shuffle tree and stored as one partial, and the
// total adds the nchunk x 8 partials in a fixed order.  So a solve gives the
// same bits whatever group of blocks the batch gives it.
template <int NR> __device__ __forceinline__ double *group_part(const GroupCtx &g)
{
    return g.S->part + (size_t)(g.red & 1) * g.S->nchunk * 8 * 2;
}

// Stores chunk c's partials of the per-site values v (this thread's site).
template <int NR> __device__ void chunk_put(const GroupCtx &g, int c, double (&v)[NR])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    if (lane == 0) {
        double *buf = group_part<NR>(g);
#pragma unroll
        for (int k = 0; k < NR; ++k) buf[((size_t)c * 8 + warp) * 2 + k] = v[k];
    }
}

// Barrier, then every block adds all partials in the same fixed order (thread t
// takes entries t, t + 256, ...; then a fixed tree), so all blocks agree.
template <int NR> __device__ bool group_total(GroupCtx &g, double (&v)[NR])
{
    __shared__ double sm[8][NR];
    if (!group_sync(g)) return false;
    const double *buf = group_part<NR>(g);
    g.red++;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = g.S->nchunk * 8;
#pragma unroll
    for (int k = 0; k < NR; ++k) v[k] = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
#pragma unroll
        for (int k = 0; k < NR; ++k) v[k] += __ldcg(buf + (size_t)j * 2 + k);
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NR; ++k) sm[warp][k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w][k];
        v[k] = t;
    }
    __syncthreads();
    return true;
}

template <int P, bool DAG, bool HX>
__device__ void group_hop(const GroupCtx &g, HopArgs A, const char *in, const char *x, char *out, int p, double a,
                          double b)
{
    A.in[0] = A.in[1] = in;
    A.x[0] = A.x[1] = x;
    A.out[0] = A.out[1] = out;
    A.a = a;
    A.b = b;
    for (int i = g.gb * blockDim.x + threadIdx.x; i < A.vh; i += g.G * blockDim.x)
        hop_site<P, 18, DAG, HX, 1>(A, p, i, 0);
}

// out = Mhat^dagger Mhat in (4 hops, a barrier after each).
template <int P>
__device__ bool group_mdagm(GroupCtx &g, const HopArgs &A, double mass, const char *in, char *out, char *t_o,
                            char *t_e)
{
    const double a = mass + 4.0, c = 1.0 / (4.0 * (mass + 4.0));
    group_hop<P, false, false>(g, A, in, nullptr, t_o, 1, 0.0, 1.0);
    if (!group_sync(g)) return false;
    group_hop<P, false, true>(g, A, t_o, in, t_e, 0, a, -c);
    if (!group_sync(g)) return false;
    group_hop<P, true, false>(g, A, t_e, nullptr, t_o, 1, 0.0, 1.0);
    if (!group_sync(g)) return false;
    group_hop<P, true, true>(g, A, t_o, t_e, out, 0, a, -c);
    return true;   // the caller's next step reads only its own sites of `out`
}

// Half-field bytes of precision P on the device (as half_field_bytes).
template <int P> __host__ __device__ constexpr size_t half_bytes_of(int vh)
{
    return (size_t)vh * (24 * Prec<P>::bytes + (Prec<P>::scaled ? 4 : 0));
}

// One 256-thread block per SM: the inner-precision and FP64 hop bodies inlined
// together need up to 255 registers per thread.  P: storage precision of the
// iterated residual, the direction and the operator's intermediate fields
// (FP32, FP16 or BF16; FP32 arithmetic).
template <int P>
__global__ void __launch_bounds__(256, 1) cg_persistent_kernel(const PSolve *__restrict__ solves,
                                                                const int *__restrict__ block_solve, int *err,
                                                                long long limit)
{
    const PSolve *S = solves + block_solve[blockIdx.x];
    GroupCtx g{S, (int)blockIdx.x - S->block0, S->nblocks, 0u, 0, limit, err};
    const int vh = S->hs.vh;
    const size_t h64 = (size_t)vh * 192, h32 = (size_t)vh * 96, hp = half_bytes_of<P>(vh);
    const FieldRef<PREC_F64> fb{(char *)S->b, h64, vh}, fx{S->x, h64, vh}, fr{S->r, h64, vh}, fax{S->ax, h64, vh};
    const FieldRef<P> frs{S->rs, hp, vh}, fps{S->ps, hp, vh}, faps{S->aps, hp, vh};
    const FieldRef<PREC_F32> fxs{S->xs, h32, vh};
    const int i0 = g.gb * blockDim.x + threadIdx.x, stride = g.G * blockDim.x;

    // |b|^2, then x = 0, r = b, rs = ps = (FP32) b, xs = 0 on this block's sites
    for (int c = g.gb; c < S->nchunk; c += g.G) {
        const int i = c * 256 + threadIdx.x;
        double v[1] = {0.0};
        if (i < vh) {
            double bv[24];
            fb.load(i, bv);
            double s = 0.0;
            for (int k = 0; k < 24; ++k) s = fma(bv[k], bv[k], s);
            v[0] = s;
            fr.store(i, bv);
            float f[24];
            for (int k = 0; k < 24; ++k) f[k] = (float)bv[k];
            frs.store(i, f);
            fps.store(i, f);
            for (int k = 0; k < 24; ++k) { bv[k] = 0.0; f[k] = 0.0f; }
            fx.store(i, bv);
            fxs.store(i, f);
        }
        chunk_put(g, c, v);
    }
    double one[1];
    if (!group_total(g, one)) return;
    const double b2 = one[0];
    int status = WD_OK, it = 0, nupd = 0, it_update = 0;
    double r2t = b2;
    if (b2 > 0.0) {
        const double stop2 = SOLVE_TARGET * SOLVE_TARGET * S->tol * S->tol * b2;
        double r2 = b2, maxr = sqrt(b2);
        bool converged = false;
        while (it < S->maxiter) {
            if (!group_mdagm<P>(g, S->hs, S->mass, S->ps, S->aps, S->tso, S->tse)) return;
            double pap[1];
            for (int c = g.gb; c < S->nchunk; c += g.G) {
                const int i = c * 256 + threadIdx.x;
                double v[1] = {0.0};
                if (i < vh) {
                    float pv[24], av[24];
                    fps.load(i, pv);
                    faps.load(i, av);
                    float t = 0.0f;
                    for (int k = 0; k < 24; ++k) t = fmaf(pv[k], av[k], t);
                    v[0] = (double)t;
                }
                chunk_put(g, c, v);
            }
            if (!group_total(g, pap)) return;
            if (!(pap[0] > 0.0)) { status = WD_ENOCONV; break; }
            const double alpha = r2 / pap[0];
            double rr[1];
            for (int c = g.gb; c < S->nchunk; c += g.G) {
                const int i = c * 256 + threadIdx.x;
                double v[1] = {0.0};
                if (i < vh) {
                    float rv[24], av[24], pv[24], xv[24];
                    frs.load(i, rv);
                    faps.load(i, av);
                    fps.load(i, pv);
                    fxs.load(i, xv);
                    const float af = (float)alpha;
                    float t = 0.0f;
                    for (int k = 0; k < 24; ++k) {
                        rv[k] = fmaf(-af, av[k], rv[k]);
                        t = fmaf(rv[k], rv[k], t);
                        xv[k] = fmaf(af, pv[k], xv[k]);
                    }
                    frs.store(i, rv);
                    fxs.store(i, xv);
                    v[0] = (double)t;
                }
                chunk_put(g, c, v);
            }
            if (!group_total(g, rr)) return;
            ++it;
            double r2new = rr[0];
            const double rn = sqrt(r2new);
            if (rn > maxr) maxr = rn;
            if (rn < S->delta * maxr || r2new <= stop2 || it - it_update >= RELIABLE_MAX_GAP) {
                it_update = it;
                // reliable update: x += xs (FP64), true residual with the FP64 operator
                for (int i = i0; i < vh; i += stride) {
                    double xv[24];
                    float sv[24];
                    fx.load(i, xv);
                    fxs.load(i, sv);
                    for (int k = 0; k < 24; ++k) { xv[k] += (double)sv[k]; sv[k] = 0.0f; }
                    fx.store(i, xv);
                    fxs.store(i, sv);
                }
                if (!group_sync(g)) return;
                if (!group_mdagm<PREC_F64>(g, S->hd, S->mass, S->x, S->ax, S->to64, S->te64)) return;
                double t2[1];
                for (int c = g.gb; c < S->nchunk; c += g.G) {
                    const int i = c * 256 + threadIdx.x;
                    double v[1] = {0.0};
                    if (i < vh) {
                        double bv[24], av[24];
                        fb.load(i, bv);
                        fax.load(i, av);
                        double s = 0.0;
                        float f[24];
                        for (int k = 0; k < 24; ++k) {
                            bv[k] -= av[k];
                            s = fma(bv[k], bv[k], s);
                            f[k] = (float)bv[k];
                        }
                        fr.store(i, bv);
                        frs.store(i, f);
                        v[0] = s;
                    }
                    chunk_put(g, c, v);
                }
                if (!group_total(g, t2)) return;
                ++nupd;
                r2t = t2[0];
                if (r2t <= stop2) { converged = true; break; }
                if (!(r2t < 1e300)) { status = WD_ENOCONV; break; }
                r2new = r2t;
                maxr = sqrt(r2t);
            }
            const float beta = (float)(r2new / r2);
            for (int i = i0; i < vh; i += stride) {
                float rv[24], pv[24];
                frs.load(i, rv);
                fps.load(i, pv);
                for (int k = 0; k < 24; ++k) pv[k] = fmaf(beta, pv[k], rv[k]);
                fps.store(i, pv);
            }
            if (!group_sync(g)) return;
            r2 = r2new;
        }
        if (!converged && status == WD_OK) status = WD_ENOCONV;
    }
    if (g.gb == 0 && threadIdx.x == 0) {
        S->out_int[0] = status;
        S->out_int[1] = it;
        S->out_int[2] = nupd;
        S->out_rel[0] = b2 > 0.0 ? sqrt(r2t / b2) : 0.0;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

int check_desc(const wd_solve_desc &d, int mode)
{
    if (!d.gauge || !d.x_e || !d.b_e) return set_error(WD_EINVAL, "NULL gauge or field in a solve descriptor");
    if (((uintptr_t)d.x_e & 15u) || ((uintptr_t)d.b_e & 15u)) return set_error(WD_EINVAL, "misaligned field");
    if (!(d.tol > 0.0)) return set_error(WD_EINVAL, "tol must be > 0");
    if (d.opts.maxiter < 1) return set_error(WD_EINVAL, "maxiter must be >= 1");
    if (!valid_prec(d.opts.inner_prec)) return set_error(WD_EINVAL, "bad inner precision");
    if (!valid_recon(d.opts.inner_recon) || !valid_recon(d.opts.outer_recon))
        return set_error(WD_EINVAL, "bad link reconstruction");
    if (d.opts.outer_prec != WD_F64 && d.opts.outer_prec != WD_DF)
        return set_error(WD_EINVAL, "outer precision must be WD_F64 or WD_DF");
    if (mode == WD_BATCH_PERSISTENT) {
        if (d.opts.inner_prec == WD_F64 || d.opts.inner_recon != 18 || d.opts.outer_recon != 18 || !d.opts.reliable ||
            d.opts.outer_prec != WD_F64)
            return set_error(WD_EINVAL, "the persistent batch runs mixed-precision reliable-update CG "
                                        "(FP32, FP16 or BF16 inner) with 18-real links and FP64 updates only");
        if (!(d.opts.delta > 0.0 && d.opts.delta < 1.0)) return set_error(WD_EINVAL, "delta must be in (0, 1)");
    }
    if (mode == WD_BATCH_GRAPH && (d.opts.inner_prec == WD_F64 || !d.opts.reliable))
        return set_error(WD_EINVAL, "the graph batch runs mixed-precision reliable-update CG");
    return WD_OK;
}

int run_persistent(wd_ctx *ctx, int n, const wd_solve_desc *d, wd_cg_stats *stats, cudaStream_t s)
{
    // one kernel per launch: every solve of the batch has the same inner precision
    const int inner = d[0].opts.inner_prec;
    for (int k = 1; k < n; ++k)
        if (d[k].opts.inner_prec != inner)
            return set_error(WD_EINVAL, "the solves of a persistent batch must share their inner precision");
    const void *kernel = inner == WD_F16    ? (const void *)cg_persistent_kernel<PREC_F16>
                         : inner == WD_BF16 ? (const void *)cg_persistent_kernel<PREC_BF16>
                                            : (const void *)cg_persistent_kernel<PREC_F32>;
    int per_sm = 0;
    WD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0));
    const int capacity = per_sm * ctx->num_sms;
    if (capacity < 1) return set_error(WD_ECUDA, "persistent kernel cannot be resident");
    // host-side fault injection for tests: WD_FAULT=barrier_missing makes each
    // group wait for one block more than it has, so its first barrier times out
    const char *fault = std::getenv("WD_FAULT");
    const int extra = (fault && std::strstr(fault, "barrier_missing")) ? 1 : 0;
    double limit_s = 1.0;
    if (const char *ls = std::getenv("WD_BARRIER_TIMEOUT_S")) limit_s = std::atof(ls);
    const long long limit = (long long)(limit_s * device_clock_khz(ctx->device) * 1e3);

    int done = 0;
    while (done < n) {
        // next wave: as many solves as fit one block each, groups sized by volume
        int m = std::min(n - done, capacity);
        double vtot = 0.0;
        for (int k = 0; k < m; ++k) vtot += d[done + k].gauge->geo.Vh;
        std::vector<int> nb(m);
        int used = 0;
        for (int k = 0; k < m; ++k) {
            const int vh = d[done + k].gauge->geo.Vh;
            const int maxb = (vh + 255) / 256;
            int want = (int)std::floor((double)(capacity - m) * vh / vtot) + 1;
            nb[k] = std::max(1, std::min(want, maxb));
            used += nb[k];
        }
        // hand out what rounding left to the largest groups that can take it
        for (int k = 0; used < capacity && k < m; ++k) {
            const int maxb = (d[done + k].gauge->geo.Vh + 255) / 256;
            while (used < capacity && nb[k] < maxb && nb[k] < 4 * (int)std::ceil((double)capacity * d[done + k].gauge->geo.Vh / vtot)) {
                ++nb[k];
                ++used;
            }
        }
        // device memory: workspace fields + per-solve sync/partials/outputs
        std::vector<PSolve> ps(m);
        std::vector<int> bmap(used);
        size_t bytes = 0;
        std::vector<size_t> off(m);
        for (int k = 0; k < m; ++k) {
            const int vh = d[done + k].gauge->geo.Vh;
            off[k] = bytes;
            bytes += 4 * ((size_t)vh * 192 + 256) + 5 * (half_field_bytes(vh, inner) + 256) + ((size_t)vh * 96 + 256) +
                     256 + 4096 +
                     (size_t)((vh + 255) / 256) * 8 * 2 * 2 * sizeof(double) + 256;
        }
        DevBuf work, meta;
        if (cudaMalloc(&work.p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return set_error(WD_ENOMEM, "cudaMalloc of %zu bytes for the persistent batch failed", bytes);
        }
        WD_CUDA_TRY(cudaMemsetAsync(work.p, 0, bytes, s));
        int b0 = 0;
        for (int k = 0; k < m; ++k) {
            const wd_solve_desc &dk = d[done + k];
            PSolve &P = ps[k];
            std::memset(&P, 0, sizeof(P));
            WD_TRY(hop_setup(dk.gauge, inner, 18, P.hs));
            WD_TRY(hop_setup(dk.gauge, WD_F64, 18, P.hd));
            P.hs.nparity = P.hd.nparity = 1;
            const int vh = dk.gauge->geo.Vh;
            char *q = (char *)work.p + off[k];
            auto take = [&q](size_t nbytes) {
                char *r = q;
                q += (nbytes + 255) & ~size_t(255);
                return r;
            };
            P.b = (const char *)dk.b_e;
            P.x = (char *)dk.x_e;
            P.r = take((size_t)vh * 192);
            P.ax = take((size_t)vh * 192);
            P.to64 = take((size_t)vh * 192);
            P.te64 = take((size_t)vh * 192);
            const size_t hp = half_field_bytes(vh, inner);
            P.rs = take(hp);
            P.ps = take(hp);
            P.aps = take(hp);
            P.tso = take(hp);
            P.tse = take(hp);
            P.xs = take((size_t)vh * 96);
            P.bar = (unsigned *)take(256);
            P.out_int = (int *)take(64);
            P.out_rel = (double *)take(64);
            P.nchunk = (vh + 255) / 256;
            P.part = (double *)take((size_t)P.nchunk * 8 * 2 * 2 * sizeof(double));
            P.mass = dk.mass;
            P.tol = dk.tol;
            P.delta = dk.opts.delta;
            P.maxiter = dk.opts.maxiter;
            P.block0 = b0;
            P.nblocks = nb[k];
            P.barrier_target = nb[k] + extra;
            for (int b = 0; b < nb[k]; ++b) bmap[b0 + b] = k;
            b0 += nb[k];
        }
        const size_t mbytes = sizeof(PSolve) * m + sizeof(int) * used + 64;
        if (cudaMalloc(&meta.p, mbytes) != cudaSuccess) {
            cudaGetLastError();
            return set_error(WD_ENOMEM, "cudaMalloc of the batch descriptors failed");
        }
        PSolve *d_ps = (PSolve *)meta.p;
        int *d_map = (int *)((char *)meta.p + sizeof(PSolve) * m);
        int *d_err = d_map + used;
        WD_CUDA_TRY(cudaMemcpyAsync(d_ps, ps.data(), sizeof(PSolve) * m, cudaMemcpyHostToDevice, s));
        WD_CUDA_TRY(cudaMemcpyAsync(d_map, bmap.data(), sizeof(int) * used, cudaMemcpyHostToDevice, s));
        WD_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), s));
        void *args[] = {(void *)&d_ps, (void *)&d_map, (void *)&d_err, (void *)&limit};
        WD_CUDA_TRY(cudaLaunchCooperativeKernel(kernel, dim3(used), dim3(256), args, 0, s));
        WD_CUDA_TRY(cudaStreamSynchronize(s));
        int herr = 0;
        WD_CUDA_TRY(cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost));
        for (int k = 0; k < m; ++k) {
            int oi[3];
            double rel = 0.0;
            WD_CUDA_TRY(cudaMemcpy(oi, ps[k].out_int, sizeof(oi), cudaMemcpyDeviceToHost));
            WD_CUDA_TRY(cudaMemcpy(&rel, ps[k].out_rel, sizeof(double), cudaMemcpyDeviceToHost));
            if (stats) {
                wd_cg_stats &st = stats[done + k];
                st.status = herr ? WD_ETIMEOUT : oi[0];
                st.iters = oi[1];
                st.reliable_updates = oi[2];
                st.true_rel_resid = rel;
            }
        }
        if (herr) return set_error(WD_ETIMEOUT, "a group barrier of the persistent batch timed out");
        done += m;
    }
    return WD_OK;
}

// ---------------------------------------------------------------------------
// graph mode: the serving queue with every solve submitted at once, so that
// the solves on one gauge run as one request group (one shared-link hop launch
// per hop for all of them, in the group's device-side graph loop; ggroup.cuh)
// and the groups and the FP64 reliable updates run concurrently.
// ---------------------------------------------------------------------------
int run_graph(wd_ctx *ctx, int n, const wd_solve_desc *d, wd_cg_stats *stats)
{
    size_t budget = 0;
    for (int k = 0; k < n; ++k) budget += gs_footprint(d[k].gauge->geo.Vh, d[k].opts.inner_prec);
    rq_queue *q = nullptr;
    WD_TRY(rq_create(ctx, budget > 0 ? budget : 1, n > 0 ? n : 1, &q));
    std::vector<uint64_t> tickets(n, 0);
    int rc = WD_OK, submitted = 0;
    for (int k = 0; k < n && rc == WD_OK; ++k, ++submitted) rc = rq_submit(q, &d[k], &tickets[k]);
    int first_bad = -1, bad_status = WD_OK;
    for (int k = 0; k < submitted; ++k) {
        wd_solve_result res{};
        if (rq_wait(q, tickets[k], -1, &res) != WD_OK && rc == WD_OK) rc = WD_ECUDA;
        if (stats) {
            stats[k] = res.stats;
            stats[k].status = res.status;
        }
        if (res.status != WD_OK && first_bad < 0) {
            first_bad = k;
            bad_status = res.status;
        }
    }
    rq_destroy(q);
    if (rc != WD_OK) return rc;
    if (first_bad >= 0) return set_error(bad_status, "solve %d of the batch failed", first_bad);
    return WD_OK;
}

} // namespace
} // namespace wd

using namespace wd;

extern "C" int cg_solve_batch(wd_ctx *ctx, int n, const wd_solve_desc *descs, int mode, wd_cg_stats *stats,
                              void *stream)
{
    clear_error();
    if (!ctx || n < 0 || (n > 0 && !descs)) return set_error(WD_EINVAL, "bad arguments");
    if (mode != WD_BATCH_SEQUENTIAL && mode != WD_BATCH_GRAPH && mode != WD_BATCH_PERSISTENT)
        return set_error(WD_EINVAL, "bad batch mode %d", mode);
    for (int k = 0; k < n; ++k) WD_TRY(check_desc(descs[k], mode));
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    int rc = WD_OK;
    if (mode == WD_BATCH_SEQUENTIAL) {
        for (int k = 0; k < n; ++k) {
            wd_cg_stats st{};
            int r = cg_solve(ctx, descs[k].gauge, descs[k].mass, descs[k].x_e, descs[k].b_e, descs[k].tol,
                             &descs[k].opts, &st, stream);
            if (stats) stats[k] = st;
            if (r != WD_OK && rc == WD_OK) rc = r;
        }
        return rc;
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard dg(ctx->device);
    for (int k = 0; k < n; ++k) {
        const wd_solve_desc &d = descs[k];
        WD_TRY(wd_gauge_prepare(const_cast<wd_gauge *>(d.gauge), WD_F64, d.opts.outer_recon));
        if (outer_prec_of(d.opts) == WD_DF)
            WD_TRY(wd_gauge_prepare(const_cast<wd_gauge *>(d.gauge), WD_DF, d.opts.outer_recon));
        WD_TRY(wd_gauge_prepare(const_cast<wd_gauge *>(d.gauge), d.opts.inner_prec, d.opts.inner_recon));
        if (d.opts.autotune && mode == WD_BATCH_GRAPH)
            for (int with_x = 0; with_x < 2; ++with_x) {
                WD_TRY(hop_ensure_tuned(ctx, d.gauge, outer_prec_of(d.opts), d.opts.outer_recon, 0, with_x));
                WD_TRY(hop_ensure_tuned(ctx, d.gauge, d.opts.inner_prec, d.opts.inner_recon, 0, with_x));
            }
    }
    clear_error();
    if (mode == WD_BATCH_PERSISTENT) {
        rc = run_persistent(ctx, n, descs, stats, s);
    } else {
        // the solves run on their own streams: first let the work queued on the
        // caller's stream (which may still be writing the sources) finish
        WD_CUDA_TRY(cudaStreamSynchronize(s));
        rc = run_graph(ctx, n, descs, stats);
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats)
        for (int k = 0; k < n; ++k) stats[k].seconds = secs;
    return rc;
}
