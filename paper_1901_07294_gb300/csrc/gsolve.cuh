// One mixed-precision reliable-update CG solve driven by a CUDA graph with a
// device-side loop.
//
// Shared by the graph batch mode and the request queue.  A solve owns its
// workspace, a stream, per-solve reduction scratch and a graph whose only
// top-level node is a conditional WHILE node.  Its body is one CG iteration
// (4 hop launches and 3 BLAS kernels, every CG scalar in device memory)
// followed by a one-thread control kernel that tracks max |r| and the
// iteration counts and keeps the loop going until a reliable update is due
// (|r| < delta max|r|, |r|^2 <= tol^2 |b|^2, a breakdown, RELIABLE_MAX_GAP
// iterations without an update, maxiter) or GS_LAUNCH_CAP iterations have run
// in this launch.  The host then reads the scalars and does the FP64 reliable
// update (x += x_lo, r = b - A x) and the convergence test: one host round
// trip per update instead of one per fixed number of iterations, and no
// iterations past the point where an update was due.
#pragma once

#include <cmath>
#include <cstring>

#include "blas_host.cuh"

namespace wd {

constexpr int GS_LAUNCH_CAP = 32;   // iterations at most per graph launch

// Device scalar slots of a graph-driven solve (see also OpDotAlphaDev):
// s[0] |r|^2, s[1] pAp, s[2] alpha, s[3] true |r|^2, s[4] previous |r|^2,
// s[5] beta = s[0] / s[4] for the next direction update, s[6] breakdown flag, s[8] max |r| since the last update, s[9] iterations in
// this launch, s[10] iterations since the last update, s[11] iterations in
// total, s[12] tol^2 |b|^2, s[13] delta, s[14] maxiter, s[15] GS_LAUNCH_CAP.
constexpr int GS_NSCAL = 16;

// One solve's bookkeeping after an iteration: max |r| since the last update,
// the iteration counts, and whether its loop must stop (breakdown, a residual
// that is not finite, an update due, convergence, maxiter, RELIABLE_MAX_GAP
// iterations without an update, or the per-launch cap s[15]).
__device__ __forceinline__ bool gs_member_step(double *s)
{
    const double r2 = s[0];
    const double rn = sqrt(r2);
    double maxr = s[8];
    if (rn > maxr) maxr = rn;
    s[8] = maxr;
    const double n_launch = s[9] + 1.0, n_gap = s[10] + 1.0, n_total = s[11] + 1.0;
    s[9] = n_launch;
    s[10] = n_gap;
    s[11] = n_total;
    const bool finite = r2 == r2 && r2 < 1e300;
    s[5] = s[4] > 0.0 ? r2 / s[4] : 0.0;   // once here, not per site in OpXpayDev
    return s[6] != 0.0 || !finite || rn < s[13] * maxr || r2 <= s[12] || n_total >= s[14] ||
           n_gap >= (double)RELIABLE_MAX_GAP || n_launch >= s[15];
}

// The loop condition of the WHILE node, evaluated after each iteration.
template <int UNUSED = 0>
__global__ void gs_control_kernel(double *s, cudaGraphConditionalHandle cond)
{
    grid_dependency_enter();
    if (threadIdx.x != 0) return;
    cudaGraphSetConditional(cond, gs_member_step(s) ? 0u : 1u);
}

struct GSolve {
    // problem
    const wd_gauge *gauge = nullptr;
    double mass = 0, tol = 0;
    void *x = nullptr;
    const void *b = nullptr;
    wd_cg_opts opts{};
    int vh = 0, prec = WD_F32;
    // resources
    cudaStream_t s = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond = 0;
    void *mem = nullptr;
    double *h = nullptr;   // pinned host copy of the scalars
    char *r = nullptr, *ax = nullptr, *t_o = nullptr, *t_e = nullptr;
    char *rs = nullptr, *ps = nullptr, *aps = nullptr, *tso = nullptr, *tse = nullptr, *xs = nullptr;
    double *scal = nullptr;   // device scalars, see OpDotAlphaDev
    RedScratch red{};
    // state
    double b2 = 0, stop2 = 0, maxr = 0;
    int iters = 0, updates = 0, status = WD_OK, iters_at_update = 0;
    bool active = true;
    bool broke = false;   // the last launch stopped on a breakdown (set by gs_after_begin)
    // an FP64 recomputation of the true residual is in flight: the double-word
    // one said converged, and convergence is declared only on the FP64 value
    bool confirming = false;
    bool update_fp64 = false;   // the update in flight uses the FP64 operator
    bool update_check = false;  // ... and the iterated residual's convergence triggered it
    bool fp64_only = false;     // an FP64 convergence check failed: all further updates in FP64
    double rel = 1.0;
};

inline size_t gs_footprint(int vh, int prec)
{
    return 4 * ((size_t)vh * 192 + 256) + 5 * (half_field_bytes(vh, prec) + 256) + (size_t)vh * 96 + 256 + 512 +
           (size_t)MAX_RED_BLOCKS * MAX_NR * 8 + 256;
}

namespace gs_detail {

inline int mdagm(const wd_gauge *g, int prec, int recon, double mass, const char *in, char *out, char *t_o,
                 char *t_e, cudaStream_t s)
{
    const double a = mass + 4.0, c = 1.0 / (4.0 * (mass + 4.0));
    WD_TRY(eo_hop(g, prec, recon, t_o, in, nullptr, WD_ODD, 0.0, 1.0, 0, s));
    WD_TRY(eo_hop(g, prec, recon, t_e, t_o, in, WD_EVEN, a, -c, 0, s));
    WD_TRY(eo_hop(g, prec, recon, t_o, t_e, nullptr, WD_ODD, 0.0, 1.0, 1, s));
    WD_TRY(eo_hop(g, prec, recon, out, t_o, t_e, WD_EVEN, a, -c, 1, s));
    return WD_OK;
}

template <typename Op> inline int launch(const wd_ctx *ctx, const Op &op, int nsite, RedScratch rs, cudaStream_t s)
{
    cudaError_t e = wd_launch(blas_kernel<Op>, dim3(blas_grid_for<Op>(ctx, nsite)), dim3(BLAS_THREADS), 0, s, op, nsite, rs);
    return e == cudaSuccess ? WD_OK : set_error(WD_ECUDA, "BLAS launch failed: %s", cudaGetErrorString(e));
}

// One iteration, starting with the direction update p = r + beta p
// (beta = s[5] = s[0]/s[4]; s[4] = +inf, s[5] = 0 give p = r).  A launch therefore ends right
// after a residual update, and a host-side reliable update that replaces r
// and s[0] between launches is picked up by the next direction update, as in
// the sequential solver.
template <int PS> int iteration(const wd_ctx *ctx, GSolve &q)
{
    const int vh = q.vh;
    auto FS = [&](const void *p) { return field_ref<PS>(p, vh); };
    auto FX = [&](const void *p) { return field_ref<PREC_F32>(p, vh); };
    WD_TRY(launch(ctx, OpXpayDev<PS>{FS(q.rs), FS(q.ps), q.scal}, vh, q.red, q.s));
    WD_TRY(mdagm(q.gauge, PS, q.opts.inner_recon, q.mass, q.ps, q.aps, q.tso, q.tse, q.s));
    WD_TRY(launch(ctx, OpDotAlphaDev<PS>{FS(q.ps), FS(q.aps), q.scal}, vh, q.red, q.s));
    OpCgUpdateDev<PREC_F32, PS> up{
        OpCgUpdate<PREC_F32, PS>{FX(q.xs), FS(q.rs), FS(q.ps), FS(q.aps), q.scal + 2, nullptr}, q.scal};
    WD_TRY(launch(ctx, up, vh, q.red, q.s));
    return WD_OK;
}

// r = b - A x (FP64; A applied in precision op, FP64 or double-word FP32);
// r_lo = r; |r|^2 -> h[7] (asynchronous).
template <int PS> int residual_reseed(const wd_ctx *ctx, GSolve &q, int op)
{
    const int vh = q.vh;
    auto apply = [&](int prec, const char *in, char *out) {
        return mdagm(q.gauge, prec, q.opts.outer_recon, q.mass, in, out, q.t_o, q.t_e, q.s);
    };
    auto blas = [&](const auto &o) { return launch(ctx, o, vh, q.red, q.s); };
    WD_TRY(true_residual(op, vh, (const char *)q.x, (const char *)q.b, q.r, q.ax, q.scal + 3, apply, blas));
    WD_TRY(launch(ctx, OpConvert<PS, PREC_F64>{field_ref<PS>(q.rs, vh), field_ref<PREC_F64>(q.r, vh)}, vh, q.red,
                  q.s));
    WD_CUDA_TRY(cudaMemcpyAsync(q.h + 7, q.scal + 3, sizeof(double), cudaMemcpyDeviceToHost, q.s));
    return WD_OK;
}

// x += x_lo, then residual_reseed in FP64 or the solve's outer precision (q.update_fp64).
template <int PS> int reliable_update(const wd_ctx *ctx, GSolve &q)
{
    const int vh = q.vh;
    auto F64 = [&](const void *p) { return field_ref<PREC_F64>(p, vh); };
    auto FX = [&](const void *p) { return field_ref<PREC_F32>(p, vh); };
    WD_TRY(launch(ctx, OpAxpby<PREC_F32, PREC_F64>{FX(q.xs), F64(q.x), 1.0, 1.0}, vh, q.red, q.s));
    WD_CUDA_TRY(cudaMemsetAsync(q.xs, 0, half_field_bytes(vh, WD_F32), q.s));
    return residual_reseed<PS>(ctx, q, q.update_fp64 ? WD_F64 : outer_prec_of(q.opts));
}

template <int PS> int init(const wd_ctx *ctx, GSolve &q, bool with_graph)
{
    const int vh = q.vh;
    auto F64 = [&](const void *p) { return field_ref<PREC_F64>(p, vh); };
    auto FS = [&](const void *p) { return field_ref<PS>(p, vh); };
    WD_CUDA_TRY(cudaMemsetAsync(q.mem, 0, gs_footprint(vh, PS), q.s));
    WD_TRY(launch(ctx, OpNorm2<PREC_F64>{F64(q.b), q.scal}, vh, q.red, q.s));
    WD_CUDA_TRY(cudaMemsetAsync(q.x, 0, (size_t)vh * 192, q.s));
    WD_CUDA_TRY(cudaMemcpyAsync(q.r, q.b, (size_t)vh * 192, cudaMemcpyDeviceToDevice, q.s));
    WD_TRY(launch(ctx, OpConvert<PS, PREC_F64>{FS(q.rs), F64(q.r)}, vh, q.red, q.s));
    WD_CUDA_TRY(cudaMemcpyAsync(q.ps, q.rs, half_field_bytes(vh, PS), cudaMemcpyDeviceToDevice, q.s));
    static const double inf = INFINITY;   // s[4] = inf: the first direction update gives p = r
    WD_CUDA_TRY(cudaMemcpyAsync(q.scal + 4, &inf, sizeof(double), cudaMemcpyHostToDevice, q.s));
    WD_CUDA_TRY(cudaMemcpyAsync(q.h, q.scal, sizeof(double), cudaMemcpyDeviceToHost, q.s));
    if (!with_graph) return WD_OK;
    // build the graph node by node (no stream capture): a WHILE node whose
    // body is one iteration and the control kernel
    cudaGraph_t graph;
    WD_CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaError_t ge = cudaGraphConditionalHandleCreate(&q.cond, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = q.cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    if (ge == cudaSuccess) ge = cudaGraphAddNode(&loop, graph, nullptr, nullptr, 0, &cp);
    if (ge != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_error(WD_ECUDA, "creating the solve loop failed: %s", cudaGetErrorString(ge));
    }
    GraphSink sink;
    sink.graph = cp.conditional.phGraph_out[0];
    graph_sink() = &sink;
    int rc = iteration<PS>(ctx, q);
    if (rc == WD_OK && wd_launch(gs_control_kernel<0>, dim3(1), dim3(32), 0, q.s, q.scal, q.cond) != cudaSuccess)
        rc = set_error(WD_ECUDA, "adding the loop control failed");
    graph_sink() = nullptr;
    if (rc == WD_OK && sink.err != cudaSuccess)
        rc = set_error(WD_ECUDA, "building the solve graph failed: %s", cudaGetErrorString(sink.err));
    if (rc != WD_OK) {
        cudaGraphDestroy(graph);
        return rc;
    }
    cudaError_t ce = cudaGraphInstantiate(&q.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return set_error(WD_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
    return WD_OK;
}

} // namespace gs_detail

#define WD_GS_DISPATCH(prec, CALL)                                            \
    switch (prec) {                                                           \
    case WD_F16: { constexpr int PS = PREC_F16; return CALL; }                \
    case WD_BF16: { constexpr int PS = PREC_BF16; return CALL; }              \
    default: { constexpr int PS = PREC_F32; return CALL; }                    \
    }

// Allocates a solve's device workspace, pinned scalars and stream.  Returns
// WD_ENOMEM if the workspace does not fit.
inline int gs_alloc(GSolve &q)
{
    q.vh = q.gauge->geo.Vh;
    q.prec = q.opts.inner_prec;
    const size_t bytes = gs_footprint(q.vh, q.prec);
    if (cudaMalloc(&q.mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        q.mem = nullptr;
        return set_error(WD_ENOMEM, "cudaMalloc of %zu bytes of solve workspace failed", bytes);
    }
    WD_CUDA_TRY(cudaMallocHost(&q.h, GS_NSCAL * sizeof(double)));
    WD_CUDA_TRY(cudaStreamCreateWithFlags(&q.s, cudaStreamNonBlocking));
    return WD_OK;
}

// Lays the solve's fields out in its workspace (from gs_alloc, or reused from
// an earlier solve with the same footprint), enqueues the initial state and,
// with graph = true, builds the solve's own graph (a member of a request group
// runs in its group's graph instead).  Allocates no device memory.
inline int gs_bind(const wd_ctx *ctx, GSolve &q, bool graph = true)
{
    q.vh = q.gauge->geo.Vh;
    q.prec = q.opts.inner_prec;
    q.iters = q.updates = q.iters_at_update = 0;
    q.status = WD_OK;
    q.active = true;
    q.rel = 1.0;
    std::memset(q.h, 0, GS_NSCAL * sizeof(double));
    char *p = (char *)q.mem;
    auto take = [&p](size_t n) {
        char *r = p;
        p += (n + 255) & ~size_t(255);
        return r;
    };
    const size_t h64 = (size_t)q.vh * 192, hs = half_field_bytes(q.vh, q.prec);
    q.r = take(h64); q.ax = take(h64); q.t_o = take(h64); q.t_e = take(h64);
    q.rs = take(hs); q.ps = take(hs); q.aps = take(hs); q.tso = take(hs); q.tse = take(hs);
    q.xs = take((size_t)q.vh * 96);
    q.scal = (double *)take(256);
    q.red.ticket = (unsigned *)take(256);
    q.red.partials = (double *)take((size_t)MAX_RED_BLOCKS * MAX_NR * 8);
    WD_GS_DISPATCH(q.prec, gs_detail::init<PS>(ctx, q, graph));
}

// gs_alloc + gs_bind.
inline int gs_setup(const wd_ctx *ctx, GSolve &q)
{
    WD_TRY(gs_alloc(q));
    return gs_bind(ctx, q);
}

// After gs_bind's work has finished: reads |b|^2, prepares the test and
// enqueues the loop's constants (s[8..15]); launch_cap: iterations at most per
// launch of the solve's own graph (a group member passes no limit: its group
// counts the iterations of a launch).
inline void gs_start(GSolve &q, double launch_cap = (double)GS_LAUNCH_CAP)
{
    q.confirming = q.update_fp64 = q.update_check = q.fp64_only = false;
    q.b2 = q.h[0];
    q.stop2 = SOLVE_TARGET * SOLVE_TARGET * q.tol * q.tol * q.b2;
    q.maxr = std::sqrt(q.b2);
    if (!(q.b2 > 0.0)) {
        q.active = false;
        q.rel = 0.0;
        if (!std::isfinite(q.b2)) q.status = WD_EINVAL;   // poisoned source
        return;
    }
    double *c = q.h + 8;
    c[0] = q.maxr;
    c[1] = c[2] = c[3] = 0.0;
    c[4] = q.stop2;
    c[5] = q.opts.delta;
    c[6] = (double)q.opts.maxiter;
    c[7] = launch_cap;
    if (cudaMemcpyAsync(q.scal + 8, c, 8 * sizeof(double), cudaMemcpyHostToDevice, q.s) != cudaSuccess ||
        cudaStreamSynchronize(q.s) != cudaSuccess) {
        cudaGetLastError();
        q.active = false;
        q.status = WD_ECUDA;
    }
}

// Enqueues one launch (the device loop runs until an update is due or
// GS_LAUNCH_CAP iterations) and the scalar read-back.
inline int gs_launch(GSolve &q)
{
    WD_CUDA_TRY(cudaMemsetAsync(q.scal + 9, 0, sizeof(double), q.s));
    WD_CUDA_TRY(cudaGraphLaunch(q.exec, q.s));
    WD_CUDA_TRY(cudaMemcpyAsync(q.h, q.scal, GS_NSCAL * sizeof(double), cudaMemcpyDeviceToHost, q.s));
    return WD_OK;
}

// First half of the work after a launch has finished: if the loop stopped
// for a reliable update or the convergence test (not merely at the
// per-launch cap), enqueues the FP64 update on the solve's stream and sets
// *pending; the caller then waits for the stream and calls gs_after_update.
inline int gs_after_begin(const wd_ctx *ctx, GSolve &q, bool &pending)
{
    pending = false;
    q.iters = (int)q.h[11];
    const double r2 = q.h[0];
    q.broke = q.h[6] != 0.0 || !std::isfinite(r2);
    const double rn = std::sqrt(r2);
    q.maxr = q.h[8];
    if (!(q.broke || rn < q.opts.delta * q.maxr || r2 <= q.stop2 || q.iters >= q.opts.maxiter ||
          (int)q.h[10] >= RELIABLE_MAX_GAP))
        return WD_OK;
    q.iters_at_update = q.iters;
    // an update that the iterated residual's convergence (or maxiter) triggered
    // is a convergence check: FP64 directly, as are all updates after a failed one
    q.update_check = r2 <= q.stop2 || q.iters >= q.opts.maxiter;
    q.update_fp64 = q.update_check || q.fp64_only || outer_prec_of(q.opts) == WD_F64;
    int rc;
    switch (q.prec) {
    case WD_F16: rc = gs_detail::reliable_update<PREC_F16>(ctx, q); break;
    case WD_BF16: rc = gs_detail::reliable_update<PREC_BF16>(ctx, q); break;
    default: rc = gs_detail::reliable_update<PREC_F32>(ctx, q); break;
    }
    if (rc) return rc;
    pending = true;
    return WD_OK;
}

// Second half, once the update's work has finished: reads the true residual,
// ends the solve or enqueues the restart scalars on the stream.  It does not
// wait for them: the next launch on the same stream runs after them, and the
// host writes the scalar buffer again only after that launch has finished.
// When a double-word residual meets the target, an FP64 recomputation is
// enqueued instead and q.confirming set: the caller waits for the stream again
// and calls this once more, and only the FP64 value can end the solve.
inline int gs_after_update(const wd_ctx *ctx, GSolve &q)
{
    const double r2t = q.h[7];
    const bool fp64 = q.confirming || q.update_fp64;
    if (outer_prec_of(q.opts) != WD_F64 && r2t > q.stop2 && (q.confirming || q.update_check)) q.fp64_only = true;
    q.confirming = false;
    q.update_check = false;
    q.updates++;
    q.rel = std::sqrt(r2t / q.b2);
    if (r2t <= q.stop2) {
        if (!fp64) {
            int rc;
            switch (q.prec) {
            case WD_F16: rc = gs_detail::residual_reseed<PREC_F16>(ctx, q, WD_F64); break;
            case WD_BF16: rc = gs_detail::residual_reseed<PREC_BF16>(ctx, q, WD_F64); break;
            default: rc = gs_detail::residual_reseed<PREC_F32>(ctx, q, WD_F64); break;
            }
            if (rc) return rc;
            q.confirming = true;
            return WD_OK;
        }
        q.active = false;
        return WD_OK;
    }
    if (q.iters >= q.opts.maxiter || !std::isfinite(r2t)) {
        q.active = false;
        q.status = WD_ENOCONV;
        return WD_OK;
    }
    // continue from the true residual; restart the direction after a breakdown
    // s[0] = true |r|^2, so the next direction update uses beta = |r_true|^2 / |r_old|^2
    // (s[4] still holds |r_old|^2); after a breakdown restart with p = r (s[4] = inf)
    WD_CUDA_TRY(cudaMemcpyAsync(q.scal, &q.h[7], sizeof(double), cudaMemcpyHostToDevice, q.s));
    if (q.broke) {
        static const double restart[3] = {INFINITY, 0.0, 0.0};   // s[4], s[5], s[6]
        WD_CUDA_TRY(cudaMemcpyAsync(q.scal + 4, restart, sizeof(restart), cudaMemcpyHostToDevice, q.s));
    } else {
        // beta = |r_true|^2 / |r_old|^2 (s[4] is unchanged; the same division as on the device)
        q.h[5] = q.h[4] > 0.0 ? r2t / q.h[4] : 0.0;
        WD_CUDA_TRY(cudaMemcpyAsync(q.scal + 5, q.h + 5, sizeof(double), cudaMemcpyHostToDevice, q.s));
    }
    q.maxr = std::sqrt(r2t);
    q.h[8] = q.maxr;   // s[8] = max |r| = the true |r|, s[10] = 0 iterations since the update
    q.h[10] = 0.0;
    WD_CUDA_TRY(cudaMemcpyAsync(q.scal + 8, q.h + 8, sizeof(double), cudaMemcpyHostToDevice, q.s));
    WD_CUDA_TRY(cudaMemcpyAsync(q.scal + 10, q.h + 10, sizeof(double), cudaMemcpyHostToDevice, q.s));
    return WD_OK;
}

// After a launch has finished: reliable update and convergence test when the
// loop stopped for one of them (both halves above, waiting for each).
inline int gs_after(const wd_ctx *ctx, GSolve &q)
{
    bool pending = false;
    WD_TRY(gs_after_begin(ctx, q, pending));
    if (!pending) return WD_OK;
    do {
        WD_CUDA_TRY(cudaStreamSynchronize(q.s));
        WD_TRY(gs_after_update(ctx, q));
    } while (q.confirming);
    WD_CUDA_TRY(cudaStreamSynchronize(q.s));
    return WD_OK;
}

// Drops the solve's graph but keeps workspace, scalars and stream for reuse.
inline void gs_release_graph(GSolve &q)
{
    if (q.s) cudaStreamSynchronize(q.s);
    if (q.exec) cudaGraphExecDestroy(q.exec);
    q.exec = nullptr;
}

inline void gs_release(GSolve &q)
{
    if (q.s) cudaStreamSynchronize(q.s);
    if (q.exec) cudaGraphExecDestroy(q.exec);
    if (q.s) cudaStreamDestroy(q.s);
    if (q.mem) cudaFree(q.mem);
    if (q.h) cudaFreeHost(q.h);
    q.exec = nullptr;
    q.s = nullptr;
    q.mem = nullptr;
    q.h = nullptr;
}

} // namespace wd
