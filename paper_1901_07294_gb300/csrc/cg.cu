// Conjugate gradient on the even-odd normal equations Mhat^dagger Mhat x = b.
//
// Sec. II-A names CG as the solver that dominates the run time of lattice
// QCD.  The operator is the Schur complement of D on the even sites,
//     Mhat = (m+4) - H_eo H_oe / (4(m+4)),   Mhat^dagger = gamma5 Mhat gamma5,
// applied as four even-odd hop launches with fused axpby epilogues.
//
// Mixed precision follows the reliable-update scheme of Sleijpen and van der
// Vorst (1996), in the GPU form of Clark et al. (2010): the iterated residual,
// search direction and operator run in a low storage precision (FP32, FP16
// or BF16 storage, FP32 arithmetic), while FP64 holds the solution, the true
// residual b - A x (recomputed at every reliable update with the FP64
// operator, or with the double-word FP32 one when outer_prec = WD_DF; a
// double-word residual that meets the target is confirmed with the FP64
// operator before the solve ends) and every global inner product.  An update is triggered when the
// iterated residual has fallen by `delta` since the last one, and always
// before convergence is declared; it folds the low-precision solution
// increment into x, recomputes r in FP64, re-seeds the low-precision
// residual from it and keeps the search direction.  With reliable = 0 the
// solver does iterative refinement instead: restarted low-precision CG runs
// to a relative residual `delta` on the current FP64 residual.
#include <chrono>
#include <cmath>

#include "blas_host.cuh"
#include "gsolve.cuh"

namespace wd {

namespace {

struct Bump {
    char *p;
    char *take(size_t n)
    {
        char *r = p;
        p += (n + 255) & ~size_t(255);
        return r;
    }
};

// out = Mhat^dagger Mhat in, on even half fields of precision P.
int apply_mdagm(const wd_gauge *g, int prec, int recon, double mass, const char *in, char *out, char *t_o,
                char *t_e, cudaStream_t s)
{
    const double a = mass + 4.0, c = 1.0 / (4.0 * (mass + 4.0));
    WD_TRY(eo_hop(g, prec, recon, t_o, in, nullptr, WD_ODD, 0.0, 1.0, 0, s));   // H_oe in
    WD_TRY(eo_hop(g, prec, recon, t_e, t_o, in, WD_EVEN, a, -c, 0, s));        // Mhat in
    WD_TRY(eo_hop(g, prec, recon, t_o, t_e, nullptr, WD_ODD, 0.0, 1.0, 1, s)); // g5 H_oe g5 t
    WD_TRY(eo_hop(g, prec, recon, out, t_o, t_e, WD_EVEN, a, -c, 1, s));      // Mhat^dagger t
    return WD_OK;
}

int read_scalars(wd_ctx *ctx, int first, int n, cudaStream_t s)
{
    WD_CUDA_TRY(cudaMemcpyAsync(ctx->h_scal + first, ctx->d_scal + first, n * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
    WD_CUDA_TRY(cudaStreamSynchronize(s));
    return WD_OK;
}

template <int PS, int PX>
int cg_run(wd_ctx *ctx, const wd_gauge *g, double mass, char *x, const char *b, double tol, const wd_cg_opts &o,
           wd_cg_stats &st, cudaStream_t s)
{
    const int vh = g->geo.Vh;
    const size_t h64 = half_field_bytes(vh, WD_F64), hs = half_field_bytes(vh, PS), hx = half_field_bytes(vh, PX);
    char *w = nullptr;
    WD_TRY(ctx_workspace(ctx, 4 * (h64 + 256) + 5 * (hs + 256) + hx + 256, &w));
    Bump bp{w};
    char *r = bp.take(h64), *ax = bp.take(h64), *t_o = bp.take(h64), *t_e = bp.take(h64);
    char *rs = bp.take(hs), *ps = bp.take(hs), *aps = bp.take(hs), *tso = bp.take(hs), *tse = bp.take(hs);
    char *xs = bp.take(hx);
    double *d = ctx->d_scal, *h = ctx->h_scal;

    auto F64 = [&](const void *p) { return field_ref<PREC_F64>(p, vh); };
    auto FS = [&](const void *p) { return field_ref<PS>(p, vh); };
    auto FX = [&](const void *p) { return field_ref<PX>(p, vh); };
    // the reliable updates' operator (FP64 or double-word) and BLAS launcher
    const int outer = outer_prec_of(o);
    auto mdagm_outer = [&](int prec, const char *in, char *out) {
        return apply_mdagm(g, prec, o.outer_recon, mass, in, out, t_o, t_e, s);
    };
    auto blas = [&](const auto &op) { return run_blas(ctx, op, vh, s); };

    WD_TRY(run_blas(ctx, OpNorm2<PREC_F64>{F64(b), d + 0}, vh, s));
    WD_TRY(read_scalars(ctx, 0, 1, s));
    const double b2 = h[0];
    WD_CUDA_TRY(cudaMemsetAsync(x, 0, h64, s));
    st.iters = 0;
    st.reliable_updates = 0;
    if (!(b2 > 0.0)) {
        st.true_rel_resid = 0.0;
        WD_CUDA_TRY(cudaStreamSynchronize(s));
        return std::isfinite(b2) ? WD_OK : set_error(WD_EINVAL, "source is not finite");
    }
    WD_CUDA_TRY(cudaMemcpyAsync(r, b, h64, cudaMemcpyDeviceToDevice, s));
    WD_TRY(run_blas(ctx, OpConvert<PS, PREC_F64>{FS(rs), F64(r)}, vh, s));
    WD_CUDA_TRY(cudaMemcpyAsync(ps, rs, hs, cudaMemcpyDeviceToDevice, s));
    WD_CUDA_TRY(cudaMemsetAsync(xs, 0, hx, s));

    const double stop2 = SOLVE_TARGET * SOLVE_TARGET * tol * tol * b2;
    // plain FP64 CG: the iterated residual is already FP64, so the true
    // residual is recomputed only to confirm convergence
    const bool reliable = PS == PREC_F64 ? true : o.reliable != 0;
    const double delta = PS == PREC_F64 ? 0.0 : o.delta;
    double r2 = b2, maxr = std::sqrt(b2), r2_restart = b2, r2_true = b2;
    bool converged = false;
    bool fp64_only = false;   // set once an FP64 convergence check has failed
    int status = WD_OK;
    int it = 0, it_update = 0;
    while (it < o.maxiter) {
        WD_TRY(apply_mdagm(g, PS, o.inner_recon, mass, ps, aps, tso, tse, s));
        WD_TRY(run_blas(ctx, OpDotReAlpha<PS>{FS(ps), FS(aps), r2, d + 1}, vh, s));   // d1 = pAp, d2 = alpha
        WD_TRY(run_blas(ctx, OpCgUpdate<PX, PS>{FX(xs), FS(rs), FS(ps), FS(aps), d + 2, d + 3}, vh, s));
        WD_TRY(read_scalars(ctx, 1, 3, s));
        ++it;
        const double pap = h[1];
        double r2_new = h[3];
        if (!(pap > 0.0) || !std::isfinite(r2_new)) {
            status = set_error(WD_ENOCONV, "CG breakdown at iteration %d (pAp = %g, |r|^2 = %g)", it, pap, r2_new);
            break;
        }
        const double rn = std::sqrt(r2_new);
        if (rn > maxr) maxr = rn;
        bool update;
        // a reliable update also when the low-precision residual has gone
        // RELIABLE_MAX_GAP iterations without one (it can stall above
        // delta * max|r| once rounding noise dominates)
        if (reliable)
            update = (rn < delta * maxr) || (r2_new <= stop2) || (PS != PREC_F64 && it - it_update >= RELIABLE_MAX_GAP);
        else update = r2_new <= std::fmax(stop2, delta * delta * r2_restart);
        if (update) {
            // x += x_lo (FP64), then the true residual with the FP64 operator
            WD_TRY(run_blas(ctx, OpAxpby<PX, PREC_F64>{FX(xs), F64(x), 1.0, 1.0}, vh, s));
            WD_CUDA_TRY(cudaMemsetAsync(xs, 0, hx, s));
            // an update that the iterated residual's convergence triggered is a
            // convergence check: FP64 directly, as are all updates after a failed check
            const bool check = r2_new <= stop2;
            const int op = (check || fp64_only) ? WD_F64 : outer;
            WD_TRY(true_residual(op, vh, x, b, r, ax, d + 4, mdagm_outer, blas));
            WD_TRY(read_scalars(ctx, 4, 1, s));
            r2_true = h[4];
            ++st.reliable_updates;
            if (r2_true <= stop2 && op != WD_F64) {
                // the double-word residual meets the target: only the FP64 one may end the solve
                WD_TRY(true_residual(WD_F64, vh, x, b, r, ax, d + 4, mdagm_outer, blas));
                WD_TRY(read_scalars(ctx, 4, 1, s));
                r2_true = h[4];
                ++st.reliable_updates;
                if (r2_true > stop2) fp64_only = true;
            }
            if (check && outer != WD_F64 && r2_true > stop2) fp64_only = true;
            it_update = it;
            if (r2_true <= stop2) {
                converged = true;
                break;
            }
            if (!std::isfinite(r2_true)) {
                status = set_error(WD_ENOCONV, "true residual is not finite at iteration %d", it);
                break;
            }
            WD_TRY(run_blas(ctx, OpConvert<PS, PREC_F64>{FS(rs), F64(r)}, vh, s));
            r2_new = r2_true;
            maxr = std::sqrt(r2_true);
            if (!reliable) {   // iterative refinement: restart the inner CG on the new residual
                WD_CUDA_TRY(cudaMemcpyAsync(ps, rs, hs, cudaMemcpyDeviceToDevice, s));
                r2 = r2_true;
                r2_restart = r2_true;
                continue;
            }
        }
        const double beta = r2_new / r2;
        WD_TRY(run_blas(ctx, OpAxpby<PS, PS>{FS(rs), FS(ps), 1.0, beta}, vh, s));   // p = r + beta p
        r2 = r2_new;
    }
    if (!converged && status == WD_OK) {
        WD_TRY(run_blas(ctx, OpAxpby<PX, PREC_F64>{FX(xs), F64(x), 1.0, 1.0}, vh, s));
        WD_TRY(true_residual(WD_F64, vh, x, b, r, ax, d + 4, mdagm_outer, blas));
        WD_TRY(read_scalars(ctx, 4, 1, s));
        r2_true = h[4];
        status = set_error(WD_ENOCONV, "CG did not converge in %d iterations (relative residual %.3e)", it,
                           std::sqrt(r2_true / b2));
    }
    WD_CUDA_TRY(cudaStreamSynchronize(s));
    st.iters = it;
    st.true_rel_resid = std::sqrt(r2_true / b2);
    return status;
}

// The same solve driven by a CUDA graph with a device-side loop (gsolve.cuh):
// one host synchronisation per reliable update instead of one per iteration.  Runs on
// the solve's own stream; the call is synchronous either way.
int cg_run_graph(wd_ctx *ctx, const wd_gauge *g, double mass, char *x, const char *b, double tol,
                 const wd_cg_opts &o, wd_cg_stats &st)
{
    GSolve q;
    q.gauge = g;
    q.mass = mass;
    q.tol = tol;
    q.x = x;
    q.b = b;
    q.opts = o;
    int rc = gs_setup(ctx, q);
    if (rc == WD_OK && cudaStreamSynchronize(q.s) != cudaSuccess) rc = set_error(WD_ECUDA, "solve set-up failed");
    if (rc == WD_OK) gs_start(q);
    while (rc == WD_OK && q.active) {
        rc = gs_launch(q);
        if (rc == WD_OK && cudaStreamSynchronize(q.s) != cudaSuccess) rc = set_error(WD_ECUDA, "graph replay failed");
        if (rc == WD_OK) rc = gs_after(ctx, q);
    }
    gs_release(q);
    st.iters = q.iters;
    st.reliable_updates = q.updates;
    st.true_rel_resid = q.rel;
    if (rc != WD_OK) return rc;
    if (q.status == WD_ENOCONV)
        return set_error(WD_ENOCONV, "CG did not converge in %d iterations (relative residual %.3e)", q.iters, q.rel);
    if (q.status != WD_OK) return set_error(q.status, "CG failed");
    return WD_OK;
}

} // namespace

int cg_dispatch(wd_ctx *ctx, const wd_gauge *g, double mass, char *x, const char *b, double tol,
                const wd_cg_opts &o, wd_cg_stats &st, cudaStream_t s)
{
    if (o.use_graph && o.inner_prec != WD_F64 && o.reliable) {
        // the graph runs on the solve's own stream: first let the work queued on
        // the caller's stream (which may still be writing b) finish
        WD_CUDA_TRY(cudaStreamSynchronize(s));
        return cg_run_graph(ctx, g, mass, x, b, tol, o, st);
    }
    switch (o.inner_prec) {
    case WD_F64: return cg_run<PREC_F64, PREC_F64>(ctx, g, mass, x, b, tol, o, st, s);
    case WD_F32: return cg_run<PREC_F32, PREC_F32>(ctx, g, mass, x, b, tol, o, st, s);
    case WD_F16: return cg_run<PREC_F16, PREC_F32>(ctx, g, mass, x, b, tol, o, st, s);
    default: return cg_run<PREC_BF16, PREC_F32>(ctx, g, mass, x, b, tol, o, st, s);
    }
}

} // namespace wd

using namespace wd;

extern "C" {

int cg_solve(wd_ctx *ctx, const wd_gauge *g, double mass, void *x_e, const void *b_e, double tol,
             const wd_cg_opts *opts, wd_cg_stats *stats, void *stream)
{
    clear_error();
    if (!ctx || !g || !x_e || !b_e || !opts) return set_error(WD_EINVAL, "NULL argument");
    if (((uintptr_t)x_e & 15u) || ((uintptr_t)b_e & 15u)) return set_error(WD_EINVAL, "fields must be 16-byte aligned");
    if (x_e == b_e) return set_error(WD_EINVAL, "x must not alias b");
    if (!(tol > 0.0)) return set_error(WD_EINVAL, "tol must be > 0");
    if (!valid_prec(opts->inner_prec)) return set_error(WD_EINVAL, "bad inner precision %d", opts->inner_prec);
    if (!valid_recon(opts->inner_recon) || !valid_recon(opts->outer_recon))
        return set_error(WD_EINVAL, "bad link reconstruction");
    if (opts->outer_prec != WD_F64 && opts->outer_prec != WD_DF)
        return set_error(WD_EINVAL, "outer precision must be WD_F64 or WD_DF");
    if (opts->maxiter < 1) return set_error(WD_EINVAL, "maxiter must be >= 1");
    if (opts->inner_prec != WD_F64 && !(opts->delta > 0.0 && opts->delta < 1.0))
        return set_error(WD_EINVAL, "delta must be in (0, 1)");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard dg(ctx->device);
    // build the gauge layouts up front so that no allocation happens mid-solve
    const int outer = outer_prec_of(*opts);
    WD_TRY(wd_gauge_prepare(const_cast<wd_gauge *>(g), WD_F64, opts->outer_recon));
    if (outer == WD_DF) WD_TRY(wd_gauge_prepare(const_cast<wd_gauge *>(g), WD_DF, opts->outer_recon));
    WD_TRY(wd_gauge_prepare(const_cast<wd_gauge *>(g), opts->inner_prec, opts->inner_recon));
    if (opts->autotune) {
        for (int with_x = 0; with_x < 2; ++with_x) {
            WD_TRY(hop_ensure_tuned(ctx, g, WD_F64, opts->outer_recon, 0, with_x));
            if (outer == WD_DF) WD_TRY(hop_ensure_tuned(ctx, g, WD_DF, opts->outer_recon, 0, with_x));
            WD_TRY(hop_ensure_tuned(ctx, g, opts->inner_prec, opts->inner_recon, 0, with_x));
        }
    }
    clear_error();
    wd_cg_stats st{};
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = cg_dispatch(ctx, g, mass, (char *)x_e, (const char *)b_e, tol, *opts, st, (cudaStream_t)stream);
    st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    st.status = rc;
    if (stats) *stats = st;
    return rc;
}

} // extern "C"
