// BiCGStab on the even-odd Schur system Mhat x_e = b_e, and the full-system
// solve D x = b by even-odd reduction.
//
// The paper names only CG (Sec. II-A); these are the steps either side of the
// CG path.  Mhat = (m+4) - H_eo H_oe / (4(m+4)) is not Hermitian, so BiCGStab
// (van der Vorst 1992) applies to it directly, at two Mhat applications (four
// even-odd hops) per iteration, the cost of one CG iteration on the normal
// equations, without squaring the condition number.
//
// Mixed precision: the iterated vectors (r, r^, p, v, s, t) and the operator
// run in the low storage precision, the solution increment in FP32, and FP64
// holds the solution, the true residual b - Mhat x (FP64 operator) and every
// global inner product.  With reliable = 1 the iterated residual is replaced
// by the true one whenever it has fallen by `delta` since the last
// replacement (residual replacement, van der Vorst and Ye 2000, the
// counterpart of reliable updates in CG); rho and beta are recomputed from it
// and the Krylov state is kept.  With reliable = 0 each correction restarts
// BiCGStab on the current FP64 residual (iterative refinement).  Convergence
// is always confirmed with the FP64 residual.
//
// Full system (reading of the even-odd reduction):
//   b^_e = b_e + H_eo b_o / (2(m+4));   Mhat x_e = b^_e;
//   x_o = (b_o + H_oe x_e / 2) / (m+4).
// With that x_o the odd rows of D x = b hold exactly and the even rows leave
// b^_e - Mhat x_e, so the Schur system is solved to tol |b| / |b^_e|.  The
// Schur solve is BiCGStab on Mhat or CG on Mhat^dagger Mhat x_e = Mhat^dagger
// b^_e with defect correction on the Schur residual.
#include <chrono>
#include <cmath>

#include "bicg_ops.cuh"
#include "blas_host.cuh"

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

int read_scal(wd_ctx *ctx, int first, int n, cudaStream_t s)
{
    WD_CUDA_TRY(cudaMemcpyAsync(ctx->h_scal + first, ctx->d_scal + first, n * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
    WD_CUDA_TRY(cudaStreamSynchronize(s));
    return WD_OK;
}

// out = Mhat in (dagger = 0) or Mhat^dagger in, even half fields of precision prec.
int apply_mhat(const wd_gauge *g, int prec, int recon, double mass, const char *in, char *out, char *t_o, int dagger,
               cudaStream_t s)
{
    const double a = mass + 4.0, c = 1.0 / (4.0 * (mass + 4.0));
    WD_TRY(eo_hop(g, prec, recon, t_o, in, nullptr, WD_ODD, 0.0, 1.0, dagger, s));
    WD_TRY(eo_hop(g, prec, recon, out, t_o, in, WD_EVEN, a, -c, dagger, s));
    return WD_OK;
}

template <int PS, int PX>
int bicg_run(wd_ctx *ctx, const wd_gauge *g, double mass, char *x, const char *b, double tol, const wd_cg_opts &o,
             wd_cg_stats &st, cudaStream_t s)
{
    const int vh = g->geo.Vh;
    const size_t h64 = half_field_bytes(vh, WD_F64), hs = half_field_bytes(vh, PS), hx = half_field_bytes(vh, PX);
    char *w = nullptr;
    WD_TRY(ctx_workspace(ctx, 3 * (h64 + 256) + 7 * (hs + 256) + hx + 256, &w));
    Bump bp{w};
    char *r = bp.take(h64), *ax = bp.take(h64), *t_o = bp.take(h64);
    char *rs = bp.take(hs), *rh = bp.take(hs), *ps = bp.take(hs), *vs = bp.take(hs), *ss = bp.take(hs);
    char *ts = bp.take(hs), *tso = bp.take(hs);
    char *xs = bp.take(hx);
    double *d = ctx->d_scal, *h = ctx->h_scal;
    auto F64 = [&](const void *p) { return field_ref<PREC_F64>(p, vh); };
    auto FS = [&](const void *p) { return field_ref<PS>(p, vh); };
    auto FX = [&](const void *p) { return field_ref<PX>(p, vh); };
    // the reliable updates' operator (FP64 or double-word) and BLAS launcher
    const int outer = outer_prec_of(o);
    auto mhat_outer = [&](int prec, const char *in, char *out) {
        return apply_mhat(g, prec, o.outer_recon, mass, in, out, t_o, 0, s);
    };
    auto blas = [&](const auto &op) { return run_blas(ctx, op, vh, s); };

    WD_TRY(run_blas(ctx, OpNorm2<PREC_F64>{F64(b), d + 0}, vh, s));
    WD_TRY(read_scal(ctx, 0, 1, s));
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
    WD_CUDA_TRY(cudaMemsetAsync(xs, 0, hx, s));
    auto restart = [&]() -> int {
        WD_CUDA_TRY(cudaMemsetAsync(ps, 0, hs, s));
        WD_CUDA_TRY(cudaMemsetAsync(vs, 0, hs, s));
        return run_blas(ctx, OpBicgRestart<PS>{FS(rs), FS(rh), d}, vh, s);
    };
    WD_TRY(restart());

    const double stop2 = SOLVE_TARGET * SOLVE_TARGET * tol * tol * b2;
    const bool reliable = PS == PREC_F64 ? true : o.reliable != 0;
    const double delta = PS == PREC_F64 ? 0.0 : o.delta;
    double maxr = std::sqrt(b2), r2_restart = b2, r2_true = b2;
    bool converged = false;
    int status = WD_OK;
    int it = 0, it_update = 0;
    bool fp64_only = false;   // set once an FP64 convergence check has failed
    while (it < o.maxiter) {
        WD_TRY(run_blas(ctx, OpBicgP<PS>{FS(rs), FS(ps), FS(vs), d}, vh, s));
        WD_TRY(apply_mhat(g, PS, o.inner_recon, mass, ps, vs, tso, 0, s));
        WD_TRY(run_blas(ctx, OpBicgAlpha<PS>{FS(rh), FS(vs), d}, vh, s));
        WD_TRY(run_blas(ctx, OpBicgS<PS>{FS(rs), FS(vs), FS(ss), d}, vh, s));
        WD_TRY(apply_mhat(g, PS, o.inner_recon, mass, ss, ts, tso, 0, s));
        WD_TRY(run_blas(ctx, OpBicgOmega<PS>{FS(ts), FS(ss), d}, vh, s));
        WD_TRY(run_blas(ctx, OpBicgUpdate<PX, PS>{FX(xs), FS(ps), FS(ss), FS(ts), FS(rh), FS(rs), d}, vh, s));
        WD_TRY(read_scal(ctx, BS_R2, BS_FLAG - BS_R2 + 1, s));
        ++it;
        const double r2 = h[BS_R2];
        const bool breakdown = h[BS_FLAG] != 0.0 || !std::isfinite(r2);
        const double rn = std::sqrt(r2);
        if (rn > maxr) maxr = rn;
        bool update = breakdown;
        if (reliable)
            update = update || (rn < delta * maxr) || (r2 <= stop2) ||
                     (PS != PREC_F64 && it - it_update >= RELIABLE_MAX_GAP);
        else update = update || r2 <= std::fmax(stop2, delta * delta * r2_restart);
        if (!update) continue;
        // x += x_lo (FP64), then the true residual with the FP64 operator
        WD_TRY(run_blas(ctx, OpAxpby<PX, PREC_F64>{FX(xs), F64(x), 1.0, 1.0}, vh, s));
        WD_CUDA_TRY(cudaMemsetAsync(xs, 0, hx, s));
        // an update that the iterated residual's convergence triggered is a
        // convergence check: FP64 directly, as are all updates after a failed check
        const bool check = r2 <= stop2;
        const int op = (check || fp64_only) ? WD_F64 : outer;
        WD_TRY(true_residual(op, vh, x, b, r, ax, d + 4, mhat_outer, blas));
        WD_TRY(read_scal(ctx, 4, 1, s));
        r2_true = h[4];
        ++st.reliable_updates;
        if (r2_true <= stop2 && op != WD_F64) {
            // the double-word residual meets the target: only the FP64 one may end the solve
            WD_TRY(true_residual(WD_F64, vh, x, b, r, ax, d + 4, mhat_outer, blas));
            WD_TRY(read_scal(ctx, 4, 1, s));
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
            status = set_error(WD_ENOCONV, "BiCGStab: true residual is not finite at iteration %d", it);
            break;
        }
        WD_TRY(run_blas(ctx, OpConvert<PS, PREC_F64>{FS(rs), F64(r)}, vh, s));
        maxr = std::sqrt(r2_true);
        if (breakdown || !reliable) {
            r2_restart = r2_true;
            WD_TRY(restart());
        } else {
            WD_TRY(run_blas(ctx, OpBicgRho<PS>{FS(rh), FS(rs), d}, vh, s));
        }
    }
    if (!converged && status == WD_OK) {
        WD_TRY(run_blas(ctx, OpAxpby<PX, PREC_F64>{FX(xs), F64(x), 1.0, 1.0}, vh, s));
        WD_TRY(true_residual(WD_F64, vh, x, b, r, ax, d + 4, mhat_outer, blas));
        WD_TRY(read_scal(ctx, 4, 1, s));
        r2_true = h[4];
        status = set_error(WD_ENOCONV, "BiCGStab did not converge in %d iterations (relative residual %.3e)", it,
                           std::sqrt(r2_true / b2));
    }
    WD_CUDA_TRY(cudaStreamSynchronize(s));
    st.iters = it;
    st.true_rel_resid = std::sqrt(r2_true / b2);
    return status;
}

int bicg_dispatch(wd_ctx *ctx, const wd_gauge *g, double mass, char *x, const char *b, double tol,
                  const wd_cg_opts &o, wd_cg_stats &st, cudaStream_t s)
{
    switch (o.inner_prec) {
    case WD_F64: return bicg_run<PREC_F64, PREC_F64>(ctx, g, mass, x, b, tol, o, st, s);
    case WD_F32: return bicg_run<PREC_F32, PREC_F32>(ctx, g, mass, x, b, tol, o, st, s);
    case WD_F16: return bicg_run<PREC_F16, PREC_F32>(ctx, g, mass, x, b, tol, o, st, s);
    default: return bicg_run<PREC_BF16, PREC_F32>(ctx, g, mass, x, b, tol, o, st, s);
    }
}

int check_solve_args(wd_ctx *ctx, const wd_gauge *g, const void *x, const void *b, double tol, const wd_cg_opts *o)
{
    if (!ctx || !g || !x || !b || !o) return set_error(WD_EINVAL, "NULL argument");
    if (((uintptr_t)x & 15u) || ((uintptr_t)b & 15u)) return set_error(WD_EINVAL, "fields must be 16-byte aligned");
    if (x == b) return set_error(WD_EINVAL, "x must not alias b");
    if (!(tol > 0.0)) return set_error(WD_EINVAL, "tol must be > 0");
    if (!valid_prec(o->inner_prec)) return set_error(WD_EINVAL, "bad inner precision %d", o->inner_prec);
    if (!valid_recon(o->inner_recon) || !valid_recon(o->outer_recon))
        return set_error(WD_EINVAL, "bad link reconstruction");
    if (o->outer_prec != WD_F64 && o->outer_prec != WD_DF)
        return set_error(WD_EINVAL, "outer precision must be WD_F64 or WD_DF");
    if (o->maxiter < 1) return set_error(WD_EINVAL, "maxiter must be >= 1");
    if (o->inner_prec != WD_F64 && !(o->delta > 0.0 && o->delta < 1.0))
        return set_error(WD_EINVAL, "delta must be in (0, 1)");
    return WD_OK;
}

int prepare_layouts(wd_ctx *ctx, const wd_gauge *g, const wd_cg_opts &o)
{
    // FP64 links for the full-system steps; the reliable updates' links if double-word
    WD_TRY(wd_gauge_prepare(const_cast<wd_gauge *>(g), WD_F64, o.outer_recon));
    if (outer_prec_of(o) == WD_DF) WD_TRY(wd_gauge_prepare(const_cast<wd_gauge *>(g), WD_DF, o.outer_recon));
    WD_TRY(wd_gauge_prepare(const_cast<wd_gauge *>(g), o.inner_prec, o.inner_recon));
    if (o.autotune) {
        for (int with_x = 0; with_x < 2; ++with_x) {
            WD_TRY(hop_ensure_tuned(ctx, g, WD_F64, o.outer_recon, 0, with_x));
            if (outer_prec_of(o) == WD_DF) WD_TRY(hop_ensure_tuned(ctx, g, WD_DF, o.outer_recon, 0, with_x));
            WD_TRY(hop_ensure_tuned(ctx, g, o.inner_prec, o.inner_recon, 0, with_x));
        }
        WD_TRY(hop_ensure_tuned(ctx, g, WD_F64, o.outer_recon, 1, 1));
    }
    clear_error();
    return WD_OK;
}

// CG on the normal equations of Mhat x_e = bh with defect correction on the
// Schur residual: each pass solves Mhat^dagger Mhat e = Mhat^dagger rh (rh the
// current Schur residual) and adds e to x_e, until |rh| <= tol |bh|.  The
// normal equations are solved to a relative residual chosen from the last
// pass, since |Mhat^dagger r| small only bounds |r| up to cond(Mhat).
int cgne_schur(wd_ctx *ctx, const wd_gauge *g, double mass, char *x_e, const char *bh, double bh2, double tol,
               const wd_cg_opts &o, wd_cg_stats &st, cudaStream_t s)
{
    const int vh = g->geo.Vh;
    const size_t h64 = half_field_bytes(vh, WD_F64);
    char *aux = nullptr;
    WD_TRY(ctx_aux_workspace(ctx, 4 * (h64 + 256), &aux));
    Bump bp{aux};
    char *rh = bp.take(h64), *c = bp.take(h64), *e = bp.take(h64), *t_o = bp.take(h64);
    double *d = ctx->d_scal, *h = ctx->h_scal;
    auto F64 = [&](const void *p) { return field_ref<PREC_F64>(p, vh); };
    WD_CUDA_TRY(cudaMemsetAsync(x_e, 0, h64, s));
    WD_CUDA_TRY(cudaMemcpyAsync(rh, bh, h64, cudaMemcpyDeviceToDevice, s));
    double r2 = bh2, tol_ne = tol;
    const double target2 = SOLVE_TARGET * SOLVE_TARGET * tol * tol * bh2;
    st.iters = 0;
    st.reliable_updates = 0;
    for (int pass = 0; pass < 8; ++pass) {
        WD_TRY(apply_mhat(g, WD_F64, o.outer_recon, mass, rh, c, t_o, 1, s));
        wd_cg_stats cs{};
        const int rc = cg_dispatch(ctx, g, mass, e, c, tol_ne, o, cs, s);
        st.iters += cs.iters;
        st.reliable_updates += cs.reliable_updates;
        if (rc != WD_OK && rc != WD_ENOCONV) return rc;
        WD_TRY(run_blas(ctx, OpAxpby<PREC_F64, PREC_F64>{F64(e), F64(x_e), 1.0, 1.0}, vh, s));
        WD_TRY(apply_mhat(g, WD_F64, o.outer_recon, mass, x_e, c, t_o, 0, s));
        WD_TRY(run_blas(ctx, OpXmyNorm<PREC_F64>{F64(bh), F64(c), F64(rh), d + 4}, vh, s));
        WD_TRY(read_scal(ctx, 4, 1, s));
        r2 = h[4];
        if (r2 <= target2) return WD_OK;
        if (!std::isfinite(r2)) return set_error(WD_ENOCONV, "CGNE: Schur residual is not finite");
        if (rc == WD_ENOCONV || st.iters >= o.maxiter) break;
        // next pass: aim at half the remaining factor, relative to this residual
        tol_ne = std::fmax(0.5 * std::sqrt(target2 / r2), 1e-15);
    }
    return set_error(WD_ENOCONV, "CGNE did not reach the Schur residual %.3e (reached %.3e)", tol,
                     std::sqrt(r2 / bh2));
}

int full_solve(wd_ctx *ctx, const wd_gauge *g, double mass, char *x, const char *b, double tol, int solver,
               const wd_cg_opts &o, wd_cg_stats &st, cudaStream_t s)
{
    const int vh = g->geo.Vh;
    const size_t h64 = half_field_bytes(vh, WD_F64);
    const char *b_e = b, *b_o = b + h64;
    char *x_e = x, *x_o = x + h64;
    double *d = ctx->d_scal, *h = ctx->h_scal;
    const double a = mass + 4.0;
    auto F64 = [&](const void *p) { return field_ref<PREC_F64>(p, vh); };
    // b^_e, held in the odd half of x until x_o is formed
    char *bh = x_o;
    WD_TRY(eo_hop(g, WD_F64, o.outer_recon, bh, b_o, b_e, WD_EVEN, 1.0, 1.0 / (2.0 * a), 0, s));
    WD_TRY(run_blas(ctx, OpNorm2<PREC_F64>{F64(b), d + 0}, 2 * vh, s));
    WD_TRY(run_blas(ctx, OpNorm2<PREC_F64>{F64(bh), d + 1}, vh, s));
    WD_TRY(read_scal(ctx, 0, 2, s));
    const double b2 = h[0], bh2 = h[1];
    st.iters = 0;
    st.reliable_updates = 0;
    if (!std::isfinite(b2) || !std::isfinite(bh2)) return set_error(WD_EINVAL, "source is not finite");
    if (!(b2 > 0.0)) {
        WD_CUDA_TRY(cudaMemsetAsync(x, 0, 2 * h64, s));
        WD_CUDA_TRY(cudaStreamSynchronize(s));
        st.true_rel_resid = 0.0;
        return WD_OK;
    }
    int rc = WD_OK;
    if (!(bh2 > 0.0)) {
        WD_CUDA_TRY(cudaMemsetAsync(x_e, 0, h64, s));
    } else {
        const double tol_hat = tol * std::sqrt(b2 / bh2);
        if (solver == WD_SOLVER_BICGSTAB) {
            rc = bicg_dispatch(ctx, g, mass, x_e, bh, tol_hat, o, st, s);
        } else {
            rc = cgne_schur(ctx, g, mass, x_e, bh, bh2, tol_hat, o, st, s);
        }
        if (rc != WD_OK && rc != WD_ENOCONV) return rc;
    }
    // x_o = (b_o + H_oe x_e / 2) / (m+4), then the true residual |b - D x| / |b|
    WD_TRY(eo_hop(g, WD_F64, o.outer_recon, x_o, x_e, b_o, WD_ODD, 1.0 / a, 1.0 / (2.0 * a), 0, s));
    char *aux = nullptr;
    WD_TRY(ctx_aux_workspace(ctx, 2 * (2 * h64 + 256), &aux));
    Bump bp{aux};
    char *dx = bp.take(2 * h64), *res = bp.take(2 * h64);
    WD_TRY(full_hop(g, WD_F64, o.outer_recon, dx, x, a, -0.5, s));
    WD_TRY(run_blas(ctx, OpXmyNorm<PREC_F64>{F64(b), F64(dx), F64(res), d + 4}, 2 * vh, s));
    WD_TRY(read_scal(ctx, 4, 1, s));
    st.true_rel_resid = std::sqrt(h[4] / b2);
    if (rc == WD_ENOCONV) return rc;
    if (!(st.true_rel_resid <= tol))
        return set_error(WD_ENOCONV, "full solve reached relative residual %.3e > %.3e", st.true_rel_resid, tol);
    return WD_OK;
}

} // namespace

} // namespace wd

using namespace wd;

extern "C" {

int bicgstab_solve(wd_ctx *ctx, const wd_gauge *g, double mass, void *x_e, const void *b_e, double tol,
                   const wd_cg_opts *opts, wd_cg_stats *stats, void *stream)
{
    clear_error();
    WD_TRY(check_solve_args(ctx, g, x_e, b_e, tol, opts));
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard dg(ctx->device);
    WD_TRY(prepare_layouts(ctx, g, *opts));
    wd_cg_stats st{};
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = bicg_dispatch(ctx, g, mass, (char *)x_e, (const char *)b_e, tol, *opts, st, (cudaStream_t)stream);
    st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    st.status = rc;
    if (stats) *stats = st;
    return rc;
}

int wilson_solve(wd_ctx *ctx, const wd_gauge *g, double mass, void *x, const void *b, double tol, int solver,
                 const wd_cg_opts *opts, wd_cg_stats *stats, void *stream)
{
    clear_error();
    WD_TRY(check_solve_args(ctx, g, x, b, tol, opts));
    if (solver != WD_SOLVER_CGNE && solver != WD_SOLVER_BICGSTAB)
        return set_error(WD_EINVAL, "solver = %d is not a wd_solver value", solver);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard dg(ctx->device);
    WD_TRY(prepare_layouts(ctx, g, *opts));
    wd_cg_stats st{};
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = full_solve(ctx, g, mass, (char *)x, (const char *)b, tol, solver, *opts, st, (cudaStream_t)stream);
    st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    st.status = rc;
    if (stats) *stats = st;
    return rc;
}

} // extern "C"
