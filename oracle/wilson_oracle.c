/*
 * FP64 CPU oracle for the Wilson-Dirac operator and its CG solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it and shares no code,
 * header, table or helper with it.
 *
 * It is the plain definition, written for readability, not speed:
 *   - fields in lexicographic array-of-structures order,
 *       site = x + Lx*(y + Ly*(z + Lz*t)),
 *       spinor double[V][4 spin][3 colour][re,im],
 *       links  double[V][4 mu][3][3][re,im]  (mu = 0,1,2,3 = x,y,z,t),
 *   - the full 4x4 Dirac matrices of the chiral basis (no spin-projection
 *     shortcut), plain 3x3 complex matrix products,
 *   - periodic boundaries by modulo arithmetic,
 *   - no FMA contraction (compiled with -ffp-contract=off).
 *
 * Passages followed (arXiv:1901.07294, Meyer et al., "SVE-enabling Lattice QCD
 * Codes"):
 *   Sec. II-A, Eq. (1): the hopping term D_h, quark field psi^{ia}_x with 4
 *     spin and 3 colour indices, SU(3) links U_{x,mu} on nearest-neighbour
 *     links, constant Dirac matrices gamma_mu.
 *   Sec. II-A: the linear system with the Dirac operator is solved by CG.
 *   The paper names no other solver; BiCGStab on Mhat and the full-system
 *   solve by even-odd reduction are the textbook steps either side of the CG
 *   path (van der Vorst 1992 for BiCGStab; reading R5 for the reduction).
 *
 * Readings where the paper is silent (each is also stated where it is used):
 *   R1 sign convention: the library's hopping sum is
 *        H psi(x) = sum_mu (1-gamma_mu) U_mu(x) psi(x+mu)
 *                        + (1+gamma_mu) U_mu(x-mu)^dagger psi(x-mu),
 *      related to Eq. (1) by D_h = gamma5 H gamma5.  Eq. (1) itself is also
 *      implemented (convention 1) so that this identity is tested.
 *   R2 normalisation: D = (m+4) - H/2 (Wilson mass term; Eq. (1) is the bare
 *      hopping term).
 *   R3 gamma basis: Hermitian Euclidean chiral basis (see gamma_basis()),
 *      gamma5 = gamma0 gamma1 gamma2 gamma3 = diag(1,1,-1,-1).
 *   R4 boundaries: periodic in all four directions.
 *   R5 even-odd: Mhat = (m+4) - H_eo H_oe / (4(m+4)) on even sites (the exact
 *      Schur complement of D), Mhat^dagger = gamma5 Mhat gamma5, CG on
 *      Mhat^dagger Mhat.
 *
 * Pins (tests, CPU only): dense-matrix brute force on 2^4 and 4x2x2x4
 * lattices, closed-form free-field plane-wave action and spectrum,
 * gamma5-hermiticity, gauge covariance, Clifford algebra of the basis, the
 * Schur-complement identity against a dense inverse, the CG solution against
 * a dense solve and the free-field momentum-space inverse; BiCGStab and the
 * full-system solve against a dense solve of D and the free-field inverse
 * D(p)^{-1} = (a - i gamma.s) / (a^2 + s^2), a = m + sum(1 - cos p), s = sin p.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* ------------------------------------------------------------------ */
/* Dirac matrices (reading R3)                                          */
/* ------------------------------------------------------------------ */
static void gamma_basis(int mu, cplx g[4][4])
{
    memset(g, 0, 16 * sizeof(cplx));
    switch (mu) {
    case 0: /* gamma_x */
        g[0][3] = I;  g[1][2] = I;  g[2][1] = -I; g[3][0] = -I;
        break;
    case 1: /* gamma_y */
        g[0][3] = -1; g[1][2] = 1;  g[2][1] = 1;  g[3][0] = -1;
        break;
    case 2: /* gamma_z */
        g[0][2] = I;  g[1][3] = -I; g[2][0] = -I; g[3][1] = I;
        break;
    case 3: /* gamma_t */
        g[0][2] = 1;  g[1][3] = 1;  g[2][0] = 1;  g[3][1] = 1;
        break;
    }
}

static void mat4_mul(cplx a[4][4], cplx b[4][4], cplx out[4][4])
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += a[i][k] * b[k][j];
            out[i][j] = s;
        }
}

/* gamma_mu for mu = 0..3; mu = 4 gives gamma5 = gamma0 gamma1 gamma2 gamma3. */
static void gamma_matrix(int mu, cplx g[4][4])
{
    if (mu < 4) {
        gamma_basis(mu, g);
        return;
    }
    cplx a[4][4], b[4][4], t[4][4];
    gamma_basis(0, a);
    for (int nu = 1; nu < 4; ++nu) {
        gamma_basis(nu, b);
        mat4_mul(a, b, t);
        memcpy(a, t, sizeof(t));
    }
    memcpy(g, a, sizeof(a));
}

/* Exported for the tests: out = double[4][4][2]. */
void oracle_gamma(int mu, double *out)
{
    cplx g[4][4];
    gamma_matrix(mu, g);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            out[2 * (4 * i + j)] = creal(g[i][j]);
            out[2 * (4 * i + j) + 1] = cimag(g[i][j]);
        }
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Lattice geometry (reading R4: periodic)                              */
/* ------------------------------------------------------------------ */
static void site_coords(const int d[4], int64_t s, int c[4])
{
    c[0] = (int)(s % d[0]); s /= d[0];
    c[1] = (int)(s % d[1]); s /= d[1];
    c[2] = (int)(s % d[2]); s /= d[2];
    c[3] = (int)s;
}

static int64_t site_index(const int d[4], const int c[4])
{
    return c[0] + (int64_t)d[0] * (c[1] + (int64_t)d[1] * (c[2] + (int64_t)d[2] * c[3]));
}

static int64_t neighbour(const int d[4], const int c[4], int mu, int step)
{
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[mu] = ((n[mu] + step) % d[mu] + d[mu]) % d[mu];
    return site_index(d, n);
}

static int site_parity(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

static int64_t volume(const int d[4]) { return (int64_t)d[0] * d[1] * d[2] * d[3]; }

/* ------------------------------------------------------------------ */
/* Hopping term                                                         */
/* ------------------------------------------------------------------ */
/*
 * out(x) = sum_mu [ P_f(mu) (x) U_mu(x)            ] psi(x+mu)
 *               + [ P_b(mu) (x) U_mu(x-mu)^dagger  ] psi(x-mu)
 * with spin matrices
 *   convention 0 (library H, reading R1): P_f = 1 - gamma_mu, P_b = 1 + gamma_mu
 *   convention 1 (Eq. (1) literally):     P_f = 1 + gamma_mu, P_b = 1 - gamma_mu
 * Only sites of parity out_parity are written (out_parity < 0: all sites);
 * the other sites of out are set to zero.  Since every neighbour of a site
 * has the opposite parity, out_parity = p gives the block H_{p,1-p}.
 */
void oracle_hop(const int dims[4], const double *links, const double *psi, double *out,
                int out_parity, int convention)
{
    const cplx *U = (const cplx *)links;
    const cplx *in = (const cplx *)psi;
    cplx *o = (cplx *)out;
    cplx Pf[4][4][4], Pb[4][4][4];
    double sf = (convention == 0) ? -1.0 : 1.0;
    for (int mu = 0; mu < 4; ++mu) {
        cplx g[4][4];
        gamma_matrix(mu, g);
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                cplx id = (a == b) ? 1.0 : 0.0;
                Pf[mu][a][b] = id + sf * g[a][b];
                Pb[mu][a][b] = id - sf * g[a][b];
            }
    }
    const int64_t V = volume(dims);
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < V; ++s) {
        int c[4];
        site_coords(dims, s, c);
        cplx acc[4][3];
        memset(acc, 0, sizeof(acc));
        if (out_parity < 0 || site_parity(c) == out_parity) {
            for (int mu = 0; mu < 4; ++mu) {
                int64_t sp = neighbour(dims, c, mu, +1);
                int64_t sm = neighbour(dims, c, mu, -1);
                const cplx *Uf = U + (s * 4 + mu) * 9;   /* U_mu(x)      */
                const cplx *Ub = U + (sm * 4 + mu) * 9;  /* U_mu(x - mu) */
                const cplx *pf = in + sp * 12;
                const cplx *pb = in + sm * 12;
                cplx wf[4][3], wb[4][3];
                /* colour: w[b][i] = sum_j U[i][j] psi[b][j]  (forward)
                 *         w[b][i] = sum_j conj(U[j][i]) psi[b][j]  (backward) */
                for (int b = 0; b < 4; ++b)
                    for (int i = 0; i < 3; ++i) {
                        cplx f = 0, g = 0;
                        for (int j = 0; j < 3; ++j) {
                            f += Uf[3 * i + j] * pf[3 * b + j];
                            g += conj(Ub[3 * j + i]) * pb[3 * b + j];
                        }
                        wf[b][i] = f;
                        wb[b][i] = g;
                    }
                /* spin: acc[a][i] += sum_b P[a][b] w[b][i] */
                for (int a = 0; a < 4; ++a)
                    for (int i = 0; i < 3; ++i) {
                        cplx t = 0;
                        for (int b = 0; b < 4; ++b) t += Pf[mu][a][b] * wf[b][i] + Pb[mu][a][b] * wb[b][i];
                        acc[a][i] += t;
                    }
            }
        }
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 3; ++i) o[s * 12 + 3 * a + i] = acc[a][i];
    }
}

/* out(x) = G psi(x) for the spin matrix G = gamma_mu (mu = 0..3) or gamma5 (mu = 4). */
void oracle_gamma_apply(int64_t V, int mu, const double *psi, double *out)
{
    cplx g[4][4];
    gamma_matrix(mu, g);
    const cplx *in = (const cplx *)psi;
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < V; ++s) {
        cplx t[4][3];
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 3; ++i) {
                cplx v = 0;
                for (int b = 0; b < 4; ++b) v += g[a][b] * in[s * 12 + 3 * b + i];
                t[a][i] = v;
            }
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 3; ++i) o[s * 12 + 3 * a + i] = t[a][i];
    }
}

/* D psi = (m+4) psi - H psi / 2   (readings R1, R2), full lattice. */
void oracle_dirac(const int dims[4], const double *links, const double *psi, double mass, double *out)
{
    const int64_t V = volume(dims);
    double *h = (double *)malloc((size_t)V * 24 * sizeof(double));
    oracle_hop(dims, links, psi, h, -1, 0);
    const double a = mass + 4.0;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < V * 24; ++k) out[k] = a * psi[k] - 0.5 * h[k];
    free(h);
}

/*
 * Even-odd Schur complement (reading R5), on full-lattice arrays whose odd
 * sites are ignored on input and set to zero on output:
 *   Mhat x_e = (m+4) x_e - H_eo H_oe x_e / (4(m+4)).
 * dagger = 1 applies Mhat^dagger = gamma5 Mhat gamma5 literally.
 */
void oracle_mhat(const int dims[4], const double *links, double mass, int dagger,
                 const double *in, double *out)
{
    const int64_t V = volume(dims);
    const size_t nb = (size_t)V * 24 * sizeof(double);
    double *src = (double *)malloc(nb);
    double *t_o = (double *)malloc(nb);
    double *s_e = (double *)malloc(nb);
    if (dagger) oracle_gamma_apply(V, 4, in, src);
    else memcpy(src, in, nb);
    oracle_hop(dims, links, src, t_o, 1, 0);   /* H_oe x_e */
    oracle_hop(dims, links, t_o, s_e, 0, 0);   /* H_eo (H_oe x_e) */
    const double a = mass + 4.0, c = 1.0 / (4.0 * (mass + 4.0));
    for (int64_t s = 0; s < V; ++s) {
        int co[4];
        site_coords(dims, s, co);
        int even = (site_parity(co) == 0);
        for (int k = 0; k < 24; ++k)
            t_o[s * 24 + k] = even ? (a * src[s * 24 + k] - c * s_e[s * 24 + k]) : 0.0;
    }
    if (dagger) oracle_gamma_apply(V, 4, t_o, out);
    else memcpy(out, t_o, nb);
    free(src); free(t_o); free(s_e);
}

/* A x = Mhat^dagger Mhat x  (the CG normal operator). */
void oracle_mdagm(const int dims[4], const double *links, double mass, const double *in, double *out)
{
    const int64_t V = volume(dims);
    double *t = (double *)malloc((size_t)V * 24 * sizeof(double));
    oracle_mhat(dims, links, mass, 0, in, t);
    oracle_mhat(dims, links, mass, 1, t, out);
    free(t);
}

/* ------------------------------------------------------------------ */
/* Conjugate gradient (Sec. II-A names CG as the solver)                 */
/* ------------------------------------------------------------------ */
static double re_dot(int64_t n, const double *a, const double *b)
{
    /* Re <a, b> = sum_k a_k b_k over interleaved re/im reals */
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/*
 * Textbook CG (Hestenes-Stiefel) on A x = b, A = Mhat^dagger Mhat, x_0 = 0.
 * When the recursively updated residual satisfies |r|/|b| <= tol the true
 * residual b - A x is computed; if that is still above tol the iteration
 * restarts from it (r = p = b - A x).  Returns the iteration count (negative
 * if maxiter was reached) and the final true relative residual.
 */
int oracle_cg(const int dims[4], const double *links, double mass, const double *b, double *x,
              double tol, int maxiter, double *true_rel_resid)
{
    const int64_t V = volume(dims), n = V * 24;
    const size_t nb = (size_t)n * sizeof(double);
    double *r = (double *)malloc(nb), *p = (double *)malloc(nb), *ap = (double *)malloc(nb);
    memset(x, 0, nb);
    memcpy(r, b, nb);
    memcpy(p, b, nb);
    const double bb = re_dot(n, b, b);
    double rr = bb;
    int it = 0, converged = 0;
    double rel = 1.0;
    if (bb == 0.0) { converged = 1; rel = 0.0; }
    while (!converged && it < maxiter) {
        oracle_mdagm(dims, links, mass, p, ap);
        ++it;
        const double alpha = rr / re_dot(n, p, ap);
        for (int64_t k = 0; k < n; ++k) {
            x[k] += alpha * p[k];
            r[k] -= alpha * ap[k];
        }
        double rr_new = re_dot(n, r, r);
        if (sqrt(rr_new / bb) <= tol) {
            oracle_mdagm(dims, links, mass, x, ap);
            for (int64_t k = 0; k < n; ++k) r[k] = b[k] - ap[k];
            rr_new = re_dot(n, r, r);
            rel = sqrt(rr_new / bb);
            if (rel <= tol) { converged = 1; break; }
            memcpy(p, r, nb);
            rr = rr_new;
            continue;
        }
        const double beta = rr_new / rr;
        for (int64_t k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
        rr = rr_new;
    }
    if (!converged) {
        oracle_mdagm(dims, links, mass, x, ap);
        for (int64_t k = 0; k < n; ++k) r[k] = b[k] - ap[k];
        rel = bb > 0.0 ? sqrt(re_dot(n, r, r) / bb) : 0.0;
    }
    if (true_rel_resid) *true_rel_resid = rel;
    free(r); free(p); free(ap);
    return converged ? it : -it;
}

/* ------------------------------------------------------------------ */
/* BiCGStab on Mhat x = b and the full-system solve D x = b            */
/* ------------------------------------------------------------------ */
/* <a, b> = sum conj(a_k) b_k over the complex entries of two real arrays of
 * n = 2 * (number of complex entries) interleaved re/im reals. */
static cplx c_dot(int64_t n, const double *a, const double *b)
{
    double re = 0.0, im = 0.0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (int64_t k = 0; k < n; k += 2) {
        re += a[k] * b[k] + a[k + 1] * b[k + 1];
        im += a[k] * b[k + 1] - a[k + 1] * b[k];
    }
    return re + I * im;
}

/* y = x + c z on interleaved complex arrays (c complex). */
static void c_axpy(int64_t n, const double *x, cplx c, const double *z, double *y)
{
    const double cr = creal(c), ci = cimag(c);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; k += 2) {
        const double zr = z[k], zi = z[k + 1];
        y[k] = x[k] + cr * zr - ci * zi;
        y[k + 1] = x[k + 1] + cr * zi + ci * zr;
    }
}

/*
 * Textbook BiCGStab (van der Vorst, SIAM J. Sci. Stat. Comput. 13 (1992) 631)
 * on Mhat x = b, x_0 = 0, shadow residual r^ = b, complex inner products.
 * Each iteration: rho = <r^, r>; beta = (rho / rho_old)(alpha / omega);
 * p = r + beta (p - omega v); v = Mhat p; alpha = rho / <r^, v>;
 * s = r - alpha v; t = Mhat s; omega = <t, s> / <t, t>;
 * x += alpha p + omega s; r = s - omega t.
 * When the iterated residual (s, or r) satisfies |.|/|b| <= tol the true
 * residual b - Mhat x is computed; if that is still above tol the iteration
 * restarts from it (r = r^ = b - Mhat x, p = v = 0, rho_old = alpha = omega = 1).
 * A zero rho, <r^, v> or <t, t> is a breakdown: the iteration restarts the same
 * way.  Arrays are full-lattice; odd sites are ignored on input and are zero on
 * output.  Returns the iteration count (negative if not converged) and the
 * final true relative residual.
 */
int oracle_bicgstab(const int dims[4], const double *links, double mass, const double *b, double *x,
                    double tol, int maxiter, double *true_rel_resid)
{
    const int64_t V = volume(dims), n = V * 24;
    const size_t nb = (size_t)n * sizeof(double);
    double *be = (double *)malloc(nb), *r = (double *)malloc(nb), *rh = (double *)malloc(nb);
    double *p = (double *)malloc(nb), *v = (double *)malloc(nb), *s = (double *)malloc(nb);
    double *t = (double *)malloc(nb), *w = (double *)malloc(nb);
    /* b restricted to even sites */
    for (int64_t q = 0; q < V; ++q) {
        int co[4];
        site_coords(dims, q, co);
        const int even = site_parity(co) == 0;
        for (int k = 0; k < 24; ++k) be[q * 24 + k] = even ? b[q * 24 + k] : 0.0;
    }
    memset(x, 0, nb);
    const double bb = creal(c_dot(n, be, be));
    int it = 0, converged = 0;
    double rel = bb > 0.0 ? 1.0 : 0.0;
    if (bb == 0.0) converged = 1;
    int restart = 1;
    cplx rho_old = 1.0, alpha = 1.0, omega = 1.0;
    while (!converged && it < maxiter) {
        if (restart) {
            oracle_mhat(dims, links, mass, 0, x, w);
            for (int64_t k = 0; k < n; ++k) r[k] = be[k] - w[k];
            memcpy(rh, r, nb);
            memset(p, 0, nb);
            memset(v, 0, nb);
            rho_old = alpha = omega = 1.0;
            restart = 0;
        }
        const cplx rho = c_dot(n, rh, r);
        if (rho == 0.0) { restart = 1; ++it; continue; }
        const cplx beta = (rho / rho_old) * (alpha / omega);
        c_axpy(n, p, -omega, v, w);          /* w = p - omega v */
        c_axpy(n, r, beta, w, p);            /* p = r + beta w */
        oracle_mhat(dims, links, mass, 0, p, v);
        ++it;
        const cplx rhv = c_dot(n, rh, v);
        if (rhv == 0.0) { restart = 1; continue; }
        alpha = rho / rhv;
        c_axpy(n, r, -alpha, v, s);          /* s = r - alpha v */
        int check = 0;
        if (sqrt(creal(c_dot(n, s, s)) / bb) <= tol) {
            c_axpy(n, x, alpha, p, x);
            check = 1;
        } else {
            oracle_mhat(dims, links, mass, 0, s, t);
            const double tt = creal(c_dot(n, t, t));
            if (tt == 0.0) { c_axpy(n, x, alpha, p, x); restart = 1; continue; }
            omega = c_dot(n, t, s) / tt;
            c_axpy(n, x, alpha, p, x);
            c_axpy(n, x, omega, s, x);
            c_axpy(n, s, -omega, t, r);      /* r = s - omega t */
            rho_old = rho;
            if (sqrt(creal(c_dot(n, r, r)) / bb) <= tol) check = 1;
        }
        if (check) {
            oracle_mhat(dims, links, mass, 0, x, w);
            for (int64_t k = 0; k < n; ++k) w[k] = be[k] - w[k];
            rel = sqrt(creal(c_dot(n, w, w)) / bb);
            if (rel <= tol) converged = 1;
            else restart = 1;
        }
    }
    if (!converged && bb > 0.0) {
        oracle_mhat(dims, links, mass, 0, x, w);
        for (int64_t k = 0; k < n; ++k) w[k] = be[k] - w[k];
        rel = sqrt(creal(c_dot(n, w, w)) / bb);
    }
    if (true_rel_resid) *true_rel_resid = rel;
    free(be); free(r); free(rh); free(p); free(v); free(s); free(t); free(w);
    return converged ? it : -it;
}

/*
 * The full system D x = b by even-odd reduction (reading R5):
 *   b^_e = b_e + H_eo b_o / (2(m+4)),
 *   Mhat x_e = b^_e  (BiCGStab above),
 *   x_o = (b_o + H_oe x_e / 2) / (m+4).
 * With this x_o the odd rows of D x = b hold exactly and the even rows leave
 * the residual b^_e - Mhat x_e, so the Schur system is solved to
 * tol |b| / |b^_e|.  Returns the BiCGStab iteration count (negative if not
 * converged) and the true relative residual |b - D x| / |b|.
 */
int oracle_solve_full(const int dims[4], const double *links, double mass, const double *b, double *x,
                      double tol, int maxiter, double *true_rel_resid)
{
    const int64_t V = volume(dims), n = V * 24;
    const size_t nb = (size_t)n * sizeof(double);
    double *bo = (double *)malloc(nb), *bh = (double *)malloc(nb), *h = (double *)malloc(nb);
    int *odd = (int *)malloc((size_t)V * sizeof(int));
    for (int64_t q = 0; q < V; ++q) {
        int co[4];
        site_coords(dims, q, co);
        odd[q] = site_parity(co);
        for (int k = 0; k < 24; ++k) bo[q * 24 + k] = odd[q] ? b[q * 24 + k] : 0.0;
    }
    const double a = mass + 4.0;
    oracle_hop(dims, links, bo, h, 0, 0);                 /* H_eo b_o on even sites */
    for (int64_t q = 0; q < V; ++q)
        for (int k = 0; k < 24; ++k)
            bh[q * 24 + k] = odd[q] ? 0.0 : b[q * 24 + k] + h[q * 24 + k] / (2.0 * a);
    const double b2 = creal(c_dot(n, b, b)), bh2 = creal(c_dot(n, bh, bh));
    int it = 0;
    if (bh2 > 0.0) {
        double rel_e = 0.0;
        it = oracle_bicgstab(dims, links, mass, bh, x, tol * sqrt(b2 / bh2), maxiter, &rel_e);
    } else {
        memset(x, 0, nb);
    }
    oracle_hop(dims, links, x, h, 1, 0);                  /* H_oe x_e on odd sites */
    for (int64_t q = 0; q < V; ++q)
        if (odd[q])
            for (int k = 0; k < 24; ++k) x[q * 24 + k] = (b[q * 24 + k] + 0.5 * h[q * 24 + k]) / a;
    if (true_rel_resid) {
        oracle_dirac(dims, links, x, mass, h);
        for (int64_t k = 0; k < n; ++k) h[k] = b[k] - h[k];
        *true_rel_resid = b2 > 0.0 ? sqrt(creal(c_dot(n, h, h)) / b2) : 0.0;
    }
    free(bo); free(bh); free(h); free(odd);
    return it;
}
