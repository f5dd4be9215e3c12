/*
 * Seeded synthetic inputs for the Wilson-Dirac operator: smoothed SU(3) gauge
 * links and Gaussian quark-field sources.
 *
 * This module is shared by the FP64 oracle and the GPU path as their common
 * input source.  It holds none of the operator's arithmetic: it only draws
 * random numbers and turns them into unitary matrices.
 *
 * Random numbers.  SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: output n of stream `seed` is mix(seed + (n+1)*0x9E3779B97F4A7C15),
 * which is exactly the n-th value the sequential generator returns after being
 * seeded with `seed`.  Every matrix and every spinor component has a fixed
 * counter, so the bytes do not depend on the thread count.  Uniforms take the
 * top 53 bits; normals come from the Box-Muller transform.
 *
 * Links ("smoothed SU(3)").  For matrix k, draw a complex Gaussian 3x3 matrix
 * A (re and im of each entry N(0,1)), form the traceless Hermitian
 * H = (A + A^dagger)/2 - tr(H)/3, and set U = exp(i eps H).  The exponential is
 * a Taylor series after scaling by 2^-s, squared back s times.  U is then
 * re-unitarised (row 0 normalised, row 1 Gram-Schmidt, row 2 = conj(row0 x
 * row1)) so that U U^dagger = 1 and det U = 1 to rounding.
 *
 * Layouts (canonical, array-of-structures, FP64, interleaved re/im):
 *   links  : double[n][3][3][2]  (for a gauge field n = 4V, matrix k = 4*site+mu)
 *   spinor : double[V][4 spin][3 colour][2]
 */
#include <math.h>
#include <stdint.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t splitmix64_at(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + (n + 1u) * GOLDEN_GAMMA;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Gaussian pair number k of stream `seed` (uses counters 2k and 2k+1). */
static void gauss_pair(uint64_t seed, uint64_t k, double *g0, double *g1)
{
    const double two53 = 9007199254740992.0;               /* 2^53 */
    double u1 = ((double)(splitmix64_at(seed, 2 * k) >> 11) + 1.0) / two53; /* (0,1] */
    double u2 = (double)(splitmix64_at(seed, 2 * k + 1) >> 11) / two53;     /* [0,1) */
    double r = sqrt(-2.0 * log(u1));
    double th = 6.283185307179586476925286766559 * u2;
    *g0 = r * cos(th);
    *g1 = r * sin(th);
}

/* Raw counter-based stream, exposed so the tests can check it against the
 * sequential definition of SplitMix64. */
uint64_t synth_splitmix64_at(uint64_t seed, uint64_t n) { return splitmix64_at(seed, n); }

/* n Gaussian N(0,1) reals: out[j] = normal number j of stream `seed`. */
void synth_gaussian(int64_t n, uint64_t seed, double *out)
{
    int64_t npair = (n + 1) / 2;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < npair; ++k) {
        double g0, g1;
        gauss_pair(seed, (uint64_t)k, &g0, &g1);
        out[2 * k] = g0;
        if (2 * k + 1 < n) out[2 * k + 1] = g1;
    }
}

/* ---- small complex 3x3 helpers (re/im split, no <complex.h>) ---- */
typedef struct { double re, im; } c64;

static void mat_mul3(const c64 a[9], const c64 b[9], c64 out[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < 3; ++k) {
                re += a[3 * i + k].re * b[3 * k + j].re - a[3 * i + k].im * b[3 * k + j].im;
                im += a[3 * i + k].re * b[3 * k + j].im + a[3 * i + k].im * b[3 * k + j].re;
            }
            out[3 * i + j].re = re;
            out[3 * i + j].im = im;
        }
}

static void reunitarise(c64 u[9])
{
    /* row 0: normalise */
    double n0 = 0.0;
    for (int j = 0; j < 3; ++j) n0 += u[j].re * u[j].re + u[j].im * u[j].im;
    n0 = 1.0 / sqrt(n0);
    for (int j = 0; j < 3; ++j) { u[j].re *= n0; u[j].im *= n0; }
    /* row 1: remove the row-0 component, normalise */
    double pr = 0.0, pi = 0.0; /* <row0, row1> = sum conj(r0) r1 */
    for (int j = 0; j < 3; ++j) {
        pr += u[j].re * u[3 + j].re + u[j].im * u[3 + j].im;
        pi += u[j].re * u[3 + j].im - u[j].im * u[3 + j].re;
    }
    for (int j = 0; j < 3; ++j) {
        u[3 + j].re -= pr * u[j].re - pi * u[j].im;
        u[3 + j].im -= pr * u[j].im + pi * u[j].re;
    }
    double n1 = 0.0;
    for (int j = 0; j < 3; ++j) n1 += u[3 + j].re * u[3 + j].re + u[3 + j].im * u[3 + j].im;
    n1 = 1.0 / sqrt(n1);
    for (int j = 0; j < 3; ++j) { u[3 + j].re *= n1; u[3 + j].im *= n1; }
    /* row 2 = conj(row0 x row1) */
    for (int k = 0; k < 3; ++k) {
        int a = (k + 1) % 3, b = (k + 2) % 3;
        double re = (u[a].re * u[3 + b].re - u[a].im * u[3 + b].im) -
                    (u[b].re * u[3 + a].re - u[b].im * u[3 + a].im);
        double im = (u[a].re * u[3 + b].im + u[a].im * u[3 + b].re) -
                    (u[b].re * u[3 + a].im + u[b].im * u[3 + a].re);
        u[6 + k].re = re;
        u[6 + k].im = -im;
    }
}

/* U = exp(i eps H) for matrix number k of stream `seed`. */
static void su3_near_identity(uint64_t seed, uint64_t k, double eps, c64 u[9])
{
    double g[18];
    for (int p = 0; p < 9; ++p) gauss_pair(seed, 9 * k + (uint64_t)p, &g[2 * p], &g[2 * p + 1]);
    c64 a[9], h[9];
    for (int e = 0; e < 9; ++e) { a[e].re = g[2 * e]; a[e].im = g[2 * e + 1]; }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { /* (A + A^dagger)/2 */
            h[3 * i + j].re = 0.5 * (a[3 * i + j].re + a[3 * j + i].re);
            h[3 * i + j].im = 0.5 * (a[3 * i + j].im - a[3 * j + i].im);
        }
    double tr = (h[0].re + h[4].re + h[8].re) / 3.0;
    h[0].re -= tr; h[4].re -= tr; h[8].re -= tr;
    h[0].im = h[4].im = h[8].im = 0.0;
    /* M = i eps H */
    c64 m[9];
    double fro = 0.0;
    for (int e = 0; e < 9; ++e) {
        m[e].re = -eps * h[e].im;
        m[e].im = eps * h[e].re;
        fro += m[e].re * m[e].re + m[e].im * m[e].im;
    }
    fro = sqrt(fro);
    int s = 0;
    while (fro > 0.25) { fro *= 0.5; ++s; }
    double sc = ldexp(1.0, -s);
    for (int e = 0; e < 9; ++e) { m[e].re *= sc; m[e].im *= sc; }
    /* Taylor series: sum_{n=0}^{18} M^n / n! */
    c64 term[9], sum[9], tmp[9];
    for (int e = 0; e < 9; ++e) { term[e].re = term[e].im = 0.0; }
    term[0].re = term[4].re = term[8].re = 1.0;
    for (int e = 0; e < 9; ++e) sum[e] = term[e];
    for (int n = 1; n <= 18; ++n) {
        mat_mul3(term, m, tmp);
        double inv = 1.0 / (double)n;
        for (int e = 0; e < 9; ++e) {
            term[e].re = tmp[e].re * inv;
            term[e].im = tmp[e].im * inv;
            sum[e].re += term[e].re;
            sum[e].im += term[e].im;
        }
    }
    for (int q = 0; q < s; ++q) {
        mat_mul3(sum, sum, tmp);
        for (int e = 0; e < 9; ++e) sum[e] = tmp[e];
    }
    reunitarise(sum);
    for (int e = 0; e < 9; ++e) u[e] = sum[e];
}

/* n SU(3) matrices, out = double[n][3][3][2]. */
void synth_su3(int64_t n, double eps, uint64_t seed, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        c64 u[9];
        su3_near_identity(seed, (uint64_t)k, eps, u);
        for (int e = 0; e < 9; ++e) {
            out[18 * k + 2 * e] = u[e].re;
            out[18 * k + 2 * e + 1] = u[e].im;
        }
    }
}
