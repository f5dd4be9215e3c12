// Device-side building blocks: storage traits, 16-byte plane loads/stores,
// complex multiply-add, link reconstruction.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace wd {

enum { PREC_F64 = 0, PREC_F32 = 1, PREC_F16 = 2, PREC_BF16 = 3, PREC_DF = 4 };

// First statement of every kernel launched through wd_launch, which launches
// with programmatic dependent launch.  The wait returns once all grids this
// one depends on programmatically have completed and their memory operations
// are visible (at once for a kernel launched without such a dependency); no
// access to global memory may precede it, so an early start can neither read
// a result before it is written nor overwrite an input its predecessor still
// reads.  The trigger then lets the next kernel be dispatched as soon as every
// block of this one has passed it: at most two grids of a chain are resident,
// the running one and its waiting successor.
__device__ __forceinline__ void grid_dependency_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---- double-word FP32 ("double-float") arithmetic ---------------------------
// A value is the unevaluated sum hi + lo of two FP32 numbers, |lo| <= ulp(hi)
// after normalisation: 48 significand bits from FP32 instructions, for a part
// whose FP64 rate is 1/64 of its FP32 rate.  The building blocks are the
// error-free transformations of Knuth (TwoSum), Dekker (Fast2Sum) and the FMA
// form of TwoProduct; the operations are the "sloppy" double-word sum and the
// double-word product of Joldes, Muller and Popescu (ACM TOMS 44, 2017), and
// fma(x, y, z) = z + x y is one step of the compensated dot product of Ogita,
// Rump and Oishi (SIAM J. Sci. Comput. 26, 2005): the rounding errors of the
// running sum and of the products gather in lo, which is left unnormalised
// between steps.  Every error is of order 2^-48 times the magnitude of the
// terms involved, which is what a residual b - A x needs.  Intrinsics keep the
// compiler from contracting or reordering the error terms.
// Conversions between FP64 and FP32 issue on the FP64 pipe, so the ones
// around the double-word arithmetic and in the FP64 BLAS work on the bit
// patterns instead.  The rare operands they do not cover go to functions kept
// out of line: a branch, where an inlined fallback would be predicated and
// cost its FP64 instructions on every element.
static __device__ __noinline__ double f32_to_f64_rare(float f) { return (double)f; }

// f32_to_f64: exact widening of a float (subnormal, inf, NaN out of line)
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned u = __float_as_uint(f), e = (u >> 23) & 0xffu;
    if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));   // +-0
    if (e == 0u || e == 0xffu) return f32_to_f64_rare(f);
    const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e - 127u + 1023u) << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

// the FP64 route of the double -> double-word split, out of line
static __device__ __noinline__ float2 f64_split_rare(double v)
{
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(int v) : hi((float)v), lo(0.0f) {}
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __device__ explicit df(float v) : hi(v), lo(0.0f) {}
    // hi = v rounded to 24 significant bits, to nearest even (an integer add
    // below bit 29 of the pattern, whose carry moves into the exponent: the
    // FP32 rounding of v), lo = v - hi, a signed remainder of at most 28 bits
    // rounded to 24 (|lo| <=
    // ulp(hi)/2, error <= 2^-24 |lo| <= 2^-48 |v|); integer operations and one
    // integer-to-float conversion while both parts are normal FP32 numbers
    // (2^-74 <= |v| < 2^126), and for +-0; otherwise (tiny, huge, inf, NaN)
    // hi = RN(v), lo = RN(v - hi) in FP64, out of line.
    __device__ explicit df(double v)
    {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
        if ((b << 1) == 0ull) {   // +-0
            hi = __uint_as_float((unsigned)(b >> 32));
            lo = 0.0f;
        } else if (e >= 949u && e <= 1148u) {
            const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
            const unsigned long long r = (b + 0x0fffffffull + ((b >> 29) & 1ull)) & ~0x1fffffffull;
            const unsigned er = (unsigned)(r >> 52) & 0x7ffu;
            hi = __uint_as_float(sign | ((er - 896u) << 23) | ((unsigned)(r >> 29) & 0x7fffffu));
            // |v| - |hi| in units of 2^(e - 1075), the last significand bit of v
            const int d = (int)(long long)((b & 0x7fffffffffffffffull) - (r & 0x7fffffffffffffffull));
            // as a float its exponent field is 127 + log2|d|; adding e - 1075
            // (>= -126 here) keeps it a normal number
            lo = d ? __uint_as_float((__float_as_uint(__int2float_rn(d)) + ((e - 1075u) << 23)) ^ sign) : 0.0f;
        } else {
            const float2 t = f64_split_rare(v);
            hi = t.x;
            lo = t.y;
        }
    }
    __device__ explicit operator double() const { return f32_to_f64(hi) + f32_to_f64(lo); }
    __device__ explicit operator float() const { return __fadd_rn(hi, lo); }
};
// Value conversion between compute types: float -> double by bit pattern,
// everything else as a cast.
template <typename To, typename From> __device__ __forceinline__ To to_real(From v) { return (To)v; }
template <> __device__ __forceinline__ double to_real<double, float>(float v) { return f32_to_f64(v); }

// s + e = a + b exactly, s = RN(a + b)
__device__ __forceinline__ df df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// the same for |a| >= |b| (or a = 0)
__device__ __forceinline__ df df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_normalize(df x) { return df_two_sum(x.hi, x.lo); }
__device__ __forceinline__ df operator-(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df operator+(df x, df y)
{
    const df s = df_two_sum(x.hi, y.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return df_fast_two_sum(p, e);
}
// sign factors of the projectors (s = +1 or -1 only)
__device__ __forceinline__ df operator*(int s, df x) { return s < 0 ? -x : x; }
__device__ __forceinline__ df &operator+=(df &x, df y) { return x = x + y; }
__device__ __forceinline__ df &operator-=(df &x, df y) { return x = x - y; }
// z + x y, one compensated dot-product step (result not normalised).  The
// global float and double fma stay visible beside this overload.
using ::fma;
__device__ __forceinline__ df fma(df x, df y, df z)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    const df s = df_two_sum(z.hi, p);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(e, z.lo))};
}

// Storage traits.  `real` is the compute type; `per16` reals fit in one 16-byte
// vector; half types carry a per-site FP32 scale plane for spinors.
template <int P> struct Prec;
template <> struct Prec<PREC_F64> { using real = double; static constexpr int per16 = 2;  static constexpr int bytes = 8; static constexpr bool scaled = false; };
template <> struct Prec<PREC_F32> { using real = float;  static constexpr int per16 = 4;  static constexpr int bytes = 4; static constexpr bool scaled = false; };
template <> struct Prec<PREC_F16> { using real = float;  static constexpr int per16 = 8;  static constexpr int bytes = 2; static constexpr bool scaled = true; };
template <> struct Prec<PREC_BF16>{ using real = float;  static constexpr int per16 = 8;  static constexpr int bytes = 2; static constexpr bool scaled = true; };
template <> struct Prec<PREC_DF>  { using real = df;     static constexpr int per16 = 2;  static constexpr int bytes = 8; static constexpr bool scaled = false; };

template <typename T> struct cpx { T re, im; };

// Storage precision of the links that go with fields of precision P.  Link
// entries are bounded by 1 in magnitude, so they need no exponent range; for
// BF16 fields they are kept in FP16, which has 3 more mantissa bits.
__host__ __device__ constexpr int link_prec(int p) { return p == PREC_BF16 ? PREC_F16 : p; }

// z + x*y and z + conj(x)*y with real FMAs (the two complex multiply-add
// forms of Sec. III-D, Eq. (2), which SVE gets from a pair of FCMLA).
template <typename T> __device__ __forceinline__ cpx<T> cfma(cpx<T> x, cpx<T> y, cpx<T> z)
{
    z.re = fma(x.re, y.re, z.re); z.re = fma(-x.im, y.im, z.re);
    z.im = fma(x.re, y.im, z.im); z.im = fma(x.im, y.re, z.im);
    return z;
}
template <typename T> __device__ __forceinline__ cpx<T> cfma_conj(cpx<T> x, cpx<T> y, cpx<T> z)
{
    z.re = fma(x.re, y.re, z.re); z.re = fma(x.im, y.im, z.re);
    z.im = fma(x.re, y.im, z.im); z.im = fma(-x.im, y.re, z.im);
    return z;
}
template <typename T> __device__ __forceinline__ cpx<T> cmul(cpx<T> x, cpx<T> y)
{
    cpx<T> z;
    z.re = x.re * y.re; z.re = fma(-x.im, y.im, z.re);
    z.im = x.re * y.im; z.im = fma(x.im, y.re, z.im);
    return z;
}
template <typename T> __device__ __forceinline__ cpx<T> cmul_conj(cpx<T> x, cpx<T> y)
{
    cpx<T> z;
    z.re = x.re * y.re; z.re = fma(x.im, y.im, z.re);
    z.im = x.re * y.im; z.im = fma(-x.im, y.re, z.im);
    return z;
}

// ---- 16-byte vector <-> reals -------------------------------------------
__device__ __forceinline__ uint4 ldg16(const void *p)
{
    return __ldg(reinterpret_cast<const uint4 *>(p));
}
// As ldg16, without allocating the line in L1.
__device__ __forceinline__ uint4 ldg16_na(const void *p)
{
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p));
    return r;
}
__device__ __forceinline__ void stg16(void *p, uint4 v) { *reinterpret_cast<uint4 *>(p) = v; }

// Hint: bring the 128-byte line holding p into L2 (no register result).
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int P> __device__ __forceinline__ void unpack16(uint4 w, typename Prec<P>::real *r, float scale);
template <> __device__ __forceinline__ void unpack16<PREC_F64>(uint4 w, double *r, float)
{
    r[0] = __hiloint2double(w.y, w.x);
    r[1] = __hiloint2double(w.w, w.z);
}
template <> __device__ __forceinline__ void unpack16<PREC_F32>(uint4 w, float *r, float)
{
    r[0] = __uint_as_float(w.x); r[1] = __uint_as_float(w.y);
    r[2] = __uint_as_float(w.z); r[3] = __uint_as_float(w.w);
}
template <> __device__ __forceinline__ void unpack16<PREC_F16>(uint4 w, float *r, float s)
{
    const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __half2 h = *reinterpret_cast<const __half2 *>(&u[k]);
        float2 f = __half22float2(h);
        r[2 * k] = f.x * s; r[2 * k + 1] = f.y * s;
    }
}
template <> __device__ __forceinline__ void unpack16<PREC_BF16>(uint4 w, float *r, float s)
{
    const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&u[k]);
        float2 f = __bfloat1622float2(h);
        r[2 * k] = f.x * s; r[2 * k + 1] = f.y * s;
    }
}

// ---- 16-bit values read straight from their 32-bit storage words ----------
// H selects the low (0: the real part) or high (1: the imaginary part) half of
// a word that holds two 16-bit values.  h16_f32 converts one exactly; h16_add
// and h16_sub take one operand as stored: sm_100 and later have FP32 additions
// with a 16-bit operand (exact widening, one rounding), so x + y and x - y
// cost one instruction where a conversion and an addition took two, with the
// same result bit for bit.
template <int P, int H> __device__ __forceinline__ float h16_f32(unsigned w)
{
    if constexpr (P == PREC_BF16) return __uint_as_float(H ? (w & 0xffff0000u) : (w << 16));
    else {
        float r;
        if constexpr (H) asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; cvt.f32.f16 %0, h;}" : "=f"(r) : "r"(w));
        else asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; cvt.f32.f16 %0, l;}" : "=f"(r) : "r"(w));
        return r;
    }
}
// value(H of w) + c
template <int P, int H> __device__ __forceinline__ float h16_add(unsigned w, float c)
{
    float r;
    if constexpr (P == PREC_BF16) {
        if constexpr (H) asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; add.rn.f32.bf16 %0, h, %2;}" : "=f"(r) : "r"(w), "f"(c));
        else asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; add.rn.f32.bf16 %0, l, %2;}" : "=f"(r) : "r"(w), "f"(c));
    } else {
        if constexpr (H) asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; add.rn.f32.f16 %0, h, %2;}" : "=f"(r) : "r"(w), "f"(c));
        else asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; add.rn.f32.f16 %0, l, %2;}" : "=f"(r) : "r"(w), "f"(c));
    }
    return r;
}
// value(H of w) - c
template <int P, int H> __device__ __forceinline__ float h16_sub(unsigned w, float c)
{
    float r;
    if constexpr (P == PREC_BF16) {
        if constexpr (H) asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; sub.rn.f32.bf16 %0, h, %2;}" : "=f"(r) : "r"(w), "f"(c));
        else asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; sub.rn.f32.bf16 %0, l, %2;}" : "=f"(r) : "r"(w), "f"(c));
    } else {
        if constexpr (H) asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; sub.rn.f32.f16 %0, h, %2;}" : "=f"(r) : "r"(w), "f"(c));
        else asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; sub.rn.f32.f16 %0, l, %2;}" : "=f"(r) : "r"(w), "f"(c));
    }
    return r;
}
// u + SIGMA v for u = half HU of wu and v = half HV of wv (SIGMA = +1 or -1):
// the widened operand is the one the instruction cannot take as stored.
template <int P, int HU, int HV, int SIGMA> __device__ __forceinline__ float h16_pm(unsigned wu, unsigned wv)
{
    if constexpr (SIGMA > 0) return h16_add<P, HV>(wv, h16_f32<P, HU>(wu));
    else return h16_sub<P, HU>(wu, h16_f32<P, HV>(wv));
}

template <> __device__ __forceinline__ void unpack16<PREC_DF>(uint4 w, df *r, float)
{
    r[0] = {__uint_as_float(w.x), __uint_as_float(w.y)};
    r[1] = {__uint_as_float(w.z), __uint_as_float(w.w)};
}

template <int P> __device__ __forceinline__ uint4 pack16(const typename Prec<P>::real *r, float inv_scale);
template <> __device__ __forceinline__ uint4 pack16<PREC_F64>(const double *r, float)
{
    uint4 w;
    w.x = __double2loint(r[0]); w.y = __double2hiint(r[0]);
    w.z = __double2loint(r[1]); w.w = __double2hiint(r[1]);
    return w;
}
template <> __device__ __forceinline__ uint4 pack16<PREC_F32>(const float *r, float)
{
    return make_uint4(__float_as_uint(r[0]), __float_as_uint(r[1]), __float_as_uint(r[2]), __float_as_uint(r[3]));
}
// stored normalised: hi = RN(hi + lo)
template <> __device__ __forceinline__ uint4 pack16<PREC_DF>(const df *r, float)
{
    const df a = df_normalize(r[0]), b = df_normalize(r[1]);
    return make_uint4(__float_as_uint(a.hi), __float_as_uint(a.lo), __float_as_uint(b.hi), __float_as_uint(b.lo));
}
template <> __device__ __forceinline__ uint4 pack16<PREC_F16>(const float *r, float is)
{
    unsigned u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __half2 h = __floats2half2_rn(r[2 * k] * is, r[2 * k + 1] * is);
        u[k] = *reinterpret_cast<unsigned *>(&h);
    }
    return make_uint4(u[0], u[1], u[2], u[3]);
}
template <> __device__ __forceinline__ uint4 pack16<PREC_BF16>(const float *r, float is)
{
    unsigned u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __nv_bfloat162 h = __floats2bfloat162_rn(r[2 * k] * is, r[2 * k + 1] * is);
        u[k] = *reinterpret_cast<unsigned *>(&h);
    }
    return make_uint4(u[0], u[1], u[2], u[3]);
}

// ---- spinor fields ------------------------------------------------------
// Half field: planes of 16-byte vectors, plane k at byte offset k*Vh*16; half
// types then hold an FP32 scale plane.
template <int P> struct Spinor {
    using real = typename Prec<P>::real;
    static constexpr int nplane = 24 / Prec<P>::per16;
    static constexpr size_t site_bytes = 24 * Prec<P>::bytes + (Prec<P>::scaled ? 4 : 0);

    __device__ static __forceinline__ void prefetch(const char *f, int vh, int i)
    {
#pragma unroll
        for (int k = 0; k < nplane; ++k) prefetch_l2(f + ((size_t)k * vh + i) * 16);
        if (Prec<P>::scaled) prefetch_l2(reinterpret_cast<const float *>(f + (size_t)nplane * vh * 16) + i);
    }

    // The stored values without the per-site scale, which is returned (1 for
    // unscaled types); lets a linear consumer apply the scale once at the end.
    __device__ static __forceinline__ float load_unscaled(const char *f, int vh, int i, real (&v)[24])
    {
        float s = 1.0f;
        if (Prec<P>::scaled) s = __ldg(reinterpret_cast<const float *>(f + (size_t)nplane * vh * 16) + i);
#pragma unroll
        for (int k = 0; k < nplane; ++k) {
            uint4 w = ldg16(f + ((size_t)k * vh + i) * 16);
            unpack16<P>(w, v + k * Prec<P>::per16, 1.0f);
        }
        return s;
    }

    // 16-bit types: the twelve storage words (spin s, colour c in word 3s+c,
    // real part low) and the per-site scale.
    __device__ static __forceinline__ float load_words(const char *f, int vh, int i, unsigned (&u)[12])
    {
        static_assert(Prec<P>::scaled, "16-bit storage only");
        const float s = __ldg(reinterpret_cast<const float *>(f + (size_t)nplane * vh * 16) + i);
#pragma unroll
        for (int k = 0; k < nplane; ++k) {
            const uint4 w = ldg16(f + ((size_t)k * vh + i) * 16);
            u[4 * k] = w.x; u[4 * k + 1] = w.y; u[4 * k + 2] = w.z; u[4 * k + 3] = w.w;
        }
        return s;
    }

    __device__ static __forceinline__ void load(const char *f, int vh, int i, real (&v)[24])
    {
        float s = 1.0f;
        if (Prec<P>::scaled) s = __ldg(reinterpret_cast<const float *>(f + (size_t)nplane * vh * 16) + i);
#pragma unroll
        for (int k = 0; k < nplane; ++k) {
            uint4 w = ldg16(f + ((size_t)k * vh + i) * 16);
            unpack16<P>(w, v + k * Prec<P>::per16, s);
        }
    }
    __device__ static __forceinline__ void store(char *f, int vh, int i, const real (&v)[24])
    {
        float is = 1.0f;
        if (Prec<P>::scaled) {
            float m = 0.0f;
#pragma unroll
            for (int k = 0; k < 24; ++k) m = fmaxf(m, fabsf((float)v[k]));
            reinterpret_cast<float *>(f + (size_t)nplane * vh * 16)[i] = m;
            is = m > 0.0f ? 1.0f / m : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < nplane; ++k) stg16(f + ((size_t)k * vh + i) * 16, pack16<P>(v + k * Prec<P>::per16, is));
    }
};

// ---- gauge links --------------------------------------------------------
// Per (parity, mu): `nmain` planes of 16-byte vectors, then a tail plane with
// the remaining reals (8 or 4 bytes per site) when RECON*bytes is not a
// multiple of 16.  Reals are the row-major matrix entries (re, im), the first
// RECON of the 18.
template <int P, int RECON> struct Link {
    using real = typename Prec<P>::real;
    static constexpr int per16 = Prec<P>::per16;
    static constexpr int nmain = RECON / per16;
    static constexpr int ntail = RECON % per16;   // reals in the tail plane
    static constexpr size_t site_bytes = (size_t)RECON * Prec<P>::bytes;

    __device__ static __forceinline__ void prefetch(const char *blk, int vh, int i)
    {
#pragma unroll
        for (int k = 0; k < nmain; ++k) prefetch_l2(blk + ((size_t)k * vh + i) * 16);
        if constexpr (ntail > 0) prefetch_l2(blk + (size_t)nmain * vh * 16 + (size_t)i * ntail * Prec<P>::bytes);
    }

    // NA: the 16-byte planes bypass L1 allocation (a link read once per call
    // would only evict neighbour spinors that other threads of the block reuse)
    template <bool NA = false>
    __device__ static __forceinline__ void load_raw(const char *blk, int vh, int i, real (&u)[18])
    {
#pragma unroll
        for (int k = 0; k < nmain; ++k) {
            const char *a = blk + ((size_t)k * vh + i) * 16;
            const uint4 w = NA ? ldg16_na(a) : ldg16(a);
            unpack16<P>(w, u + k * per16, 1.0f);
        }
        if constexpr (ntail > 0) {
            const char *tp = blk + (size_t)nmain * vh * 16;
            if constexpr (P == PREC_F32) {          // 2 floats
                float2 t = __ldg(reinterpret_cast<const float2 *>(tp) + i);
                u[nmain * per16] = t.x; u[nmain * per16 + 1] = t.y;
            } else if constexpr (ntail == 2) {      // 2 halves
                unsigned t = __ldg(reinterpret_cast<const unsigned *>(tp) + i);
                float2 f;
                if constexpr (P == PREC_F16) f = __half22float2(*reinterpret_cast<__half2 *>(&t));
                else f = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&t));
                u[nmain * per16] = f.x; u[nmain * per16 + 1] = f.y;
            } else {                                // 4 halves
                uint2 t = __ldg(reinterpret_cast<const uint2 *>(tp) + i);
                float2 f0, f1;
                if constexpr (P == PREC_F16) {
                    f0 = __half22float2(*reinterpret_cast<__half2 *>(&t.x));
                    f1 = __half22float2(*reinterpret_cast<__half2 *>(&t.y));
                } else {
                    f0 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&t.x));
                    f1 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&t.y));
                }
                u[nmain * per16] = f0.x; u[nmain * per16 + 1] = f0.y;
                u[nmain * per16 + 2] = f1.x; u[nmain * per16 + 3] = f1.y;
            }
        }
    }

    // Full 3x3 matrix; with RECON = 12 the third row is conj(row0 x row1).
    template <bool NA = false>
    __device__ static __forceinline__ void load(const char *blk, int vh, int i, cpx<real> (&U)[3][3])
    {
        real u[18];
        load_raw<NA>(blk, vh, i, u);
#pragma unroll
        for (int r = 0; r < (RECON == 18 ? 3 : 2); ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) { U[r][c].re = u[6 * r + 2 * c]; U[r][c].im = u[6 * r + 2 * c + 1]; }
        if constexpr (RECON == 12) {
            // row 2 = conj(row 0 x row 1): U[2][c] = conj(U0a U1b - U0b U1a) with
            // a = c+1, b = c+2 (mod 3).  FP32 (latency-bound kernels): two
            // products and a difference, chains of depth 3; FP64 and the 16-bit
            // formats (arithmetic-bound): one four-term FMA chain per part, 8
            // operations instead of 10 (measured on 32^4: FP32 full 81.4 against
            // 84.2 us; FP16 full 69.9 against 71.3 us).
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int a = (c + 1) % 3, b = (c + 2) % 3;
                const cpx<real> x = U[0][a], y = U[1][b], z = U[0][b], w = U[1][a];
                if constexpr (P == PREC_F32) {
                    const cpx<real> t = cmul(x, y), s = cmul(z, w);
                    U[2][c].re = t.re - s.re;
                    U[2][c].im = -(t.im - s.im);
                } else {
                    real re = x.re * y.re;
                    re = fma(-x.im, y.im, re);
                    re = fma(-z.re, w.re, re);
                    re = fma(z.im, w.im, re);
                    real im = -(x.re * y.im);
                    im = fma(-x.im, y.re, im);
                    im = fma(z.re, w.im, im);
                    im = fma(z.im, w.re, im);
                    U[2][c].re = re;
                    U[2][c].im = im;
                }
            }
        }
    }
};

} // namespace wd
