// Aligned double-float: the arithmetic of the register-resident FFT lines.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers, as in dd.cuh,
// with one more invariant: every hi of a line is an integer multiple of the
// line's quantum q, a power of two chosen from the line's largest value so
// that |hi| <= 2^19 q. Sums and differences of such values stay multiples of
// q, and while they stay below 2^24 q they are exact in FP32: an addition
// costs one FP32 add on the high parts and one on the low parts, where a
// double-float addition needs Knuth's TwoSum (six operations) and two more.
// Only products leave the grid; each is rounded back onto it (the rounding
// constant 1.5 * 2^23 * q moves the product's bits below q out of the high
// part) and the exact remainder, from one FMA, goes to the low part.
//
// Error: the low parts are plain FP32 of magnitude about q, so each operation
// adds an absolute error of about 2^-24 q = 2^-43 times the line's bound,
// against about 2^-48 of each value in double-float: well inside what the
// convolution needs (its error is absolute against the line's norm anyway).
//
// Growth: a radix-8 butterfly takes components bounded by 2^19 q to at most
// 9.7 times that, and the next stage's twiddle product to 13.7 times; the next
// stage therefore runs at quantum 16 q, where the bound is again 2^19. The
// magic-constant rounding needs |x| <= 2^22 q and the butterfly's sums stay
// below 2^23 q.
//
// Every operation uses the _rn intrinsics, which the compiler neither
// contracts into FMAs nor reassociates.
#pragma once

#include "dd.cuh"

namespace mvd {

#if defined(__CUDA_ARCH__)
#define ADF_ADD(a, b) __fadd_rn((a), (b))
#define ADF_SUB(a, b) __fsub_rn((a), (b))
#define ADF_MUL(a, b) __fmul_rn((a), (b))
#define ADF_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#else
#define ADF_ADD(a, b) ((a) + (b))
#define ADF_SUB(a, b) ((a) - (b))
#define ADF_MUL(a, b) ((a) * (b))
#define ADF_FMA(a, b, c) fmaf((a), (b), (c))
#endif

// the rounding constant 1.5 * 2^23 * q of quantum q = 2^e, as FP32 bits
__host__ __device__ __forceinline__ float adf_const_exp2(int e) {
    // 1.5 * 2^(e + 23): biased exponent e + 23 + 127, mantissa 0.5
    int be = e + 150;
    be = be < 1 ? 1 : (be > 254 ? 254 : be);
#if defined(__CUDA_ARCH__)
    return __int_as_float((be << 23) | 0x400000);
#else
    union {
        int i;
        float f;
    } u;
    u.i = (be << 23) | 0x400000;
    return u.f;
#endif
}

// exponent e of the quantum q = 2^e for values bounded by m (|x| <= m):
// m < 2^E with E the exponent just above m, q = 2^(E - H), so m < 2^H q
template <int H = 19>
__host__ __device__ __forceinline__ int adf_exp_for(float m) {
#if defined(__CUDA_ARCH__)
    const int bits = __float_as_int(m);
#else
    union {
        float f;
        int i;
    } u;
    u.f = m;
    const int bits = u.i;
#endif
    int be = (bits >> 23) & 0xff;  // m in [2^(be-127), 2^(be-126))
    if (be < 40) be = 40;          // zero and tiny lines: q far below anything they hold
    return be - 126 - H;
}

// rounding onto the grid of the constant c: nearest multiple of q, |x| <= 2^22 q
__host__ __device__ __forceinline__ float adf_round(float x, float c) { return ADF_SUB(ADF_ADD(x, c), c); }

// any pair -> aligned on c's grid (|x.hi| <= 2^22 q); 4 ops
__host__ __device__ __forceinline__ dd adf_align(dd x, float c) {
    const float h = adf_round(x.hi, c);
    return {h, ADF_ADD(ADF_SUB(x.hi, h), x.lo)};
}
__host__ __device__ __forceinline__ dd adf_add(dd a, dd b) { return {ADF_ADD(a.hi, b.hi), ADF_ADD(a.lo, b.lo)}; }
__host__ __device__ __forceinline__ dd adf_sub(dd a, dd b) { return {ADF_SUB(a.hi, b.hi), ADF_SUB(a.lo, b.lo)}; }
__host__ __device__ __forceinline__ dd adf_neg(dd a) { return {-a.hi, -a.lo}; }

// a * k (k a double-float constant), aligned on c's grid; 6 ops. The FMA
// gives the exact product minus the rounded high part (at most 3q/4, so its
// own rounding is below 2^-24 q); a.lo * k.lo (below 2^-24 q) is dropped.
__host__ __device__ __forceinline__ dd adf_mulk(dd a, dd k, float c) {
    const float h = adf_round(ADF_MUL(a.hi, k.hi), c);
    float r = ADF_FMA(a.hi, k.hi, -h);
    r = ADF_FMA(a.hi, k.lo, r);
    r = ADF_FMA(a.lo, k.hi, r);
    return {h, r};
}

// x * w (w a double-float twiddle), aligned on c's grid; 28 ops
__host__ __device__ __forceinline__ cdd adf_cmul(cdd x, cdd w, float c) {
    const dd p1 = adf_mulk(x.re, w.re, c), p2 = adf_mulk(x.im, w.im, c);
    const dd p3 = adf_mulk(x.re, w.im, c), p4 = adf_mulk(x.im, w.re, c);
    return {adf_sub(p1, p2), adf_add(p3, p4)};
}
__host__ __device__ __forceinline__ cdd adf_calign(cdd x, float c) { return {adf_align(x.re, c), adf_align(x.im, c)}; }
__host__ __device__ __forceinline__ cdd adf_cadd(cdd a, cdd b) { return {adf_add(a.re, b.re), adf_add(a.im, b.im)}; }
__host__ __device__ __forceinline__ cdd adf_csub(cdd a, cdd b) { return {adf_sub(a.re, b.re), adf_sub(a.im, b.im)}; }
template <int S>
__host__ __device__ __forceinline__ cdd adf_mul_si(cdd a) {  // times S i, exact
    return S < 0 ? cdd{a.im, adf_neg(a.re)} : cdd{adf_neg(a.im), a.re};
}

// largest |hi| component of a value (the line bound; the low parts are below
// the previous grid's quantum and the bound has a factor 2 of slack)
__host__ __device__ __forceinline__ float adf_absmax(cdd x, float m) {
    return fmaxf(m, fmaxf(fabsf(x.re.hi), fabsf(x.im.hi)));
}

// small DFTs y[m] = sum_r v[r] exp(s 2 pi i r m / R) on aligned values
// (inputs bounded by 2^19 q, c the grid's constant)
template <int R, int S>
struct DftA;

template <int S>
struct DftA<2, S> {
    __host__ __device__ __forceinline__ static void run(cdd* v, float) {
        const cdd a = v[0], b = v[1];
        v[0] = adf_cadd(a, b);
        v[1] = adf_csub(a, b);
    }
};

template <int S>
struct DftA<4, S> {
    __host__ __device__ __forceinline__ static void run(cdd* v, float) {
        const cdd t0 = adf_cadd(v[0], v[2]), t1 = adf_csub(v[0], v[2]);
        const cdd t2 = adf_cadd(v[1], v[3]), t3 = adf_mul_si<S>(adf_csub(v[1], v[3]));
        v[0] = adf_cadd(t0, t2);
        v[2] = adf_csub(t0, t2);
        v[1] = adf_cadd(t1, t3);
        v[3] = adf_csub(t1, t3);
    }
};

template <int S>
struct DftA<8, S> {
    __host__ __device__ __forceinline__ static void run(cdd* v, float c) {
        cdd e[4] = {v[0], v[2], v[4], v[6]};
        cdd o[4] = {v[1], v[3], v[5], v[7]};
        DftA<4, S>::run(e, c);
        DftA<4, S>::run(o, c);
        // o1 (1 + S i) h and o3 (-1 + S i) h with h = sqrt(2)/2: one exact
        // sum and one product by h per part
        const dd hd = MVD_DD(0.70710678118654752440);
        const dd o1s = S > 0 ? o[1].im : adf_neg(o[1].im), o1r = S > 0 ? o[1].re : adf_neg(o[1].re);
        const dd o3s = S > 0 ? o[3].im : adf_neg(o[3].im), o3r = S > 0 ? o[3].re : adf_neg(o[3].re);
        const dd a1 = adf_sub(o[1].re, o1s), b1 = adf_add(o[1].im, o1r);
        const dd a3 = adf_add(o[3].re, o3s), b3 = adf_sub(o3r, o[3].im);
        const cdd w1{adf_mulk(a1, hd, c), adf_mulk(b1, hd, c)};
        const cdd w3{adf_neg(adf_mulk(a3, hd, c)), adf_mulk(b3, hd, c)};
        const cdd w2 = adf_mul_si<S>(o[2]);
        v[0] = adf_cadd(e[0], o[0]);
        v[4] = adf_csub(e[0], o[0]);
        v[1] = adf_cadd(e[1], w1);
        v[5] = adf_csub(e[1], w1);
        v[2] = adf_cadd(e[2], w2);
        v[6] = adf_csub(e[2], w2);
        v[3] = adf_cadd(e[3], w3);
        v[7] = adf_csub(e[3], w3);
    }
};

// growth of the grid exponent over a stage of radix R (the bound after the
// butterfly and the next twiddle product, over 2^19 q, rounded up)
__host__ __device__ constexpr int adf_stage_shift(int R) { return R == 8 ? 4 : (R == 4 ? 3 : 2); }

// ---------------------------------------------------------------------------
// Mixed radix (the shared-memory Stockham lines). These run with inputs
// bounded by 2^18 q (one more bit of headroom: the 3 x 3 length-9 butterfly's
// second products reach 8.5 times its input bound) and the generic growth
// bound: a radix-R butterfly and the next twiddle take components bounded by
// B to at most R sqrt(2) B.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int adf_gen_shift(int R) {
    return R == 2 ? 2 : (R <= 5 ? 3 : 4);  // ceil(log2(R sqrt 2)) for R = 2..10
}

// a * k for an FP32-exact constant k, aligned on c's grid; 4 ops
__host__ __device__ __forceinline__ dd adf_mulf(dd a, float k, float c) {
    const float h = adf_round(ADF_MUL(a.hi, k), c);
    return {h, ADF_FMA(a.lo, k, ADF_FMA(a.hi, k, -h))};
}
__host__ __device__ __forceinline__ cdd adf_cmulk(cdd a, dd k, float c) {
    return {adf_mulk(a.re, k, c), adf_mulk(a.im, k, c)};
}

template <int S>
struct DftA<3, S> {
    __host__ __device__ __forceinline__ static void run(cdd* v, float c) {
        const cdd t = adf_cadd(v[1], v[2]);
        const cdd u = adf_csub(v[1], v[2]);
        const dd hd = MVD_DD(0.86602540378443864676);  // sin(2 pi / 3)
        const cdd m = adf_cadd(v[0], cdd{adf_mulf(t.re, -0.5f, c), adf_mulf(t.im, -0.5f, c)});
        const cdd j = adf_mul_si<S>(adf_cmulk(u, hd, c));
        v[0] = adf_cadd(v[0], t);
        v[1] = adf_cadd(m, j);
        v[2] = adf_csub(m, j);
    }
};

template <int S>
struct DftA<5, S> {
    __host__ __device__ __forceinline__ static void run(cdd* v, float c) {
        const dd c1 = MVD_DD(0.30901699437494742410), c2 = MVD_DD(-0.80901699437494742410);
        const dd s1 = MVD_DD(0.95105651629515357212), s2 = MVD_DD(0.58778525229247312917);
        const cdd t1 = adf_cadd(v[1], v[4]), u1 = adf_csub(v[1], v[4]);
        const cdd t2 = adf_cadd(v[2], v[3]), u2 = adf_csub(v[2], v[3]);
        const cdd a0 = v[0];
        const cdd m1 = adf_cadd(a0, adf_cadd(adf_cmulk(t1, c1, c), adf_cmulk(t2, c2, c)));
        const cdd m2 = adf_cadd(a0, adf_cadd(adf_cmulk(t1, c2, c), adf_cmulk(t2, c1, c)));
        const cdd j1 = adf_mul_si<S>(adf_cadd(adf_cmulk(u1, s1, c), adf_cmulk(u2, s2, c)));
        const cdd j2 = adf_mul_si<S>(adf_csub(adf_cmulk(u1, s2, c), adf_cmulk(u2, s1, c)));
        v[0] = adf_cadd(a0, adf_cadd(t1, t2));
        v[1] = adf_cadd(m1, j1);
        v[4] = adf_csub(m1, j1);
        v[2] = adf_cadd(m2, j2);
        v[3] = adf_csub(m2, j2);
    }
};

// length 6 as 2 x 3 with coprime factors (Good-Thomas): no twiddles between
template <int S>
struct DftA<6, S> {
    __host__ __device__ __forceinline__ static void run(cdd* v, float c) {
        cdd a[3] = {adf_cadd(v[0], v[3]), adf_cadd(v[2], v[5]), adf_cadd(v[4], v[1])};
        cdd b[3] = {adf_csub(v[0], v[3]), adf_csub(v[2], v[5]), adf_csub(v[4], v[1])};
        DftA<3, S>::run(a, c);
        DftA<3, S>::run(b, c);
        v[0] = a[0], v[4] = a[1], v[2] = a[2];
        v[3] = b[0], v[1] = b[1], v[5] = b[2];
    }
};

// length 9 as 3 x 3 (Cooley-Tukey) with the internal twiddles exp(s 2 pi i m / 9)
template <int S>
struct DftA<9, S> {
    __host__ __device__ __forceinline__ static cdd root(int m) {
        const double cr = m == 1 ? 0.76604444311897803520 : m == 2 ? 0.17364817766693034885 : -0.93969262078590838405;
        const double si = m == 1 ? 0.64278760968653932632 : m == 2 ? 0.98480775301220805936 : 0.34202014332566873304;
        return cdd{MVD_DD(cr), MVD_DD(S * si)};
    }
    __host__ __device__ __forceinline__ static void run(cdd* v, float c) {
        cdd c0[3] = {v[0], v[3], v[6]};
        cdd c1[3] = {v[1], v[4], v[7]};
        cdd c2[3] = {v[2], v[5], v[8]};
        DftA<3, S>::run(c0, c);
        DftA<3, S>::run(c1, c);
        DftA<3, S>::run(c2, c);
        c1[1] = adf_cmul(c1[1], root(1), c);
        c2[1] = adf_cmul(c2[1], root(2), c);
        c1[2] = adf_cmul(c1[2], root(2), c);
        c2[2] = adf_cmul(c2[2], root(4), c);
        cdd r0[3] = {c0[0], c1[0], c2[0]};
        cdd r1[3] = {c0[1], c1[1], c2[1]};
        cdd r2[3] = {c0[2], c1[2], c2[2]};
        DftA<3, S>::run(r0, c);
        DftA<3, S>::run(r1, c);
        DftA<3, S>::run(r2, c);
        v[0] = r0[0], v[3] = r0[1], v[6] = r0[2];
        v[1] = r1[0], v[4] = r1[1], v[7] = r1[2];
        v[2] = r2[0], v[5] = r2[1], v[8] = r2[2];
    }
};

}  // namespace mvd
