// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits, built from
// the error-free transformations of Knuth (TwoSum), Dekker (FastTwoSum) and
// the FMA-based exact product (TwoProd). Used for the forward blur
// b = psi * P_v, whose FP32 FFT rounding (absolute, scaled by the whole
// volume's norm) would swamp dim voxels of b.
//
// These steps rely on IEEE round-to-nearest FP32 adds without
// reassociation; the library is never built with fast-math.
#pragma once

#include "fft.cuh"

namespace mvd {

struct dd {
    float hi, lo;
};

__device__ __forceinline__ dd dd_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {  // needs |a| >= |b| (or a == 0)
    const float s = a + b;
    return {s, b - (s - a)};
}
// Sum without the final renormalisation: hi is the rounded sum of the high
// parts, lo collects that rounding error and both low parts (8 FP32 ops instead
// of 11). hi + lo carries the same error as the renormalised sum; |lo| may grow
// to a few ulp(hi) over chained additions, which the multiplications below
// (all ending in FastTwoSum) bring back. Where heavy cancellation leaves lo
// larger than hi, the values involved are themselves of the order of the
// operands' last bits, so the absolute error stays at that level.
__device__ __forceinline__ dd dd_add(dd x, dd y) {
    const dd s = dd_two_sum(x.hi, y.hi);
    return {s.hi, s.lo + (x.lo + y.lo)};
}
__device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd{-y.hi, -y.lo}); }
__device__ __forceinline__ dd dd_mul(dd x, dd y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return dd_fast_two_sum(p, e);
}
__device__ __forceinline__ dd dd_from(float a) { return {a, 0.f}; }

// complex double-float, 16 bytes (loads and stores as float4)
struct __align__(16) cdd {
    dd re, im;
};

__device__ __forceinline__ cdd cadd(cdd a, cdd b) { return {dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
__device__ __forceinline__ cdd csub(cdd a, cdd b) { return {dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; }
// x.y + sg * z.w with one TwoSum: both high products and their exact errors
// (TwoProd by FMA) plus the cross terms, renormalised once (19 ops).
template <int SG>
__device__ __forceinline__ dd dd_dot2(dd x, dd y, dd z, dd w) {
    const float p = x.hi * y.hi, q = z.hi * w.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    float f = fmaf(z.hi, w.hi, -q);
    f = fmaf(z.hi, w.lo, f);
    f = fmaf(z.lo, w.hi, f);
    const dd t = dd_two_sum(p, SG > 0 ? q : -q);
    return dd_fast_two_sum(t.hi, t.lo + (SG > 0 ? e + f : e - f));
}
__device__ __forceinline__ cdd cmul(cdd a, cdd b) {
    return {dd_dot2<-1>(a.re, b.re, a.im, b.im), dd_dot2<+1>(a.re, b.im, a.im, b.re)};
}
// x.y + sg * z.w as an unevaluated pair, without the final renormalisation
// (16 ops): hi the rounded sum of the high products, lo its TwoSum error
// plus the products' exact errors and cross terms. For a consumer that
// re-aligns its input anyway (the aligned line transforms).
template <int SG>
__device__ __forceinline__ dd dd_dot2_pair(dd x, dd y, dd z, dd w) {
    const float p = x.hi * y.hi, q = z.hi * w.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    float f = fmaf(z.hi, w.hi, -q);
    f = fmaf(z.hi, w.lo, f);
    f = fmaf(z.lo, w.hi, f);
    const dd t = dd_two_sum(p, SG > 0 ? q : -q);
    return {t.hi, t.lo + (SG > 0 ? e + f : e - f)};
}
__device__ __forceinline__ cdd cmul_pair(cdd a, cdd b) {
    return {dd_dot2_pair<-1>(a.re, b.re, a.im, b.im), dd_dot2_pair<+1>(a.re, b.im, a.im, b.re)};
}
__device__ __forceinline__ cdd cconj(cdd a) { return {a.re, dd{-a.im.hi, -a.im.lo}}; }
__device__ __forceinline__ cdd chalf(cdd a) {  // exact
    return {dd{0.5f * a.re.hi, 0.5f * a.re.lo}, dd{0.5f * a.im.hi, 0.5f * a.im.lo}};
}
template <int S>
__device__ __forceinline__ cdd mul_si(cdd a) {  // exact
    return S < 0 ? cdd{a.im, dd{-a.re.hi, -a.re.lo}} : cdd{dd{-a.im.hi, -a.im.lo}, a.re};
}
__device__ __forceinline__ cdd czero_dd() { return {dd{0.f, 0.f}, dd{0.f, 0.f}}; }
__device__ __forceinline__ cdd cdd_load(const cdd* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {dd{v.x, v.y}, dd{v.z, v.w}};
}
__device__ __forceinline__ cdd cdd_load_cg(const cdd* p) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
    return {dd{v.x, v.y}, dd{v.z, v.w}};
}
__device__ __forceinline__ cdd cdd_load_nc(const cdd* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {dd{v.x, v.y}, dd{v.z, v.w}};
}
__device__ __forceinline__ void cdd_store(cdd* p, cdd a) {
    *reinterpret_cast<float4*>(p) = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo);
}

// 16-byte asynchronous global -> shared copy (L2 only); with !valid nothing is
// read and the 16 bytes are zero-filled (src then only needs to be a valid
// address)
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src, bool valid) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// constant (cos, S sin) pairs as double-float: hi = fl32(c), lo = fl32(c - hi)
#define MVD_DD(c) dd{(float)(c), (float)((c) - (double)(float)(c))}

// exp(s 2 pi i m / L) from the forward table tw[m] = exp(-2 pi i m / L)
template <int S>
__device__ __forceinline__ cdd twiddle_dd(const cdd* __restrict__ tw, int m) {
    cdd w = cdd_load_nc(tw + m);
    if (S > 0) w.im = dd{-w.im.hi, -w.im.lo};
    return w;
}

// ---------------------------------------------------------------------------
// small DFTs in double-float: y[m] = sum_r v[r] exp(s 2 pi i r m / R)
// ---------------------------------------------------------------------------
template <int R, int S>
struct DftDD;

template <int S>
struct DftDD<2, S> {
    __device__ __forceinline__ static void run(cdd* v) {
        const cdd a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <int S>
struct DftDD<4, S> {
    __device__ __forceinline__ static void run(cdd* v) {
        const cdd t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        const cdd t2 = cadd(v[1], v[3]), t3 = mul_si<S>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <int S>
struct DftDD<8, S> {
    __device__ __forceinline__ static void run(cdd* v) {
        cdd e[4] = {v[0], v[2], v[4], v[6]};
        cdd o[4] = {v[1], v[3], v[5], v[7]};
        DftDD<4, S>::run(e);
        DftDD<4, S>::run(o);
        // o1 (1 + S i) h = h (re - S im, im + S re);
        // o3 (-1 + S i) h = h (-(re + S im), S re - im): one add and one product by h per part
        const dd hd = MVD_DD(0.70710678118654752440);  // sqrt(2)/2
        auto sg = [](dd x) { return S > 0 ? x : dd{-x.hi, -x.lo}; };
        const dd a1 = dd_sub(o[1].re, sg(o[1].im)), b1 = dd_add(o[1].im, sg(o[1].re));
        const dd a3 = dd_add(o[3].re, sg(o[3].im)), b3 = dd_sub(sg(o[3].re), o[3].im);
        const dd m3 = dd_mul(hd, a3);
        const cdd o1{dd_mul(hd, a1), dd_mul(hd, b1)};
        const cdd o3{dd{-m3.hi, -m3.lo}, dd_mul(hd, b3)};
        const cdd o2 = mul_si<S>(o[2]);
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

template <int S>
struct DftDD<3, S> {
    __device__ __forceinline__ static void run(cdd* v) {
        const double c = -0.5, h = 0.86602540378443864676;  // cos(2pi/3), sin(2pi/3)
        const cdd t = cadd(v[1], v[2]);
        const cdd u = csub(v[1], v[2]);
        const dd cd = MVD_DD(c), hd = MVD_DD(h);
        const cdd m = cadd(v[0], cdd{dd_mul(cd, t.re), dd_mul(cd, t.im)});
        const cdd j = mul_si<S>(cdd{dd_mul(hd, u.re), dd_mul(hd, u.im)});
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, j);
        v[2] = csub(m, j);
    }
};

template <int S>
struct DftDD<5, S> {
    __device__ __forceinline__ static void run(cdd* v) {
        const dd c1 = MVD_DD(0.30901699437494742410), c2 = MVD_DD(-0.80901699437494742410);
        const dd s1 = MVD_DD(0.95105651629515357212), s2 = MVD_DD(0.58778525229247312917);
        const cdd t1 = cadd(v[1], v[4]), u1 = csub(v[1], v[4]);
        const cdd t2 = cadd(v[2], v[3]), u2 = csub(v[2], v[3]);
        const cdd a0 = v[0];
        auto sc = [](dd k, cdd x) { return cdd{dd_mul(k, x.re), dd_mul(k, x.im)}; };
        const cdd m1 = cadd(a0, cadd(sc(c1, t1), sc(c2, t2)));
        const cdd m2 = cadd(a0, cadd(sc(c2, t1), sc(c1, t2)));
        const cdd j1 = mul_si<S>(cadd(sc(s1, u1), sc(s2, u2)));
        const cdd j2 = mul_si<S>(csub(sc(s2, u1), sc(s1, u2)));
        v[0] = cadd(a0, cadd(t1, t2));
        v[1] = cadd(m1, j1);
        v[4] = csub(m1, j1);
        v[2] = cadd(m2, j2);
        v[3] = csub(m2, j2);
    }
};

template <int S>
struct Root9<cdd, S> {
    __device__ __forceinline__ static cdd get(int m) {
        // cos, sin of 2 pi m / 9 for m = 1, 2, 4, as double-float
        const double c = m == 1 ? 0.76604444311897803520 : m == 2 ? 0.17364817766693034885 : -0.93969262078590838405;
        const double s = m == 1 ? 0.64278760968653932632 : m == 2 ? 0.98480775301220805936 : 0.34202014332566873304;
        return cdd{MVD_DD(c), MVD_DD(S * s)};
    }
};

template <int S>
struct DftDD<6, S> {
    __device__ __forceinline__ static void run(cdd* v) { dft6<mvd::DftDD, S>(v); }
};

template <int S>
struct DftDD<9, S> {
    __device__ __forceinline__ static void run(cdd* v) { dft9<mvd::DftDD, S>(v); }
};

}  // namespace mvd
