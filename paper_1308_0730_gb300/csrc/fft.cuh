// Device-side FFT building blocks: complex helpers, radix-2/3/4/5/8 DFT
// butterflies and a shared-memory Stockham (self-sorting) driver that runs
// the same length-L transform on a batch of lines held in shared memory.
//
// Stockham stage with radix R after Ns points have been combined (Ns starts
// at 1 and is multiplied by R after each stage): for butterfly j in [0, L/R)
// with k = j mod Ns,
//   v[r] = A[j + r L/R] * exp(s 2 pi i r k / (Ns R)),   r = 0..R-1
//   v    = DFT_R(v)   (sign s)
//   B[(j / Ns) Ns R + k + r Ns] = v[r]
// which leaves the output in natural order after the last stage. s = -1 is
// the forward transform, s = +1 the (unnormalised) inverse.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace mvd {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by s*i (s = -1 forward, +1 inverse)
template <int S>
__device__ __forceinline__ float2 mul_si(float2 a) {
    return S < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// Factor the sequential update multiplies psi by, from v = c - 1 (c the view's
// back-projected ratio): with view weight w and Tikhonov lambda (one-step-late
// form, factor c / (1 + lambda psi)) it is 1 + w (c / (1 + lambda psi) - 1)
// = 1 + w (v - lambda psi) / (1 + lambda psi); plainly 1 + v. With a zero
// boundary c is first divided by the sensitivity (inv_s = 1 / s).
__device__ __forceinline__ float update_factor(float v, float psi, const float* wt, long i, float lam,
                                               const float* inv_s = nullptr) {
    if (inv_s) v = (v + 1.f) * __ldg(inv_s + i) - 1.f;
    if (!wt && lam == 0.f) return v + 1.f;
    const float w = wt ? __ldg(wt + i) : 1.f;
    return lam == 0.f ? 1.f + w * v : 1.f + w * (v - lam * psi) / (1.f + lam * psi);
}

// exp(s 2 pi i m / L) from the forward table tw[m] = exp(-2 pi i m / L)
template <int S>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int m) {
    float2 w = __ldg(tw + m);
    if (S > 0) w.y = -w.y;
    return w;
}

// ---------------------------------------------------------------------------
// small DFTs: y[m] = sum_r v[r] exp(s 2 pi i r m / R)
// ---------------------------------------------------------------------------
template <int R, int S>
struct Dft;

template <int S>
struct Dft<2, S> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <int S>
struct Dft<4, S> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        float2 t2 = cadd(v[1], v[3]), t3 = mul_si<S>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <int S>
struct Dft<8, S> {
    __device__ __forceinline__ static void run(float2* v) {
        // split into even / odd radix-4 DFTs, then combine with exp(s 2 pi i m / 8)
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, S>::run(e);
        Dft<4, S>::run(o);
        const float h = 0.70710678118654752440f;  // sqrt(2)/2
        // w1 = h (1 + s i), w2 = s i, w3 = h (-1 + s i)
        float2 o1 = make_float2(h * (o[1].x - S * o[1].y), h * (o[1].y + S * o[1].x));
        float2 o2 = mul_si<S>(o[2]);
        float2 o3 = make_float2(h * (-o[3].x - S * o[3].y), h * (-o[3].y + S * o[3].x));
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
struct Dft<3, S> {
    __device__ __forceinline__ static void run(float2* v) {
        const float c = -0.5f, h = 0.86602540378443864676f;  // cos(2pi/3), sin(2pi/3)
        float2 t = cadd(v[1], v[2]);
        float2 u = csub(v[1], v[2]);
        float2 m = make_float2(v[0].x + c * t.x, v[0].y + c * t.y);
        float2 j = mul_si<S>(cscale(u, h));
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, j);
        v[2] = csub(m, j);
    }
};

template <int S>
struct Dft<5, S> {
    __device__ __forceinline__ static void run(float2* v) {
        const float c1 = 0.30901699437494742410f;   // cos(2pi/5)
        const float c2 = -0.80901699437494742410f;  // cos(4pi/5)
        const float s1 = 0.95105651629515357212f;   // sin(2pi/5)
        const float s2 = 0.58778525229247312917f;   // sin(4pi/5)
        float2 t1 = cadd(v[1], v[4]), u1 = csub(v[1], v[4]);
        float2 t2 = cadd(v[2], v[3]), u2 = csub(v[2], v[3]);
        float2 a0 = v[0];
        float2 m1 = make_float2(a0.x + c1 * t1.x + c2 * t2.x, a0.y + c1 * t1.y + c2 * t2.y);
        float2 m2 = make_float2(a0.x + c2 * t1.x + c1 * t2.x, a0.y + c2 * t1.y + c1 * t2.y);
        float2 j1 = mul_si<S>(make_float2(s1 * u1.x + s2 * u2.x, s1 * u1.y + s2 * u2.y));
        float2 j2 = mul_si<S>(make_float2(s2 * u1.x - s1 * u2.x, s2 * u1.y - s1 * u2.y));
        v[0] = make_float2(a0.x + t1.x + t2.x, a0.y + t1.y + t2.y);
        v[1] = cadd(m1, j1);
        v[4] = csub(m1, j1);
        v[2] = cadd(m2, j2);
        v[3] = csub(m2, j2);
    }
};

// ---------------------------------------------------------------------------
// composite small DFTs, generic in the element type T (float2 here, complex
// double-float in dd.cuh) and in the family D of prime-length DFTs
// ---------------------------------------------------------------------------

// Prime-factor (Good-Thomas) DFTs of lengths 6 = 2 x 3 and 10 = 2 x 5: input
// n = (N2 n1 + 2 n2) mod N with N1 = 2, output k with k = k1 (mod 2) and
// k = k2 (mod N2); the exponent n k then splits into a 2-point and an
// N2-point part, so there are no twiddles between the two. The 2-point DFTs
// over n1 are the sums (k1 = 0) and differences (k1 = 1) of the pairs below.
template <template <int, int> class D, int S, typename T>
__device__ __forceinline__ void dft6(T* v) {
    T a[3] = {cadd(v[0], v[3]), cadd(v[2], v[5]), cadd(v[4], v[1])};
    T b[3] = {csub(v[0], v[3]), csub(v[2], v[5]), csub(v[4], v[1])};
    D<3, S>::run(a);
    D<3, S>::run(b);
    v[0] = a[0], v[4] = a[1], v[2] = a[2];
    v[3] = b[0], v[1] = b[1], v[5] = b[2];
}

template <template <int, int> class D, int S, typename T>
__device__ __forceinline__ void dft10(T* v) {
    T a[5] = {cadd(v[0], v[5]), cadd(v[2], v[7]), cadd(v[4], v[9]), cadd(v[6], v[1]), cadd(v[8], v[3])};
    T b[5] = {csub(v[0], v[5]), csub(v[2], v[7]), csub(v[4], v[9]), csub(v[6], v[1]), csub(v[8], v[3])};
    D<5, S>::run(a);
    D<5, S>::run(b);
    v[0] = a[0], v[6] = a[1], v[2] = a[2], v[8] = a[3], v[4] = a[4];
    v[5] = b[0], v[1] = b[1], v[7] = b[2], v[3] = b[3], v[9] = b[4];
}

// exp(s 2 pi i m / 9) as an element of type T (specialised per type)
template <typename T, int S>
struct Root9;

template <int S>
struct Root9<float2, S> {
    __device__ __forceinline__ static float2 get(int m) {
        // cos, sin of 2 pi m / 9 for m = 1, 2, 4
        const float c = m == 1 ? 0.76604444311897803520f : m == 2 ? 0.17364817766693034885f : -0.93969262078590838405f;
        const float s = m == 1 ? 0.64278760968653932632f : m == 2 ? 0.98480775301220805936f : 0.34202014332566873304f;
        return make_float2(c, S * s);
    }
};

// Length-9 DFT as 3 x 3 (Cooley-Tukey): 3-point DFTs over n1 of x[3 n1 + n2]
// (c_n2), twiddles exp(s 2 pi i n2 k1 / 9), 3-point DFTs over n2, output at
// k1 + 3 k2.
template <template <int, int> class D, int S, typename T>
__device__ __forceinline__ void dft9(T* v) {
    T c0[3] = {v[0], v[3], v[6]};
    T c1[3] = {v[1], v[4], v[7]};
    T c2[3] = {v[2], v[5], v[8]};
    D<3, S>::run(c0);
    D<3, S>::run(c1);
    D<3, S>::run(c2);
    c1[1] = cmul(c1[1], Root9<T, S>::get(1));
    c2[1] = cmul(c2[1], Root9<T, S>::get(2));
    c1[2] = cmul(c1[2], Root9<T, S>::get(2));
    c2[2] = cmul(c2[2], Root9<T, S>::get(4));
    T r0[3] = {c0[0], c1[0], c2[0]};
    T r1[3] = {c0[1], c1[1], c2[1]};
    T r2[3] = {c0[2], c1[2], c2[2]};
    D<3, S>::run(r0);
    D<3, S>::run(r1);
    D<3, S>::run(r2);
    v[0] = r0[0], v[3] = r0[1], v[6] = r0[2];
    v[1] = r1[0], v[4] = r1[1], v[7] = r1[2];
    v[2] = r2[0], v[5] = r2[1], v[8] = r2[2];
}

template <int S>
struct Dft<6, S> {
    __device__ __forceinline__ static void run(float2* v) { dft6<mvd::Dft, S>(v); }
};

template <int S>
struct Dft<10, S> {
    __device__ __forceinline__ static void run(float2* v) { dft10<mvd::Dft, S>(v); }
};

template <int S>
struct Dft<9, S> {
    __device__ __forceinline__ static void run(float2* v) { dft9<mvd::Dft, S>(v); }
};

// ---------------------------------------------------------------------------
// one Stockham butterfly (see the file header)
// ---------------------------------------------------------------------------

// floor(n / d) for 0 <= n and n + d < 2^22, from inv = the FP32 reciprocal of d
// (correctly rounded): (n + 1/2) / d lies at least 1/(2d) from an integer and
// the two roundings move it by less than (n/d + 1) 2^-23, so the truncation is
// exact. Replaces the integer divisions of the butterfly indexing.
__device__ __forceinline__ int small_div(int n, float inv) { return __float2int_rz(((float)n + 0.5f) * inv); }

// Per-stage constants of the Stockham indexing: nb = L / R butterflies per
// line, Ns combined so far.
struct StageIdx {
    int nb, Ns;
    float inv_nb, inv_ns;
    __device__ __forceinline__ StageIdx(int L, int R, int ns)
        : nb(L / R), Ns(ns), inv_nb(1.0f / (float)(L / R)), inv_ns(1.0f / (float)ns) {}
};

template <int R, int S>
__device__ __forceinline__ void stockham_bfly(const float2* __restrict__ A, float2* __restrict__ B, int j,
                                              const StageIdx& si, const float2* __restrict__ tw) {
    const int jq = small_div(j, si.inv_ns);
    const int k = j - jq * si.Ns;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = A[j + r * si.nb];
    if (si.Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twiddle<S>(tw, (r - 1) * si.Ns + k));
    }
    Dft<R, S>::run(v);
    const int d = jq * si.Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) B[d + r * si.Ns] = v[r];
}

// All butterflies of one stage (radix R, Ns combined so far) over `nlines`
// lines, spread over the block's threads.
template <int R, int S>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ A, float2* __restrict__ B, int nlines,
                                               int ls, int L, int Ns, const float2* __restrict__ tw) {
    const StageIdx si(L, R, Ns);
    const int total = nlines * si.nb;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int line = small_div(t, si.inv_nb);
        const int j = t - line * si.nb;
        stockham_bfly<R, S>(A + line * ls, B + line * ls, j, si, tw);
    }
}

// Transforms `nlines` lines of length p.L stored at A + line*ls (line stride
// ls >= L), using B (same shape) as the ping-pong buffer. All threads of the
// block take part; the call begins and ends with the data synchronised.
// Returns the buffer (A or B) that holds the result.
// Twiddles: p.tw is the axis's natural table (w^m, m < L), followed by its
// radix-8 and radix-16 stage-ordered copies and then by its copy in the
// stage order of this plan (p.tw + 3L): stage s >= 1 (Ns combined before it,
// radix R) keeps w^(r k L / (Ns R)) at (earlier stages' entries) +
// (r - 1) Ns + k, so consecutive butterflies read consecutive entries.
template <int S>
__device__ float2* fft_lines(float2* A, float2* B, int nlines, int ls, const FftPlan& p) {
    int Ns = 1;
    const float2* tw = p.tw + 3 * p.L;
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.radix[s];
        switch (R) {
            case 8: stockham_stage<8, S>(A, B, nlines, ls, p.L, Ns, tw); break;
            case 4: stockham_stage<4, S>(A, B, nlines, ls, p.L, Ns, tw); break;
            case 2: stockham_stage<2, S>(A, B, nlines, ls, p.L, Ns, tw); break;
            case 3: stockham_stage<3, S>(A, B, nlines, ls, p.L, Ns, tw); break;
            case 6: stockham_stage<6, S>(A, B, nlines, ls, p.L, Ns, tw); break;
            case 9: stockham_stage<9, S>(A, B, nlines, ls, p.L, Ns, tw); break;
            case 10: stockham_stage<10, S>(A, B, nlines, ls, p.L, Ns, tw); break;
            default: stockham_stage<5, S>(A, B, nlines, ls, p.L, Ns, tw); break;
        }
        if (s > 0) tw += (R - 1) * Ns;
        __syncthreads();
        float2* t = A;
        A = B;
        B = t;
        Ns *= R;
    }
    return A;
}

// Global loads of data that other blocks of the same launch may have written
// (the persistent batch kernel) must bypass L1: CO selects L2-only loads.
template <bool CO>
__device__ __forceinline__ float2 ld2(const float2* p) {
    if constexpr (CO)
        return __ldcg(p);
    else
        return *p;
}
template <bool CO>
__device__ __forceinline__ float ld1(const float* p) {
    if constexpr (CO)
        return __ldcg(p);
    else
        return *p;
}

}  // namespace mvd
