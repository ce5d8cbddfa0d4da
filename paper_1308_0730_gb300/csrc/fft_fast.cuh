// Register-resident line FFT with a compile-time plan.
//
// A line of length L (a power of two, 16 <= L <= 4096) is held by TPL = L/16
// threads, thread t owning the 16 elements t + TPL*q, q = 0..15 ("natural"
// distribution). The Stockham stages of the plan (radix 16 while 16 divides
// the remaining length, then one radix 2, 4 or 8 stage) work on registers:
// stage (R, Ns) butterfly j reads elements j + r*L/R and, for a thread
// holding butterflies j = t + TPL*m, those are exactly its own elements
// m + r*(16/R). Between stages the outputs go through a padded shared-memory
// line (one write, one read per element); the last stage leaves its outputs
// in natural order in registers, so a pass can load its input straight from
// global memory into the first stage and store the last stage's registers
// straight back.
#pragma once

#include "fft.cuh"

namespace mvd {

// 16-point DFT as 4 x 4: radix-4 over n1 for each n2, twiddle w^(n2 k1),
// radix-4 over n2 for each k1 (n = 4 n1 + n2, k = k1 + 4 k2).
template <int S>
struct Dft<16, S> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 a[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            float2 x[4] = {v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]};
            Dft<4, S>::run(x);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = x[k1];
        }
        // w^m = cos(2 pi m / 16) + S i sin(2 pi m / 16)
        const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
        const float h = 0.70710678118654752440f;
        // (n2, k1) = (1,1) m=1 ; (1,2) m=2 ; (1,3) m=3 ; (2,1) m=2 ; (2,2) m=4 ; (2,3) m=6 ;
        //            (3,1) m=3 ; (3,2) m=6 ; (3,3) m=9
        a[1][1] = cmul(a[1][1], make_float2(c1, S * s1));
        a[1][2] = cmul(a[1][2], make_float2(h, S * h));
        a[1][3] = cmul(a[1][3], make_float2(s1, S * c1));
        a[2][1] = cmul(a[2][1], make_float2(h, S * h));
        a[2][2] = mul_si<S>(a[2][2]);
        a[2][3] = cmul(a[2][3], make_float2(-h, S * h));
        a[3][1] = cmul(a[3][1], make_float2(s1, S * c1));
        a[3][2] = cmul(a[3][2], make_float2(-h, S * h));
        a[3][3] = cmul(a[3][3], make_float2(-c1, -S * s1));
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 x[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
            Dft<4, S>::run(x);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = x[k2];
        }
    }
};

constexpr int kE = 16;  // elements per thread

__host__ __device__ constexpr int plan_n16(int L) {
    int n = 0;
    while (L % 16 == 0 && L >= 16) {
        L /= 16;
        ++n;
    }
    return n;
}
__host__ __device__ constexpr int plan_rem(int L) {
    while (L % 16 == 0 && L >= 16) L /= 16;
    return L;  // 1, 2, 4 or 8 for a power of two
}
__host__ __device__ constexpr int plan_radix(int L, int s) {
    return s < plan_n16(L) ? 16 : (s == plan_n16(L) && plan_rem(L) > 1 ? plan_rem(L) : 0);
}
__host__ __device__ constexpr int plan_nst(int L) { return plan_n16(L) + (plan_rem(L) > 1 ? 1 : 0); }
__host__ __device__ constexpr bool fast_length(int L) {
    return L >= 16 && L <= 4096 && (L & (L - 1)) == 0;
}

// Twiddles in stage order: the FP32 natural table of a length L (w^m, m < L)
// is followed by its radix-8 stage-ordered copy (the 8-point-per-thread
// lines) and then its radix-16 one (these lines), where stage s >= 1 (NS
// points combined before it, radix R) keeps w^(r k L / (NS R)) at
// tw_stage_off16(L, s) + (r - 1) NS + k: a warp's consecutive k read
// consecutive entries.
__host__ __device__ constexpr int tw_stage_off16(int L, int ST) {
    int off = 0, ns = 1;
    for (int s = 0; s < ST; ++s) {
        const int R = plan_radix(L, s);
        if (s > 0) off += (R - 1) * ns;
        ns *= R;
    }
    return off;
}

// padded shared-memory index of element i of a line: one pad slot per 16
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
// line stride in float2: L + L/16 (+1 to shift lines across banks)
__host__ __device__ constexpr int line_stride(int L) { return L + L / 16 + 1; }

template <int L, int S, bool WARP_LOCAL>
struct LineFFT {
    static constexpr int TPL = L / kE;
    static constexpr int NST = plan_nst(L);

    __device__ __forceinline__ static void sync() {
        if (WARP_LOCAL && TPL <= 32)
            __syncwarp();
        else
            __syncthreads();
    }

    template <int ST, int NS>
    __device__ __forceinline__ static void stage(float2 (&v)[kE], float2* sm, int t, const float2* __restrict__ tw) {
        if constexpr (ST < NST) {
            constexpr int R = plan_radix(L, ST);
            constexpr int B = kE / R;  // butterflies per thread
            constexpr bool LAST = (ST == NST - 1);
#pragma unroll
            for (int m = 0; m < B; ++m) {
                float2 x[R];
#pragma unroll
                for (int r = 0; r < R; ++r) x[r] = v[m + r * B];
                const int j = t + TPL * m;
                const int k = j % NS;
                if (NS > 1) {
                    constexpr int OFF = tw_stage_off16(L, ST);
#pragma unroll
                    for (int r = 1; r < R; ++r) x[r] = cmul(x[r], twiddle<S>(tw + 2 * L, OFF + (r - 1) * NS + k));
                }
                Dft<R, S>::run(x);
                if (LAST) {
#pragma unroll
                    for (int r = 0; r < R; ++r) v[m + r * B] = x[r];
                } else {
                    const int d = (j / NS) * NS * R + k;
#pragma unroll
                    for (int r = 0; r < R; ++r) sm[pad16(d + r * NS)] = x[r];
                }
            }
            if constexpr (!LAST) {
                sync();
#pragma unroll
                for (int q = 0; q < kE; ++q) v[q] = sm[pad16(t + TPL * q)];
                sync();
                stage<ST + 1, NS * R>(v, sm, t, tw);
            }
        }
    }

    // v: natural distribution in and out; sm: this line's exchange buffer
    __device__ __forceinline__ static void run(float2 (&v)[kE], float2* sm, int t, const float2* __restrict__ tw) {
        stage<0, 1>(v, sm, t, tw);
    }
};

}  // namespace mvd
