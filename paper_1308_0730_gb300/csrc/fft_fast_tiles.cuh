// Tile-level device functions of the register-resident FFT passes
// (power-of-two line lengths), shared by the per-volume kernels
// (fft_fast.cu) and the persistent batch kernel (batch.cu). A tile is what
// one 256-thread block handles. CO = true turns loads of data written inside
// the same launch (spectrum, estimate) into L2 loads, as the batch kernel
// requires.
#pragma once

#include "dd.cuh"
#include "fft_fast.cuh"

namespace mvd {

constexpr int kFastThreads = 256;

// tile sizes: x rows per tile, y lines per tile, z columns per tile
__host__ __device__ constexpr int fast_x_rows(int L) { return 2 * (kFastThreads / (L / kE)); }
__host__ __device__ constexpr int fast_y_lines(int L) { return kFastThreads / (L / kE); }
__host__ __device__ constexpr int fast_z_cols(int L) {
    return (kFastThreads / (L / kE)) >= 8 ? kFastThreads / (L / kE) : 8;
}
__host__ __device__ constexpr size_t fast_x_smem(int L) { return (size_t)fast_x_rows(L) * line_stride(L) * sizeof(float2); }
__host__ __device__ constexpr size_t fast_y_smem(int L) { return (size_t)fast_y_lines(L) * line_stride(L) * sizeof(float2); }
__host__ __device__ constexpr size_t fast_z_smem(int L) { return (size_t)fast_z_cols(L) * line_stride(L) * sizeof(float2); }

// y pass: Xh*Z contiguous lines of length Y; lines of one warp are adjacent
template <int L, int S, bool CO>
__device__ __forceinline__ void fast_y_tile(float2* __restrict__ spec, long nlines, const float2* __restrict__ tw,
                                            long tile, float2* sm) {
    using F = LineFFT<L, S, true>;
    constexpr int TPL = F::TPL;
    constexpr int LPC = kFastThreads / TPL;
    const int li = threadIdx.x / TPL, t = threadIdx.x - li * TPL;
    const long line = tile * LPC + li;
    const bool ok = line < nlines;
    float2* g = spec + line * L;
    float2 v[kE];
#pragma unroll
    for (int q = 0; q < kE; ++q) v[q] = ok ? ld2<CO>(g + t + TPL * q) : make_float2(0.f, 0.f);
    F::run(v, sm + li * line_stride(L), t, tw);
    if (ok) {
#pragma unroll
        for (int q = 0; q < kE; ++q) g[t + TPL * q] = v[q];
    }
}

// z pass: Q lines (consecutive y) of one kx plane; thread = q + Q * t so each
// warp reads rows of consecutive y. Needs Q * L/16 threads per block.
template <int L, bool MUL, bool CO>
__device__ __forceinline__ void fast_z_tile(float2* __restrict__ spec, const float2* __restrict__ K, int Y, long YZ,
                                            int ntiles_y, float scale, const float2* __restrict__ tw, long tile,
                                            float2* sm) {
    constexpr int TPL = L / kE;
    constexpr int Q = fast_z_cols(L);
    const int q = threadIdx.x % Q, t = threadIdx.x / Q;
    const int kx = (int)(tile / ntiles_y);
    const int y0 = (int)(tile - (long)kx * ntiles_y) * Q;
    const bool ok = y0 + q < Y;
    const long base = (long)kx * YZ + y0 + q;
    float2* line_sm = sm + q * line_stride(L);
    float2 v[kE];
#pragma unroll
    for (int i = 0; i < kE; ++i) v[i] = ok ? ld2<CO>(spec + base + (long)(t + TPL * i) * Y) : make_float2(0.f, 0.f);
    LineFFT<L, -1, false>::run(v, line_sm, t, tw);
    if (MUL) {
#pragma unroll
        for (int i = 0; i < kE; ++i) {
            const float2 k = ok ? __ldg(K + base + (long)(t + TPL * i) * Y) : make_float2(0.f, 0.f);
            v[i] = cmul(v[i], k);
        }
        __syncthreads();  // the exchange buffer is reused by the inverse transform
        LineFFT<L, +1, false>::run(v, line_sm, t, tw);
    } else {
#pragma unroll
        for (int i = 0; i < kE; ++i) v[i] = cscale(v[i], scale);
    }
    if (ok) {
#pragma unroll
        for (int i = 0; i < kE; ++i) spec[base + (long)(t + TPL * i) * Y] = v[i];
    }
}

// x passes: P pairs of rows per tile (rows rho0+p and rho0+P+p form pair p)
struct XFast {
    const float* src;
    float2* spec;
    const float* phi;
    float* psi;
    long YZ;
    float eps;
    const float2* tw;
    const float* wt;   // when set, the update applies the fraction wt of the change (partial overlap)
    float lam;         // Tikhonov regularisation of the update (0 = none)
    const float* inv_s;  // zero boundary: 1 / sensitivity of the update's view, or none
};

// write the packed forward spectra (natural order in registers) as the two
// half spectra of each pair, coalesced over rows
template <int L>
__device__ __forceinline__ void x_store_halves(const XFast& a, float2 (&v)[kE], float2* sm, int p, int t, long rho0,
                                               int nrows) {
    constexpr int TPL = L / kE, P = kFastThreads / TPL, LS = line_stride(L), XH = L / 2 + 1;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kE; ++q) sm[p * LS + pad16(t + TPL * q)] = v[q];
    __syncthreads();
    constexpr int NTOT = XH * 2 * P, NIT = (NTOT + kFastThreads - 1) / kFastThreads;
#pragma unroll
    for (int i = 0; i < NIT; ++i) {
        const int idx = threadIdx.x + i * kFastThreads;
        const int k = idx / (2 * P), row = idx - k * 2 * P;
        if (idx >= NTOT || row >= nrows) continue;
        const int pp = row < P ? row : row - P;
        const float2 zk = sm[pp * LS + pad16(k)];
        const float2 zm = cconj(sm[pp * LS + pad16(k == 0 ? 0 : L - k)]);
        float2 val;
        if (row < P) {
            val = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
        } else {
            const float2 d = csub(zk, zm);
            val = make_float2(0.5f * d.y, -0.5f * d.x);
        }
        a.spec[(long)k * a.YZ + rho0 + row] = val;
    }
}

// read both half spectra of each pair and build Z = A + i B (natural order)
template <int L, bool CO>
__device__ __forceinline__ void x_load_packed(const XFast& a, float2 (&v)[kE], float2* sm, int p, int t, long rho0,
                                              int nrows) {
    constexpr int TPL = L / kE, P = kFastThreads / TPL, LS = line_stride(L), XH = L / 2 + 1;
    constexpr int NTOT = XH * 2 * P, NIT = (NTOT + kFastThreads - 1) / kFastThreads;
    // rows < P -> line p (A), rows >= P -> line P + p (B); all loads of a
    // thread are issued before the first shared-memory store
    float2 tmp[NIT];
#pragma unroll
    for (int i = 0; i < NIT; ++i) {
        const int idx = threadIdx.x + i * kFastThreads;
        const int k = idx / (2 * P), row = idx - k * 2 * P;
        tmp[i] = make_float2(0.f, 0.f);
        if (idx < NTOT && row < nrows) {
            const long at = (long)k * a.YZ + rho0 + row;
            tmp[i] = ld2<CO>(a.spec + at);
        }
    }
#pragma unroll
    for (int i = 0; i < NIT; ++i) {
        const int idx = threadIdx.x + i * kFastThreads;
        const int k = idx / (2 * P), row = idx - k * 2 * P;
        if (idx < NTOT) sm[row * LS + pad16(k)] = tmp[i];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kE; ++q) {
        const int k = t + TPL * q;
        if (k <= L / 2) {
            const float2 A = sm[p * LS + pad16(k)], B = sm[(P + p) * LS + pad16(k)];
            v[q] = make_float2(A.x - B.y, A.y + B.x);
        } else {
            const float2 A = sm[p * LS + pad16(L - k)], B = sm[(P + p) * LS + pad16(L - k)];
            v[q] = make_float2(A.x + B.y, B.x - A.y);  // conj(A) + i conj(B)
        }
    }
    __syncthreads();
}

template <int L, bool CO>
__device__ __forceinline__ void fast_x_forward_tile(const XFast& a, long tile, float2* sm) {
    constexpr int TPL = L / kE, P = kFastThreads / TPL, LS = line_stride(L);
    const int p = threadIdx.x / TPL, t = threadIdx.x - p * TPL;
    const long rho0 = tile * 2 * P;
    const int nrows = (int)min((long)2 * P, a.YZ - rho0);
    const bool oka = p < nrows, okb = P + p < nrows;
    const float* ra = a.src + (rho0 + p) * L;
    const float* rb = a.src + (rho0 + P + p) * L;
    float2 v[kE];
#pragma unroll
    for (int q = 0; q < kE; ++q) {
        const int n = t + TPL * q;
        v[q] = make_float2(oka ? ld1<CO>(ra + n) : 0.f, okb ? ld1<CO>(rb + n) : 0.f);
    }
    LineFFT<L, -1, true>::run(v, sm + p * LS, t, a.tw);
    x_store_halves<L>(a, v, sm, p, t, rho0, nrows);
}

// MODE 0: ratio -> forward ; 1: psi update ; 2: plain real output ;
// 4: acc *= c (the combined update's product of view factors; acc in a.psi)
template <int L, int MODE, bool CO>
__device__ __forceinline__ void fast_x_inverse_tile(const XFast& a, long tile, float2* sm) {
    constexpr int TPL = L / kE, P = kFastThreads / TPL, LS = line_stride(L);
    const int p = threadIdx.x / TPL, t = threadIdx.x - p * TPL;
    const long rho0 = tile * 2 * P;
    const int nrows = (int)min((long)2 * P, a.YZ - rho0);
    const bool oka = p < nrows, okb = P + p < nrows;
    float2 v[kE];
    x_load_packed<L, CO>(a, v, sm, p, t, rho0, nrows);
    const long ra = (rho0 + p) * L, rb = (rho0 + P + p) * L;
    // the epilogue's operand rows (phi for the ratio, psi for the update) are
    // fetched now so that their loads overlap the inverse transform
    float2 w[kE];
    if (MODE == 0) {
#pragma unroll
        for (int q = 0; q < kE; ++q) {
            const int n = t + TPL * q;
            w[q] = make_float2(oka ? __ldg(a.phi + ra + n) : 0.f, okb ? __ldg(a.phi + rb + n) : 0.f);
        }
    } else if (MODE == 1 || MODE == 4) {
#pragma unroll
        for (int q = 0; q < kE; ++q) {
            const int n = t + TPL * q;
            w[q] = make_float2(oka ? ld1<CO>(a.psi + ra + n) : 0.f, okb ? ld1<CO>(a.psi + rb + n) : 0.f);
        }
    }
    LineFFT<L, +1, true>::run(v, sm + p * LS, t, a.tw);
    if (MODE == 0) {
#pragma unroll
        for (int q = 0; q < kE; ++q) {
            // r - 1 (see the generic ratio pass): the update adds the 1 back
            const float xa = oka ? w[q].x / fmaxf(v[q].x, a.eps) - 1.f : 0.f;
            const float xb = okb ? w[q].y / fmaxf(v[q].y, a.eps) - 1.f : 0.f;
            v[q] = make_float2(xa, xb);
        }
        LineFFT<L, -1, true>::run(v, sm + p * LS, t, a.tw);
        x_store_halves<L>(a, v, sm, p, t, rho0, nrows);
    } else {
#pragma unroll
        for (int q = 0; q < kE; ++q) {
            const int n = t + TPL * q;
            if (MODE == 1) {
                // v = c - 1 (weights and regularisation: update_factor)
                if (oka)
                    a.psi[ra + n] = fmaxf(w[q].x * update_factor(v[q].x, w[q].x, a.wt, ra + n, a.lam, a.inv_s), a.eps);
                if (okb)
                    a.psi[rb + n] = fmaxf(w[q].y * update_factor(v[q].y, w[q].y, a.wt, rb + n, a.lam, a.inv_s), a.eps);
            } else if (MODE == 4) {  // combined update: multiply this view's factor into the product
                if (oka) a.psi[ra + n] = w[q].x * (v[q].x + 1.f) * (a.inv_s ? __ldg(a.inv_s + ra + n) : 1.f);
                if (okb) a.psi[rb + n] = w[q].y * (v[q].y + 1.f) * (a.inv_s ? __ldg(a.inv_s + rb + n) : 1.f);
            } else {
                if (oka) a.psi[ra + n] = v[q].x;
                if (okb) a.psi[rb + n] = v[q].y;
            }
        }
    }
}

}  // namespace mvd
