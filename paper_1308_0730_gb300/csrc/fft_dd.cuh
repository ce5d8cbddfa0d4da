// Double-float passes (tile-level device functions, generic mixed-radix
// plans). Same layout as the FP32 passes: spectrum S2[kx][z][y] of complex
// double-float (16 bytes), two real x-lines per complex line. The forward
// blur b = psi * P_v runs entirely in double-float; the ratio pass rounds b to
// FP32, forms r - 1 = phi / max(b, eps) - 1, transforms it along x in FP32
// and stores that spectrum exactly as double-float, so that the
// back-projection's y and z passes (and the kernel multiply) run in
// double-float too; the update pass reads S2 rounded to FP32.
//
// CO = true makes loads of data written inside the same launch L2 loads (the
// persistent batch kernel).
#pragma once

#include "adf.cuh"
#include "dd.cuh"
#include "fft_generic.cuh"

namespace mvd {

// One Stockham butterfly and the multi-line drivers, as in fft.cuh (tw: the
// axis's natural double-float table, followed by its radix-8 and its
// plan-ordered copies; the drivers read the plan-ordered one). The
// first stage runs in double-float and records the largest component of its
// outputs; the later stages run in aligned double-float (adf.cuh) on one grid
// per tile, chosen from that bound (the tile's lines are neighbours in the
// volume or its spectrum, and the error this leaves is absolute against the
// tile's largest line, far inside what the convolution needs).
template <int R, int S, bool ALN>
__device__ __forceinline__ void dd_bfly_math(cdd (&v)[R], int k, const StageIdx& si, const cdd* __restrict__ tw,
                                             float c, float& mx) {
    if constexpr (ALN) {  // a later stage: Ns > 1
        v[0] = adf_calign(v[0], c);
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = adf_cmul(v[r], twiddle_dd<S>(tw, (r - 1) * si.Ns + k), c);
        DftA<R, S>::run(v, c);
    } else {
        if (si.Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twiddle_dd<S>(tw, (r - 1) * si.Ns + k));
        }
        DftDD<R, S>::run(v);
#pragma unroll
        for (int r = 0; r < R; ++r) mx = adf_absmax(v[r], mx);
    }
}

template <int R, int S, bool ALN>
__device__ __forceinline__ void stockham_stage_dd(const cdd* __restrict__ A, cdd* __restrict__ B, int nlines, int ls,
                                                  int L, int Ns, const cdd* __restrict__ tw, float c, float& mx) {
    const StageIdx si(L, R, Ns);
    const int total = nlines * si.nb;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int line = small_div(t, si.inv_nb);
        const int j = t - line * si.nb;
        const int jq = small_div(j, si.inv_ns);
        const int k = j - jq * si.Ns;
        const cdd* a = A + line * ls;
        cdd* b = B + line * ls;
        cdd v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = a[j + r * si.nb];
        dd_bfly_math<R, S, ALN>(v, k, si, tw, c, mx);
        const int d = jq * si.Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) b[d + r * si.Ns] = v[r];
    }
}

// A stage whose input comes straight from global memory (element e of line l
// at g + l*gls + e*ges; lines >= nl read as zero; L2-only loads when CO)
// and/or whose output goes straight to global memory (lines >= nl skipped);
// the other side is the shared-memory line buffer (stride ls). LF maps
// consecutive threads to consecutive lines (coalesced when gls = 1), else to
// consecutive butterflies of a line (coalesced when ges = 1).
template <int R, int S, bool GIN, bool GOUT, bool CO, bool LF, bool ALN>
__device__ __forceinline__ void stockham_stage_dd_io(const cdd* __restrict__ A, cdd* __restrict__ B, const cdd* gin,
                                                     cdd* gout, long gls, long ges, int nlines, int nl, int ls, int L,
                                                     int Ns, const cdd* __restrict__ tw, float c, float& mx) {
    const StageIdx si(L, R, Ns);
    const int total = nlines * si.nb;
    const float inv_nl = 1.0f / (float)nlines;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int line, j;
        if (LF) {
            j = small_div(t, inv_nl);
            line = t - j * nlines;
        } else {
            line = small_div(t, si.inv_nb);
            j = t - line * si.nb;
        }
        const int jq = small_div(j, si.inv_ns);
        const int k = j - jq * si.Ns;
        const bool ok = line < nl;
        cdd v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (GIN) {
                const cdd* q = gin + (long)line * gls + (long)(j + r * si.nb) * ges;
                v[r] = ok ? (CO ? cdd_load_cg(q) : cdd_load(q)) : czero_dd();
            } else {
                v[r] = A[line * ls + j + r * si.nb];
            }
        }
        dd_bfly_math<R, S, ALN>(v, k, si, tw, c, mx);
        const int d = jq * si.Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (GOUT) {
                if (ok) cdd_store(gout + (long)line * gls + (long)(d + r * si.Ns) * ges, v[r]);
            } else {
                B[line * ls + d + r * si.Ns] = v[r];
            }
        }
    }
}

template <int S, bool GIN, bool GOUT, bool CO, bool LF, bool ALN>
__device__ __forceinline__ void stage_dd_io(int R, const cdd* A, cdd* B, const cdd* gin, cdd* gout, long gls,
                                            long ges, int nlines, int nl, int ls, int L, int Ns, const cdd* tw,
                                            float c, float& mx) {
#define MVD_DD_IO(RR) \
    stockham_stage_dd_io<RR, S, GIN, GOUT, CO, LF, ALN>(A, B, gin, gout, gls, ges, nlines, nl, ls, L, Ns, tw, c, mx)
    switch (R) {
        case 8: MVD_DD_IO(8); break;
        case 4: MVD_DD_IO(4); break;
        case 2: MVD_DD_IO(2); break;
        case 3: MVD_DD_IO(3); break;
        case 6: MVD_DD_IO(6); break;
        case 9: MVD_DD_IO(9); break;
        default: MVD_DD_IO(5); break;
    }
#undef MVD_DD_IO
}

// the first stage's bound: each warp's largest component into w[warp]
__device__ __forceinline__ void dd_publish_bound(float mx, float* w) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = mx;
}
// grid exponent of stage s >= 1 (e: that of stage s - 1; w: the first stage's
// warp bounds, read after the barrier that ends it). The first stage's
// outputs are bounded by m; the twiddle products stay below sqrt(2) m.
__device__ __forceinline__ int dd_stage_exp(int s, int e, int prev_radix, const float* w) {
    if (s > 1) return e + adf_gen_shift(prev_radix);
    float m = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, w[i]);
    return adf_exp_for<18>(1.5f * m);
}

// Transforms nl (<= nlines) lines of length p.L. With GIN the first stage
// reads them from global memory g (element e of line l at g + l*gls + e*ges),
// else from the shared-memory buffer A; with GOUT the last stage writes them
// back to g, else to shared memory. The stages between go through the
// shared-memory buffers A/B (nlines lines at stride ls). GIN and GOUT together
// need p.nst >= 2 (one stage would read and write the same global elements).
// Starts and ends with the block synchronised; returns the shared buffer that
// holds the result when !GOUT.
template <int S, bool GIN, bool GOUT, bool CO, bool LF>
__device__ cdd* fft_lines_dd_io(cdd* g, long gls, long ges, cdd* A, cdd* B, int nlines, int nl, int ls,
                                const FftPlan& p, const cdd* tw) {
    __shared__ float wmax[32];
    int Ns = 1, e = 0;
    tw += 2 * p.L;  // the stage-ordered copy for this plan
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.radix[s];
        const bool first = s == 0, last = s == p.nst - 1;
        float mx = 0.f, c = 0.f;
        if (!first) {
            e = dd_stage_exp(s, e, p.radix[s > 0 ? s - 1 : 0], wmax);
            c = adf_const_exp2(e);
        }
        if (GIN && first && GOUT && last)
            stage_dd_io<S, true, true, CO, LF, false>(R, A, B, g, g, gls, ges, nlines, nl, ls, p.L, Ns, tw, c, mx);
        else if (GIN && first)
            stage_dd_io<S, true, false, CO, LF, false>(R, A, B, g, g, gls, ges, nlines, nl, ls, p.L, Ns, tw, c, mx);
        else if (first && GOUT && last)
            stage_dd_io<S, false, true, CO, LF, false>(R, A, B, g, g, gls, ges, nlines, nl, ls, p.L, Ns, tw, c, mx);
        else if (first)
            stage_dd_io<S, false, false, CO, LF, false>(R, A, B, g, g, gls, ges, nlines, nl, ls, p.L, Ns, tw, c, mx);
        else if (GOUT && last)
            stage_dd_io<S, false, true, CO, LF, true>(R, A, B, g, g, gls, ges, nlines, nl, ls, p.L, Ns, tw, c, mx);
        else
            stage_dd_io<S, false, false, CO, LF, true>(R, A, B, g, g, gls, ges, nlines, nl, ls, p.L, Ns, tw, c, mx);
        if (first) dd_publish_bound(mx, wmax);
        if (!first) tw += (R - 1) * Ns;
        __syncthreads();
        cdd* t = A;
        A = B;
        B = t;
        Ns *= R;
    }
    return A;
}

// plan radices as FftPlan, twiddles from a double-float table of length L
template <int S>
__device__ cdd* fft_lines_dd(cdd* A, cdd* B, int nlines, int ls, const FftPlan& p, const cdd* tw) {
    __shared__ float wmax[32];
    int Ns = 1, e = 0;
    tw += 2 * p.L;  // the stage-ordered copy for this plan
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.radix[s];
        float mx = 0.f, c = 0.f;
        if (s > 0) {
            e = dd_stage_exp(s, e, p.radix[s - 1], wmax);
            c = adf_const_exp2(e);
        }
#define MVD_DD_ST(RR)                                                                        \
    do {                                                                                     \
        if (s == 0)                                                                          \
            stockham_stage_dd<RR, S, false>(A, B, nlines, ls, p.L, Ns, tw, c, mx);           \
        else                                                                                 \
            stockham_stage_dd<RR, S, true>(A, B, nlines, ls, p.L, Ns, tw, c, mx);            \
    } while (0)
        switch (R) {
            case 8: MVD_DD_ST(8); break;
            case 4: MVD_DD_ST(4); break;
            case 2: MVD_DD_ST(2); break;
            case 3: MVD_DD_ST(3); break;
            case 6: MVD_DD_ST(6); break;
            case 9: MVD_DD_ST(9); break;
            default: MVD_DD_ST(5); break;
        }
#undef MVD_DD_ST
        if (s == 0) dd_publish_bound(mx, wmax);
        if (s > 0) tw += (R - 1) * Ns;
        __syncthreads();
        cdd* t = A;
        A = B;
        B = t;
        Ns *= R;
    }
    return A;
}


// half the lines of the FP32 tiles (elements are twice as large)
__host__ __device__ inline int dd_x_pairs(int X) {
    const int p = gen_x_pairs(X) / 2;
    return p < 1 ? 1 : p;
}
__host__ __device__ inline int dd_y_lines(int Y) {
    const int p = gen_y_lines(Y) / 2;
    return p < 1 ? 1 : p;
}
__host__ __device__ inline int dd_z_cols(int Z, int Y) {
    const int q = gen_z_cols(Z, Y) / 2;
    return q < 1 ? 1 : q;
}
__host__ __device__ inline long dd_x_tiles(int X, long YZ) { return gen_div_up(YZ, 2 * dd_x_pairs(X)); }
__host__ __device__ inline long dd_y_tiles(int Y, int Xh, int Z) { return gen_div_up((long)Xh * Z, dd_y_lines(Y)); }
__host__ __device__ inline long dd_z_tiles(int Z, int Y, int Xh) { return (long)Xh * gen_div_up(Y, dd_z_cols(Z, Y)); }
__host__ __device__ inline size_t dd_x_smem(int X) { return (size_t)2 * dd_x_pairs(X) * (X + 1) * sizeof(cdd); }
__host__ __device__ inline size_t dd_y_smem(int Y) { return (size_t)2 * dd_y_lines(Y) * (Y + 1) * sizeof(cdd); }
// z line stride: odd, so that 16-byte accesses of consecutive lines hit distinct banks
__host__ __device__ inline int dd_z_ls(int Z) { return (Z + 1) | 1; }
__host__ __device__ inline size_t dd_z_smem(int Z, int Y) { return (size_t)2 * dd_z_cols(Z, Y) * dd_z_ls(Z) * sizeof(cdd); }

struct DdX {
    int X, Xh, P, ls;
    long YZ;
    FftPlan plan;           // radices of X
    const cdd* tw2;         // double-float twiddles of X
    const float* src;       // real rows
    cdd* S2;                // double-float spectrum
    const float* phi;       // observed view
    float eps;
    float2* S;              // ratio: the FP32 spectrum of r - 1 goes here when set, else into S2
};

__host__ __device__ inline DdX dd_x_args(int X, long YZ, const FftPlan& plan, const cdd* tw2) {
    DdX a{};
    a.X = X;
    a.Xh = X / 2 + 1;
    a.P = dd_x_pairs(X);
    a.ls = X + 1;
    a.YZ = YZ;
    a.plan = plan;
    a.tw2 = tw2;
    return a;
}

template <bool CO>
__device__ void dd_x_forward_tile(const DdX& a, long tile, cdd* sm) {
    cdd* A = sm;
    cdd* B = sm + a.P * a.ls;
    const long rho0 = tile * 2 * a.P;
    const int nrows = (int)min((long)2 * a.P, a.YZ - rho0);
    const int n2 = a.P * a.X;
    // pair p = rows (p, P+p): complex line a + i b, exact in double-float
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int p = t / a.X, n = t - p * a.X;
        const float va = p < nrows ? ld1<CO>(a.src + (rho0 + p) * a.X + n) : 0.f;
        const float vb = a.P + p < nrows ? ld1<CO>(a.src + (rho0 + a.P + p) * a.X + n) : 0.f;
        A[p * a.ls + n] = cdd{dd_from(va), dd_from(vb)};
    }
    __syncthreads();
    const cdd* F = fft_lines_dd<-1>(A, B, a.P, a.ls, a.plan, a.tw2);
    const int P2 = 2 * a.P;
    for (int t = threadIdx.x; t < a.Xh * P2; t += blockDim.x) {
        const int k = t / P2, row = t - k * P2;
        if (row >= nrows) continue;
        const int p = row < a.P ? row : row - a.P;
        const cdd zk = F[p * a.ls + k];
        const cdd zm = cconj(F[p * a.ls + (k == 0 ? 0 : a.X - k)]);
        cdd val;
        if (row < a.P) {
            val = chalf(cadd(zk, zm));
        } else {  // (zk - zm) / (2i)
            const cdd d = chalf(csub(zk, zm));
            val = cdd{d.im, dd{-d.re.hi, -d.re.lo}};
        }
        cdd_store(a.S2 + (long)k * a.YZ + rho0 + row, val);
    }
}

// double-float spectrum -> inverse x -> b (rounded to FP32) -> r - 1 with
// r = phi / max(b, eps) -> FP32 forward x -> back into S2 (exact as
// double-float), where the back-projection's y and z passes continue in
// double-float
// the unpacked half spectra of the P transformed complex lines in F (rows
// p and P + p of the tile) into S2
__device__ __forceinline__ void dd_x_unpack_store(const DdX& a, const cdd* F, long rho0, int nrows) {
    const int P2 = 2 * a.P;
    for (int t = threadIdx.x; t < a.Xh * P2; t += blockDim.x) {
        const int k = t / P2, row = t - k * P2;
        if (row >= nrows) continue;
        const int p = row < a.P ? row : row - a.P;
        const cdd zk = F[p * a.ls + k];
        const cdd zm = cconj(F[p * a.ls + (k == 0 ? 0 : a.X - k)]);
        cdd val;
        if (row < a.P) {
            val = chalf(cadd(zk, zm));
        } else {  // (zk - zm) / (2i)
            const cdd d = chalf(csub(zk, zm));
            val = cdd{d.im, dd{-d.re.hi, -d.re.lo}};
        }
        cdd_store(a.S2 + (long)k * a.YZ + rho0 + row, val);
    }
}

// gather the half spectra of the tile's row pairs from S2 into A (rows < P)
// and B, then form the full spectrum of each complex line A + iB in A
template <bool CO>
__device__ __forceinline__ void dd_x_gather_lines(const DdX& a, cdd* A, cdd* B, long rho0, int nrows) {
    const int P2 = 2 * a.P;
    for (int t = threadIdx.x; t < a.Xh * P2; t += blockDim.x) {
        const int k = t / P2, row = t - k * P2;
        cdd v = czero_dd();
        if (row < nrows) v = CO ? cdd_load_cg(a.S2 + (long)k * a.YZ + rho0 + row) : cdd_load(a.S2 + (long)k * a.YZ + rho0 + row);
        if (row < a.P)
            A[row * a.ls + k] = v;
        else
            B[(row - a.P) * a.ls + k] = v;
    }
    __syncthreads();
    const int half = (a.X + 1) / 2;
    for (int t = threadIdx.x; t < a.P * a.Xh; t += blockDim.x) {
        const int p = t / a.Xh, k = t - p * a.Xh;
        const cdd av = A[p * a.ls + k], bv = B[p * a.ls + k];
        A[p * a.ls + k] = cdd{dd_sub(av.re, bv.im), dd_add(av.im, bv.re)};
        if (k >= 1 && k < half) A[p * a.ls + (a.X - k)] = cdd{dd_add(av.re, bv.im), dd_sub(bv.re, av.im)};
    }
    __syncthreads();
}

// The back-projection's last pass in double-float: inverse x of S2, the
// result (c - 1) rounded to FP32 once, then MODE 1: psi = max(psi .
// update_factor, eps); MODE 4: acc = acc . c . inv_s (the combined update's
// product); MODE 0: psi = the rounded result (plain real output).
struct DdXU {
    DdX x;
    float* psi;
    const float* wt;
    float lam;
    const float* inv_s;
};

template <bool CO, int MODE>
__device__ void dd_x_update_tile(const DdXU& u, long tile, cdd* sm) {
    const DdX& a = u.x;
    cdd* A = sm;
    cdd* B = sm + a.P * a.ls;
    const long rho0 = tile * 2 * a.P;
    const int nrows = (int)min((long)2 * a.P, a.YZ - rho0);
    dd_x_gather_lines<CO>(a, A, B, rho0, nrows);
    const cdd* R = fft_lines_dd<+1>(A, B, a.P, a.ls, a.plan, a.tw2);
    const int n2 = a.P * a.X;
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int p = t / a.X, n = t - p * a.X;
        const cdd z = R[p * a.ls + n];
        const float cv[2] = {z.re.hi + z.re.lo, z.im.hi + z.im.lo};  // c - 1 of rows p and P + p
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = p + h * a.P;
            if (row >= nrows) continue;
            const long i = (rho0 + row) * a.X + n;
            if (MODE == 0) {
                u.psi[i] = cv[h];
                continue;
            }
            const float ps = u.psi[i];
            if (MODE == 1)
                u.psi[i] = fmaxf(ps * update_factor(cv[h], ps, u.wt, i, u.lam, u.inv_s), a.eps);
            else
                u.psi[i] = ps * (cv[h] + 1.f) * (u.inv_s ? __ldg(u.inv_s + i) : 1.f);
        }
    }
}

template <bool CO>
__device__ void dd_x_ratio_tile(const DdX& a, long tile, cdd* sm) {
    cdd* A = sm;
    cdd* B = sm + a.P * a.ls;
    const long rho0 = tile * 2 * a.P;
    const int nrows = (int)min((long)2 * a.P, a.YZ - rho0);
    const int P2 = 2 * a.P;
    for (int t = threadIdx.x; t < a.Xh * P2; t += blockDim.x) {
        const int k = t / P2, row = t - k * P2;
        cdd v = czero_dd();
        if (row < nrows) v = CO ? cdd_load_cg(a.S2 + (long)k * a.YZ + rho0 + row) : cdd_load(a.S2 + (long)k * a.YZ + rho0 + row);
        if (row < a.P)
            A[row * a.ls + k] = v;
        else
            B[(row - a.P) * a.ls + k] = v;
    }
    __syncthreads();
    const int half = (a.X + 1) / 2;
    for (int t = threadIdx.x; t < a.P * a.Xh; t += blockDim.x) {
        const int p = t / a.Xh, k = t - p * a.Xh;
        const cdd av = A[p * a.ls + k], bv = B[p * a.ls + k];
        // A + iB and, at -k, conj(A) + i conj(B)
        A[p * a.ls + k] = cdd{dd_sub(av.re, bv.im), dd_add(av.im, bv.re)};
        if (k >= 1 && k < half) A[p * a.ls + (a.X - k)] = cdd{dd_add(av.re, bv.im), dd_sub(bv.re, av.im)};
    }
    __syncthreads();
    cdd* R = fft_lines_dd<+1>(A, B, a.P, a.ls, a.plan, a.tw2);
    // FP32 buffers in the other half of shared memory
    float2* F0 = reinterpret_cast<float2*>(R == A ? B : A);
    float2* F1 = F0 + a.P * a.ls;
    const int n2 = a.P * a.X;
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int p = t / a.X, n = t - p * a.X;
        const cdd z = R[p * a.ls + n];
        const float ba = z.re.hi + z.re.lo, bb = z.im.hi + z.im.lo;
        float ra = 0.f, rb = 0.f;
        if (p < nrows) ra = __ldg(a.phi + (rho0 + p) * a.X + n) / fmaxf(ba, a.eps) - 1.f;
        if (a.P + p < nrows) rb = __ldg(a.phi + (rho0 + a.P + p) * a.X + n) / fmaxf(bb, a.eps) - 1.f;
        F0[p * a.ls + n] = make_float2(ra, rb);
    }
    __syncthreads();
    const float2* F = fft_lines<-1>(F0, F1, a.P, a.ls, a.plan);
    // unpack into the FP32 spectrum (as gen_unpack_store, with this tile's P)
    for (int t = threadIdx.x; t < a.Xh * P2; t += blockDim.x) {
        const int k = t / P2, row = t - k * P2;
        if (row >= nrows) continue;
        const int p = row < a.P ? row : row - a.P;
        const float2 zk = F[p * a.ls + k];
        const float2 zm = cconj(F[p * a.ls + (k == 0 ? 0 : a.X - k)]);
        float2 val;
        if (row < a.P) {
            val = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
        } else {
            const float2 d = csub(zk, zm);
            val = make_float2(0.5f * d.y, -0.5f * d.x);
        }
        if (a.S)
            a.S[(long)k * a.YZ + rho0 + row] = val;
        else
            cdd_store(a.S2 + (long)k * a.YZ + rho0 + row, cdd{dd_from(val.x), dd_from(val.y)});
    }
}

struct DdY {
    int L, ls, P;
    long nlines;
    FftPlan plan;
    const cdd* tw2;
    cdd* S2;
};

__host__ __device__ inline DdY dd_y_args(int Y, int Xh, int Z, const FftPlan& plan, const cdd* tw2, cdd* S2) {
    DdY a{};
    a.L = Y;
    a.ls = Y + 1;
    a.P = dd_y_lines(Y);
    a.nlines = (long)Xh * Z;
    a.plan = plan;
    a.tw2 = tw2;
    a.S2 = S2;
    return a;
}

template <bool CO, int S>
__device__ void dd_y_tile(const DdY& a, long tile, cdd* sm) {
    cdd* A = sm;
    cdd* B = sm + a.P * a.ls;
    const long l0 = tile * a.P;
    const int nl = (int)min((long)a.P, a.nlines - l0);
    if (a.plan.nst >= 2) {
        // the tile's lines staged by asynchronous copies, all in flight at once
        // (lines past the end zero-filled); the last stage writes global memory
        const cdd* src = a.S2 + l0 * a.L;
        for (int t = threadIdx.x; t < a.P * a.L; t += blockDim.x) {
            const int line = t / a.L, y = t - line * a.L;
            const bool ok = line < nl;
            cp_async16(A + line * a.ls + y, ok ? src + (long)line * a.L + y : a.S2, ok);
        }
        cp_async_wait_all();
        __syncthreads();
        fft_lines_dd_io<S, false, true, CO, false>(a.S2 + l0 * a.L, a.L, 1, A, B, a.P, nl, a.ls, a.plan, a.tw2);
        return;
    }
    for (int t = threadIdx.x; t < a.P * a.L; t += blockDim.x) {
        const int line = t / a.L, y = t - line * a.L;
        cdd v = czero_dd();
        if (line < nl) v = CO ? cdd_load_cg(a.S2 + (l0 + line) * a.L + y) : cdd_load(a.S2 + (l0 + line) * a.L + y);
        A[line * a.ls + y] = v;
    }
    __syncthreads();
    const cdd* R = fft_lines_dd<S>(A, B, a.P, a.ls, a.plan, a.tw2);
    for (int t = threadIdx.x; t < nl * a.L; t += blockDim.x) {
        const int line = t / a.L, y = t - line * a.L;
        cdd_store(a.S2 + (l0 + line) * a.L + y, R[line * a.ls + y]);
    }
}

struct DdZ {
    int Z, Y, Q, ls, ntiles_y;
    long YZ;
    FftPlan plan;
    const cdd* tw2;
    cdd* S2;
    const cdd* K2;  // double-float kernel spectrum (MUL)
    dd scale;       // forward-only scale
};

__host__ __device__ inline DdZ dd_z_args(int Z, int Y, long YZ, const FftPlan& plan, const cdd* tw2, cdd* S2,
                                         const cdd* K2, dd scale) {
    DdZ a{};
    a.Z = Z;
    a.Y = Y;
    a.Q = dd_z_cols(Z, Y);
    a.ls = dd_z_ls(Z);
    a.ntiles_y = (int)gen_div_up(Y, a.Q);
    a.YZ = YZ;
    a.plan = plan;
    a.tw2 = tw2;
    a.S2 = S2;
    a.K2 = K2;
    a.scale = scale;
    return a;
}

template <bool CO, bool MUL>
__device__ void dd_z_tile(const DdZ& a, long tile, cdd* sm) {
    cdd* A = sm;
    cdd* B = sm + a.Q * a.ls;
    const int kx = (int)(tile / a.ntiles_y);
    const int y0 = (int)(tile - (long)kx * a.ntiles_y) * a.Q;
    const int nq = min(a.Q, a.Y - y0);
    const long base = (long)kx * a.YZ + y0;
    const int n = a.Z * a.Q;
    if (MUL && a.plan.nst >= 1) {  // columns: element z of column q at base + z*Y + q; threads run along q
        // the tile's columns staged by asynchronous copies (consecutive copies take
        // consecutive columns: Q * 16 contiguous bytes per z), all in flight at once
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int z = t / a.Q, q = t - z * a.Q;
            const bool ok = q < nq;
            cp_async16(A + q * a.ls + z, ok ? a.S2 + base + (long)z * a.Y + q : a.S2, ok);
        }
        cp_async_wait_all();
        __syncthreads();
        cdd* F = fft_lines_dd_io<-1, false, false, CO, true>(a.S2 + base, 1, a.Y, A, B, a.Q, nq, a.ls, a.plan, a.tw2);
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int z = t / a.Q, q = t - z * a.Q;
            if (q < nq) F[q * a.ls + z] = cmul(F[q * a.ls + z], cdd_load_nc(a.K2 + base + (long)z * a.Y + q));
        }
        __syncthreads();
        fft_lines_dd_io<+1, false, true, CO, true>(a.S2 + base, 1, a.Y, F, F == A ? B : A, a.Q, nq, a.ls, a.plan,
                                                   a.tw2);
        return;
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int z = t / a.Q, q = t - z * a.Q;
        cdd v = czero_dd();
        if (q < nq) v = CO ? cdd_load_cg(a.S2 + base + (long)z * a.Y + q) : cdd_load(a.S2 + base + (long)z * a.Y + q);
        A[q * a.ls + z] = v;
    }
    __syncthreads();
    cdd* F = fft_lines_dd<-1>(A, B, a.Q, a.ls, a.plan, a.tw2);
    cdd* O = F == A ? B : A;
    if (MUL) {
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int z = t / a.Q, q = t - z * a.Q;
            if (q < nq) F[q * a.ls + z] = cmul(F[q * a.ls + z], cdd_load_nc(a.K2 + base + (long)z * a.Y + q));
        }
        __syncthreads();
        F = fft_lines_dd<+1>(F, O, a.Q, a.ls, a.plan, a.tw2);
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int z = t / a.Q, q = t - z * a.Q;
        if (q < nq) {
            cdd v = F[q * a.ls + z];
            if (!MUL) v = cdd{dd_mul(v.re, a.scale), dd_mul(v.im, a.scale)};
            cdd_store(a.S2 + base + (long)z * a.Y + q, v);
        }
    }
}

}  // namespace mvd
