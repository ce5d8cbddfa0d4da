// FFT passes specialised for power-of-two line lengths (16..4096), built on
// the register-resident LineFFT. Same layout and contract as the generic
// passes in fft_passes.cu (spectrum S[kx][z][y], two real x-lines per complex
// line, 1/M folded into the kernel spectra); the host picks these whenever
// the axis length allows.
#include <type_traits>

#include "fft_fast.cuh"

namespace mvd {

namespace {

constexpr int kThreads = 256;

inline int div_up(long a, long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// y pass: Xh*Z contiguous lines of length Y; lines of one warp are adjacent
// ---------------------------------------------------------------------------
template <int L, int S>
__global__ void __launch_bounds__(kThreads) k_y_fast(float2* __restrict__ spec, long nlines,
                                                     const float2* __restrict__ tw) {
    using F = LineFFT<L, S, true>;
    constexpr int TPL = F::TPL;
    constexpr int LPC = kThreads / TPL;
    extern __shared__ float2 sm[];
    const int li = threadIdx.x / TPL, t = threadIdx.x - li * TPL;
    const long line = (long)blockIdx.x * LPC + li;
    const bool ok = line < nlines;
    float2* g = spec + line * L;
    float2 v[kE];
#pragma unroll
    for (int q = 0; q < kE; ++q) v[q] = ok ? g[t + TPL * q] : make_float2(0.f, 0.f);
    F::run(v, sm + li * line_stride(L), t, tw);
    if (ok) {
#pragma unroll
        for (int q = 0; q < kE; ++q) g[t + TPL * q] = v[q];
    }
}

// ---------------------------------------------------------------------------
// z pass: Q lines (consecutive y) of one kx plane; thread = q + Q * t so each
// warp reads rows of consecutive y
// ---------------------------------------------------------------------------
template <int L>
__host__ __device__ constexpr int z_q() {
    return (kThreads / (L / kE)) >= 8 ? kThreads / (L / kE) : 8;
}

template <int L, bool MUL>
__global__ void __launch_bounds__(512) k_z_fast(float2* __restrict__ spec, const float2* __restrict__ K, int Y,
                                                 long YZ, int ntiles_y, float scale, const float2* __restrict__ tw) {
    constexpr int TPL = L / kE;
    constexpr int Q = z_q<L>();
    extern __shared__ float2 sm[];
    const int q = threadIdx.x % Q, t = threadIdx.x / Q;
    const int kx = blockIdx.x / ntiles_y;
    const int y0 = (blockIdx.x - kx * ntiles_y) * Q;
    const bool ok = y0 + q < Y;
    const long base = (long)kx * YZ + y0 + q;
    float2* line_sm = sm + q * line_stride(L);
    float2 v[kE];
#pragma unroll
    for (int i = 0; i < kE; ++i) v[i] = ok ? spec[base + (long)(t + TPL * i) * Y] : make_float2(0.f, 0.f);
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

// ---------------------------------------------------------------------------
// x passes: P pairs of rows per block (rows rho0+p and rho0+P+p form pair p)
// ---------------------------------------------------------------------------
struct XFast {
    const float* src;
    float2* spec;
    const float* phi;
    float* psi;
    long YZ;
    float eps;
    const float2* tw;
};

// write the packed forward spectra (natural order in registers) as the two
// half spectra of each pair, coalesced over rows
template <int L>
__device__ __forceinline__ void x_store_halves(const XFast& a, float2 (&v)[kE], float2* sm, int p, int t, long rho0,
                                               int nrows) {
    constexpr int TPL = L / kE, P = kThreads / TPL, LS = line_stride(L), XH = L / 2 + 1;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kE; ++q) sm[p * LS + pad16(t + TPL * q)] = v[q];
    __syncthreads();
    constexpr int NTOT = XH * 2 * P, NIT = (NTOT + kThreads - 1) / kThreads;
#pragma unroll
    for (int i = 0; i < NIT; ++i) {
        const int idx = threadIdx.x + i * kThreads;
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
template <int L>
__device__ __forceinline__ void x_load_packed(const XFast& a, float2 (&v)[kE], float2* sm, int p, int t, long rho0,
                                              int nrows) {
    constexpr int TPL = L / kE, P = kThreads / TPL, LS = line_stride(L), XH = L / 2 + 1;
    constexpr int NTOT = XH * 2 * P, NIT = (NTOT + kThreads - 1) / kThreads;
    // rows < P -> line p (A), rows >= P -> line P + p (B); all loads of a
    // thread are issued before the first shared-memory store
    float2 tmp[NIT];
#pragma unroll
    for (int i = 0; i < NIT; ++i) {
        const int idx = threadIdx.x + i * kThreads;
        const int k = idx / (2 * P), row = idx - k * 2 * P;
        tmp[i] = (idx < NTOT && row < nrows) ? a.spec[(long)k * a.YZ + rho0 + row] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < NIT; ++i) {
        const int idx = threadIdx.x + i * kThreads;
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

template <int L>
__global__ void __launch_bounds__(kThreads) k_x_forward_fast(XFast a) {
    constexpr int TPL = L / kE, P = kThreads / TPL, LS = line_stride(L);
    extern __shared__ float2 sm[];
    const int p = threadIdx.x / TPL, t = threadIdx.x - p * TPL;
    const long rho0 = (long)blockIdx.x * 2 * P;
    const int nrows = (int)min((long)2 * P, a.YZ - rho0);
    const bool oka = p < nrows, okb = P + p < nrows;
    const float* ra = a.src + (rho0 + p) * L;
    const float* rb = a.src + (rho0 + P + p) * L;
    float2 v[kE];
#pragma unroll
    for (int q = 0; q < kE; ++q) {
        const int n = t + TPL * q;
        v[q] = make_float2(oka ? __ldg(ra + n) : 0.f, okb ? __ldg(rb + n) : 0.f);
    }
    LineFFT<L, -1, true>::run(v, sm + p * LS, t, a.tw);
    x_store_halves<L>(a, v, sm, p, t, rho0, nrows);
}

template <int L, int MODE>  // MODE 0: ratio -> forward ; 1: psi update ; 2: plain real output
__global__ void __launch_bounds__(kThreads) k_x_inverse_fast(XFast a) {
    constexpr int TPL = L / kE, P = kThreads / TPL, LS = line_stride(L);
    extern __shared__ float2 sm[];
    const int p = threadIdx.x / TPL, t = threadIdx.x - p * TPL;
    const long rho0 = (long)blockIdx.x * 2 * P;
    const int nrows = (int)min((long)2 * P, a.YZ - rho0);
    const bool oka = p < nrows, okb = P + p < nrows;
    float2 v[kE];
    x_load_packed<L>(a, v, sm, p, t, rho0, nrows);
    const long ra = (rho0 + p) * L, rb = (rho0 + P + p) * L;
    // the epilogue's operand rows (phi for the ratio, psi for the update) are
    // fetched now so that their loads overlap the inverse transform
    float2 w[kE];
    if (MODE < 2) {
        const float* src = MODE == 0 ? a.phi : a.psi;
#pragma unroll
        for (int q = 0; q < kE; ++q) {
            const int n = t + TPL * q;
            w[q] = make_float2(oka ? src[ra + n] : 0.f, okb ? src[rb + n] : 0.f);
        }
    }
    LineFFT<L, +1, true>::run(v, sm + p * LS, t, a.tw);
    if (MODE == 0) {
#pragma unroll
        for (int q = 0; q < kE; ++q) {
            const float xa = oka ? w[q].x / fmaxf(v[q].x, a.eps) : 0.f;
            const float xb = okb ? w[q].y / fmaxf(v[q].y, a.eps) : 0.f;
            v[q] = make_float2(xa, xb);
        }
        LineFFT<L, -1, true>::run(v, sm + p * LS, t, a.tw);
        x_store_halves<L>(a, v, sm, p, t, rho0, nrows);
    } else {
#pragma unroll
        for (int q = 0; q < kE; ++q) {
            const int n = t + TPL * q;
            if (MODE == 1) {
                if (oka) a.psi[ra + n] = fmaxf(w[q].x * v[q].x, a.eps);
                if (okb) a.psi[rb + n] = fmaxf(w[q].y * v[q].y, a.eps);
            } else {
                if (oka) a.psi[ra + n] = v[q].x;
                if (okb) a.psi[rb + n] = v[q].y;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// dispatch over the supported lengths
// ---------------------------------------------------------------------------
template <typename F>
bool dispatch_len(int L, F&& f) {
    switch (L) {
        case 16: f(std::integral_constant<int, 16>{}); return true;
        case 32: f(std::integral_constant<int, 32>{}); return true;
        case 64: f(std::integral_constant<int, 64>{}); return true;
        case 128: f(std::integral_constant<int, 128>{}); return true;
        case 256: f(std::integral_constant<int, 256>{}); return true;
        case 512: f(std::integral_constant<int, 512>{}); return true;
        case 1024: f(std::integral_constant<int, 1024>{}); return true;
        case 2048: f(std::integral_constant<int, 2048>{}); return true;
        default: return false;
    }
}

}  // namespace

bool fft_fast_supported(int L) { return fast_length(L) && L <= 2048; }
bool fft_fast_z_supported(int L) { return fast_length(L) && L <= 1024; }

mvd_status fft_y_fast(const FftGeom& g, float2* S, int inverse, cudaStream_t st) {
    mvd_status rc = MVD_ERR_UNSUPPORTED;
    const long nlines = (long)g.Xh * g.Z;
    dispatch_len(g.Y, [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        constexpr int TPL = L / kE, LPC = kThreads / TPL;
        const size_t smem = (size_t)LPC * line_stride(L) * sizeof(float2);
        auto kern = inverse ? k_y_fast<L, +1> : k_y_fast<L, -1>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            rc = cuda_status(e, "fft y (fast) attr");
            return;
        }
        prof_begin(KC_Y, st);
        kern<<<div_up(nlines, LPC), kThreads, smem, st>>>(S, nlines, g.py.tw);
        prof_end(KC_Y, st);
        count_launch();
        rc = check_launch("fft y (fast)");
    });
    return rc;
}

static mvd_status z_fast(const FftGeom& g, float2* S, const float2* K, float scale, bool mul, cudaStream_t st) {
    mvd_status rc = MVD_ERR_UNSUPPORTED;
    if (!fft_fast_z_supported(g.Z)) return rc;
    dispatch_len(g.Z, [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        constexpr int TPL = L / kE, Q = z_q<L>();
        const int threads = Q * TPL;
        const int ntiles = div_up(g.Y, Q);
        const size_t smem = (size_t)Q * line_stride(L) * sizeof(float2);
        if constexpr (L <= 1024) {
            auto kern = mul ? k_z_fast<L, true> : k_z_fast<L, false>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) {
                rc = cuda_status(e, "fft z (fast) attr");
                return;
            }
            const int cls = mul ? KC_Z_MUL : KC_SETUP;
            prof_begin(cls, st);
            kern<<<g.Xh * ntiles, threads, smem, st>>>(S, K, g.Y, g.YZ, ntiles, scale, g.pz.tw);
            prof_end(cls, st);
            count_launch();
            rc = check_launch("fft z (fast)");
        }
    });
    return rc;
}

mvd_status fft_z_mul_fast(const FftGeom& g, float2* S, const float2* K, cudaStream_t st) {
    return z_fast(g, S, K, 1.f, true, st);
}

mvd_status fft_z_forward_scaled_fast(const FftGeom& g, float2* S, float scale, cudaStream_t st) {
    return z_fast(g, S, nullptr, scale, false, st);
}

static mvd_status x_fast(const FftGeom& g, int mode, const float* src, float2* S, const float* phi, float* psi,
                         float eps, cudaStream_t st) {
    mvd_status rc = MVD_ERR_UNSUPPORTED;
    XFast a{src, S, phi, psi, g.YZ, eps, g.px.tw};
    dispatch_len(g.X, [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        constexpr int TPL = L / kE, P = kThreads / TPL;
        const size_t smem = (size_t)2 * P * line_stride(L) * sizeof(float2);
        const int grid = div_up(g.YZ, 2 * P);
        void (*kern)(XFast) = nullptr;
        int cls = KC_SETUP;
        if (mode == 3) {
            kern = k_x_forward_fast<L>;
            cls = KC_X_FORWARD;
        } else if (mode == 0) {
            kern = k_x_inverse_fast<L, 0>;
            cls = KC_X_RATIO;
        } else if (mode == 1) {
            kern = k_x_inverse_fast<L, 1>;
            cls = KC_X_UPDATE;
        } else {
            kern = k_x_inverse_fast<L, 2>;
        }
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            rc = cuda_status(e, "fft x (fast) attr");
            return;
        }
        prof_begin(cls, st);
        kern<<<grid, kThreads, smem, st>>>(a);
        prof_end(cls, st);
        count_launch();
        rc = check_launch("fft x (fast)");
    });
    return rc;
}

mvd_status fft_forward_real_fast(const FftGeom& g, const float* src, float2* S, cudaStream_t st) {
    return x_fast(g, 3, src, S, nullptr, nullptr, 0.f, st);
}
mvd_status fft_x_ratio_fast(const FftGeom& g, float2* S, const float* phi, float eps, cudaStream_t st) {
    return x_fast(g, 0, nullptr, S, phi, nullptr, eps, st);
}
mvd_status fft_x_update_fast(const FftGeom& g, const float2* S, float* psi, float eps, cudaStream_t st) {
    return x_fast(g, 1, nullptr, const_cast<float2*>(S), nullptr, psi, eps, st);
}
mvd_status fft_inverse_real_fast(const FftGeom& g, const float2* S, float* dst, cudaStream_t st) {
    return x_fast(g, 2, nullptr, const_cast<float2*>(S), nullptr, dst, 0.f, st);
}

}  // namespace mvd
