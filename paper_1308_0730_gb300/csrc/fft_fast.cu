// FFT passes specialised for power-of-two line lengths (16..4096), built on
// the register-resident LineFFT. Same layout and contract as the generic
// passes in fft_passes.cu (spectrum S[kx][z][y], two real x-lines per complex
// line, 1/M folded into the kernel spectra); the host picks these whenever
// the axis length allows.
#include <type_traits>

#include "fft_fast_tiles.cuh"

namespace mvd {

namespace {

constexpr int kThreads = 256;

inline int div_up(long a, long b) { return (int)((a + b - 1) / b); }

template <int L, int S>
__global__ void __launch_bounds__(kThreads) k_y_fast(float2* __restrict__ spec, long nlines,
                                                     const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    fast_y_tile<L, S, false>(spec, nlines, tw, blockIdx.x, sm);
}

template <int L>
__host__ __device__ constexpr int z_q() {
    return fast_z_cols(L);
}

template <int L, bool MUL>
__global__ void __launch_bounds__(512) k_z_fast(float2* __restrict__ spec, const float2* __restrict__ K, int Y,
                                                 long YZ, int ntiles_y, float scale, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    fast_z_tile<L, MUL, false>(spec, K, Y, YZ, ntiles_y, scale, tw, blockIdx.x, sm);
}

template <int L>
__global__ void __launch_bounds__(kThreads) k_x_forward_fast(XFast a) {
    extern __shared__ float2 sm[];
    fast_x_forward_tile<L, false>(a, blockIdx.x, sm);
}

template <int L, int MODE>  // MODE 0: ratio -> forward ; 1: psi update ; 2: plain real output
__global__ void __launch_bounds__(kThreads) k_x_inverse_fast(XFast a) {
    extern __shared__ float2 sm[];
    fast_x_inverse_tile<L, MODE, false>(a, blockIdx.x, sm);
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
                         float eps, cudaStream_t st, const float* wt = nullptr, float lam = 0.f,
                         const float* inv_s = nullptr) {
    mvd_status rc = MVD_ERR_UNSUPPORTED;
    XFast a{src, S, phi, psi, g.YZ, eps, g.px.tw, wt, lam, inv_s};
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
        } else if (mode == 4) {
            kern = k_x_inverse_fast<L, 4>;
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
mvd_status fft_x_update_fast(const FftGeom& g, const float2* S, float* psi, float eps, cudaStream_t st,
                             const float* wt, float lam, const float* inv_s) {
    return x_fast(g, 1, nullptr, const_cast<float2*>(S), nullptr, psi, eps, st, wt, lam, inv_s);
}
mvd_status fft_x_accumulate_fast(const FftGeom& g, const float2* S, float* acc, cudaStream_t st,
                                 const float* inv_s) {
    return x_fast(g, 4, nullptr, const_cast<float2*>(S), nullptr, acc, 0.f, st, nullptr, 0.f, inv_s);
}
mvd_status fft_inverse_real_fast(const FftGeom& g, const float2* S, float* dst, cudaStream_t st) {
    return x_fast(g, 2, nullptr, const_cast<float2*>(S), nullptr, dst, 0.f, st);
}

}  // namespace mvd
