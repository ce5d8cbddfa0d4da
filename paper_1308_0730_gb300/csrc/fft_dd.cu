// Kernels and launchers of the double-float forward-blur passes (tile
// functions in fft_dd.cuh).
#include <type_traits>

#include "fft_dd.cuh"
#include "fft_dd_fast.cuh"

namespace mvd {

namespace {

// generic double-float passes: three blocks per SM (their tiles' shared
// memory allows three; the registers of the radix-9/10 butterflies would
// otherwise leave room for two)
constexpr int kDdGenBlocks = 3;

__global__ void __launch_bounds__(kGenThreads, kDdGenBlocks) k_dd_x_forward(DdX a) {
    extern __shared__ cdd smd[];
    dd_x_forward_tile<false>(a, blockIdx.x, smd);
}

__global__ void __launch_bounds__(kGenThreads, kDdGenBlocks) k_dd_x_ratio(DdX a) {
    extern __shared__ cdd smd[];
    dd_x_ratio_tile<false>(a, blockIdx.x, smd);
}

template <int MODE>
__global__ void __launch_bounds__(kGenThreads, kDdGenBlocks) k_dd_x_update(DdXU u) {
    extern __shared__ cdd smd[];
    dd_x_update_tile<false, MODE>(u, blockIdx.x, smd);
}

template <int S>
__global__ void __launch_bounds__(kGenThreads, kDdGenBlocks) k_dd_y(DdY a) {
    extern __shared__ cdd smd[];
    dd_y_tile<false, S>(a, blockIdx.x, smd);
}

template <bool MUL>
__global__ void __launch_bounds__(kGenThreads, kDdGenBlocks) k_dd_z(DdZ a) {
    extern __shared__ cdd smd[];
    dd_z_tile<false, MUL>(a, blockIdx.x, smd);
}

// register-resident double-float passes (power-of-two lengths)
template <int L, int S, int IO = 0>
__global__ void __launch_bounds__(kDdThreads, 4) k_ddf_y(cdd* S2, long nlines, const cdd* tw2, float2* S1) {
    extern __shared__ cdd smd[];
    ddf_y_tile<L, S, false, IO>(S2, nlines, tw2, blockIdx.x, smd, S1);
}

template <int L, bool MUL>
__global__ void __launch_bounds__(512) k_ddf_z(cdd* S2, const cdd* K2, int Y, long YZ, int ntiles_y, dd scale,
                                               const cdd* tw2) {
    extern __shared__ cdd smd[];
    ddf_z_tile<L, MUL, false>(S2, K2, Y, YZ, ntiles_y, scale, tw2, blockIdx.x, smd);
}

template <int L>
__global__ void __launch_bounds__(kDdThreads, 2) k_ddf_z2_pipe(cdd* S2, const cdd* K2, int Y, long YZ, int ntiles_y,
                                                              const cdd* tw2, long ntiles) {
    extern __shared__ cdd smd[];
    ddf_z2_pipe<L>(S2, K2, Y, YZ, ntiles_y, tw2, ntiles, smd);
}

template <int L>
__global__ void __launch_bounds__(kDdThreads, 4) k_ddf_x_forward(DdXFast a) {
    extern __shared__ cdd smd[];
    ddf_x_forward_tile<L, false>(a, blockIdx.x, smd);
}

template <int L>
__global__ void __launch_bounds__(kDdThreads) k_ddf_x_inverse(DdXFast a) {
    extern __shared__ cdd smd[];
    ddf_x_inverse_tile<L, false>(a, blockIdx.x, smd);
}

template <int L>
__global__ void __launch_bounds__(kDdThreads, 4) k_ddf_x_ratio(DdXFast a) {
    extern __shared__ cdd smd[];
    ddf_x_ratio_tile<L, false>(a, blockIdx.x, smd);
}

template <int L, int MODE>
__global__ void __launch_bounds__(kDdThreads, 4) k_ddf_x_update(DdXUpd a) {
    extern __shared__ cdd smd[];
    ddf_x_update_tile<L, MODE>(a, blockIdx.x, smd);
}




template <typename F>
bool with_dd_len(int L, F&& f) {
    switch (L) {
        case 32: f(std::integral_constant<int, 32>{}); return true;
        case 64: f(std::integral_constant<int, 64>{}); return true;
        case 128: f(std::integral_constant<int, 128>{}); return true;
        case 256: f(std::integral_constant<int, 256>{}); return true;
        case 512: f(std::integral_constant<int, 512>{}); return true;
        case 1024: f(std::integral_constant<int, 1024>{}); return true;
        default: return false;
    }
}

template <typename K, typename... Args>
mvd_status launch_raw(K kern, long grid, int threads, size_t smem, cudaStream_t st, const char* name, int cls,
                      Args... args) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e, name);
    prof_begin(cls, st);
    kern<<<(unsigned)grid, threads, smem, st>>>(args...);
    prof_end(cls, st);
    count_launch();
    return check_launch(name);
}

// blocks of a persistent launch: as many as fit on every SM at once, at most one per tile
template <typename K>
long persistent_grid(K kern, int threads, size_t smem, long ntiles) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long g = (long)per_sm * (sms > 0 ? sms : 1);
    return g < ntiles ? g : ntiles;
}

DdXFast ddf_args(const FftGeom& g) {
    DdXFast a{};
    a.YZ = g.YZ;
    a.tw2 = g.tw2x;
    a.plan = g.px;
    return a;
}

template <typename K, typename A>
mvd_status launch(K kern, const A& a, long grid, size_t smem, cudaStream_t st, const char* name, int cls) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e, name);
    prof_begin(cls, st);
    kern<<<(unsigned)grid, kGenThreads, smem, st>>>(a);
    prof_end(cls, st);
    count_launch();
    return check_launch(name);
}

}  // namespace

mvd_status dd_forward_real(const FftGeom& g, const float* src, cdd* S2, cudaStream_t st) {
    if (g.fast && dd_fast_length(g.X)) {
        mvd_status rc = MVD_ERR_UNSUPPORTED;
        DdXFast a = ddf_args(g);
        a.src = src;
        a.S2 = S2;
        with_dd_len(g.X, [&](auto Lc) {
            constexpr int L = decltype(Lc)::value;
            rc = launch_raw(k_ddf_x_forward<L>, gen_div_up(g.YZ, 2 * ddf_pairs(L)), kDdThreads, ddf_x_smem(L), st,
                            "dd x forward (fast)", KC_DD_X_FORWARD, a);
        });
        return rc;
    }
    DdX a = dd_x_args(g.X, g.YZ, g.px, g.tw2x);
    a.src = src;
    a.S2 = S2;
    return launch(k_dd_x_forward, a, dd_x_tiles(g.X, g.YZ), dd_x_smem(g.X), st, "dd x forward", KC_DD_X_FORWARD);
}

bool dd_fast_x(const FftGeom& g) { return g.fast && dd_fast_length(g.X); }

mvd_status dd_x_inverse_real(const FftGeom& g, const cdd* S2, float* dst, cudaStream_t st) {
    if (!(g.fast && dd_fast_length(g.X))) {
        set_error("dd x inverse: length %d has no register-resident double-float transform", g.X);
        return MVD_ERR_UNSUPPORTED;
    }
    mvd_status rc = MVD_ERR_UNSUPPORTED;
    DdXFast a = ddf_args(g);
    a.S2 = const_cast<cdd*>(S2);
    a.dst = dst;
    with_dd_len(g.X, [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        rc = launch_raw(k_ddf_x_inverse<L>, gen_div_up(g.YZ, 2 * ddf_pairs(L)), kDdThreads, ddf_x_smem(L), st,
                        "dd x inverse (fast)", KC_DD_X_RATIO, a);
    });
    return rc;
}

mvd_status dd_x_ratio(const FftGeom& g, cdd* S2, const float* phi, float eps, cudaStream_t st, float2* S) {
    if (g.fast && dd_fast_length(g.X)) {
        mvd_status rc = MVD_ERR_UNSUPPORTED;
        DdXFast a = ddf_args(g);
        a.S2 = S2;
        a.S = S;
        a.phi = phi;
        a.eps = eps;
        with_dd_len(g.X, [&](auto Lc) {
            constexpr int L = decltype(Lc)::value;
            rc = launch_raw(k_ddf_x_ratio<L>, gen_div_up(g.YZ, 2 * ddf_pairs(L)), kDdThreads, ddf_ratio_smem(L), st,
                            "dd x ratio (fast)", KC_DD_X_RATIO, a);
        });
        return rc;
    }
    DdX a = dd_x_args(g.X, g.YZ, g.px, g.tw2x);
    a.S2 = S2;
    a.S = S;
    a.phi = phi;
    a.eps = eps;
    return launch(k_dd_x_ratio, a, dd_x_tiles(g.X, g.YZ), dd_x_smem(g.X), st, "dd x ratio", KC_DD_X_RATIO);
}

mvd_status dd_y(const FftGeom& g, cdd* S2, int inverse, cudaStream_t st) {
    if (g.fast && dd_fast_length(g.Y)) {
        mvd_status rc = MVD_ERR_UNSUPPORTED;
        const long nl = (long)g.Xh * g.Z;
        with_dd_len(g.Y, [&](auto Lc) {
            constexpr int L = decltype(Lc)::value;
            rc = launch_raw(inverse ? k_ddf_y<L, +1> : k_ddf_y<L, -1>, gen_div_up(nl, ddf_y_lines(L)), kDdThreads,
                            ddf_y_smem(L), st, "dd y (fast)", KC_DD_Y, S2, nl, g.tw2y, (float2*)nullptr);
        });
        return rc;
    }
    DdY a = dd_y_args(g.Y, g.Xh, g.Z, g.py, g.tw2y, S2);
    return launch(inverse ? k_dd_y<+1> : k_dd_y<-1>, a, dd_y_tiles(g.Y, g.Xh, g.Z), dd_y_smem(g.Y), st, "dd y",
                  KC_DD_Y);
}

bool dd_fast_yx(const FftGeom& g) { return g.fast && dd_fast_length(g.X) && dd_fast_length(g.Y); }

mvd_status dd_y_from_f32(const FftGeom& g, const float2* S1, cdd* S2, cudaStream_t st) {
    if (!dd_fast_yx(g)) {
        set_error("dd y from FP32: needs register-resident x and y lengths, got %d x %d", g.X, g.Y);
        return MVD_ERR_UNSUPPORTED;
    }
    mvd_status rc = MVD_ERR_UNSUPPORTED;
    const long nl = (long)g.Xh * g.Z;
    with_dd_len(g.Y, [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        rc = launch_raw(k_ddf_y<L, -1, 1>, gen_div_up(nl, ddf_y_lines(L)), kDdThreads, ddf_y_smem(L), st,
                        "dd y (FP32 in)", KC_DD_Y, S2, nl, g.tw2y, const_cast<float2*>(S1));
    });
    return rc;
}

mvd_status dd_x_update_generic(const FftGeom& g, const cdd* S2, float* psi, float eps, cudaStream_t st,
                               const float* wt, float lam, const float* inv_s, int accumulate) {
    DdXU u{};
    u.x = dd_x_args(g.X, g.YZ, g.px, g.tw2x);
    u.x.S2 = const_cast<cdd*>(S2);
    u.x.eps = eps;
    u.psi = psi;
    u.wt = wt;
    u.lam = lam;
    u.inv_s = inv_s;
    return launch(accumulate ? k_dd_x_update<4> : k_dd_x_update<1>, u, dd_x_tiles(g.X, g.YZ), dd_x_smem(g.X), st,
                  "dd x update", KC_X_UPDATE);
}

mvd_status dd_x_inverse_real_generic(const FftGeom& g, const cdd* S2, float* dst, cudaStream_t st) {
    DdXU u{};
    u.x = dd_x_args(g.X, g.YZ, g.px, g.tw2x);
    u.x.S2 = const_cast<cdd*>(S2);
    u.psi = dst;
    return launch(k_dd_x_update<0>, u, dd_x_tiles(g.X, g.YZ), dd_x_smem(g.X), st, "dd x inverse", KC_X_UPDATE);
}

mvd_status dd_x_update(const FftGeom& g, const cdd* S2, float* psi, float eps, cudaStream_t st, const float* wt,
                       float lam, const float* inv_s, int accumulate) {
    if (!dd_fast_x(g)) return dd_x_update_generic(g, S2, psi, eps, st, wt, lam, inv_s, accumulate);
    mvd_status rc = MVD_ERR_UNSUPPORTED;
    DdXUpd a{S2, psi, g.YZ, eps, g.tw2x, wt, lam, inv_s};
    with_dd_len(g.X, [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        rc = launch_raw(accumulate ? k_ddf_x_update<L, 4> : k_ddf_x_update<L, 1>, gen_div_up(g.YZ, 2 * ddf_pairs(L)),
                        kDdThreads, ddf_ratio_smem(L), st, "dd x update", KC_X_UPDATE, a);
    });
    return rc;
}

static mvd_status ddf_z(const FftGeom& g, cdd* S2, const cdd* K2, dd scale, bool mul, cudaStream_t st) {
    mvd_status rc = MVD_ERR_UNSUPPORTED;
    with_dd_len(g.Z, [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        constexpr int Q = ddf_z_cols(L);
        const int threads = Q * (L / kE8);
        const int nty = (int)gen_div_up(g.Y, Q);
        rc = launch_raw(mul ? k_ddf_z<L, true> : k_ddf_z<L, false>, (long)g.Xh * nty, threads, ddf_z_smem(L), st,
                        "dd z (fast)", mul ? KC_DD_Z_MUL : KC_SETUP, S2, K2, g.Y, g.YZ, nty, scale, g.tw2z);
    });
    return rc;
}

mvd_status dd_z_mul(const FftGeom& g, cdd* S2, const cdd* K2, cudaStream_t st) {
    if (g.fast && ddf_z2_length(g.Z)) {
        mvd_status rc = MVD_ERR_UNSUPPORTED;
        with_dd_len(g.Z, [&](auto Lc) {
            constexpr int L = decltype(Lc)::value;
            if constexpr (ddf_z2_length(L)) {
                constexpr int Q = ddf_z_cols(L);
                const int nty = (int)gen_div_up(g.Y, Q);
                const long nt = (long)g.Xh * nty;
                const size_t smem = ddf_z2_pipe_smem(L);
                rc = launch_raw(k_ddf_z2_pipe<L>, persistent_grid(k_ddf_z2_pipe<L>, Q * (L / kE8), smem, nt),
                                Q * (L / kE8), smem, st, "dd z", KC_DD_Z_MUL, S2, K2, g.Y, g.YZ, nty, g.tw2z, nt);
            }
        });
        return rc;
    }
    if (g.fast && dd_fast_length(g.Z)) return ddf_z(g, S2, K2, dd{1.f, 0.f}, true, st);
    DdZ a = dd_z_args(g.Z, g.Y, g.YZ, g.pz, g.tw2z, S2, K2, dd{1.f, 0.f});
    return launch(k_dd_z<true>, a, dd_z_tiles(g.Z, g.Y, g.Xh), dd_z_smem(g.Z, g.Y), st, "dd z", KC_DD_Z_MUL);
}

mvd_status dd_z_forward_scaled(const FftGeom& g, cdd* S2, double scale, cudaStream_t st) {
    const float hi = (float)scale;
    if (g.fast && dd_fast_length(g.Z)) return ddf_z(g, S2, nullptr, dd{hi, (float)(scale - (double)hi)}, false, st);
    DdZ a = dd_z_args(g.Z, g.Y, g.YZ, g.pz, g.tw2z, S2, nullptr, dd{hi, (float)(scale - (double)hi)});
    return launch(k_dd_z<false>, a, dd_z_tiles(g.Z, g.Y, g.Xh), dd_z_smem(g.Z, g.Y), st, "dd z forward", KC_SETUP);
}

}  // namespace mvd
