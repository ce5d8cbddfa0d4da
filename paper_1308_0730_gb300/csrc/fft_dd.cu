// Kernels and launchers of the double-float forward-blur passes (tile
// functions in fft_dd.cuh).
#include "fft_dd.cuh"

namespace mvd {

namespace {

__global__ void __launch_bounds__(kGenThreads) k_dd_x_forward(DdX a) {
    extern __shared__ cdd smd[];
    dd_x_forward_tile<false>(a, blockIdx.x, smd);
}

__global__ void __launch_bounds__(kGenThreads) k_dd_x_ratio(DdX a) {
    extern __shared__ cdd smd[];
    dd_x_ratio_tile<false>(a, blockIdx.x, smd);
}

template <int S>
__global__ void __launch_bounds__(kGenThreads) k_dd_y(DdY a) {
    extern __shared__ cdd smd[];
    dd_y_tile<false, S>(a, blockIdx.x, smd);
}

template <bool MUL>
__global__ void __launch_bounds__(kGenThreads) k_dd_z(DdZ a) {
    extern __shared__ cdd smd[];
    dd_z_tile<false, MUL>(a, blockIdx.x, smd);
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
    DdX a = dd_x_args(g.X, g.YZ, g.px, g.tw2x);
    a.src = src;
    a.S2 = S2;
    return launch(k_dd_x_forward, a, dd_x_tiles(g.X, g.YZ), dd_x_smem(g.X), st, "dd x forward", KC_DD_X_FORWARD);
}

mvd_status dd_x_ratio(const FftGeom& g, const cdd* S2, const float* phi, float eps, float2* S, cudaStream_t st) {
    DdX a = dd_x_args(g.X, g.YZ, g.px, g.tw2x);
    a.S2 = const_cast<cdd*>(S2);
    a.phi = phi;
    a.eps = eps;
    a.S = S;
    return launch(k_dd_x_ratio, a, dd_x_tiles(g.X, g.YZ), dd_x_smem(g.X), st, "dd x ratio", KC_DD_X_RATIO);
}

mvd_status dd_y(const FftGeom& g, cdd* S2, int inverse, cudaStream_t st) {
    DdY a = dd_y_args(g.Y, g.Xh, g.Z, g.py, g.tw2y, S2);
    return launch(inverse ? k_dd_y<+1> : k_dd_y<-1>, a, dd_y_tiles(g.Y, g.Xh, g.Z), dd_y_smem(g.Y), st, "dd y",
                  KC_DD_Y);
}

mvd_status dd_z_mul(const FftGeom& g, cdd* S2, const cdd* K2, cudaStream_t st) {
    DdZ a = dd_z_args(g.Z, g.Y, g.YZ, g.pz, g.tw2z, S2, K2, dd{1.f, 0.f});
    return launch(k_dd_z<true>, a, dd_z_tiles(g.Z, g.Y, g.Xh), dd_z_smem(g.Z, g.Y), st, "dd z", KC_DD_Z_MUL);
}

mvd_status dd_z_forward_scaled(const FftGeom& g, cdd* S2, double scale, cudaStream_t st) {
    const float hi = (float)scale;
    DdZ a = dd_z_args(g.Z, g.Y, g.YZ, g.pz, g.tw2z, S2, nullptr, dd{hi, (float)(scale - (double)hi)});
    return launch(k_dd_z<false>, a, dd_z_tiles(g.Z, g.Y, g.Xh), dd_z_smem(g.Z, g.Y), st, "dd z forward", KC_SETUP);
}

}  // namespace mvd
