// Periodic 3D convolution by FFT, split into line passes over HBM.
//
// Spectrum layout S[kx][z][y] (y fastest), kx in [0, Xh), Xh = X/2 + 1: the
// half spectrum of the real volume along x, stored plane by plane so that the
// x pass writes rows of consecutive y and the y and z passes read and write
// whole lines (y) or contiguous row segments (z) of one plane.
//
// One view update (Eq. 220 with the sequential order) runs as
//   xf : psi                  -> S      (real-to-complex along x)
//   y+ : S                    -> S      (forward along y)
//   zk : S                    -> S      (forward along z, times FFT(P_v)/M, inverse along z)
//   y- : S                    -> S
//   xr : S, phi_v             -> S      (inverse along x, r = phi/max(b,eps), forward along x)
//   y+, zk (FFT(P_v^comp)/M), y-
//   xu : S, psi               -> psi    (inverse along x, psi = max(psi . c, eps))
// The 1/M of the inverse transform is folded into the kernel spectra.
//
// Real lines are transformed two at a time: rows a and b of a tile form one
// complex line a + i b; after the complex FFT, A[k] = (Z[k] + conj Z[-k]) / 2
// and B[k] = (Z[k] - conj Z[-k]) / (2i). The inverse builds Z = A + i B from
// the two Hermitian half spectra and returns a (real part) and b (imaginary).
#include "fft_generic.cuh"

namespace mvd {

namespace {

__global__ void __launch_bounds__(kGenThreads) k_x_forward(GenX a) {
    extern __shared__ float2 sm[];
    gen_x_forward_tile<false>(a, blockIdx.x, sm);
}

__global__ void __launch_bounds__(kGenThreads) k_x_ratio(GenX a) {
    extern __shared__ float2 sm[];
    gen_x_ratio_tile<false>(a, blockIdx.x, sm);
}

template <int MODE>
__global__ void __launch_bounds__(kGenThreads) k_x_inverse(GenX a) {
    extern __shared__ float2 sm[];
    gen_x_inverse_tile<false, MODE>(a, blockIdx.x, sm);
}

template <int S>
__global__ void __launch_bounds__(kGenThreads) k_y(GenY a) {
    extern __shared__ float2 sm[];
    gen_y_tile<false, S>(a, blockIdx.x, sm);
}

template <bool MUL>
__global__ void __launch_bounds__(kGenThreads) k_z(GenZ a) {
    extern __shared__ float2 sm[];
    gen_z_tile<false, MUL>(a, blockIdx.x, sm);
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

GenX make_x(const FftGeom& g) { return gen_x_args(g.X, g.YZ, g.px); }

}  // namespace

mvd_status fft_forward_real_generic(const FftGeom& g, const float* src, float2* S, cudaStream_t st) {
    GenX a = make_x(g);
    a.src = src;
    a.S = S;
    return launch(k_x_forward, a, gen_x_tiles(g.X, g.YZ), gen_x_smem(g.X), st, "fft x forward", KC_X_FORWARD);
}

mvd_status fft_x_ratio_generic(const FftGeom& g, float2* S, const float* phi, float eps, cudaStream_t st) {
    GenX a = make_x(g);
    a.S = S;
    a.phi = phi;
    a.eps = eps;
    return launch(k_x_ratio, a, gen_x_tiles(g.X, g.YZ), gen_x_smem(g.X), st, "fft x ratio", KC_X_RATIO);
}

mvd_status fft_x_update_generic(const FftGeom& g, const float2* S, float* psi, float eps, cudaStream_t st,
                                const float* wt, float lam, const float* inv_s) {
    GenX a = make_x(g);
    a.S = const_cast<float2*>(S);
    a.psi = psi;
    a.eps = eps;
    a.wt = wt;
    a.lam = lam;
    a.inv_s = inv_s;
    return launch(k_x_inverse<1>, a, gen_x_tiles(g.X, g.YZ), gen_x_smem(g.X), st, "fft x update", KC_X_UPDATE);
}

mvd_status fft_x_accumulate_generic(const FftGeom& g, const float2* S, float* acc, cudaStream_t st,
                                    const float* inv_s) {
    GenX a = make_x(g);
    a.S = const_cast<float2*>(S);
    a.psi = acc;
    a.inv_s = inv_s;
    return launch(k_x_inverse<4>, a, gen_x_tiles(g.X, g.YZ), gen_x_smem(g.X), st, "fft x accumulate", KC_X_UPDATE);
}

mvd_status fft_inverse_real_generic(const FftGeom& g, const float2* S, float* dst, cudaStream_t st) {
    GenX a = make_x(g);
    a.S = const_cast<float2*>(S);
    a.psi = dst;
    return launch(k_x_inverse<0>, a, gen_x_tiles(g.X, g.YZ), gen_x_smem(g.X), st, "fft x inverse", KC_SETUP);
}

mvd_status fft_x_inverse_dd(const FftGeom& g, const cdd* S2, float* dst, cudaStream_t st) {
    if (dd_fast_x(g)) return dd_x_inverse_real(g, S2, dst, st);
    return dd_x_inverse_real_generic(g, S2, dst, st);
}

mvd_status fft_y_generic(const FftGeom& g, float2* S, int inverse, cudaStream_t st) {
    GenY a = gen_y_args(g.Y, g.Xh, g.Z, g.py, S);
    return launch(inverse ? k_y<+1> : k_y<-1>, a, gen_y_tiles(g.Y, g.Xh, g.Z), gen_y_smem(g.Y), st, "fft y", KC_Y);
}

mvd_status fft_z_mul_generic(const FftGeom& g, float2* S, const float2* K, cudaStream_t st) {
    GenZ a = gen_z_args(g.Z, g.Y, g.YZ, g.pz, S, K, 1.f);
    return launch(k_z<true>, a, gen_z_tiles(g.Z, g.Y, g.Xh), gen_z_smem(g.Z, g.Y), st, "fft z", KC_Z_MUL);
}

mvd_status fft_z_forward_scaled_generic(const FftGeom& g, float2* S, float scale, cudaStream_t st) {
    GenZ a = gen_z_args(g.Z, g.Y, g.YZ, g.pz, S, nullptr, scale);
    return launch(k_z<false>, a, gen_z_tiles(g.Z, g.Y, g.Xh), gen_z_smem(g.Z, g.Y), st, "fft z forward", KC_SETUP);
}

// ---------------------------------------------------------------------------
// public passes: the register-resident kernels when the axis length is a
// supported power of two (and the generic engine is not forced), else the
// generic shared-memory Stockham kernels above
// ---------------------------------------------------------------------------
mvd_status fft_forward_real(const FftGeom& g, const float* src, float2* S, cudaStream_t st) {
    if (g.fast && fft_fast_supported(g.X)) return fft_forward_real_fast(g, src, S, st);
    return fft_forward_real_generic(g, src, S, st);
}
mvd_status fft_x_ratio(const FftGeom& g, float2* S, const float* phi, float eps, cudaStream_t st) {
    if (g.fast && fft_fast_supported(g.X)) return fft_x_ratio_fast(g, S, phi, eps, st);
    return fft_x_ratio_generic(g, S, phi, eps, st);
}
mvd_status fft_x_update(const FftGeom& g, const float2* S, float* psi, float eps, cudaStream_t st,
                        const float* wt, float lam, const float* inv_s) {
    if (g.fast && fft_fast_supported(g.X)) return fft_x_update_fast(g, S, psi, eps, st, wt, lam, inv_s);
    return fft_x_update_generic(g, S, psi, eps, st, wt, lam, inv_s);
}
mvd_status fft_x_accumulate(const FftGeom& g, const float2* S, float* acc, cudaStream_t st, const float* inv_s) {
    if (g.fast && fft_fast_supported(g.X)) return fft_x_accumulate_fast(g, S, acc, st, inv_s);
    return fft_x_accumulate_generic(g, S, acc, st, inv_s);
}
mvd_status fft_inverse_real(const FftGeom& g, const float2* S, float* dst, cudaStream_t st) {
    if (g.fast && fft_fast_supported(g.X)) return fft_inverse_real_fast(g, S, dst, st);
    return fft_inverse_real_generic(g, S, dst, st);
}
mvd_status fft_y(const FftGeom& g, float2* S, int inverse, cudaStream_t st) {
    if (g.fast && fft_fast_supported(g.Y)) return fft_y_fast(g, S, inverse, st);
    return fft_y_generic(g, S, inverse, st);
}
mvd_status fft_z_mul(const FftGeom& g, float2* S, const float2* K, cudaStream_t st) {
    if (g.fast && fft_fast_z_supported(g.Z)) return fft_z_mul_fast(g, S, K, st);
    return fft_z_mul_generic(g, S, K, st);
}
mvd_status fft_z_forward_scaled(const FftGeom& g, float2* S, float scale, cudaStream_t st) {
    if (g.fast && fft_fast_z_supported(g.Z)) return fft_z_forward_scaled_fast(g, S, scale, st);
    return fft_z_forward_scaled_generic(g, S, scale, st);
}

}  // namespace mvd
