// Zero boundary: the volume continued by zeros instead of periodically.
//
// The engines work on a periodic grid padded on every axis by at least the
// largest PSF half-width (rounded up to a {2,3,5}-smooth size). The views and
// the estimate hold the user's volume in the low corner and zeros elsewhere,
// and the estimate's padding is cleared after every update, so each periodic
// convolution on the padded grid equals, on the user's volume, the convolution
// with a zero boundary (no term wraps into data). For this forward model the
// update is the ML-EM step of Shepp and Vardi (1982): the back-projected ratio
// is divided by the sensitivity s_v = 1 * P_v^comp (the back-projection of the
// indicator of the user's volume), which is 1 in the periodic case.
#include "common.cuh"
#include "dd.cuh"

namespace mvd {

namespace {

constexpr int kThreads = 256;

inline int grid_for(long n) {
    const long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

struct Geo {
    int X, Y, Z;     // padded grid
    int X0, Y0, Z0;  // user volume (low corner)
};

__device__ __forceinline__ bool inside(const Geo& g, long i, long* user_index) {
    const int x = (int)(i % g.X), y = (int)((i / g.X) % g.Y), z = (int)(i / ((long)g.X * g.Y));
    if (x >= g.X0 || y >= g.Y0 || z >= g.Z0) return false;
    if (user_index) *user_index = (long)x + (long)g.X0 * (y + (long)g.Y0 * z);
    return true;
}

// dst (padded) = src (user layout) inside, 0 outside
__global__ void k_pad(const float* src, Geo g, float* dst) {
    const long n = (long)g.X * g.Y * g.Z;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        long u = 0;
        dst[i] = inside(g, i, &u) ? src[u] : 0.f;
    }
}

// dst (user layout) = src (padded) inside
__global__ void k_crop(const float* src, Geo g, float* dst) {
    const long n = (long)g.X0 * g.Y0 * g.Z0;
    for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) {
        const int x = (int)(u % g.X0), y = (int)((u / g.X0) % g.Y0), z = (int)(u / ((long)g.X0 * g.Y0));
        dst[u] = src[(long)x + (long)g.X * (y + (long)g.Y * z)];
    }
}

__global__ void k_clear_padding(float* v, Geo g) {
    const long n = (long)g.X * g.Y * g.Z;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        if (!inside(g, i, nullptr)) v[i] = 0.f;
}

__global__ void k_indicator(float* v, Geo g) {
    const long n = (long)g.X * g.Y * g.Z;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        v[i] = inside(g, i, nullptr) ? 1.f : 0.f;
}

// 1 / s inside (s > 0 there: the compound kernel's centre tap is positive); 1 outside
__global__ void k_inverse_inside(float* s, Geo g) {
    const long n = (long)g.X * g.Y * g.Z;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        s[i] = inside(g, i, nullptr) ? 1.f / s[i] : 1.f;
}

inline Geo geo_of(const mvd_ctx* c) {
    return Geo{c->dims[0], c->dims[1], c->dims[2], c->udims[0], c->udims[1], c->udims[2]};
}

mvd_status launched(const char* what) {
    count_launch();
    return check_launch(what);
}

}  // namespace

mvd_status pad_volume(const mvd_ctx* c, const float* user, float* padded, cudaStream_t st) {
    k_pad<<<grid_for(c->M), kThreads, 0, st>>>(user, geo_of(c), padded);
    return launched("pad volume");
}

mvd_status crop_volume(const mvd_ctx* c, const float* padded, float* user, cudaStream_t st) {
    k_crop<<<grid_for(c->uM), kThreads, 0, st>>>(padded, geo_of(c), user);
    return launched("crop volume");
}

mvd_status clear_padding(const mvd_ctx* c, float* padded, cudaStream_t st) {
    k_clear_padding<<<grid_for(c->M), kThreads, 0, st>>>(padded, geo_of(c));
    return launched("clear padding");
}

// 1 / (indicator * K_v) for every view into c->d_invs (nv padded volumes):
// double-float convolution with the precise engine's kernel spectra where the
// x length allows, else the direct engine (direct contexts) or FP32 FFT passes.
mvd_status compute_inverse_sensitivity(mvd_ctx* c) {
    const Geo g = geo_of(c);
    const long M = c->M;
    cudaStream_t st = c->stream;
    float* ind = c->d_r;  // scratch volume: the indicator
    k_indicator<<<grid_for(M), kThreads, 0, st>>>(ind, g);
    MVD_TRY(launched("indicator"));
    for (int v = 0; v < c->nv; ++v) {
        float* s = c->d_invs + (size_t)v * M;
        const int* kd = &c->kd[3 * v];
        const float* K = c->d_comp + c->koff[v];
        if (c->path == MVD_PATH_DIRECT) {
            MVD_TRY(direct_conv(c->dims, ind, K, kd, s, st));
        } else if (c->precise && c->d_KP2 && dd_fast_x(c->geom)) {
            const size_t ns = (size_t)c->geom.Xh * c->geom.YZ;
            const cdd* Kc2 = reinterpret_cast<const cdd*>(reinterpret_cast<const float4*>(c->d_KP2) + ns * (2 * v + 1));
            MVD_TRY(dd_forward_real(c->geom, ind, c->d_S2, st));
            MVD_TRY(dd_y(c->geom, c->d_S2, 0, st));
            MVD_TRY(dd_z_mul(c->geom, c->d_S2, Kc2, st));
            MVD_TRY(dd_y(c->geom, c->d_S2, 1, st));
            MVD_TRY(dd_x_inverse_real(c->geom, c->d_S2, s, st));
        } else {
            // FP32: the kernel's spectrum in the work spectrum's twin (placed kernel -> x, y, z)
            float2* spec = nullptr;
            const size_t ns = (size_t)c->geom.Xh * c->geom.YZ;
            cudaError_t e = cudaMalloc(&spec, ns * sizeof(float2));
            if (e != cudaSuccess) return cuda_status(e, "sensitivity spectrum");
            mvd_status rc = place_kernel(c->dims, K, kd, s, st);
            if (rc == MVD_OK) rc = fft_forward_real(c->geom, s, spec, st);
            if (rc == MVD_OK) rc = fft_y(c->geom, spec, 0, st);
            if (rc == MVD_OK) rc = fft_z_forward_scaled(c->geom, spec, (float)(1.0 / (double)M), st);
            if (rc == MVD_OK) rc = fft_forward_real(c->geom, ind, c->d_S, st);
            if (rc == MVD_OK) rc = fft_y(c->geom, c->d_S, 0, st);
            if (rc == MVD_OK) rc = fft_z_mul(c->geom, c->d_S, spec, st);
            if (rc == MVD_OK) rc = fft_y(c->geom, c->d_S, 1, st);
            if (rc == MVD_OK) rc = fft_inverse_real(c->geom, c->d_S, s, st);
            cudaStreamSynchronize(st);
            cudaFree(spec);
            MVD_TRY(rc);
        }
        k_inverse_inside<<<grid_for(M), kThreads, 0, st>>>(s, g);
        MVD_TRY(launched("inverse sensitivity"));
    }
    return MVD_OK;
}

}  // namespace mvd
