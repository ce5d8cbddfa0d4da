// Zero and mirror boundaries: the volume continued by zeros, or by its
// half-sample symmetric reflection, instead of periodically.
//
// The engines work on a periodic grid padded on every axis by at least the
// largest PSF half-width h (zero) or 2h (mirror), rounded up to a
// {2,3,5}-smooth size. The views hold the user's volume in the low corner and
// zeros elsewhere, so the ratio phi / b vanishes in the padding.
//
// Zero: the estimate's padding is cleared after every update, so each
// periodic convolution on the padded grid equals, on the user's volume, the
// convolution with a zero boundary (no term wraps into data).
//
// Mirror: the estimate's halo (h voxels past each face, the high side at
// D..D+h-1, the low side wrapped to D'-h..D'-1) holds its reflection, so the
// forward blur sees the reflected continuation. The back-projection of the
// ratio on the padded grid spreads into the halo without aliasing (D' >= D+2h)
// and is folded back: every voxel adds the values at its reflections.
//
// For both forward models the update is the ML-EM step of Shepp and Vardi
// (1982): the back-projected ratio is divided by the sensitivity s_v (the
// back-projection of the indicator of the user's volume), which is 1 in the
// periodic case.
#include "common.cuh"
#include "dd.cuh"
#include "fft.cuh"

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
    int hx, hy, hz;  // halo (mirror boundary)
};

// Positions on one padded axis that reflect onto user coordinate j: j itself,
// -1-j (stored at D'-1-j) when j < h, 2D-1-j when j >= D-h. Returns the count.
__device__ __forceinline__ int axis_images(int j, int D, int Dp, int h, int pos[3]) {
    int n = 0;
    pos[n++] = j;
    if (j < h) pos[n++] = Dp - 1 - j;
    if (j >= D - h) pos[n++] = 2 * D - 1 - j;
    return n;
}

// The user coordinate a padded position reflects from, or -1 outside the halo.
__device__ __forceinline__ int axis_source(int p, int D, int Dp, int h) {
    if (p < D) return p;
    if (p < D + h) return 2 * D - 1 - p;
    if (p >= Dp - h) return Dp - 1 - p;
    return -1;
}

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

// padding outside the user's volume: the reflection in the halo, 0 beyond
__global__ void k_mirror_fill(float* v, Geo g) {
    const long n = (long)g.X * g.Y * g.Z;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.X), y = (int)((i / g.X) % g.Y), z = (int)(i / ((long)g.X * g.Y));
        if (x < g.X0 && y < g.Y0 && z < g.Z0) continue;
        const int sx = axis_source(x, g.X0, g.X, g.hx), sy = axis_source(y, g.Y0, g.Y, g.hy),
                  sz = axis_source(z, g.Z0, g.Z, g.hz);
        v[i] = (sx < 0 || sy < 0 || sz < 0) ? 0.f : v[(long)sx + (long)g.X * (sy + (long)g.Y * sz)];
    }
}

// The reflections of user voxel (x, y, z) on the padded grid; fold() sums
// cp + off over them (plain loads: k_fold_inplace reads what it writes).
struct Images {
    int px[3], py[3], pz[3];
    int nx, ny, nz;
};

__device__ __forceinline__ Images images_of(const Geo& g, int x, int y, int z) {
    Images m;
    m.nx = axis_images(x, g.X0, g.X, g.hx, m.px);
    m.ny = axis_images(y, g.Y0, g.Y, g.hy, m.py);
    m.nz = axis_images(z, g.Z0, g.Z, g.hz, m.pz);
    return m;
}

__device__ __forceinline__ float fold(const Geo& g, const Images& m, const float* cp, float off) {
    float s = 0.f;
    for (int c = 0; c < m.nz; ++c)
        for (int b = 0; b < m.ny; ++b)
            for (int a = 0; a < m.nx; ++a)
                s += cp[(long)m.px[a] + (long)g.X * (m.py[b] + (long)g.Y * m.pz[c])] + off;
    return s;
}

// psi = max(psi . F, eps) for every user voxel, F the folded back-projection
// f = fold(cp + off) . inv_s composed with the view weight w and Tikhonov
// lambda as in the periodic update (1 + w (f - 1 - lambda psi) / (1 + lambda
// psi)), written to the voxel and to its reflections in the halo (each halo
// position has one source voxel, so no two threads write the same address)
__global__ void k_mirror_update(float* psi, const float* cp, float off, const float* inv_s, float eps, Geo g,
                                const float* wt, float lam) {
    const long n = (long)g.X0 * g.Y0 * g.Z0;
    for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) {
        const int x = (int)(u % g.X0), y = (int)((u / g.X0) % g.Y0), z = (int)(u / ((long)g.X0 * g.Y0));
        const Images m = images_of(g, x, y, z);
        const long i = (long)x + (long)g.X * (y + (long)g.Y * z);
        const float p = psi[i];
        const float f = update_factor(fold(g, m, cp, off) * __ldg(inv_s + i) - 1.f, p, wt, i, lam);
        const float v = fmaxf(p * f, eps);
        for (int c = 0; c < m.nz; ++c)
            for (int b = 0; b < m.ny; ++b)
                for (int a = 0; a < m.nx; ++a)
                    psi[(long)m.px[a] + (long)g.X * (m.py[b] + (long)g.Y * m.pz[c])] = v;
    }
}

// combined update: prod *= fold(cp + off) . inv_s at every user voxel
__global__ void k_mirror_accumulate(float* prod, const float* cp, float off, const float* inv_s, Geo g) {
    const long n = (long)g.X0 * g.Y0 * g.Z0;
    for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) {
        const int x = (int)(u % g.X0), y = (int)((u / g.X0) % g.Y0), z = (int)(u / ((long)g.X0 * g.Y0));
        const long i = (long)x + (long)g.X * (y + (long)g.Y * z);
        prod[i] *= fold(g, images_of(g, x, y, z), cp, off) * __ldg(inv_s + i);
    }
}

// the fold in place (inside voxels only; each reads its own reflections)
__global__ void k_fold_inplace(float* v, Geo g) {
    const long n = (long)g.X0 * g.Y0 * g.Z0;
    for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) {
        const int x = (int)(u % g.X0), y = (int)((u / g.X0) % g.Y0), z = (int)(u / ((long)g.X0 * g.Y0));
        v[(long)x + (long)g.X * (y + (long)g.Y * z)] = fold(g, images_of(g, x, y, z), v, 0.f);
    }
}

inline Geo geo_of(const mvd_ctx* c) {
    return Geo{c->dims[0],  c->dims[1],  c->dims[2],  c->udims[0], c->udims[1],
               c->udims[2], c->halo[0], c->halo[1], c->halo[2]};
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

mvd_status mirror_fill(const mvd_ctx* c, float* padded, cudaStream_t st) {
    k_mirror_fill<<<grid_for(c->M), kThreads, 0, st>>>(padded, geo_of(c));
    return launched("mirror fill");
}

mvd_status mirror_update(const mvd_ctx* c, const float* cp, float off, const float* inv_s, cudaStream_t st,
                         const float* wt, float lam) {
    k_mirror_update<<<grid_for(c->uM), kThreads, 0, st>>>(c->d_psi, cp, off, inv_s, c->eps, geo_of(c), wt, lam);
    return launched("mirror update");
}

mvd_status mirror_accumulate(const mvd_ctx* c, const float* cp, float off, const float* inv_s, float* prod,
                             cudaStream_t st) {
    k_mirror_accumulate<<<grid_for(c->uM), kThreads, 0, st>>>(prod, cp, off, inv_s, geo_of(c));
    return launched("mirror accumulate");
}

mvd_status finish_padding(const mvd_ctx* c, float* padded, cudaStream_t st) {
    if (c->boundary == MVD_BOUNDARY_ZERO) return clear_padding(c, padded, st);
    if (c->boundary == MVD_BOUNDARY_MIRROR) return mirror_fill(c, padded, st);
    return MVD_OK;
}

// 1 / s_v for every view into c->d_invs (nv padded volumes): s_v is the
// indicator of the user's volume convolved with P_v^comp on the padded grid
// (folded for the mirror boundary), with the context's engine and precision.
mvd_status compute_inverse_sensitivity(mvd_ctx* c) {
    const Geo g = geo_of(c);
    const long M = c->M;
    cudaStream_t st = c->stream;
    float* ind = c->d_r;  // scratch volume: the indicator
    k_indicator<<<grid_for(M), kThreads, 0, st>>>(ind, g);
    MVD_TRY(launched("indicator"));
    const FftGeom& fg = c->geom;
    const size_t ns = (size_t)fg.Xh * fg.YZ;
    for (int v = 0; v < c->nv; ++v) {
        float* s = c->d_invs + (size_t)v * M;
        if (c->path == MVD_PATH_DIRECT) {
            MVD_TRY(direct_conv(c->dims, ind, c->d_comp + c->koff[v], &c->kd[3 * v], s, st));
        } else if (c->precise) {
            const cdd* Kc2 = reinterpret_cast<const cdd*>(reinterpret_cast<const float4*>(c->d_KP2) + ns * (2 * v + 1));
            MVD_TRY(dd_forward_real(fg, ind, c->d_S2, st));
            MVD_TRY(dd_y(fg, c->d_S2, 0, st));
            MVD_TRY(dd_z_mul(fg, c->d_S2, Kc2, st));
            MVD_TRY(dd_y(fg, c->d_S2, 1, st));
            MVD_TRY(fft_x_inverse_dd(fg, c->d_S2, s, st));
        } else {
            MVD_TRY(fft_forward_real(fg, ind, c->d_S, st));
            MVD_TRY(fft_y(fg, c->d_S, 0, st));
            MVD_TRY(fft_z_mul(fg, c->d_S, c->d_K + ns * (2 * v + 1), st));
            MVD_TRY(fft_y(fg, c->d_S, 1, st));
            MVD_TRY(fft_inverse_real(fg, c->d_S, s, st));
        }
        if (c->boundary == MVD_BOUNDARY_MIRROR) {
            k_fold_inplace<<<grid_for(c->uM), kThreads, 0, st>>>(s, g);
            MVD_TRY(launched("fold sensitivity"));
        }
        k_inverse_inside<<<grid_for(M), kThreads, 0, st>>>(s, g);
        MVD_TRY(launched("inverse sensitivity"));
    }
    return MVD_OK;
}

}  // namespace mvd
