// Direct periodic 3D convolution for small kernels, with the update's
// elementwise steps fused into the epilogue:
//   ratio : r   = phi / max(psi * P, eps)        (Eq. 15 / Eq. 51, first half)
//   update: psi = max(psi . (r * K), eps)         (Eq. 15 / Eq. 220, second half)
// (f * k)(x) = sum_d k(d) f((x - d) mod dims), d = tap index - (K-1)/2.
//
// Each block computes a TX x TY x TZ output tile. The input tile plus the
// kernel's halo (periodically wrapped) and the kernel taps are staged in
// shared memory; every thread accumulates TZ outputs along z, so each input
// value it loads feeds up to TZ FMAs.
#include "common.cuh"
#include "fft.cuh"

namespace mvd {

namespace {

constexpr int TX = 32, TZ = 4;
constexpr size_t kMaxSmem = 200 * 1024;

// tile height TY (8, 4, 2 or 1 rows of 32 threads): the largest whose input
// tile + halo and kernel taps fit in shared memory
inline size_t smem_bytes(const int kd[3], int ty) {
    const size_t T = (size_t)kd[0] * kd[1] * kd[2];
    const size_t tile = (size_t)(TX + kd[0] - 1) * (ty + kd[1] - 1) * (TZ + kd[2] - 1);
    return (T + tile) * sizeof(float);
}
inline int pick_ty(const int kd[3]) {
    for (int ty : {8, 4, 2, 1})
        if (smem_bytes(kd, ty) <= kMaxSmem) return ty;
    return 0;
}

struct DArgs {
    int X, Y, Z, Kx, Ky, Kz;
    const float* in;
    const float* k;
    const float* phi;
    float* out;  // r (ratio), psi (update) or plain output
    float eps;
    const float* wt;  // update: when set, apply the fraction wt of the change (partial overlap)
    float lam;        // update: Tikhonov regularisation (0 = none)
    const float* inv_s;  // update / accumulate: zero boundary, 1 / sensitivity
};

// MODE 0: out = phi / max(conv, eps); MODE 1: out = max(out . conv, eps); MODE 2: out = conv;
// MODE 3: out += conv; MODE 4: out *= conv (the combined update's product)
template <int MODE, int TY>
__global__ void __launch_bounds__(TX * TY) k_direct(DArgs a) {
    extern __shared__ float smem[];
    const int T = a.Kx * a.Ky * a.Kz;
    float* sk = smem;
    float* st = smem + T;
    const int WX = TX + a.Kx - 1, WY = TY + a.Ky - 1, WZ = TZ + a.Kz - 1;
    const int hx = (a.Kx - 1) / 2, hy = (a.Ky - 1) / 2, hz = (a.Kz - 1) / 2;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;

    for (int i = threadIdx.x; i < T; i += blockDim.x) sk[i] = __ldg(a.k + i);
    const int nt = WX * WY * WZ;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        const int ix = i % WX, r = i / WX, iy = r % WY, iz = r / WY;
        int gx = (x0 - hx + ix) % a.X;
        if (gx < 0) gx += a.X;
        int gy = (y0 - hy + iy) % a.Y;
        if (gy < 0) gy += a.Y;
        int gz = (z0 - hz + iz) % a.Z;
        if (gz < 0) gz += a.Z;
        st[i] = __ldg(a.in + (long)gx + (long)a.X * (gy + (long)a.Y * gz));
    }
    __syncthreads();

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;  // ty < TY
    float acc[TZ];
#pragma unroll
    for (int o = 0; o < TZ; ++o) acc[o] = 0.f;
    // output o at tile z index o uses input plane i = o + (Kz-1) - kz
    for (int ky = 0; ky < a.Ky; ++ky) {
        const int iy = ty + (a.Ky - 1) - ky;
        for (int kx = 0; kx < a.Kx; ++kx) {
            const int ix = tx + (a.Kx - 1) - kx;
            const float* col = st + ix + WX * iy;
            const float* kcol = sk + kx + a.Kx * ky;
            for (int i = 0; i < WZ; ++i) {
                const float v = col[(long)WX * WY * i];
#pragma unroll
                for (int o = 0; o < TZ; ++o) {
                    const int kz = o + (a.Kz - 1) - i;
                    if (kz >= 0 && kz < a.Kz) acc[o] = fmaf(kcol[a.Kx * a.Ky * kz], v, acc[o]);
                }
            }
        }
    }
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= a.X || gy >= a.Y) return;
#pragma unroll
    for (int o = 0; o < TZ; ++o) {
        const int gz = z0 + o;
        if (gz >= a.Z) break;
        const long g = (long)gx + (long)a.X * (gy + (long)a.Y * gz);
        if (MODE == 0)
            a.out[g] = __ldg(a.phi + g) / fmaxf(acc[o], a.eps);
        else if (MODE == 1)
        {
            const float p = a.out[g];
            a.out[g] = fmaxf(p * (a.wt || a.lam != 0.f || a.inv_s ? update_factor(acc[o] - 1.f, p, a.wt, g, a.lam,
                                                                                    a.inv_s)
                                                                   : acc[o]),
                             a.eps);
        }
        else if (MODE == 2)
            a.out[g] = acc[o];
        else if (MODE == 3)
            a.out[g] += acc[o];
        else  // MODE 4: combined update, multiply this view's factor into the product
            a.out[g] *= a.inv_s ? acc[o] * __ldg(a.inv_s + g) : acc[o];
    }
}

template <int MODE, int TY>
mvd_status launch_ty(const DArgs& a, size_t sm, cudaStream_t st, const char* name) {
    cudaError_t e = cudaFuncSetAttribute(k_direct<MODE, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_status(e, name);
    dim3 grid((a.X + TX - 1) / TX, (a.Y + TY - 1) / TY, (a.Z + TZ - 1) / TZ);
    const int cls = MODE == 0 ? KC_DIRECT_RATIO : (MODE == 1 || MODE == 4) ? KC_DIRECT_UPDATE : KC_DIRECT_CONV;
    prof_begin(cls, st);
    k_direct<MODE, TY><<<grid, TX * TY, sm, st>>>(a);
    prof_end(cls, st);
    count_launch();
    return check_launch(name);
}

template <int MODE>
mvd_status launch(const DArgs& a, const int kd[3], cudaStream_t st, const char* name, int ty_req = 0) {
    const int ty = (ty_req == 8 || ty_req == 4 || ty_req == 2 || ty_req == 1) && smem_bytes(kd, ty_req) <= kMaxSmem
                       ? ty_req
                       : pick_ty(kd);
    if (ty == 0) {
        set_error("%s: kernel box %dx%dx%d too large for the direct engine", name, kd[0], kd[1], kd[2]);
        return MVD_ERR_UNSUPPORTED;
    }
    const size_t sm = smem_bytes(kd, ty);
    switch (ty) {
        case 8: return launch_ty<MODE, 8>(a, sm, st, name);
        case 4: return launch_ty<MODE, 4>(a, sm, st, name);
        case 2: return launch_ty<MODE, 2>(a, sm, st, name);
        default: return launch_ty<MODE, 1>(a, sm, st, name);
    }
}

DArgs make(const int dims[3], const float* in, const float* k, const int kd[3]) {
    DArgs a{};
    a.X = dims[0];
    a.Y = dims[1];
    a.Z = dims[2];
    a.Kx = kd[0];
    a.Ky = kd[1];
    a.Kz = kd[2];
    a.in = in;
    a.k = k;
    return a;
}

}  // namespace

bool direct_supported(const int kd[3]) { return pick_ty(kd) > 0; }

int direct_tile_heights(const int kd[3], int out[4]) {
    int n = 0;
    for (int ty : {8, 4, 2, 1})
        if (smem_bytes(kd, ty) <= kMaxSmem) out[n++] = ty;
    return n;
}

mvd_status direct_ratio(const int dims[3], const float* psi, const float* k, const int kd[3],
                        const float* phi, float eps, float* r, cudaStream_t st, int ty) {
    DArgs a = make(dims, psi, k, kd);
    a.phi = phi;
    a.out = r;
    a.eps = eps;
    return launch<0>(a, kd, st, "direct ratio", ty);
}

mvd_status direct_update(const int dims[3], const float* r, const float* k, const int kd[3],
                         float* psi, float eps, cudaStream_t st, int ty, const float* wt, float lam,
                         const float* inv_s) {
    DArgs a = make(dims, r, k, kd);
    a.out = psi;
    a.eps = eps;
    a.wt = wt;
    a.lam = lam;
    a.inv_s = inv_s;
    return launch<1>(a, kd, st, "direct update", ty);
}

mvd_status direct_accumulate(const int dims[3], const float* r, const float* k, const int kd[3], float* prod,
                             cudaStream_t st, int ty, const float* inv_s) {
    DArgs a = make(dims, r, k, kd);
    a.out = prod;
    a.inv_s = inv_s;
    return launch<4>(a, kd, st, "direct accumulate", ty);
}

mvd_status direct_conv(const int dims[3], const float* in, const float* k, const int kd[3], float* out,
                       cudaStream_t st) {
    DArgs a = make(dims, in, k, kd);
    a.out = out;
    return launch<2>(a, kd, st, "direct conv");
}

mvd_status direct_conv_add(const int dims[3], const float* in, const float* k, const int kd[3], float* out,
                           cudaStream_t st) {
    DArgs a = make(dims, in, k, kd);
    a.out = out;
    return launch<3>(a, kd, st, "direct conv add");
}

}  // namespace mvd
