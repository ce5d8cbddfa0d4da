// Device-side set-up work: compound kernels (Eq. 222 / Eq. 230 / Eq. 240),
// kernel placement on the periodic grid, view statistics (psi0 and input
// validation) and small helpers.
//
// Kernels are functions on Z^3 supported on a centred odd box; kernel algebra
// (P_v^* * P_w * P_w^*) is linear convolution of those small functions. The
// compound kernel of view v is zero outside P_v^*'s box, so every factor is
// evaluated on that box only.
#include "box_sum.cuh"
#include "common.cuh"

namespace mvd {

namespace {

constexpr int kThreads = 256;

struct Box {
    int kx, ky, kz;  // sizes
    __device__ __forceinline__ int hx() const { return (kx - 1) / 2; }
    __device__ __forceinline__ int hy() const { return (ky - 1) / 2; }
    __device__ __forceinline__ int hz() const { return (kz - 1) / 2; }
    __device__ __forceinline__ int size() const { return kx * ky * kz; }
    // value at offset (dx,dy,dz) from the centre
    __device__ __forceinline__ float at(const float* k, int dx, int dy, int dz) const {
        return __ldg(k + (dx + hx()) + kx * ((dy + hy()) + ky * (dz + hz())));
    }
};

__device__ __forceinline__ void offset_of(const Box& b, int i, int& dx, int& dy, int& dz) {
    dx = i % b.kx - b.hx();
    const int r = i / b.kx;
    dy = r % b.ky - b.hy();
    dz = r / b.ky - b.hz();
}

// Q(d) = sum_e P(e) P(e - d)   (P * P^*), on the box of size 2K-1; one warp per d
__global__ void k_autocorr(const float* P, Box b, float* Q, Box q) {
    const int i = (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5);
    if (i >= q.size()) return;
    int dx, dy, dz;
    offset_of(q, i, dx, dy, dz);
    // e and e - d both inside b
    const int zlo = max(-b.hz(), dz - b.hz()), zhi = min(b.hz(), dz + b.hz());
    const int ylo = max(-b.hy(), dy - b.hy()), yhi = min(b.hy(), dy + b.hy());
    const int xlo = max(-b.hx(), dx - b.hx()), xhi = min(b.hx(), dx + b.hx());
    const float s = warp_box_sum(xlo, xhi, ylo, yhi, zlo, zhi, [&](int ex, int ey, int ez, float acc) {
        return fmaf(b.at(P, ex, ey, ez), b.at(P, ex - dx, ey - dy, ez - dz), acc);
    });
    if ((threadIdx.x & 31) == 0) Q[i] = s;
}

// out(d) = P^*(d) = P(-d)
__global__ void k_mirror(const float* P, Box b, float* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.size()) return;
    int dx, dy, dz;
    offset_of(b, i, dx, dy, dz);
    out[i] = b.at(P, -dx, -dy, -dz);
}

// out(d) *= sum_e P^*(e) G(d - e)  for d on P's box  (P^*(e) = P(-e)); one warp per d
__global__ void k_mul_conv(const float* P, Box b, const float* G, Box g, float* out) {
    const int i = (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5);
    if (i >= b.size()) return;
    int dx, dy, dz;
    offset_of(b, i, dx, dy, dz);
    const int zlo = max(-b.hz(), dz - g.hz()), zhi = min(b.hz(), dz + g.hz());
    const int ylo = max(-b.hy(), dy - g.hy()), yhi = min(b.hy(), dy + g.hy());
    const int xlo = max(-b.hx(), dx - g.hx()), xhi = min(b.hx(), dx + g.hx());
    const float s = warp_box_sum(xlo, xhi, ylo, yhi, zlo, zhi, [&](int ex, int ey, int ez, float acc) {
        return fmaf(b.at(P, -ex, -ey, -ez), g.at(G, dx - ex, dy - ey, dz - ez), acc);
    });
    if ((threadIdx.x & 31) == 0) out[i] *= s;
}

// out(d) *= P^*(d)
__global__ void k_mul_mirror(const float* P, Box b, float* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.size()) return;
    int dx, dy, dz;
    offset_of(b, i, dx, dy, dz);
    out[i] *= b.at(P, -dx, -dy, -dz);
}

// one block: out /= sum(out) (sum in FP64); flag if the sum is not > 0
__global__ void k_normalize(float* out, int n, int* bad) {
    __shared__ double part[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += out[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    const double tot = part[0];
    if (!(tot > 0.0)) {
        if (threadIdx.x == 0) *bad = 1;
        return;
    }
    const float inv = (float)(1.0 / tot);
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] *= inv;
}

__global__ void k_place(const float* k, Box b, int X, int Y, int Z, float* vol) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.size()) return;
    int dx, dy, dz;
    offset_of(b, i, dx, dy, dz);
    const int x = (dx % X + X) % X, y = (dy % Y + Y) % Y, z = (dz % Z + Z) % Z;
    vol[(long)x + (long)X * (y + (long)Y * z)] = __ldg(k + i);
}

// sum of all values (FP64) and a flag for negative or non-finite values
// Sum (FP64) and validity of n floats. Four consecutive values are added in
// FP32 before the FP64 accumulation (at most three FP32 roundings of a
// four-term sum, relative 2e-7 of it; exact for photon counts below 2^22):
// the FP64 adds are the slow part of this pass on a GPU with few FP64 units.
__global__ void k_stats(const float* v, long n, double* sum, int* bad) {
    __shared__ double part[kThreads];
    double s = 0.0;
    int b = 0;
    const long n4 = n / 4;  // v is 16-byte aligned (device allocation)
    const float4* v4 = reinterpret_cast<const float4*>(v);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n4; i += (long)gridDim.x * blockDim.x) {
        const float4 x = __ldg(v4 + i);
        if (!(x.x >= 0.f) || isinf(x.x) || !(x.y >= 0.f) || isinf(x.y) || !(x.z >= 0.f) || isinf(x.z) ||
            !(x.w >= 0.f) || isinf(x.w))
            b = 1;
        s += (double)((x.x + x.y) + (x.z + x.w));
    }
    for (long i = 4 * n4 + blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float x = v[i];
        if (!(x >= 0.f) || isinf(x)) b = 1;
        s += x;
    }
    part[threadIdx.x] = s;
    if (b) atomicOr(bad, 1);
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(sum, part[0]);
}

__global__ void k_check_positive(const float* v, long n, int* bad) {
    int b = 0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float x = v[i];
        if (!(x > 0.f) || isinf(x)) b = 1;
    }
    if (b) atomicOr(bad, 1);
}

// combined update: psi = max(psi . prod^e, eps) (e = 1/N for the geometric mean,
// 1 for the plain product); rounding can leave a factor slightly below 0
__global__ void k_apply_product(float* psi, const float* prod, long n, float e, float eps) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float p = fmaxf(prod[i], 0.f);
        const float f = e == 1.f ? p : powf(p, e);
        psi[i] = fmaxf(psi[i] * f, eps);
    }
}

// partial overlap: weights must lie in [0, 1]
__global__ void k_check_unit(const float* w, long n, int* bad) {
    int b = 0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float x = w[i];
        if (!(x >= 0.f && x <= 1.f)) b = 1;
    }
    if (b) atomicOr(bad, 1);
}

// per voxel the number of views with w > 0: sums over the covered voxels
// (stats[0] covered voxels, stats[1] sum of counts) and the minimum count
__global__ void k_overlap_stats(const float* w, int nv, long M, unsigned long long* stats, int* mincount) {
    __shared__ unsigned long long s_cov, s_sum;
    __shared__ int s_min;
    if (threadIdx.x == 0) {
        s_cov = 0;
        s_sum = 0;
        s_min = 1 << 30;
    }
    __syncthreads();
    unsigned long long cov = 0, sum = 0;
    int mn = 1 << 30;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < M; i += (long)gridDim.x * blockDim.x) {
        int n = 0;
        for (int v = 0; v < nv; ++v) n += w[(size_t)v * M + i] > 0.f;
        if (n > 0) {
            ++cov;
            sum += n;
            mn = min(mn, n);
        }
    }
    atomicAdd(&s_cov, cov);
    atomicAdd(&s_sum, sum);
    atomicMin(&s_min, mn);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(stats, s_cov);
        atomicAdd(stats + 1, s_sum);
        atomicMin(mincount, s_min);
    }
}

// w_v *= min(1, T / sum_v w_v) per voxel
__global__ void k_normalize_weights(float* w, int nv, long M, float T) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < M; i += (long)gridDim.x * blockDim.x) {
        float S = 0.f;
        for (int v = 0; v < nv; ++v) S += w[(size_t)v * M + i];
        if (S > T) {
            const float f = T / S;
            for (int v = 0; v < nv; ++v) w[(size_t)v * M + i] *= f;
        }
    }
}

__global__ void k_fill(float* p, long n, float v) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) p[i] = v;
}

inline Box box_of(const int* kd) { return Box{kd[0], kd[1], kd[2]}; }
inline int blocks_for(long n) { return (int)((n + kThreads - 1) / kThreads); }
inline int warp_blocks_for(long n) { return (int)((n * 32 + kThreads - 1) / kThreads); }  // one warp per output
inline int grid_stride_blocks(long n) {
    long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 152 * 8 ? (b < 1 ? 1 : b) : 152 * 8);
}

}  // namespace

mvd_status autocorr_all(int n_views, const float* d_psf, const long* koff, const int* kd, float* d_q, long qstride,
                        cudaStream_t st) {
    for (int w = 0; w < n_views; ++w) MVD_TRY(autocorr_kernel(d_psf + koff[w], kd + 3 * w, d_q + (size_t)w * qstride, st));
    return MVD_OK;
}

mvd_status build_compound(int n_views, const float* d_psf, const long* koff, const int* kd, int v,
                          int variant, float* d_out, const float* d_q, long qstride, cudaStream_t st) {
    const Box bv = box_of(kd + 3 * v);
    const float* Pv = d_psf + koff[v];
    k_mirror<<<blocks_for(bv.kx * bv.ky * bv.kz), kThreads, 0, st>>>(Pv, bv, d_out);
    count_launch();
    MVD_TRY(check_launch("compound mirror"));
    if (variant != MVD_PLAIN) {
        for (int w = 0; w < n_views; ++w) {
            if (w == v) continue;
            const Box bw = box_of(kd + 3 * w);
            const float* Pw = d_psf + koff[w];
            if (variant == MVD_EFFICIENT) {  // Q_w = P_w * P_w^*, computed once per view by autocorr_all
                const Box bq{2 * bw.kx - 1, 2 * bw.ky - 1, 2 * bw.kz - 1};
                k_mul_conv<<<warp_blocks_for(bv.kx * bv.ky * bv.kz), kThreads, 0, st>>>(Pv, bv, d_q + (size_t)w * qstride,
                                                                                        bq, d_out);
            } else if (variant == MVD_OPT1) {
                k_mul_conv<<<warp_blocks_for(bv.kx * bv.ky * bv.kz), kThreads, 0, st>>>(Pv, bv, Pw, bw, d_out);
            } else {
                k_mul_mirror<<<blocks_for(bv.kx * bv.ky * bv.kz), kThreads, 0, st>>>(Pv, bv, d_out);
            }
            count_launch();
            MVD_TRY(check_launch("compound product"));
        }
    }
    return MVD_OK;
}

mvd_status mirror_kernel(const float* k, const int kd[3], float* out, cudaStream_t st) {
    const Box b = box_of(kd);
    k_mirror<<<blocks_for((long)b.kx * b.ky * b.kz), kThreads, 0, st>>>(k, b, out);
    count_launch();
    return check_launch("mirror kernel");
}

mvd_status autocorr_kernel(const float* P, const int kd[3], float* Q, cudaStream_t st) {
    const Box b = box_of(kd);
    const Box q{2 * b.kx - 1, 2 * b.ky - 1, 2 * b.kz - 1};
    k_autocorr<<<warp_blocks_for((long)q.kx * q.ky * q.kz), kThreads, 0, st>>>(P, b, Q, q);
    count_launch();
    return check_launch("autocorrelation");
}

mvd_status normalize_kernel(float* d_k, int n, int* d_bad, cudaStream_t st) {
    k_normalize<<<1, 1024, 0, st>>>(d_k, n, d_bad);
    count_launch();
    return check_launch("normalise kernel");
}

mvd_status place_kernel(const int dims[3], const float* k, const int kd[3], float* vol, cudaStream_t st) {
    const long M = (long)dims[0] * dims[1] * dims[2];
    MVD_CUDA(cudaMemsetAsync(vol, 0, M * sizeof(float), st));
    const Box b = box_of(kd);
    k_place<<<blocks_for(b.kx * b.ky * b.kz), kThreads, 0, st>>>(k, b, dims[0], dims[1], dims[2], vol);
    count_launch();
    return check_launch("place kernel");
}

mvd_status view_stats(const float* views, long n, double* d_sum, int* d_bad, cudaStream_t st) {
    k_stats<<<grid_stride_blocks(n), kThreads, 0, st>>>(views, n, d_sum, d_bad);
    count_launch();
    return check_launch("view statistics");
}

mvd_status check_positive(const float* p, long n, int* d_bad, cudaStream_t st) {
    k_check_positive<<<grid_stride_blocks(n), kThreads, 0, st>>>(p, n, d_bad);
    count_launch();
    return check_launch("check estimate");
}

mvd_status apply_product(float* psi, const float* prod, long n, float e, float eps, cudaStream_t st) {
    k_apply_product<<<grid_stride_blocks(n), kThreads, 0, st>>>(psi, prod, n, e, eps);
    count_launch();
    return check_launch("apply product");
}

mvd_status weights_check(const float* w, long n, int* d_bad, cudaStream_t st) {
    k_check_unit<<<grid_stride_blocks(n), kThreads, 0, st>>>(w, n, d_bad);
    count_launch();
    return check_launch("check weights");
}

mvd_status weights_overlap(const float* w, int nv, long M, unsigned long long* d_stats, int* d_min, cudaStream_t st) {
    k_overlap_stats<<<grid_stride_blocks(M), kThreads, 0, st>>>(w, nv, M, d_stats, d_min);
    count_launch();
    return check_launch("overlap counts");
}

mvd_status weights_normalize(float* w, int nv, long M, float T, cudaStream_t st) {
    k_normalize_weights<<<grid_stride_blocks(M), kThreads, 0, st>>>(w, nv, M, T);
    count_launch();
    return check_launch("normalise weights");
}

mvd_status fill(float* p, long n, float v, cudaStream_t st) {
    k_fill<<<grid_stride_blocks(n), kThreads, 0, st>>>(p, n, v);
    count_launch();
    return check_launch("fill");
}

}  // namespace mvd
