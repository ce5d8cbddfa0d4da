// Differentiation of the unrolled sequential update (mvd_unrolled_forward /
// mvd_unrolled_backward) and the Gaussian PSF model used for PSF calibration.
//
// One view update, as a chain of elementary steps (Eq. 15 / Eq. 220; floors
// pass a gradient only where they are inactive):
//   b = psi * P ; b' = max(b, eps) ; r = phi / b' ; c = r * K ;
//   t = psi . c ; psi' = max(t, eps)
// Its adjoint for an incoming gradient g = dL/dpsi':
//   tb = g [t > eps] ; psi_bar = tb . c ; cb = tb . psi
//   rb = cb * K^* (transpose of a convolution = convolution with the mirror)
//   K_bar(d) += sum_x cb(x) r(x - d)
//   phi_bar += rb / b' ; bb = -rb . r / b' [b > eps]
//   psi_bar += bb * P^* ; P_bar(d) += sum_x bb(x) psi(x - d)
// The forward keeps the estimate at the start of every iteration (one volume
// per iteration). The backward takes the iterations in reverse; for each it
// replays the iteration's view updates from its checkpoint with the same
// engine as the forward (keeping the N estimates before the updates) and then
// recomputes each update's intermediates (b, r, c) in the adjoint step, so
// device memory is (iterations + 1) checkpoints, N replayed estimates and a
// few work volumes and kernel spectra.
// K_bar flows back through the compound kernel (Eq. 222 / 230 / 240 and its
// normalisation) to every PSF, P_bar through the PSF normalisation to the raw
// PSF values; the gradient of the flat start psi0 = mean of the views is
// spread over every view voxel. Contexts on the FFT engine run the volume
// work through the FFT passes (backward_fft); contexts on the direct engine
// use direct convolutions and a tiled correlation.
#include <cmath>
#include <vector>

#include "box_sum.cuh"
#include "common.cuh"
#include "dd.cuh"

namespace mvd {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(long n) { return (int)((n + kThreads - 1) / kThreads); }
inline int grid_stride(long n) {
    const long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

// ---------------------------------------------------------------------------
// elementwise steps
// ---------------------------------------------------------------------------

// r = phi / max(b, eps)
__global__ void k_ratio(const float* b, const float* phi, float eps, float* r, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        r[i] = phi[i] / fmaxf(b[i], eps);
}

// r = phi / max(b, eps) and r - 1 (the back-projection transforms r - 1:
// c = (r - 1) * K + 1 because K sums to 1, and r - 1 is small where psi fits)
__global__ void k_ratio_m1(const float* b, const float* phi, float eps, float* r, float* rm1, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float q = phi[i] / fmaxf(b[i], eps);
        r[i] = q;
        rm1[i] = q - 1.f;
    }
}

__global__ void k_add_one(float* x, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) x[i] += 1.f;
}

// tb = g [psi c > eps] ; gnew = tb c ; cb = tb psi
__global__ void k_adj_update(const float* psi, const float* c, const float* g, float eps, float* gnew, float* cb,
                             long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float p = psi[i], cc = c[i];
        const float tb = p * cc > eps ? g[i] : 0.f;
        gnew[i] = tb * cc;
        cb[i] = tb * p;
    }
}

// phi_bar += rb / b' ; bb = -rb r / b' [b > eps]
__global__ void k_adj_ratio(const float* rb, const float* b, const float* r, float eps, float* gphi, float* bb, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float bv = b[i], bp = fmaxf(bv, eps), rbv = rb[i];
        gphi[i] += rbv / bp;
        bb[i] = bv > eps ? -rbv * r[i] / bp : 0.f;
    }
}

__global__ void k_sum(const float* x, long n, double* out) {
    __shared__ double part[kThreads];
    double s = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) s += x[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, part[0]);
}

// x += sum / count (the flat start's share for every view voxel)
__global__ void k_add_mean(float* x, long n, const double* sum, double count) {
    const float add = (float)(*sum / count);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) x[i] += add;
}

// out(x) = in((-x) mod dims): the mirrored volume, whose spectrum is the
// conjugate (correlation with a volume = convolution with its mirror)
__global__ void k_mirror_volume(const float* in, int X, int Y, int Z, float* out) {
    const long n = (long)X * Y * Z;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int x = (int)(i % X), y = (int)((i / X) % Y), z = (int)(i / ((long)X * Y));
        const int mx = x ? X - x : 0, my = y ? Y - y : 0, mz = z ? Z - z : 0;
        out[i] = in[(long)mx + (long)X * (my + (long)Y * mz)];
    }
}

__global__ void k_add_volume(float* y, const float* x, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) y[i] += x[i];
}

// ---------------------------------------------------------------------------
// out(d) += sum_x a(x) b((x - d) mod dims) for d on a centred box: each block
// takes a 32 x 4 x 4 tile of x, stages a there and b over the tile widened by
// the box, and writes one partial sum per tap; a second kernel adds the
// partials of all tiles in FP64.
// ---------------------------------------------------------------------------
constexpr int CX = 32, CY = 4, CZ = 4;

__global__ void __launch_bounds__(kThreads) k_corr_partial(const float* a, const float* b, int X, int Y, int Z, int Kx,
                                                           int Ky, int Kz, float* partial) {
    extern __shared__ float sm[];
    const int hx = (Kx - 1) / 2, hy = (Ky - 1) / 2, hz = (Kz - 1) / 2;
    const int WX = CX + Kx - 1, WY = CY + Ky - 1, WZ = CZ + Kz - 1;
    float* sa = sm;                // CX*CY*CZ
    float* sb = sm + CX * CY * CZ;  // WX*WY*WZ, origin at tile - h (so b(x - d) sits at local x - d + h)
    const int ntx = (X + CX - 1) / CX, nty = (Y + CY - 1) / CY;
    const int tile = blockIdx.x;
    const int x0 = (tile % ntx) * CX, y0 = ((tile / ntx) % nty) * CY, z0 = (tile / (ntx * nty)) * CZ;
    for (int i = threadIdx.x; i < CX * CY * CZ; i += blockDim.x) {
        const int lx = i % CX, ly = (i / CX) % CY, lz = i / (CX * CY);
        const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
        sa[i] = (gx < X && gy < Y && gz < Z) ? a[(long)gx + (long)X * (gy + (long)Y * gz)] : 0.f;
    }
    const int nw = WX * WY * WZ;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) {
        const int lx = i % WX, ly = (i / WX) % WY, lz = i / (WX * WY);
        int gx = (x0 - hx + lx) % X;
        if (gx < 0) gx += X;
        int gy = (y0 - hy + ly) % Y;
        if (gy < 0) gy += Y;
        int gz = (z0 - hz + lz) % Z;
        if (gz < 0) gz += Z;
        sb[i] = b[(long)gx + (long)X * (gy + (long)Y * gz)];
    }
    __syncthreads();
    const int T = Kx * Ky * Kz;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const int dx = t % Kx - hx, dy = (t / Kx) % Ky - hy, dz = t / (Kx * Ky) - hz;
        float s = 0.f;
        for (int lz = 0; lz < CZ; ++lz)
            for (int ly = 0; ly < CY; ++ly) {
                const float* ar = sa + CX * (ly + CY * lz);
                const float* br = sb + (hx - dx) + WX * ((ly - dy + hy) + WY * (lz - dz + hz));
#pragma unroll 8
                for (int lx = 0; lx < CX; ++lx) s = fmaf(ar[lx], br[lx], s);
            }
        partial[(long)tile * T + t] = s;
    }
}

__global__ void k_corr_reduce(const float* partial, long ntiles, int T, float* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    double s = 0.0;
    for (long i = 0; i < ntiles; ++i) s += partial[i * T + t];
    out[t] += (float)s;
}

// ---------------------------------------------------------------------------
// kernel space (centred odd boxes): the compound kernel's vector-Jacobian
// product, K = U / sum(U), U = A . prod_w C_w, A = P_v^*
// ---------------------------------------------------------------------------
struct KBox {
    int kx, ky, kz;
    __device__ __forceinline__ int hx() const { return (kx - 1) / 2; }
    __device__ __forceinline__ int hy() const { return (ky - 1) / 2; }
    __device__ __forceinline__ int hz() const { return (kz - 1) / 2; }
    __device__ __forceinline__ int size() const { return kx * ky * kz; }
    __device__ __forceinline__ int index(int dx, int dy, int dz) const {
        return (dx + hx()) + kx * ((dy + hy()) + ky * (dz + hz()));
    }
    __device__ __forceinline__ void offset(int i, int& dx, int& dy, int& dz) const {
        dx = i % kx - hx();
        dy = (i / kx) % ky - hy();
        dz = i / (kx * ky) - hz();
    }
};

// One warp per output value (blocks of kThreads threads hold kThreads / 32
// outputs); i = the output's index, uniform within the warp.
__device__ __forceinline__ int warp_item() { return (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5); }
inline int warp_blocks(long n) { return (int)((n * 32 + kThreads - 1) / kThreads); }

// out(d) = sum_e a(e) g(d - e), d and e on box a
__global__ void k_kconv(const float* a, KBox ba, const float* g, KBox bg, float* out) {
    const int i = warp_item();
    if (i >= ba.size()) return;
    int dx, dy, dz;
    ba.offset(i, dx, dy, dz);
    const float s = warp_box_sum(max(-ba.hx(), dx - bg.hx()), min(ba.hx(), dx + bg.hx()),
                                 max(-ba.hy(), dy - bg.hy()), min(ba.hy(), dy + bg.hy()),
                                 max(-ba.hz(), dz - bg.hz()), min(ba.hz(), dz + bg.hz()),
                                 [&](int ex, int ey, int ez, float acc) {
                                     return fmaf(a[ba.index(ex, ey, ez)], g[bg.index(dx - ex, dy - ey, dz - ez)], acc);
                                 });
    if ((threadIdx.x & 31) == 0) out[i] = s;
}

// ab(e) += sum_d cb(d) g(d - e)   (adjoint of k_kconv in a), d and e on box a
__global__ void k_kconv_ta(const float* cb, KBox ba, const float* g, KBox bg, float* ab) {
    const int i = warp_item();
    if (i >= ba.size()) return;
    int ex, ey, ez;
    ba.offset(i, ex, ey, ez);
    const float s = warp_box_sum(max(-ba.hx(), ex - bg.hx()), min(ba.hx(), ex + bg.hx()),
                                 max(-ba.hy(), ey - bg.hy()), min(ba.hy(), ey + bg.hy()),
                                 max(-ba.hz(), ez - bg.hz()), min(ba.hz(), ez + bg.hz()),
                                 [&](int dx, int dy, int dz, float acc) {
                                     return fmaf(cb[ba.index(dx, dy, dz)], g[bg.index(dx - ex, dy - ey, dz - ez)], acc);
                                 });
    if ((threadIdx.x & 31) == 0) ab[i] += s;
}

// gb(f) = sum_e cb(e + f) a(e)   (adjoint of k_kconv in g), f on box g
__global__ void k_kconv_tg(const float* cb, const float* a, KBox ba, float* gb, KBox bg) {
    const int i = warp_item();
    if (i >= bg.size()) return;
    int fx, fy, fz;
    bg.offset(i, fx, fy, fz);
    const float s = warp_box_sum(max(-ba.hx(), -ba.hx() - fx), min(ba.hx(), ba.hx() - fx),
                                 max(-ba.hy(), -ba.hy() - fy), min(ba.hy(), ba.hy() - fy),
                                 max(-ba.hz(), -ba.hz() - fz), min(ba.hz(), ba.hz() - fz),
                                 [&](int ex, int ey, int ez, float acc) {
                                     return fmaf(cb[ba.index(ex + fx, ey + fy, ez + fz)], a[ba.index(ex, ey, ez)], acc);
                                 });
    if ((threadIdx.x & 31) == 0) gb[i] = s;
}

// Q(f) = sum_g P(g) P(g - f): pb(h) += sum_f qb(f) (P(h - f) + P(h + f)), h on box p,
// f on box q (the two terms as two box sums: h - f in box p, h + f in box p)
__global__ void k_autocorr_vjp(const float* qb, KBox bq, const float* p, KBox bp, float* pb) {
    const int i = warp_item();
    if (i >= bp.size()) return;
    int hx, hy, hz;
    bp.offset(i, hx, hy, hz);
    const float s1 = warp_box_sum(max(-bq.hx(), hx - bp.hx()), min(bq.hx(), hx + bp.hx()),
                                  max(-bq.hy(), hy - bp.hy()), min(bq.hy(), hy + bp.hy()),
                                  max(-bq.hz(), hz - bp.hz()), min(bq.hz(), hz + bp.hz()),
                                  [&](int fx, int fy, int fz, float acc) {
                                      return fmaf(qb[bq.index(fx, fy, fz)], p[bp.index(hx - fx, hy - fy, hz - fz)], acc);
                                  });
    const float s2 = warp_box_sum(max(-bq.hx(), -bp.hx() - hx), min(bq.hx(), bp.hx() - hx),
                                  max(-bq.hy(), -bp.hy() - hy), min(bq.hy(), bp.hy() - hy),
                                  max(-bq.hz(), -bp.hz() - hz), min(bq.hz(), bp.hz() - hz),
                                  [&](int fx, int fy, int fz, float acc) {
                                      return fmaf(qb[bq.index(fx, fy, fz)], p[bp.index(hx + fx, hy + fy, hz + fz)], acc);
                                  });
    if ((threadIdx.x & 31) == 0) pb[i] += s1 + s2;
}

// pb(d) += ab(-d)
__global__ void k_mirror_add(const float* ab, KBox b, float* pb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.size()) return;
    int dx, dy, dz;
    b.offset(i, dx, dy, dz);
    pb[i] += ab[b.index(-dx, -dy, -dz)];
}

// out(d) += vol(d mod dims) for d on the centred box b (a full correlation
// volume cropped to the kernel's support)
__global__ void k_crop_add(const float* vol, int X, int Y, int Z, KBox b, float* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.size()) return;
    int dx, dy, dz;
    b.offset(i, dx, dy, dz);
    const int x = ((dx % X) + X) % X, y = ((dy % Y) + Y) % Y, z = ((dz % Z) + Z) % Z;
    out[i] += vol[(long)x + (long)X * (y + (long)Y * z)];
}

constexpr int kMaxViews = 32;
struct FactorPtrs {
    const float* c[kMaxViews];  // C_w on box v (nullptr for w == v or no factor)
};

// One block: U = A . prod C ; s = sum U ; K = U / s ; kk = sum(Kb . K) ;
// Ub = (Kb - kk) / s ; Ab = Ub . prod C ; Cb_w = Ub . A . prod_{u != w} C_u
__global__ void k_compound_back(const float* A, FactorPtrs C, int nv, int T, const float* Kb, float* U, float* Ab,
                                float* Cb /* nv * T */) {
    __shared__ double part[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < T; i += blockDim.x) {
        float u = A[i];
        for (int w = 0; w < nv; ++w)
            if (C.c[w]) u *= C.c[w][i];
        U[i] = u;
        s += u;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    const double su = part[0];
    __syncthreads();
    double k = 0.0;
    for (int i = threadIdx.x; i < T; i += blockDim.x) k += (double)Kb[i] * (U[i] / su);
    part[threadIdx.x] = k;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    const double kk = part[0];
    for (int i = threadIdx.x; i < T; i += blockDim.x) {
        const float ub = (float)((Kb[i] - kk) / su);
        float prod = 1.f;
        for (int w = 0; w < nv; ++w)
            if (C.c[w]) prod *= C.c[w][i];
        Ab[i] = ub * prod;
        for (int w = 0; w < nv; ++w) {
            if (!C.c[w]) continue;
            float q = ub * A[i];
            for (int u = 0; u < nv; ++u)
                if (C.c[u] && u != w) q *= C.c[u][i];
            Cb[(long)w * T + i] = q;
        }
    }
}

__global__ void k_add(float* y, const float* x, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}

inline KBox kbox(const int* kd) { return KBox{kd[0], kd[1], kd[2]}; }

#define LAUNCH_CHECK(name)          \
    do {                            \
        count_launch();             \
        MVD_TRY(check_launch(name)); \
    } while (0)

template <typename T>
mvd_status alloc(T** p, size_t n, const char* what) {
    cudaError_t e = cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return cuda_status(e, what);
    }
    return MVD_OK;
}

constexpr size_t kCorrMaxSmem = 227 * 1024;
inline size_t corr_smem(const int kd[3]) {
    return sizeof(float) *
           ((size_t)CX * CY * CZ + (size_t)(CX + kd[0] - 1) * (CY + kd[1] - 1) * (CZ + kd[2] - 1));
}

mvd_status copy_volume(float* dst, const float* src, long n, cudaStream_t st) {
    const cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? MVD_OK : cuda_status(e, "volume copy");
}

mvd_status corr_to_box(const float* a, const float* b, const int dims[3], const int kd[3], float* out_acc,
                       float* partial, cudaStream_t st) {
    const int X = dims[0], Y = dims[1], Z = dims[2];
    const long ntiles = (long)((X + CX - 1) / CX) * ((Y + CY - 1) / CY) * ((Z + CZ - 1) / CZ);
    const size_t smem = corr_smem(kd);
    if (smem > kCorrMaxSmem) {
        set_error("kernel-gradient correlation: box %dx%dx%d needs %zu bytes of shared memory", kd[0], kd[1], kd[2],
                  smem);
        return MVD_ERR_UNSUPPORTED;
    }
    MVD_CUDA(cudaFuncSetAttribute(k_corr_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    prof_begin(KC_KERNEL_GRAD, st);
    k_corr_partial<<<(unsigned)ntiles, kThreads, smem, st>>>(a, b, X, Y, Z, kd[0], kd[1], kd[2], partial);
    const int T = kd[0] * kd[1] * kd[2];
    k_corr_reduce<<<blocks_for(T), kThreads, 0, st>>>(partial, ntiles, T, out_acc);
    prof_end(KC_KERNEL_GRAD, st);
    count_launch(2);
    MVD_TRY(check_launch("kernel-gradient correlation"));
    return MVD_OK;
}

}  // namespace

// scratch of the compound-kernel VJP, sized for the largest box
struct VjpScratch {
    float *A = nullptr, *U = nullptr, *Ab = nullptr, *Cb = nullptr, *Cf = nullptr, *Q = nullptr, *Gb = nullptr;
    long qmax = 1;
    mvd_status alloc_for(const mvd_ctx* c) {
        long tmax = 1;
        for (int w = 0; w < c->nv; ++w) {
            const int* k = &c->kd[3 * w];
            tmax = std::max(tmax, (long)k[0] * k[1] * k[2]);
            qmax = std::max(qmax, (long)(2 * k[0] - 1) * (2 * k[1] - 1) * (2 * k[2] - 1));
        }
        MVD_TRY(alloc(&A, tmax, "vjp A"));
        MVD_TRY(alloc(&U, tmax, "vjp U"));
        MVD_TRY(alloc(&Ab, tmax, "vjp Ab"));
        MVD_TRY(alloc(&Cb, (size_t)c->nv * tmax, "vjp Cb"));
        MVD_TRY(alloc(&Cf, (size_t)c->nv * tmax, "vjp C"));
        MVD_TRY(alloc(&Q, (size_t)c->nv * qmax, "vjp Q"));
        return alloc(&Gb, qmax, "vjp Gb");
    }
    void release() {
        for (float* p : {A, U, Ab, Cb, Cf, Q, Gb})
            if (p) cudaFree(p);
        A = U = Ab = Cb = Cf = Q = Gb = nullptr;
    }
};

// compound-kernel VJP for view v: Pb[w] += d K_v / d Pn_w applied to Kb
static mvd_status compound_vjp(mvd_ctx* c, int v, const float* Kb, float* Pb, const VjpScratch& sc, cudaStream_t st) {
    const int nv = c->nv;
    const int* dv = &c->kd[3 * v];
    const int Tv = dv[0] * dv[1] * dv[2];
    const KBox bv = kbox(dv);
    const float* Pv = c->d_psf + c->koff[v];
    const long qmax = sc.qmax;
    float *A = sc.A, *U = sc.U, *Ab = sc.Ab, *Cb = sc.Cb, *Cf = sc.Cf, *Q = sc.Q, *Gb = sc.Gb;
    mvd_status stt = MVD_OK;
    do {
        if ((stt = mirror_kernel(Pv, dv, A, st)) != MVD_OK) break;
        FactorPtrs fp{};
        if (c->variant != MVD_PLAIN) {
            for (int w = 0; w < nv && stt == MVD_OK; ++w) {
                if (w == v) continue;
                const int* dw = &c->kd[3 * w];
                const float* Pw = c->d_psf + c->koff[w];
                float* Cw = Cf + (size_t)w * Tv;
                if (c->variant == MVD_EFFICIENT) {
                    float* Qw = Q + (size_t)w * qmax;
                    const int qd[3] = {2 * dw[0] - 1, 2 * dw[1] - 1, 2 * dw[2] - 1};
                    if ((stt = autocorr_kernel(Pw, dw, Qw, st)) != MVD_OK) break;
                    k_kconv<<<warp_blocks(Tv), kThreads, 0, st>>>(A, bv, Qw, kbox(qd), Cw);
                } else if (c->variant == MVD_OPT1) {
                    k_kconv<<<warp_blocks(Tv), kThreads, 0, st>>>(A, bv, Pw, kbox(dw), Cw);
                } else {
                    cudaError_t e = cudaMemcpyAsync(Cw, A, sizeof(float) * Tv, cudaMemcpyDeviceToDevice, st);
                    if (e != cudaSuccess) {
                        stt = cuda_status(e, "vjp factor copy");
                        break;
                    }
                }
                if (c->variant != MVD_OPT2) count_launch();
                if ((stt = check_launch("vjp factor")) != MVD_OK) break;
                fp.c[w] = Cw;
            }
            if (stt != MVD_OK) break;
        }
        k_compound_back<<<1, 1024, 0, st>>>(A, fp, nv, Tv, Kb, U, Ab, Cb);
        count_launch();
        if ((stt = check_launch("vjp compound")) != MVD_OK) break;
        for (int w = 0; w < nv && c->variant != MVD_PLAIN; ++w) {
            if (w == v) continue;
            const int* dw = &c->kd[3 * w];
            const int Tw = dw[0] * dw[1] * dw[2];
            const float* Pw = c->d_psf + c->koff[w];
            float* Pbw = Pb + c->koff[w];
            const float* Cbw = Cb + (size_t)w * Tv;
            if (c->variant == MVD_OPT2) {  // C_w = A
                k_add<<<blocks_for(Tv), kThreads, 0, st>>>(Ab, Cbw, Tv);
                count_launch();
                continue;
            }
            const int qd[3] = {2 * dw[0] - 1, 2 * dw[1] - 1, 2 * dw[2] - 1};
            const float* G = c->variant == MVD_EFFICIENT ? Q + (size_t)w * qmax : Pw;
            const KBox bg = c->variant == MVD_EFFICIENT ? kbox(qd) : kbox(dw);
            k_kconv_ta<<<warp_blocks(Tv), kThreads, 0, st>>>(Cbw, bv, G, bg, Ab);
            count_launch();
            k_kconv_tg<<<warp_blocks(bg.kx * bg.ky * bg.kz), kThreads, 0, st>>>(Cbw, A, bv, Gb, bg);
            count_launch();
            if (c->variant == MVD_EFFICIENT) {
                k_autocorr_vjp<<<warp_blocks(Tw), kThreads, 0, st>>>(Gb, bg, Pw, kbox(dw), Pbw);
            } else {
                k_add<<<blocks_for(Tw), kThreads, 0, st>>>(Pbw, Gb, Tw);
            }
            count_launch();
            if ((stt = check_launch("vjp chain")) != MVD_OK) break;
        }
        if (stt != MVD_OK) break;
        k_mirror_add<<<blocks_for(Tv), kThreads, 0, st>>>(Ab, bv, Pb + c->koff[v]);
        count_launch();
        stt = check_launch("vjp mirror");
    } while (false);
    return stt;
}

// Circular convolutions through the FP32 FFT engine: spectra of kernels or
// volumes (full 3D transform, scaled by 1/M) and products with them.
struct FftConv {
    mvd_ctx* c;
    float2* S;  // work spectrum
    cudaStream_t st;
    mvd_status spectrum(const float* vol, float2* spec) const {
        MVD_TRY(fft_forward_real(c->geom, vol, spec, st));
        MVD_TRY(fft_y(c->geom, spec, 0, st));
        return fft_z_forward_scaled(c->geom, spec, (float)(1.0 / (double)c->M), st);
    }
    mvd_status conv(const float* in, const float2* spec, float* out) const {
        MVD_TRY(fft_forward_real(c->geom, in, S, st));
        MVD_TRY(fft_y(c->geom, S, 0, st));
        MVD_TRY(fft_z_mul(c->geom, S, spec, st));
        MVD_TRY(fft_y(c->geom, S, 1, st));
        return fft_inverse_real(c->geom, S, out, st);
    }
};

// The reverse pass on the FFT engine (contexts whose path is FFT). Per update:
// b = psi * P, r, c = (r - 1) * K + 1 recomputed; r_bar = c_bar * K^*,
// psi_bar += b_bar * P^* (mirrored kernels' spectra); K_bar and P_bar are the
// full correlations c_bar * mirror(r) and b_bar * mirror(psi), cropped to the
// kernel box. FFT rounding is absolute (it scales with the whole volume's
// norm), while the view gradient r_bar / b is largest where b is dim, so when
// the forward ran in double-float, b, r_bar and the b_bar * P^* term are
// double-float convolutions too; c and the cropped correlations (sums over
// the whole volume) stay FP32.
static mvd_status backward_fft(mvd_ctx* c, const float* grad_psi, float* const* grad_views, float* Kb, float* Pb,
                               double* dsum) {
    const long M = c->M;
    const int nv = c->nv;
    cudaStream_t st = c->stream;
    const FftGeom& g = c->geom;
    const size_t ns = (size_t)g.Xh * g.YZ;
    float *work = nullptr, *stage = nullptr, *kt = nullptr;
    float2 *spec = nullptr, *specA = nullptr, *S = nullptr;
    cdd* specDD = nullptr;
    int Tmax = 1;
    for (int v = 0; v < nv; ++v) Tmax = std::max(Tmax, c->kd[3 * v] * c->kd[3 * v + 1] * c->kd[3 * v + 2]);
    mvd_status stt = MVD_OK;
    do {
        if ((stt = alloc(&work, (size_t)10 * M, "adjoint work")) != MVD_OK) break;
        if ((stt = alloc(&stage, (size_t)nv * M, "replayed estimates")) != MVD_OK) break;
        if ((stt = alloc(&kt, (size_t)Tmax, "mirrored kernel")) != MVD_OK) break;
        if ((stt = alloc(&spec, (size_t)4 * nv * ns, "kernel spectra")) != MVD_OK) break;
        if ((stt = alloc(&specA, ns, "volume spectrum")) != MVD_OK) break;
        if ((stt = alloc(&S, ns, "work spectrum")) != MVD_OK) break;
        float *B = work, *R = work + M, *C = work + 2 * M, *CB = work + 3 * M, *RB = work + 4 * M,
              *BB = work + 5 * M, *G = work + 6 * M, *G2 = work + 7 * M, *MIR = work + 8 * M, *TMP = work + 9 * M;
        const FftConv F{c, S, st};
        const bool dd = c->precise && c->d_KP2 && c->d_S2 && dd_fast_x(g);
        // double-float spectra of the mirrored kernels: 2v P^*, 2v+1 K^*
        if (dd && (stt = alloc(reinterpret_cast<float4**>(&specDD), (size_t)2 * nv * ns, "mirrored spectra")) != MVD_OK)
            break;
        for (int v = 0; v < nv && dd && stt == MVD_OK; ++v) {
            const int* kd = &c->kd[3 * v];
            for (int j = 0; j < 2 && stt == MVD_OK; ++j) {
                cdd* dst = specDD + (size_t)(2 * v + j) * ns;
                if ((stt = mirror_kernel((j == 0 ? c->d_psf : c->d_comp) + c->koff[v], kd, kt, st)) != MVD_OK) break;
                if ((stt = place_kernel(c->dims, kt, kd, TMP, st)) != MVD_OK) break;
                if ((stt = dd_forward_real(g, TMP, dst, st)) != MVD_OK) break;
                if ((stt = dd_y(g, dst, 0, st)) != MVD_OK) break;
                stt = dd_z_forward_scaled(g, dst, 1.0 / (double)M, st);
            }
        }
        if (stt != MVD_OK) break;
        auto dd_conv = [&](const float* in, const cdd* K2, float* out) -> mvd_status {
            MVD_TRY(dd_forward_real(g, in, c->d_S2, st));
            MVD_TRY(dd_y(g, c->d_S2, 0, st));
            MVD_TRY(dd_z_mul(g, c->d_S2, K2, st));
            MVD_TRY(dd_y(g, c->d_S2, 1, st));
            return dd_x_inverse_real(g, c->d_S2, out, st);
        };
        // spectra per view: 4v P, 4v+1 K, 4v+2 P^*, 4v+3 K^*
        for (int v = 0; v < nv && stt == MVD_OK; ++v) {
            const int* kd = &c->kd[3 * v];
            const float* ks[2] = {c->d_psf + c->koff[v], c->d_comp + c->koff[v]};
            for (int j = 0; j < 4 && stt == MVD_OK; ++j) {
                const float* k = ks[j & 1];
                if (j >= 2) {
                    if ((stt = mirror_kernel(k, kd, kt, st)) != MVD_OK) break;
                    k = kt;
                }
                if ((stt = place_kernel(c->dims, k, kd, TMP, st)) != MVD_OK) break;
                stt = F.spectrum(TMP, spec + (size_t)(4 * v + j) * ns);
            }
        }
        if (stt != MVD_OK) break;
        cudaMemsetAsync(Kb, 0, sizeof(float) * c->ktotal, st);
        cudaMemsetAsync(Pb, 0, sizeof(float) * c->ktotal, st);
        for (int v = 0; v < nv; ++v) cudaMemsetAsync(grad_views[v], 0, sizeof(float) * M, st);
        if ((stt = copy_volume(G, grad_psi, M, st)) != MVD_OK) break;
        for (long u = (long)c->ckpt_iters * nv - 1; u >= 0 && stt == MVD_OK; --u) {
            const int v = (int)(u % nv);
            if (v == nv - 1) {  // replay iteration u / nv from its checkpoint with the forward's engine
                stt = copy_volume(c->d_psi, c->d_ckpt + (size_t)(u / nv) * M, M, st);
                for (int w = 0; w < nv && stt == MVD_OK; ++w) {
                    stt = copy_volume(stage + (size_t)w * M, c->d_psi, M, st);
                    if (stt == MVD_OK && w < nv - 1) stt = one_update(c, w);
                }
                if (stt != MVD_OK) break;
            }
            const KBox box = kbox(&c->kd[3 * v]);
            const float* psi = stage + (size_t)v * M;
            const float* phi = c->d_views + (size_t)v * M;
            const float2* sP = spec + (size_t)(4 * v) * ns;
            const float2* sK = sP + ns;
            const float2* sPm = sP + 2 * ns;
            const float2* sKm = sP + 3 * ns;
            // forward intermediates
            if (dd) {
                const cdd* Kp2 = reinterpret_cast<const cdd*>(reinterpret_cast<const float4*>(c->d_KP2) + ns * (2 * v));
                if ((stt = dd_conv(psi, Kp2, B)) != MVD_OK) break;
            } else if ((stt = F.conv(psi, sP, B)) != MVD_OK) {
                break;
            }
            k_ratio_m1<<<grid_stride(M), kThreads, 0, st>>>(B, phi, c->eps, R, TMP, M);
            count_launch();
            if ((stt = F.conv(TMP, sK, C)) != MVD_OK) break;
            k_add_one<<<grid_stride(M), kThreads, 0, st>>>(C, M);
            count_launch();
            // adjoint
            k_adj_update<<<grid_stride(M), kThreads, 0, st>>>(psi, C, G, c->eps, G2, CB, M);
            count_launch();
            if ((stt = dd ? dd_conv(CB, specDD + (size_t)(2 * v + 1) * ns, RB) : F.conv(CB, sKm, RB)) != MVD_OK) break;
            k_mirror_volume<<<grid_stride(M), kThreads, 0, st>>>(R, c->dims[0], c->dims[1], c->dims[2], MIR);
            count_launch();
            if ((stt = F.spectrum(MIR, specA)) != MVD_OK) break;
            if ((stt = F.conv(CB, specA, TMP)) != MVD_OK) break;
            k_crop_add<<<blocks_for(box.kx * box.ky * box.kz), kThreads, 0, st>>>(
                TMP, c->dims[0], c->dims[1], c->dims[2], box, Kb + c->koff[v]);
            count_launch();
            k_adj_ratio<<<grid_stride(M), kThreads, 0, st>>>(RB, B, R, c->eps, grad_views[v], BB, M);
            count_launch();
            if ((stt = dd ? dd_conv(BB, specDD + (size_t)(2 * v) * ns, TMP) : F.conv(BB, sPm, TMP)) != MVD_OK) break;
            k_add_volume<<<grid_stride(M), kThreads, 0, st>>>(G2, TMP, M);
            count_launch();
            k_mirror_volume<<<grid_stride(M), kThreads, 0, st>>>(psi, c->dims[0], c->dims[1], c->dims[2], MIR);
            count_launch();
            if ((stt = F.spectrum(MIR, specA)) != MVD_OK) break;
            if ((stt = F.conv(BB, specA, TMP)) != MVD_OK) break;
            k_crop_add<<<blocks_for(box.kx * box.ky * box.kz), kThreads, 0, st>>>(
                TMP, c->dims[0], c->dims[1], c->dims[2], box, Pb + c->koff[v]);
            count_launch();
            if ((stt = check_launch("adjoint step")) != MVD_OK) break;
            std::swap(G, G2);
        }
        if (stt != MVD_OK) break;
        if (c->ckpt_flat) {  // psi0 = mean of all views
            cudaMemsetAsync(dsum, 0, sizeof(double), st);
            k_sum<<<grid_stride(M), kThreads, 0, st>>>(G, M, dsum);
            count_launch();
            for (int v = 0; v < nv; ++v) {
                k_add_mean<<<grid_stride(M), kThreads, 0, st>>>(grad_views[v], M, dsum, (double)M * nv);
                count_launch();
            }
            stt = check_launch("flat start");
        }
    } while (false);
    const cudaError_t se = cudaStreamSynchronize(st);
    if (stt == MVD_OK && se != cudaSuccess) stt = cuda_status(se, "adjoint sync");
    cudaFree(work);
    cudaFree(stage);
    cudaFree(kt);
    cudaFree(spec);
    cudaFree(specA);
    cudaFree(S);
    cudaFree(specDD);
    return stt;
}

}  // namespace mvd

using namespace mvd;

extern "C" {

mvd_status mvd_unrolled_forward(mvd_ctx* c, int n_iter) {
    clear_error();
    if (!c) {
        set_error("mvd_unrolled_forward: NULL context");
        return MVD_ERR_ARG;
    }
    if (c->state < 2) {
        set_error("mvd_unrolled_forward: kernels not precomputed");
        return MVD_ERR_STATE;
    }
    if (!c->views_ok) {
        set_error("mvd_unrolled_forward: the last mvd_set_views failed; load valid views first");
        return MVD_ERR_STATE;
    }
    if (n_iter < 0) {
        set_error("mvd_unrolled_forward: n_iter < 0");
        return MVD_ERR_ARG;
    }
    if (c->d_w || c->lambda != 0.f || c->boundary != MVD_BOUNDARY_PERIODIC) {
        set_error("mvd_unrolled_forward: not defined for a context with view weights, regularisation or a zero "
                  "boundary");
        return MVD_ERR_UNSUPPORTED;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    if (c->d_ckpt) cudaFree(c->d_ckpt);
    c->d_ckpt = nullptr;
    c->ckpt_iters = -1;
    mvd_status st = alloc(&c->d_ckpt, (size_t)(n_iter + 1) * c->M, "checkpoints");
    // the run starts from the flat estimate (whose value depends on the views)
    if (st == MVD_OK) st = mvd_set_estimate(c, nullptr, 0);
    for (int k = 0; k <= n_iter && st == MVD_OK; ++k) {
        cudaError_t e = cudaMemcpyAsync(c->d_ckpt + (size_t)k * c->M, c->d_psi, sizeof(float) * c->M,
                                        cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) {
            st = cuda_status(e, "checkpoint copy");
            break;
        }
        for (int v = 0; v < c->nv && k < n_iter && st == MVD_OK; ++v) st = one_update(c, v);
    }
    if (st == MVD_OK) {
        c->ckpt_iters = n_iter;
        c->ckpt_flat = 1;
    }
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    return st;
}

mvd_status mvd_unrolled_backward(mvd_ctx* c, const float* grad_psi, float* const* grad_views,
                                 float* const* grad_psfs) {
    clear_error();
    if (!c || !grad_psi || !grad_views || !grad_psfs) {
        set_error("mvd_unrolled_backward: NULL argument");
        return MVD_ERR_ARG;
    }
    if (c->ckpt_iters < 0 || !c->d_ckpt) {
        set_error("mvd_unrolled_backward: no unrolled forward run to differentiate");
        return MVD_ERR_STATE;
    }
    if (c->nv > kMaxViews) {
        set_error("mvd_unrolled_backward: at most %d views", kMaxViews);
        return MVD_ERR_UNSUPPORTED;
    }
    for (int v = 0; v < c->nv; ++v) {
        if (!grad_views[v] || !grad_psfs[v]) {
            set_error("mvd_unrolled_backward: gradient buffer %d is NULL", v);
            return MVD_ERR_ARG;
        }
        if (c->path != MVD_PATH_FFT &&
            (!direct_supported(&c->kd[3 * v]) || corr_smem(&c->kd[3 * v]) > kCorrMaxSmem)) {
            set_error("mvd_unrolled_backward: PSF %d too large for the direct engine", v);
            return MVD_ERR_UNSUPPORTED;
        }
    }
    const bool use_fft = c->path == MVD_PATH_FFT;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    const long M = c->M;
    const int nv = c->nv;
    cudaStream_t st = c->stream;
    long ntiles = (long)((c->dims[0] + CX - 1) / CX) * ((c->dims[1] + CY - 1) / CY) * ((c->dims[2] + CZ - 1) / CZ);
    int Tmax = 1;
    for (int v = 0; v < nv; ++v) Tmax = std::max(Tmax, c->kd[3 * v] * c->kd[3 * v + 1] * c->kd[3 * v + 2]);
    float *work = nullptr, *stage = nullptr, *partial = nullptr, *Kb = nullptr, *Pb = nullptr, *mir = nullptr;
    double* dsum = nullptr;
    mvd_status stt = MVD_OK;
    do {
        if ((stt = alloc(&Kb, (size_t)c->ktotal, "kernel gradients")) != MVD_OK) break;
        if ((stt = alloc(&Pb, (size_t)c->ktotal, "PSF gradients")) != MVD_OK) break;
        if ((stt = alloc(&dsum, 1, "sum")) != MVD_OK) break;
        if (use_fft) {
            if ((stt = backward_fft(c, grad_psi, grad_views, Kb, Pb, dsum)) != MVD_OK) break;
        } else {
            if ((stt = alloc(&work, (size_t)8 * M, "adjoint work")) != MVD_OK) break;
            if ((stt = alloc(&stage, (size_t)nv * M, "replayed estimates")) != MVD_OK) break;
            if ((stt = alloc(&partial, (size_t)ntiles * Tmax, "correlation partials")) != MVD_OK) break;
            if ((stt = alloc(&mir, (size_t)2 * Tmax, "mirrored kernels")) != MVD_OK) break;
            float *B = work, *R = work + M, *C = work + 2 * M, *CB = work + 3 * M, *RB = work + 4 * M,
                  *BB = work + 5 * M, *G = work + 6 * M, *G2 = work + 7 * M;
            cudaMemsetAsync(Kb, 0, sizeof(float) * c->ktotal, st);
            cudaMemsetAsync(Pb, 0, sizeof(float) * c->ktotal, st);
            for (int v = 0; v < nv; ++v) cudaMemsetAsync(grad_views[v], 0, sizeof(float) * M, st);
            cudaMemcpyAsync(G, grad_psi, sizeof(float) * M, cudaMemcpyDeviceToDevice, st);
            for (long u = (long)c->ckpt_iters * nv - 1; u >= 0 && stt == MVD_OK; --u) {
                const int v = (int)(u % nv);
                if (v == nv - 1) {  // replay iteration u / nv from its checkpoint
                    stt = copy_volume(c->d_psi, c->d_ckpt + (size_t)(u / nv) * M, M, st);
                    for (int w = 0; w < nv && stt == MVD_OK; ++w) {
                        stt = copy_volume(stage + (size_t)w * M, c->d_psi, M, st);
                        if (stt == MVD_OK && w < nv - 1) stt = one_update(c, w);
                    }
                    if (stt != MVD_OK) break;
                }
                const int* kd = &c->kd[3 * v];
                const float* psi = stage + (size_t)v * M;
                const float* phi = c->d_views + (size_t)v * M;
                const float* P = c->d_psf + c->koff[v];
                const float* K = c->d_comp + c->koff[v];
                float* Ks = mir;
                float* Ps = mir + Tmax;
                if ((stt = mirror_kernel(K, kd, Ks, st)) != MVD_OK) break;
                if ((stt = mirror_kernel(P, kd, Ps, st)) != MVD_OK) break;
                // forward intermediates
                if ((stt = direct_conv(c->dims, psi, P, kd, B, st)) != MVD_OK) break;
                k_ratio<<<grid_stride(M), kThreads, 0, st>>>(B, phi, c->eps, R, M);
                count_launch();
                if ((stt = direct_conv(c->dims, R, K, kd, C, st)) != MVD_OK) break;
                // adjoint
                k_adj_update<<<grid_stride(M), kThreads, 0, st>>>(psi, C, G, c->eps, G2, CB, M);
                count_launch();
                if ((stt = direct_conv(c->dims, CB, Ks, kd, RB, st)) != MVD_OK) break;
                if ((stt = corr_to_box(CB, R, c->dims, kd, Kb + c->koff[v], partial, st)) != MVD_OK) break;
                k_adj_ratio<<<grid_stride(M), kThreads, 0, st>>>(RB, B, R, c->eps, grad_views[v], BB, M);
                count_launch();
                if ((stt = direct_conv_add(c->dims, BB, Ps, kd, G2, st)) != MVD_OK) break;
                if ((stt = corr_to_box(BB, psi, c->dims, kd, Pb + c->koff[v], partial, st)) != MVD_OK) break;
                if ((stt = check_launch("adjoint step")) != MVD_OK) break;
                std::swap(G, G2);
            }
            if (stt != MVD_OK) break;
            if (c->ckpt_flat) {  // psi0 = mean of all views
                cudaMemsetAsync(dsum, 0, sizeof(double), st);
                k_sum<<<grid_stride(M), kThreads, 0, st>>>(G, M, dsum);
                count_launch();
                for (int v = 0; v < nv; ++v) {
                    k_add_mean<<<grid_stride(M), kThreads, 0, st>>>(grad_views[v], M, dsum, (double)M * nv);
                    count_launch();
                }
                if ((stt = check_launch("flat start")) != MVD_OK) break;
            }
        }  // direct engine
        VjpScratch sc;
        stt = sc.alloc_for(c);
        for (int v = 0; v < nv && stt == MVD_OK; ++v) stt = compound_vjp(c, v, Kb + c->koff[v], Pb, sc, st);
        cudaStreamSynchronize(st);
        sc.release();
        if (stt != MVD_OK) break;
        // PSF normalisation Pn = p / sum(p), on the host in FP64
        std::vector<float> pb(c->ktotal), pn(c->ktotal);
        cudaError_t e = cudaMemcpyAsync(pb.data(), Pb, sizeof(float) * c->ktotal, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pn.data(), c->d_psf, sizeof(float) * c->ktotal, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            stt = cuda_status(e, "PSF gradients");
            break;
        }
        for (int v = 0; v < nv; ++v) {
            const long T = (long)c->kd[3 * v] * c->kd[3 * v + 1] * c->kd[3 * v + 2];
            double dot = 0.0;
            for (long i = 0; i < T; ++i) dot += (double)pb[c->koff[v] + i] * pn[c->koff[v] + i];
            for (long i = 0; i < T; ++i) grad_psfs[v][i] = (float)(((double)pb[c->koff[v] + i] - dot) / c->psf_sum[v]);
        }
    } while (false);
    if (c->ckpt_iters > 0)  // the replays moved the estimate: restore psi_K
        cudaMemcpyAsync(c->d_psi, c->d_ckpt + (size_t)c->ckpt_iters * M, sizeof(float) * M, cudaMemcpyDeviceToDevice,
                        st);
    cudaStreamSynchronize(st);
    cudaFree(work);
    cudaFree(stage);
    cudaFree(partial);
    cudaFree(Kb);
    cudaFree(Pb);
    cudaFree(mir);
    cudaFree(dsum);
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    return stt;
}

// ---------------------------------------------------------------------------
// Gaussian PSF model (host, FP64): exp(-d^T S^-1 d / 2) on a centred box,
// S = R diag(v) R^T with v = sigma_xy^2 on the lateral axes and sigma_ax^2 on
// `axis`, R a rotation about y by angle_deg, normalised to sum 1.
// ---------------------------------------------------------------------------
namespace {
struct GaussTerms {
    std::vector<double> g, dq_dxy, dq_dax;
    double sum;
};

GaussTerms gauss_terms(double sxy, double sax, double angle_deg, int axis, const int box[3]) {
    const double t = angle_deg * M_PI / 180.0, cs = std::cos(t), sn = std::sin(t);
    const int hx = (box[0] - 1) / 2, hy = (box[1] - 1) / 2, hz = (box[2] - 1) / 2;
    const long T = (long)box[0] * box[1] * box[2];
    GaussTerms r;
    r.g.resize(T);
    r.dq_dxy.resize(T);
    r.dq_dax.resize(T);
    r.sum = 0.0;
    for (long i = 0; i < T; ++i) {
        const double dx = (double)(i % box[0] - hx), dy = (double)((i / box[0]) % box[1] - hy),
                     dz = (double)(i / ((long)box[0] * box[1]) - hz);
        // body-frame coordinates R^T d (R rotates x towards z about y)
        const double u[3] = {cs * dx - sn * dz, dy, sn * dx + cs * dz};
        double lat = 0.0, ax = 0.0;
        for (int a = 0; a < 3; ++a) (a == axis ? ax : lat) += u[a] * u[a];
        const double q = lat / (sxy * sxy) + ax / (sax * sax);
        r.g[i] = std::exp(-0.5 * q);
        r.dq_dxy[i] = -2.0 * lat / (sxy * sxy * sxy);
        r.dq_dax[i] = -2.0 * ax / (sax * sax * sax);
        r.sum += r.g[i];
    }
    return r;
}
}  // namespace

mvd_status mvd_gaussian_psf(double sigma_xy, double sigma_ax, double angle_deg, int axis, const int box[3],
                            float* out) {
    clear_error();
    if (!box || !out || !(sigma_xy > 0) || !(sigma_ax > 0) || axis < 0 || axis > 2) {
        set_error("mvd_gaussian_psf: bad arguments");
        return MVD_ERR_ARG;
    }
    for (int a = 0; a < 3; ++a)
        if (box[a] < 1 || box[a] % 2 == 0) {
            set_error("mvd_gaussian_psf: box sizes must be odd");
            return MVD_ERR_SHAPE;
        }
    GaussTerms g = gauss_terms(sigma_xy, sigma_ax, angle_deg, axis, box);
    for (size_t i = 0; i < g.g.size(); ++i) out[i] = (float)(g.g[i] / g.sum);
    return MVD_OK;
}

mvd_status mvd_gaussian_psf_vjp(double sigma_xy, double sigma_ax, double angle_deg, int axis, const int box[3],
                                const float* grad_psf, double grad_sigma[2]) {
    clear_error();
    if (!box || !grad_psf || !grad_sigma || !(sigma_xy > 0) || !(sigma_ax > 0) || axis < 0 || axis > 2) {
        set_error("mvd_gaussian_psf_vjp: bad arguments");
        return MVD_ERR_ARG;
    }
    GaussTerms g = gauss_terms(sigma_xy, sigma_ax, angle_deg, axis, box);
    // P = g / G ; dP/ds = (dg/ds - P sum(dg/ds)) / G ; dg/ds = -g dq/ds / 2
    double sxy = 0.0, sax = 0.0, pxy = 0.0, pax = 0.0;
    for (size_t i = 0; i < g.g.size(); ++i) {
        const double dgx = -0.5 * g.g[i] * g.dq_dxy[i], dga = -0.5 * g.g[i] * g.dq_dax[i];
        sxy += dgx;
        sax += dga;
        pxy += grad_psf[i] * dgx;
        pax += grad_psf[i] * dga;
    }
    double pp = 0.0;
    for (size_t i = 0; i < g.g.size(); ++i) pp += grad_psf[i] * (g.g[i] / g.sum);
    grad_sigma[0] = (pxy - pp * sxy) / g.sum;
    grad_sigma[1] = (pax - pp * sax) / g.sum;
    return MVD_OK;
}

}  // extern "C"
