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
// device memory is (iterations + views + 9) volumes.
// K_bar flows back through the compound kernel (Eq. 222 / 230 / 240 and its
// normalisation) to every PSF, P_bar through the PSF normalisation to the raw
// PSF values; the gradient of the flat start psi0 = mean of the views is
// spread over every view voxel. All volume work here uses the direct
// (spatial) engine in FP32.
#include <cmath>
#include <vector>

#include "common.cuh"

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
    __device__ __forceinline__ bool in(int dx, int dy, int dz) const {
        return dx >= -hx() && dx <= hx() && dy >= -hy() && dy <= hy() && dz >= -hz() && dz <= hz();
    }
    __device__ __forceinline__ int index(int dx, int dy, int dz) const {
        return (dx + hx()) + kx * ((dy + hy()) + ky * (dz + hz()));
    }
    __device__ __forceinline__ void offset(int i, int& dx, int& dy, int& dz) const {
        dx = i % kx - hx();
        dy = (i / kx) % ky - hy();
        dz = i / (kx * ky) - hz();
    }
};

// out(d) = sum_e a(e) g(d - e), d and e on box a
__global__ void k_kconv(const float* a, KBox ba, const float* g, KBox bg, float* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ba.size()) return;
    int dx, dy, dz;
    ba.offset(i, dx, dy, dz);
    float s = 0.f;
    for (int ez = max(-ba.hz(), dz - bg.hz()); ez <= min(ba.hz(), dz + bg.hz()); ++ez)
        for (int ey = max(-ba.hy(), dy - bg.hy()); ey <= min(ba.hy(), dy + bg.hy()); ++ey)
            for (int ex = max(-ba.hx(), dx - bg.hx()); ex <= min(ba.hx(), dx + bg.hx()); ++ex)
                s = fmaf(a[ba.index(ex, ey, ez)], g[bg.index(dx - ex, dy - ey, dz - ez)], s);
    out[i] = s;
}

// ab(e) += sum_d cb(d) g(d - e)   (adjoint of k_kconv in a), d and e on box a
__global__ void k_kconv_ta(const float* cb, KBox ba, const float* g, KBox bg, float* ab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ba.size()) return;
    int ex, ey, ez;
    ba.offset(i, ex, ey, ez);
    float s = 0.f;
    for (int dz = max(-ba.hz(), ez - bg.hz()); dz <= min(ba.hz(), ez + bg.hz()); ++dz)
        for (int dy = max(-ba.hy(), ey - bg.hy()); dy <= min(ba.hy(), ey + bg.hy()); ++dy)
            for (int dx = max(-ba.hx(), ex - bg.hx()); dx <= min(ba.hx(), ex + bg.hx()); ++dx)
                s = fmaf(cb[ba.index(dx, dy, dz)], g[bg.index(dx - ex, dy - ey, dz - ez)], s);
    ab[i] += s;
}

// gb(f) = sum_e cb(e + f) a(e)   (adjoint of k_kconv in g), f on box g
__global__ void k_kconv_tg(const float* cb, const float* a, KBox ba, float* gb, KBox bg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= bg.size()) return;
    int fx, fy, fz;
    bg.offset(i, fx, fy, fz);
    float s = 0.f;
    for (int ez = max(-ba.hz(), -ba.hz() - fz); ez <= min(ba.hz(), ba.hz() - fz); ++ez)
        for (int ey = max(-ba.hy(), -ba.hy() - fy); ey <= min(ba.hy(), ba.hy() - fy); ++ey)
            for (int ex = max(-ba.hx(), -ba.hx() - fx); ex <= min(ba.hx(), ba.hx() - fx); ++ex)
                s = fmaf(cb[ba.index(ex + fx, ey + fy, ez + fz)], a[ba.index(ex, ey, ez)], s);
    gb[i] = s;
}

// Q(f) = sum_g P(g) P(g - f): pb(h) += sum_f qb(f) (P(h - f) + P(h + f)), h on box p
__global__ void k_autocorr_vjp(const float* qb, KBox bq, const float* p, KBox bp, float* pb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= bp.size()) return;
    int hx, hy, hz;
    bp.offset(i, hx, hy, hz);
    float s = 0.f;
    for (int fz = -bq.hz(); fz <= bq.hz(); ++fz)
        for (int fy = -bq.hy(); fy <= bq.hy(); ++fy)
            for (int fx = -bq.hx(); fx <= bq.hx(); ++fx) {
                float pp = 0.f;
                if (bp.in(hx - fx, hy - fy, hz - fz)) pp += p[bp.index(hx - fx, hy - fy, hz - fz)];
                if (bp.in(hx + fx, hy + fy, hz + fz)) pp += p[bp.index(hx + fx, hy + fy, hz + fz)];
                s = fmaf(qb[bq.index(fx, fy, fz)], pp, s);
            }
    pb[i] += s;
}

// pb(d) += ab(-d)
__global__ void k_mirror_add(const float* ab, KBox b, float* pb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.size()) return;
    int dx, dy, dz;
    b.offset(i, dx, dy, dz);
    pb[i] += ab[b.index(-dx, -dy, -dz)];
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
    k_corr_partial<<<(unsigned)ntiles, kThreads, smem, st>>>(a, b, X, Y, Z, kd[0], kd[1], kd[2], partial);
    LAUNCH_CHECK("kernel-gradient correlation");
    const int T = kd[0] * kd[1] * kd[2];
    k_corr_reduce<<<blocks_for(T), kThreads, 0, st>>>(partial, ntiles, T, out_acc);
    LAUNCH_CHECK("kernel-gradient reduction");
    return MVD_OK;
}

}  // namespace

// compound-kernel VJP for view v: Pb[w] += d K_v / d Pn_w applied to Kb
static mvd_status compound_vjp(mvd_ctx* c, int v, const float* Kb, float* Pb, cudaStream_t st) {
    const int nv = c->nv;
    const int* dv = &c->kd[3 * v];
    const int Tv = dv[0] * dv[1] * dv[2];
    const KBox bv = kbox(dv);
    const float* Pv = c->d_psf + c->koff[v];
    long qmax = 1;
    for (int w = 0; w < nv; ++w) {
        const int* k = &c->kd[3 * w];
        qmax = std::max(qmax, (long)(2 * k[0] - 1) * (2 * k[1] - 1) * (2 * k[2] - 1));
    }
    float *A, *U, *Ab, *Cb, *Cf, *Q, *Gb;
    MVD_TRY(alloc(&A, Tv, "vjp A"));
    MVD_TRY(alloc(&U, Tv, "vjp U"));
    MVD_TRY(alloc(&Ab, Tv, "vjp Ab"));
    MVD_TRY(alloc(&Cb, (size_t)nv * Tv, "vjp Cb"));
    MVD_TRY(alloc(&Cf, (size_t)nv * Tv, "vjp C"));
    MVD_TRY(alloc(&Q, (size_t)nv * qmax, "vjp Q"));
    MVD_TRY(alloc(&Gb, qmax, "vjp Gb"));
    auto cleanup = [&]() {
        cudaFree(A);
        cudaFree(U);
        cudaFree(Ab);
        cudaFree(Cb);
        cudaFree(Cf);
        cudaFree(Q);
        cudaFree(Gb);
    };
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
                    k_kconv<<<blocks_for(Tv), kThreads, 0, st>>>(A, bv, Qw, kbox(qd), Cw);
                } else if (c->variant == MVD_OPT1) {
                    k_kconv<<<blocks_for(Tv), kThreads, 0, st>>>(A, bv, Pw, kbox(dw), Cw);
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
            k_kconv_ta<<<blocks_for(Tv), kThreads, 0, st>>>(Cbw, bv, G, bg, Ab);
            count_launch();
            k_kconv_tg<<<blocks_for(bg.kx * bg.ky * bg.kz), kThreads, 0, st>>>(Cbw, A, bv, Gb, bg);
            count_launch();
            if (c->variant == MVD_EFFICIENT) {
                k_autocorr_vjp<<<blocks_for(Tw), kThreads, 0, st>>>(Gb, bg, Pw, kbox(dw), Pbw);
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
    const cudaError_t se = cudaStreamSynchronize(st);
    if (stt == MVD_OK && se != cudaSuccess) stt = cuda_status(se, "vjp sync");
    cleanup();
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
    if (n_iter < 0) {
        set_error("mvd_unrolled_forward: n_iter < 0");
        return MVD_ERR_ARG;
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
        if (!direct_supported(&c->kd[3 * v]) || corr_smem(&c->kd[3 * v]) > kCorrMaxSmem) {
            set_error("mvd_unrolled_backward: PSF %d too large for the direct engine", v);
            return MVD_ERR_UNSUPPORTED;
        }
    }
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
        if ((stt = alloc(&work, (size_t)8 * M, "adjoint work")) != MVD_OK) break;
        if ((stt = alloc(&stage, (size_t)nv * M, "replayed estimates")) != MVD_OK) break;
        if ((stt = alloc(&partial, (size_t)ntiles * Tmax, "correlation partials")) != MVD_OK) break;
        if ((stt = alloc(&Kb, (size_t)c->ktotal, "kernel gradients")) != MVD_OK) break;
        if ((stt = alloc(&Pb, (size_t)c->ktotal, "PSF gradients")) != MVD_OK) break;
        if ((stt = alloc(&mir, (size_t)2 * Tmax, "mirrored kernels")) != MVD_OK) break;
        if ((stt = alloc(&dsum, 1, "sum")) != MVD_OK) break;
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
        for (int v = 0; v < nv && stt == MVD_OK; ++v) stt = compound_vjp(c, v, Kb + c->koff[v], Pb, st);
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
