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
#include "fft.cuh"

namespace mvd {

namespace {

constexpr int kThreads = 256;

inline int div_up(long a, long b) { return (int)((a + b - 1) / b); }

// rows (2P per tile) and smem line stride for the x pass
struct XTile {
    int P;
    int ls;
};
inline XTile x_tile(int X) {
    int P = (int)(16384 / (2 * (long)X));  // ~64 KB of ping-pong buffers
    if (P < 1) P = 1;
    if (P > 16) P = 16;
    return {P, X + 1};
}
inline int y_lines(int Y) {
    int P = 4096 / Y;
    if (P < 1) P = 1;
    if (P > 16) P = 16;
    return P;
}
inline int z_cols(int Z, int Y) {
    int Q = 4096 / Z;
    if (Q < 1) Q = 1;
    if (Q > 16) Q = 16;
    if (Q > Y) Q = Y;
    return Q;
}

struct XArgs {
    int X, Xh, P, ls;
    long YZ;
    FftPlan plan;
    const float* src;  // real rows (forward from a real volume)
    float2* S;
    const float* phi;  // ratio epilogue
    float* psi;        // update epilogue / real output
    float eps;
};

// rows rho0 .. rho0+2P-1 of the (y,z) row space; pair p = (row p, row P+p)
__device__ __forceinline__ void load_real_pairs(const XArgs& a, float2* A, long rho0, int nrows,
                                                const float* __restrict__ src) {
    const int n2 = 2 * a.P * a.X;
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int row = t / a.X, n = t - row * a.X;
        const float v = row < nrows ? src[(rho0 + row) * a.X + n] : 0.f;
        const int p = row < a.P ? row : row - a.P;
        reinterpret_cast<float*>(A + p * a.ls + n)[row < a.P ? 0 : 1] = v;
    }
}

// after a forward complex FFT of the packed pairs: write both half spectra
__device__ __forceinline__ void unpack_store(const XArgs& a, const float2* F, long rho0, int nrows) {
    const int P2 = 2 * a.P;
    const int n = a.Xh * P2;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int k = t / P2, row = t - k * P2;
        if (row >= nrows) continue;
        const int p = row < a.P ? row : row - a.P;
        const float2 zk = F[p * a.ls + k];
        const int km = k == 0 ? 0 : a.X - k;
        const float2 zm = cconj(F[p * a.ls + km]);
        float2 val;
        if (row < a.P) {
            val = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
        } else {
            const float2 d = csub(zk, zm);
            val = make_float2(0.5f * d.y, -0.5f * d.x);
        }
        a.S[(long)k * a.YZ + rho0 + row] = val;
    }
}

// read both half spectra of the pairs and build Z = A + i B over the full line
__device__ __forceinline__ void load_spectrum_pairs(const XArgs& a, float2* A, float2* B, long rho0,
                                                    int nrows) {
    const int P2 = 2 * a.P;
    const int n = a.Xh * P2;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int k = t / P2, row = t - k * P2;
        const float2 v = row < nrows ? a.S[(long)k * a.YZ + rho0 + row] : make_float2(0.f, 0.f);
        if (row < a.P)
            A[row * a.ls + k] = v;
        else
            B[(row - a.P) * a.ls + k] = v;
    }
    __syncthreads();
    const int half = (a.X + 1) / 2;
    const int m = a.P * a.Xh;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const int p = t / a.Xh, k = t - p * a.Xh;
        const float2 av = A[p * a.ls + k], bv = B[p * a.ls + k];
        A[p * a.ls + k] = make_float2(av.x - bv.y, av.y + bv.x);  // A + iB
        if (k >= 1 && k < half)                                  // conj(A) + i conj(B) at -k
            A[p * a.ls + (a.X - k)] = make_float2(av.x + bv.y, bv.x - av.y);
    }
    __syncthreads();
}

// MODE 0: real volume -> spectrum
__global__ void __launch_bounds__(kThreads) k_x_forward(XArgs a) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* B = sm + a.P * a.ls;
    const long rho0 = (long)blockIdx.x * 2 * a.P;
    const int nrows = (int)min((long)2 * a.P, a.YZ - rho0);
    load_real_pairs(a, A, rho0, nrows, a.src);
    __syncthreads();
    const float2* F = fft_lines<-1>(A, B, a.P, a.ls, a.plan);
    unpack_store(a, F, rho0, nrows);
}

// spectrum -> inverse x -> r = phi / max(b, eps) -> forward x -> spectrum
__global__ void __launch_bounds__(kThreads) k_x_ratio(XArgs a) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* B = sm + a.P * a.ls;
    const long rho0 = (long)blockIdx.x * 2 * a.P;
    const int nrows = (int)min((long)2 * a.P, a.YZ - rho0);
    load_spectrum_pairs(a, A, B, rho0, nrows);
    float2* R = fft_lines<+1>(A, B, a.P, a.ls, a.plan);
    float2* O = R == A ? B : A;
    const int n2 = 2 * a.P * a.X;
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int row = t / a.X, n = t - row * a.X;
        const int p = row < a.P ? row : row - a.P;
        float* cell = reinterpret_cast<float*>(R + p * a.ls + n) + (row < a.P ? 0 : 1);
        float r = 0.f;
        if (row < nrows) {
            const float b = *cell;
            r = __ldg(a.phi + (rho0 + row) * a.X + n) / fmaxf(b, a.eps);
        }
        *cell = r;
    }
    __syncthreads();
    const float2* F = fft_lines<-1>(R, O, a.P, a.ls, a.plan);
    unpack_store(a, F, rho0, nrows);
}

// MODE update: spectrum -> inverse x -> psi = max(psi . c, eps)
// MODE store : spectrum -> inverse x -> dst (plain real output)
template <bool UPDATE>
__global__ void __launch_bounds__(kThreads) k_x_inverse(XArgs a) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* B = sm + a.P * a.ls;
    const long rho0 = (long)blockIdx.x * 2 * a.P;
    const int nrows = (int)min((long)2 * a.P, a.YZ - rho0);
    load_spectrum_pairs(a, A, B, rho0, nrows);
    const float2* R = fft_lines<+1>(A, B, a.P, a.ls, a.plan);
    const int n2 = nrows * a.X;
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int row = t / a.X, n = t - row * a.X;
        const int p = row < a.P ? row : row - a.P;
        const float c = reinterpret_cast<const float*>(R + p * a.ls + n)[row < a.P ? 0 : 1];
        float* dst = a.psi + (rho0 + row) * a.X + n;
        if (UPDATE)
            *dst = fmaxf(*dst * c, a.eps);
        else
            *dst = c;
    }
}

struct LineArgs {
    int L, ls, P;
    long nlines;
    FftPlan plan;
    float2* S;
};

// complex FFT along y: the spectrum is nlines = Xh*Z contiguous lines of Y
template <int S>
__global__ void __launch_bounds__(kThreads) k_y(LineArgs a) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* B = sm + a.P * a.ls;
    const long l0 = (long)blockIdx.x * a.P;
    const int nl = (int)min((long)a.P, a.nlines - l0);
    const int n = a.P * a.L;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int line = t / a.L, y = t - line * a.L;
        A[line * a.ls + y] = line < nl ? a.S[(l0 + line) * a.L + y] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* R = fft_lines<S>(A, B, a.P, a.ls, a.plan);
    const int m = nl * a.L;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const int line = t / a.L, y = t - line * a.L;
        a.S[(l0 + line) * a.L + y] = R[line * a.ls + y];
    }
}

struct ZArgs {
    int Z, Y, Q, ls, ntiles_y;
    long YZ;
    FftPlan plan;
    float2* S;
    const float2* K;
    float scale;
};

// along z at fixed (kx, y0..y0+Q-1): MUL=true  -> forward, times K, inverse
//                                   MUL=false -> forward, times scale
template <bool MUL>
__global__ void __launch_bounds__(kThreads) k_z(ZArgs a) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* B = sm + a.Q * a.ls;
    const int kx = blockIdx.x / a.ntiles_y;
    const int y0 = (blockIdx.x - kx * a.ntiles_y) * a.Q;
    const int nq = min(a.Q, a.Y - y0);
    const long base = (long)kx * a.YZ + y0;
    const int n = a.Z * a.Q;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int z = t / a.Q, q = t - z * a.Q;
        A[q * a.ls + z] = q < nq ? a.S[base + (long)z * a.Y + q] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* F = fft_lines<-1>(A, B, a.Q, a.ls, a.plan);
    float2* O = F == A ? B : A;
    if (MUL) {
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int z = t / a.Q, q = t - z * a.Q;
            if (q < nq) F[q * a.ls + z] = cmul(F[q * a.ls + z], __ldg(a.K + base + (long)z * a.Y + q));
        }
        __syncthreads();
        F = fft_lines<+1>(F, O, a.Q, a.ls, a.plan);
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int z = t / a.Q, q = t - z * a.Q;
        if (q < nq) {
            float2 v = F[q * a.ls + z];
            if (!MUL) v = cscale(v, a.scale);
            a.S[base + (long)z * a.Y + q] = v;
        }
    }
}

XArgs make_x(const FftGeom& g) {
    XTile t = x_tile(g.X);
    XArgs a{};
    a.X = g.X;
    a.Xh = g.Xh;
    a.P = t.P;
    a.ls = t.ls;
    a.YZ = g.YZ;
    a.plan = g.px;
    return a;
}

size_t x_smem(const XArgs& a) { return (size_t)2 * a.P * a.ls * sizeof(float2); }

template <typename K>
mvd_status launch_x(K kern, const XArgs& a, cudaStream_t st, const char* name, int cls) {
    const size_t sm = x_smem(a);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_status(e, name);
    prof_begin(cls, st);
    kern<<<div_up(a.YZ, 2 * a.P), kThreads, sm, st>>>(a);
    prof_end(cls, st);
    count_launch();
    return check_launch(name);
}

}  // namespace

mvd_status fft_forward_real_generic(const FftGeom& g, const float* src, float2* S, cudaStream_t st) {
    XArgs a = make_x(g);
    a.src = src;
    a.S = S;
    return launch_x(k_x_forward, a, st, "fft x forward", KC_X_FORWARD);
}

mvd_status fft_x_ratio_generic(const FftGeom& g, float2* S, const float* phi, float eps, cudaStream_t st) {
    XArgs a = make_x(g);
    a.S = S;
    a.phi = phi;
    a.eps = eps;
    return launch_x(k_x_ratio, a, st, "fft x ratio", KC_X_RATIO);
}

mvd_status fft_x_update_generic(const FftGeom& g, const float2* S, float* psi, float eps, cudaStream_t st) {
    XArgs a = make_x(g);
    a.S = const_cast<float2*>(S);
    a.psi = psi;
    a.eps = eps;
    return launch_x(k_x_inverse<true>, a, st, "fft x update", KC_X_UPDATE);
}

mvd_status fft_inverse_real_generic(const FftGeom& g, const float2* S, float* dst, cudaStream_t st) {
    XArgs a = make_x(g);
    a.S = const_cast<float2*>(S);
    a.psi = dst;
    return launch_x(k_x_inverse<false>, a, st, "fft x inverse", KC_SETUP);
}

mvd_status fft_y_generic(const FftGeom& g, float2* S, int inverse, cudaStream_t st) {
    LineArgs a{};
    a.L = g.Y;
    a.ls = g.Y + 1;
    a.P = y_lines(g.Y);
    a.nlines = (long)g.Xh * g.Z;
    a.plan = g.py;
    a.S = S;
    const size_t sm = (size_t)2 * a.P * a.ls * sizeof(float2);
    auto kern = inverse ? k_y<+1> : k_y<-1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_status(e, "fft y attr");
    prof_begin(KC_Y, st);
    kern<<<div_up(a.nlines, a.P), kThreads, sm, st>>>(a);
    prof_end(KC_Y, st);
    count_launch();
    return check_launch("fft y");
}

static mvd_status launch_z(const FftGeom& g, float2* S, const float2* K, float scale, bool mul,
                           cudaStream_t st) {
    ZArgs a{};
    a.Z = g.Z;
    a.Y = g.Y;
    a.Q = z_cols(g.Z, g.Y);
    a.ls = g.Z + 1;
    a.ntiles_y = div_up(g.Y, a.Q);
    a.YZ = g.YZ;
    a.plan = g.pz;
    a.S = S;
    a.K = K;
    a.scale = scale;
    const size_t sm = (size_t)2 * a.Q * a.ls * sizeof(float2);
    auto kern = mul ? k_z<true> : k_z<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_status(e, "fft z attr");
    const int cls = mul ? KC_Z_MUL : KC_SETUP;
    prof_begin(cls, st);
    kern<<<g.Xh * a.ntiles_y, kThreads, sm, st>>>(a);
    prof_end(cls, st);
    count_launch();
    return check_launch("fft z");
}

mvd_status fft_z_mul_generic(const FftGeom& g, float2* S, const float2* K, cudaStream_t st) {
    return launch_z(g, S, K, 1.f, true, st);
}

mvd_status fft_z_forward_scaled_generic(const FftGeom& g, float2* S, float scale, cudaStream_t st) {
    return launch_z(g, S, nullptr, scale, false, st);
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
mvd_status fft_x_update(const FftGeom& g, const float2* S, float* psi, float eps, cudaStream_t st) {
    if (g.fast && fft_fast_supported(g.X)) return fft_x_update_fast(g, S, psi, eps, st);
    return fft_x_update_generic(g, S, psi, eps, st);
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
