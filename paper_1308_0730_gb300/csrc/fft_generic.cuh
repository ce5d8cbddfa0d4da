// Generic (any {2,3,5}-smooth length) FFT passes as tile-level device
// functions: the per-volume kernels (fft_passes.cu) run one tile per block,
// the persistent batch kernel (batch.cu) runs whichever tile its work queue
// hands out. CO = true makes every load of data written inside the same
// launch (spectrum, estimate) an L2 load, as the batch kernel requires.
//
// Layout and contract as in fft_passes.cu: spectrum S[kx][z][y], two real
// x-lines per complex line, 1/M folded into the kernel spectra.
#pragma once

#include "dd.cuh"
#include "fft.cuh"

namespace mvd {

constexpr int kGenThreads = 256;

// rows (2P per tile) for the x pass: about 64 KB of ping-pong buffers
__host__ __device__ inline int gen_x_pairs(int X) {
    int P = 16384 / (2 * X);
    return P < 1 ? 1 : (P > 16 ? 16 : P);
}
__host__ __device__ inline int gen_y_lines(int Y) {
    int P = 4096 / Y;
    return P < 1 ? 1 : (P > 16 ? 16 : P);
}
__host__ __device__ inline int gen_z_cols(int Z, int Y) {
    int Q = 4096 / Z;
    Q = Q < 1 ? 1 : (Q > 16 ? 16 : Q);
    return Q > Y ? Y : Q;
}
__host__ __device__ inline long gen_div_up(long a, long b) { return (a + b - 1) / b; }

// tiles per pass and shared memory (bytes) per tile
__host__ __device__ inline long gen_x_tiles(int X, long YZ) { return gen_div_up(YZ, 2 * gen_x_pairs(X)); }
__host__ __device__ inline long gen_y_tiles(int Y, int Xh, int Z) { return gen_div_up((long)Xh * Z, gen_y_lines(Y)); }
__host__ __device__ inline long gen_z_tiles(int Z, int Y, int Xh) { return (long)Xh * gen_div_up(Y, gen_z_cols(Z, Y)); }
__host__ __device__ inline size_t gen_x_smem(int X) { return (size_t)2 * gen_x_pairs(X) * (X + 1) * sizeof(float2); }
__host__ __device__ inline size_t gen_y_smem(int Y) { return (size_t)2 * gen_y_lines(Y) * (Y + 1) * sizeof(float2); }
__host__ __device__ inline size_t gen_z_smem(int Z, int Y) {
    return (size_t)2 * gen_z_cols(Z, Y) * (Z + 1) * sizeof(float2);
}

struct GenX {
    int X, Xh, P, ls;
    long YZ;
    FftPlan plan;
    const float* src;  // real rows (forward from a real volume)
    float2* S;
    const float* phi;  // ratio epilogue
    float* psi;        // update epilogue / real output
    float eps;
    const float* wt;   // when set, the update applies the fraction wt of the change (partial overlap)
    float lam;         // Tikhonov regularisation of the update (0 = none)
    const float* inv_s;  // zero boundary: 1 / sensitivity of the update's view, or none
};

__host__ __device__ inline GenX gen_x_args(int X, long YZ, const FftPlan& plan) {
    GenX a{};
    a.X = X;
    a.Xh = X / 2 + 1;
    a.P = gen_x_pairs(X);
    a.ls = X + 1;
    a.YZ = YZ;
    a.plan = plan;
    return a;
}

// rows rho0 .. rho0+2P-1 of the (y,z) row space; pair p = (row p, row P+p)
template <bool CO>
__device__ __forceinline__ void gen_load_real_pairs(const GenX& a, float2* A, long rho0, int nrows) {
    const int n2 = 2 * a.P * a.X;
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int row = t / a.X, n = t - row * a.X;
        const float v = row < nrows ? ld1<CO>(a.src + (rho0 + row) * a.X + n) : 0.f;
        const int p = row < a.P ? row : row - a.P;
        reinterpret_cast<float*>(A + p * a.ls + n)[row < a.P ? 0 : 1] = v;
    }
}

// after a forward complex FFT of the packed pairs: write both half spectra
__device__ __forceinline__ void gen_unpack_store(const GenX& a, const float2* F, long rho0, int nrows) {
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
template <bool CO>
__device__ __forceinline__ void gen_load_spectrum_pairs(const GenX& a, float2* A, float2* B, long rho0, int nrows) {
    const int P2 = 2 * a.P;
    const int n = a.Xh * P2;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int k = t / P2, row = t - k * P2;
        float2 v = make_float2(0.f, 0.f);
        if (row < nrows) {
            const long at = (long)k * a.YZ + rho0 + row;
            v = ld2<CO>(a.S + at);
        }
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

// real volume -> spectrum, one tile of 2P rows
template <bool CO>
__device__ void gen_x_forward_tile(const GenX& a, long tile, float2* sm) {
    float2* A = sm;
    float2* B = sm + a.P * a.ls;
    const long rho0 = tile * 2 * a.P;
    const int nrows = (int)min((long)2 * a.P, a.YZ - rho0);
    gen_load_real_pairs<CO>(a, A, rho0, nrows);
    __syncthreads();
    const float2* F = fft_lines<-1>(A, B, a.P, a.ls, a.plan);
    gen_unpack_store(a, F, rho0, nrows);
}

// spectrum -> inverse x -> r = phi / max(b, eps) -> forward x of r - 1 -> spectrum
// (transforming r - 1 instead of r keeps the large mean of r out of the FP32
// back-projection's rounding; the update adds the 1 back, since K sums to 1)
template <bool CO>
__device__ void gen_x_ratio_tile(const GenX& a, long tile, float2* sm) {
    float2* A = sm;
    float2* B = sm + a.P * a.ls;
    const long rho0 = tile * 2 * a.P;
    const int nrows = (int)min((long)2 * a.P, a.YZ - rho0);
    gen_load_spectrum_pairs<CO>(a, A, B, rho0, nrows);
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
            r = __ldg(a.phi + (rho0 + row) * a.X + n) / fmaxf(b, a.eps) - 1.f;
        }
        *cell = r;  // r - 1: the back-projection transforms r - 1 and adds 1 back
    }
    __syncthreads();
    const float2* F = fft_lines<-1>(R, O, a.P, a.ls, a.plan);
    gen_unpack_store(a, F, rho0, nrows);
}

// UPDATE: spectrum -> inverse x -> psi = max(psi . c, eps); else plain real output
// MODE 0: plain real output ; 1: psi update ; 4: acc *= c (the combined
// update's product of view factors; acc in a.psi)
template <bool CO, int MODE>
__device__ void gen_x_inverse_tile(const GenX& a, long tile, float2* sm) {
    float2* A = sm;
    float2* B = sm + a.P * a.ls;
    const long rho0 = tile * 2 * a.P;
    const int nrows = (int)min((long)2 * a.P, a.YZ - rho0);
    gen_load_spectrum_pairs<CO>(a, A, B, rho0, nrows);
    const float2* R = fft_lines<+1>(A, B, a.P, a.ls, a.plan);
    const int n2 = nrows * a.X;
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int row = t / a.X, n = t - row * a.X;
        const int p = row < a.P ? row : row - a.P;
        const float c = reinterpret_cast<const float*>(R + p * a.ls + n)[row < a.P ? 0 : 1];
        float* dst = a.psi + (rho0 + row) * a.X + n;
        if (MODE == 1) {  // c here is (r - 1) * K: the factor is c + 1 (K sums to 1), see update_factor
            const float old = ld1<CO>(dst);
            *dst = fmaxf(old * update_factor(c, old, a.wt, (rho0 + row) * a.X + n, a.lam, a.inv_s), a.eps);
        }
        else if (MODE == 4)
            *dst = ld1<CO>(dst) * (c + 1.f) * (a.inv_s ? __ldg(a.inv_s + (rho0 + row) * a.X + n) : 1.f);
        else
            *dst = c;
    }
}

struct GenY {
    int L, ls, P;
    long nlines;
    FftPlan plan;
    float2* S;
};

__host__ __device__ inline GenY gen_y_args(int Y, int Xh, int Z, const FftPlan& plan, float2* S) {
    GenY a{};
    a.L = Y;
    a.ls = Y + 1;
    a.P = gen_y_lines(Y);
    a.nlines = (long)Xh * Z;
    a.plan = plan;
    a.S = S;
    return a;
}

// complex FFT along y: the spectrum is nlines = Xh*Z contiguous lines of Y
template <bool CO, int S>
__device__ void gen_y_tile(const GenY& a, long tile, float2* sm) {
    float2* A = sm;
    float2* B = sm + a.P * a.ls;
    const long l0 = tile * a.P;
    const int nl = (int)min((long)a.P, a.nlines - l0);
    const int n = a.P * a.L;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int line = t / a.L, y = t - line * a.L;
        A[line * a.ls + y] = line < nl ? ld2<CO>(a.S + (l0 + line) * a.L + y) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* R = fft_lines<S>(A, B, a.P, a.ls, a.plan);
    const int m = nl * a.L;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const int line = t / a.L, y = t - line * a.L;
        a.S[(l0 + line) * a.L + y] = R[line * a.ls + y];
    }
}

struct GenZ {
    int Z, Y, Q, ls, ntiles_y;
    long YZ;
    FftPlan plan;
    float2* S;
    const float2* K;
    float scale;
};

__host__ __device__ inline GenZ gen_z_args(int Z, int Y, long YZ, const FftPlan& plan, float2* S, const float2* K,
                                           float scale) {
    GenZ a{};
    a.Z = Z;
    a.Y = Y;
    a.Q = gen_z_cols(Z, Y);
    a.ls = Z + 1;
    a.ntiles_y = (int)gen_div_up(Y, a.Q);
    a.YZ = YZ;
    a.plan = plan;
    a.S = S;
    a.K = K;
    a.scale = scale;
    return a;
}

// along z at fixed (kx, y0..y0+Q-1): MUL -> forward, times K, inverse;
// otherwise forward, times scale
template <bool CO, bool MUL>
__device__ void gen_z_tile(const GenZ& a, long tile, float2* sm) {
    float2* A = sm;
    float2* B = sm + a.Q * a.ls;
    const int kx = (int)(tile / a.ntiles_y);
    const int y0 = (int)(tile - (long)kx * a.ntiles_y) * a.Q;
    const int nq = min(a.Q, a.Y - y0);
    const long base = (long)kx * a.YZ + y0;
    const int n = a.Z * a.Q;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int z = t / a.Q, q = t - z * a.Q;
        A[q * a.ls + z] = q < nq ? ld2<CO>(a.S + base + (long)z * a.Y + q) : make_float2(0.f, 0.f);
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

}  // namespace mvd
