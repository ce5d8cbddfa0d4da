// Register-resident double-float line FFT and forward-blur tiles for
// power-of-two lengths 32..1024 (same scheme as fft_fast.cuh, 8 elements per
// thread: a line of length L is held by TPL = L/8 threads, thread t owning
// elements t + TPL*q; radix-8 Stockham stages, then one radix 2 or 4 stage;
// padded shared-memory exchanges between stages).
#pragma once

#include "adf.cuh"
#include "dd.cuh"
#include "fft_fast.cuh"

namespace mvd {

constexpr int kE8 = 8;
constexpr int kDdThreads = 256;

__host__ __device__ constexpr int plan8_n(int L) {
    int n = 0;
    while (L % 8 == 0 && L >= 8) {
        L /= 8;
        ++n;
    }
    return n;
}
__host__ __device__ constexpr int plan8_rem(int L) {
    while (L % 8 == 0 && L >= 8) L /= 8;
    return L;  // 1, 2 or 4
}
__host__ __device__ constexpr int plan8_radix(int L, int s) {
    return s < plan8_n(L) ? 8 : (s == plan8_n(L) && plan8_rem(L) > 1 ? plan8_rem(L) : 0);
}
__host__ __device__ constexpr int plan8_nst(int L) { return plan8_n(L) + (plan8_rem(L) > 1 ? 1 : 0); }
__host__ __device__ constexpr bool dd_fast_length(int L) { return L >= 32 && L <= 1024 && (L & (L - 1)) == 0; }

// Twiddles in stage order: the natural table of a length L (w^m, m < L) is
// followed by the stage-ordered one, where stage s >= 1 (NS points combined
// before it, radix R) keeps w^(r k L / (NS R)) at tw_stage_off(L, s) +
// (r - 1) NS + k: a warp's consecutive k read consecutive entries (in natural
// order they would sit L / (NS R) entries apart).
__host__ __device__ constexpr int tw_stage_off(int L, int ST) {
    int off = 0, ns = 1;
    for (int s = 0; s < ST; ++s) {
        const int R = plan8_radix(L, s);
        if (s > 0) off += (R - 1) * ns;
        ns *= R;
    }
    return off;
}

// padded index: one pad slot per 8 elements; line stride shifts lines across banks
__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }
__host__ __device__ constexpr int line_stride8(int L) { return L + L / 8 + 1; }

// Arithmetic: aligned double-float (adf.cuh). run() first takes the largest
// component of the line (a reduction over its threads), puts every value on
// the grid of that bound's quantum, and each later stage moves to a grid 16
// times coarser (the growth bound of a radix-8 stage); butterfly sums are then
// exact FP32 adds, and only the products (twiddles, sqrt(2)/2) are rounded
// back onto the grid. The result is an unevaluated pair per component (hi on
// the last stage's grid, lo the remainder).
// DB > 0: the exchanges alternate between the line's buffer at sm and a second
// one at sm + DB (cdd elements), so a stage may write while slower threads of
// the line still read the previous stage's buffer: one barrier per exchange
// instead of two.
// TWS: the stage-ordered twiddles are a copy in shared memory at padded index
// pad8(i) (the z tile: its Q columns share every twiddle, so a warp's reads
// are broadcasts of few distinct words); else tw is the global natural table,
// followed by the stage-ordered one (read-only path).
// QI: with !WARP_LOCAL, the block interleaves QI lines (line = thread % QI).
// The line-bound reduction keeps its partial maxima in the line buffer's pad
// slots (cdd index 9k + 8, which no exchange touches).
template <int L, int S, bool WARP_LOCAL, int DB = 0, bool TWS = false, int QI = 1>
struct LineFFTDD {
    static constexpr int TPL = L / kE8;
    static constexpr int NST = plan8_nst(L);

    // WARP_LOCAL: the TPL threads of a line are contiguous, so a line longer
    // than a warp synchronises on its own named barrier (id bar, TPL threads)
    // instead of the whole block: the lines of a block then drift apart and
    // their warps stop queueing on the same pipes at the same time.
    __device__ __forceinline__ static void sync(int bar) {
        if constexpr (WARP_LOCAL && TPL <= 32)
            __syncwarp();
        else if constexpr (WARP_LOCAL)
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(TPL) : "memory");
        else
            __syncthreads();
    }

    __device__ __forceinline__ static float* red_slot(cdd* sm, int g) {
        return reinterpret_cast<float*>(sm + 9 * (g >> 2) + 8) + (g & 3);
    }

    // largest |hi| component over the line's TPL threads
    __device__ __forceinline__ static float line_bound(const cdd (&v)[kE8], cdd* sm, int t, int bar) {
        float m = 0.f;
#pragma unroll
        for (int q = 0; q < kE8; ++q) m = adf_absmax(v[q], m);
        if constexpr (WARP_LOCAL) {
            constexpr int W = TPL < 32 ? TPL : 32;
#pragma unroll
            for (int o = 1; o < W; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if constexpr (TPL > 32) {
                if ((t & 31) == 0) *red_slot(sm, t >> 5) = m;
                sync(bar);
#pragma unroll
                for (int g = 0; g < TPL / 32; ++g) m = fmaxf(m, *red_slot(sm, g));
            }
        } else {
            constexpr int LPW = QI >= 32 ? 1 : 32 / QI;  // a line's lanes in one warp
            constexpr int G = TPL / LPW;
            static_assert(G <= 16, "line-bound groups exceed the pad slots");
#pragma unroll
            for (int o = QI; o < 32; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (t % LPW == 0) *red_slot(sm, t / LPW) = m;
            __syncthreads();
#pragma unroll
            for (int g = 0; g < G; ++g) m = fmaxf(m, *red_slot(sm, g));
        }
        return m;
    }

    template <int ST, int NS>
    __device__ __forceinline__ static void stage(cdd (&v)[kE8], cdd* sm, int t, const cdd* __restrict__ tw, int bar,
                                                 int e0) {
        if constexpr (ST < NST) {
            constexpr int R = plan8_radix(L, ST);
            constexpr int B = kE8 / R;
            constexpr bool LAST = (ST == NST - 1);
            const float c = adf_const_exp2(e0 + 4 * ST);  // every stage before this one is radix 8
#pragma unroll
            for (int m = 0; m < B; ++m) {
                cdd x[R];
#pragma unroll
                for (int r = 0; r < R; ++r) x[r] = v[m + r * B];
                const int j = t + TPL * m;
                const int k = j % NS;
                if (NS > 1) {
                    constexpr int OFF = tw_stage_off(L, ST);
                    x[0] = adf_calign(x[0], c);
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        cdd w;
                        if constexpr (TWS) {
                            w = cdd_load(tw + pad8(OFF + (r - 1) * NS + k));
                            if (S > 0) w.im = dd{-w.im.hi, -w.im.lo};
                        } else {
                            w = twiddle_dd<S>(tw + L, OFF + (r - 1) * NS + k);
                        }
                        x[r] = adf_cmul(x[r], w, c);
                    }
                }
                DftA<R, S>::run(x, c);
                if (LAST) {
#pragma unroll
                    for (int r = 0; r < R; ++r) v[m + r * B] = x[r];
                } else {
                    const int d = (j / NS) * NS * R + k;
                    cdd* buf = sm + ((DB > 0 && (ST & 1)) ? DB : 0);
#pragma unroll
                    for (int r = 0; r < R; ++r) cdd_store(buf + pad8(d + r * NS), x[r]);
                }
            }
            if constexpr (!LAST) {
                const cdd* buf = sm + ((DB > 0 && (ST & 1)) ? DB : 0);
                sync(bar);
#pragma unroll
                for (int q = 0; q < kE8; ++q) v[q] = cdd_load(buf + pad8(t + TPL * q));
                if constexpr (DB == 0) sync(bar);
                stage<ST + 1, NS * R>(v, sm, t, tw, bar, e0);
            }
        }
    }

    // bar: the line's named barrier (1 + its index in the block) when WARP_LOCAL
    __device__ __forceinline__ static void run(cdd (&v)[kE8], cdd* sm, int t, const cdd* __restrict__ tw,
                                               int bar = 1) {
        const int e0 = adf_exp_for(line_bound(v, sm, t, bar));
        const float c0 = adf_const_exp2(e0);
#pragma unroll
        for (int q = 0; q < kE8; ++q) v[q] = adf_calign(v[q], c0);
        stage<0, 1>(v, sm, t, tw, bar, e0);
    }
};

// The same register-resident plan in FP32 (float2 elements; tw is the FP32
// natural table of L, followed by its radix-8 stage-ordered copy): used for
// the back-projection's forward x transform of r - 1, whose
// input the double-float inverse leaves in exactly this distribution. Its
// exchanges pad one slot per 16 float2 (128 bytes; one per 8 would put the
// 16th element of a half-warp's load on the bank of the first); a line uses
// L + L/16 + 1 float2 of shared memory, inside the double-float line's region.
template <int L, int S, bool WARP_LOCAL>
struct LineFFT8F {
    static constexpr int TPL = L / kE8;
    static constexpr int NST = plan8_nst(L);

    // WARP_LOCAL: the TPL threads of a line are contiguous, so a line longer
    // than a warp synchronises on its own named barrier (id bar, TPL threads)
    // instead of the whole block: the lines of a block then drift apart and
    // their warps stop queueing on the same pipes at the same time.
    __device__ __forceinline__ static void sync(int bar) {
        if constexpr (WARP_LOCAL && TPL <= 32)
            __syncwarp();
        else if constexpr (WARP_LOCAL)
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(TPL) : "memory");
        else
            __syncthreads();
    }

    template <int ST, int NS>
    __device__ __forceinline__ static void stage(float2 (&v)[kE8], float2* sm, int t, const float2* __restrict__ tw,
                                                 int bar) {
        if constexpr (ST < NST) {
            constexpr int R = plan8_radix(L, ST);
            constexpr int B = kE8 / R;
            constexpr bool LAST = (ST == NST - 1);
#pragma unroll
            for (int m = 0; m < B; ++m) {
                float2 x[R];
#pragma unroll
                for (int r = 0; r < R; ++r) x[r] = v[m + r * B];
                const int j = t + TPL * m;
                const int k = j % NS;
                if (NS > 1) {
                    constexpr int OFF = tw_stage_off(L, ST);
#pragma unroll
                    for (int r = 1; r < R; ++r) x[r] = cmul(x[r], twiddle<S>(tw + L, OFF + (r - 1) * NS + k));
                }
                Dft<R, S>::run(x);
                if (LAST) {
#pragma unroll
                    for (int r = 0; r < R; ++r) v[m + r * B] = x[r];
                } else {
                    const int d = (j / NS) * NS * R + k;
#pragma unroll
                    for (int r = 0; r < R; ++r) sm[pad16(d + r * NS)] = x[r];
                }
            }
            if constexpr (!LAST) {
                sync(bar);
#pragma unroll
                for (int q = 0; q < kE8; ++q) v[q] = sm[pad16(t + TPL * q)];
                sync(bar);
                stage<ST + 1, NS * R>(v, sm, t, tw, bar);
            }
        }
    }

    __device__ __forceinline__ static void run(float2 (&v)[kE8], float2* sm, int t, const float2* __restrict__ tw,
                                               int bar = 1) {
        stage<0, 1>(v, sm, t, tw, bar);
    }
};

// tile geometry
__host__ __device__ constexpr int ddf_pairs(int L) { return kDdThreads / (L / kE8); }  // x pass: pairs per tile
__host__ __device__ constexpr int ddf_y_lines(int L) { return kDdThreads / (L / kE8); }
__host__ __device__ constexpr int ddf_z_cols(int L) {
    return (kDdThreads / (L / kE8)) >= 4 ? kDdThreads / (L / kE8) : 4;
}
// half-spectrum rows (XH = L/2 + 1 values) of the x-pass gather, unpadded:
// the pair line reads them in ascending runs (k <= L/2) and descending runs
// (L - k), and a padded row would split a quarter-warp's descending run over
// a pad slot (two wavefronts). The gather's quarter-warp writes 8 rows of one
// k (odd stride: distinct banks) or, with two pairs, 4 rows of k and k + 1
// (stride 2 mod 8). The x passes' 2P gathered rows and their P transformed
// lines share the buffer (the two phases are separated by a barrier). With two
// pairs per tile (L = 1024) the unpacking's 2 lines of a quarter-warp collide
// on the banks at a line stride of one pad slot; + 3 spreads them.
__host__ __device__ constexpr int x_half_stride8(int L) { return L / 2 + 1 + (ddf_pairs(L) == 2 ? 1 : 0); }
__host__ __device__ constexpr int x_line_stride8(int L) { return L + L / 8 + (ddf_pairs(L) == 2 ? 3 : 1); }
__host__ __device__ constexpr size_t ddf_x_smem(int L) {
    return (size_t)(2 * ddf_pairs(L) * x_half_stride8(L) > ddf_pairs(L) * x_line_stride8(L)
                        ? 2 * ddf_pairs(L) * x_half_stride8(L)
                        : ddf_pairs(L) * x_line_stride8(L)) *
           sizeof(cdd);
}
__host__ __device__ constexpr size_t ddf_y_smem(int L) { return (size_t)ddf_y_lines(L) * line_stride8(L) * sizeof(cdd); }
// z lines: a warp holds Q interleaved columns (q = thread % Q); with Q = 4 a
// stride of L + L/8 + 1 puts columns q and q + 1 one bank apart, so the
// exchanges of neighbouring threads collide (two wavefronts per quarter-warp);
// + 2 spreads them over distinct banks
__host__ __device__ constexpr int z_line_stride8(int L) { return L + L / 8 + (ddf_z_cols(L) == 4 ? 2 : 1); }
__host__ __device__ constexpr size_t ddf_z_smem(int L) {
    return (size_t)2 * ddf_z_cols(L) * z_line_stride8(L) * sizeof(cdd);
}

template <bool CO>
__device__ __forceinline__ cdd ld_cdd(const cdd* p) {
    if constexpr (CO)
        return cdd_load_cg(p);
    else
        return cdd_load(p);
}

// IO selects where the lines come from:
//   0: the double-float spectrum S2, in place;
//   1: read the FP32 spectrum S1 (each value widened exactly), write S2.
// IO 1 takes the ratio pass's FP32 spectrum of r - 1 (exact FP32 values, so
// nothing is lost against storing them as double-float) at half the bytes.
template <int L, int S, bool CO, int IO = 0>
__device__ __forceinline__ void ddf_y_tile(cdd* __restrict__ S2, long nlines, const cdd* __restrict__ tw2, long tile,
                                           cdd* sm, float2* __restrict__ S1 = nullptr) {
    using F = LineFFTDD<L, S, true>;
    constexpr int TPL = F::TPL, LPC = kDdThreads / TPL;
    const int li = threadIdx.x / TPL, t = threadIdx.x - li * TPL;
    const long line = tile * LPC + li;
    const bool ok = line < nlines;
    cdd* g = S2 + line * L;
    float2* g1 = S1 + line * L;
    cdd v[kE8];
#pragma unroll
    for (int q = 0; q < kE8; ++q) {
        if constexpr (IO == 1) {
            const float2 f = ok ? (CO ? __ldcg(g1 + t + TPL * q) : g1[t + TPL * q]) : make_float2(0.f, 0.f);
            v[q] = cdd{dd_from(f.x), dd_from(f.y)};
        } else {
            v[q] = ok ? ld_cdd<CO>(g + t + TPL * q) : czero_dd();
        }
    }
    F::run(v, sm + li * line_stride8(L), t, tw2, 1 + li);
    if (ok) {
#pragma unroll
        for (int q = 0; q < kE8; ++q) cdd_store(g + t + TPL * q, v[q]);
    }
}

// z: forward, times the double-float kernel spectrum, inverse (MUL); or
// forward times a scale. Needs Q * L/8 threads.
template <int L, bool MUL, bool CO>
__device__ __forceinline__ void ddf_z_tile(cdd* __restrict__ S2, const cdd* __restrict__ K2, int Y, long YZ,
                                           int ntiles_y, dd scale, const cdd* __restrict__ tw2, long tile, cdd* sm) {
    constexpr int TPL = L / kE8, Q = ddf_z_cols(L);
    const int q = threadIdx.x % Q, t = threadIdx.x / Q;
    const int kx = (int)(tile / ntiles_y);
    const int y0 = (int)(tile - (long)kx * ntiles_y) * Q;
    const bool ok = y0 + q < Y;
    const long base = (long)kx * YZ + y0 + q;
    cdd* line_sm = sm + q * z_line_stride8(L);
    cdd v[kE8];
#pragma unroll
    for (int i = 0; i < kE8; ++i) v[i] = ok ? ld_cdd<CO>(S2 + base + (long)(t + TPL * i) * Y) : czero_dd();
    using FF = LineFFTDD<L, -1, false, Q * z_line_stride8(L), false, Q>;
    using FI = LineFFTDD<L, +1, false, Q * z_line_stride8(L), false, Q>;
    FF::run(v, line_sm, t, tw2);
    if (MUL) {
#pragma unroll
        for (int i = 0; i < kE8; ++i) v[i] = cmul(v[i], ok ? cdd_load_nc(K2 + base + (long)(t + TPL * i) * Y) : czero_dd());
        __syncthreads();
        FI::run(v, line_sm, t, tw2);
    } else {
#pragma unroll
        for (int i = 0; i < kE8; ++i) v[i] = cdd{dd_mul(v[i].re, scale), dd_mul(v[i].im, scale)};
    }
    if (ok) {
#pragma unroll
        for (int i = 0; i < kE8; ++i) cdd_store(S2 + base + (long)(t + TPL * i) * Y, v[i]);
    }
}

// z pass (forward x spectrum x inverse) with the twiddles in shared memory:
// the Q column lines, then the stage-ordered twiddle table at pad8(i) (loaded
// from the global table, the compiler hoists later stages' twiddles above the
// stage barriers and holds them in registers).
__host__ __device__ constexpr bool ddf_z2_length(int L) { return L >= 128 && L <= 512 && (L & (L - 1)) == 0; }
__host__ __device__ constexpr int z2_tw_offset(int L) { return ddf_z_cols(L) * z_line_stride8(L); }
__host__ __device__ constexpr size_t ddf_z2_smem(int L) {
    return (size_t)(z2_tw_offset(L) + L + L / 8) * sizeof(cdd);
}

// The z pass as a persistent, software-pipelined loop: each block walks the
// tiles blockIdx.x, blockIdx.x + gridDim.x, ... and, while it transforms one
// tile, the next tile's columns of S2 and of the kernel spectrum are already
// in flight into shared memory by asynchronous copies. Every thread copies
// exactly the elements it will itself read (thread-private slots
// i * 256 + thread), so neither the copies' completion (cp.async.wait_group
// of its own groups) nor the reuse of the slots needs a barrier. Two blocks
// per SM (the twiddles, the column lines and both staging areas take 110 KB
// for L = 512); measured faster than three blocks of the unpipelined tile.
__host__ __device__ constexpr size_t ddf_z2_pipe_smem(int L) {
    return ddf_z2_smem(L) + (size_t)2 * kE8 * kDdThreads * sizeof(cdd);
}

template <int L>
__device__ __forceinline__ void ddf_z2_pipe(cdd* __restrict__ S2, const cdd* __restrict__ K2, int Y, long YZ,
                                            int ntiles_y, const cdd* __restrict__ tw2, long ntiles, cdd* sm) {
    constexpr int TPL = L / kE8, Q = ddf_z_cols(L);
    const int q = threadIdx.x % Q, t = threadIdx.x / Q;
    cdd* tws = sm + z2_tw_offset(L);
    cdd* line_sm = sm + q * z_line_stride8(L);
    cdd* stS = sm + z2_tw_offset(L) + L + L / 8 + threadIdx.x;  // slot i at stS[i * 256]
    cdd* stK = stS + kE8 * kDdThreads;
    const long step = (long)TPL * Y;
    // element i of this thread's column of tile `tile` sits at col_off(tile) + i * step
    auto col_off = [&](long tile, bool& ok) {
        const int kx = (int)(tile / ntiles_y);
        const int y0 = (int)(tile - (long)kx * ntiles_y) * Q;
        ok = y0 + q < Y;
        return (long)kx * YZ + y0 + q + (long)t * Y;
    };
    auto issue = [&](cdd* slots, const cdd* src, long tile) {
        bool ok;
        const long off = col_off(tile, ok);
#pragma unroll
        for (int i = 0; i < kE8; ++i) cp_async16(slots + i * kDdThreads, ok ? src + off + i * step : src, ok);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    for (int m = threadIdx.x; m < L; m += Q * TPL) cp_async16(tws + pad8(m), tw2 + L + m, true);
    long tile = blockIdx.x;
    if (tile < ntiles) {
        issue(stS, S2, tile);
        issue(stK, K2, tile);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();  // the twiddle table is shared
    for (; tile < ntiles; tile += gridDim.x) {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        const long next = tile + gridDim.x;
        cdd v[kE8];
#pragma unroll
        for (int i = 0; i < kE8; ++i) v[i] = stS[i * kDdThreads];
        if (next < ntiles) issue(stS, S2, next);
        LineFFTDD<L, -1, false, 0, true, Q>::run(v, line_sm, t, tws);
#pragma unroll
        for (int i = 0; i < kE8; ++i) v[i] = cmul_pair(v[i], stK[i * kDdThreads]);
        if (next < ntiles) issue(stK, K2, next);
        // no barrier here nor at the loop's end: the next transform writes the
        // column lines only after its bound reduction's block barrier, which
        // every thread reaches after its last read of the previous transform
        LineFFTDD<L, +1, false, 0, true, Q>::run(v, line_sm, t, tws);
        bool ok;
        long o = col_off(tile, ok);
        if (ok) {
            cdd* col = S2 + o;
#pragma unroll
            for (int i = 0; i < kE8; ++i) cdd_store(col + i * step, v[i]);
        }
    }
}

struct DdXFast {
    const float* src;  // real rows
    cdd* S2;
    const float* phi;
    long YZ;
    float eps;
    const cdd* tw2;
    FftPlan plan;      // FP32 plan of X (radices + FP32 twiddles) for the r - 1 transform
    float* dst;        // real rows written by the plain inverse
    float2* S;         // ratio: the FP32 spectrum of r - 1 goes here when set, else into S2
};

// unpack the packed forward double-float spectra (natural order in registers
// of pair p) into the two half spectra, coalesced over rows
template <int L>
__device__ __forceinline__ void ddf_store_halves(const DdXFast& a, cdd (&v)[kE8], cdd* sm, int p, int t, long rho0,
                                                 int nrows) {
    constexpr int TPL = L / kE8, P = ddf_pairs(L), LS = x_line_stride8(L), XH = L / 2 + 1;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kE8; ++q) cdd_store(sm + p * LS + pad8(t + TPL * q), v[q]);
    __syncthreads();
    for (int idx = threadIdx.x; idx < XH * 2 * P; idx += kDdThreads) {
        const int k = idx / (2 * P), row = idx - k * 2 * P;
        if (row >= nrows) continue;
        const int pp = row < P ? row : row - P;
        // zk and zm are outputs of one aligned line (one grid, below 2^23 q):
        // their sums and differences are exact FP32 adds
        const cdd zk = cdd_load(sm + pp * LS + pad8(k));
        const cdd zm = cconj(cdd_load(sm + pp * LS + pad8(k == 0 ? 0 : L - k)));
        cdd val;
        if (row < P) {
            val = chalf(adf_cadd(zk, zm));
        } else {
            const cdd d = chalf(adf_csub(zk, zm));
            val = cdd{d.im, dd{-d.re.hi, -d.re.lo}};
        }
        cdd_store(a.S2 + (long)k * a.YZ + rho0 + row, val);
    }
}

template <int L, bool CO>
__device__ __forceinline__ void ddf_x_forward_tile(const DdXFast& a, long tile, cdd* sm) {
    constexpr int TPL = L / kE8, P = ddf_pairs(L), LS = x_line_stride8(L);
    const int p = threadIdx.x / TPL, t = threadIdx.x - p * TPL;
    const long rho0 = tile * 2 * P;
    const int nrows = (int)min((long)2 * P, a.YZ - rho0);
    const bool oka = p < nrows, okb = P + p < nrows;
    const float* ra = a.src + (rho0 + p) * L;
    const float* rb = a.src + (rho0 + P + p) * L;
    cdd v[kE8];
#pragma unroll
    for (int q = 0; q < kE8; ++q) {
        const int n = t + TPL * q;
        v[q] = cdd{dd_from(oka ? ld1<CO>(ra + n) : 0.f), dd_from(okb ? ld1<CO>(rb + n) : 0.f)};
    }
    LineFFTDD<L, -1, true>::run(v, sm + p * LS, t, a.tw2, 1 + p);
    ddf_store_halves<L>(a, v, sm, p, t, rho0, nrows);
}

// issue the asynchronous copies of the half spectra of rows rho0 + p (A) and
// rho0 + P + p (B) of a tile into shared memory (rows < P -> row p, rows >= P
// -> row P + p, at stride HS); every copy is in flight before any completes
template <int L>
__device__ __forceinline__ void ddf_gather_issue(const DdXFast& a, long rho0, int nrows, cdd* sm) {
    constexpr int P = ddf_pairs(L), HS = x_half_stride8(L), XH = L / 2 + 1;
    for (int idx = threadIdx.x; idx < XH * 2 * P; idx += kDdThreads) {
        const int k = idx / (2 * P), row = idx - k * 2 * P;
        const bool ok = row < nrows;
        cp_async16(sm + row * HS + k, ok ? a.S2 + (long)k * a.YZ + rho0 + row : a.S2, ok);
    }
}

// the full spectrum of the complex line A + iB of pair p from the gathered halves
template <int L>
__device__ __forceinline__ void ddf_pair_line(const cdd* sm, int p, int t, cdd (&v)[kE8]) {
    constexpr int TPL = L / kE8, P = ddf_pairs(L), HS = x_half_stride8(L);
#pragma unroll
    for (int q = 0; q < kE8; ++q) {
        const int k = t + TPL * q;
        const int kk = k <= L / 2 ? k : L - k;
        const cdd A = cdd_load(sm + p * HS + kk), B = cdd_load(sm + (P + p) * HS + kk);
        v[q] = k <= L / 2 ? cdd{dd_sub(A.re, B.im), dd_add(A.im, B.re)}    // A + iB
                          : cdd{dd_add(A.re, B.im), dd_sub(B.re, A.im)};   // conj(A) + i conj(B)
    }
}

// gather the half spectra of rows rho0 + p (A) and rho0 + P + p (B) of a
// tile and form the full spectrum of the complex line A + iB in v
template <int L, bool CO>
__device__ __forceinline__ void ddf_gather_pair(const DdXFast& a, long rho0, int nrows, int p, int t, cdd* sm,
                                                cdd (&v)[kE8]) {
    ddf_gather_issue<L>(a, rho0, nrows, sm);
    cp_async_wait_all();
    __syncthreads();
    ddf_pair_line<L>(sm, p, t, v);
}

// double-float spectrum -> inverse x -> real rows (rounded to FP32) in dst
template <int L, bool CO>
__device__ __forceinline__ void ddf_x_inverse_tile(const DdXFast& a, long tile, cdd* sm) {
    constexpr int TPL = L / kE8, P = ddf_pairs(L), LS = x_line_stride8(L);
    const int p = threadIdx.x / TPL, t = threadIdx.x - p * TPL;
    const long rho0 = tile * 2 * P;
    const int nrows = (int)min((long)2 * P, a.YZ - rho0);
    cdd v[kE8];
    ddf_gather_pair<L, CO>(a, rho0, nrows, p, t, sm, v);
    __syncthreads();
    LineFFTDD<L, +1, true>::run(v, sm + p * LS, t, a.tw2, 1 + p);
    const long ra = (rho0 + p) * L, rb = (rho0 + P + p) * L;
#pragma unroll
    for (int q = 0; q < kE8; ++q) {
        const int n = t + TPL * q;
        if (p < nrows) a.dst[ra + n] = v[q].re.hi + v[q].re.lo;
        if (P + p < nrows) a.dst[rb + n] = v[q].im.hi + v[q].im.lo;
    }
}

// shared memory of the ratio pass: the x-pass buffer, then the 2P observed rows
__host__ __device__ constexpr size_t ddf_ratio_smem(int L) {
    return ddf_x_smem(L) + (size_t)2 * ddf_pairs(L) * L * sizeof(float);
}

// double-float spectrum -> inverse x -> b -> r - 1 = phi / max(b, eps) - 1
// -> FP32 forward x -> the FP32 spectrum of r - 1 into S (or, without S, into
// S2 as double-float). The half spectra and the observed rows are staged in
// shared memory by asynchronous copies that are all in flight at once, so no
// register holds them across the inverse transform.
template <int L, bool CO>
__device__ __forceinline__ void ddf_x_ratio_tile(const DdXFast& a, long tile, cdd* sm) {
    constexpr int TPL = L / kE8, P = ddf_pairs(L), LS = x_line_stride8(L), XH = L / 2 + 1;
    const int p = threadIdx.x / TPL, t = threadIdx.x - p * TPL;
    const long rho0 = tile * 2 * P;
    const int nrows = (int)min((long)2 * P, a.YZ - rho0);
    const bool oka = p < nrows, okb = P + p < nrows;
    float* phs = reinterpret_cast<float*>(reinterpret_cast<char*>(sm) + ddf_x_smem(L));  // 2P rows of L
    ddf_gather_issue<L>(a, rho0, nrows, sm);
    {
        // the observed rows rho0 .. rho0 + nrows - 1 are contiguous: 2P * L floats
        const float* src = a.phi + rho0 * L;
        for (int c = threadIdx.x; c < 2 * P * L / 4; c += kDdThreads) {
            const bool ok = c * 4 < nrows * L;
            cp_async16(phs + 4 * c, ok ? src + 4 * c : a.phi, ok);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    cdd v[kE8];
    ddf_pair_line<L>(sm, p, t, v);
    __syncthreads();
    LineFFTDD<L, +1, true>::run(v, sm + p * LS, t, a.tw2, 1 + p);
    // r - 1 of both rows as one complex FP32 line, forward x in registers (the
    // double-float inverse leaves the line in the same distribution; its last
    // shared-memory read was followed by a barrier, so the line's shared
    // memory is free)
    float2 f[kE8];
#pragma unroll
    for (int q = 0; q < kE8; ++q) {
        const int n = t + TPL * q;
        // r - 1 = (phi - b') / b' with b' = max(b, eps): the difference is
        // exact where phi and b' are within a factor 2 (Sterbenz), so r - 1
        // keeps its relative precision as r approaches 1; the quotient is the
        // fast division intrinsic (2 ulp, b' far inside its range)
        const float ba = fmaxf(v[q].re.hi + v[q].re.lo, a.eps), bb = fmaxf(v[q].im.hi + v[q].im.lo, a.eps);
        const float xa = oka ? __fdividef(phs[p * L + n] - ba, ba) : 0.f;
        const float xb = okb ? __fdividef(phs[(P + p) * L + n] - bb, bb) : 0.f;
        f[q] = make_float2(xa, xb);
    }
    // each FP32 line lives inside its own line's double-float region (the
    // threads of a line are the only ones touching it until the barrier)
    float2* Fp = reinterpret_cast<float2*>(sm + p * LS);
    LineFFT8F<L, -1, true>::run(f, Fp, t, a.plan.tw, 1 + p);
#pragma unroll
    for (int q = 0; q < kE8; ++q) Fp[pad16(t + TPL * q)] = f[q];
    __syncthreads();
    for (int idx = threadIdx.x; idx < XH * 2 * P; idx += kDdThreads) {
        const int k = idx / (2 * P), row = idx - k * 2 * P;
        if (row >= nrows) continue;
        const int pp = row < P ? row : row - P;
        const float2* F = reinterpret_cast<const float2*>(sm + pp * LS);
        const float2 zk = F[pad16(k)];
        const float2 zm = cconj(F[pad16(k == 0 ? 0 : L - k)]);
        float2 val;
        if (row < P) {
            val = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
        } else {
            const float2 d = csub(zk, zm);
            val = make_float2(0.5f * d.y, -0.5f * d.x);
        }
        if (a.S)
            a.S[(long)k * a.YZ + rho0 + row] = val;
        else
            cdd_store(a.S2 + (long)k * a.YZ + rho0 + row, cdd{dd_from(val.x), dd_from(val.y)});
    }
}

// The back-projection's last pass in precise mode: the double-float half
// spectra of the tile's rows and the rows' current estimate are staged in
// shared memory by asynchronous copies, the inverse x transform runs in
// double-float and gives c - 1, and
//   MODE 1: psi = max(psi . update_factor(c - 1), eps)   (weights, lambda, 1/s)
//   MODE 4: acc = acc . c . inv_s                         (combined update)
// (c - 1 rounded to FP32 once, at the end).
struct DdXUpd {
    const cdd* S2;        // double-float half spectrum S2[kx][rho]
    float* psi;           // estimate (MODE 1) or product (MODE 4), rows of X floats
    long YZ;
    float eps;
    const cdd* tw2;       // double-float twiddles of X
    const float* wt;      // view weights or none
    float lam;            // Tikhonov lambda
    const float* inv_s;   // 1 / sensitivity or none
};

template <int L, int MODE>
__device__ __forceinline__ void ddf_x_update_tile(const DdXUpd& a, long tile, cdd* sm) {
    constexpr int TPL = L / kE8, P = ddf_pairs(L), LS = x_line_stride8(L);
    const int p = threadIdx.x / TPL, t = threadIdx.x - p * TPL;
    const long rho0 = tile * 2 * P;
    const int nrows = (int)min((long)2 * P, a.YZ - rho0);
    const bool oka = p < nrows, okb = P + p < nrows;
    float* ps = reinterpret_cast<float*>(reinterpret_cast<char*>(sm) + ddf_x_smem(L));  // 2P rows
    DdXFast g{};
    g.S2 = const_cast<cdd*>(a.S2);
    g.YZ = a.YZ;
    ddf_gather_issue<L>(g, rho0, nrows, sm);
    {
        const float* src = a.psi + rho0 * L;
        for (int c = threadIdx.x; c < 2 * P * L / 4; c += kDdThreads) {
            const bool ok = c * 4 < nrows * L;
            cp_async16(ps + 4 * c, ok ? src + 4 * c : a.psi, ok);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    cdd v[kE8];
    ddf_pair_line<L>(sm, p, t, v);
    __syncthreads();
    LineFFTDD<L, +1, true>::run(v, sm + p * LS, t, a.tw2, 1 + p);
    const long ra = (rho0 + p) * L, rb = (rho0 + P + p) * L;
#pragma unroll
    for (int q = 0; q < kE8; ++q) {
        const int n = t + TPL * q;
        const float ca = v[q].re.hi + v[q].re.lo, cb = v[q].im.hi + v[q].im.lo;  // c - 1
        const float pa = ps[p * L + n], pb = ps[(P + p) * L + n];
        if (MODE == 1) {
            if (oka) a.psi[ra + n] = fmaxf(pa * update_factor(ca, pa, a.wt, ra + n, a.lam, a.inv_s), a.eps);
            if (okb) a.psi[rb + n] = fmaxf(pb * update_factor(cb, pb, a.wt, rb + n, a.lam, a.inv_s), a.eps);
        } else {
            if (oka) a.psi[ra + n] = pa * (ca + 1.f) * (a.inv_s ? __ldg(a.inv_s + ra + n) : 1.f);
            if (okb) a.psi[rb + n] = pb * (cb + 1.f) * (a.inv_s ? __ldg(a.inv_s + rb + n) : 1.f);
        }
    }
}

}  // namespace mvd
