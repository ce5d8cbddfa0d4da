// Shared internals of the mvd library: error reporting, launch accounting,
// the FFT plan type and the context struct.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "mvd.h"

namespace mvd {

// ---------------------------------------------------------------------------
// errors and accounting
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

extern std::atomic<unsigned long long> g_launches;
inline void count_launch(unsigned n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Optional per-kernel timing (mvd_profile_*): a pair of CUDA events on the
// launching stream around each launch of a given class.
enum KernelClass {
    KC_X_FORWARD = 0,
    KC_Y,
    KC_Z_MUL,
    KC_X_RATIO,
    KC_X_UPDATE,
    KC_DIRECT_RATIO,
    KC_DIRECT_UPDATE,
    KC_DD_X_FORWARD,
    KC_DD_Y,
    KC_DD_Z_MUL,
    KC_DD_X_RATIO,
    KC_SETUP,
    KC_DIRECT_CONV,  // plain direct convolutions (adjoint)
    KC_KERNEL_GRAD,  // kernel-gradient correlations (adjoint)
    KC_COUNT
};
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st);
bool profiling_on();

// Converts the last CUDA error (after a launch) into a status.
mvd_status check_launch(const char* what);
mvd_status cuda_status(cudaError_t e, const char* what);

#define MVD_TRY(expr)                          \
    do {                                       \
        mvd_status _st = (expr);               \
        if (_st != MVD_OK) return _st;         \
    } while (0)

#define MVD_CUDA(call)                                           \
    do {                                                         \
        cudaError_t _e = (call);                                 \
        if (_e != cudaSuccess) return ::mvd::cuda_status(_e, #call); \
    } while (0)

// ---------------------------------------------------------------------------
// FFT plan: one line length L = prod(radix[s]); tw[m] = exp(-2 pi i m / L)
// (device table, computed in FP64 on the host and rounded to FP32).
// ---------------------------------------------------------------------------
constexpr int kMaxStages = 16;

struct FftPlan {
    int L;
    int nst;
    int radix[kMaxStages];
    const float2* tw;
};

// Radix plan for a {2,3,5}-smooth length; false if L has another prime factor.
// dd: the plan also drives double-float passes (no radix 10 there).
bool make_radix_plan(int L, FftPlan* p, bool dd);

// ---------------------------------------------------------------------------
// kernel launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
struct cdd;  // complex double-float (dd.cuh)

struct FftGeom {
    int X, Y, Z, Xh;
    long YZ;
    FftPlan px, py, pz;
    bool fast;                       // use the register-resident kernels where the length allows
    const cdd *tw2x, *tw2y, *tw2z;  // double-float twiddle tables (precise forward blur)
};

// Spectrum layout: S[kx][z][y] (y fastest), kx in [0, Xh), Xh = X/2 + 1.
mvd_status fft_forward_real(const FftGeom& g, const float* src, float2* S, cudaStream_t st);
mvd_status fft_y(const FftGeom& g, float2* S, int inverse, cudaStream_t st);
mvd_status fft_z_mul(const FftGeom& g, float2* S, const float2* K, cudaStream_t st);
mvd_status fft_z_forward_scaled(const FftGeom& g, float2* S, float scale, cudaStream_t st);
mvd_status fft_x_ratio(const FftGeom& g, float2* S, const float* phi, float eps, cudaStream_t st);
mvd_status fft_x_update(const FftGeom& g, const float2* S, float* psi, float eps, cudaStream_t st,
                        const float* wt = nullptr, float lam = 0.f,
                        const float* inv_s = nullptr);  // weights of the change, Tikhonov lambda, 1 / sensitivity
mvd_status fft_inverse_real(const FftGeom& g, const float2* S, float* dst, cudaStream_t st);
// inverse x of a double-float spectrum to real (after the y and z passes)
mvd_status fft_x_inverse_dd(const FftGeom& g, const cdd* S2, float* dst, cudaStream_t st);
// combined update: acc *= c, c the back-projected factor of the spectrum of (r - 1) * K (+ 1)
mvd_status fft_x_accumulate(const FftGeom& g, const float2* S, float* acc, cudaStream_t st,
                            const float* inv_s = nullptr);
mvd_status fft_x_accumulate_generic(const FftGeom& g, const float2* S, float* acc, cudaStream_t st,
                                    const float* inv_s = nullptr);
mvd_status fft_x_accumulate_fast(const FftGeom& g, const float2* S, float* acc, cudaStream_t st,
                                 const float* inv_s = nullptr);

// double-float forward blur (fft_dd.cu): spectrum of complex double-float
mvd_status dd_forward_real(const FftGeom& g, const float* src, cdd* S2, cudaStream_t st);
mvd_status dd_y(const FftGeom& g, cdd* S2, int inverse, cudaStream_t st);
// register-resident x and y lengths: the back-projection's forward y pass can
// take the ratio pass's FP32 spectrum of r - 1 (exact FP32 values) into S2
bool dd_fast_yx(const FftGeom& g);
mvd_status dd_y_from_f32(const FftGeom& g, const float2* S1, cdd* S2, cudaStream_t st);
// the double-float x inverse of S2 to real rows (rounded to FP32), generic lengths
mvd_status dd_x_inverse_real_generic(const FftGeom& g, const cdd* S2, float* dst, cudaStream_t st);
// the double-float x inverse of S2 -> the update of psi (accumulate: the combined
// update's product), any smooth length
mvd_status dd_x_update(const FftGeom& g, const cdd* S2, float* psi, float eps, cudaStream_t st, const float* wt,
                       float lam, const float* inv_s, int accumulate);
mvd_status dd_x_update_generic(const FftGeom& g, const cdd* S2, float* psi, float eps, cudaStream_t st,
                               const float* wt, float lam, const float* inv_s, int accumulate);

mvd_status dd_z_mul(const FftGeom& g, cdd* S2, const cdd* K2, cudaStream_t st);
mvd_status dd_z_forward_scaled(const FftGeom& g, cdd* S2, double scale, cudaStream_t st);
// the inverse x of b (double-float) -> r - 1 -> FP32 forward x, written to the
// FP32 spectrum S when given, else exactly into S2
mvd_status dd_x_ratio(const FftGeom& g, cdd* S2, const float* phi, float eps, cudaStream_t st, float2* S = nullptr);
// double-float spectrum -> real volume (x inverse, rounded to FP32); X of 32..1024, a power of two
mvd_status dd_x_inverse_real(const FftGeom& g, const cdd* S2, float* dst, cudaStream_t st);
bool dd_fast_x(const FftGeom& g);
// update pass reading the double-float spectrum (rounded to FP32)

// register-resident variants for power-of-two lengths (fft_fast.cu)
bool fft_fast_supported(int L);
bool fft_fast_z_supported(int L);
mvd_status fft_forward_real_fast(const FftGeom& g, const float* src, float2* S, cudaStream_t st);
mvd_status fft_y_fast(const FftGeom& g, float2* S, int inverse, cudaStream_t st);
mvd_status fft_z_mul_fast(const FftGeom& g, float2* S, const float2* K, cudaStream_t st);
mvd_status fft_z_forward_scaled_fast(const FftGeom& g, float2* S, float scale, cudaStream_t st);
mvd_status fft_x_ratio_fast(const FftGeom& g, float2* S, const float* phi, float eps, cudaStream_t st);
mvd_status fft_x_update_fast(const FftGeom& g, const float2* S, float* psi, float eps, cudaStream_t st,
                             const float* wt = nullptr, float lam = 0.f, const float* inv_s = nullptr);
mvd_status fft_inverse_real_fast(const FftGeom& g, const float2* S, float* dst, cudaStream_t st);

// Direct (spatial) periodic convolution with fused epilogues.
bool direct_supported(const int kd[3]);
// ty = output tile height (8, 4, 2 or 1 rows of 32 x 4 outputs); 0 = the
// largest whose staging fits in shared memory
mvd_status direct_ratio(const int dims[3], const float* psi, const float* k, const int kd[3],
                        const float* phi, float eps, float* r, cudaStream_t st, int ty = 0);
mvd_status direct_update(const int dims[3], const float* r, const float* k, const int kd[3],
                         float* psi, float eps, cudaStream_t st, int ty = 0, const float* wt = nullptr,
                         float lam = 0.f, const float* inv_s = nullptr);
int direct_tile_heights(const int kd[3], int out[4]);  // tile heights that fit, largest first
// prod *= r * k (the combined update's product of view factors)
mvd_status direct_accumulate(const int dims[3], const float* r, const float* k, const int kd[3], float* prod,
                             cudaStream_t st, int ty = 0, const float* inv_s = nullptr);
mvd_status direct_conv(const int dims[3], const float* in, const float* k, const int kd[3],
                       float* out, cudaStream_t st);

// Compound-kernel precompute and helpers.
// compound kernel of view v into d_out; for MVD_EFFICIENT d_q holds Q_w = P_w * P_w^*
// of every view w (autocorr_all) at stride qstride
mvd_status build_compound(int n_views, const float* d_psf, const long* koff_h, const int* kd_h, int v,
                          int variant, float* d_out, const float* d_q, long qstride, cudaStream_t st);
mvd_status autocorr_all(int n_views, const float* d_psf, const long* koff_h, const int* kd_h, float* d_q,
                        long qstride, cudaStream_t st);
mvd_status normalize_kernel(float* d_k, int n, int* d_bad, cudaStream_t st);
mvd_status mirror_kernel(const float* k, const int kd[3], float* out, cudaStream_t st);
mvd_status autocorr_kernel(const float* P, const int kd[3], float* Q, cudaStream_t st);  // Q box = 2K-1
mvd_status direct_conv_add(const int dims[3], const float* in, const float* k, const int kd[3], float* out,
                           cudaStream_t st);
mvd_status one_update(mvd_ctx* c, int v);
// zero / mirror boundary (boundary.cu)
mvd_status pad_volume(const mvd_ctx* c, const float* user, float* padded, cudaStream_t st);
mvd_status crop_volume(const mvd_ctx* c, const float* padded, float* user, cudaStream_t st);
mvd_status clear_padding(const mvd_ctx* c, float* padded, cudaStream_t st);
// mirror: the halo holds the reflection of the volume, the rest of the padding 0
mvd_status mirror_fill(const mvd_ctx* c, float* padded, cudaStream_t st);
// mirror: psi = max(psi . fold(cp + off) . inv_s, eps) inside, reflection refreshed;
// cp is the back-projection on the padded grid (minus off)
mvd_status mirror_update(const mvd_ctx* c, const float* cp, float off, const float* inv_s, cudaStream_t st,
                         const float* wt = nullptr, float lam = 0.f);
// combined update with the mirror boundary: prod *= fold(cp + off) / s_v on the user's voxels
mvd_status mirror_accumulate(const mvd_ctx* c, const float* cp, float off, const float* inv_s, float* prod,
                             cudaStream_t st);
// the estimate's padding after it was written inside: zeroed or reflected
mvd_status finish_padding(const mvd_ctx* c, float* padded, cudaStream_t st);
mvd_status compute_inverse_sensitivity(mvd_ctx* c);
// view v's pass from the current estimate: with prod == nullptr the
// sequential update psi = max(psi . c_v, eps); else prod *= c_v
mvd_status view_pass(mvd_ctx* c, int v, float* prod);
mvd_status place_kernel(const int dims[3], const float* k, const int kd[3], float* vol,
                        cudaStream_t st);
mvd_status view_stats(const float* views, long n, double* d_sum, int* d_bad, cudaStream_t st);
mvd_status fill(float* p, long n, float v, cudaStream_t st);
mvd_status apply_product(float* psi, const float* prod, long n, float e, float eps, cudaStream_t st);
// partial overlap weights: range check, overlap counts, per-voxel normalisation
mvd_status weights_check(const float* w, long n, int* d_bad, cudaStream_t st);
mvd_status weights_overlap(const float* w, int nv, long M, unsigned long long* d_stats, int* d_min, cudaStream_t st);
mvd_status weights_normalize(float* w, int nv, long M, float T, cudaStream_t st);
mvd_status check_positive(const float* p, long n, int* d_bad, cudaStream_t st);

}  // namespace mvd

// ---------------------------------------------------------------------------
// the context
// ---------------------------------------------------------------------------
struct mvd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int dims[3] = {0, 0, 0};
    long M = 0;
    int nv = 0;
    std::vector<int> kd;     // 3 per view
    std::vector<long> koff;  // offset of each view's box in the packed kernel arrays
    long ktotal = 0;

    float* d_views = nullptr;  // nv * M
    float* d_psi = nullptr;    // M
    float* d_r = nullptr;      // M (direct-path ratio; scratch for kernel placement)
    float* d_psf = nullptr;    // packed normalised PSFs
    float* d_comp = nullptr;   // packed compound kernels
    float* d_ktmp = nullptr;   // precompute scratch
    double* d_red = nullptr;   // reduction scratch
    int* d_flag = nullptr;

    // FFT engine
    mvd::FftGeom geom{};
    int precise = 1;         // 1 MVD_PRECISE, 2 MVD_MIXED (double-float forward blur), 0 MVD_FAST
    float2* d_tw = nullptr;  // twiddle tables (x, y, z)
    float2* d_S = nullptr;   // work spectrum Xh*Y*Z
    // kernel spectra, each Xh*Y*Z, slot 2v = P_v and 2v+1 = P_v^comp: FP32
    // in fast mode (d_K), double-float in precise and mixed mode (d_KP2);
    // mixed mode also keeps P_v^comp in FP32 for its back-projection, slot v
    // of d_K
    float2* d_K = nullptr;
    mvd::cdd* d_tw2 = nullptr;  // double-float twiddle tables (x, y, z)
    mvd::cdd* d_S2 = nullptr;   // double-float work spectrum (precise mode)
    mvd::cdd* d_KP2 = nullptr;  // 2*nv double-float kernel spectra (precise mode)

    // one instantiated graph per schedule (one iteration each)
    struct Graph {
        cudaGraphExec_t exec;
        unsigned nodes;
    };
    std::map<std::vector<int>, Graph> graphs;

    // unrolled iteration for differentiation: psi at the start of every
    // iteration, then psi_K (n_iter + 1 volumes)
    float* d_ckpt = nullptr;
    long ckpt_iters = -1;
    int ckpt_flat = 0;           // the unrolled run started from the flat estimate
    std::vector<double> psf_sum;  // sums of the raw PSFs (normalisation)

    int state = 0;  // 1 created, 2 kernels precomputed
    int variant = -1;
    int path_opt = MVD_PATH_AUTO;
    int direct_ty = 0;  // direct-engine tile height chosen by the autotuner (0 = default)
    float* d_prod = nullptr;  // combined update: product of the view factors (M)
    float* d_w = nullptr;     // partial overlap: normalised weights of every view (nv * M), or none
    float weight_norm = 0.f;  // the normalisation target T of the weights
    float lambda = 0.f;       // Tikhonov regularisation of the sequential update (0 = none)

    // zero / mirror boundary: the engines run on a padded grid (dims, M); the
    // user's volume (udims, uM) sits in its low corner; halo = largest PSF
    // half-width per axis (the mirror boundary keeps psi's reflection there)
    int boundary = 0;                 // mvd_boundary
    int udims[3] = {0, 0, 0};
    int halo[3] = {0, 0, 0};
    long uM = 0;
    float* d_invs = nullptr;  // 1 / sensitivity per view (nv padded volumes)
    float* d_stage = nullptr; // user-layout staging volume (uM)
    float* d_bp = nullptr;    // mirror boundary, combined update: the back-projection (d_prod holds the product)
    int path = MVD_PATH_AUTO;
    float psi0 = 0.f, eps = 0.f;
    bool eps_user = false;  // eps given at create (else 1e-4 psi0 of the current views)
    bool views_ok = true;   // false after mvd_set_views rejected its input
};
