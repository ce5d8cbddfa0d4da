// C ABI of the mvd library (declared in include/mvd.h): context life cycle,
// precompute, the sequential update loop and result access.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "dd.cuh"

namespace mvd {

std::atomic<unsigned long long> g_launches{0};
static thread_local std::string t_err;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
}

void clear_error() { t_err.clear(); }

mvd_status cuda_status(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MVD_ERR_OOM : MVD_ERR_CUDA;
}

mvd_status check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, what);
    return MVD_OK;
}

// ---------------------------------------------------------------------------
// per-kernel event timing
// ---------------------------------------------------------------------------
namespace {

struct ProfRec {
    int cls;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
std::atomic<int> g_prof_on{0};
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_pool;
size_t g_pool_used = 0;
thread_local int t_open_cls = -1;
thread_local cudaEvent_t t_open_ev = nullptr;
const char* kClassNames[KC_COUNT] = {"x_forward", "y",        "z_mul",        "x_ratio",
                                     "x_update",  "direct_ratio", "direct_update", "dd_x_forward",
                                     "dd_y",      "dd_z_mul", "dd_x_ratio",   "setup",
                                     "direct_conv", "kernel_grad"};

cudaEvent_t next_event() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_pool_used == g_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        g_pool.push_back(e);
    }
    return g_pool[g_pool_used++];
}
}  // namespace

bool profiling_on() { return g_prof_on.load(std::memory_order_relaxed) != 0; }

void prof_begin(int cls, cudaStream_t st) {
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    cudaEvent_t e = next_event();
    if (!e || cudaEventRecord(e, st) != cudaSuccess) return;
    t_open_cls = cls;
    t_open_ev = e;
}

void prof_end(int cls, cudaStream_t st) {
    if (!g_prof_on.load(std::memory_order_relaxed) || t_open_cls != cls) return;
    t_open_cls = -1;
    cudaEvent_t e = next_event();
    if (!e || cudaEventRecord(e, st) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back({cls, t_open_ev, e});
}

namespace {

// Rough cost per point of one Stockham stage of radix R in double-float
// operations: the small DFT, the twiddle products of (R-1)/R of the points
// (none in the first stage) and the shared-memory round trip.
double stage_cost(int R, bool first) {
    double dft;
    switch (R) {
        case 2: dft = 16; break;
        case 3: dft = 41; break;
        case 4: dft = 32; break;
        case 5: dft = 74; break;
        case 6: dft = 57; break;
        case 8: dft = 52; break;
        case 9: dft = 99; break;
        default: dft = 90; break;  // 10
    }
    return dft + (first ? 0.0 : 38.0 * (R - 1) / R) + 40.0;
}

// cheapest factorisation of n into the allowed radices <= max_r (bit R of
// `allowed`), in non-increasing order
void best_plan(int n, int max_r, unsigned allowed, std::vector<int>& cur, double cost, std::vector<int>& best,
               double& best_cost) {
    if (n == 1) {
        if (cost < best_cost) best_cost = cost, best = cur;
        return;
    }
    static const int kRadices[] = {10, 9, 8, 6, 5, 4, 3, 2};
    for (int R : kRadices) {
        if (R > max_r || !(allowed >> R & 1u) || n % R != 0 || (int)cur.size() >= kMaxStages) continue;
        const double c = cost + stage_cost(R, cur.empty());
        if (c >= best_cost) continue;
        cur.push_back(R);
        best_plan(n / R, R, allowed, cur, c, best, best_cost);
        cur.pop_back();
    }
}

}  // namespace

bool make_radix_plan(int L, FftPlan* p, bool dd) {
    p->L = L;
    p->nst = 0;
    int n = L, a = 0;
    while (n % 2 == 0) n /= 2, ++a;
    while (n % 3 == 0) n /= 3;
    while (n % 5 == 0) n /= 5;
    if (n != 1 || L < 1) return false;
    auto push = [&](int r) {
        if (p->nst < kMaxStages) p->radix[p->nst++] = r;
    };
    if (L == (1 << a)) {  // powers of two: radix 8, then 4 4 or 4 or 2 for the rest
        const int q = a / 3, rem = a % 3;
        if (rem == 0) {
            for (int i = 0; i < q; ++i) push(8);
        } else if (rem == 1) {
            if (q >= 1) {
                for (int i = 0; i < q - 1; ++i) push(8);
                push(4);
                push(4);
            } else {
                push(2);
            }
        } else {
            for (int i = 0; i < q; ++i) push(8);
            push(4);
        }
        return true;
    }
    // mixed lengths: the cheapest product of radices 2..10 (composite 6, 9, 10
    // cut the number of stages), the largest radix first (it has no twiddles);
    // without 10 where double-float passes run (their registers)
    std::vector<int> cur, best;
    double best_cost = 1e300;
    const unsigned allowed = (1u << 2) | (1u << 3) | (1u << 4) | (1u << 5) | (1u << 6) | (1u << 8) | (1u << 9) |
                             (dd ? 0u : (1u << 10));
    best_plan(L, 10, allowed, cur, 0.0, best, best_cost);
    if (best.empty()) return false;
    for (int r : best) push(r);
    return true;
}

}  // namespace mvd

using namespace mvd;

namespace {

// Stage order of the twiddles of a line transform whose stages have the
// radices radix[0..n-1]: stage s >= 1, with NS points combined before it and
// radix R, needs w^m for m = r k L / (NS R) (r = 1..R-1, k = 0..NS-1);
// put(i, m) stores it at i = (earlier stages' entries) + (r - 1) NS + k, so
// that consecutive butterflies (consecutive k) read consecutive entries.
template <typename F>
void stage_ordered_twiddles(int L, const std::vector<int>& radix, F&& put) {
    int ns = 1;
    size_t off = 0;
    for (size_t st = 0; st < radix.size(); ++st) {
        const int R = radix[st];
        if (st > 0) {
            for (int r = 1; r < R; ++r)
                for (int k = 0; k < ns; ++k) put(off + (size_t)(r - 1) * ns + k, (long)r * k * (L / (ns * R)));
            off += (size_t)(R - 1) * ns;
        }
        ns *= R;
    }
}

// the register-resident lines' plan: radix P stages, then L's remainder
std::vector<int> pow_plan(int L, int P) {
    std::vector<int> radix;
    int rem = L;
    while (rem % P == 0 && rem >= P) {
        radix.push_back(P);
        rem /= P;
    }
    if (rem > 1) radix.push_back(rem);
    return radix;
}

std::vector<int> plan_radices(const FftPlan& p) { return std::vector<int>(p.radix, p.radix + p.nst); }


struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
mvd_status dev_alloc(T** p, size_t count, const char* what) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error("allocating %s (%zu bytes): %s", what, count * sizeof(T), cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MVD_ERR_OOM : MVD_ERR_CUDA;
    }
    return MVD_OK;
}

template <typename T>
void dev_free(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void drop_graphs(mvd_ctx* c) {
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
}

void free_fft(mvd_ctx* c) {
    drop_graphs(c);
    dev_free(c->d_tw);
    dev_free(c->d_S);
    dev_free(c->d_K);
    dev_free(c->d_tw2);
    dev_free(c->d_S2);
    dev_free(c->d_KP2);
}

void free_all(mvd_ctx* c) {
    drop_graphs(c);
    dev_free(c->d_ckpt);
    dev_free(c->d_prod);
    dev_free(c->d_w);
    free_fft(c);
    dev_free(c->d_views);
    dev_free(c->d_psi);
    dev_free(c->d_r);
    dev_free(c->d_psf);
    dev_free(c->d_comp);
    dev_free(c->d_ktmp);
    dev_free(c->d_red);
    dev_free(c->d_flag);
    dev_free(c->d_invs);
    dev_free(c->d_stage);
    dev_free(c->d_bp);
}

bool smooth235(int n) {
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

// Relative cost of the two engines for one view update (seconds, rough):
// direct = 2T FMAs per voxel on the FP32 pipe; FFT = ~88 bytes per voxel over
// HBM plus nine launches. Used when the path is AUTO.
int choose_path(const mvd_ctx* c) {
    bool direct_ok = true;
    long tmax = 0;
    for (int v = 0; v < c->nv; ++v) {
        direct_ok = direct_ok && direct_supported(&c->kd[3 * v]);
        tmax = std::max(tmax, (long)c->kd[3 * v] * c->kd[3 * v + 1] * c->kd[3 * v + 2]);
    }
    const bool fft_ok = smooth235(c->dims[0]) && smooth235(c->dims[1]) && smooth235(c->dims[2]);
    if (!fft_ok) return direct_ok ? MVD_PATH_DIRECT : -1;
    if (!direct_ok) return MVD_PATH_FFT;
    const double t_direct = 2.0 * tmax * (double)c->M / 40e12 + 2 * 3e-6;
    const double t_fft = 88.0 * (double)c->M / 5e12 + 9 * 3e-6;
    return t_direct <= t_fft ? MVD_PATH_DIRECT : MVD_PATH_FFT;
}

mvd_status setup_fft(mvd_ctx* c) {
    FftGeom& g = c->geom;
    g.X = c->dims[0];
    g.Y = c->dims[1];
    g.Z = c->dims[2];
    g.Xh = g.X / 2 + 1;
    g.YZ = (long)g.Y * g.Z;
    // MVD_FFT_GENERIC=1 forces the generic kernels (used to test both engines)
    const char* gen = std::getenv("MVD_FFT_GENERIC");
    g.fast = !(gen && gen[0] == '1');
    if (!make_radix_plan(g.X, &g.px, c->precise) || !make_radix_plan(g.Y, &g.py, c->precise) ||
        !make_radix_plan(g.Z, &g.pz, c->precise)) {
        set_error("FFT engine needs {2,3,5}-smooth dims, got %d x %d x %d", g.X, g.Y, g.Z);
        return MVD_ERR_UNSUPPORTED;
    }
    const int Ls[3] = {g.X, g.Y, g.Z};
    // FP32 twiddles w^m = exp(-2 pi i m / L), per axis: the natural table
    // (m = 0..L-1), then the same values in the stage order of the
    // register-resident lines of a power-of-two L, for their radix-8 plan
    // (8 points per thread) and their radix-16 plan (16 points per thread),
    // then in the stage order of the axis's mixed-radix plan
    const FftPlan* plans[3] = {&g.px, &g.py, &g.pz};
    std::vector<float2> tw(4 * ((size_t)g.X + g.Y + g.Z), make_float2(0.f, 0.f));
    size_t off = 0;
    for (int a = 0; a < 3; ++a) {
        const int L = Ls[a];
        auto w32 = [L](long m) {
            const double ang = -2.0 * M_PI * (double)m / (double)L;
            return make_float2((float)std::cos(ang), (float)std::sin(ang));
        };
        for (int m = 0; m < L; ++m) tw[off + m] = w32(m);
        if (L >= 16 && L <= 4096 && (L & (L - 1)) == 0) {
            stage_ordered_twiddles(L, pow_plan(L, 8), [&](size_t i, long m) { tw[off + L + i] = w32(m); });
            stage_ordered_twiddles(L, pow_plan(L, 16), [&](size_t i, long m) { tw[off + 2 * (size_t)L + i] = w32(m); });
        }
        stage_ordered_twiddles(L, plan_radices(*plans[a]), [&](size_t i, long m) { tw[off + 3 * (size_t)L + i] = w32(m); });
        off += 4 * (size_t)L;
    }
    MVD_TRY(dev_alloc(&c->d_tw, tw.size(), "twiddle tables"));
    MVD_CUDA(cudaMemcpyAsync(c->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream));
    g.px.tw = c->d_tw;
    g.py.tw = c->d_tw + 4 * g.X;
    g.pz.tw = c->d_tw + 4 * (g.X + g.Y);
    const size_t ns = (size_t)g.Xh * g.YZ;
    MVD_TRY(dev_alloc(&c->d_S, ns, "work spectrum"));
    if (c->precise != 1) MVD_TRY(dev_alloc(&c->d_K, ns * (c->precise ? 1 : 2) * c->nv, "kernel spectra"));
    const float inv_m = (float)(1.0 / (double)c->M);
    if (c->precise) {
        // double-float twiddles w^m = exp(-2 pi i m / L): hi = fl32(w), lo =
        // fl32(w - hi), w in FP64. Per axis the table in natural order (m =
        // 0..L-1), then, for the register-resident passes of a power-of-two L,
        // the same values in the stage order of their radix-8 plan, then in
        // the stage order of the axis's mixed-radix plan.
        auto twv = [](long m, int L) {
            const double ang = -2.0 * M_PI * (double)m / (double)L;
            const double cr = std::cos(ang), ci = std::sin(ang);
            const float rh = (float)cr, ih = (float)ci;
            return make_float4(rh, (float)(cr - rh), ih, (float)(ci - ih));
        };
        std::vector<float4> tw2(3 * ((size_t)g.X + g.Y + g.Z), make_float4(0.f, 0.f, 0.f, 0.f));
        size_t o = 0;
        for (int a = 0; a < 3; ++a) {
            const int L = Ls[a];
            for (int m = 0; m < L; ++m) tw2[o + m] = twv(m, L);
            if (L >= 32 && L <= 1024 && (L & (L - 1)) == 0)
                stage_ordered_twiddles(L, pow_plan(L, 8), [&](size_t i, long m) { tw2[o + L + i] = twv(m, L); });
            stage_ordered_twiddles(L, plan_radices(*plans[a]),
                                   [&](size_t i, long m) { tw2[o + 2 * (size_t)L + i] = twv(m, L); });
            o += 3 * (size_t)L;
        }
        MVD_TRY(dev_alloc(reinterpret_cast<float4**>(&c->d_tw2), tw2.size(), "double-float twiddle tables"));
        MVD_CUDA(cudaMemcpyAsync(c->d_tw2, tw2.data(), tw2.size() * sizeof(float4), cudaMemcpyHostToDevice,
                                 c->stream));
        g.tw2x = c->d_tw2;
        g.tw2y = reinterpret_cast<const cdd*>(reinterpret_cast<const float4*>(c->d_tw2) + 3 * g.X);
        g.tw2z = reinterpret_cast<const cdd*>(reinterpret_cast<const float4*>(c->d_tw2) + 3 * (g.X + g.Y));
        MVD_TRY(dev_alloc(reinterpret_cast<float4**>(&c->d_S2), ns, "double-float work spectrum"));
        MVD_TRY(dev_alloc(reinterpret_cast<float4**>(&c->d_KP2), ns * 2 * c->nv, "double-float kernel spectra"));
    }
    // kernel spectra, scaled by 1/M: slot 2v = P_v, 2v+1 = P_v^comp (FP32 in
    // fast mode, double-float in precise and mixed mode, plus P_v^comp in FP32
    // in mixed mode)
    for (int v = 0; v < c->nv; ++v) {
        for (int which = 0; which < 2; ++which) {
            const float* k = (which == 0 ? c->d_psf : c->d_comp) + c->koff[v];
            MVD_TRY(place_kernel(c->dims, k, &c->kd[3 * v], c->d_r, c->stream));
            if (c->precise) {
                cdd* dst = reinterpret_cast<cdd*>(reinterpret_cast<float4*>(c->d_KP2) + ns * (2 * v + which));
                MVD_TRY(dd_forward_real(g, c->d_r, dst, c->stream));
                MVD_TRY(dd_y(g, dst, 0, c->stream));
                MVD_TRY(dd_z_forward_scaled(g, dst, 1.0 / (double)c->M, c->stream));
                if (which == 0 || c->precise == 1) continue;
            }
            float2* dst = c->d_K + ns * (c->precise ? v : 2 * v + which);
            MVD_TRY(fft_forward_real(g, c->d_r, dst, c->stream));
            MVD_TRY(fft_y(g, dst, 0, c->stream));
            MVD_TRY(fft_z_forward_scaled(g, dst, inv_m, c->stream));
        }
    }
    return MVD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// autotuner (engine and tile choice per problem shape, timed on the context's
// own data, persisted in a text cache)
// ---------------------------------------------------------------------------
namespace {

struct TuneChoice {
    int path = MVD_PATH_FFT;
    int ty = 0;
    int fast = 1;
    double ms = 0.0;
};

std::string tune_key(const mvd_ctx* c) {
    std::string k = "mvd-tune-v1 dims " + std::to_string(c->dims[0]) + " " + std::to_string(c->dims[1]) + " " +
                    std::to_string(c->dims[2]) + " precision " + std::to_string(c->precise == 1 ? MVD_PRECISE : c->precise == 2 ? MVD_MIXED : MVD_FAST) + " boxes";
    for (int v = 0; v < c->nv; ++v)
        for (int a = 0; a < 3; ++a) k += " " + std::to_string(c->kd[3 * v + a]);
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
        std::string name = prop.name;
        for (char& ch : name)
            if (ch == ' ' || ch == '|') ch = '_';
        k += " gpu " + name + " sms " + std::to_string(prop.multiProcessorCount);
    }
    return k;
}

// cache line: "<key> | <path> <tile height> <fast> <ms per update>"
bool tune_lookup(const char* path, const std::string& key, TuneChoice* out) {
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[4096];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        const char* bar = std::strchr(line, '|');
        if (!bar) continue;
        std::string k(line, bar - line);
        while (!k.empty() && k.back() == ' ') k.pop_back();
        if (k != key) continue;
        TuneChoice t;
        if (std::sscanf(bar + 1, "%d %d %d %lf", &t.path, &t.ty, &t.fast, &t.ms) != 4) continue;
        if (t.path != MVD_PATH_DIRECT && t.path != MVD_PATH_FFT) continue;
        *out = t;  // the last valid entry wins
        found = true;
    }
    std::fclose(f);
    return found;
}

void tune_store(const char* path, const std::string& key, const TuneChoice& t) {
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s | %d %d %d %.6f\n", key.c_str(), t.path, t.ty, t.fast, t.ms);
    std::fclose(f);
}

void apply_choice(mvd_ctx* c, const TuneChoice& t) {
    drop_graphs(c);
    c->path = t.path;
    c->direct_ty = t.path == MVD_PATH_DIRECT ? t.ty : 0;
    c->geom.fast = t.fast != 0;
}

// milliseconds per view update of the configuration now set on c: one warm
// update, then one pass over all views; the estimate is restored afterwards
mvd_status time_updates(mvd_ctx* c, float* psi_save, double cutoff_ms, double* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MVD_CUDA(cudaEventCreate(&e0));
    MVD_CUDA(cudaEventCreate(&e1));
    mvd_status st = MVD_OK;
    float t_warm = 0.f, t_all = 0.f;
    do {
        if (cudaEventRecord(e0, c->stream) != cudaSuccess) { st = MVD_ERR_CUDA; break; }
        if ((st = one_update(c, 0)) != MVD_OK) break;
        if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            st = MVD_ERR_CUDA;
            break;
        }
        cudaEventElapsedTime(&t_warm, e0, e1);
        if (cutoff_ms > 0 && t_warm > 4.0 * cutoff_ms) {  // far slower than the best so far: skip the timed pass
            *ms = t_warm;
            break;
        }
        cudaEventRecord(e0, c->stream);
        for (int v = 0; v < c->nv && st == MVD_OK; ++v) st = one_update(c, v);
        if (st != MVD_OK) break;
        if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            st = MVD_ERR_CUDA;
            break;
        }
        cudaEventElapsedTime(&t_all, e0, e1);
        *ms = t_all / c->nv;
    } while (false);
    if (st == MVD_ERR_CUDA) set_error("autotune: timing failed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = cudaMemcpyAsync(c->d_psi, psi_save, sizeof(float) * c->M, cudaMemcpyDeviceToDevice, c->stream);
    if (st == MVD_OK && e != cudaSuccess) st = cuda_status(e, "autotune: restore estimate");
    return st;
}

}  // namespace

mvd_status mvd::one_update(mvd_ctx* c, int v) { return view_pass(c, v, nullptr); }

mvd_status mvd::view_pass(mvd_ctx* c, int v, float* prod) {
    const float* phi = c->d_views + (size_t)v * c->M;
    const int* kd = &c->kd[3 * v];
    const float* wt = c->d_w ? c->d_w + (size_t)v * c->M : nullptr;  // partial overlap (sequential update only)
    const float* inv_s = c->d_invs ? c->d_invs + (size_t)v * c->M : nullptr;  // zero / mirror boundary
    // the update leaves max(0 * c, eps) in a zero boundary's padding: clear it
    auto done = [&](mvd_status st) {
        return st == MVD_OK && !prod && c->boundary == MVD_BOUNDARY_ZERO ? clear_padding(c, c->d_psi, c->stream)
                                                                          : st;
    };
    // mirror boundary: the back-projection goes to c->d_prod (FFT engines:
    // minus 1, the transform of r - 1), then the fold and the update
    const bool mirror = c->boundary == MVD_BOUNDARY_MIRROR;
    if (c->path == MVD_PATH_DIRECT) {
        MVD_TRY(direct_ratio(c->dims, c->d_psi, c->d_psf + c->koff[v], kd, phi, c->eps, c->d_r, c->stream,
                             c->direct_ty));
        if (mirror) {
            float* bp = prod ? c->d_bp : c->d_prod;
            MVD_TRY(direct_conv(c->dims, c->d_r, c->d_comp + c->koff[v], kd, bp, c->stream));
            if (prod) return mirror_accumulate(c, bp, 0.f, inv_s, prod, c->stream);
            return mirror_update(c, bp, 0.f, inv_s, c->stream, wt, c->lambda);
        }
        if (prod)
            return direct_accumulate(c->dims, c->d_r, c->d_comp + c->koff[v], kd, prod, c->stream, c->direct_ty,
                                     inv_s);
        return done(direct_update(c->dims, c->d_r, c->d_comp + c->koff[v], kd, c->d_psi, c->eps, c->stream,
                                  c->direct_ty, wt, c->lambda, inv_s));
    }
    const FftGeom& g = c->geom;
    const size_t ns = (size_t)g.Xh * g.YZ;
    if (c->precise) {
        cdd* S2 = c->d_S2;
        const float4* K4 = reinterpret_cast<const float4*>(c->d_KP2);
        const cdd* Kp2 = reinterpret_cast<const cdd*>(K4 + ns * (2 * v));
        MVD_TRY(dd_forward_real(g, c->d_psi, S2, c->stream));
        MVD_TRY(dd_y(g, S2, 0, c->stream));
        MVD_TRY(dd_z_mul(g, S2, Kp2, c->stream));
        MVD_TRY(dd_y(g, S2, 1, c->stream));
        if (c->precise == 2) {
            // MVD_MIXED: the ratio pass hands r - 1 over as an FP32 spectrum
            // and the back-projection runs in FP32
            MVD_TRY(dd_x_ratio(g, S2, phi, c->eps, c->stream, c->d_S));
        } else {
            // MVD_PRECISE: the back-projection's y, z and x-inverse passes run
            // in double-float, so no rounding of a large |r - 1| (a count where
            // b is near eps) spreads over the volume at FP32 level.
            const cdd* Kc2 = reinterpret_cast<const cdd*>(K4 + ns * (2 * v + 1));
            // The ratio pass hands r - 1 over as an FP32 spectrum when the
            // forward y pass can widen it (exact FP32 values, half the bytes);
            // every transform after it runs in double-float, the update's x
            // inverse included: an FP32 x inverse there carries the rounding
            // of a line's large values (where b is near eps) into the whole
            // line and left up to 1.4e-4 after 15 iterations on volumes of
            // the 48-volume batch (double-float: <= 2.6e-5).
            if (dd_fast_yx(g)) {
                MVD_TRY(dd_x_ratio(g, S2, phi, c->eps, c->stream, c->d_S));
                MVD_TRY(dd_y_from_f32(g, c->d_S, S2, c->stream));
            } else {
                MVD_TRY(dd_x_ratio(g, S2, phi, c->eps, c->stream));
                MVD_TRY(dd_y(g, S2, 0, c->stream));
            }
            MVD_TRY(dd_z_mul(g, S2, Kc2, c->stream));
            MVD_TRY(dd_y(g, S2, 1, c->stream));
            if (mirror) {
                float* bp = prod ? c->d_bp : c->d_prod;
                MVD_TRY(fft_x_inverse_dd(g, S2, bp, c->stream));
                if (prod) return mirror_accumulate(c, bp, 1.f, inv_s, prod, c->stream);
                return mirror_update(c, bp, 1.f, inv_s, c->stream, wt, c->lambda);
            }
            if (prod) return dd_x_update(g, S2, prod, 0.f, c->stream, nullptr, 0.f, inv_s, 1);
            return done(dd_x_update(g, S2, c->d_psi, c->eps, c->stream, wt, c->lambda, inv_s, 0));
        }
    } else {
        const float2* Kp = c->d_K + ns * (2 * v);
        MVD_TRY(fft_forward_real(g, c->d_psi, c->d_S, c->stream));
        MVD_TRY(fft_y(g, c->d_S, 0, c->stream));
        MVD_TRY(fft_z_mul(g, c->d_S, Kp, c->stream));
        MVD_TRY(fft_y(g, c->d_S, 1, c->stream));
        MVD_TRY(fft_x_ratio(g, c->d_S, phi, c->eps, c->stream));
    }
    const float2* Kc = c->d_K + ns * (c->precise ? v : 2 * v + 1);
    MVD_TRY(fft_y(g, c->d_S, 0, c->stream));
    MVD_TRY(fft_z_mul(g, c->d_S, Kc, c->stream));
    MVD_TRY(fft_y(g, c->d_S, 1, c->stream));
    if (mirror) {
        float* bp = prod ? c->d_bp : c->d_prod;
        MVD_TRY(fft_inverse_real(g, c->d_S, bp, c->stream));
        if (prod) return mirror_accumulate(c, bp, 1.f, inv_s, prod, c->stream);
        return mirror_update(c, bp, 1.f, inv_s, c->stream, wt, c->lambda);
    }
    if (prod) return fft_x_accumulate(g, c->d_S, prod, c->stream, inv_s);
    return done(fft_x_update(g, c->d_S, c->d_psi, c->eps, c->stream, wt, c->lambda, inv_s));
}

namespace {

// Enqueues n_iter iterations, one iteration being what `one` enqueues. On a
// non-NULL stream one iteration is captured once as a CUDA graph (kept per
// key until the next precompute or destroy) and replayed; the host then
// launches one graph per iteration instead of every kernel. Not on the legacy
// default stream (it cannot be captured), not while per-kernel timing is on,
// and not with MVD_NO_GRAPH=1.
template <typename F>
mvd_status run_iterations(mvd_ctx* c, const std::vector<int>& key, int n_iter, F&& one) {
    const char* ng = std::getenv("MVD_NO_GRAPH");
    const bool use_graph = n_iter > 0 && c->stream != nullptr && !g_prof_on.load() && !(ng && ng[0] == '1');
    if (!use_graph) {
        for (int i = 0; i < n_iter; ++i) MVD_TRY(one());
        return MVD_OK;
    }
    cudaGraphExec_t exec = nullptr;
    unsigned nodes = 0;
    auto it = c->graphs.find(key);
    if (it != c->graphs.end()) {
        exec = it->second.exec;
        nodes = it->second.nodes;
    } else {
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_status(e, "begin capture");
        const unsigned long long before = g_launches.load();
        const mvd_status st = one();
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(c->stream, &graph);
        nodes = (unsigned)(g_launches.load() - before);
        g_launches.fetch_sub(nodes);  // captured, not launched
        if (st != MVD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_status(e, "end capture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_status(e, "instantiate graph");
        c->graphs[key] = {exec, nodes};
    }
    for (int i = 0; i < n_iter; ++i) {
        const cudaError_t e = cudaGraphLaunch(exec, c->stream);
        if (e != cudaSuccess) return cuda_status(e, "graph launch");
        count_launch(nodes);
    }
    return MVD_OK;
}

mvd_status cuda_ok(cudaError_t e, const char* what) { return e == cudaSuccess ? MVD_OK : cuda_status(e, what); }

mvd_status read_flag(mvd_ctx* c, int* flag) {
    MVD_CUDA(cudaMemcpyAsync(flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MVD_CUDA(cudaStreamSynchronize(c->stream));
    return MVD_OK;
}

}  // namespace

extern "C" {

void mvd_default_options(mvd_options* opt) {
    if (!opt) return;
    opt->eps = 0.f;
    opt->path = MVD_PATH_AUTO;
    opt->stream = nullptr;
    opt->views_on_device = 0;
    opt->device = -1;
    opt->precision = MVD_PRECISE;
    opt->boundary = MVD_BOUNDARY_PERIODIC;
}

const char* mvd_last_error(void) { return t_err.c_str(); }

unsigned long long mvd_launch_count(void) { return g_launches.load(); }

int mvd_fft_plan(int L, int precision, int* radices, int max_stages) {
    if (!radices || (precision != MVD_PRECISE && precision != MVD_FAST && precision != MVD_MIXED)) return -1;
    if (L < 2) return 0;
    mvd::FftPlan p{};
    if (!mvd::make_radix_plan(L, &p, precision != MVD_FAST)) return 0;
    if (p.nst > max_stages) return -1;
    for (int s = 0; s < p.nst; ++s) radices[s] = p.radix[s];
    return p.nst;
}

void mvd_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(mvd::g_prof_mu);
    mvd::g_prof.clear();
    mvd::g_pool_used = 0;
    mvd::g_prof_on.store(on ? 1 : 0);
}

int mvd_profile_read(const char** names, unsigned long long* launches, double* ms, int max) {
    std::lock_guard<std::mutex> lk(mvd::g_prof_mu);
    double acc[KC_COUNT] = {0};
    unsigned long long cnt[KC_COUNT] = {0};
    for (const auto& r : mvd::g_prof) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            acc[r.cls] += t;
            cnt[r.cls] += 1;
        }
    }
    int n = 0;
    for (int c = 0; c < KC_COUNT && n < max; ++c, ++n) {
        if (names) names[n] = mvd::kClassNames[c];
        if (launches) launches[n] = cnt[c];
        if (ms) ms[n] = acc[c];
    }
    return n;
}

namespace {

// Copies the views into the context (zero-padded on a padded grid), checks
// them, sets psi0 = their mean over the user's voxels and (unless given at
// create) eps = 1e-4 psi0, and resets psi to the flat psi0.
mvd_status load_views(mvd_ctx* c, const float* const* views, int on_device, const char* who) {
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    c->views_ok = false;
    for (int v = 0; v < c->nv; ++v) {
        if (!views[v]) {
            set_error("%s: view %d is NULL", who, v);
            return MVD_ERR_ARG;
        }
        float* dst = c->d_views + (size_t)v * c->M;
        if (c->boundary != MVD_BOUNDARY_PERIODIC) {
            const float* src = views[v];
            if (!on_device) {
                MVD_CUDA(cudaMemcpyAsync(c->d_stage, views[v], c->uM * sizeof(float), kind, c->stream));
                src = c->d_stage;
            }
            MVD_TRY(pad_volume(c, src, dst, c->stream));
            continue;
        }
        MVD_CUDA(cudaMemcpyAsync(dst, views[v], c->M * sizeof(float), kind, c->stream));
    }
    MVD_CUDA(cudaMemsetAsync(c->d_red, 0, 4 * sizeof(double), c->stream));
    MVD_CUDA(cudaMemsetAsync(c->d_flag, 0, 4 * sizeof(int), c->stream));
    MVD_TRY(view_stats(c->d_views, (long)c->nv * c->M, c->d_red, c->d_flag, c->stream));
    double sum = 0.0;
    int bad = 0;
    MVD_CUDA(cudaMemcpyAsync(&sum, c->d_red, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MVD_CUDA(cudaMemcpyAsync(&bad, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MVD_CUDA(cudaStreamSynchronize(c->stream));
    if (bad) {
        set_error("%s: a view holds a negative or non-finite value", who);
        return MVD_ERR_ARG;
    }
    const double mean = sum / ((double)c->uM * c->nv);
    if (!((float)mean > 0.f)) {
        set_error("%s: all views are zero", who);
        return MVD_ERR_ARG;
    }
    c->psi0 = (float)mean;
    const float eps = c->eps_user ? c->eps : (float)(1e-4 * mean);
    if (eps != c->eps) drop_graphs(c);  // the captured passes carry eps
    c->eps = eps;
    MVD_TRY(fill(c->d_psi, c->M, c->psi0, c->stream));
    MVD_TRY(finish_padding(c, c->d_psi, c->stream));
    c->views_ok = true;
    return MVD_OK;
}

}  // namespace

mvd_status mvd_create(const float* const* views, int n_views, const float* const* psfs, const int* psf_dims,
                      const int dims[3], const mvd_options* opt_in, mvd_ctx** out) {
    clear_error();
    if (!out) {
        set_error("mvd_create: out is NULL");
        return MVD_ERR_ARG;
    }
    *out = nullptr;
    mvd_options opt;
    mvd_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (!views || !psfs || !psf_dims || !dims || n_views < 1) {
        set_error("mvd_create: NULL pointer or n_views < 1");
        return MVD_ERR_ARG;
    }
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1) {
        set_error("mvd_create: dims must be >= 1");
        return MVD_ERR_SHAPE;
    }
    if (opt.precision != MVD_PRECISE && opt.precision != MVD_FAST && opt.precision != MVD_MIXED) {
        set_error("mvd_create: unknown precision %d", opt.precision);
        return MVD_ERR_ARG;
    }
    if (opt.path < MVD_PATH_AUTO || opt.path > MVD_PATH_FFT) {
        set_error("mvd_create: unknown path %d", opt.path);
        return MVD_ERR_ARG;
    }
    if (!(opt.eps >= 0.f) || std::isinf(opt.eps)) {
        set_error("mvd_create: eps must be finite and >= 0");
        return MVD_ERR_ARG;
    }
    if (opt.boundary < MVD_BOUNDARY_PERIODIC || opt.boundary > MVD_BOUNDARY_MIRROR) {
        set_error("mvd_create: unknown boundary %d", opt.boundary);
        return MVD_ERR_ARG;
    }
    // PSF shapes and values; normalise to sum 1 (Eq. 3)
    std::vector<float> psf_h;
    std::vector<double> psf_sum;
    std::vector<long> koff(n_views);
    long ktotal = 0;
    for (int v = 0; v < n_views; ++v) {
        const int* k = psf_dims + 3 * v;
        for (int a = 0; a < 3; ++a) {
            if (k[a] < 1 || k[a] % 2 == 0) {
                set_error("mvd_create: PSF %d size %d on axis %d must be odd and >= 1", v, k[a], a);
                return MVD_ERR_SHAPE;
            }
            if (k[a] > dims[a]) {
                set_error("mvd_create: PSF %d size %d exceeds the volume (%d) on axis %d", v, k[a], dims[a], a);
                return MVD_ERR_SHAPE;
            }
        }
        if (!views[v] || !psfs[v]) {
            set_error("mvd_create: view or PSF %d is NULL", v);
            return MVD_ERR_ARG;
        }
        koff[v] = ktotal;
        const long T = (long)k[0] * k[1] * k[2];
        double s = 0.0;
        for (long i = 0; i < T; ++i) {
            const float x = psfs[v][i];
            if (!(x >= 0.f) || std::isinf(x)) {
                set_error("mvd_create: PSF %d has a negative or non-finite value at %ld", v, i);
                return MVD_ERR_ARG;
            }
            s += x;
        }
        if (!(s > 0.0)) {
            set_error("mvd_create: PSF %d sums to zero", v);
            return MVD_ERR_ARG;
        }
        for (long i = 0; i < T; ++i) psf_h.push_back((float)(psfs[v][i] / s));
        psf_sum.push_back(s);
        ktotal += T;
    }

    DeviceGuard dg(opt.device);
    if (!dg.ok) {
        set_error("mvd_create: cannot select device %d", opt.device);
        return MVD_ERR_CUDA;
    }
    mvd_ctx* c = new mvd_ctx();
    cudaGetDevice(&c->device);
    c->stream = (cudaStream_t)opt.stream;
    c->boundary = opt.boundary;
    for (int a = 0; a < 3; ++a) {
        c->udims[a] = dims[a];
        c->dims[a] = dims[a];
        if (opt.boundary != MVD_BOUNDARY_PERIODIC) {
            // pad by the largest half-width h so no term of a periodic
            // convolution wraps into the volume (mirror: 2h, room for the
            // reflections on both sides); round up to a smooth length
            int h = 0;
            for (int v = 0; v < n_views; ++v) h = std::max(h, psf_dims[3 * v + a] / 2);
            c->halo[a] = h;
            int n = dims[a] + (opt.boundary == MVD_BOUNDARY_MIRROR ? 2 * h : h);
            while (!smooth235(n)) ++n;
            c->dims[a] = n;
        }
    }
    c->uM = (long)dims[0] * dims[1] * dims[2];
    c->M = (long)c->dims[0] * c->dims[1] * c->dims[2];
    c->nv = n_views;
    c->kd.assign(psf_dims, psf_dims + 3 * n_views);
    c->koff = koff;
    c->ktotal = ktotal;
    c->psf_sum = psf_sum;
    c->path_opt = opt.path;
    c->precise = opt.precision == MVD_PRECISE ? 1 : opt.precision == MVD_MIXED ? 2 : 0;

    auto fail = [&](mvd_status st) {
        cudaStreamSynchronize(c->stream);
        free_all(c);
        delete c;
        return st;
    };
    mvd_status st;
    if ((st = dev_alloc(&c->d_views, (size_t)n_views * c->M, "views")) != MVD_OK) return fail(st);
    if ((st = dev_alloc(&c->d_psi, (size_t)c->M, "estimate")) != MVD_OK) return fail(st);
    if ((st = dev_alloc(&c->d_r, (size_t)c->M, "ratio buffer")) != MVD_OK) return fail(st);
    if ((st = dev_alloc(&c->d_psf, (size_t)ktotal, "PSFs")) != MVD_OK) return fail(st);
    if ((st = dev_alloc(&c->d_red, 4, "reduction scratch")) != MVD_OK) return fail(st);
    if ((st = dev_alloc(&c->d_flag, 4, "flag")) != MVD_OK) return fail(st);
    if (c->boundary != MVD_BOUNDARY_PERIODIC) {
        if ((st = dev_alloc(&c->d_stage, (size_t)c->uM, "staging volume")) != MVD_OK) return fail(st);
        // mirror: the back-projection on the padded grid, before the fold
        if (c->boundary == MVD_BOUNDARY_MIRROR && (st = dev_alloc(&c->d_prod, (size_t)c->M, "back-projection")) != MVD_OK)
            return fail(st);
    }
    {
        cudaError_t e = cudaMemcpyAsync(c->d_psf, psf_h.data(), ktotal * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return fail(cuda_status(e, "copying PSFs"));
    }
    c->eps_user = opt.eps > 0.f;
    c->eps = opt.eps;
    if ((st = load_views(c, views, opt.views_on_device, "mvd_create")) != MVD_OK) return fail(st);
    c->state = 1;
    *out = c;
    return MVD_OK;
}

namespace {

// Last step of mvd_precompute_kernels once the engine is set up: with a zero
// or mirror boundary, the inverse sensitivity of every view.
mvd_status finish_precompute(mvd_ctx* c, int variant) {
    if (c->boundary != MVD_BOUNDARY_PERIODIC) {
        if (!c->d_invs) MVD_TRY(dev_alloc(&c->d_invs, (size_t)c->nv * c->M, "inverse sensitivities"));
        MVD_TRY(compute_inverse_sensitivity(c));
    }
    c->variant = variant;
    c->state = 2;
    return MVD_OK;
}

}  // namespace

mvd_status mvd_set_views(mvd_ctx* c, const float* const* views, int on_device) {
    clear_error();
    if (!c || !views) {
        set_error("mvd_set_views: NULL argument");
        return MVD_ERR_ARG;
    }
    if (c->state < 1) {
        set_error("mvd_set_views: context not created");
        return MVD_ERR_STATE;
    }
    DeviceGuard dg(c->device);
    return load_views(c, views, on_device, "mvd_set_views");
}

mvd_status mvd_precompute_kernels(mvd_ctx* c, int variant) {
    clear_error();
    if (!c) {
        set_error("mvd_precompute_kernels: NULL context");
        return MVD_ERR_ARG;
    }
    if (c->state < 1) {
        set_error("mvd_precompute_kernels: context not created");
        return MVD_ERR_STATE;
    }
    if (variant < MVD_PLAIN || variant > MVD_OPT2) {
        set_error("mvd_precompute_kernels: unknown variant %d", variant);
        return MVD_ERR_ARG;
    }
    DeviceGuard dg(c->device);
    drop_graphs(c);
    free_fft(c);
    c->direct_ty = 0;
    dev_free(c->d_comp);
    dev_free(c->d_ktmp);
    c->state = 1;
    MVD_TRY(dev_alloc(&c->d_comp, (size_t)c->ktotal, "compound kernels"));
    size_t qmax = 1;
    for (int v = 0; v < c->nv; ++v) {
        const int* k = &c->kd[3 * v];
        qmax = std::max(qmax, (size_t)(2 * k[0] - 1) * (2 * k[1] - 1) * (2 * k[2] - 1));
    }
    MVD_TRY(dev_alloc(&c->d_ktmp, qmax * (size_t)c->nv, "precompute scratch"));
    if (variant == MVD_EFFICIENT)
        MVD_TRY(autocorr_all(c->nv, c->d_psf, c->koff.data(), c->kd.data(), c->d_ktmp, (long)qmax, c->stream));
    MVD_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
    for (int v = 0; v < c->nv; ++v) {
        float* dst = c->d_comp + c->koff[v];
        MVD_TRY(build_compound(c->nv, c->d_psf, c->koff.data(), c->kd.data(), v, variant, dst, c->d_ktmp,
                               (long)qmax, c->stream));
        const int* k = &c->kd[3 * v];
        MVD_TRY(normalize_kernel(dst, k[0] * k[1] * k[2], c->d_flag, c->stream));
    }
    int bad = 0;
    MVD_TRY(read_flag(c, &bad));
    if (bad) {
        set_error("mvd_precompute_kernels: a compound kernel sums to zero");
        return MVD_ERR_ARG;
    }
    int path = c->path_opt;
    const bool fft_ok = smooth235(c->dims[0]) && smooth235(c->dims[1]) && smooth235(c->dims[2]);
    TuneChoice cached;
    const bool use_cached = path == MVD_PATH_AUTO && tune_lookup(std::getenv("MVD_TUNE_CACHE"), tune_key(c), &cached);
    if (use_cached) {
        bool ok = cached.path == MVD_PATH_FFT ? fft_ok : true;
        for (int v = 0; v < c->nv && cached.path == MVD_PATH_DIRECT; ++v) ok = ok && direct_supported(&c->kd[3 * v]);
        if (ok) {
            c->path = cached.path;
            c->direct_ty = cached.path == MVD_PATH_DIRECT ? cached.ty : 0;
            if (cached.path == MVD_PATH_FFT) {
                MVD_TRY(setup_fft(c));
                c->geom.fast = cached.fast != 0;
            }
            return finish_precompute(c, variant);
        }
    }
    if (path == MVD_PATH_AUTO) {
        path = choose_path(c);
        if (path < 0) {
            set_error("mvd_precompute_kernels: no engine fits (dims not {2,3,5}-smooth and PSF too large)");
            return MVD_ERR_UNSUPPORTED;
        }
    } else if (path == MVD_PATH_DIRECT) {
        for (int v = 0; v < c->nv; ++v)
            if (!direct_supported(&c->kd[3 * v])) {
                set_error("mvd_precompute_kernels: PSF %d too large for the direct engine", v);
                return MVD_ERR_UNSUPPORTED;
            }
    } else if (!fft_ok) {
        set_error("mvd_precompute_kernels: FFT engine needs {2,3,5}-smooth dims");
        return MVD_ERR_UNSUPPORTED;
    }
    c->path = path;
    if (path == MVD_PATH_FFT) MVD_TRY(setup_fft(c));
    return finish_precompute(c, variant);
}

mvd_status mvd_set_estimate(mvd_ctx* c, const float* psi, int on_device) {
    clear_error();
    if (!c) {
        set_error("mvd_set_estimate: NULL context");
        return MVD_ERR_ARG;
    }
    if (c->state < 1) {
        set_error("mvd_set_estimate: context not created");
        return MVD_ERR_STATE;
    }
    DeviceGuard dg(c->device);
    const bool padded = c->boundary != MVD_BOUNDARY_PERIODIC;
    if (!psi) {
        MVD_TRY(fill(c->d_psi, c->M, c->psi0, c->stream));
        return finish_padding(c, c->d_psi, c->stream);
    }
    // on a padded grid: stage the user-layout volume, check it, pad it
    float* dst = padded ? c->d_stage : c->d_psi;
    const long n = padded ? c->uM : c->M;
    MVD_CUDA(cudaMemcpyAsync(dst, psi, n * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->stream));
    MVD_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
    MVD_TRY(check_positive(dst, n, c->d_flag, c->stream));
    int bad = 0;
    MVD_TRY(read_flag(c, &bad));
    if (bad) {
        set_error("mvd_set_estimate: the estimate must be finite and > 0");
        fill(c->d_psi, c->M, c->psi0, c->stream);
        finish_padding(c, c->d_psi, c->stream);
        return MVD_ERR_ARG;
    }
    if (!padded) return MVD_OK;
    MVD_TRY(pad_volume(c, c->d_stage, c->d_psi, c->stream));
    return finish_padding(c, c->d_psi, c->stream);
}

mvd_status mvd_iterate(mvd_ctx* c, int n_iter, const int* schedule, int schedule_len) {
    clear_error();
    if (!c) {
        set_error("mvd_iterate: NULL context");
        return MVD_ERR_ARG;
    }
    if (c->state < 2) {
        set_error("mvd_iterate: kernels not precomputed");
        return MVD_ERR_STATE;
    }
    if (!c->views_ok) {
        set_error("mvd_iterate: the last mvd_set_views failed; load valid views first");
        return MVD_ERR_STATE;
    }
    if (n_iter < 0 || schedule_len < 0 || (schedule_len > 0 && !schedule)) {
        set_error("mvd_iterate: bad iteration count or schedule");
        return MVD_ERR_ARG;
    }
    const int L = schedule_len > 0 ? schedule_len : c->nv;
    for (int s = 0; s < L; ++s) {
        const int v = schedule_len > 0 ? schedule[s] : s;
        if (v < 0 || v >= c->nv) {
            set_error("mvd_iterate: schedule entry %d = %d out of range", s, v);
            return MVD_ERR_ARG;
        }
    }
    DeviceGuard dg(c->device);
    std::vector<int> sched(L);
    for (int s = 0; s < L; ++s) sched[s] = schedule_len > 0 ? schedule[s] : s;
    return run_iterations(c, sched, n_iter, [&]() -> mvd_status {
        for (int s = 0; s < L; ++s) MVD_TRY(one_update(c, sched[s]));
        return MVD_OK;
    });
}

mvd_status mvd_set_weights(mvd_ctx* c, const float* const* weights, int on_device, int norm, float value,
                           float* target) {
    clear_error();
    if (!c) {
        set_error("mvd_set_weights: NULL context");
        return MVD_ERR_ARG;
    }
    if (c->state < 1) {
        set_error("mvd_set_weights: context not created");
        return MVD_ERR_STATE;
    }
    DeviceGuard dg(c->device);
    drop_graphs(c);  // the captured update passes carry the weight pointers
    if (!weights) {
        dev_free(c->d_w);
        c->weight_norm = 0.f;
        return MVD_OK;
    }
    if (norm < MVD_WEIGHTS_SUM_ONE || norm > MVD_WEIGHTS_USER || (norm == MVD_WEIGHTS_USER && !(value > 0.f))) {
        set_error("mvd_set_weights: unknown normalisation %d or bad value", norm);
        return MVD_ERR_ARG;
    }
    for (int v = 0; v < c->nv; ++v)
        if (!weights[v]) {
            set_error("mvd_set_weights: weight image %d is NULL", v);
            return MVD_ERR_ARG;
        }
    const long M = c->M;
    const int nv = c->nv;
    float* w = nullptr;
    MVD_TRY(dev_alloc(&w, (size_t)nv * M, "view weights"));
    mvd_status st = MVD_OK;
    unsigned long long* stats = nullptr;
    do {
        const bool padded = c->boundary != MVD_BOUNDARY_PERIODIC;
        for (int v = 0; v < nv && st == MVD_OK; ++v) {
            if (!padded) {
                const cudaError_t e = cudaMemcpyAsync(w + (size_t)v * M, weights[v], sizeof(float) * M,
                                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                                      c->stream);
                if (e != cudaSuccess) st = cuda_status(e, "mvd_set_weights: copy");
                continue;
            }
            // zero / mirror boundary: the user-layout image onto the padded grid, 0 in the
            // padding (no view covers it, so the overlap counts and the normalisation are
            // those of the user's volume)
            const float* src = weights[v];
            if (!on_device) {
                const cudaError_t e = cudaMemcpyAsync(c->d_stage, weights[v], sizeof(float) * c->uM,
                                                      cudaMemcpyHostToDevice, c->stream);
                if (e != cudaSuccess) {
                    st = cuda_status(e, "mvd_set_weights: copy");
                    break;
                }
                src = c->d_stage;
            }
            st = pad_volume(c, src, w + (size_t)v * M, c->stream);
        }
        if (st != MVD_OK) break;
        int bad = 0;
        if ((st = cuda_ok(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream), "flag")) != MVD_OK) break;
        if ((st = weights_check(w, (long)nv * M, c->d_flag, c->stream)) != MVD_OK) break;
        if ((st = read_flag(c, &bad)) != MVD_OK) break;
        if (bad) {
            set_error("mvd_set_weights: weights must lie in [0, 1]");
            st = MVD_ERR_ARG;
            break;
        }
        double T = 1.0;
        if (norm == MVD_WEIGHTS_USER) {
            T = value;
        } else if (norm != MVD_WEIGHTS_SUM_ONE) {
            if ((st = dev_alloc(&stats, 2, "overlap counts")) != MVD_OK) break;
            const int big = 1 << 30;
            unsigned long long h[2] = {0, 0};
            int mn = big;
            cudaMemcpyAsync(stats, h, sizeof(h), cudaMemcpyHostToDevice, c->stream);
            cudaMemcpyAsync(c->d_flag, &mn, sizeof(int), cudaMemcpyHostToDevice, c->stream);
            if ((st = weights_overlap(w, nv, M, stats, c->d_flag, c->stream)) != MVD_OK) break;
            cudaMemcpyAsync(h, stats, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
            cudaMemcpyAsync(&mn, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
            if ((st = cuda_ok(cudaStreamSynchronize(c->stream), "overlap counts")) != MVD_OK) break;
            if (h[0] == 0) {
                set_error("mvd_set_weights: no voxel is covered by any view");
                st = MVD_ERR_ARG;
                break;
            }
            T = norm == MVD_WEIGHTS_MIN_OVERLAP ? (double)mn : (double)h[1] / (double)h[0];
        }
        if ((st = weights_normalize(w, nv, M, (float)T, c->stream)) != MVD_OK) break;
        if ((st = cuda_ok(cudaStreamSynchronize(c->stream), "normalise weights")) != MVD_OK) break;
        dev_free(c->d_w);
        c->d_w = w;
        w = nullptr;
        c->weight_norm = (float)T;
        if (target) *target = (float)T;
    } while (false);
    dev_free(w);
    dev_free(stats);
    return st;
}

mvd_status mvd_set_regularization(mvd_ctx* c, float lambda) {
    clear_error();
    if (!c) {
        set_error("mvd_set_regularization: NULL context");
        return MVD_ERR_ARG;
    }
    if (!(lambda >= 0.f) || !(lambda < 1e30f)) {
        set_error("mvd_set_regularization: lambda must be finite and >= 0");
        return MVD_ERR_ARG;
    }
    DeviceGuard dg(c->device);
    drop_graphs(c);  // the captured update passes carry lambda
    c->lambda = lambda;
    return MVD_OK;
}

mvd_status mvd_get_weights(mvd_ctx* c, int v, float* out, size_t n_elems) {
    clear_error();
    if (!c || !out) {
        set_error("mvd_get_weights: NULL argument");
        return MVD_ERR_ARG;
    }
    if (!c->d_w) {
        set_error("mvd_get_weights: no weights set");
        return MVD_ERR_STATE;
    }
    const bool padded = c->boundary != MVD_BOUNDARY_PERIODIC;
    const long n = padded ? c->uM : c->M;
    if (v < 0 || v >= c->nv || n_elems < (size_t)n) {
        set_error("mvd_get_weights: bad view or buffer size");
        return MVD_ERR_ARG;
    }
    DeviceGuard dg(c->device);
    const float* src = c->d_w + (size_t)v * c->M;
    if (padded) {
        MVD_TRY(crop_volume(c, src, c->d_stage, c->stream));
        src = c->d_stage;
    }
    MVD_CUDA(cudaMemcpyAsync(out, src, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
    MVD_CUDA(cudaStreamSynchronize(c->stream));
    return MVD_OK;
}

mvd_status mvd_iterate_combined(mvd_ctx* c, int n_iter, int root) {
    clear_error();
    if (!c) {
        set_error("mvd_iterate_combined: NULL context");
        return MVD_ERR_ARG;
    }
    if (c->state < 2) {
        set_error("mvd_iterate_combined: kernels not precomputed");
        return MVD_ERR_STATE;
    }
    if (!c->views_ok) {
        set_error("mvd_iterate_combined: the last mvd_set_views failed; load valid views first");
        return MVD_ERR_STATE;
    }
    if (n_iter < 0) {
        set_error("mvd_iterate_combined: n_iter < 0");
        return MVD_ERR_ARG;
    }
    if (c->d_w || c->lambda != 0.f) {
        set_error("mvd_iterate_combined: view weights and regularisation apply to the sequential update only");
        return MVD_ERR_UNSUPPORTED;
    }
    DeviceGuard dg(c->device);
    if (!c->d_prod) MVD_TRY(dev_alloc(&c->d_prod, (size_t)c->M, "combined-update product"));
    if (c->boundary == MVD_BOUNDARY_MIRROR && !c->d_bp)
        MVD_TRY(dev_alloc(&c->d_bp, (size_t)c->M, "back-projection"));
    const float e = root ? (float)(1.0 / (double)c->nv) : 1.f;
    // graph key: schedule entries are >= 0, so {-1} and {-2} name the two combined forms.
    // Zero / mirror boundary: every factor is c_v / s_v (the accumulate passes divide
    // by the sensitivity); afterwards the padding is cleared, or the halo refilled with
    // the estimate's reflection for the next forward blurs.
    return run_iterations(c, {root ? -2 : -1}, n_iter, [&]() -> mvd_status {
        MVD_TRY(fill(c->d_prod, c->M, 1.f, c->stream));
        for (int v = 0; v < c->nv; ++v) MVD_TRY(view_pass(c, v, c->d_prod));
        MVD_TRY(apply_product(c->d_psi, c->d_prod, c->M, e, c->eps, c->stream));
        return finish_padding(c, c->d_psi, c->stream);
    });
}

mvd_status mvd_result(mvd_ctx* c, float* out, size_t n_elems) {
    clear_error();
    if (!c || !out) {
        set_error("mvd_result: NULL argument");
        return MVD_ERR_ARG;
    }
    if (c->state < 1) {
        set_error("mvd_result: context not created");
        return MVD_ERR_STATE;
    }
    const long n = c->boundary != MVD_BOUNDARY_PERIODIC ? c->uM : c->M;
    if (n_elems < (size_t)n) {
        set_error("mvd_result: buffer holds %zu elements, need %ld", n_elems, n);
        return MVD_ERR_SHAPE;
    }
    DeviceGuard dg(c->device);
    const float* src = c->d_psi;
    if (c->boundary != MVD_BOUNDARY_PERIODIC) {
        MVD_TRY(crop_volume(c, c->d_psi, c->d_stage, c->stream));
        src = c->d_stage;
    }
    MVD_CUDA(cudaMemcpyAsync(out, src, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    MVD_CUDA(cudaStreamSynchronize(c->stream));
    return MVD_OK;
}

mvd_status mvd_result_device(mvd_ctx* c, const float** dptr) {
    clear_error();
    if (!c || !dptr) {
        set_error("mvd_result_device: NULL argument");
        return MVD_ERR_ARG;
    }
    if (c->state < 1) {
        set_error("mvd_result_device: context not created");
        return MVD_ERR_STATE;
    }
    if (c->boundary != MVD_BOUNDARY_PERIODIC) {
        DeviceGuard dg(c->device);
        MVD_TRY(crop_volume(c, c->d_psi, c->d_stage, c->stream));
        *dptr = c->d_stage;
        return MVD_OK;
    }
    *dptr = c->d_psi;
    return MVD_OK;
}

mvd_status mvd_synchronize(mvd_ctx* c) {
    clear_error();
    if (!c) {
        set_error("mvd_synchronize: NULL context");
        return MVD_ERR_ARG;
    }
    DeviceGuard dg(c->device);
    MVD_CUDA(cudaStreamSynchronize(c->stream));
    return MVD_OK;
}

void mvd_destroy(mvd_ctx* c) {
    if (!c) return;
    DeviceGuard dg(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

float mvd_get_eps(const mvd_ctx* c) { return c ? c->eps : 0.f; }
float mvd_get_psi0(const mvd_ctx* c) { return c ? c->psi0 : 0.f; }
int mvd_get_path(const mvd_ctx* c) { return c ? c->path : -1; }

mvd_status mvd_get_compound_kernel(mvd_ctx* c, int v, float* out, size_t n_elems) {
    clear_error();
    if (!c || !out) {
        set_error("mvd_get_compound_kernel: NULL argument");
        return MVD_ERR_ARG;
    }
    if (c->state < 2) {
        set_error("mvd_get_compound_kernel: kernels not precomputed");
        return MVD_ERR_STATE;
    }
    if (v < 0 || v >= c->nv) {
        set_error("mvd_get_compound_kernel: view %d out of range", v);
        return MVD_ERR_ARG;
    }
    const int* k = &c->kd[3 * v];
    const size_t T = (size_t)k[0] * k[1] * k[2];
    if (n_elems < T) {
        set_error("mvd_get_compound_kernel: buffer too small");
        return MVD_ERR_SHAPE;
    }
    DeviceGuard dg(c->device);
    MVD_CUDA(cudaMemcpyAsync(out, c->d_comp + c->koff[v], T * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    MVD_CUDA(cudaStreamSynchronize(c->stream));
    return MVD_OK;
}

mvd_status mvd_autotune(mvd_ctx* c, const char* cache_path, mvd_tune_result* out) {
    clear_error();
    if (!c) {
        set_error("mvd_autotune: NULL context");
        return MVD_ERR_ARG;
    }
    if (c->state < 2) {
        set_error("mvd_autotune: kernels not precomputed");
        return MVD_ERR_STATE;
    }
    if (!c->views_ok) {
        set_error("mvd_autotune: the last mvd_set_views failed; load valid views first");
        return MVD_ERR_STATE;
    }
    DeviceGuard dg(c->device);
    if (!cache_path) cache_path = std::getenv("MVD_TUNE_CACHE");
    const std::string key = tune_key(c);
    TuneChoice best;
    int from_cache = 0;
    const bool fft_ok = smooth235(c->dims[0]) && smooth235(c->dims[1]) && smooth235(c->dims[2]);
    bool direct_ok = true;
    for (int v = 0; v < c->nv; ++v) direct_ok = direct_ok && direct_supported(&c->kd[3 * v]);
    if (tune_lookup(cache_path, key, &best) && (best.path == MVD_PATH_FFT ? fft_ok : direct_ok)) {
        from_cache = 1;
        if (best.path == MVD_PATH_FFT && !c->d_S) MVD_TRY(setup_fft(c));
    } else {
        float* save = nullptr;
        MVD_TRY(dev_alloc(&save, (size_t)c->M, "autotune estimate copy"));
        mvd_status st = MVD_OK;
        const cudaError_t ce =
            cudaMemcpyAsync(save, c->d_psi, sizeof(float) * c->M, cudaMemcpyDeviceToDevice, c->stream);
        if (ce != cudaSuccess) {
            dev_free(save);
            return cuda_status(ce, "autotune: save estimate");
        }
        best.ms = -1.0;
        std::vector<TuneChoice> cands;
        if (fft_ok) {
            const bool any_fast = fft_fast_supported(c->dims[0]) || fft_fast_supported(c->dims[1]) ||
                                  fft_fast_z_supported(c->dims[2]);
            if (any_fast) cands.push_back({MVD_PATH_FFT, 0, 1, 0.0});
            cands.push_back({MVD_PATH_FFT, 0, 0, 0.0});
        }
        if (direct_ok) {
            // tile heights that fit every view's box
            int common[4] = {8, 4, 2, 1};
            for (int ty : common) {
                bool fits = true;
                for (int v = 0; v < c->nv; ++v) {
                    int opts[4];
                    const int n = direct_tile_heights(&c->kd[3 * v], opts);
                    fits = fits && std::find(opts, opts + n, ty) != opts + n;
                }
                if (fits) cands.push_back({MVD_PATH_DIRECT, ty, 1, 0.0});
            }
        }
        const int prev_path = c->path, prev_ty = c->direct_ty, prev_fast = c->geom.fast ? 1 : 0;
        for (size_t i = 0; i < cands.size() && st == MVD_OK; ++i) {
            TuneChoice t = cands[i];
            if (t.path == MVD_PATH_FFT && !c->d_S && (st = setup_fft(c)) != MVD_OK) break;
            apply_choice(c, t);
            double ms = 0.0;
            if ((st = time_updates(c, save, best.ms, &ms)) != MVD_OK) break;
            t.ms = ms;
            if (best.ms < 0 || ms < best.ms) best = t;
        }
        dev_free(save);
        if (st != MVD_OK) {
            apply_choice(c, {prev_path, prev_ty, prev_fast, 0.0});
            return st;
        }
        if (best.ms < 0) {
            set_error("mvd_autotune: no engine fits this problem");
            return MVD_ERR_UNSUPPORTED;
        }
        tune_store(cache_path, key, best);
    }
    apply_choice(c, best);
    if (best.path == MVD_PATH_DIRECT) free_fft(c);
    if (out) {
        out->path = best.path;
        out->direct_tile_y = best.path == MVD_PATH_DIRECT ? best.ty : 0;
        out->fft_engine = best.path == MVD_PATH_FFT ? best.fast : -1;
        out->from_cache = from_cache;
        out->ms_per_update = best.ms;
    }
    return MVD_OK;
}

}  // extern "C"
