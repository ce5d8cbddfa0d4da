// Batched form: many independent deconvolution problems (contexts of uneven
// size and view count) advanced together by one launch. Two executions:
//
// MVD_BATCH_BRANCHES. One CUDA graph in which every volume's whole run (its
// n_iter iterations of view updates, each the single-volume engine's kernels)
// is an independent branch. The graph executor runs kernels of different
// branches side by side, so small volumes, whose kernels fill only part of
// the GPU, and the tails of large kernels overlap with other volumes' work.
// Branches start largest volume first.
//
// MVD_BATCH_PERSISTENT. ONE persistent kernel launch, described below.
//
// Work queue. Every view update of every volume is the same 9 passes
// (x-forward, y+, z*K_v, y-, x-ratio, y+, z*K_v^comp, y-, x-update); each
// pass splits into independent tiles. The host lists all tiles of the job in
// phase order (iteration, view slot, pass; volumes inside a phase), as
// "entries" (one per volume and phase) with a contiguous task range each.
// Blocks take task ids from one global counter. A task may start once every
// tile of the same volume's previous entry is done: each volume has one
// monotonic completion counter, and the entry stores the count it needs.
// A block only waits for tasks with smaller ids, which blocks that are
// already running took, so the smallest unfinished task can always run and
// the queue drains without assuming co-resident blocks.
//
// Waits are bounded: after poll_limit polls a block sets the error flag and
// leaves; every block stops taking tasks once the flag is set, and the host
// reports MVD_ERR_TIMEOUT. Loads of data other blocks wrote during the launch
// (spectra, estimates) go to L2 (ld.global.cg), completions are published
// with a fence before the counter increment, and waits read the counter with
// acquire semantics.
#include <algorithm>
#include <type_traits>
#include <cstdlib>
#include <vector>

#include "fft_dd.cuh"
#include "fft_dd_fast.cuh"
#include "fft_fast_tiles.cuh"
#include "fft_generic.cuh"

struct mvd_batch;

namespace mvd {

namespace {

enum Pass { XF = 0, YF1, Z1, YI1, XR, YF2, Z2, YI2, XU, NPASS };

struct VolDesc {
    int X, Y, Z, Xh, nv;
    long YZ, M;
    FftPlan px, py, pz;
    float* psi;
    const float* views;
    float2* S;
    const float2* K;  // 2*nv spectra of Xh*Y*Z
    float eps;
    int fx, fy, fz;  // register-resident tiles on this axis (length 64, 128 or 256)
    int precise;     // forward blur in double-float (passes XF..XR)
    cdd* S2;
    const cdd* KP2;  // nv double-float spectra of P_v
    const cdd *tw2x, *tw2y, *tw2z;
};

struct Entry {
    long begin;                 // first task id
    unsigned long long target;  // completed tiles of this volume needed before starting
    int vol, pass, view;
    int ntiles, tpt;  // tiles of this pass, tiles per task
};

struct BatchArgs {
    const VolDesc* vols;
    const Entry* entries;
    int n_entries;
    long total;
    unsigned long long* next;  // task counter
    unsigned long long* done;  // per-volume completed tiles
    int* error;
    long long poll_limit;
};

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

template <typename F>
__device__ __forceinline__ void with_len(int L, F&& f) {
    switch (L) {
        case 64: f(std::integral_constant<int, 64>{}); break;
        case 128: f(std::integral_constant<int, 128>{}); break;
        default: f(std::integral_constant<int, 256>{}); break;
    }
}

// precise mode, axes of length 64, 128 or 256: register-resident
// double-float passes (the same tiles as the single-volume engine)
__device__ bool run_tile_ddf(const VolDesc& d, int pass, int view, long tile, cdd* sm) {
    const size_t ns = (size_t)d.Xh * d.YZ;
    switch (pass) {
        case XF:
        case XR: {
            if (!d.fx) return false;
            const DdXFast a{d.psi, d.S2, d.views + (size_t)view * d.M, d.YZ, d.eps, d.tw2x, d.px};
            with_len(d.X, [&](auto Lc) {
                constexpr int L = decltype(Lc)::value;
                if (pass == XF)
                    ddf_x_forward_tile<L, true>(a, tile, sm);
                else
                    ddf_x_ratio_tile<L, true>(a, tile, sm);
            });
            return true;
        }
        case Z1:
        case Z2: {
            if (!d.fz) return false;
            const cdd* K2 = reinterpret_cast<const cdd*>(reinterpret_cast<const float4*>(d.KP2) +
                                                         ns * (2 * view + (pass == Z2 ? 1 : 0)));
            with_len(d.Z, [&](auto Lc) {
                constexpr int L = decltype(Lc)::value;
                const int nty = (int)gen_div_up(d.Y, ddf_z_cols(L));
                ddf_z_tile<L, true, true>(d.S2, K2, d.Y, d.YZ, nty, dd{1.f, 0.f}, d.tw2z, tile, sm);
            });
            return true;
        }
        default: {  // y passes
            if (!d.fy) return false;
            const long nl = (long)d.Xh * d.Z;
            const bool inv = pass == YI1 || pass == YI2;
            with_len(d.Y, [&](auto Lc) {
                constexpr int L = decltype(Lc)::value;
                if (inv)
                    ddf_y_tile<L, +1, true>(d.S2, nl, d.tw2y, tile, sm);
                else
                    ddf_y_tile<L, -1, true>(d.S2, nl, d.tw2y, tile, sm);
            });
            return true;
        }
    }
}

// precise mode: every pass but the update runs in double-float
__device__ void run_tile_dd(const VolDesc& d, int pass, int view, long tile, cdd* sm) {
    const size_t ns = (size_t)d.Xh * d.YZ;
    if (run_tile_ddf(d, pass, view, tile, sm)) return;
    switch (pass) {
        case XF: {
            DdX a = dd_x_args(d.X, d.YZ, d.px, d.tw2x);
            a.src = d.psi;
            a.S2 = d.S2;
            dd_x_forward_tile<true>(a, tile, sm);
            break;
        }
        case YF1:
        case YF2:
            dd_y_tile<true, -1>(dd_y_args(d.Y, d.Xh, d.Z, d.py, d.tw2y, d.S2), tile, sm);
            break;
        case YI1:
        case YI2:
            dd_y_tile<true, +1>(dd_y_args(d.Y, d.Xh, d.Z, d.py, d.tw2y, d.S2), tile, sm);
            break;
        case Z1:
        case Z2: {
            const cdd* K2 = reinterpret_cast<const cdd*>(reinterpret_cast<const float4*>(d.KP2) +
                                                         ns * (2 * view + (pass == Z2 ? 1 : 0)));
            dd_z_tile<true, true>(dd_z_args(d.Z, d.Y, d.YZ, d.pz, d.tw2z, d.S2, K2, dd{1.f, 0.f}), tile, sm);
            break;
        }
        default: {  // XR
            DdX a = dd_x_args(d.X, d.YZ, d.px, d.tw2x);
            a.S2 = d.S2;
            a.phi = d.views + (size_t)view * d.M;
            a.eps = d.eps;
            dd_x_ratio_tile<true>(a, tile, sm);
            break;
        }
    }
}

__device__ void run_tile(const VolDesc& d, int pass, int view, long tile, float2* sm) {
    const size_t ns = (size_t)d.Xh * d.YZ;
    if (d.precise && pass != XU) {
        run_tile_dd(d, pass, view, tile, reinterpret_cast<cdd*>(sm));
        return;
    }
    switch (pass) {
        case XF: {
            if (d.fx) {
                const XFast a{d.psi, d.S, nullptr, nullptr, d.YZ, 0.f, d.px.tw};
                with_len(d.X, [&](auto Lc) { fast_x_forward_tile<decltype(Lc)::value, true>(a, tile, sm); });
            } else {
                GenX a = gen_x_args(d.X, d.YZ, d.px);
                a.src = d.psi;
                a.S = d.S;
                gen_x_forward_tile<true>(a, tile, sm);
            }
            break;
        }
        case YF1:
        case YF2:
        case YI1:
        case YI2: {
            const bool inv = pass == YI1 || pass == YI2;
            if (d.fy) {
                const long nl = (long)d.Xh * d.Z;
                with_len(d.Y, [&](auto Lc) {
                    constexpr int L = decltype(Lc)::value;
                    if (inv)
                        fast_y_tile<L, +1, true>(d.S, nl, d.py.tw, tile, sm);
                    else
                        fast_y_tile<L, -1, true>(d.S, nl, d.py.tw, tile, sm);
                });
            } else if (inv) {
                gen_y_tile<true, +1>(gen_y_args(d.Y, d.Xh, d.Z, d.py, d.S), tile, sm);
            } else {
                gen_y_tile<true, -1>(gen_y_args(d.Y, d.Xh, d.Z, d.py, d.S), tile, sm);
            }
            break;
        }
        case Z1:
        case Z2: {
            const float2* K = d.K + ns * (2 * view + (pass == Z2 ? 1 : 0));
            if (d.fz) {
                with_len(d.Z, [&](auto Lc) {
                    constexpr int L = decltype(Lc)::value;
                    const int nty = (int)gen_div_up(d.Y, fast_z_cols(L));
                    fast_z_tile<L, true, true>(d.S, K, d.Y, d.YZ, nty, 1.f, d.pz.tw, tile, sm);
                });
            } else {
                gen_z_tile<true, true>(gen_z_args(d.Z, d.Y, d.YZ, d.pz, d.S, K, 1.f), tile, sm);
            }
            break;
        }
        case XR: {
            if (d.fx) {
                const XFast a{nullptr, d.S, d.views + (size_t)view * d.M, nullptr, d.YZ, d.eps, d.px.tw};
                with_len(d.X, [&](auto Lc) { fast_x_inverse_tile<decltype(Lc)::value, 0, true>(a, tile, sm); });
            } else {
                GenX a = gen_x_args(d.X, d.YZ, d.px);
                a.S = d.S;
                a.phi = d.views + (size_t)view * d.M;
                a.eps = d.eps;
                gen_x_ratio_tile<true>(a, tile, sm);
            }
            break;
        }
        default: {  // XU
            if (d.precise) {  // the double-float x inverse of the double-float spectrum
                if (d.fx) {
                    const DdXUpd a{d.S2, d.psi, d.YZ, d.eps, d.tw2x, nullptr, 0.f, nullptr};
                    with_len(d.X, [&](auto Lc) {
                        ddf_x_update_tile<decltype(Lc)::value, 1>(a, tile, reinterpret_cast<cdd*>(sm));
                    });
                } else {
                    DdXU u{};
                    u.x = dd_x_args(d.X, d.YZ, d.px, d.tw2x);
                    u.x.S2 = d.S2;
                    u.x.eps = d.eps;
                    u.psi = d.psi;
                    dd_x_update_tile<true, 1>(u, tile, reinterpret_cast<cdd*>(sm));
                }
            } else if (d.fx) {
                const XFast a{nullptr, d.S, nullptr, d.psi, d.YZ, d.eps, d.px.tw};
                with_len(d.X, [&](auto Lc) { fast_x_inverse_tile<decltype(Lc)::value, 1, true>(a, tile, sm); });
            } else {
                GenX a = gen_x_args(d.X, d.YZ, d.px);
                a.S = d.S;
                a.psi = d.psi;
                a.eps = d.eps;
                gen_x_inverse_tile<true, 1>(a, tile, sm);
            }
            break;
        }
    }
}

__global__ void __launch_bounds__(kGenThreads, 2) k_batch(BatchArgs a) {
    extern __shared__ float2 sm[];
    __shared__ long s_task;
    __shared__ int s_entry, s_stop;
    int cur = 0;  // entry cursor of thread 0: task ids of a block only increase
    long nxt = 0;
    if (threadIdx.x == 0) nxt = (long)atomicAdd(a.next, 1ull);
    for (;;) {
        if (threadIdx.x == 0) {
            const long task = nxt;
            int stop = 0;
            if (task >= a.total || *(volatile int*)a.error) {
                stop = 1;
            } else {
                while (cur + 1 < a.n_entries && a.entries[cur + 1].begin <= task) ++cur;
                const Entry e = a.entries[cur];
                long long polls = 0;
                while (ld_acquire(a.done + e.vol) < e.target) {
                    if (++polls > a.poll_limit || *(volatile int*)a.error) {
                        atomicExch(a.error, 1);
                        stop = 1;
                        break;
                    }
                    __nanosleep(128);
                }
                // the next id is fetched now; its latency overlaps this task's work
                if (!stop) nxt = (long)atomicAdd(a.next, 1ull);
            }
            s_task = task;
            s_entry = cur;
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) break;
        const Entry e = a.entries[s_entry];
        const long first = (s_task - e.begin) * e.tpt;
        const int count = (int)min((long)e.tpt, (long)e.ntiles - first);
        const VolDesc& d = a.vols[e.vol];
        for (int k = 0; k < count; ++k) {
            run_tile(d, e.pass, e.view, first + k, sm);
            __syncthreads();
        }
        __threadfence();  // each thread's stores of this task reach gpu scope ...
        __syncthreads();  // ... before the block publishes its tiles as done
        if (threadIdx.x == 0) atomicAdd(a.done + e.vol, (unsigned long long)count);
    }
}

// tiles of one pass, and elements each tile transforms
void pass_tiles(const VolDesc& d, int pass, long* ntiles, long* elems) {
    if (d.precise) {  // double-float tiles, the update's x inverse included
        switch (pass) {
            case XF:
            case XR:
            case XU:
                if (d.fx) {
                    *ntiles = gen_div_up(d.YZ, 2L * ddf_pairs(d.X));
                    *elems = 2L * ddf_pairs(d.X) * d.X * 4;
                    return;
                }
                *ntiles = dd_x_tiles(d.X, d.YZ);
                *elems = 2L * dd_x_pairs(d.X) * d.X * 4;  // double-float work counts about 4x
                return;
            case Z1:
            case Z2:
                if (d.fz) {
                    *ntiles = (long)d.Xh * gen_div_up(d.Y, ddf_z_cols(d.Z));
                    *elems = (long)ddf_z_cols(d.Z) * d.Z * 4;
                    return;
                }
                *ntiles = dd_z_tiles(d.Z, d.Y, d.Xh);
                *elems = (long)dd_z_cols(d.Z, d.Y) * d.Z * 4;
                return;
            default:
                if (d.fy) {
                    *ntiles = gen_div_up((long)d.Xh * d.Z, ddf_y_lines(d.Y));
                    *elems = (long)ddf_y_lines(d.Y) * d.Y * 4;
                    return;
                }
                *ntiles = dd_y_tiles(d.Y, d.Xh, d.Z);
                *elems = (long)dd_y_lines(d.Y) * d.Y * 4;
                return;
        }
    }
    switch (pass) {
        case XF:
        case XR:
        case XU:
            if (d.fx) {
                *ntiles = gen_div_up(d.YZ, fast_x_rows(d.X));
                *elems = (long)fast_x_rows(d.X) * d.X;
            } else {
                *ntiles = gen_x_tiles(d.X, d.YZ);
                *elems = 2L * gen_x_pairs(d.X) * d.X;
            }
            return;
        case Z1:
        case Z2:
            if (d.fz) {
                *ntiles = (long)d.Xh * gen_div_up(d.Y, fast_z_cols(d.Z));
                *elems = (long)fast_z_cols(d.Z) * d.Z;
            } else {
                *ntiles = gen_z_tiles(d.Z, d.Y, d.Xh);
                *elems = (long)gen_z_cols(d.Z, d.Y) * d.Z;
            }
            return;
        default:
            if (d.fy) {
                *ntiles = gen_div_up((long)d.Xh * d.Z, fast_y_lines(d.Y));
                *elems = (long)fast_y_lines(d.Y) * d.Y;
            } else {
                *ntiles = gen_y_tiles(d.Y, d.Xh, d.Z);
                *elems = (long)gen_y_lines(d.Y) * d.Y;
            }
            return;
    }
}

bool batch_fast_len(int L) { return L == 64 || L == 128 || L == 256; }

}  // namespace

}  // namespace mvd

using namespace mvd;

struct mvd_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n = 0, n_iter = 0;
    VolDesc* d_vols = nullptr;
    Entry* d_entries = nullptr;
    int n_entries = 0;
    long total = 0;
    unsigned long long* d_counters = nullptr;  // [0] next task, [1..n] done per volume
    int* d_error = nullptr;
    int grid = 0;
    size_t smem = 0;
    long long poll_limit = 0;
    int mode = MVD_BATCH_PERSISTENT;
    unsigned graph_nodes = 0;  // kernels in one run (branches mode)
    cudaGraphExec_t exec = nullptr;
};

namespace {

void batch_free(mvd_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->d_vols) cudaFree(b->d_vols);
    if (b->d_entries) cudaFree(b->d_entries);
    if (b->d_counters) cudaFree(b->d_counters);
    if (b->d_error) cudaFree(b->d_error);
    delete b;
}

// One graph whose branches are the volumes' whole runs, captured from the
// single-volume engine with each context's work redirected to a branch stream.
mvd_status capture_branches(mvd_batch* b, mvd_ctx* const* ctxs) {
    const int n = b->n;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (double)ctxs[x]->M * ctxs[x]->nv > (double)ctxs[y]->M * ctxs[y]->nv;
    });
    std::vector<cudaStream_t> streams(n, nullptr);
    std::vector<cudaEvent_t> joins(n, nullptr);
    cudaEvent_t fork = nullptr;
    mvd_status st = MVD_OK;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&streams[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&joins[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) st = cuda_status(e, "batch branch streams");
    bool capturing = false;
    if (st == MVD_OK) {
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) st = cuda_status(e, "batch capture");
        capturing = st == MVD_OK;
    }
    const unsigned long long before = g_launches.load();
    if (st == MVD_OK && (e = cudaEventRecord(fork, b->stream)) != cudaSuccess) st = cuda_status(e, "batch fork");
    for (int k = 0; k < n && st == MVD_OK; ++k) {
        mvd_ctx* c = ctxs[order[k]];
        if ((e = cudaStreamWaitEvent(streams[k], fork, 0)) != cudaSuccess) {
            st = cuda_status(e, "batch branch start");
            break;
        }
        cudaStream_t own = c->stream;
        c->stream = streams[k];
        for (int it = 0; it < b->n_iter && st == MVD_OK; ++it)
            for (int v = 0; v < c->nv && st == MVD_OK; ++v) st = one_update(c, v);
        c->stream = own;
        if (st != MVD_OK) break;
        if ((e = cudaEventRecord(joins[k], streams[k])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(b->stream, joins[k], 0)) != cudaSuccess)
            st = cuda_status(e, "batch branch join");
    }
    b->graph_nodes = (unsigned)(g_launches.load() - before);
    g_launches.fetch_sub(b->graph_nodes);  // captured, not launched
    if (capturing) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->stream, &graph);
        if (st == MVD_OK && e != cudaSuccess) st = cuda_status(e, "batch capture end");
        if (st == MVD_OK) {
            e = cudaGraphInstantiate(&b->exec, graph, 0);
            if (e != cudaSuccess) st = cuda_status(e, "batch graph");
        }
        if (graph) cudaGraphDestroy(graph);
    }
    for (int k = 0; k < n; ++k) {
        if (joins[k]) cudaEventDestroy(joins[k]);
        if (streams[k]) cudaStreamDestroy(streams[k]);
    }
    if (fork) cudaEventDestroy(fork);
    return st;
}

mvd_status enqueue(mvd_batch* b) {
    MVD_CUDA(cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned long long) * (b->n + 1), b->stream));
    MVD_CUDA(cudaMemsetAsync(b->d_error, 0, sizeof(int), b->stream));
    BatchArgs a{b->d_vols, b->d_entries, b->n_entries, b->total, b->d_counters, b->d_counters + 1, b->d_error,
                b->poll_limit};
    k_batch<<<b->grid, kGenThreads, b->smem, b->stream>>>(a);
    count_launch();
    return check_launch("batch kernel");
}

}  // namespace

extern "C" {

mvd_status mvd_batch_create(mvd_ctx* const* ctxs, int n, int n_iter, mvd_batch** out) {
    return mvd_batch_create_mode(ctxs, n, n_iter, MVD_BATCH_AUTO, out);
}

mvd_status mvd_batch_create_mode(mvd_ctx* const* ctxs, int n, int n_iter, int mode, mvd_batch** out) {
    clear_error();
    if (!out || !ctxs || n < 1 || n_iter < 0 || mode < MVD_BATCH_AUTO || mode > MVD_BATCH_BRANCHES) {
        set_error("mvd_batch_create: bad arguments");
        return MVD_ERR_ARG;
    }
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        const mvd_ctx* c = ctxs[i];
        if (!c) {
            set_error("mvd_batch_create: context %d is NULL", i);
            return MVD_ERR_ARG;
        }
        if (c->state < 2 || !c->views_ok) {
            set_error("mvd_batch_create: context %d is not precomputed or holds rejected views", i);
            return MVD_ERR_STATE;
        }
        if (c->device != ctxs[0]->device || c->stream != ctxs[0]->stream) {
            set_error("mvd_batch_create: all contexts must share one device and one stream");
            return MVD_ERR_ARG;
        }
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) {
                set_error("mvd_batch_create: context %d appears twice", i);
                return MVD_ERR_ARG;
            }
    }
    bool all_fft = true, any_weights = false;
    for (int i = 0; i < n; ++i) {
        all_fft = all_fft && ctxs[i]->path == MVD_PATH_FFT;
        any_weights = any_weights || ctxs[i]->d_w != nullptr || ctxs[i]->lambda != 0.f || ctxs[i]->boundary != 0;
    }
    const bool branches_ok = ctxs[0]->stream != nullptr && !profiling_on();
    if (mode == MVD_BATCH_AUTO) mode = branches_ok ? MVD_BATCH_BRANCHES : MVD_BATCH_PERSISTENT;
    if (mode == MVD_BATCH_PERSISTENT && any_weights) {
        set_error("mvd_batch_create: the persistent kernel applies neither view weights, regularisation nor the "
                  "zero boundary");
        return MVD_ERR_UNSUPPORTED;
    }
    if (mode == MVD_BATCH_PERSISTENT && !all_fft) {
        set_error("mvd_batch_create: the persistent kernel needs every context on the FFT engine");
        return MVD_ERR_UNSUPPORTED;
    }
    if (mode == MVD_BATCH_BRANCHES && !branches_ok) {
        set_error("mvd_batch_create: graph branches need a non-NULL stream and per-kernel timing off");
        return MVD_ERR_UNSUPPORTED;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (ctxs[0]->device != prev) cudaSetDevice(ctxs[0]->device);
    mvd_batch* b = new mvd_batch();
    b->device = ctxs[0]->device;
    b->stream = ctxs[0]->stream;
    b->n = n;
    b->n_iter = n_iter;
    b->mode = mode;
    auto fail = [&](mvd_status st) {
        batch_free(b);
        if (prev >= 0 && prev != ctxs[0]->device) cudaSetDevice(prev);
        return st;
    };
    if (mode == MVD_BATCH_BRANCHES) {
        const mvd_status st = capture_branches(b, ctxs);
        if (st != MVD_OK) return fail(st);
        if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
        *out = b;
        return MVD_OK;
    }

    std::vector<VolDesc> vols(n);
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
        const mvd_ctx* c = ctxs[i];
        const FftGeom& g = c->geom;
        VolDesc& d = vols[i];
        d.X = g.X;
        d.Y = g.Y;
        d.Z = g.Z;
        d.Xh = g.Xh;
        d.nv = c->nv;
        d.YZ = g.YZ;
        d.M = c->M;
        d.px = g.px;
        d.py = g.py;
        d.pz = g.pz;
        d.psi = c->d_psi;
        d.views = c->d_views;
        d.S = c->d_S;
        d.K = c->d_K;
        d.eps = c->eps;
        d.fx = g.fast && batch_fast_len(g.X);
        d.fy = g.fast && batch_fast_len(g.Y);
        d.fz = g.fast && batch_fast_len(g.Z);
        d.precise = c->precise;
        d.S2 = c->d_S2;
        d.KP2 = c->d_KP2;
        d.tw2x = g.tw2x;
        d.tw2y = g.tw2y;
        d.tw2z = g.tw2z;
        smem = std::max({smem, d.fx ? fast_x_smem(g.X) : gen_x_smem(g.X), d.fy ? fast_y_smem(g.Y) : gen_y_smem(g.Y),
                         d.fz ? fast_z_smem(g.Z) : gen_z_smem(g.Z, g.Y)});
        if (d.precise)
            smem = std::max({smem, d.fx ? ddf_ratio_smem(g.X) : dd_x_smem(g.X), d.fy ? ddf_y_smem(g.Y) : dd_y_smem(g.Y),
                             d.fz ? ddf_z_smem(g.Z) : dd_z_smem(g.Z, g.Y)});
    }
    // Entries (default schedule: views 0..nv-1 per iteration). Each volume's
    // own entries stay in order; across volumes they are merged by the
    // fraction of the volume's work done at the entry's midpoint, so that
    // every stretch of the queue holds passes of all volumes (volumes with
    // few views or small passes do not queue behind the others' last views).
    struct Pending {
        double key;
        int vol;
        Entry e;
    };
    std::vector<Pending> pend;
    for (int i = 0; i < n; ++i) {
        std::vector<Entry> own;
        std::vector<double> work;
        unsigned long long done_i = 0;
        double total_i = 0.0;
        for (int it = 0; it < n_iter; ++it)
            for (int s = 0; s < vols[i].nv; ++s)
                for (int p = 0; p < NPASS; ++p) {
                    long nt = 0, el = 0;
                    pass_tiles(vols[i], p, &nt, &el);
                    // a task covers several small tiles (about 16K elements of work)
                    const int tpt = (int)std::min(8L, std::max(1L, 16384 / std::max(1L, el)));
                    own.push_back({0, done_i, i, p, s, (int)nt, tpt});
                    work.push_back((double)nt * (double)el);
                    total_i += (double)nt * (double)el;
                    done_i += (unsigned long long)nt;
                }
        double cum = 0.0;
        for (size_t k = 0; k < own.size(); ++k) {
            pend.push_back({(cum + 0.5 * work[k]) / std::max(total_i, 1.0), i, own[k]});
            cum += work[k];
        }
    }
    std::stable_sort(pend.begin(), pend.end(), [](const Pending& a, const Pending& b) {
        return a.key < b.key || (a.key == b.key && a.vol < b.vol);
    });
    std::vector<Entry> entries;
    entries.reserve(pend.size());
    long task = 0;
    for (const Pending& q : pend) {
        Entry e = q.e;
        e.begin = task;
        task += gen_div_up((long)e.ntiles, (long)e.tpt);
        entries.push_back(e);
    }
    b->n_entries = (int)entries.size();
    b->total = task;
    b->smem = smem;
    const char* pl = std::getenv("MVD_BATCH_POLL_LIMIT");
    b->poll_limit = pl ? std::atoll(pl) : (1LL << 21);  // about 1-2 s of polling
    // test hook: MVD_BATCH_STALL_ENTRY=k makes entry k wait for a count no
    // task will ever reach, so its wait runs out (failure detection test)
    const char* stall = std::getenv("MVD_BATCH_STALL_ENTRY");
    if (stall && b->n_entries > 0) {
        const int k = std::atoi(stall);
        if (k >= 0 && k < b->n_entries) entries[k].target = ~0ull;
    }
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_vols, sizeof(VolDesc) * n)) != cudaSuccess) return fail(cuda_status(e, "batch descriptors"));
    if ((e = cudaMalloc(&b->d_entries, sizeof(Entry) * std::max<size_t>(1, entries.size()))) != cudaSuccess)
        return fail(cuda_status(e, "batch entries"));
    if ((e = cudaMalloc(&b->d_counters, sizeof(unsigned long long) * (n + 1))) != cudaSuccess)
        return fail(cuda_status(e, "batch counters"));
    if ((e = cudaMalloc(&b->d_error, sizeof(int))) != cudaSuccess) return fail(cuda_status(e, "batch flag"));
    e = cudaMemcpyAsync(b->d_vols, vols.data(), sizeof(VolDesc) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !entries.empty())
        e = cudaMemcpyAsync(b->d_entries, entries.data(), sizeof(Entry) * entries.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail(cuda_status(e, "batch tables"));
    e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(cuda_status(e, "batch kernel attributes"));
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kGenThreads, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return fail(cuda_status(e, "batch occupancy"));
    b->grid = std::max(1, per_sm) * sms;
    // one persistent launch (plus two counter resets) captured as a graph
    if (b->stream != nullptr) {
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail(cuda_status(e, "batch capture"));
        const unsigned long long before = g_launches.load();
        mvd_status st = enqueue(b);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->stream, &graph);
        g_launches.fetch_sub(g_launches.load() - before);
        if (st != MVD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return fail(st);
        }
        if (e != cudaSuccess) return fail(cuda_status(e, "batch capture end"));
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(cuda_status(e, "batch graph"));
    }
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    *out = b;
    return MVD_OK;
}

mvd_status mvd_batch_run(mvd_batch* b) {
    clear_error();
    if (!b) {
        set_error("mvd_batch_run: NULL batch");
        return MVD_ERR_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    mvd_status st = MVD_OK;
    if (b->exec) {
        cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
        if (e != cudaSuccess)
            st = cuda_status(e, "mvd_batch_run: graph launch");
        else
            count_launch(b->mode == MVD_BATCH_BRANCHES ? b->graph_nodes : 1);
    } else {
        st = enqueue(b);
    }
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return st;
}

mvd_status mvd_batch_wait(mvd_batch* b) {
    clear_error();
    if (!b) {
        set_error("mvd_batch_wait: NULL batch");
        return MVD_ERR_ARG;
    }
    int flag = 0;
    if (b->d_error) MVD_CUDA(cudaMemcpyAsync(&flag, b->d_error, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    MVD_CUDA(cudaStreamSynchronize(b->stream));
    if (flag) {
        set_error("mvd_batch_wait: a block gave up waiting for a dependency (poll limit %lld)", b->poll_limit);
        return MVD_ERR_TIMEOUT;
    }
    return MVD_OK;
}

long long mvd_batch_tasks(const mvd_batch* b) {
    if (!b) return 0;
    return b->mode == MVD_BATCH_BRANCHES ? (long long)b->graph_nodes : b->total;
}

int mvd_batch_mode(const mvd_batch* b) { return b ? b->mode : -1; }

void mvd_batch_destroy(mvd_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
}

}  // extern "C"
