// Allocation-free view update (mvd_update_direct_noalloc).
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// owned by a caching allocator that must see every allocation (a raw
// cudaMalloc or cudaFree also synchronises the whole device), and acquisition
// loops that allocate everything at start-up and must not allocate while
// frames stream in. For them this entry point runs one view update with the
// direct engine without allocating: the caller passes every input and output,
// and the one intermediate the update needs (the ratio r = phi / max(psi * P,
// eps)) lives in the file-scope device array below.
//
// Host code never takes the array's address directly: in host code its name
// is a host-side stand-in, not a device address. The device address is
// fetched once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on that device.
#include <mutex>

#include "common.cuh"

namespace {

// Ratio scratch shared by every call on a device; every GPU that loads the
// library holds it (8 MiB) until the process exits.
constexpr long kNoAllocMaxVoxels = 2L * 1024 * 1024;
__device__ __align__(256) float g_noalloc_ratio[kNoAllocMaxVoxels];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float* g_ratio_ptr[kMaxDevices] = {nullptr};

mvd_status ratio_scratch(float** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mvd::cuda_status(e, "mvd_update_direct_noalloc: current device");
    if (dev < 0 || dev >= kMaxDevices) {
        mvd::set_error("mvd_update_direct_noalloc: device %d out of range", dev);
        return MVD_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_ratio_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_ratio);
        if (e != cudaSuccess) return mvd::cuda_status(e, "mvd_update_direct_noalloc: cudaGetSymbolAddress");
        g_ratio_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_ratio_ptr[dev];
    return MVD_OK;
}

}  // namespace

extern "C" mvd_status mvd_update_direct_noalloc(float* psi, const float* phi, const float* psf, const float* comp,
                                                const int dims[3], const int kdims[3], float eps, void* stream) {
    mvd::clear_error();
    if (!psi || !phi || !psf || !comp || !dims || !kdims) {
        mvd::set_error("mvd_update_direct_noalloc: NULL argument");
        return MVD_ERR_ARG;
    }
    if (!(eps > 0.f)) {
        mvd::set_error("mvd_update_direct_noalloc: eps must be > 0");
        return MVD_ERR_ARG;
    }
    long M = 1;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || kdims[a] < 1 || kdims[a] % 2 == 0 || kdims[a] > dims[a]) {
            mvd::set_error("mvd_update_direct_noalloc: bad sizes on axis %d (volume %d, kernel %d)", a, dims[a],
                           kdims[a]);
            return MVD_ERR_SHAPE;
        }
        M *= dims[a];
    }
    if (M > kNoAllocMaxVoxels) {
        mvd::set_error("mvd_update_direct_noalloc: volume has %ld voxels, the allocation-free scratch holds at most %ld",
                       M, kNoAllocMaxVoxels);
        return MVD_ERR_SHAPE;
    }
    if (!mvd::direct_supported(kdims)) {
        mvd::set_error("mvd_update_direct_noalloc: kernel box %dx%dx%d too large for the direct engine", kdims[0],
                       kdims[1], kdims[2]);
        return MVD_ERR_UNSUPPORTED;
    }
    // every buffer must be device (or managed) memory of the current device:
    // the scratch below is this device's, and the kernels read X*Y*Z and
    // Kx*Ky*Kz floats behind the pointers
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mvd::cuda_status(e, "mvd_update_direct_noalloc: current device");
    const void* bufs[4] = {psi, phi, psf, comp};
    const char* names[4] = {"psi", "phi", "psf", "comp"};
    for (int i = 0; i < 4; ++i) {
        cudaPointerAttributes at{};
        e = cudaPointerGetAttributes(&at, bufs[i]);
        if (e != cudaSuccess) {
            cudaGetLastError();
            mvd::set_error("mvd_update_direct_noalloc: %s is not a CUDA pointer", names[i]);
            return MVD_ERR_ARG;
        }
        const bool ok = (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
        if (!ok) {
            mvd::set_error("mvd_update_direct_noalloc: %s is not device memory of the current device %d", names[i],
                           dev);
            return MVD_ERR_ARG;
        }
    }
    float* r = nullptr;
    MVD_TRY(ratio_scratch(&r));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // r is written in full before it is read, so nothing needs clearing
    MVD_TRY(mvd::direct_ratio(dims, psi, psf, kdims, phi, eps, r, st));
    return mvd::direct_update(dims, r, comp, kdims, psi, eps, st);
}
