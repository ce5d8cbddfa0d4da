// Warp-cooperative sums over small 3D boxes of kernel offsets (compound-kernel
// algebra and its vector-Jacobian product): one warp per output value.
#pragma once

#include <cuda_runtime.h>

namespace mvd {

// Sum over the box [xlo,xhi] x [ylo,yhi] x [zlo,zhi] of the terms that
// f(ex, ey, ez, acc) adds to acc (one FMA each), by one warp: lanes stride
// over the flattened (ey, ex) plane (stepped incrementally, no division in the
// loop), z runs serially; the lanes' partial sums are combined with shuffles.
// Every lane of the warp must call it and every lane returns the total.
template <typename F>
__device__ __forceinline__ float warp_box_sum(int xlo, int xhi, int ylo, int yhi, int zlo, int zhi, F&& f) {
    const int lane = threadIdx.x & 31;
    const int nx = xhi - xlo + 1, ny = yhi - ylo + 1;
    float s = 0.f;
    if (nx > 0 && ny > 0) {
        const int n2 = nx * ny;
        for (int ez = zlo; ez <= zhi; ++ez) {
            int ey = ylo + lane / nx, ex = xlo + lane % nx;
            for (int i = lane; i < n2; i += 32) {
                s = f(ex, ey, ez, s);
                ex += 32;
                while (ex > xhi) {
                    ex -= nx;
                    ++ey;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

}  // namespace mvd
