// Brushing and linking (Sec. 3.5): the cells selected by a pixel ROI of the
// plot are one run [first, last] of the curve order; the linked 3D view tests
// cells against ROIs given as inclusive ranges of curve keys.  Both selections
// are written as a byte mask over the cells in the caller's input order
// (mask[perm[k]] for the k-th cell of the curve order).
#include <cuda_runtime.h>
#include <stdint.h>

#include "dvl_internal.h"

namespace dvl {

namespace {

constexpr uint32_t MAX_RANGES = MAX_SELECT_RANGES;

// mask[perm[k]] = 1 for k in [first, last] (the mask is cleared before).
__global__ void k_roi_mask(const uint32_t* __restrict__ perm, uint64_t first, uint64_t last, uint8_t* mask)
{
    for (uint64_t k = first + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k <= last;
         k += (uint64_t)gridDim.x * blockDim.x)
        mask[perm[k]] = 1;
}

// mask[perm[k]] = 1 if keys[k] lies in one of the R inclusive ranges.
__global__ __launch_bounds__(256) void k_select_keys(const unsigned long long* __restrict__ keys,
                                                     const uint32_t* __restrict__ perm, uint64_t n,
                                                     const unsigned long long* __restrict__ ranges, uint32_t R,
                                                     uint8_t* mask)
{
    __shared__ unsigned long long s_r[2 * MAX_RANGES];
    for (uint32_t i = threadIdx.x; i < 2 * R; i += blockDim.x) s_r[i] = ranges[i];
    __syncthreads();
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[k];
        uint8_t sel = 0;
        for (uint32_t r = 0; r < R; ++r) sel |= (key >= s_r[2 * r] && key <= s_r[2 * r + 1]) ? 1 : 0;
        mask[perm[k]] = sel;
    }
}

unsigned grid_for(uint64_t work)
{
    uint64_t b = (work + 255) / 256;
    if (b > 148ull * 16) b = 148ull * 16;
    return b ? (unsigned)b : 1u;
}

}  // namespace

cudaError_t launch_roi_mask(cudaStream_t s, const uint32_t* perm, uint64_t n, uint64_t first, uint64_t last,
                            uint8_t* mask)
{
    cudaError_t e = cudaMemsetAsync(mask, 0, n, s);
    if (e != cudaSuccess || n == 0 || last < first) return e;
    k_roi_mask<<<grid_for(last - first + 1), 256, 0, s>>>(perm, first, last, mask);
    return cudaGetLastError();
}

cudaError_t launch_select_keys(cudaStream_t s, const unsigned long long* keys, const uint32_t* perm, uint64_t n,
                               const unsigned long long* ranges, uint32_t R, uint8_t* mask)
{
    if (n == 0) return cudaSuccess;
    if (R > MAX_RANGES) return cudaErrorInvalidValue;
    k_select_keys<<<grid_for(n), 256, 0, s>>>(keys, perm, n, ranges, R, mask);
    return cudaGetLastError();
}

}  // namespace dvl
