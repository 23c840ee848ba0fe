// Line-plot rasterisation of the bins (the RasterizeLines step after the
// update, Sec. 4, Fig. 1): a headless H x W image per call, row 0 at the top,
// column p = bin p.  A bin value v in [0, 1] (mean of the normalised values,
// or its alpha) maps to row r = clamp(floor((1 - v)(H - 1) + 1/2), 0, H - 1)
// in correctly rounded float32 steps.  Field m's polyline covers, in column
// p, the rows between r_p and its shares of the segments to the neighbouring
// columns, r_p - trunc((r_p - r_{p-1})/2) and r_p + trunc((r_{p+1} - r_p)/2);
// bit m of lines[row][p] marks it.  bars[row][p] = 1 from r_p of the bar field
// down to the baseline.
//
// One thread per (column, block of rows): it derives its column's row range
// per field from three neighbouring bin values and writes its rows; the
// threads of a warp hold consecutive columns, so every row store is
// coalesced.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dvl_internal.h"

namespace dvl {

namespace {

constexpr int RASTER_ROWS = 32;           // rows per thread

__device__ __forceinline__ int plot_row(float v, uint32_t H)
{
    const float y = __fadd_rn(__fmul_rn(__fsub_rn(1.0f, v), (float)(H - 1)), 0.5f);
    const int r = (int)floorf(y);
    return min(max(r, 0), (int)H - 1);
}

__global__ __launch_bounds__(256) void k_raster(const float* __restrict__ val, uint32_t M, uint32_t W, uint32_t H,
                                                uint32_t bar_field, uint8_t* __restrict__ lines,
                                                uint8_t* __restrict__ bars)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= W) return;
    int lo[DVL_MAX_FIELDS], hi[DVL_MAX_FIELDS];
    int rbar = (int)H;
    for (uint32_t m = 0; m < M; ++m) {
        const float* v = val + (uint64_t)m * W;
        const int r = plot_row(v[p], H);
        int l = r, h = r;
        if (p > 0) {
            const int a = r - (r - plot_row(v[p - 1], H)) / 2;
            l = min(l, a);
            h = max(h, a);
        }
        if (p + 1 < W) {
            const int b = r + (plot_row(v[p + 1], H) - r) / 2;
            l = min(l, b);
            h = max(h, b);
        }
        lo[m] = l;
        hi[m] = h;
        if (m == bar_field) rbar = r;
    }
    const uint32_t r0 = blockIdx.y * RASTER_ROWS, r1 = min(r0 + RASTER_ROWS, H);
    for (uint32_t row = r0; row < r1; ++row) {
        uint32_t bits = 0;
        for (uint32_t m = 0; m < M; ++m)
            bits |= ((int)row >= lo[m] && (int)row <= hi[m]) ? (1u << m) : 0u;
        if (lines) lines[(uint64_t)row * W + p] = (uint8_t)bits;
        if (bars) bars[(uint64_t)row * W + p] = (int)row >= rbar ? 1 : 0;
    }
}

}  // namespace

cudaError_t launch_raster(cudaStream_t s, const float* values, uint32_t M, uint32_t W, uint32_t H,
                          uint32_t bar_field, uint8_t* lines, uint8_t* bars)
{
    if (W == 0 || H == 0) return cudaSuccess;
    const dim3 grid((W + 255) / 256, (H + RASTER_ROWS - 1) / RASTER_ROWS);
    k_raster<<<grid, 256, 0, s>>>(values, M, W, H, bar_field, lines, bars);
    return cudaGetLastError();
}

}  // namespace dvl
