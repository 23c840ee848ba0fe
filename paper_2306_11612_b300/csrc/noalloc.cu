// dvl_update_noalloc: one DVL update over caller-owned device buffers that
// never allocates device memory.
//
// Who needs it: code that may not call cudaMalloc/cudaFree at the point where
// it wants a volume-line update -- for example a render or UI callback running
// under a memory budget that another system owns, a host process that shares
// the GPU through a fixed memory pool, or a driver layer that must not
// introduce device-wide synchronisation (cudaFree synchronises the device).
// Such a caller owns its inputs and outputs; the only working memory the
// update needs beyond them (per-update constants, the prefix-scan tile states,
// the per-chunk prefix sums and the data-range words) lives here, in one
// file-scope device array of fixed size that every GPU which loads this
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "dvl_internal.h"

namespace {

using namespace dvl;

// Fixed scratch: 4 MiB.  Header (constants, data range, counters, TF domain)
// first, then 8 bytes of tile state and 8 bytes of chunk prefix per warp for
// every scan tile of TILE cells; kMaxCells is the documented cap, which fits.
constexpr size_t kScratchBytes = 4u << 20;
constexpr size_t kHeaderBytes = 4096;
constexpr size_t kPerTileBytes = 8 + 8 * WARPS;
constexpr uint64_t kMaxCells = 476749824ull;                      // documented in dvl.h
constexpr uint64_t kMaxTiles = (kMaxCells + TILE - 1) / TILE;
static_assert(kHeaderBytes + kMaxTiles * kPerTileBytes <= kScratchBytes, "scratch too small for the cap");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Header {
    DataMeta meta;
    UpdateConsts consts;
    uint32_t err;
    uint32_t counters[4];
    float dom[2 * DVL_MAX_FIELDS];
};
static_assert(sizeof(Header) <= kHeaderBytes, "scratch header too large");

// Device address of the scratch array per device, looked up once per device
// (with that device current) the first time the entry point runs there.
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_for(int device, unsigned char** out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

__global__ void k_max_level(uint64_t n, const uint8_t* __restrict__ level, DataMeta* meta)
{
    uint32_t m = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, (uint32_t)level[i]);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&meta->max_level, m);
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" int dvl_update_noalloc(void* cuda_stream, uint64_t n_cells, uint32_t n_fields,
                                  const float* fields, size_t pitch, const uint8_t* level,
                                  uint32_t n_entries, const float* alpha, const float* domain,
                                  const dvl_params* p, const dvl_bins* out)
{
    // ---- argument checks (no CUDA calls) ----
    if (!p || !out || !domain) return DVL_ERR_ARG;
    if (n_cells > kMaxCells) return DVL_ERR_RANGE;          // beyond the fixed scratch
    if (n_fields < 1 || n_fields > DVL_MAX_FIELDS) return DVL_ERR_ARG;
    if (n_entries < 2 || n_entries > DVL_MAX_TF_ENTRIES || !alpha) return DVL_ERR_ARG;
    if (p->width < 1 || p->width > DVL_MAX_WIDTH) return DVL_ERR_ARG;
    if (!(p->P >= 0.0f) || !std::isfinite(p->P) || !(p->min_importance >= 0.0f) ||
        !std::isfinite(p->min_importance) || p->min_imp_mode > 1 || p->vmax_mode > 1 || p->width_mode > 1 ||
        p->want_alpha)
        return DVL_ERR_ARG;
    if (!out->sum || !out->min || !out->max || !out->count || !out->mean || !out->y ||
        out->mem_kind != DVL_MEM_DEVICE)
        return DVL_ERR_ARG;
    if (n_cells && (!fields || !level || !aligned(fields, 16) || !aligned(level, 4) ||
                    pitch % 4 != 0 || pitch < (n_cells + 3) / 4 * 4))
        return DVL_ERR_ARG;
    for (uint32_t m = 0; m < n_fields; ++m) {
        const float lo = domain[m], hi = domain[n_fields + m];
        const bool dflt = std::isnan(lo) && std::isnan(hi);
        if (!dflt && !(std::isfinite(lo) && std::isfinite(hi) && lo < hi)) return DVL_ERR_ARG;
    }
    if (p->width > 0 && (uint64_t)n_fields * p->width > (1ull << 31)) return DVL_ERR_ARG;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return DVL_ERR_CUDA;
    unsigned char* base = nullptr;
    if (scratch_for(device, &base) != cudaSuccess) {
        cudaGetLastError();
        return DVL_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    Header* h = reinterpret_cast<Header*>(base);
    const uint64_t n_tiles = (n_cells + TILE - 1) / TILE;
    unsigned long long* tile_status = reinterpret_cast<unsigned long long*>(base + kHeaderBytes);
    unsigned long long* chunk_prefix = tile_status + kMaxTiles;

    // ---- reset the parts of the shared scratch that must start fresh ----
    uint32_t init[2 * DVL_MAX_FIELDS + 2];
    for (int m = 0; m < DVL_MAX_FIELDS; ++m) { init[m] = 0xFFFFFFFFu; init[DVL_MAX_FIELDS + m] = 0u; }
    init[2 * DVL_MAX_FIELDS] = 0u;       // max_level
    init[2 * DVL_MAX_FIELDS + 1] = 0u;
    cudaError_t e = cudaMemcpyAsync(&h->meta, init, sizeof init, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&h->err, 0, sizeof(uint32_t), s);
    float dom[2 * DVL_MAX_FIELDS];
    for (uint32_t k = 0; k < 2 * n_fields; ++k) dom[k] = domain[k];
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->dom, dom, 2 * n_fields * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { cudaGetLastError(); return DVL_ERR_CUDA; }

    // ---- data range and deepest level, then the regular update kernels ----
    launch_field_ranges(s, n_cells, n_fields, fields, pitch, &h->meta, &h->err);
    if (n_cells) {
        int blocks = (int)std::min<uint64_t>((n_cells + 255) / 256, 148ull * 8);
        k_max_level<<<blocks, 256, 0, s>>>(n_cells, level, &h->meta);
    }
    UpdateArgs a{};
    a.n = n_cells;
    a.M = n_fields;
    a.T = n_entries;
    a.W = p->width;
    a.val = fields;
    a.pitch = pitch;
    a.lev = level;
    a.tf = alpha;
    a.dom = h->dom;
    a.meta = &h->meta;
    a.consts = &h->consts;
    a.tile_status = tile_status;
    a.chunk_prefix = chunk_prefix;
    a.counters = h->counters;
    a.sum = out->sum;
    a.vmin = reinterpret_cast<uint32_t*>(out->min);
    a.vmax = reinterpret_cast<uint32_t*>(out->max);
    a.count = out->count;
    a.mean = out->mean;
    a.y = out->y;
    a.err = &h->err;
    a.spin_limit = 1 << 22;
    a.fault_no_publish = 0;
    a.prm = *p;
    a.events = nullptr;
    (void)n_tiles;
    e = launch_update(s, a);
    if (e != cudaSuccess) { cudaGetLastError(); return DVL_ERR_CUDA; }

    // ---- wait, then report device-side errors of this call ----
    uint32_t err = 0;
    e = cudaMemcpyAsync(&err, &h->err, sizeof err, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cudaGetLastError(); return DVL_ERR_CUDA; }
    if (err & ERR_TIMEOUT) return DVL_ERR_TIMEOUT;
    if (err) return DVL_ERR_RANGE;
    return DVL_OK;
}
