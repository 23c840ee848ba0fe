// Internal declarations shared by the host orchestration (dvl_api.cu) and the
// kernels (sfc_sort.cu, update.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/dvl.h"

namespace dvl {

// ---- update geometry -------------------------------------------------------
// One warp owns a chunk of CHUNK consecutive cells (curve order); a CTA of
// WARPS warps owns one tile of the device-wide prefix scan.  A lane handles 4
// consecutive cells per step (one float4 per field, one u32 of levels).
constexpr int WARPS = 8;
constexpr int CHUNK = 2048;
constexpr int STEP = 128;                 // cells per warp step (32 lanes x 4)
constexpr int STEPS = CHUNK / STEP;
constexpr int TILE = WARPS * CHUNK;       // 16384 cells
constexpr int PAD = 2048;                 // field/level arrays padded to a chunk

// Position of cell i in the per-cell TF entry rows.  Each chunk of CHUNK
// cells is kept piece-major: its STEPS warp steps of STEP cells are cut into
// 4 pieces of 32 cells, and piece p of every step is stored before piece
// p + 1 of any (position p * 32 * STEPS + s * 32 + j for cell s * STEP +
// p * 32 + j of the chunk).  A run of 512 positions then holds one piece of
// each of the chunk's 16 steps, so a warp reading 16 bytes a lane sees the
// same step in lanes 2 s and 2 s + 1 from one such run to the next, while a
// step's cells still fill whole 32-byte sectors.  Pieces of 32 cells (and so
// every aligned group of 4 or 16) stay contiguous.
__host__ __device__ __forceinline__ uint64_t ent_pos(uint64_t i)
{
    static_assert(CHUNK == 2048 && STEP == 128, "entry layout: 16 steps of 4 pieces a chunk");
    return (i & ~(uint64_t)(CHUNK - 1)) | ((i >> 5) & 3u) << 9 | ((i >> 7) & 15u) << 5 | (i & 31u);
}

// ---- radix sort geometry ---------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_KPT = 16;                // keys per thread
constexpr int RS_TILE = RS_THREADS * RS_KPT;   // 4096 keys per tile
constexpr int RS_BITS = 8;
constexpr int RS_RADIX = 1 << RS_BITS;

// ---- device error bits (dvl_ctx::d_err) -------------------------------------
enum : uint32_t {
    ERR_TIMEOUT = 1u,       // a bounded wait gave up
    ERR_RANGE = 2u,         // width bound not representable / bad input value
    ERR_LEVEL = 4u,         // cell level too high
    ERR_COORD = 8u,         // cell outside the logical grid
    ERR_NONFINITE = 16u,    // non-finite field value
};

// Per-update constants, written on the device by k_prepare / k_consts and
// read by the update kernels.  Plain struct (also copied back for stats).
struct UpdateConsts {
    float lo[DVL_MAX_FIELDS];     // TF domain lower bound per field
    float s[DVL_MAX_FIELDS];      // float32 reciprocal of the domain span (0 if empty)
    float vmax, inv_vmax, f_upper, qscale;   // qscale = 2^Q
    float P, min_imp;
    int32_t Q, i, j, pow_n2;      // pow_n2 = 2P if exact mode, else -1
    int32_t min_imp_mode, width_shift;       // width_shift = 1 (2^L) or 3 (8^L)
    int32_t linear, pad0;
    uint64_t F;                   // total width, set by the last scan tile
    uint64_t F_div_W, F_mod_W;    // F = F_div_W * W + F_mod_W (for pixel bounds)
};

// Data-set metadata computed on the device at load time.
struct DataMeta {
    uint32_t dmin[DVL_MAX_FIELDS];   // order-preserving bits of the data min
    uint32_t dmax[DVL_MAX_FIELDS];
    uint32_t max_level;
    uint32_t pad;
    unsigned long long key_or;       // OR of all keys (significant bits)
    uint32_t dpos[DVL_MAX_FIELDS];   // bits of the smallest positive value (0xFFFFFFFF: none)
};

}  // namespace dvl

// ---- kernel launchers (all asynchronous on `s`) -----------------------------
namespace dvl {

// sfc_sort.cu
void launch_validate(cudaStream_t s, uint64_t n, const int32_t* lower, const uint8_t* level,
                     uint32_t M, float* const* fields, size_t pitch, DataMeta* meta, uint32_t* err);
// Per-field min/max into meta->dmin/dmax; with `positive` also the smallest
// positive value into meta->dpos (the clamp of the log scale).
void launch_field_ranges(cudaStream_t s, uint64_t n, uint32_t M, const float* fields, size_t pitch,
                         DataMeta* meta, uint32_t* err, bool positive = false);
void launch_keys(cudaStream_t s, uint64_t n, const int32_t* lower, size_t pitch, const uint8_t* level,
                 int sfc, unsigned long long* keys, uint32_t* vals, uint32_t* hist /*8*256*/,
                 DataMeta* meta);
// One stable LSD pass over digit (key >> shift) & 255.  `status` holds
// n_tiles*256 words tagged with `epoch` (never cleared between passes).
cudaError_t launch_onesweep(cudaStream_t s, uint64_t n, const unsigned long long* kin,
                            const uint32_t* vin, unsigned long long* kout, uint32_t* vout,
                            int shift, const uint32_t* hist_digit, unsigned long long* status,
                            uint32_t epoch, uint32_t* tile_counter, uint32_t* err, int64_t spin_limit);
// fout[m][k] = fin[m][perm[k]]; a field whose bit is set in log_mask is
// stored as its log10 scale (logscale.cuh), values <= 0 taking meta->dpos[m].
void launch_gather(cudaStream_t s, uint64_t n, const uint32_t* perm, uint32_t M, const float* fin,
                   size_t pitch_in, const uint8_t* lin, float* fout, size_t pitch_out, uint8_t* lout,
                   uint32_t log_mask = 0, const DataMeta* meta = nullptr);

// bins.cu: TF-independent value tables (per data set and TF domain) and the
// per-pixel range queries that replace the placement pass.
//
// Per field, over steps of STEP cells grouped in blocks of VT_BLOCK steps:
// the fixed-point sum of t = floor(t * 2^95) of every step as an exclusive
// prefix within its block (loc) plus an exclusive prefix over the blocks
// (blk), so the prefix up to step s is blk[s / VT_BLOCK] + loc[s]; and the
// (min, max) of t per step (raw), over the block's steps up to and including
// it (pre) and from it to the block's end (suf), with a sparse table of the
// blocks' (min, max) over power-of-two runs of blocks (bmm).
constexpr int VT_BLOCK = 32;
struct ValueTableArgs {
    uint64_t n;
    const float* val;          // M x pitch, curve order
    size_t pitch;
    const UpdateConsts* consts;   // lo / s of the domains the tables are built for
    uint64_t n_steps;          // ceil(n / STEP)
    uint64_t n_blocks;         // ceil(n_steps / VT_BLOCK)
    ulonglong2* loc;           // M x (n_steps + 1), u128 as (lo, hi)
    ulonglong2* blk;           // M x (n_blocks + 1), u128 as (lo, hi)
    float2* raw;               // M x n_steps
    float2* pre;               // M x n_steps
    float2* suf;               // M x n_steps
    float2* bmm;               // M x b_levels x n_blocks: level l, entry i = blocks [i, i + 2^l)
    int b_levels;              // floor(log2(n_blocks)) + 1 (0 when there are no blocks)
    ulonglong2* seg;           // M x ceil(n_blocks / 2048): segment sums of blk, then their prefixes
    uint8_t* ent;              // if not null: the cells' TF entries are written in the same pass
    uint32_t T;                //   (UpdateArgs::ent; T <= 256 entries)
    uint32_t* err;             // error word (ERR_TIMEOUT when a bounded wait runs out)
};
struct QueryArgs {
    const UpdateConsts* consts;
    const unsigned long long* chunk_prefix;
    const unsigned long long* step_sums;
    unsigned long long* H;     // W + 1: cells whose span starts before pixel j's first position
    uint8_t* S;                // W + 1: the last of them also touches pixel j
    // Per boundary j and field m, the partial-step terms of its two pixels
    // over the 128-cell step holding cell H(j)-1: side 0 = cells of that step
    // before H(j) (pixel j-1's tail), side 1 = cells from pixel j's first cell
    // to the step's end (its head).  Index ((j * 2 + side) * M + m).
    ulonglong2* psum;          // fixed-point sums of t (lo, hi words)
    float2* pmm;               // min, max of t (3, -1 if empty)
    // The pixel queries read boundary j of these arrays at j * hstride: a
    // width that divides a wider one of the same scan shares its boundaries
    // (ceil(j F / W) = ceil(r j F / (r W))), so it reads every r-th entry.
    uint32_t hstride;
    // Alpha means (null when not asked for): pass A's per-step and per-chunk
    // sums of the cells' fixed-point alpha (see UpdateArgs::astep) and, per
    // boundary, the two partial-step sums (index as psum).
    const unsigned long long* astep;
    const unsigned long long* achunk;
    unsigned long long* apart;
    uint64_t a_chunks;         // chunks per field row of astep / achunk (pass A's count)
};
// Sparse-table levels over n_blocks blocks: floor(log2(n_blocks)) + 1.
int value_table_levels(uint64_t n_blocks);
uint64_t value_table_segments(uint64_t n_blocks);

// update.cu
struct UpdateArgs {
    uint64_t n;
    uint32_t M, T, W;
    const float* val;          // M x pitch, curve order
    size_t pitch;
    const uint8_t* lev;        // pitch bytes, curve order
    const float* tf;           // M x T alpha tables
    const float* dom;          // 2*M: lo[M], hi[M]  (NaN,NaN = data range)
    const DataMeta* meta;
    UpdateConsts* consts;
    unsigned long long* tile_status;   // n_tiles scan status words
    unsigned long long* chunk_prefix;  // n_chunks
    unsigned long long* step_sums;     // n_chunks * STEPS width totals per warp step, or
                                       // null (then the placement pass recomputes widths)
    uint32_t* counters;        // [0] tile ticket, [1] tiles done
    double* sum;               // M x W
    uint32_t* vmin;            // M x W (float bits)
    uint32_t* vmax;            // M x W (float bits)
    uint32_t* count;           // W
    float* mean;               // M x W
    float* y;                  // M x W
    double* asum;              // M x W alpha sums, or null (no alpha means)
    float* amean;              // M x W alpha means (when asum)
    // Alpha means in the same read of the cells as the widths: pass A adds the
    // cells' alpha per field in fixed point, a_fx = rint(alpha 2^29), per warp
    // step (astep: M x n_chunks * STEPS, the exclusive prefix of the steps
    // within their chunk) and per chunk (achunk: M x (n_chunks + 1), turned
    // into the exclusive prefix over chunks by the chunk scan); apart holds
    // the pixel boundaries' partial-step sums ((W + 1) x 2 x M).  Null: no
    // alpha sums are asked for.
    unsigned long long* astep;
    unsigned long long* achunk;
    unsigned long long* apart;
    uint32_t* err;
    int64_t spin_limit;
    int fault_no_publish;
    dvl_params prm;
    cudaEvent_t* events;       // 5 events recorded between the stages, or null
    // range-query bins (null vt: the placement pass k_passB* is used instead)
    const ValueTableArgs* vt;
    int vt_build;              // rebuild the value tables after k_prepare
    // Per-cell TF entries for the current TF domains and T <= 256, M rows of
    // pitch bytes at positions ent_pos(c): entry m of cell c = min(floor(t T),
    // T - 1) (the alpha-table index of Sec. 3.3's normalised value), and in
    // row M the cells' levels at the same positions.  They depend on the data,
    // the domains and T only (the level row on the data only), so pass A
    // streams them (M + 1 bytes a cell) instead of the field values.  Null:
    // pass A reads the fields.
    uint8_t* ent;
    int ent_build;             // rebuild the entries after k_prepare
    int ent_lev_build;         // rewrite the level row (new data set)
    unsigned long long* H;
    uint8_t* S;
    ulonglong2* psum;          // boundary partial sums (see QueryArgs)
    float2* pmm;
};
// Batched updates: K transfer functions x V viewports.
constexpr uint32_t MAX_BATCH_TF = DVL_MAX_BATCH_TF;
struct PairDesc {              // one (TF, viewport) pair of a batch
    uint32_t k, W;
    uint64_t bin_off;          // element offset of its M x W bin arrays
    uint64_t cnt_off;          // element offset of its W counts
    uint64_t hs_off;           // element offset of its W + 1 pixel bounds
    uint64_t src_hs_off;       // bounds its pixels read: its own, or those of a
    uint32_t hstride;          //   wider pair of the same TF (every hstride-th)
    uint32_t derived;          // 1: its bounds are not computed (src is another pair)
};
struct BatchArgs {
    uint32_t K, G;             // TFs, TFs per shared-memory group of pass A
    const float* tfs;          // K x M x T alpha tables
    UpdateConsts* consts;      // K
    unsigned long long* tile_status;   // K x n_tiles
    unsigned long long* chunk_prefix;  // K x n_chunks
    unsigned long long* step_sums;     // K x n_chunks x STEPS
    uint64_t n_tiles, n_chunks;
    const PairDesc* pairs;     // device, n_pairs
    uint32_t n_pairs, max_W;
    double* sum;
    uint32_t* vmin;
    uint32_t* vmax;
    float* mean;
    float* y;
    uint32_t* count;
    unsigned long long* H;
    uint8_t* S;
    ulonglong2* psum;          // 2 x M per pixel bound (offset hs_off * 2 * M)
    float2* pmm;
    uint32_t* tickets;         // 2K + 1, zeroed per batch: [1 + k] TF k's chunk-scan block
                               // counter, [1 + K + g] pass A's chunk counter of TF group g
    int resid;                 // pass A CTAs per SM (persistent grid)
    int sm_count;
    // Device clock (%globaltimer, ns) of the batch's execution: [0] when the
    // first kernel started, [1] when the last of its pixel-query blocks ended.
    unsigned long long* stamps;
};
// The stamps of the last batch of a context (device memory, 2 words).
const unsigned long long* batch_stamps(const dvl_ctx* c);
cudaError_t launch_prepare_batch(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b);
cudaError_t launch_passA_batch(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b);
// Resident pass-A batch CTAs per SM for groups of G tables (0 = does not fit).
cudaError_t passA_batch_occupancy(const UpdateArgs& a, uint32_t G, int* blocks);
cudaError_t launch_bins_batch(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b, const ValueTableArgs& v);

cudaError_t launch_value_tables(cudaStream_t s, uint32_t M, const ValueTableArgs& v);
cudaError_t launch_bins(cudaStream_t s, const UpdateArgs& a, const QueryArgs& qa, const ValueTableArgs& v);
cudaError_t launch_update(cudaStream_t s, const UpdateArgs& a);
// Load the per-edit kernels of M fields into the current context ahead of
// their first launch (update.cu: widths and scan; bins.cu: value tables and
// pixel queries).
cudaError_t preload_update_kernels(uint32_t M);
// The per-cell TF entries (a.ent) for the domains of a.consts and T = a.T.
cudaError_t launch_entries(cudaStream_t s, const UpdateArgs& a);
cudaError_t preload_bins_kernels(uint32_t M);
// Alpha tables from control points (M x K -> M x T), flags values outside [0,1].
cudaError_t launch_ctrl_table(cudaStream_t s, uint32_t M, uint32_t K, uint32_t T, const float* ctrl, float* tf,
                              uint32_t* err);
// Adjoint of the alpha means of the last update: gtab (M x T, zeroed by the
// caller) += per (cell, pixel) g[m][p] / count[p] at the cell's entry; then
// grad_ctrl (M x K) = gtab through the interpolation weights.
// gpart: scratch of backward_gpart_elems(M, T, n) doubles for the histogram
// adjoint (deterministic, no global atomics), or null for the atomic one.
cudaError_t launch_backward(cudaStream_t s, const UpdateArgs& a, const float* g, double* gtab, uint32_t K,
                            float* grad_ctrl, double* gpart);
size_t backward_gpart_elems(uint32_t M, uint32_t T, uint64_t n, uint32_t W);   // 0: tables too large for it
cudaError_t launch_widths(cudaStream_t s, const UpdateArgs& a, unsigned long long* q);

// raster.cu: line-plot image of M x W bin values (lines: bit m per field,
// bars of one field), H x W bytes each, row-major; either may be null.
cudaError_t launch_raster(cudaStream_t s, const float* values, uint32_t M, uint32_t W, uint32_t H,
                          uint32_t bar_field, uint8_t* lines, uint8_t* bars);

// select.cu: brushing and linking masks over the cells in input order.
constexpr uint32_t MAX_SELECT_RANGES = 1024;
cudaError_t launch_roi_mask(cudaStream_t s, const uint32_t* perm, uint64_t n, uint64_t first, uint64_t last,
                            uint8_t* mask);
cudaError_t launch_select_keys(cudaStream_t s, const unsigned long long* keys, const uint32_t* perm, uint64_t n,
                               const unsigned long long* ranges, uint32_t R, uint8_t* mask);

// Opts a kernel in to `bytes` of dynamic shared memory.  Always set: the
// 48 KB default covers static plus dynamic memory, and several kernels have
// static arrays of their own.
template <typename K>
cudaError_t smem_attr(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Sets a kernel's dynamic shared-memory limit once per device and size: the
// batched launches are also recorded into CUDA graphs, where the call is
// avoided by setting the limit on the first uncaptured launch.  `cache` holds
// the largest size set so far per device (one cache per kernel).
constexpr int MAX_DEVICES = 64;
template <typename K>
cudaError_t smem_attr_once(K kernel, size_t bytes, std::atomic<size_t> (&cache)[MAX_DEVICES])
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return smem_attr(kernel, bytes);
    if (bytes <= cache[dev].load(std::memory_order_relaxed)) return cudaSuccess;
    e = smem_attr(kernel, bytes);
    if (e == cudaSuccess) cache[dev].store(bytes, std::memory_order_relaxed);
    return e;
}

// Dispatch on the field count of `a` to fn<1..8>(...).
#define DVL_DISPATCH_M(fn, ...)                   \
    switch (a.M) {                                \
        case 1: return fn<1>(__VA_ARGS__);        \
        case 2: return fn<2>(__VA_ARGS__);        \
        case 3: return fn<3>(__VA_ARGS__);        \
        case 4: return fn<4>(__VA_ARGS__);        \
        case 5: return fn<5>(__VA_ARGS__);        \
        case 6: return fn<6>(__VA_ARGS__);        \
        case 7: return fn<7>(__VA_ARGS__);        \
        case 8: return fn<8>(__VA_ARGS__);        \
        default: return cudaErrorInvalidValue;    \
    }

}  // namespace dvl
