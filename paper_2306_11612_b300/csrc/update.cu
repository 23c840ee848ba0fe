// Per-edit stage of the DVL computation (paper Sec. 3-4), run on every alpha
// transfer-function or data change over the cells in curve order.
//
//   k_prepare   TF domains, Eq. 5/6 max-variation approximation, fixed-point
//               exponent; clears bins and scan state (one launch).
//   k_passA_ring  per cell: TF alpha per field, variation V (Eq. 1),
//               importance f (Eq. 3), fixed-point width q; width totals per
//               warp step and per chunk (and, for alpha means, the cells'
//               fixed-point alpha sums per step and chunk), each chunk's
//               totals also added into its scan block's sum; k_chunk_scan
//               then gives the exclusive prefix of every chunk and the total
//               F (Eq. 4).  k_passA: the same with direct loads and a decoupled
//               look-back per tile (rows that are not 16-byte aligned).
//   The bins are range queries over TF-independent value tables (bins.cu).
//   k_passB     places every cell into the pixels its [E, E+q) span touches
//               (Sec. 3.2), recomputing every width, with global atomics only
//               when the pixel changes or the chunk ends (used by the
//               allocation-free entry point, which keeps no value tables).
//   k_finalize  per pixel: mean = sum / count, alpha of the mean (Sec. 3.3).
//
// Widths are integers q = rint(f * 2^Q) < 2^32 with Q chosen so that the total
// stays below 2^62: the prefix sum is exact and independent of summation order,
// so the cell-to-pixel assignment is bit-identical to a sequential CPU
// evaluation.  Every float operation that decides an integer (TF entry, width)
// is a correctly rounded float32 operation (explicit __f*_r? intrinsics; this
// file is built with -fmad=false).
#include <cuda_runtime.h>
#include <stdint.h>

#include "bulk.cuh"
#include "cell_math.cuh"
#include "consts.cuh"
#include "dvl_internal.h"

namespace dvl {

namespace {
__global__ void k_prepare(UpdateArgs a, uint64_t n_status)
{
    // clear bins and scan state
    const uint64_t MW = (uint64_t)a.M * a.W;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < MW;
         i += (uint64_t)gridDim.x * blockDim.x) {
        a.sum[i] = 0.0;
        if (a.asum) a.asum[i] = 0.0;
        a.vmin[i] = 0xFFFFFFFFu;
        a.vmax[i] = 0u;
        if (i < a.W) a.count[i] = 0u;
    }
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_status;
         i += (uint64_t)gridDim.x * blockDim.x)
        a.tile_status[i] = 0ull;
    if (blockIdx.x != 0) return;
    if (threadIdx.x == 0) {
        a.counters[0] = 0u;
        a.counters[1] = 0u;
    }
    prepare_consts_block(a);
}

// Exact max V over all cells (the reduction Sec. 3.4 avoids; optional mode).
template <int M>
__global__ __launch_bounds__(256) void k_vmax_exact(UpdateArgs a)
{
    extern __shared__ float s_tf[];
    load_table<M>(s_tf, a.tf, a.T);
    __syncthreads();
    Cell<M, POW_GEN> cc;
    cc.load(a.consts, a.T);
    float best = 0.0f;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        float t[M];
#pragma unroll
        for (int m = 0; m < M; ++m) t[m] = norm_t(a.val[m * a.pitch + i], cc.lo[m], cc.s[m]);
        best = fmaxf(best, cc.variation(t, s_tf));
    }
    for (int o = 16; o; o >>= 1) best = fmaxf(best, __shfl_xor_sync(FULL, best, o));
    if ((threadIdx.x & 31) == 0 && best > 0.0f)
        atomicMax(reinterpret_cast<unsigned int*>(&a.consts->vmax), __float_as_uint(best));
}

__global__ void k_consts(UpdateArgs a) { finish_consts(a.consts, a, a.meta->max_level); }

// ---------------------------------------------------------------------------
// Pass A: widths, chunk sums, decoupled look-back scan over tiles
// ---------------------------------------------------------------------------

// Sum of the fixed-point widths of one lane's 4 cells at idx.  AL: also adds
// the cells' fixed-point alphas per field to ax (the u32 tables lie `aoff`
// bytes after the float tables).
template <int M, int PM, bool FULLSTEP, bool P2, bool AL = false>
__device__ __forceinline__ unsigned long long widths4_of(const Cell<M, PM>& cc, const UpdateArgs& a,
                                                         const float* s_tf, const uint32_t* cm, uint64_t idx,
                                                         const float (&v)[4][M], uint32_t L4, uint32_t aoff = 0,
                                                         uint32_t* ax = nullptr)
{
    unsigned long long acc = 0;
    if (P2 && PM == POW_ONE) {
        // pairs of cells in float32x2 form
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
            uint32_t axa[M], axb[M], qa, qb;
            cc.template width2_p2<AL>(v[j], v[j + 1], (L4 >> (8 * j)) & 0xFF, (L4 >> (8 * j + 8)) & 0xFF, cm, aoff,
                                      axa, axb, qa, qb);
            const bool ina = FULLSTEP || idx + j < a.n, inb = FULLSTEP || idx + j + 1 < a.n;
            if (ina) acc += qa;
            if (inb) acc += qb;
            if (AL) {
#pragma unroll
                for (int m = 0; m < M; ++m) ax[m] += (ina ? axa[m] : 0u) + (inb ? axb[m] : 0u);
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t q;
            uint32_t axj[M];
#pragma unroll
            for (int m = 0; m < M; ++m) axj[m] = 0;
            if (P2) {
                q = AL ? cc.width_p2_alpha(v[j], (L4 >> (8 * j)) & 0xFF, cm, aoff, axj)
                       : cc.width_p2(v[j], (L4 >> (8 * j)) & 0xFF, cm);
            } else {
                float t[M];
#pragma unroll
                for (int m = 0; m < M; ++m) t[m] = norm_t(v[j][m], cc.lo[m], cc.s[m]);
                q = AL ? cc.width_alpha(t, (L4 >> (8 * j)) & 0xFF, s_tf,
                                        reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(s_tf) + aoff), axj)
                       : cc.width(t, (L4 >> (8 * j)) & 0xFF, s_tf);
            }
            if (FULLSTEP || idx + j < a.n) {
                acc += q;
                if (AL) {
#pragma unroll
                    for (int m = 0; m < M; ++m) ax[m] += axj[m];
                }
            }
        }
    }
    return acc;
}

template <int M, int PM, bool FULLSTEP, bool P2, bool AL = false>
__device__ __forceinline__ unsigned long long widths4(const Cell<M, PM>& cc, const UpdateArgs& a,
                                                      const float* s_tf, const uint32_t* cm, uint64_t idx,
                                                      uint32_t aoff = 0, uint32_t* ax = nullptr)
{
    float v[4][M];
    uint32_t L4;
    load4<M>(a.val, a.pitch, a.lev, idx, v, L4);
    return widths4_of<M, PM, FULLSTEP, P2, AL>(cc, a, s_tf, cm, idx, v, L4, aoff, ax);
}

// Byte j of w (j a compile-time constant): one byte permute.
__device__ __forceinline__ uint32_t byte_at(uint32_t w, int j) { return __byte_perm(w, 0u, 0x4440u | (uint32_t)j); }

// Sum of the fixed-point widths of one lane's 4 cells from their TF entries
// (E[m]: the 4 cells' entries of field m, one byte each, cell j in byte j);
// AL: also adds their fixed-point alphas per field to ax.  Whole steps only.
template <int M, int PM, bool AL>
__device__ __forceinline__ unsigned long long widths4_ent(const Cell<M, PM>& cc, const uint32_t (&E)[M],
                                                          uint32_t L4, const uint32_t* tb, uint32_t aoff,
                                                          uint32_t* ax, uint32_t four, uint32_t w23)
{
    unsigned long long acc = 0;
    if (PM == POW_ONE) {
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
            uint32_t ea[M], eb[M], axa[M], axb[M], qa, qb;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                ea[m] = byte_at(E[m], j);
                eb[m] = byte_at(E[m], j + 1);
            }
            cc.template width2_ent<AL>(ea, eb, byte_at(L4, j), byte_at(L4, j + 1), tb, aoff, axa, axb, qa, qb, four,
                                       w23);
            acc += (unsigned long long)qa + qb;
            if (AL) {
#pragma unroll
                for (int m = 0; m < M; ++m) ax[m] += axa[m] + axb[m];
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t e[M];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                e[m] = (E[m] >> (8 * j)) & 0xFFu;
                if (AL) ax[m] += lds_u32(tb[m] + 4u * e[m] + aoff);
            }
            acc += cc.width_ent(e, (L4 >> (8 * j)) & 0xFF, tb);
        }
    }
    return acc;
}

// The TF entries of every cell for the current domains (k_prepare's lo and
// s), T <= 256: the same entry as the width paths read, min(floor(t T), T),
// with entry T (a copy of T - 1 in the tables) stored as T - 1, at the
// cells' entry positions (ent_pos).  Four cells per thread; the rows'
// padding past the last cell is read and written too (its entries are never
// used).
template <int M>
__global__ __launch_bounds__(256) void k_entries(UpdateArgs a)
{
    const UpdateConsts* C = a.consts;
    const float Tf = (float)a.T;
    const uint32_t Tm1 = a.T - 1;
    const uint64_t n4 = (a.n + 3) / 4;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n4; i += (uint64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const float lo = C->lo[m], sc = C->s[m];
            const float4 x = __ldg(reinterpret_cast<const float4*>(a.val + m * a.pitch) + i);
            const float c[4] = {x.x, x.y, x.z, x.w};
            uint32_t packed = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t e = floor_small(__fmul_rn(norm_t(c[j], lo, sc), Tf));
                packed |= (e < Tm1 ? e : Tm1) << (8 * j);
            }
            *reinterpret_cast<uint32_t*>(a.ent + m * a.pitch + ent_pos(4 * i)) = packed;
        }
    }
}

// Row M of the entries: the cells' levels at their entry positions (once per
// data set).  16 cells per thread, padding included.
__global__ __launch_bounds__(256) void k_ent_levels(UpdateArgs a)
{
    const uint64_t n16 = (a.n + 15) / 16;
    uint8_t* row = a.ent + (uint64_t)a.M * a.pitch;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n16; i += (uint64_t)gridDim.x * blockDim.x)
        *reinterpret_cast<uint4*>(row + ent_pos(16 * i)) = __ldg(reinterpret_cast<const uint4*>(a.lev) + i);
}

// One warp of a pass-A CTA, with the tile's chunk totals in lanes 0..7: chunk
// offsets within the tile, the tile's exclusive prefix by decoupled look-back
// (bounded waits), the chunk prefixes, and F after the last tile.
// Decoupled look-back of scan unit `unit` > 0 by one warp: the sum of the
// units before it, from their published aggregates (FLAG_A) back to the
// nearest inclusive prefix (FLAG_P), 32 units per round.  Waits are bounded
// (spin_limit polls, then the unit counts as 0 and ERR_TIMEOUT is raised).
__device__ __forceinline__ unsigned long long look_back(const UpdateArgs& a, const unsigned long long* status,
                                                        uint64_t unit, int lane)
{
    unsigned long long excl = 0;
    int64_t end = (int64_t)unit - 1;              // window [end-31, end]
    while (true) {
        const int64_t j = end - lane;
        unsigned long long s = FLAG_P;            // before unit 0: neutral
        if (j >= 0) {
            long long spins = 0;
            while (true) {
                s = ld_relaxed(status + j);
                if (s >> 62) break;
                if (++spins > a.spin_limit) {
                    atomicOr(a.err, ERR_TIMEOUT);
                    s = FLAG_P;                   // give up: count it as 0
                    break;
                }
                __nanosleep(100);
            }
        }
        const unsigned pmask = __ballot_sync(FULL, (s & FLAG_P) != 0);
        // lanes up to and including the nearest inclusive prefix contribute
        const int first = pmask ? __ffs(pmask) - 1 : 31;
        const unsigned long long contrib = lane <= first ? (s & VAL_MASK) : 0ull;
        excl += warp_sum_u64(contrib);
        if (pmask) return excl;
        end -= 32;
    }
}

__device__ __forceinline__ void tile_scan(const UpdateArgs& a, uint32_t tile, uint32_t n_tiles, int lane,
                                          unsigned long long w /* lane < WARPS: chunk total of warp lane */)
{
    unsigned long long incl = warp_incl_scan_u64(w, lane);
    const unsigned long long agg = __shfl_sync(FULL, incl, WARPS - 1);
    unsigned long long* status = a.tile_status;
    const bool skip = a.fault_no_publish && tile == 0;
    if (lane == 0 && !skip) st_relaxed(status + tile, (tile == 0 ? FLAG_P : FLAG_A) | agg);
    unsigned long long excl = 0;
    if (tile > 0) {
        excl = look_back(a, status, tile, lane);
        if (lane == 0 && !skip) st_relaxed(status + tile, FLAG_P | (excl + agg));
    }
    if (lane < WARPS) a.chunk_prefix[(uint64_t)tile * WARPS + lane] = excl + incl - w;
    if (lane == 0 && tile == n_tiles - 1) {
        UpdateConsts* C = a.consts;
        unsigned long long F = excl + agg;
        int linear = 0;
        if (F == 0 && a.n > 0) { F = a.n; linear = 1; }   // all widths 0: equal widths
        C->F = F;
        C->linear = linear;
        C->F_div_W = F / a.W;
        C->F_mod_W = F % a.W;
    }
}

// P2: the table size is a power of two (fast TF entries, see width_p2)
template <int M, int PM, bool P2>
__global__ __launch_bounds__(WARPS * 32) void k_passA(UpdateArgs a, uint32_t n_tiles)
{
    extern __shared__ float s_tf[];
    __shared__ unsigned long long s_wsum[WARPS];
    __shared__ unsigned long long s_lane[WARPS][STEPS][32];   // per-lane step sums
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // The tile comes from a ticket (the look-back needs tickets in the order
    // CTAs start), so it is known only after the barrier.  The first step's
    // cell loads are issued before it for the tile a CTA usually gets (its
    // block index) and redone after it if the ticket differs, so that their
    // latency overlaps the table load and the CTA's set-up.
    const uint32_t guess = blockIdx.x;
    float v0[4][M];
    uint32_t L0 = 0;
    {
        const uint64_t gb = ((uint64_t)guess * WARPS + warp) * CHUNK;
        if (gb + CHUNK <= a.n) load4<M>(a.val, a.pitch, a.lev, gb + lane * 4, v0, L0);
    }
    load_table<M>(s_tf, a.tf, a.T);
    if (tid == 0) s_tile = atomicAdd(&a.counters[0], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t chunk = (uint64_t)tile * WARPS + warp;
    const uint64_t base = chunk * CHUNK;
    const bool full = base + CHUNK <= a.n;
    if (full && tile != guess) load4<M>(a.val, a.pitch, a.lev, base + lane * 4, v0, L0);
    Cell<M, PM> cc;
    cc.load(a.consts, a.T);
    uint32_t cm[M];
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(s_tf);
#pragma unroll
    for (int m = 0; m < M; ++m) cm[m] = sb + 4u * (uint32_t)(m * (a.T + 1)) - 4u * BITS_2P23;

    unsigned long long acc = 0;
    if (full) {
        {
            const unsigned long long l = widths4_of<M, PM, true, P2>(cc, a, s_tf, cm, base + lane * 4, v0, L0);
            s_lane[warp][0][lane] = l;
            acc += l;
        }
#pragma unroll 2
        for (int st = 1; st < STEPS; ++st) {
            const unsigned long long l = widths4<M, PM, true, P2>(cc, a, s_tf, cm, base + st * STEP + lane * 4);
            s_lane[warp][st][lane] = l;
            acc += l;
        }
    } else {
        for (int st = 0; st < STEPS; ++st) {
            const uint64_t idx = base + st * STEP + lane * 4;
            const unsigned long long l = idx < a.n ? widths4<M, PM, false, P2>(cc, a, s_tf, cm, idx) : 0ull;
            s_lane[warp][st][lane] = l;
            acc += l;
        }
    }
    __syncwarp();
    if (a.step_sums && lane < STEPS) {
        // lane st adds up step st (rows rotated by lane to spread the banks)
        unsigned long long tot = 0;
        for (int k = 0; k < 32; ++k) tot += s_lane[warp][lane][(k + lane) & 31];
        a.step_sums[chunk * STEPS + lane] = tot;
    }
    acc = warp_sum_u64(acc);
    if (lane == 0) s_wsum[warp] = acc;
    __syncthreads();
    if (warp != 0) return;
    tile_scan(a, tile, n_tiles, lane, lane < WARPS ? s_wsum[lane] : 0ull);
}

// Pass A with the cells streamed into shared memory by bulk copies, in a
// persistent grid (as many CTAs as fit on the GPU at once) whose warps run
// independently: global warp g starts with chunk g and claims each next chunk
// from a counter when it starts the previous one (G warps in the grid: the
// claims start at G), writing each chunk's width total; k_chunk_scan then
// turns the totals into the exclusive chunk prefixes and F.
// No warp ever waits for another (no tile barrier, no look-back), so the
// stream of copies never stalls on the scan's chain of tiles.
//
// Every warp owns a ring of D slots.  Streaming the field values a slot is
// one warp step (128 cells: M field rows of 512 B and 128 level bytes) and the
// step totals come from two warp reductions per step; streaming the per-cell
// TF entries a slot is one or two 512-position runs of the entry order
// (ent_pos), each lane stays on one step for the whole chunk, and the totals
// are reduced once per chunk.  Lanes 0..M keep D slots in flight, refilling a
// slot as soon as the warp has read it and running on into the warp's next
// chunk, so a warp's loads never wait on its own arithmetic and the bytes in
// flight cost no registers.  Partial chunks (the data set's end) read the
// field values from global memory directly.  A wait that runs out (bounded
// polls) stops the warp: it waits once more, bounded, for each copy it still
// has in flight, raises ERR_TIMEOUT and returns.
// The chunk scan's blocks (k_chunk_scan): SCAN_SPAN chunks each; the width
// pass adds each chunk's totals into its block's segment sums (status words
// of quantity q at status + q * n_blocks, cleared by k_prepare).
constexpr int SCAN_THREADS = 256, SCAN_PER_THREAD = 2, SCAN_SPAN = SCAN_THREADS * SCAN_PER_THREAD;
constexpr int SCAN_Q = 1 + DVL_MAX_FIELDS;                 // quantities at most
constexpr uint32_t RING_WAIT_POLLS = 4096;      // mbarrier polls (<= 1 ms each) before a wait gives up

// Requests warp step idx into a slot: lanes 0..M-1 copy one field row each,
// lane M the levels, lane 0 arms the barrier with the step's byte count (a
// copy may complete first: the phase cannot end before that arrival).  Called
// by the whole warp after every lane has finished reading the slot.
// EN: the field rows are the cells' TF entries instead of their values, and
// the level row is the entries' row M (both at the entry positions ent_pos).
// With EN > 0 a slot holds EN runs of 512 entry positions (each one 32-cell
// piece of every warp step of a chunk): M entry rows and the level row of
// en_unit(EN) bytes each.
__host__ __device__ constexpr int en_unit(int EN) { return EN * 4 * STEP; }
template <int M, int EN>
__device__ __forceinline__ void ring_issue(int lane, uint32_t slot, uint32_t bar, const UpdateArgs& a, uint64_t idx)
{
    constexpr uint32_t ROW = EN ? en_unit(EN) : STEP * 4, LROW = EN ? en_unit(EN) : STEP;
    if (lane <= M) {
        proxy_fence_shared();          // the warp's reads of the slot before the copy's writes
        if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(M * ROW + LROW));
        if (EN) {
            bulk_g2s(slot + (uint32_t)lane * ROW, a.ent + lane * a.pitch + idx, ROW, bar);   // row M: the levels
        } else if (lane < M) {
            bulk_g2s(slot + (uint32_t)lane * ROW, a.val + lane * a.pitch + idx, ROW, bar);
        } else {
            bulk_g2s(slot + (uint32_t)(M * ROW), a.lev + idx, LROW, bar);
        }
    }
}

// chunk totals go to chunk_prefix (turned into prefixes by k_chunk_scan).
// AL: the cells' fixed-point alphas are summed per field as well (per step
// into astep, per chunk into achunk); tf_bytes then covers the float tables
// and their u32 twins (aoff = half of it).
// EN: whole steps stream the cells' TF entries (a.ent) instead of their
// field values, M + 1 bytes a cell (partial chunks still read the fields).
template <int M, int PM, bool P2, int D, int MINB, bool AL = false, int EN = 0>
__global__ __launch_bounds__(WARPS * 32, MINB) void k_passA_ring(UpdateArgs a, uint64_t n_chunks, uint32_t tf_bytes)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int EN_UNIT = en_unit(EN), EN_H = EN > 0 ? EN : 1;
    constexpr uint32_t SLOT = EN ? (M + 1) * EN_UNIT : M * STEP * 4 + STEP;
    constexpr int UNIT = EN ? EN_UNIT : STEP, UNITS = CHUNK / UNIT;   // cells per slot, slots per chunk
    float* s_tf = reinterpret_cast<float*>(smem);
    const uint32_t aoff = tf_bytes / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned char* ring = smem + tf_bytes + (size_t)warp * D * SLOT;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t ring_s = sbase + tf_bytes + (uint32_t)warp * D * SLOT;
    const uint32_t bar_s = sbase + tf_bytes + (uint32_t)(WARPS * D * SLOT) + (uint32_t)warp * D * 8u;
    // first chunk by position, then the next unclaimed one from a counter
    // (dynamic: the grid's last chunks end together whatever the chunk count)
    const uint64_t G = (uint64_t)gridDim.x * WARPS;
    uint64_t chunk = (uint64_t)blockIdx.x * WARPS + warp;
    auto claim = [&]() {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(&a.counters[0], 1u);
        return G + __shfl_sync(FULL, c, 0);
    };
    auto full = [&](uint64_t c) { return c < n_chunks && (c + 1) * CHUNK <= a.n; };
    bool cur_full = full(chunk);
    // fault injection (tests): the first warp also waits on a barrier that
    // nothing completes, so its bounded wait runs out
    const uint32_t never_s = sbase + tf_bytes + (uint32_t)(WARPS * D * SLOT) + (uint32_t)(WARPS * D * 8);
    const bool inject = a.fault_no_publish && blockIdx.x == 0 && warp == 0;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < D; ++k) mbar_init(bar_s + 8u * k, 1);
        if (tid == 0) mbar_init(never_s, 1);
        mbar_init_fence();
    }
    __syncwarp();
    int inflight = 0;                  // copies issued and not yet consumed (warp-uniform)
    if (cur_full) {
#pragma unroll
        for (int k = 0; k < D; ++k) ring_issue<M, EN>(lane, ring_s + k * SLOT, bar_s + 8u * k, a, chunk * CHUNK + k * UNIT);
        inflight = D;
    }
    load_table<M>(s_tf, a.tf, a.T);
    if (AL) load_table_fx<M>(reinterpret_cast<uint32_t*>(smem + aoff), a.tf, a.T);
    __syncthreads();
    Cell<M, PM> cc;
    cc.load(a.consts, a.T);
    uint32_t cm[M], tb[M];
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(s_tf);
#pragma unroll
    for (int m = 0; m < M; ++m) {
        tb[m] = sb + 4u * (uint32_t)(m * (a.T + 1));
        cm[m] = tb[m] - 4u * BITS_2P23;
    }
    const uint64_t n_steps_all = n_chunks * STEPS;
    const uint64_t scan_blocks = (n_chunks + SCAN_SPAN - 1) / SCAN_SPAN;
    // 4 and wshift << 23 as values the compiler cannot fold (see width2_ent)
    const uint32_t four = 4u + (a.T >> 31), w23 = (uint32_t)cc.wshift << 23;

    int k = 0;                         // next slot to consume
    uint32_t phase = 0;                // its parity
    bool late = false;                 // a wait gave up
    const bool injected = inject && !mbar_wait(never_s, 0, (uint32_t)min((int64_t)RING_WAIT_POLLS, a.spin_limit),
                                               1000u);
    while (chunk < n_chunks) {
        const uint64_t base = chunk * CHUNK;
        const uint64_t nxt = claim();
        const bool nxt_full = full(nxt);
        unsigned long long acc = 0, mine = 0;
        unsigned long long amine[M];                    // this lane's step: alpha sums per field
#pragma unroll
        for (int m = 0; m < M; ++m) amine[m] = 0;
        auto alpha_step = [&](uint32_t (&ax)[M], int st) {
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const unsigned long long t = warp_total_small(ax[m]);     // <= 128 x 2^29
                if (AL && lane == st) amine[m] = t;
            }
        };
        if (cur_full) {
#pragma unroll 1
            for (int st = 0; st < UNITS; ++st) {
                // a wait that runs out (for any lane) ends the warp's work
                if (!__all_sync(FULL, mbar_wait(bar_s + 8u * k, phase, RING_WAIT_POLLS))) {
                    late = true;
                    break;
                }
                --inflight;
                float v[4][M];
                uint4 W4[EN_H][M], LV[EN_H];    // EN: the lane's 16 cells of each half (one byte each)
                uint32_t L4 = 0;
                if constexpr (EN) {
#pragma unroll
                    for (int h = 0; h < EN_H; ++h) {
#pragma unroll
                        for (int m = 0; m < M; ++m)
                            W4[h][m] = reinterpret_cast<const uint4*>(ring + k * SLOT + m * EN_UNIT + h * 512)[lane];
                        LV[h] = reinterpret_cast<const uint4*>(ring + k * SLOT + M * EN_UNIT + h * 512)[lane];
                    }
                } else {
                    const float4* f4 = reinterpret_cast<const float4*>(ring + k * SLOT);
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        const float4 x = f4[m * 32 + lane];
                        v[0][m] = x.x; v[1][m] = x.y; v[2][m] = x.z; v[3][m] = x.w;
                    }
                    L4 = reinterpret_cast<const uint32_t*>(ring + k * SLOT + M * STEP * 4)[lane];
                }
                __syncwarp();             // every lane has read the slot
                {
                    const int s2 = st + D;
                    if (s2 < UNITS) {
                        ring_issue<M, EN>(lane, ring_s + k * SLOT, bar_s + 8u * k, a, base + s2 * UNIT);
                        ++inflight;
                    } else if (nxt_full) {
                        ring_issue<M, EN>(lane, ring_s + k * SLOT, bar_s + 8u * k, a, nxt * CHUNK + (s2 - UNITS) * UNIT);
                        ++inflight;
                    }
                }
                if constexpr (EN) {
                    // each 512-position run of the slot holds one piece of
                    // every step of the chunk (ent_pos): lane l has 16 cells
                    // of step l >> 1 in each, the same step in every slot, so
                    // its sums run over the chunk and meet their other half
                    // (lane l ^ 1) at its end
#pragma unroll
                    for (int w = 0; w < 4 * EN_H; ++w) {
                        uint32_t E[M], ax[M];
                        const int h = w >> 2, c = w & 3;
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const uint4& q = W4[h][m];
                            E[m] = c == 0 ? q.x : c == 1 ? q.y : c == 2 ? q.z : q.w;
                            ax[m] = 0;
                        }
                        const uint32_t L = c == 0 ? LV[h].x : c == 1 ? LV[h].y : c == 2 ? LV[h].z : LV[h].w;
                        acc += widths4_ent<M, PM, AL>(cc, E, L, tb, aoff, ax, four, w23);
                        if (AL) {
#pragma unroll
                            for (int m = 0; m < M; ++m) amine[m] += ax[m];
                        }
                    }
                } else {
                    uint32_t ax[M];
#pragma unroll
                    for (int m = 0; m < M; ++m) ax[m] = 0;
                    const unsigned long long l =
                        widths4_of<M, PM, true, P2, AL>(cc, a, s_tf, cm, base + st * STEP + lane * 4, v, L4, aoff, ax);
                    const unsigned long long tot = warp_total_small(l);
                    if (lane == st) mine = tot;
                    acc += tot;
                    if (AL) alpha_step(ax, st);
                }
                if (++k == D) { k = 0; phase ^= 1u; }
            }
            if constexpr (EN) {
                if (!late) {
                    // step totals (both halves of a step; lane s < 16 keeps
                    // step s), then the chunk total
                    acc += __shfl_xor_sync(FULL, acc, 1);
                    mine = __shfl_sync(FULL, acc, (2 * lane) & 31);
                    if (AL) {
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            amine[m] += __shfl_xor_sync(FULL, amine[m], 1);
                            amine[m] = __shfl_sync(FULL, amine[m], (2 * lane) & 31);
                        }
                    }
#pragma unroll
                    for (int o = 2; o < 32; o <<= 1) acc += __shfl_xor_sync(FULL, acc, o);
                }
            }
        } else {
            if (nxt_full) {
                // nothing of this chunk is in flight: the next one's first steps
                int kk = k;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    ring_issue<M, EN>(lane, ring_s + kk * SLOT, bar_s + 8u * kk, a, nxt * CHUNK + j * UNIT);
                    if (++kk == D) kk = 0;
                }
                inflight += D;
            }
            for (int st = 0; st < STEPS; ++st) {
                const uint64_t idx = base + st * STEP + lane * 4;
                uint32_t ax[M];
#pragma unroll
                for (int m = 0; m < M; ++m) ax[m] = 0;
                const unsigned long long l =
                    idx < a.n ? widths4<M, PM, false, P2, AL>(cc, a, s_tf, cm, idx, aoff, ax) : 0ull;
                const unsigned long long tot = warp_total_small(l);
                if (lane == st) mine = tot;
                acc += tot;
                if (AL) alpha_step(ax, st);
            }
        }
        if (late) break;
        if (a.step_sums && lane < STEPS) a.step_sums[chunk * STEPS + lane] = mine;
        if (lane == 0) {
            a.chunk_prefix[chunk] = acc;
            atomicAdd(a.tile_status + chunk / SCAN_SPAN, acc);          // the scan block's sum
        }
        if (AL) {
            // per field: the steps' alpha sums as an exclusive prefix within
            // the chunk, and the chunk total
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const unsigned long long am = lane < STEPS ? amine[m] : 0ull;
                const unsigned long long incl = warp_incl_scan_u64(am, lane);
                if (lane < STEPS) a.astep[(uint64_t)m * n_steps_all + chunk * STEPS + lane] = incl - am;
                if (lane == STEPS - 1) {
                    a.achunk[(uint64_t)m * (n_chunks + 1) + chunk] = incl;
                    atomicAdd(a.tile_status + (1 + m) * scan_blocks + chunk / SCAN_SPAN, incl);
                }
            }
        }
        chunk = nxt;
        cur_full = nxt_full;
    }
    if (late) {
        // the copies still in flight fill the slots from k on, in order: each
        // is waited for once more (bounded) before the warp stops
        for (; inflight > 0; --inflight) {
            mbar_wait(bar_s + 8u * k, phase, RING_WAIT_POLLS);
            if (++k == D) { k = 0; phase ^= 1u; }
        }
    }
    if ((late || injected) && lane == 0) atomicOr(a.err, ERR_TIMEOUT);
}

// The chunk totals (in chunk_prefix) become exclusive prefixes in one launch
// over blocks of SCAN_SPAN chunks: the width pass has already summed each
// block's chunks into its status word, so a block scans its own chunks and
// adds the sum of the earlier blocks' words (one round of loads; no block
// waits for another).  The last block also writes F (Eq. 4's total) and the
// all-zero fallback, as tile_scan does.  With alpha sums (achunk) the block
// scans each field's chunk alpha sums the same way, warp q summing quantity
// q's earlier blocks (quantity 0: widths, q >= 1: field q - 1's alphas;
// status words of quantity q at status + q * gridDim.x), and the last block
// writes each field's alpha total at achunk[m][n_chunks].
__global__ __launch_bounds__(SCAN_THREADS) void k_chunk_scan(UpdateArgs a, uint64_t n_chunks,
                                                             unsigned long long* status)
{
    __shared__ unsigned long long s_warp[SCAN_Q][SCAN_THREADS / 32];
    __shared__ unsigned long long s_excl[SCAN_Q];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nq = a.achunk ? 1 + (int)a.M : 1;
    const uint32_t b = blockIdx.x;
    auto row_of = [&](int q) {
        return q == 0 ? a.chunk_prefix : a.achunk + (uint64_t)(q - 1) * (n_chunks + 1);
    };
    // block-local scans: thread tid holds chunks b0 + tid*PER .. +PER of each
    // quantity (kept in registers for the write-back)
    const uint64_t c0 = (uint64_t)b * SCAN_SPAN + (uint64_t)tid * SCAN_PER_THREAD;
    unsigned long long tq[SCAN_Q], iq[SCAN_Q], vq[SCAN_Q][SCAN_PER_THREAD];
#pragma unroll
    for (int q = 0; q < SCAN_Q; ++q) {
        tq[q] = 0;
        iq[q] = 0;
#pragma unroll
        for (int j = 0; j < SCAN_PER_THREAD; ++j) vq[q][j] = 0;
        if (q < nq) {
            const unsigned long long* row = row_of(q);
#pragma unroll
            for (int j = 0; j < SCAN_PER_THREAD; ++j) {
                vq[q][j] = c0 + j < n_chunks ? row[c0 + j] : 0ull;
                tq[q] += vq[q][j];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < SCAN_Q; ++q) {
        if (q < nq) {
            iq[q] = warp_incl_scan_u64(tq[q], lane);
            if (lane == 31) s_warp[q][warp] = iq[q];
        }
    }
    __syncthreads();
    for (int q = warp; q < nq; q += SCAN_THREADS / 32) {
        const unsigned long long* st = status + (uint64_t)q * gridDim.x;
        unsigned long long excl = 0;
        for (uint32_t i = lane; i < b; i += 32) excl += st[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) excl += __shfl_xor_sync(FULL, excl, o);
        if (lane == 0) s_excl[q] = excl;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < SCAN_Q; ++q) {
        if (q >= nq) break;
        unsigned long long wpre = 0, agg = 0;
#pragma unroll
        for (int w = 0; w < SCAN_THREADS / 32; ++w) {
            if (w < warp) wpre += s_warp[q][w];
            agg += s_warp[q][w];
        }
        unsigned long long* row = row_of(q);
        unsigned long long run = s_excl[q] + wpre + iq[q] - tq[q];
#pragma unroll
        for (int j = 0; j < SCAN_PER_THREAD; ++j) {
            if (c0 + j < n_chunks) row[c0 + j] = run;
            run += vq[q][j];
        }
        if (b == gridDim.x - 1 && tid == 0) {
            if (q == 0) {
                UpdateConsts* C = a.consts;
                unsigned long long F = s_excl[0] + agg;
                int linear = 0;
                if (F == 0 && a.n > 0) { F = a.n; linear = 1; }   // all widths 0: equal widths
                C->F = F;
                C->linear = linear;
                C->F_div_W = F / a.W;
                C->F_mod_W = F % a.W;
            } else {
                row[n_chunks] = s_excl[q] + agg;                  // the field's alpha total
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Pass B: placement and per-pixel reduction
// ---------------------------------------------------------------------------

template <int M>
struct Acc {
    float s[M], mn[M], mx[M];
    uint32_t cnt;
    __device__ __forceinline__ void reset()
    {
#pragma unroll
        for (int m = 0; m < M; ++m) { s[m] = 0.0f; mn[m] = 2.0f; mx[m] = -1.0f; }
        cnt = 0;
    }
    __device__ __forceinline__ void add(const float* t)
    {
#pragma unroll
        for (int m = 0; m < M; ++m) { s[m] += t[m]; mn[m] = fminf(mn[m], t[m]); mx[m] = fmaxf(mx[m], t[m]); }
        ++cnt;
    }
    __device__ __forceinline__ void flush_to(const UpdateArgs& a, uint32_t p) const
    {
        if (!cnt) return;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const uint64_t k = (uint64_t)m * a.W + p;
            atomicAdd(&a.sum[k], (double)s[m]);
            atomicMin(&a.vmin[k], __float_as_uint(mn[m]));   // t >= 0: bit order = value order
            atomicMax(&a.vmax[k], __float_as_uint(mx[m]));
        }
        atomicAdd(&a.count[p], cnt);
    }
    // warp-wide reduction, then one lane flushes
    __device__ __forceinline__ void warp_flush(const UpdateArgs& a, uint32_t p, int lane)
    {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
#pragma unroll
            for (int m = 0; m < M; ++m) {
                s[m] += __shfl_xor_sync(FULL, s[m], o);
                mn[m] = fminf(mn[m], __shfl_xor_sync(FULL, mn[m], o));
                mx[m] = fmaxf(mx[m], __shfl_xor_sync(FULL, mx[m], o));
            }
            cnt += __shfl_xor_sync(FULL, cnt, o);
        }
        if (lane == 0) flush_to(a, p);
        reset();
    }
};

// Exact placement of one lane's cells of a step that crosses a pixel
// boundary; consecutive cells on the same pixel are merged per lane.
template <int M>
__device__ __noinline__ void place_slow(const UpdateArgs& a, const PixelMap& pm, const float (&t)[4][M],
                                        const uint32_t (&q)[4], int nvalid, unsigned long long E)
{
    Acc<M> run;
    run.reset();
    uint32_t run_p = 0xFFFFFFFFu;
    for (int j = 0; j < nvalid; ++j) {
        const unsigned long long I = E + q[j];
        const uint32_t b1 = pm.first_pixel(E);
        const uint32_t b2 = I > E ? pm.last_pixel(I) : b1;
        for (uint32_t p = b1; p <= b2; ++p) {
            if (p != run_p) {
                run.flush_to(a, run_p);
                run.reset();
                run_p = p;
            }
            run.add(t[j]);
        }
        E = I;
    }
    run.flush_to(a, run_p);
}

// One warp step of 128 cells (4 per lane).  FULLSTEP: all cells valid.
template <int M, int PM, bool FULLSTEP>
__device__ __forceinline__ void place_step(const UpdateArgs& a, const Cell<M, PM>& cc, const float* s_tf,
                                           const PixelMap& pm, uint64_t idx, int lane, unsigned long long& pos,
                                           uint32_t& cur, unsigned long long& hi_pos, Acc<M>& acc)
{
    const int nvalid = FULLSTEP ? 4 : (idx < a.n ? (a.n - idx < 4 ? (int)(a.n - idx) : 4) : 0);
    float t[4][M];
    uint32_t q[4] = {0, 0, 0, 0};
    if (FULLSTEP || nvalid) {
        float v[4][M];
        uint32_t L4;
        load4<M>(a.val, a.pitch, a.lev, idx, v, L4);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int m = 0; m < M; ++m) t[j][m] = norm_t(v[j][m], cc.lo[m], cc.s[m]);
            uint32_t w = cc.linear ? 1u : cc.width(t[j], (L4 >> (8 * j)) & 0xFF, s_tf);
            q[j] = (FULLSTEP || j < nvalid) ? w : 0u;
        }
    }
    const unsigned long long lsum = (unsigned long long)q[0] + q[1] + q[2] + q[3];
    const unsigned long long I_last = pos + warp_total_small(lsum);
    if (I_last < hi_pos) {
        // every cell of the step lies inside pixel `cur` (pos >= C(cur) holds)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (FULLSTEP || j < nvalid) acc.add(t[j]);
    } else {
        acc.warp_flush(a, cur, lane);
        const unsigned long long incl = warp_incl_scan_u64(lsum, lane);
        place_slow<M>(a, pm, t, q, nvalid, pos + incl - lsum);
        cur = pm.first_pixel(I_last);
        hi_pos = pm.C(cur + 1);
    }
    pos = I_last;
}

template <int M, int PM>
__global__ __launch_bounds__(WARPS * 32) void k_passB(UpdateArgs a)
{
    extern __shared__ float s_tf[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    load_table<M>(s_tf, a.tf, a.T);
    __syncthreads();
    const uint64_t chunk = (uint64_t)blockIdx.x * WARPS + warp;
    const uint64_t base = chunk * CHUNK;
    if (base >= a.n) return;

    Cell<M, PM> cc;
    cc.load(a.consts, a.T);
    const UpdateConsts* C = a.consts;
    PixelMap pm{C->F_div_W, C->F_mod_W, C->F, a.W};

    unsigned long long pos = cc.linear ? base : a.chunk_prefix[chunk];
    uint32_t cur = pm.first_pixel(pos);
    unsigned long long hi_pos = pm.C(cur + 1);
    Acc<M> acc;
    acc.reset();

    const uint64_t rem = a.n - base;
    const int full = rem >= (uint64_t)CHUNK ? STEPS : (int)(rem / STEP);
#pragma unroll 1
    for (int st = 0; st < full; ++st)
        place_step<M, PM, true>(a, cc, s_tf, pm, base + st * STEP + lane * 4, lane, pos, cur, hi_pos, acc);
    if (full < STEPS && base + (uint64_t)full * STEP < a.n)
        place_step<M, PM, false>(a, cc, s_tf, pm, base + full * STEP + lane * 4, lane, pos, cur, hi_pos, acc);
    acc.warp_flush(a, cur, lane);
}

// ---------------------------------------------------------------------------
// Finalize: ApplyWeights + ApplyTransFunc (Sec. 4)
// ---------------------------------------------------------------------------

__global__ void k_finalize(UpdateArgs a)
{
    const uint64_t MW = (uint64_t)a.M * a.W;
    const float Tf = (float)a.T;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < MW;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t m = (uint32_t)(i / a.W), p = (uint32_t)(i % a.W);
        const uint32_t c = a.count[p];
        if (a.asum) a.amean[i] = c ? __double2float_rn(__ddiv_rn(a.asum[i], (double)c)) : 0.0f;
        if (c) {
            const float mean = __double2float_rn(__ddiv_rn(a.sum[i], (double)c));
            a.mean[i] = mean;
            a.y[i] = a.tf[m * a.T + tf_entry(mean, Tf, a.T - 1)];
        } else {
            a.mean[i] = 0.0f;
            a.y[i] = 0.0f;
            a.vmin[i] = 0u;
            a.vmax[i] = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// Differentiable path: control points -> alpha tables, and the adjoint of the
// per-pixel alpha means with the assignment held fixed
// ---------------------------------------------------------------------------

__global__ void k_ctrl_table(uint32_t M, uint32_t K, uint32_t T, const float* __restrict__ ctrl,
                             float* __restrict__ tf, uint32_t* err)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (uint64_t)M * K; i += stride)
        if (!(ctrl[i] >= 0.0f && ctrl[i] <= 1.0f)) atomicOr(err, ERR_RANGE);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (uint64_t)M * T; i += stride) {
        const uint32_t m = (uint32_t)(i / T), e = (uint32_t)(i % T);
        const float x = __fdiv_rn((float)(e * (K - 1)), (float)(T - 1));
        uint32_t k0 = (uint32_t)floorf(x);
        if (k0 > K - 2) k0 = K - 2;
        const float w = __fsub_rn(x, (float)k0);
        const float c0 = ctrl[m * K + k0], c1 = ctrl[m * K + k0 + 1];
        tf[i] = __fadd_rn(c0, __fmul_rn(w, __fsub_rn(c1, c0)));
    }
}

// Adds v at (field m, shared-table entry e) to the CTA's table (or to global).
__device__ __forceinline__ void gadd(double* sG, double* gtab, uint32_t T, int T1, int m, uint32_t e, double v)
{
    if (sG) atomicAdd(&sG[m * T1 + e], v);
    else atomicAdd(&gtab[(uint64_t)m * T + (e < T ? e : T - 1)], v);
}

template <int M, int PM>
__device__ __noinline__ void back_crossing_step(const UpdateArgs& a, const float* s_tf, const PixelMap& pm,
                                                uint64_t idx, unsigned long long s_start, int lane,
                                                const float* g, double* sG, double* gtab)
{
    Cell<M, PM> cc;
    cc.load(a.consts, a.T);
    const int nvalid = idx < a.n ? (a.n - idx < 4 ? (int)(a.n - idx) : 4) : 0;
    auto cell = [&](int j, float (&t)[M]) {
#pragma unroll
        for (int m = 0; m < M; ++m) t[m] = norm_t(__ldg(a.val + m * a.pitch + idx + j), cc.lo[m], cc.s[m]);
    };
    unsigned long long lsum = 0;
    for (int j = 0; j < nvalid; ++j) {
        float t[M];
        cell(j, t);
        lsum += cc.linear ? 1u : cc.width(t, __ldg(a.lev + idx + j), s_tf);
    }
    unsigned long long E = s_start + warp_incl_scan_u64(lsum, lane) - lsum;
    for (int j = 0; j < nvalid; ++j) {
        float t[M];
        cell(j, t);
        const unsigned long long I = E + (cc.linear ? 1u : cc.width(t, __ldg(a.lev + idx + j), s_tf));
        const uint32_t b1 = pm.first_pixel(E);
        const uint32_t b2 = I > E ? pm.last_pixel(I) : b1;
        for (uint32_t p = b1; p <= b2; ++p) {
            const uint32_t c = a.count[p];
            if (!c) continue;
#pragma unroll
            for (int m = 0; m < M; ++m)
                gadd(sG, gtab, a.T, cc.T1, m, floor_small(__fmul_rn(t[m], cc.Tf)),
                     (double)g[(uint64_t)m * a.W + p] / (double)c);
        }
        E = I;
    }
}

// The histogram adjoint's form of back_crossing_step, for a step whose cells
// fall in more than one pixel.  A cell that covers several pixels adds its
// weight once per pixel as before (float64 shared atomics; at most a few per
// boundary).  The cells that lie inside one pixel (nearly all) are counted per
// TF entry in the warp's own histogram h, pixel by pixel, and each pixel's
// counts are scaled by its weights g[m][p] / count[p] once, as the
// non-crossing steps are.  h is clear on entry and on return.
template <int M, int PM>
__device__ __noinline__ void back_crossing_step_hist(const UpdateArgs& a, const float* s_tf, const PixelMap& pm,
                                                     uint64_t idx, unsigned long long s_start, int lane,
                                                     const double* wtab, double* sG, uint32_t* h)
{
    Cell<M, PM> cc;
    cc.load(a.consts, a.T);
    const int T1 = cc.T1, MT1 = M * T1;
    const int nvalid = idx < a.n ? (a.n - idx < 4 ? (int)(a.n - idx) : 4) : 0;
    uint32_t e[4][M], q[4];
    unsigned long long lsum = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        q[j] = 0;
        float t[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            t[m] = j < nvalid ? norm_t(__ldg(a.val + m * a.pitch + idx + j), cc.lo[m], cc.s[m]) : 0.0f;
            e[j][m] = floor_small(__fmul_rn(t[m], cc.Tf));
        }
        if (j < nvalid) q[j] = cc.linear ? 1u : cc.width(t, __ldg(a.lev + idx + j), s_tf);
        lsum += q[j];
    }
    unsigned long long E = s_start + warp_incl_scan_u64(lsum, lane) - lsum;
    uint32_t pix[4];
    bool single[4];
    uint32_t plo = 0xFFFFFFFFu, phi = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        single[j] = false;
        pix[j] = 0;
        if (j < nvalid) {
            const unsigned long long I = E + q[j];
            const uint32_t b1 = pm.first_pixel(E);
            const uint32_t b2 = I > E ? pm.last_pixel(I) : b1;
            if (b1 == b2) {
                single[j] = true;
                pix[j] = b1;
                plo = min(plo, b1);
                phi = max(phi, b1);
            } else {
                for (uint32_t p = b1; p <= b2; ++p) {
                    if (!a.count[p]) continue;
#pragma unroll
                    for (int m = 0; m < M; ++m) atomicAdd(&sG[m * T1 + e[j][m]], wtab[(uint64_t)m * a.W + p]);
                }
            }
            E = I;
        }
    }
    plo = __reduce_min_sync(FULL, plo);
    phi = __reduce_max_sync(FULL, phi);
    if (plo > phi) return;                                      // warp-uniform: no single-pixel cell
    if (phi - plo > 8) {                                        // many narrow pixels: per-cell adds
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!single[j]) continue;
            if (!a.count[pix[j]]) continue;
#pragma unroll
            for (int m = 0; m < M; ++m) atomicAdd(&sG[m * T1 + e[j][m]], wtab[(uint64_t)m * a.W + pix[j]]);
        }
        return;
    }
    for (uint32_t p = plo; p <= phi; ++p) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (single[j] && pix[j] == p) {
#pragma unroll
                for (int m = 0; m < M; ++m) atomicAdd(&h[m * T1 + e[j][m]], 1u);
            }
        __syncwarp();
        double wc[M];
#pragma unroll
        for (int m = 0; m < M; ++m) wc[m] = wtab[(uint64_t)m * a.W + p];
        for (int i = lane; i < MT1; i += 32) {
            const uint32_t n = h[i];
            if (n) {
                h[i] = 0u;
                const int m = i / T1;
                double w = 0.0;
#pragma unroll
                for (int mm = 0; mm < M; ++mm)
                    if (mm == m) w = wc[mm];
                if (w != 0.0) atomicAdd(&sG[i], w * (double)n);
            }
        }
        __syncwarp();
    }
}

template <int M, int PM>
__global__ __launch_bounds__(WARPS * 32) void k_backward(UpdateArgs a, const float* g, double* gtab, int use_smem)
{
    extern __shared__ float s_tf[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    load_table<M>(s_tf, a.tf, a.T);
    const int T1 = (int)a.T + 1;
    double* sG = use_smem ? reinterpret_cast<double*>(s_tf + ((M * T1 + 1) & ~1)) : nullptr;
    if (sG)
        for (int i = tid; i < M * T1; i += blockDim.x) sG[i] = 0.0;
    __syncthreads();
    const uint64_t chunk = (uint64_t)blockIdx.x * WARPS + warp;
    const uint64_t base = chunk * CHUNK;
    if (base < a.n) {
        const UpdateConsts* C = a.consts;
        const bool linear = C->linear != 0;
        const PixelMap pm{C->F_div_W, C->F_mod_W, C->F, a.W};
        const uint64_t rem = a.n - base;
        const int full = rem >= (uint64_t)CHUNK ? STEPS : (int)(rem / STEP);
        const int nsteps = rem >= (uint64_t)CHUNK ? STEPS : (int)((rem + STEP - 1) / STEP);
        const unsigned long long pos0 = linear ? base : a.chunk_prefix[chunk];
        unsigned long long ssum = 0;
        if (lane < nsteps) {
            const uint64_t left = a.n - (base + (uint64_t)lane * STEP);
            ssum = linear ? (left < STEP ? left : STEP) : a.step_sums[chunk * STEPS + lane];
        }
        const unsigned long long s_end = pos0 + warp_incl_scan_u64(ssum, lane);
        const unsigned long long s_start = s_end - ssum;
        uint32_t pix = 0;
        bool crossing = true;
        if (lane < nsteps) {
            pix = pm.first_pixel(s_start);
            crossing = lane >= full || s_end >= pm.C(pix + 1);
        }
        const unsigned exact_mask = __ballot_sync(FULL, crossing) & ((1u << nsteps) - 1u);
        float lo[M], sc[M];
#pragma unroll
        for (int m = 0; m < M; ++m) { lo[m] = C->lo[m]; sc[m] = C->s[m]; }
        const float Tf = (float)a.T;
        const unsigned lt = (1u << lane) - 1u;
        for (int st = 0; st < full; ++st) {
            if (exact_mask & (1u << st)) continue;                      // warp-uniform
            const uint32_t p = __shfl_sync(FULL, pix, st);
            const uint32_t c = a.count[p];
            double wm[M];
#pragma unroll
            for (int m = 0; m < M; ++m) wm[m] = c ? (double)g[(uint64_t)m * a.W + p] / (double)c : 0.0;
            float4 x[M];
#pragma unroll
            for (int m = 0; m < M; ++m)
                x[m] = __ldg(reinterpret_cast<const float4*>(a.val + m * a.pitch + base + st * STEP + lane * 4));
#pragma unroll
            for (int j = 0; j < 4; ++j) {
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    const float v = j == 0 ? x[m].x : j == 1 ? x[m].y : j == 2 ? x[m].z : x[m].w;
                    const uint32_t e = floor_small(__fmul_rn(norm_t(v, lo[m], sc[m]), Tf));
                    // lanes with the same entry add their (equal) weights once
                    const unsigned peers = __match_any_sync(FULL, e);
                    if ((peers & lt) == 0) gadd(sG, gtab, a.T, T1, m, e, wm[m] * __popc(peers));
                }
            }
        }
        unsigned m2 = exact_mask;
        while (m2) {
            const int k = __ffs(m2) - 1;
            m2 &= m2 - 1;
            back_crossing_step<M, PM>(a, s_tf, pm, base + k * STEP + lane * 4, __shfl_sync(FULL, s_start, k), lane,
                                      g, sG, gtab);
        }
    }
    if (sG) {
        __syncthreads();
        for (int i = tid; i < M * T1; i += blockDim.x) {
            const double v = sG[i];
            if (v != 0.0) {
                const int m = i / T1;
                const uint32_t e = (uint32_t)(i - m * T1);
                atomicAdd(&gtab[(uint64_t)m * a.T + (e < a.T ? e : a.T - 1)], v);
            }
        }
    }
}

constexpr uint32_t GTAB_SEGS = 4;                 // row segments of the first reduction level

// The per-pixel weights of the adjoint, wtab[m][p] = g[m][p] / count[p] in
// float64 (0 for an empty pixel), once per call instead of once per use.
__global__ void k_backward_weights(uint32_t M, uint32_t W, const float* __restrict__ g,
                                   const uint32_t* __restrict__ count, double* __restrict__ wtab)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * W) return;
    const uint32_t c = count[i % W];
    wtab[i] = c ? (double)g[i] / (double)c : 0.0;
}

// Adjoint with per-warp entry histograms, in a persistent grid whose warps
// claim chunks from a counter.  Inside a warp step that stays in one pixel p
// every cell carries the same weight wtab[m][p] = g[m][p] / count[p], so the
// step only counts how often each TF entry occurs, in the warp's own u32
// histogram in shared memory: a lane adds each run of equal entries among its
// 4 consecutive cells with one atomic (cells close in curve order mostly
// share an entry, so fewer lanes hit the same counter at once; the run ends
// are predicates, not branches).  When the warp's pixel changes, or its chunk
// ends, the nonzero counts are packed 32 at a time through a per-warp queue
// in shared memory and scaled by the pixel's weights into the CTA's float64
// table (float64 instructions are slow on this part, so they run on full
// warps only).  Steps that cross a pixel boundary place their cells exactly
// (back_crossing_step_hist).  The next single-pixel step's cells are loaded
// while the current one is counted.  Each CTA writes its table to
// gpart[blockIdx] without atomics; k_gtab_reduce sums the CTAs in a fixed
// order.  counters[2] is the chunk counter (zeroed by the launcher).
constexpr int BQ = 64;                               // per-warp queue slots of the flush
// ENT: single-pixel steps read the cells' kept TF entries (a.ent) instead of
// normalising their field values.
template <int M, int PM, bool ENT = false>
__global__ __launch_bounds__(WARPS * 32, 3) void k_backward_hist(UpdateArgs a, const double* wtab, double* gpart)
{
    extern __shared__ float s_tf[];   // table | float64 sums | WARPS u32 histograms | WARPS flush queues
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T1 = (int)a.T + 1, MT1 = M * T1;
    load_table<M>(s_tf, a.tf, a.T);
    double* sG = reinterpret_cast<double*>(s_tf + ((MT1 + 1) & ~1));
    uint32_t* hist = reinterpret_cast<uint32_t*>(sG + MT1);
    uint32_t* h = hist + warp * MT1;
    uint32_t* qi = hist + WARPS * MT1 + warp * 2 * BQ;   // queued entry index
    uint32_t* qc = qi + BQ;                              // and its count
    for (int i = tid; i < MT1; i += blockDim.x) sG[i] = 0.0;
    for (int i = tid; i < WARPS * MT1; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const UpdateConsts* C = a.consts;
    const bool linear = C->linear != 0;
    const PixelMap pm{C->F_div_W, C->F_mod_W, C->F, a.W};
    const float Tf = (float)a.T;
    const uint64_t n_chunks = (a.n + CHUNK - 1) / CHUNK;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t cur = 0xFFFFFFFFu;
    double wc[M];
#pragma unroll
    for (int m = 0; m < M; ++m) wc[m] = 0.0;
    // scales queue slots [0, k) (k <= 32) by their field's weight into sG
    auto drain = [&](uint32_t k) {
        if ((uint32_t)lane < k) {
            const uint32_t i = qi[lane];
            const int m = (int)(i / (uint32_t)T1);
            double w = 0.0;
#pragma unroll
            for (int mm = 0; mm < M; ++mm)
                if (mm == m) w = wc[mm];
            atomicAdd(&sG[i], w * (double)qc[lane]);
        }
    };
    auto flush = [&]() {
        if (cur == 0xFFFFFFFFu) return;                            // warp-uniform
        __syncwarp();
        uint32_t fill = 0;
        for (int base = 0; base < MT1; base += 32) {
            const int i = base + lane;
            const uint32_t c = i < MT1 ? h[i] : 0u;
            const unsigned nz = __ballot_sync(FULL, c != 0u);
            if (c) {
                h[i] = 0u;
                const uint32_t pos = fill + __popc(nz & lt);
                qi[pos] = (uint32_t)i;
                qc[pos] = c;
            }
            fill += __popc(nz);
            if (fill >= 32) {
                __syncwarp();
                drain(32);
                __syncwarp();
                if ((uint32_t)lane + 32 < fill) {
                    qi[lane] = qi[lane + 32];
                    qc[lane] = qc[lane + 32];
                }
                fill -= 32;
                __syncwarp();
            }
        }
        __syncwarp();
        drain(fill);
        __syncwarp();
    };
    auto claim = [&]() {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(&a.counters[2], 1u);
        return (uint64_t)__shfl_sync(FULL, c, 0);
    };
    for (uint64_t chunk = claim(); chunk < n_chunks; chunk = claim()) {
        const uint64_t base = chunk * CHUNK;
        const uint64_t rem = a.n - base;
        const int full = rem >= (uint64_t)CHUNK ? STEPS : (int)(rem / STEP);
        const int nsteps = rem >= (uint64_t)CHUNK ? STEPS : (int)((rem + STEP - 1) / STEP);
        const unsigned long long pos0 = linear ? base : a.chunk_prefix[chunk];
        unsigned long long ssum = 0;
        if (lane < nsteps) {
            const uint64_t left = a.n - (base + (uint64_t)lane * STEP);
            ssum = linear ? (left < STEP ? left : STEP) : a.step_sums[chunk * STEPS + lane];
        }
        const unsigned long long s_end = pos0 + warp_incl_scan_u64(ssum, lane);
        const unsigned long long s_start = s_end - ssum;
        uint32_t pix = 0;
        bool crossing = true;
        if (lane < nsteps) {
            pix = pm.first_pixel(s_start);
            crossing = lane >= full || s_end >= pm.C(pix + 1);
        }
        const unsigned exact_mask = __ballot_sync(FULL, crossing) & ((1u << nsteps) - 1u);
        unsigned todo = ~exact_mask & ((1u << full) - 1u);             // single-pixel full steps
        float4 xn[M];
        uint32_t en[M];
        auto load_step = [&](int st) {
#pragma unroll
            for (int m = 0; m < M; ++m) {
                if (ENT)
                    en[m] = __ldg(reinterpret_cast<const uint32_t*>(a.ent + m * a.pitch +
                                                                    ent_pos(base + st * STEP + lane * 4)));
                else xn[m] = __ldg(reinterpret_cast<const float4*>(a.val + m * a.pitch + base + st * STEP + lane * 4));
            }
        };
        if (todo) load_step(__ffs(todo) - 1);
        while (todo) {
            const int st = __ffs(todo) - 1;
            todo &= todo - 1;
            float4 x[M];
            uint32_t ex[M];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                x[m] = xn[m];
                ex[m] = en[m];
            }
            if (todo) load_step(__ffs(todo) - 1);
            const uint32_t p = __shfl_sync(FULL, pix, st);
            if (p != cur) {                                            // warp-uniform
                flush();
                cur = p;
#pragma unroll
                for (int m = 0; m < M; ++m) wc[m] = wtab[(uint64_t)m * a.W + p];
            }
#pragma unroll
            for (int m = 0; m < M; ++m) {
                uint32_t e[4];
                if (ENT) {
                    // entry T (a copy of T - 1 in the tables) is kept as T - 1: a
                    // cell with t = 1 counts toward entry T - 1 here, which the
                    // final chain rule (k_grad_final) folds in the same way
#pragma unroll
                    for (int j = 0; j < 4; ++j) e[j] = (ex[m] >> (8 * j)) & 0xFFu;
                } else {
                    const float lo = C->lo[m], sc = C->s[m];
                    e[0] = floor_small(__fmul_rn(norm_t(x[m].x, lo, sc), Tf));
                    e[1] = floor_small(__fmul_rn(norm_t(x[m].y, lo, sc), Tf));
                    e[2] = floor_small(__fmul_rn(norm_t(x[m].z, lo, sc), Tf));
                    e[3] = floor_small(__fmul_rn(norm_t(x[m].w, lo, sc), Tf));
                }
                // run lengths from each cell to the end of its run of equal entries
                const uint32_t r3 = 1u;
                const uint32_t r2 = e[2] == e[3] ? r3 + 1u : 1u;
                const uint32_t r1 = e[1] == e[2] ? r2 + 1u : 1u;
                const uint32_t r0 = e[0] == e[1] ? r1 + 1u : 1u;
                uint32_t* hm = h + m * T1;
                atomicAdd(&hm[e[0]], r0);
                if (e[1] != e[0]) atomicAdd(&hm[e[1]], r1);
                if (e[2] != e[1]) atomicAdd(&hm[e[2]], r2);
                if (e[3] != e[2]) atomicAdd(&hm[e[3]], r3);
            }
        }
        flush();                                          // the chunk's counts (its pixel weights)
        unsigned m2 = exact_mask;
        while (m2) {
            const int k = __ffs(m2) - 1;
            m2 &= m2 - 1;
            back_crossing_step_hist<M, PM>(a, s_tf, pm, base + k * STEP + lane * 4, __shfl_sync(FULL, s_start, k),
                                           lane, wtab, sG, h);
        }
        cur = 0xFFFFFFFFu;                               // next chunk: weights reloaded
    }
    __syncthreads();
    for (int i = tid; i < MT1; i += blockDim.x) gpart[(uint64_t)blockIdx.x * MT1 + i] = sG[i];
}

// Sums the CTAs' tables in two fixed-order levels: block (x, y) adds rows y,
// y + gridDim.y, ... of 32 columns (one per lane; the warps take rows in turn
// and are combined in warp order) into part2[y]; then k_grad_final sums the
// gridDim.y partial rows per entry, folding entry T into entry T-1.
__global__ __launch_bounds__(256) void k_gtab_reduce(uint32_t MT1, uint64_t rows, const double* __restrict__ gpart,
                                                     double* __restrict__ part2)
{
    __shared__ double s[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t col = blockIdx.x * 32 + lane;
    double acc = 0.0;
    if (col < MT1)
        for (uint64_t r = blockIdx.y + (uint64_t)warp * gridDim.y; r < rows; r += 8ull * gridDim.y)
            acc += gpart[r * MT1 + col];
    s[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && col < MT1) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += s[w][lane];
        part2[(uint64_t)blockIdx.y * MT1 + col] = t;
    }
}

// The last reduction level and the chain rule in one launch, one warp per
// control point (m, k): its lanes take the table entries whose interpolation
// weights involve k (x = e (K-1)/(T-1) in [k-1, k+1]), sum each entry's
// partial rows (entry T, t = 1, folds into entry T-1), write gtab for the
// entries whose lower control point is k, and add weight x gradient in a
// fixed order: dL/dctrl[m][k] = sum_e gtab[m][e] w_k(e).
__global__ __launch_bounds__(256) void k_grad_final(uint32_t M, uint32_t K, uint32_t T,
                                                    const double* __restrict__ part2, double* __restrict__ gtab,
                                                    float* __restrict__ grad)
{
    const uint32_t wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (wid >= M * K) return;
    const uint32_t m = wid / K, k = wid % K, T1 = T + 1;
    const uint64_t lo_num = k > 0 ? (uint64_t)(k - 1) * (T - 1) : 0, hi_num = (uint64_t)(k + 1) * (T - 1);
    const uint64_t e_lo = lo_num / (K - 1), e_hi = hi_num / (K - 1) + 1;
    const uint32_t e0 = e_lo > 0 ? (uint32_t)e_lo - 1 : 0, e1 = (uint32_t)(e_hi < T - 1 ? e_hi : T - 1);
    double acc = 0.0;
    for (uint32_t e = e0 + lane; e <= e1; e += 32) {
        const uint32_t col = m * T1 + e;
        const uint32_t span = e == T - 1 ? 2u : 1u;               // entry T (t = 1) folds into T-1
        double G = 0.0;
#pragma unroll
        for (uint32_t y = 0; y < GTAB_SEGS; ++y) {
            const double* row = part2 + (uint64_t)y * M * T1 + col;
            G += row[0];
            if (span == 2u) G += row[1];
        }
        const double x = (double)e * (double)(K - 1) / (double)(T - 1);
        uint32_t k0 = (uint32_t)floor(x);
        if (k0 > K - 2) k0 = K - 2;
        const double w = x - k0;
        if (k0 == k) {
            acc += (1.0 - w) * G;
            gtab[(uint64_t)m * T + e] = G;
        }
        if (k0 + 1 == k) acc += w * G;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0) grad[wid] = (float)acc;
}

// dL/dctrl[m][k] = sum_e gtab[m][e] * (interpolation weight of k in entry e),
// from a finished gtab (the adjoint with global atomics)
__global__ void k_grad_ctrl(uint32_t M, uint32_t K, uint32_t T, const double* __restrict__ gtab,
                            float* __restrict__ grad)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * K) return;
    const uint32_t m = i / K, k = i % K;
    // only entries with x = e (K-1)/(T-1) in [k-1, k+1] weigh on control point
    // k; the range is widened by one entry on each side (the test below decides)
    const uint64_t lo_num = k > 0 ? (uint64_t)(k - 1) * (T - 1) : 0, hi_num = (uint64_t)(k + 1) * (T - 1);
    const uint64_t e_lo = lo_num / (K - 1), e_hi = hi_num / (K - 1) + 1;
    double acc = 0.0;
    for (uint32_t e = e_lo > 0 ? (uint32_t)e_lo - 1 : 0; e < T && e <= e_hi; ++e) {
        const double x = (double)e * (double)(K - 1) / (double)(T - 1);
        uint32_t k0 = (uint32_t)floor(x);
        if (k0 > K - 2) k0 = K - 2;
        const double w = x - k0, G = gtab[(uint64_t)m * T + e];
        if (k0 == k) acc += (1.0 - w) * G;
        if (k0 + 1 == k) acc += w * G;
    }
    grad[i] = (float)acc;
}

// Per-cell widths with the constants of the last update (checking aid).
template <int M>
__global__ __launch_bounds__(256) void k_widths(UpdateArgs a, unsigned long long* q)
{
    extern __shared__ float s_tf[];
    load_table<M>(s_tf, a.tf, a.T);
    __syncthreads();
    Cell<M, POW_GEN> cc;
    cc.load(a.consts, a.T);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        float t[M];
#pragma unroll
        for (int m = 0; m < M; ++m) t[m] = norm_t(a.val[m * a.pitch + i], cc.lo[m], cc.s[m]);
        q[i] = cc.linear ? 1ull : cc.width(t, a.lev[i], s_tf);
    }
}

int grid_cap(uint64_t work, int threads)
{
    uint64_t b = (work + threads - 1) / threads;
    if (b > 148ull * 8) b = 148ull * 8;
    return b ? (int)b : 1;
}

// Ring depth and register cap: D = 2 steps per warp, 4 CTAs per SM (64
// registers, 40 KB of shared memory with 256-entry tables) for up to 4 fields,
// 2 CTAs for wider cells.  (Measured on the 413.6M-cell case: depth 3 or 4
// and 5 CTAs with a 48-register cap were 0.5-1.5 % slower.)
template <int M> constexpr int ring_depth() { return 2; }
template <int M> constexpr int ring_min_blocks() { return M <= 4 ? 4 : 2; }
// Streaming the entries: slots of (M + 1) x 512 bytes at 4 CTAs per SM, or,
// once every warp of that grid has at least 6 chunks to take, slots of twice
// that at 2 CTAs per SM (the per-slot wait, copies and bookkeeping shared by
// twice the cells: 0.435 -> 0.415 ms on 413.6M cells, 85 chunks a warp;
// 0.060 -> 0.056 ms on 35.8M cells, 7.4 chunks a warp; but 5-10 % slower on
// 20M cells, 4.1 chunks a warp, where the grid's start and end show); 2
// slots deep either way.
template <int M> constexpr int ring_depth_ent() { return 2; }
template <int M> constexpr int ring_min_blocks_ent(int EN) { return EN == 1 ? ring_min_blocks<M>() : 2; }
constexpr uint64_t WIDE_SLOT_CHUNKS_PER_WARP = 6;

template <int M>
size_t ring_smem(uint32_t T, uint32_t* tf_bytes, bool alpha = false, int en = 0)
{
    // the float tables, and with alpha their u32 fixed-point twins
    *tf_bytes = (uint32_t)(((size_t)M * (T + 1) * sizeof(float) + 127) & ~(size_t)127) * (alpha ? 2u : 1u);
    const size_t slot = en ? (size_t)(M + 1) * en_unit(en) : (size_t)M * STEP * 4 + STEP;
    return *tf_bytes + (size_t)WARPS * (en ? ring_depth_ent<M>() : ring_depth<M>()) * (slot + 8) + 8;
}

// The persistent grid: as many CTAs as are resident at once (the occupancy of
// the kernel at this shared-memory size, cached per thread for the last few
// keys: an update may ask for two kernels).
template <typename K>
cudaError_t resident_ctas(K kernel, size_t smem, int* out)
{
    struct Key {
        const void* k;
        size_t smem;
        int dev, n;
    };
    constexpr int SLOTS = 4;
    thread_local Key cache[SLOTS] = {};
    thread_local int next = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    for (const Key& c : cache)
        if (c.k == (const void*)kernel && c.smem == smem && c.dev == dev) {
            *out = c.n;
            return cudaSuccess;
        }
    int per_sm = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, WARPS * 32, smem)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    cache[next] = Key{(const void*)kernel, smem, dev, (per_sm > 0 ? per_sm : 1) * sms};
    *out = cache[next].n;
    next = (next + 1) % SLOTS;
    return cudaSuccess;
}

template <int M, int PM>
cudaError_t launch_passA_ring(cudaStream_t s, const UpdateArgs& a, uint32_t n_tiles, bool p2)
{
    constexpr int D = ring_depth<M>(), MB = ring_min_blocks<M>(), DE = ring_depth_ent<M>(),
                  MB1 = ring_min_blocks_ent<M>(1), MB2 = ring_min_blocks_ent<M>(2);
    const bool alpha = a.astep != nullptr, ent = a.ent != nullptr;
    const uint64_t n_chunks = (uint64_t)n_tiles * WARPS;
    cudaError_t e;
    uint32_t tf_bytes;
    int grid = 0;
    if (ent && !alpha && p2) {
        // wide slots when every warp of their grid gets many chunks
        auto wide = k_passA_ring<M, PM, true, DE, MB2, false, 2>;
        const size_t smem2 = ring_smem<M>(a.T, &tf_bytes, false, 2);
        if ((e = smem_attr(wide, smem2)) != cudaSuccess) return e;
        if ((e = resident_ctas(wide, smem2, &grid)) != cudaSuccess) return e;
        if (n_chunks >= WIDE_SLOT_CHUNKS_PER_WARP * (uint64_t)grid * WARPS) {
            wide<<<grid, WARPS * 32, smem2, s>>>(a, n_chunks, tf_bytes);
            const uint32_t blocks = (uint32_t)((n_chunks + SCAN_SPAN - 1) / SCAN_SPAN);
            k_chunk_scan<<<blocks, SCAN_THREADS, 0, s>>>(a, n_chunks, a.tile_status);
            return cudaSuccess;
        }
    }
    const size_t smem = ring_smem<M>(a.T, &tf_bytes, alpha, ent ? 1 : 0);
    // (p2 also selects the partial chunks' entry computation in the entry-streaming kernels)
    auto kernel =
        ent ? (alpha ? (p2 ? k_passA_ring<M, PM, true, DE, MB1, true, 1> : k_passA_ring<M, PM, false, DE, MB1, true, 1>)
                     : (p2 ? k_passA_ring<M, PM, true, DE, MB1, false, 1> : k_passA_ring<M, PM, false, DE, MB1, false, 1>))
            : alpha ? (p2 ? k_passA_ring<M, PM, true, D, MB, true> : k_passA_ring<M, PM, false, D, MB, true>)
                    : (p2 ? k_passA_ring<M, PM, true, D, MB> : k_passA_ring<M, PM, false, D, MB>);
    if ((e = smem_attr(kernel, smem)) != cudaSuccess) return e;
    if ((e = resident_ctas(kernel, smem, &grid)) != cudaSuccess) return e;
    if ((uint32_t)grid > n_tiles) grid = (int)n_tiles;
    kernel<<<grid, WARPS * 32, smem, s>>>(a, n_chunks, tf_bytes);
    // the scan's block states use the (here unused) tile status words
    const uint32_t blocks = (uint32_t)((n_chunks + SCAN_SPAN - 1) / SCAN_SPAN);
    k_chunk_scan<<<blocks, SCAN_THREADS, 0, s>>>(a, n_chunks, a.tile_status);
    return cudaSuccess;
}

template <int M, int PM>
cudaError_t run_passes(cudaStream_t s, const UpdateArgs& a, uint32_t n_tiles, size_t smem)
{
    cudaError_t e;
    const bool p2 = (a.T & (a.T - 1)) == 0;          // power-of-two table size
    if ((e = smem_attr(k_passA<M, PM, true>, smem)) != cudaSuccess) return e;
    if ((e = smem_attr(k_passA<M, PM, false>, smem)) != cudaSuccess) return e;
    if ((e = smem_attr(k_passB<M, PM>, smem)) != cudaSuccess) return e;
    // the bulk copies need 16-byte aligned rows (they read whole chunks only)
    const bool ring = ((uintptr_t)a.val % 16 == 0) && ((uintptr_t)a.lev % 16 == 0) && (a.pitch % 4 == 0);
    if (a.astep && !ring) return cudaErrorInvalidValue;   // alpha sums come from the streaming pass A only
    if (a.events) cudaEventRecord(a.events[1], s);
    if (n_tiles) {
        if (ring) {
            if ((e = launch_passA_ring<M, PM>(s, a, n_tiles, p2)) != cudaSuccess) return e;
        } else if (p2) {
            k_passA<M, PM, true><<<n_tiles, WARPS * 32, smem, s>>>(a, n_tiles);
        } else {
            k_passA<M, PM, false><<<n_tiles, WARPS * 32, smem, s>>>(a, n_tiles);
        }
    }
    if (a.events) cudaEventRecord(a.events[2], s);
    if (a.vt) return cudaSuccess;          // bins come from range queries (see run_update)
    if (n_tiles) k_passB<M, PM><<<n_tiles, WARPS * 32, smem, s>>>(a);
    if (a.events) cudaEventRecord(a.events[3], s);
    return cudaSuccess;
}

template <int M>
cudaError_t run_update(cudaStream_t s, const UpdateArgs& a)
{
    const uint32_t n_tiles = (uint32_t)((a.n + TILE - 1) / TILE);
    const size_t smem = (size_t)M * (a.T + 1) * sizeof(float);
    cudaError_t e;
    if ((e = smem_attr(k_vmax_exact<M>, smem)) != cudaSuccess) return e;
    // scan status words: one per tile (direct-load pass A), or per chunk-scan
    // block and quantity (widths and, with alpha sums, each field's alphas)
    const uint64_t scan_blocks = ((uint64_t)n_tiles * WARPS + SCAN_SPAN - 1) / SCAN_SPAN;
    const uint64_t n_status = a.achunk ? (n_tiles > SCAN_Q * scan_blocks ? n_tiles : SCAN_Q * scan_blocks) : n_tiles;
    const uint64_t clear = (uint64_t)a.M * a.W > n_status ? (uint64_t)a.M * a.W : n_status;
    if (a.events) cudaEventRecord(a.events[0], s);
    k_prepare<<<grid_cap(clear, 256), 256, 0, s>>>(a, n_status);
    if (a.prm.vmax_mode == DVL_VMAX_EXACT) {
        k_vmax_exact<M><<<grid_cap(a.n, 256), 256, smem, s>>>(a);
        k_consts<<<1, 1, 0, s>>>(a);
    }
    if (a.vt && a.vt_build) {
        if ((e = launch_value_tables(s, a.M, *a.vt)) != cudaSuccess) return e;
    }
    if (a.ent && a.ent_build && a.n > 0) k_entries<M><<<grid_cap((a.n + 3) / 4, 256), 256, 0, s>>>(a);
    if (a.ent && a.ent_lev_build && a.n > 0) k_ent_levels<<<grid_cap((a.n + 15) / 16, 256), 256, 0, s>>>(a);
    e = a.prm.P == 1.0f ? run_passes<M, POW_ONE>(s, a, n_tiles, smem) : run_passes<M, POW_GEN>(s, a, n_tiles, smem);
    if (e != cudaSuccess) return e;
    if (a.vt && a.n > 0) {
        // bins as range queries over the value tables (writes final bins)
        const QueryArgs qa{a.consts, a.chunk_prefix, a.step_sums, a.H, a.S, a.psum, a.pmm, 1u,
                           a.astep, a.achunk, a.astep ? a.apart : nullptr, (uint64_t)n_tiles * WARPS};
        if ((e = launch_bins(s, a, qa, *a.vt)) != cudaSuccess) return e;
        if (a.events) cudaEventRecord(a.events[3], s);
    } else {
        // the placement pass's bins (or, with no cells, the empty bins k_prepare left)
        if (a.vt && a.events) cudaEventRecord(a.events[3], s);
        k_finalize<<<grid_cap((uint64_t)a.M * a.W, 256), 256, 0, s>>>(a);
    }
    if (a.events) cudaEventRecord(a.events[4], s);
    return cudaGetLastError();
}

size_t backward_hist_smem(uint32_t M, uint32_t T)
{
    const size_t MT1 = (size_t)M * (T + 1);
    return ((MT1 + 1) & ~(size_t)1) * sizeof(float) + MT1 * sizeof(double) + WARPS * MT1 * sizeof(uint32_t) +
           (size_t)WARPS * 2 * BQ * sizeof(uint32_t);
}

template <int M, int PM>
cudaError_t run_backward_pm(cudaStream_t s, const UpdateArgs& a, const float* g, double* gtab, double* gpart)
{
    const uint32_t n_tiles = (uint32_t)((a.n + TILE - 1) / TILE);
    cudaError_t e;
    if (gpart) {
        // histogram adjoint: per-CTA tables, then a fixed-order reduction
        const size_t smem = backward_hist_smem(M, a.T);
        auto kh = a.ent ? k_backward_hist<M, PM, true> : k_backward_hist<M, PM, false>;
        if ((e = smem_attr(kh, smem)) != cudaSuccess) return e;
        if (!n_tiles) return cudaMemsetAsync(gtab, 0, (size_t)M * a.T * sizeof(double), s);
        int grid = 0;                                 // persistent: the CTAs resident at once
        if ((e = resident_ctas(kh, smem, &grid)) != cudaSuccess) return e;
        if ((uint32_t)grid > n_tiles) grid = (int)n_tiles;
        if ((e = cudaMemsetAsync(a.counters + 2, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
        const uint32_t MT1 = M * (a.T + 1);
        double* part2 = gpart + (uint64_t)n_tiles * MT1;
        double* wtab = part2 + (uint64_t)GTAB_SEGS * MT1;             // M x W pixel weights
        k_backward_weights<<<(M * a.W + 255) / 256, 256, 0, s>>>(M, a.W, g, a.count, wtab);
        kh<<<grid, WARPS * 32, smem, s>>>(a, wtab, gpart);
        k_gtab_reduce<<<dim3((MT1 + 31) / 32, GTAB_SEGS), 256, 0, s>>>(MT1, (uint64_t)grid, gpart, part2);
        return cudaGetLastError();
    }
    const size_t table = (size_t)((M * (a.T + 1) + 1) & ~1u) * sizeof(float);
    const size_t gbytes = (size_t)M * (a.T + 1) * sizeof(double);
    const int use_smem = table + gbytes <= 96 * 1024;
    const size_t smem = table + (use_smem ? gbytes : 0);
    e = smem_attr(k_backward<M, PM>, smem);
    if (e != cudaSuccess) return e;
    if (n_tiles) k_backward<M, PM><<<n_tiles, WARPS * 32, smem, s>>>(a, g, gtab, use_smem);
    return cudaGetLastError();
}

template <int M>
cudaError_t run_backward(cudaStream_t s, const UpdateArgs& a, const float* g, double* gtab, uint32_t K,
                         float* grad_ctrl, double* gpart)
{
    cudaError_t e = a.prm.P == 1.0f ? run_backward_pm<M, POW_ONE>(s, a, g, gtab, gpart)
                                    : run_backward_pm<M, POW_GEN>(s, a, g, gtab, gpart);
    if (e != cudaSuccess) return e;
    if (gpart && a.n) {
        const uint32_t n_tiles = (uint32_t)((a.n + TILE - 1) / TILE);
        const double* part2 = gpart + (uint64_t)n_tiles * M * (a.T + 1);
        k_grad_final<<<(unsigned)((M * K + 7) / 8), 256, 0, s>>>(M, K, a.T, part2, gtab, grad_ctrl);
    } else {
        k_grad_ctrl<<<(unsigned)((M * K + 255) / 256), 256, 0, s>>>(M, K, a.T, gtab, grad_ctrl);
    }
    return cudaGetLastError();
}

template <int M>
cudaError_t run_widths(cudaStream_t s, const UpdateArgs& a, unsigned long long* q)
{
    const size_t smem = (size_t)M * (a.T + 1) * sizeof(float);
    cudaError_t e = smem_attr(k_widths<M>, smem);
    if (e != cudaSuccess) return e;
    if (a.n) k_widths<M><<<grid_cap(a.n, 256), 256, smem, s>>>(a, q);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_update(cudaStream_t s, const UpdateArgs& a) { DVL_DISPATCH_M(run_update, s, a) }

// Loads the per-edit kernels of M fields into the context now (a kernel is
// otherwise loaded at its first launch, which would add tens of ms to the
// first update after a data set is loaded).
template <int M>
cudaError_t preload_m()
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaSuccess;
    auto touch = [&](const void* f) {
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
    };
    touch((const void*)k_prepare);
    touch((const void*)k_chunk_scan);
    touch((const void*)k_finalize);
    touch((const void*)k_passA_ring<M, POW_ONE, true, ring_depth<M>(), ring_min_blocks<M>()>);
    touch((const void*)k_passA_ring<M, POW_GEN, true, ring_depth<M>(), ring_min_blocks<M>()>);
    touch((const void*)k_passA_ring<M, POW_ONE, true, ring_depth<M>(), ring_min_blocks<M>(), true>);
    touch((const void*)k_passA_ring<M, POW_ONE, true, ring_depth_ent<M>(), ring_min_blocks_ent<M>(1), false, 1>);
    touch((const void*)k_passA_ring<M, POW_ONE, true, ring_depth_ent<M>(), ring_min_blocks_ent<M>(2), false, 2>);
    touch((const void*)k_passA_ring<M, POW_ONE, true, ring_depth_ent<M>(), ring_min_blocks_ent<M>(1), true, 1>);
    touch((const void*)k_entries<M>);
    return e;
}
template <int M>
cudaError_t run_entries(cudaStream_t s, const UpdateArgs& a)
{
    if (a.n > 0) k_entries<M><<<grid_cap((a.n + 3) / 4, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_entries(cudaStream_t s, const UpdateArgs& a)
{
    DVL_DISPATCH_M(run_entries, s, a)
}

cudaError_t preload_update_kernels(uint32_t M)
{
    switch (M) {
        case 1: return preload_m<1>();
        case 2: return preload_m<2>();
        case 3: return preload_m<3>();
        case 4: return preload_m<4>();
        case 5: return preload_m<5>();
        case 6: return preload_m<6>();
        case 7: return preload_m<7>();
        case 8: return preload_m<8>();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ctrl_table(cudaStream_t s, uint32_t M, uint32_t K, uint32_t T, const float* ctrl, float* tf,
                              uint32_t* err)
{
    k_ctrl_table<<<grid_cap((uint64_t)M * T, 256), 256, 0, s>>>(M, K, T, ctrl, tf, err);
    return cudaGetLastError();
}

cudaError_t launch_backward(cudaStream_t s, const UpdateArgs& a, const float* g, double* gtab, uint32_t K,
                            float* grad_ctrl, double* gpart)
{
    DVL_DISPATCH_M(run_backward, s, a, g, gtab, K, grad_ctrl, gpart)
}

size_t backward_gpart_elems(uint32_t M, uint32_t T, uint64_t n, uint32_t W)
{
    if (backward_hist_smem(M, T) > 200 * 1024) return 0;      // tables too large: atomic adjoint
    const uint64_t n_tiles = (n + TILE - 1) / TILE;
    return (size_t)(n_tiles + GTAB_SEGS) * M * (T + 1) + (size_t)M * W;   // CTA rows, segments, weights
}

cudaError_t launch_widths(cudaStream_t s, const UpdateArgs& a, unsigned long long* q)
{
    DVL_DISPATCH_M(run_widths, s, a, q)
}

}  // namespace dvl
