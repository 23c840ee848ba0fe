// Batched updates (many transfer functions x viewports per call): the
// constants of K TFs, and one persistent pass A that reads every cell once per
// group of G TFs whose alpha tables sit in shared memory, with one decoupled
// look-back scan per TF.  The bins of all (TF, viewport) pairs are answered by
// the range queries of bins.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "cell_math.cuh"
#include "consts.cuh"
#include "dvl_internal.h"

namespace dvl {

namespace {

__device__ __forceinline__ float4 lds_f32x4(uint32_t addr)
{
    float4 r;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"(addr));
    return r;
}
// ---------------------------------------------------------------------------
// Batched updates: constants of K TFs, and pass A over all of them
// ---------------------------------------------------------------------------

__global__ void k_prepare_batch(UpdateArgs a, BatchArgs b)
{
    if (b.stamps && blockIdx.x == 0 && threadIdx.x == 0) {
        b.stamps[0] = global_ns();
        b.stamps[1] = 0ull;
    }
    UpdateArgs ak = a;
    ak.tf = b.tfs + (uint64_t)blockIdx.x * a.M * a.T;
    ak.consts = b.consts + blockIdx.x;
    for (uint32_t i = threadIdx.x; i < a.M * a.T; i += blockDim.x)
        if (!(ak.tf[i] >= 0.0f && ak.tf[i] <= 1.0f)) atomicOr(a.err, ERR_RANGE);
    prepare_consts_block(ak);
}

// Pass A for all K transfer functions of a batch (all TFs share the TF
// domains), in one persistent launch: the TFs form groups of G whose alpha
// tables fit in shared memory together; a CTA holds one group's tables at a
// time and its warps claim that group's chunks one by one (see below).  Every warp step's
// cells are loaded and normalised once per group and evaluated for all G TFs;
// per TF it writes step and chunk totals (no wait on other warps or tiles:
// k_chunk_scan_batch scans the chunk totals afterwards).  G is a compile-time constant so the TF loop unrolls; per
// cell the table offsets (all fields) and the level factor 2^(L w) are
// computed once and reused by every TF of the group.  A cell's entry of a
// field is the same for every TF of the batch (one TF domain), so the group's
// tables are stored TF-innermost -- row (field m, entry e) holds the G TFs'
// alphas, padded to G + 4 floats so that consecutive entries fall in
// different shared-memory bank groups -- and one 128-bit load fetches 4 TFs'
// alphas.  With P = 1 the
// fixed-point scale 2^Q of each TF is folded into its constants: scaling by a
// power of two is exact, so rint(max(max(V/maxV, m_b) 2^L, m_a) 2^Q) equals
// rint(max(max(V (2^Q/maxV), m_b 2^Q) 2^L, m_a 2^Q)) bit for bit.
// ENT: the cells' kept TF entries (a.ent, one byte per cell and field) are
// read instead of the field values.
template <int M, int PM, int G, int ST, bool ENT = false>
__device__ __forceinline__ void passA_batch_body(const UpdateArgs& a, const BatchArgs& b)
{
    extern __shared__ float4 s_dyn[];                  // G params, the floors, the G x M x T1 tables
    __shared__ uint32_t s_claimed;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // table stride per field: ST (a compile-time constant >= T + 1, so that
    // the unrolled TF loop addresses its tables with immediate offsets), or
    // T + 1 when ST = 0
    constexpr uint32_t RS = G + 4;                     // floats per table row (field, entry)
    const uint32_t T = a.T, T1 = ST ? (uint32_t)ST : T + 1, K = b.K, MT1 = M * T1;
    const uint32_t n_groups = (K + G - 1) / G;
    // per quad of TFs, 4 float4s: (1/maxV), (m_b), (m_a), (2^Q) of its 4 TFs
    // (see above for P = 1), so that a pair of TFs' values is one register pair
    float* s_par = reinterpret_cast<float*>(s_dyn);
    // P = 1: per level L and TF, the lower bound max(m_b 2^(L w), m_a) (x 2^Q)
    // of Eq. 3's result, since max(max(r, m_b) 2^(L w), m_a) equals
    // max(r 2^(L w), max(m_b 2^(L w), m_a)) exactly (scaling by 2^(L w) is)
    float* s_floor = reinterpret_cast<float*>(s_dyn + G);                 // (DVL_MAX_LEVEL + 1) x G
    const uint32_t floor_s = (uint32_t)__cvta_generic_to_shared(s_floor);
    float* s_tf = s_floor + (DVL_MAX_LEVEL + 1) * G;   // M x T1 rows of RS floats, TF innermost
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(s_tf);
    const UpdateConsts* C0 = b.consts;
    float lo[M], sc[M];
#pragma unroll
    for (int m = 0; m < M; ++m) { lo[m] = C0->lo[m]; sc[m] = C0->s[m]; }
    const float Tf = (float)T, P = C0->P;
    const int n2 = C0->pow_n2, wshift = C0->width_shift;
    uint32_t g0 = 0xFFFFFFFFu, gk = 0;                 // the group whose tables are loaded

    auto load_group = [&](uint32_t first) {
        g0 = first;
        gk = K - g0 < (uint32_t)G ? K - g0 : (uint32_t)G;
        for (uint32_t i = tid; i < MT1 * RS; i += blockDim.x) {
            const uint32_t row = i / RS, kk = i - row * RS, m = row / T1, e = row - m * T1;
            s_tf[i] = kk < gk ? b.tfs[((uint64_t)(g0 + kk) * M + m) * T + (e < T ? e : T - 1)] : 0.0f;
        }
        for (uint32_t kk = tid; kk < G; kk += blockDim.x) {
            float4 pr = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (kk < gk) {
                const UpdateConsts* Ck = b.consts + g0 + kk;
                const bool after = Ck->min_imp_mode == DVL_MINIMP_AFTER_POWER;
                const float mb = after ? 0.0f : Ck->min_imp, ma = after ? Ck->min_imp : 0.0f;
                const float qs = Ck->qscale;
                pr = PM == POW_ONE ? make_float4(__fmul_rn(Ck->inv_vmax, qs), __fmul_rn(mb, qs), __fmul_rn(ma, qs), qs)
                                   : make_float4(Ck->inv_vmax, mb, ma, qs);
            }
            float* q4 = s_par + (kk / 4) * 16 + (kk % 4);
            q4[0] = pr.x; q4[4] = pr.y; q4[8] = pr.z; q4[12] = pr.w;
            for (int L = 0; L <= DVL_MAX_LEVEL; ++L)
                s_floor[L * G + kk] = fmaxf(__fmul_rn(pr.y, exp2i(L * wshift)), pr.z);
        }
    };

    // Each CTA starts on group blockIdx.x mod n_groups and then visits the
    // other groups in turn; within a group its warps claim chunks one at a
    // time from the group's counter (tickets[1 + K + group]), so no warp waits
    // for another until the group's chunks run out.
    const uint64_t n_chunks = b.n_chunks;
    uint32_t* group_count = b.tickets + 1 + K;
    for (uint32_t visit = 0, gi = blockIdx.x % n_groups; visit < n_groups;
         ++visit, gi = gi + 1 == n_groups ? 0 : gi + 1) {
        if (tid == 0) s_claimed = *(volatile uint32_t*)(group_count + gi);
        __syncthreads();                               // the previous group's tables are no longer read
        const uint32_t seen = s_claimed;
        __syncthreads();                               // s_claimed is rewritten at the next visit
        if (seen >= n_chunks) continue;                // block-uniform: nothing left of this group
        load_group(gi * G);
        __syncthreads();                               // tables ready
    while (true) {
        uint32_t claimed = 0;
        if (lane == 0) claimed = atomicAdd(group_count + gi, 1u);
        claimed = __shfl_sync(FULL, claimed, 0);
        if (claimed >= n_chunks) break;                // warp-uniform
        unsigned long long ct = 0;                     // lane kk: TF kk's chunk total
        const uint64_t chunk = claimed;
        const uint64_t base = chunk * CHUNK;
        // the next step's cells are loaded while this step's TFs run (the
        // same addresses as the step itself reads, one step earlier)
        float vn[4][M];
        uint32_t En[M];                                // ENT: the 4 cells' entries of field m
        uint32_t Ln = 0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            En[m] = 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) vn[j][m] = 0.0f;
        }
        auto load_ent4 = [&](uint64_t i) {
            const uint64_t ip = ent_pos(i);            // 4 cells of one 32-cell piece
#pragma unroll
            for (int m = 0; m < M; ++m) En[m] = __ldg(reinterpret_cast<const uint32_t*>(a.ent + m * a.pitch + ip));
            Ln = __ldg(reinterpret_cast<const uint32_t*>(a.lev + i));
        };
        if (base + lane * 4 < a.n) {
            if (ENT) load_ent4(base + lane * 4);
            else load4<M>(a.val, a.pitch, a.lev, base + lane * 4, vn, Ln);
        }
        for (int st = 0; st < STEPS; ++st) {
            if (base + (uint64_t)st * STEP >= a.n) break;            // warp-uniform
            const uint64_t idx = base + st * STEP + lane * 4;
            uint32_t off[4][M];                        // shared address of row (m, entry)
            float lvl[4];
            uint32_t frow[4];                          // shared address of the cell's level row of s_floor
            bool valid[4];
            float v[4][M];
            uint32_t E[M];
            const uint32_t L4 = Ln;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                E[m] = En[m];
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j][m] = vn[j][m];
            }
            const uint64_t nidx = idx + STEP;
            if (st + 1 < STEPS && nidx < a.n) {
                if (ENT) load_ent4(nidx);
                else load4<M>(a.val, a.pitch, a.lev, nidx, vn, Ln);
            }
            if (idx < a.n) {
                // past the data set's end the entry bytes are not written:
                // those cells (masked below) read entry 0
                const uint32_t keep = ENT && idx + 4 > a.n ? (1u << (8 * (uint32_t)(a.n - idx))) - 1u : 0xFFFFFFFFu;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        const uint32_t e = ENT ? ((E[m] & keep) >> (8 * j)) & 0xFFu
                                               : floor_small(__fmul_rn(norm_t(v[j][m], lo[m], sc[m]), Tf));
                        off[j][m] = s_base + (m * T1 + e) * (RS * 4);
                    }
                    const uint32_t Lj = (L4 >> (8 * j)) & 0xFF;
                    lvl[j] = exp2i((int)Lj * wshift);
                    frow[j] = floor_s + Lj * (G * 4);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
#pragma unroll
                    for (int m = 0; m < M; ++m) off[j][m] = s_base;
                    lvl[j] = 0.0f;
                    frow[j] = floor_s;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) valid[j] = idx + j < a.n;
            // lane kk keeps TF kk's step total; a step with all 128 cells
            // present (every step but the data set's last) needs no masks.
            // TFs are evaluated 4 at a time (one 128-bit table load per field).
            unsigned long long mine = 0;
            // NQ: TFs of the quad to evaluate (4, or 0 = the group's last,
            // partial quad: gk - 4 kq of them, in a loop that is not unrolled)
            auto one_quad = [&](int kq, auto full_tag, auto nq_tag) {
                constexpr bool ALL = decltype(full_tag)::value;     // every cell present
                constexpr int NQ = decltype(nq_tag)::value;
                const int nq = NQ ? NQ : (int)gk - kq * 4;
                const float4* pq = reinterpret_cast<const float4*>(s_par) + kq * 4;
                const float4 PX = pq[0], PY = pq[1], PZ = pq[2], PW = pq[3];
                const float px[4] = {PX.x, PX.y, PX.z, PX.w}, py[4] = {PY.x, PY.y, PY.z, PY.w};
                const float pz[4] = {PZ.x, PZ.y, PZ.z, PZ.w}, pw[4] = {PW.x, PW.y, PW.z, PW.w};
                unsigned long long l[4] = {0, 0, 0, 0};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float4 a4[M];
#pragma unroll
                    for (int m = 0; m < M; ++m) a4[m] = lds_f32x4(off[j][m] + (uint32_t)kq * 16u);
                    // the 4 TFs' spreads (max - min over the fields)
                    float hi[4], lw[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        float al[M];
#pragma unroll
                        for (int m = 0; m < M; ++m) al[m] = i == 0 ? a4[m].x : i == 1 ? a4[m].y : i == 2 ? a4[m].z : a4[m].w;
                        spread_ends<M>(al, hi[i], lw[i]);
                    }
                    uint32_t q[4];
                    if (PM == POW_ONE) {
                        // Eq. 3 with the level factor precomputed, 2^Q folded into
                        // the constants and the minimum importance into s_floor,
                        // two TFs per float32x2 instruction
                        const float4 fl = lds_f32x4(frow[j] + (uint32_t)kq * 16u);
                        const float flo[4] = {fl.x, fl.y, fl.z, fl.w};
#pragma unroll
                        for (int h = 0; h < 4; h += 2) {
                            const float2 sp = sub2(make_float2(hi[h], hi[h + 1]), make_float2(lw[h], lw[h + 1]));
                            const float2 r0 = mul2(sp, make_float2(px[h], px[h + 1]));
                            const float2 x = mul2(r0, make_float2(lvl[j], lvl[j]));
                            q[h] = __float2uint_rn(fmaxf(x.x, flo[h]));
                            q[h + 1] = __float2uint_rn(fmaxf(x.y, flo[h + 1]));
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float r = fmaxf(__fmul_rn(__fsub_rn(hi[i], lw[i]), px[i]), py[i]);
                            const float f = fmaxf(pow_gen(__fmul_rn(r, lvl[j]), n2, P), pz[i]);
                            q[i] = __float2uint_rn(__fmul_rn(f, pw[i]));
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (!NQ && i >= nq) break;                     // block-uniform
                        l[i] += ALL ? q[i] : (valid[j] ? q[i] : 0u);
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (!NQ && i >= nq) break;
                    const unsigned long long tot = warp_total_small(l[i]);
                    mine = lane == kq * 4 + i ? tot : mine;
                }
            };
            using full4 = std::integral_constant<int, 4>;
            using part = std::integral_constant<int, 0>;
            const int full_quads = (int)gk / 4;
            if (base + (uint64_t)(st + 1) * STEP <= a.n) {             // warp-uniform
#pragma unroll
                for (int kq = 0; kq < G / 4; ++kq) {
                    if (kq >= full_quads) break;                       // block-uniform
                    one_quad(kq, std::true_type{}, full4{});
                }
                if ((int)gk % 4) one_quad(full_quads, std::true_type{}, part{});
            } else {                                                   // the data set's last step:
#pragma unroll 1                                                       // not unrolled (compile time)
                for (int kq = 0; kq * 4 < (int)gk; ++kq) one_quad(kq, std::false_type{}, part{});
            }
            if (lane < (int)gk) {
                b.step_sums[((uint64_t)(g0 + lane) * b.n_chunks + chunk) * STEPS + st] = mine;
                ct += mine;
            }
        }
        // the warp's chunk total of each TF of the group (lane kk: TF g0 + kk);
        // k_chunk_scan_batch turns them into prefixes
        if (lane < (int)gk) b.chunk_prefix[(uint64_t)(g0 + lane) * b.n_chunks + chunk] = ct;
    }
    }
}

// The kernel: groups of 16 TFs take 128 registers (2 CTAs per SM fill the
// register file); smaller groups are capped at 112 registers so that, at 2
// CTAs per SM, an eighth of the register file stays free for other streams'
// kernels (the serving loop runs data sets side by side, mostly with small
// batches).
template <int M, int PM, int G, int ST, bool ENT>
__global__ __launch_bounds__(WARPS * 32, 2) void k_passA_batch16(UpdateArgs a, BatchArgs b)
{
    passA_batch_body<M, PM, G, ST, ENT>(a, b);
}
template <int M, int PM, int G, int ST, bool ENT>
__global__ __maxnreg__(112) void k_passA_batch8(UpdateArgs a, BatchArgs b)
{
    passA_batch_body<M, PM, G, ST, ENT>(a, b);
}
template <int M, int PM, int G, int ST, bool ENT = false>
constexpr auto passA_batch_kernel()
{
    if constexpr (G >= 16) return k_passA_batch16<M, PM, G, ST, ENT>;
    else return k_passA_batch8<M, PM, G, ST, ENT>;
}

// The chunk totals of TF blockIdx.y become exclusive prefixes: blocks of
// BSCAN_SPAN chunks taken by tickets (tickets[1 + k]), each scanned in the
// block, published, and looked back over the earlier blocks' (decoupled
// look-back with bounded waits; status words of TF k at tile_status + k *
// n_tiles).  The last block writes the TF's F (Eq. 4's total) and the
// all-zero fallback.
constexpr int BSCAN_THREADS = 256, BSCAN_PER_THREAD = 8, BSCAN_SPAN = BSCAN_THREADS * BSCAN_PER_THREAD;

__global__ __launch_bounds__(BSCAN_THREADS) void k_chunk_scan_batch(UpdateArgs a, BatchArgs b)
{
    __shared__ unsigned long long s_warp[BSCAN_THREADS / 32];
    __shared__ unsigned long long s_excl;
    __shared__ uint32_t s_b;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t k = blockIdx.y;
    if (tid == 0) s_b = atomicAdd(&b.tickets[1 + k], 1u);
    __syncthreads();
    const uint32_t blk = s_b;
    unsigned long long* row = b.chunk_prefix + (uint64_t)k * b.n_chunks;
    unsigned long long* status = b.tile_status + (uint64_t)k * b.n_tiles;
    const uint64_t c0 = (uint64_t)blk * BSCAN_SPAN + (uint64_t)tid * BSCAN_PER_THREAD;
    unsigned long long v[BSCAN_PER_THREAD], t = 0;
#pragma unroll
    for (int j = 0; j < BSCAN_PER_THREAD; ++j) {
        v[j] = c0 + j < b.n_chunks ? row[c0 + j] : 0ull;
        t += v[j];
    }
    const unsigned long long incl = warp_incl_scan_u64(t, lane);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    unsigned long long wpre = 0, agg = 0;
#pragma unroll
    for (int w = 0; w < BSCAN_THREADS / 32; ++w) {
        if (w < warp) wpre += s_warp[w];
        agg += s_warp[w];
    }
    if (warp == 0) {
        if (lane == 0) st_relaxed(status + blk, (blk == 0 ? FLAG_P : FLAG_A) | agg);
        unsigned long long excl = 0;
        if (blk > 0) {
            int64_t end = (int64_t)blk - 1;
            while (true) {
                const int64_t jt = end - lane;
                unsigned long long sv = FLAG_P;
                if (jt >= 0) {
                    long long spins = 0;
                    while (true) {
                        sv = ld_relaxed(status + jt);
                        if (sv >> 62) break;
                        if (++spins > a.spin_limit) {
                            atomicOr(a.err, ERR_TIMEOUT);
                            sv = FLAG_P;
                            break;
                        }
                        __nanosleep(100);
                    }
                }
                const unsigned pmask = __ballot_sync(FULL, (sv & FLAG_P) != 0);
                const int first = pmask ? __ffs(pmask) - 1 : 31;
                excl += warp_sum_u64(lane <= first ? (sv & VAL_MASK) : 0ull);
                if (pmask) break;
                end -= 32;
            }
            if (lane == 0) st_relaxed(status + blk, FLAG_P | (excl + agg));
        }
        if (lane == 0) s_excl = excl;
    }
    __syncthreads();
    unsigned long long run = s_excl + wpre + incl - t;
#pragma unroll
    for (int j = 0; j < BSCAN_PER_THREAD; ++j) {
        if (c0 + j < b.n_chunks) row[c0 + j] = run;
        run += v[j];
    }
    if (blk == gridDim.x - 1 && tid == 0) {
        UpdateConsts* Ck = b.consts + k;
        unsigned long long F = s_excl + agg;
        int linear = 0;
        if (F == 0 && a.n > 0) { F = a.n; linear = 1; }   // all widths 0: equal widths
        Ck->F = F;
        Ck->linear = linear;
        Ck->F_div_W = 0;
        Ck->F_mod_W = 0;
    }
}

}  // namespace

cudaError_t launch_prepare_batch(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b)
{
    k_prepare_batch<<<b.K, 256, 0, s>>>(a, b);
    return cudaGetLastError();
}

constexpr int SMALL_T1 = 257;                    // fixed table stride for T <= 256

size_t passA_batch_smem(uint32_t M, uint32_t T, uint32_t G)
{
    const uint32_t T1 = T + 1 <= (uint32_t)SMALL_T1 ? SMALL_T1 : T + 1;
    return (size_t)G * sizeof(float4) + (size_t)(DVL_MAX_LEVEL + 1) * G * sizeof(float) +
           (size_t)(G + 4) * M * T1 * sizeof(float);
}

template <int M, int PM, int G, int ST, bool ENT>
cudaError_t run_passA_batch_gs(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b)
{
    const size_t smem = passA_batch_smem(M, a.T, G);
    static std::atomic<size_t> set_bytes[MAX_DEVICES];
    constexpr auto kernel = passA_batch_kernel<M, PM, G, ST, ENT>();
    cudaError_t e = smem_attr_once(kernel, smem, set_bytes);
    if (e != cudaSuccess) return e;
    const uint64_t work = (b.n_chunks * ((b.K + G - 1) / G) + WARPS - 1) / WARPS;   // CTAs with a chunk each
    uint64_t grid = (uint64_t)b.sm_count * b.resid;
    if (grid > work) grid = work;
    if (grid) {
        kernel<<<(unsigned)grid, WARPS * 32, smem, s>>>(a, b);
        const uint32_t blocks = (uint32_t)((b.n_chunks + BSCAN_SPAN - 1) / BSCAN_SPAN);
        k_chunk_scan_batch<<<dim3(blocks, b.K), BSCAN_THREADS, 0, s>>>(a, b);
    }
    return cudaGetLastError();
}

template <int M, int PM, int G>
cudaError_t run_passA_batch_g(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b)
{
    if (a.T + 1 > (uint32_t)SMALL_T1) return run_passA_batch_gs<M, PM, G, 0, false>(s, a, b);
    return a.ent ? run_passA_batch_gs<M, PM, G, SMALL_T1, true>(s, a, b)
                 : run_passA_batch_gs<M, PM, G, SMALL_T1, false>(s, a, b);
}

template <int M, int PM>
cudaError_t run_passA_batch(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b)
{
    switch (b.G) {
        case 4: return run_passA_batch_g<M, PM, 4>(s, a, b);
        case 8: return run_passA_batch_g<M, PM, 8>(s, a, b);
        case 16: return run_passA_batch_g<M, PM, 16>(s, a, b);
        default: return cudaErrorInvalidValue;
    }
}

template <int M>
cudaError_t run_passA_batch_m(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b)
{
    return a.prm.P == 1.0f ? run_passA_batch<M, POW_ONE>(s, a, b) : run_passA_batch<M, POW_GEN>(s, a, b);
}

cudaError_t launch_passA_batch(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b)
{
    DVL_DISPATCH_M(run_passA_batch_m, s, a, b)
}

template <int M, int PM, int G, int ST, bool ENT>
cudaError_t occupancy_passA_batch_gs(const UpdateArgs& a, int* blocks)
{
    const size_t smem = passA_batch_smem(M, a.T, G);
    *blocks = 0;
    if (smem + sizeof(unsigned long long) * WARPS * G + 16 > 227 * 1024) return cudaSuccess;
    constexpr auto kernel = passA_batch_kernel<M, PM, G, ST, ENT>();
    cudaError_t e = smem_attr(kernel, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kernel, WARPS * 32, smem);
}

template <int M, int PM, int G>
cudaError_t occupancy_passA_batch_g(const UpdateArgs& a, int* blocks)
{
    if (a.T + 1 > (uint32_t)SMALL_T1) return occupancy_passA_batch_gs<M, PM, G, 0, false>(a, blocks);
    return a.ent ? occupancy_passA_batch_gs<M, PM, G, SMALL_T1, true>(a, blocks)
                 : occupancy_passA_batch_gs<M, PM, G, SMALL_T1, false>(a, blocks);
}

template <int M, int PM>
cudaError_t occupancy_passA_batch(const UpdateArgs& a, uint32_t G, int* blocks)
{
    *blocks = 0;
    switch (G) {
        case 4: return occupancy_passA_batch_g<M, PM, 4>(a, blocks);
        case 8: return occupancy_passA_batch_g<M, PM, 8>(a, blocks);
        case 16: return occupancy_passA_batch_g<M, PM, 16>(a, blocks);
        default: return cudaSuccess;            // not a compiled group size
    }
}

template <int M>
cudaError_t occupancy_passA_batch_m(const UpdateArgs& a, uint32_t G, int* blocks)
{
    return a.prm.P == 1.0f ? occupancy_passA_batch<M, POW_ONE>(a, G, blocks)
                           : occupancy_passA_batch<M, POW_GEN>(a, G, blocks);
}

cudaError_t passA_batch_occupancy(const UpdateArgs& a, uint32_t G, int* blocks)
{
    DVL_DISPATCH_M(occupancy_passA_batch_m, a, G, blocks)
}

}  // namespace dvl
