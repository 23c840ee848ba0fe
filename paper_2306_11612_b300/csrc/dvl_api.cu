// Host side of the C ABI declared in include/dvl.h: context and state
// machine, argument validation, device memory, copies, and the ordering of
// kernel launches on the context's stream.  All compute runs in the kernels
// of sfc_sort.cu and update.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <map>
#include <string>
#include <vector>

#include "dvl_internal.h"

using namespace dvl;

struct dvl_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int state = 0;                    // 0 created, 1 loaded, 2 ordered
    std::string last_error;

    uint64_t n = 0;
    uint32_t M = 0;
    size_t pitch = 0;                 // elements per field / level row (padded)

    // unsorted inputs
    int32_t* d_lower = nullptr;       // 3 x pitch
    uint8_t* d_level_in = nullptr;    // pitch
    float* d_fin = nullptr;           // M x pitch
    // curve order
    float* d_val = nullptr;           // M x pitch
    uint8_t* d_lev = nullptr;         // pitch
    uint32_t* d_perm = nullptr;       // n
    unsigned long long* d_keys = nullptr;   // n (sorted)
    // sort scratch
    unsigned long long* d_keys_alt = nullptr;
    uint32_t* d_vals_alt = nullptr;
    uint32_t* d_hist = nullptr;       // 8 x 256
    unsigned long long* d_rs_status = nullptr;
    uint32_t* d_rs_counters = nullptr;   // 8
    uint32_t epoch = 0;
    // metadata / errors
    DataMeta* d_meta = nullptr;
    uint32_t* d_err = nullptr;
    // transfer functions
    uint32_t T = 0;
    std::vector<float> h_tf, h_dom;
    std::vector<char> tf_set;
    uint32_t log_mask = 0;            // fields on the log10 value scale (bit m)
    bool tf_dirty = false;
    bool tf_device = false;           // tables built on the device from control points
    uint32_t K_ctrl = 0;
    float* d_ctrl = nullptr;          // M x K control points
    float* d_tf = nullptr;
    float* d_dom = nullptr;
    size_t tf_cap = 0;
    // update scratch
    UpdateConsts* d_consts = nullptr;
    unsigned long long* d_tile_status = nullptr;
    unsigned long long* d_chunk_prefix = nullptr;
    unsigned long long* d_step_sums = nullptr;
    uint32_t* d_counters = nullptr;
    // bins
    uint32_t W_cap = 0, W_last = 0;
    bool have_update = false;
    double* d_sum = nullptr;
    uint32_t *d_vmin = nullptr, *d_vmax = nullptr, *d_count = nullptr;
    float *d_mean = nullptr, *d_y = nullptr;
    double* d_asum = nullptr;         // alpha sums / means (want_alpha)
    float* d_amean = nullptr;
    unsigned long long* d_astep = nullptr;    // pass A's per-step / per-chunk alpha sums (want_alpha)
    unsigned long long* d_achunk = nullptr;
    unsigned long long* d_apart = nullptr;    // boundary partial alpha sums, (W + 1) x 2 x DVL_MAX_FIELDS
    uint64_t astep_chunks = 0;                // chunks the alpha step arrays were sized for
    uint32_t alpha_cap = 0;
    double* d_gtab = nullptr;         // adjoint scratch (M x T)
    double* d_gpart = nullptr;        // per-CTA adjoint tables
    size_t gpart_cap = 0;
    float* d_gin = nullptr;           // M x W
    float* d_gout = nullptr;          // M x K
    size_t gtab_cap = 0, gin_cap = 0, gout_cap = 0;
    bool last_alpha = false;
    dvl_params last_prm{};
    // value tables for range-query bins (per data set and TF domain)
    ValueTableArgs vt{};
    bool vt_valid = false;
    std::vector<float> vt_dom;
    // per-cell TF entries (M x pitch bytes at positions ent_pos) for the
    // domains ent_dom and T = ent_T, then a row of the levels at the same
    // positions (entlev_valid: written for the current data set)
    uint8_t* d_ent = nullptr;
    bool ent_valid = false, entlev_valid = false;
    std::vector<float> ent_dom;
    uint32_t ent_T = 0;
    int use_ent = 1;
    bool last_ent = false;            // the last update's width pass streamed the entries
    uint64_t ent_gen = 0, last_ent_gen = 0;   // builds of the entries; the one the last update used
    unsigned long long* d_H = nullptr;
    uint8_t* d_S = nullptr;
    ulonglong2* d_psum = nullptr;     // boundary partial terms, 2 x M per boundary
    float2* d_pmm = nullptr;
    uint32_t HS_cap = 0;
    uint8_t* d_img = nullptr;         // line-plot images for host outputs (2 x H x W)
    size_t img_cap = 0;
    bool last_rq = false;             // the last update computed pixel bounds (range queries)
    uint8_t* d_mask = nullptr;        // selection masks for host outputs
    unsigned long long* d_ranges = nullptr;
    size_t mask_cap = 0;
    // batched updates (K TFs x viewports)
    float* d_btf = nullptr;               // K x M x T
    float* d_bdom = nullptr;              // 2 x DVL_MAX_FIELDS
    UpdateConsts* d_bconsts = nullptr;    // K
    uint32_t* d_btickets = nullptr;       // 2K + 1: unused, one scan counter per TF, one chunk counter per TF group
    unsigned long long *d_btile = nullptr, *d_bprefix = nullptr, *d_bsteps = nullptr;
    PairDesc* d_pairs = nullptr;
    double* d_bsum = nullptr;
    uint32_t *d_bvmin = nullptr, *d_bvmax = nullptr, *d_bcount = nullptr;
    float *d_bmean = nullptr, *d_by = nullptr;
    unsigned long long* d_bH = nullptr;
    uint8_t* d_bS = nullptr;
    ulonglong2* d_bpsum = nullptr;
    float2* d_bpmm = nullptr;
    unsigned long long* d_bstamps = nullptr;   // 2 words: device clock at batch start / end
    std::vector<float> b_dom_dev;               // the domains last uploaded to d_bdom
    size_t btf_cap = 0, bk_cap = 0, pairs_cap = 0, bbin_cap = 0, bcnt_cap = 0, bhs_cap = 0;
    std::vector<PairDesc> b_pairs;        // of the last batch
    bool have_batch = false;
    std::map<std::vector<uint64_t>, std::pair<int, int>> b_tuned;   // shape -> (G, CTAs per SM)
    // captured graphs by launch signature (least recently used dropped first)
    std::map<std::vector<uint64_t>, std::pair<cudaGraphExec_t, uint64_t>> b_graphs;
    uint64_t b_graph_clock = 0;
    int b_G = 0, b_resid = 0, b_replayed = 0;
    // options
    int64_t spin_limit = 1 << 22;
    int fault_no_publish = 0;
    int timing = 0;
    std::vector<std::array<cudaEvent_t, 5>> ev;   // one set per timed update
};

namespace {

int fail(dvl_ctx* c, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(dvl_ctx* c, int code, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->last_error = buf;
    }
    return code;
}

int cuda_fail(dvl_ctx* c, cudaError_t e, const char* what)
{
    cudaGetLastError();   // clear a sticky-free error so later calls can proceed
    return fail(c, e == cudaErrorMemoryAllocation ? DVL_ERR_NOMEM : DVL_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

template <typename T>
void dfree(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

template <typename T>
cudaError_t dalloc(T*& p, size_t count)
{
    dfree(p);
    if (!count) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(&p), count * sizeof(T));
}

template <typename T>
cudaError_t grow(T*& p, size_t& cap, size_t need)
{
    if (need <= cap) return cudaSuccess;
    cudaError_t e = dalloc(p, need);
    if (e == cudaSuccess) cap = need;
    return e;
}

size_t pad_to(uint64_t n, size_t q) { return (size_t)((n + q - 1) / q * q); }

void free_batch(dvl_ctx* c)
{
    dfree(c->d_btf); dfree(c->d_bdom); dfree(c->d_bconsts); dfree(c->d_btickets); dfree(c->d_btile); dfree(c->d_bprefix);
    dfree(c->d_bsteps); dfree(c->d_pairs); dfree(c->d_bsum); dfree(c->d_bvmin); dfree(c->d_bvmax);
    dfree(c->d_bcount); dfree(c->d_bmean); dfree(c->d_by); dfree(c->d_bH); dfree(c->d_bS);
    dfree(c->d_bpsum); dfree(c->d_bpmm); dfree(c->d_bstamps);
    c->b_dom_dev.clear();
    c->b_pairs.clear();
    c->btf_cap = c->bk_cap = c->pairs_cap = c->bbin_cap = c->bcnt_cap = c->bhs_cap = 0;
    for (auto& kv : c->b_graphs) cudaGraphExecDestroy(kv.second.first);
    c->b_graphs.clear();
    c->have_batch = false;
}

void free_dataset(dvl_ctx* c)
{
    dfree(c->d_lower); dfree(c->d_level_in); dfree(c->d_fin);
    dfree(c->d_val); dfree(c->d_lev); dfree(c->d_perm); dfree(c->d_keys);
    dfree(c->d_keys_alt); dfree(c->d_vals_alt); dfree(c->d_rs_status);
    dfree(c->d_tile_status); dfree(c->d_chunk_prefix); dfree(c->d_step_sums);
    dfree(c->vt.loc); dfree(c->vt.blk); dfree(c->vt.raw); dfree(c->vt.pre); dfree(c->vt.suf); dfree(c->vt.bmm); dfree(c->vt.seg);
    c->vt = ValueTableArgs{};
    c->vt_valid = false;
    dfree(c->d_ent);
    c->ent_valid = false;
    c->entlev_valid = false;
    free_batch(c);
    c->state = 0;
    c->have_update = false;
}

cudaError_t enqueue_batch(dvl_ctx* c, const UpdateArgs& a, const BatchArgs& b, const ValueTableArgs& v,
                                 bool build_vt, cudaEvent_t* ev = nullptr, bool build_ent = false)
{
    // memsets and launches only, so that the sequence can be captured; ev
    // (uncaptured runs only): 5 events around prepare, pass A and the bins
    cudaStream_t s = c->stream;
    cudaError_t e;
    if (ev) cudaEventRecord(ev[0], s);
    if ((e = cudaMemsetAsync(c->d_counters, 0, 2 * sizeof(uint32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_btickets, 0, (size_t)(2 * b.K + 1) * sizeof(uint32_t), s)) != cudaSuccess) return e;
    if (b.n_tiles &&
        (e = cudaMemsetAsync(c->d_btile, 0, (size_t)b.K * b.n_tiles * sizeof(unsigned long long), s)) != cudaSuccess)
        return e;
    if ((e = launch_prepare_batch(s, a, b)) != cudaSuccess) return e;
    if (a.n == 0) {                      // no cells: empty bins (as dvl_update)
        const size_t nb = c->b_pairs.empty() ? 0 : (size_t)(c->b_pairs.back().bin_off + (uint64_t)a.M * c->b_pairs.back().W);
        const size_t nc = c->b_pairs.empty() ? 0 : (size_t)(c->b_pairs.back().cnt_off + c->b_pairs.back().W);
        if ((e = cudaMemsetAsync(c->d_bsum, 0, nb * sizeof(double), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(c->d_bvmin, 0xFF, nb * sizeof(uint32_t), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(c->d_bvmax, 0, nb * sizeof(uint32_t), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(c->d_bmean, 0, nb * sizeof(float), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(c->d_by, 0, nb * sizeof(float), s)) != cudaSuccess) return e;
        return cudaMemsetAsync(c->d_bcount, 0, nc * sizeof(uint32_t), s);
    }
    if (build_vt && (e = launch_value_tables(s, a.M, v)) != cudaSuccess) return e;
    if (build_ent && !(build_vt && v.ent)) {             // entries alone (the table pass did not write them)
        UpdateArgs ae = a;
        ae.consts = b.consts;                            // lo / s of the batch's domains
        if ((e = launch_entries(s, ae)) != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[1], s);
    if ((e = launch_passA_batch(s, a, b)) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[2], s);
    if ((e = launch_bins_batch(s, a, b, v)) != cudaSuccess) return e;
    if (ev) {
        cudaEventRecord(ev[3], s);
        cudaEventRecord(ev[4], s);
    }
    return cudaSuccess;
}

// Maps and clears the device error word.
int take_device_error(dvl_ctx* c)
{
    uint32_t e = 0;
    CK(cudaMemcpyAsync(&e, c->d_err, sizeof e, cudaMemcpyDeviceToHost, c->stream), "read error word");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    if (!e) return DVL_OK;
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), c->stream), "clear error word");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    if (e & ERR_TIMEOUT) return fail(c, DVL_ERR_TIMEOUT, "a device-side wait exceeded its limit");
    if (e & ERR_LEVEL) return fail(c, DVL_ERR_RANGE, "a cell level exceeds %d", DVL_MAX_LEVEL);
    if (e & ERR_COORD) return fail(c, DVL_ERR_RANGE, "a cell lies outside the 2^20 logical grid");
    if (e & ERR_NONFINITE) return fail(c, DVL_ERR_RANGE, "a field value is not finite");
    if (e & ERR_RANGE)
        return fail(c, DVL_ERR_RANGE, "the importance bound is not representable, or an alpha table entry "
                                      "lies outside [0, 1]");
    return fail(c, DVL_ERR_CUDA, "unknown device error 0x%x", e);
}

cudaMemcpyKind kind_in(int mem_kind) { return mem_kind == DVL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int mem_kind) { return mem_kind == DVL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

int upload_fields(dvl_ctx* c, const float* const* fields, int mem_kind)
{
    for (uint32_t m = 0; m < c->M; ++m) {
        if (!fields[m] && c->n) return fail(c, DVL_ERR_ARG, "field %u is NULL", m);
        if (c->n)
            CK(cudaMemcpyAsync(c->d_fin + m * c->pitch, fields[m], c->n * sizeof(float), kind_in(mem_kind),
                               c->stream), "copy field");
    }
    return DVL_OK;
}

// Resets the per-field min/max words (dmin, dmax lead DataMeta) and, when
// `positive`, the smallest-positive words, then reduces `vals` into them.
int reduce_ranges(dvl_ctx* c, const float* vals, bool positive)
{
    uint32_t init[2 * DVL_MAX_FIELDS];
    for (int m = 0; m < DVL_MAX_FIELDS; ++m) { init[m] = 0xFFFFFFFFu; init[DVL_MAX_FIELDS + m] = 0u; }
    CK(cudaMemcpyAsync(c->d_meta, init, sizeof init, cudaMemcpyHostToDevice, c->stream), "write meta");
    if (positive) {
        uint32_t pos[DVL_MAX_FIELDS];
        for (int m = 0; m < DVL_MAX_FIELDS; ++m) pos[m] = 0xFFFFFFFFu;
        CK(cudaMemcpyAsync(c->d_meta->dpos, pos, sizeof pos, cudaMemcpyHostToDevice, c->stream), "write meta");
    }
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    launch_field_ranges(c->stream, c->n, c->M, vals, c->pitch, c->d_meta, c->d_err, positive);
    CK(cudaGetLastError(), "field range kernel");
    return DVL_OK;
}

int compute_ranges(dvl_ctx* c) { return reduce_ranges(c, c->d_fin, true); }

// Fields flagged in `mask` that have no positive value (synchronises).
int fields_without_positive(dvl_ctx* c, uint32_t mask, uint32_t* bad)
{
    uint32_t pos[DVL_MAX_FIELDS];
    CK(cudaMemcpyAsync(pos, c->d_meta->dpos, sizeof pos, cudaMemcpyDeviceToHost, c->stream), "read meta");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    *bad = 0;
    for (uint32_t m = 0; m < c->M; ++m)
        if ((mask >> m & 1u) && pos[m] == 0xFFFFFFFFu) *bad |= 1u << m;
    return DVL_OK;
}

// Gathers the input-order fields into curve order (levels too when lin is
// given), applying the log scale of the flagged fields; the data ranges are
// then those of the gathered values.  The value tables must be rebuilt.
int gather_values(dvl_ctx* c, const uint8_t* lin, uint8_t* lout)
{
    launch_gather(c->stream, c->n, c->d_perm, c->M, c->d_fin, c->pitch, lin, c->d_val, c->pitch, lout,
                  c->log_mask, c->d_meta);
    CK(cudaGetLastError(), "gather kernel");
    if (c->log_mask) {
        int rc = reduce_ranges(c, c->d_val, false);
        if (rc) return rc;
    }
    c->vt_valid = false;
    c->ent_valid = false;
    c->entlev_valid = false;
    return DVL_OK;
}

}  // namespace

const unsigned long long* dvl::batch_stamps(const dvl_ctx* c) { return c ? c->d_bstamps : nullptr; }

extern "C" {

const char* dvl_status_string(int s)
{
    switch (s) {
        case DVL_OK: return "ok";
        case DVL_ERR_ARG: return "invalid argument";
        case DVL_ERR_STATE: return "call not allowed in the current state";
        case DVL_ERR_NOMEM: return "out of memory";
        case DVL_ERR_CUDA: return "CUDA error";
        case DVL_ERR_RANGE: return "input outside the supported domain";
        case DVL_ERR_TIMEOUT: return "device-side wait timed out";
        case DVL_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

const char* dvl_last_error(dvl_ctx* c) { return c ? c->last_error.c_str() : ""; }

int dvl_create(dvl_ctx** out, int device, void* cuda_stream)
{
    if (!out) return DVL_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return DVL_ERR_CUDA;
    }
    if (device < 0 || device >= count) return DVL_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return DVL_ERR_CUDA;
    dvl_ctx* c = new (std::nothrow) dvl_ctx;
    if (!c) return DVL_ERR_NOMEM;
    c->device = device;
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return DVL_ERR_CUDA;
        }
        c->own_stream = true;
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc(c->d_meta, 1);
    if (e == cudaSuccess) e = dalloc(c->d_err, 1);
    if (e == cudaSuccess) e = dalloc(c->d_consts, 1);
    if (e == cudaSuccess) e = dalloc(c->d_counters, 4);
    if (e == cudaSuccess) e = dalloc(c->d_hist, 8 * RS_RADIX);
    if (e == cudaSuccess) e = dalloc(c->d_rs_counters, 8);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_consts, 0, sizeof(UpdateConsts), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        dvl_destroy(c);
        return e == cudaErrorMemoryAllocation ? DVL_ERR_NOMEM : DVL_ERR_CUDA;
    }
    *out = c;
    return DVL_OK;
}

void dvl_destroy(dvl_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_dataset(c);
    dfree(c->d_meta); dfree(c->d_err); dfree(c->d_consts); dfree(c->d_counters);
    dfree(c->d_hist); dfree(c->d_rs_counters); dfree(c->d_tf); dfree(c->d_dom);
    dfree(c->d_sum); dfree(c->d_vmin); dfree(c->d_vmax); dfree(c->d_count);
    dfree(c->d_mean); dfree(c->d_y); dfree(c->d_asum); dfree(c->d_amean); dfree(c->d_ctrl);
    dfree(c->d_astep); dfree(c->d_achunk); dfree(c->d_apart);
    c->astep_chunks = 0;
    dfree(c->d_gtab); dfree(c->d_gpart); dfree(c->d_gin); dfree(c->d_gout); dfree(c->d_H); dfree(c->d_S);
    dfree(c->d_psum); dfree(c->d_pmm); dfree(c->d_img); dfree(c->d_mask); dfree(c->d_ranges);
    for (auto& set : c->ev)
        for (auto e : set) cudaEventDestroy(e);
    free_batch(c);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int dvl_set_option(dvl_ctx* c, int option, int64_t value)
{
    if (!c) return DVL_ERR_ARG;
    switch (option) {
        case DVL_OPT_SPIN_LIMIT:
            if (value < 1) return fail(c, DVL_ERR_ARG, "spin limit must be >= 1");
            c->spin_limit = value;
            return DVL_OK;
        case DVL_OPT_FAULT_NO_PUBLISH:
            c->fault_no_publish = value ? 1 : 0;
            return DVL_OK;
        case DVL_OPT_TIMING:
            c->timing = value ? 1 : 0;
            return DVL_OK;
        case DVL_OPT_ENTRIES:
            c->use_ent = value ? 1 : 0;
            return DVL_OK;
        default:
            return fail(c, DVL_ERR_ARG, "unknown option %d", option);
    }
}

int dvl_load_amr(dvl_ctx* c, uint64_t n, const int32_t* lower, const uint8_t* level, uint32_t M,
                 const float* const* fields, int mem_kind)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (n >= (1ull << 32)) return fail(c, DVL_ERR_ARG, "n_cells must be < 2^32");
    if (M < 1 || M > DVL_MAX_FIELDS) return fail(c, DVL_ERR_ARG, "n_fields must be in [1, %d]", DVL_MAX_FIELDS);
    if (mem_kind != DVL_MEM_HOST && mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    if (n && (!lower || !level || !fields)) return fail(c, DVL_ERR_ARG, "NULL input");
    cudaSetDevice(c->device);
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    free_dataset(c);
    c->n = n;
    c->M = M;
    c->pitch = pad_to(n ? n : 1, PAD);
    const size_t p = c->pitch;
    CK(dalloc(c->d_lower, 3 * p), "alloc lower");
    CK(dalloc(c->d_level_in, p), "alloc level");
    CK(dalloc(c->d_fin, (size_t)M * p), "alloc fields");
    CK(cudaMemsetAsync(c->d_fin, 0, (size_t)M * p * sizeof(float), c->stream), "clear");
    CK(cudaMemsetAsync(c->d_level_in, 0, p, c->stream), "clear");
    if (n) {
        for (int d = 0; d < 3; ++d)
            CK(cudaMemcpyAsync(c->d_lower + d * p, lower + d * n, n * sizeof(int32_t), kind_in(mem_kind),
                               c->stream), "copy lower");
        CK(cudaMemcpyAsync(c->d_level_in, level, n, kind_in(mem_kind), c->stream), "copy level");
    }
    int rc = upload_fields(c, fields, mem_kind);
    if (rc) return rc;
    DataMeta init;
    for (int m = 0; m < DVL_MAX_FIELDS; ++m) { init.dmin[m] = 0xFFFFFFFFu; init.dmax[m] = 0u; }
    init.max_level = 0;
    init.pad = 0;
    init.key_or = 0;
    for (int m = 0; m < DVL_MAX_FIELDS; ++m) init.dpos[m] = 0xFFFFFFFFu;
    CK(cudaMemcpyAsync(c->d_meta, &init, sizeof init, cudaMemcpyHostToDevice, c->stream), "write meta");
    launch_validate(c->stream, n, c->d_lower, c->d_level_in, M, nullptr, p, c->d_meta, c->d_err);
    launch_field_ranges(c->stream, n, M, c->d_fin, p, c->d_meta, c->d_err, true);
    CK(cudaGetLastError(), "validation kernels");
    rc = take_device_error(c);     // synchronises: inputs are consumed on return
    if (rc) { free_dataset(c); return rc; }
    c->T = 0;
    c->tf_set.assign(M, 0);
    c->h_tf.clear();
    c->h_dom.assign(2 * M, NAN);
    c->log_mask = 0;
    c->tf_dirty = true;
    c->state = 1;
    return DVL_OK;
}

int dvl_build_order(dvl_ctx* c, int sfc)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (sfc != DVL_SFC_MORTON && sfc != DVL_SFC_HILBERT) return fail(c, DVL_ERR_ARG, "bad sfc");
    if (c->state < 1) return fail(c, DVL_ERR_STATE, "no data set loaded");
    cudaSetDevice(c->device);
    const uint64_t n = c->n;
    const size_t p = c->pitch;
    CK(dalloc(c->d_keys, n), "alloc keys");
    CK(dalloc(c->d_perm, n), "alloc perm");
    CK(dalloc(c->d_keys_alt, n), "alloc keys");
    CK(dalloc(c->d_vals_alt, n), "alloc vals");
    const uint64_t rs_tiles = (n + RS_TILE - 1) / RS_TILE;
    const uint64_t rs_words = (rs_tiles ? rs_tiles : 1) * RS_RADIX;
    CK(dalloc(c->d_rs_status, rs_words), "alloc sort status");
    CK(cudaMemsetAsync(c->d_rs_status, 0, rs_words * 8, c->stream), "clear");
    CK(cudaMemsetAsync(c->d_hist, 0, 8 * RS_RADIX * 4, c->stream), "clear");
    CK(cudaMemsetAsync(c->d_rs_counters, 0, 8 * 4, c->stream), "clear");
    CK(cudaMemsetAsync(&c->d_meta->key_or, 0, 8, c->stream), "clear");
    launch_keys(c->stream, n, c->d_lower, p, c->d_level_in, sfc, c->d_keys, c->d_perm, c->d_hist, c->d_meta);
    CK(cudaGetLastError(), "key kernel");
    unsigned long long key_or = 0;
    CK(cudaMemcpyAsync(&key_or, &c->d_meta->key_or, 8, cudaMemcpyDeviceToHost, c->stream), "read key bits");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    int bits = 0;
    while (bits < 64 && (key_or >> bits)) ++bits;
    const int passes = (bits + RS_BITS - 1) / RS_BITS;
    unsigned long long *kin = c->d_keys, *kout = c->d_keys_alt;
    uint32_t *vin = c->d_perm, *vout = c->d_vals_alt;
    for (int ps = 0; ps < passes; ++ps) {
        if (++c->epoch >= (1u << 24)) {     // tag space exhausted: clear and restart
            CK(cudaMemsetAsync(c->d_rs_status, 0, rs_words * 8, c->stream), "clear");
            c->epoch = 1;
        }
        CK(launch_onesweep(c->stream, n, kin, vin, kout, vout, ps * RS_BITS, c->d_hist + ps * RS_RADIX,
                           c->d_rs_status, c->epoch, c->d_rs_counters + ps, c->d_err, c->spin_limit),
           "radix pass");
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    // results live in kin/vin; make them the canonical arrays
    if (kin != c->d_keys) std::swap(c->d_keys, c->d_keys_alt);
    if (vin != c->d_perm) std::swap(c->d_perm, c->d_vals_alt);
    dfree(c->d_keys_alt);
    dfree(c->d_vals_alt);
    dfree(c->d_rs_status);
    CK(dalloc(c->d_val, (size_t)c->M * p), "alloc sorted fields");
    CK(dalloc(c->d_lev, p), "alloc sorted levels");
    CK(cudaMemsetAsync(c->d_val, 0, (size_t)c->M * p * sizeof(float), c->stream), "clear");
    CK(cudaMemsetAsync(c->d_lev, 0, p, c->stream), "clear");
    {
        int rc = gather_values(c, c->d_level_in, c->d_lev);
        if (rc) return rc;
    }
    const uint64_t tiles = (n + TILE - 1) / TILE;
    // one status word per tile, and at least one per chunk-scan block and
    // quantity (the widths and each field's alpha sums)
    const uint64_t scan_blocks = (tiles * WARPS + 511) / 512;           // chunk-scan blocks of 512 chunks
    CK(dalloc(c->d_tile_status, std::max<uint64_t>(tiles, (1 + DVL_MAX_FIELDS) * scan_blocks)), "alloc scan state");
    CK(dalloc(c->d_chunk_prefix, tiles * WARPS), "alloc scan state");
    CK(dalloc(c->d_step_sums, tiles * WARPS * STEPS), "alloc scan state");
    {
        ValueTableArgs& v = c->vt;
        v.n = n;
        v.val = c->d_val;
        v.pitch = p;
        v.consts = c->d_consts;
        v.err = c->d_err;
        v.n_steps = (n + STEP - 1) / STEP;
        v.n_blocks = (v.n_steps + VT_BLOCK - 1) / VT_BLOCK;
        v.b_levels = value_table_levels(v.n_blocks);
        const size_t M = c->M, ns = v.n_steps ? v.n_steps : 1;
        CK(dalloc(v.loc, M * (v.n_steps + 1)), "alloc value tables");
        CK(dalloc(v.blk, M * (v.n_blocks + 1)), "alloc value tables");
        CK(dalloc(v.raw, M * ns), "alloc value tables");
        CK(dalloc(v.pre, M * ns), "alloc value tables");
        CK(dalloc(v.suf, M * ns), "alloc value tables");
        CK(dalloc(v.bmm, M * (v.b_levels ? (size_t)v.b_levels * v.n_blocks : 1)), "alloc value tables");
        CK(dalloc(v.seg, M * std::max<uint64_t>(value_table_segments(v.n_blocks), 1)), "alloc value tables");
        c->vt_valid = false;
        c->ent_valid = false;
        c->entlev_valid = false;
    }
    int rc = take_device_error(c);
    if (rc) return rc;
    // the unsorted coordinates are no longer needed; fields stay for set_fields
    dfree(c->d_lower);
    dfree(c->d_level_in);
    CK(preload_update_kernels(c->M), "load update kernels");
    CK(preload_bins_kernels(c->M), "load bin kernels");
    c->state = 2;
    return DVL_OK;
}

int dvl_set_fields(dvl_ctx* c, uint32_t M, const float* const* fields, int mem_kind)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (c->state < 2) return fail(c, DVL_ERR_STATE, "order not built");
    if (M != c->M) return fail(c, DVL_ERR_ARG, "n_fields %u != loaded %u", M, c->M);
    if (mem_kind != DVL_MEM_HOST && mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    if (c->n && !fields) return fail(c, DVL_ERR_ARG, "NULL fields");
    cudaSetDevice(c->device);
    int rc = upload_fields(c, fields, mem_kind);
    if (rc) return rc;
    rc = compute_ranges(c);
    if (rc) return rc;
    uint32_t bad = 0;
    if (c->log_mask) {
        rc = fields_without_positive(c, c->log_mask, &bad);
        if (rc) return rc;
        c->log_mask &= ~bad;             // such a field falls back to the linear scale
    }
    rc = gather_values(c, nullptr, nullptr);
    if (rc) return rc;
    rc = take_device_error(c);
    if (rc) return rc;
    if (bad) return fail(c, DVL_ERR_RANGE, "log-scaled fields 0x%x have no positive value; now linear", bad);
    return DVL_OK;
}

int dvl_set_field_scale(dvl_ctx* c, uint32_t field, int scale)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (c->state < 1) return fail(c, DVL_ERR_STATE, "no data set loaded");
    if (field >= c->M) return fail(c, DVL_ERR_ARG, "field %u out of range", field);
    if (scale != DVL_SCALE_LINEAR && scale != DVL_SCALE_LOG10) return fail(c, DVL_ERR_ARG, "bad scale");
    cudaSetDevice(c->device);
    const uint32_t bit = 1u << field;
    const uint32_t mask = scale == DVL_SCALE_LOG10 ? (c->log_mask | bit) : (c->log_mask & ~bit);
    if (mask == c->log_mask) return DVL_OK;
    if (scale == DVL_SCALE_LOG10) {
        uint32_t bad = 0;
        int rc = fields_without_positive(c, bit, &bad);
        if (rc) return rc;
        if (bad) return fail(c, DVL_ERR_RANGE, "field %u has no positive value", field);
    }
    c->log_mask = mask;
    if (c->state < 2) return DVL_OK;     // applied when the order is built
    // the ranges of the input values first: a field back on the linear scale
    // takes its raw range, the others are recomputed after the gather
    int rc = reduce_ranges(c, c->d_fin, false);
    if (rc) return rc;
    rc = gather_values(c, nullptr, nullptr);
    if (rc) return rc;
    return take_device_error(c);
}

int dvl_read_values(dvl_ctx* c, uint32_t field, float* out, int mem_kind)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (c->state < 2) return fail(c, DVL_ERR_STATE, "order not built");
    if (field >= c->M) return fail(c, DVL_ERR_ARG, "field %u out of range", field);
    if (mem_kind != DVL_MEM_HOST && mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    if (c->n && !out) return fail(c, DVL_ERR_ARG, "out is NULL");
    cudaSetDevice(c->device);
    if (c->n)
        CK(cudaMemcpyAsync(out, c->d_val + field * c->pitch, c->n * sizeof(float),
                           mem_kind == DVL_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream),
           "copy values");
    if (mem_kind == DVL_MEM_HOST) return take_device_error(c);
    return DVL_OK;
}

int dvl_read_data_range(dvl_ctx* c, float* lo, float* hi)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (c->state < 1) return fail(c, DVL_ERR_STATE, "no data set loaded");
    if (!lo || !hi) return fail(c, DVL_ERR_ARG, "NULL output");
    cudaSetDevice(c->device);
    uint32_t w[2 * DVL_MAX_FIELDS];
    CK(cudaMemcpyAsync(w, c->d_meta, sizeof w, cudaMemcpyDeviceToHost, c->stream), "read meta");
    int rc = take_device_error(c);
    if (rc) return rc;
    for (uint32_t m = 0; m < c->M; ++m) {
        for (int k = 0; k < 2; ++k) {
            uint32_t u = w[k * DVL_MAX_FIELDS + m];
            u = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;     // order-preserving bits -> float bits
            float f;
            std::memcpy(&f, &u, 4);
            (k ? hi : lo)[m] = f;
        }
    }
    return DVL_OK;
}

int dvl_set_tf(dvl_ctx* c, uint32_t field, const float* alpha, uint32_t T, float lo, float hi)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (c->state < 1) return fail(c, DVL_ERR_STATE, "no data set loaded");
    if (field >= c->M) return fail(c, DVL_ERR_ARG, "field %u out of range", field);
    if (!alpha) return fail(c, DVL_ERR_ARG, "alpha is NULL");
    if (T < 2 || T > DVL_MAX_TF_ENTRIES) return fail(c, DVL_ERR_ARG, "n_entries must be in [2, %d]", DVL_MAX_TF_ENTRIES);
    for (uint32_t e = 0; e < T; ++e)
        if (!(alpha[e] >= 0.0f && alpha[e] <= 1.0f)) return fail(c, DVL_ERR_ARG, "alpha[%u] outside [0, 1]", e);
    const bool dflt = std::isnan(lo) && std::isnan(hi);
    if (!dflt && !(std::isfinite(lo) && std::isfinite(hi) && lo < hi))
        return fail(c, DVL_ERR_ARG, "domain must be finite with lo < hi, or NaN/NaN");
    if (c->tf_device) {       // leaving control-point mode: every field needs a host table again
        c->tf_device = false;
        c->tf_set.assign(c->M, 0);
        c->T = 0;
    }
    if (T != c->T) {          // a new table size invalidates the other fields' tables
        c->T = T;
        c->h_tf.assign((size_t)c->M * T, 0.0f);
        c->tf_set.assign(c->M, 0);
    }
    std::memcpy(&c->h_tf[(size_t)field * T], alpha, T * sizeof(float));
    c->h_dom[field] = lo;
    c->h_dom[c->M + field] = hi;
    c->tf_set[field] = 1;
    c->tf_dirty = true;
    return DVL_OK;
}

int dvl_set_tfs(dvl_ctx* c, uint32_t n_fields, const float* alpha, uint32_t T, const float* domain)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (c->state < 1) return fail(c, DVL_ERR_STATE, "no data set loaded");
    if (n_fields != c->M) return fail(c, DVL_ERR_ARG, "n_fields is %u, the data set has %u fields", n_fields, c->M);
    if (!alpha) return fail(c, DVL_ERR_ARG, "alpha is NULL");
    if (T < 2 || T > DVL_MAX_TF_ENTRIES) return fail(c, DVL_ERR_ARG, "n_entries must be in [2, %d]", DVL_MAX_TF_ENTRIES);
    // everything is checked before any field changes: a refused call leaves
    // the tables as they were
    const uint32_t M = c->M;
    for (size_t i = 0; i < (size_t)M * T; ++i)
        if (!(alpha[i] >= 0.0f && alpha[i] <= 1.0f))
            return fail(c, DVL_ERR_ARG, "alpha[%u][%u] outside [0, 1]", (unsigned)(i / T), (unsigned)(i % T));
    for (uint32_t m = 0; domain && m < M; ++m) {
        const float lo = domain[m], hi = domain[M + m];
        if (!(std::isnan(lo) && std::isnan(hi)) && !(std::isfinite(lo) && std::isfinite(hi) && lo < hi))
            return fail(c, DVL_ERR_ARG, "domain must be finite with lo < hi, or NaN/NaN");
    }
    for (uint32_t m = 0; m < M; ++m) {
        const int rc = dvl_set_tf(c, m, alpha + (size_t)m * T, T, domain ? domain[m] : NAN, domain ? domain[M + m] : NAN);
        if (rc) return rc;
    }
    return DVL_OK;
}

static int check_params(dvl_ctx* c, const dvl_params* p)
{
    if (!p) return fail(c, DVL_ERR_ARG, "params is NULL");
    if (!(p->P >= 0.0f) || !std::isfinite(p->P)) return fail(c, DVL_ERR_ARG, "P must be finite and >= 0");
    if (!(p->min_importance >= 0.0f) || !std::isfinite(p->min_importance))
        return fail(c, DVL_ERR_ARG, "min_importance must be finite and >= 0");
    if (p->width < 1 || p->width > DVL_MAX_WIDTH) return fail(c, DVL_ERR_ARG, "width must be in [1, %d]", DVL_MAX_WIDTH);
    if (p->min_imp_mode > 1 || p->vmax_mode > 1 || p->width_mode > 1 || p->want_alpha > 1)
        return fail(c, DVL_ERR_ARG, "bad mode");
    return DVL_OK;
}

static int ensure_update_buffers(dvl_ctx* c, uint32_t W)
{
    if (c->tf_dirty) {
        const size_t need = (size_t)c->M * c->T;
        if (need > c->tf_cap) {
            CK(dalloc(c->d_tf, need), "alloc TF");
            CK(dalloc(c->d_dom, 2 * DVL_MAX_FIELDS), "alloc TF domain");
            c->tf_cap = need;
        }
        if (!c->tf_device)
            CK(cudaMemcpyAsync(c->d_tf, c->h_tf.data(), need * sizeof(float), cudaMemcpyHostToDevice, c->stream),
               "copy TF");
        CK(cudaMemcpyAsync(c->d_dom, c->h_dom.data(), 2 * c->M * sizeof(float), cudaMemcpyHostToDevice,
                           c->stream), "copy TF domain");
        c->tf_dirty = false;
    }
    if (W > c->W_cap) {
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        const size_t MW = (size_t)c->M * W;
        CK(dalloc(c->d_sum, MW), "alloc bins");
        CK(dalloc(c->d_vmin, MW), "alloc bins");
        CK(dalloc(c->d_vmax, MW), "alloc bins");
        CK(dalloc(c->d_mean, MW), "alloc bins");
        CK(dalloc(c->d_y, MW), "alloc bins");
        CK(dalloc(c->d_count, W), "alloc bins");
        c->W_cap = W;
    }
    return DVL_OK;
}

static int ensure_alpha_buffers(dvl_ctx* c, uint32_t W)
{
    if (W > c->alpha_cap) {
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        CK(dalloc(c->d_asum, (size_t)c->M * W), "alloc alpha sums");
        CK(dalloc(c->d_amean, (size_t)c->M * W), "alloc alpha means");
        CK(dalloc(c->d_apart, (size_t)(W + 1) * 2 * DVL_MAX_FIELDS), "alloc alpha sums");
        c->alpha_cap = W;
    }
    const uint64_t chunks = (c->n + TILE - 1) / TILE * WARPS;   // pass A's chunk count
    if (chunks != c->astep_chunks || !c->d_astep) {
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        CK(dalloc(c->d_astep, (size_t)c->M * chunks * STEPS), "alloc alpha sums");
        CK(dalloc(c->d_achunk, (size_t)c->M * (chunks + 1)), "alloc alpha sums");
        c->astep_chunks = chunks;
    }
    return DVL_OK;
}

static UpdateArgs make_args(dvl_ctx* c, const dvl_params& p)
{
    UpdateArgs a;
    a.n = c->n;
    a.M = c->M;
    a.T = c->T;
    a.W = p.width;
    a.val = c->d_val;
    a.pitch = c->pitch;
    a.lev = c->d_lev;
    a.tf = c->d_tf;
    a.dom = c->d_dom;
    a.meta = c->d_meta;
    a.consts = c->d_consts;
    a.tile_status = c->d_tile_status;
    a.chunk_prefix = c->d_chunk_prefix;
    a.step_sums = c->d_step_sums;
    a.counters = c->d_counters;
    a.sum = c->d_sum;
    a.vmin = c->d_vmin;
    a.vmax = c->d_vmax;
    a.count = c->d_count;
    a.mean = c->d_mean;
    a.y = c->d_y;
    a.asum = nullptr;
    a.amean = nullptr;
    a.astep = nullptr;
    a.achunk = nullptr;
    a.apart = nullptr;
    a.vt = nullptr;
    a.vt_build = 0;
    a.ent = nullptr;
    a.ent_build = 0;
    a.ent_lev_build = 0;
    a.H = c->d_H;
    a.S = c->d_S;
    a.psum = c->d_psum;
    a.pmm = c->d_pmm;
    a.err = c->d_err;
    a.spin_limit = c->spin_limit;
    a.fault_no_publish = c->fault_no_publish;
    a.prm = p;
    a.events = nullptr;
    return a;
}

int dvl_update(dvl_ctx* c, const dvl_params* p)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    int rc = check_params(c, p);
    if (rc) return rc;
    if (c->state < 2) return fail(c, DVL_ERR_STATE, "order not built");
    for (uint32_t m = 0; m < c->M; ++m)
        if (!c->tf_set[m]) return fail(c, DVL_ERR_STATE, "field %u has no transfer function", m);
    cudaSetDevice(c->device);
    rc = ensure_update_buffers(c, p->width);
    if (rc) return rc;
    if (p->want_alpha) {
        rc = ensure_alpha_buffers(c, p->width);
        if (rc) return rc;
    }
    // bins from range queries over the value tables (which depend on the TF
    // domains); alpha means from pass A's per-step alpha sums, in the same
    // read of the cells
    if (p->width + 1 > c->HS_cap) {
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        CK(dalloc(c->d_H, p->width + 1), "alloc pixel bounds");
        CK(dalloc(c->d_S, p->width + 1), "alloc pixel bounds");
        CK(dalloc(c->d_psum, (size_t)(p->width + 1) * 2 * DVL_MAX_FIELDS), "alloc pixel bounds");
        CK(dalloc(c->d_pmm, (size_t)(p->width + 1) * 2 * DVL_MAX_FIELDS), "alloc pixel bounds");
        c->HS_cap = p->width + 1;
    }
    const bool build_vt = !c->vt_valid || c->vt_dom.size() != c->h_dom.size() ||
                          std::memcmp(c->vt_dom.data(), c->h_dom.data(), c->h_dom.size() * sizeof(float)) != 0;
    // per-cell TF entries (tables of <= 256 entries): kept per domain and T
    const bool use_ent = c->use_ent && c->T <= 256 && c->n > 0;
    bool build_ent = false;
    if (use_ent) {
        if (!c->d_ent) CK(dalloc(c->d_ent, (size_t)(c->M + 1) * c->pitch), "alloc TF entries");
        build_ent = !c->ent_valid || c->ent_T != c->T || c->ent_dom.size() != c->h_dom.size() ||
                    std::memcmp(c->ent_dom.data(), c->h_dom.data(), c->h_dom.size() * sizeof(float)) != 0;
    }
    UpdateArgs a = make_args(c, *p);
    a.vt = &c->vt;
    a.vt_build = build_vt ? 1 : 0;
    a.ent = use_ent ? c->d_ent : nullptr;
    // entries and value tables rebuilt together: the table pass writes the
    // entries as well (one read of the fields)
    const bool fuse_ent = build_ent && build_vt;
    c->vt.ent = fuse_ent ? c->d_ent : nullptr;
    c->vt.T = c->T;
    a.ent_build = build_ent && !fuse_ent ? 1 : 0;
    a.ent_lev_build = use_ent && !c->entlev_valid ? 1 : 0;
    if (p->want_alpha) {
        a.asum = c->d_asum;
        a.amean = c->d_amean;
        a.astep = c->d_astep;
        a.achunk = c->d_achunk;
        a.apart = c->d_apart;
    }
    if (c->timing) {
        std::array<cudaEvent_t, 5> set{};
        for (auto& e : set) CK(cudaEventCreate(&e), "create event");
        c->ev.push_back(set);
        a.events = c->ev.back().data();
    }
    const cudaError_t le = launch_update(c->stream, a);
    c->vt.ent = nullptr;                      // other paths (batches) never write the entries
    CK(le, "update kernels");
    if (build_vt) {
        c->vt_valid = true;
        c->vt_dom = c->h_dom;
    }
    if (build_ent) {
        c->ent_valid = true;
        c->ent_dom = c->h_dom;
        c->ent_T = c->T;
        ++c->ent_gen;
    }
    if (use_ent) c->entlev_valid = true;
    c->last_ent = use_ent;
    c->last_ent_gen = c->ent_gen;
    c->fault_no_publish = 0;
    c->W_last = p->width;
    c->last_prm = *p;
    c->last_alpha = p->want_alpha != 0;
    c->last_rq = true;
    c->have_update = true;
    return DVL_OK;
}

int dvl_rasterize(dvl_ctx* c, uint32_t height, uint32_t value_kind, uint32_t bar_field, uint8_t* lines,
                  uint8_t* bars, int mem_kind)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (!c->have_update) return fail(c, DVL_ERR_STATE, "no update has run");
    if (height < 1 || height > 65536) return fail(c, DVL_ERR_ARG, "height must be in [1, 65536]");
    if (value_kind != DVL_PLOT_MEAN && value_kind != DVL_PLOT_Y) return fail(c, DVL_ERR_ARG, "bad value_kind");
    if (bar_field >= c->M) return fail(c, DVL_ERR_ARG, "bar_field %u out of range", bar_field);
    if (!lines && !bars) return fail(c, DVL_ERR_ARG, "no output");
    if (mem_kind != DVL_MEM_HOST && mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    cudaSetDevice(c->device);
    const uint32_t W = c->W_last;
    const size_t HW = (size_t)height * W;
    uint8_t *dl = lines, *db = bars;
    if (mem_kind == DVL_MEM_HOST) {
        if (2 * HW > c->img_cap) {
            CK(cudaStreamSynchronize(c->stream), "synchronize");
            CK(dalloc(c->d_img, 2 * HW), "alloc image");
            c->img_cap = 2 * HW;
        }
        dl = lines ? c->d_img : nullptr;
        db = bars ? c->d_img + HW : nullptr;
    }
    const float* val = value_kind == DVL_PLOT_MEAN ? c->d_mean : c->d_y;
    CK(launch_raster(c->stream, val, c->M, W, height, bar_field, dl, db), "raster kernel");
    if (mem_kind == DVL_MEM_HOST) {
        if (lines) CK(cudaMemcpyAsync(lines, dl, HW, cudaMemcpyDeviceToHost, c->stream), "copy lines");
        if (bars) CK(cudaMemcpyAsync(bars, db, HW, cudaMemcpyDeviceToHost, c->stream), "copy bars");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        return take_device_error(c);
    }
    return DVL_OK;
}

static int mask_out(dvl_ctx* c, uint8_t* mask, int mem_kind, uint8_t** dev)
{
    *dev = mask;
    if (mem_kind == DVL_MEM_HOST) {
        if (c->n > c->mask_cap) {
            CK(cudaStreamSynchronize(c->stream), "synchronize");
            CK(dalloc(c->d_mask, c->n), "alloc mask");
            c->mask_cap = c->n;
        }
        *dev = c->d_mask;
    }
    return DVL_OK;
}

int dvl_brush(dvl_ctx* c, uint32_t p0, uint32_t p1, dvl_roi* out, uint8_t* mask, int mem_kind)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (!out) return fail(c, DVL_ERR_ARG, "out is NULL");
    if (!c->have_update || !c->last_rq) return fail(c, DVL_ERR_STATE, "needs a dvl_update with want_alpha = 0");
    if (p0 > p1 || p1 >= c->W_last) return fail(c, DVL_ERR_ARG, "ROI must satisfy p0 <= p1 < W");
    if (mask && mem_kind != DVL_MEM_HOST && mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    cudaSetDevice(c->device);
    int rc = take_device_error(c);
    if (rc) return rc;
    const uint32_t W = c->W_last;
    uint64_t first = 0, end = c->n;                   // selected: [first, end)
    unsigned long long h = 0;
    uint8_t st = 0;
    if (p0 > 0) {
        CK(cudaMemcpyAsync(&h, c->d_H + p0, 8, cudaMemcpyDeviceToHost, c->stream), "copy bound");
        CK(cudaMemcpyAsync(&st, c->d_S + p0, 1, cudaMemcpyDeviceToHost, c->stream), "copy bound");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        first = st ? h - 1 : h;
    }
    if (p1 + 1 < W) {
        CK(cudaMemcpyAsync(&h, c->d_H + p1 + 1, 8, cudaMemcpyDeviceToHost, c->stream), "copy bound");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        end = h;
    }
    dvl_roi r{};
    if (end > first) {
        r.first = first;
        r.last = end - 1;
        r.n_cells = end - first;
        unsigned long long k[2] = {0, 0};
        CK(cudaMemcpyAsync(&k[0], c->d_keys + r.first, 8, cudaMemcpyDeviceToHost, c->stream), "copy key");
        CK(cudaMemcpyAsync(&k[1], c->d_keys + r.last, 8, cudaMemcpyDeviceToHost, c->stream), "copy key");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        r.key_first = k[0];
        r.key_last = k[1];
    }
    if (mask) {
        uint8_t* dm = nullptr;
        if ((rc = mask_out(c, mask, mem_kind, &dm)) != DVL_OK) return rc;
        const uint64_t f = r.n_cells ? r.first : 1, l = r.n_cells ? r.last : 0;     // empty: l < f
        CK(launch_roi_mask(c->stream, c->d_perm, c->n, f, l, dm), "mask kernel");
        if (mem_kind == DVL_MEM_HOST) CK(cudaMemcpyAsync(mask, dm, c->n, cudaMemcpyDeviceToHost, c->stream), "copy mask");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
    }
    *out = r;
    return DVL_OK;
}

int dvl_select_keys(dvl_ctx* c, const uint64_t* ranges, uint32_t R, uint8_t* mask, int mem_kind)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (c->state < 2) return fail(c, DVL_ERR_STATE, "order not built");
    if (!mask || (R && !ranges)) return fail(c, DVL_ERR_ARG, "NULL argument");
    if (R > DVL_MAX_SELECT_RANGES) return fail(c, DVL_ERR_ARG, "at most %d ranges", DVL_MAX_SELECT_RANGES);
    if (mem_kind != DVL_MEM_HOST && mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    cudaSetDevice(c->device);
    if (!c->d_ranges) CK(dalloc(c->d_ranges, 2 * DVL_MAX_SELECT_RANGES), "alloc ranges");
    uint8_t* dm = nullptr;
    int rc = mask_out(c, mask, mem_kind, &dm);
    if (rc) return rc;
    if (R) CK(cudaMemcpyAsync(c->d_ranges, ranges, 2 * R * sizeof(uint64_t), cudaMemcpyHostToDevice, c->stream),
              "copy ranges");
    CK(launch_select_keys(c->stream, c->d_keys, c->d_perm, c->n, c->d_ranges, R, dm), "select kernel");
    if (mem_kind == DVL_MEM_HOST) {
        CK(cudaMemcpyAsync(mask, dm, c->n, cudaMemcpyDeviceToHost, c->stream), "copy mask");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
    }
    return DVL_OK;
}

int dvl_set_tf_ctrl(dvl_ctx* c, const float* ctrl, uint32_t K, uint32_t T, const float* domain, int mem_kind)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (c->state < 1) return fail(c, DVL_ERR_STATE, "no data set loaded");
    if (!ctrl) return fail(c, DVL_ERR_ARG, "ctrl is NULL");
    if (K < 2 || K > 1024) return fail(c, DVL_ERR_ARG, "K must be in [2, 1024]");
    if (T < 2 || T > DVL_MAX_TF_ENTRIES) return fail(c, DVL_ERR_ARG, "n_entries must be in [2, %d]", DVL_MAX_TF_ENTRIES);
    if (mem_kind != DVL_MEM_HOST && mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    const uint32_t M = c->M;
    if (mem_kind == DVL_MEM_HOST)
        for (uint32_t i = 0; i < M * K; ++i)
            if (!(ctrl[i] >= 0.0f && ctrl[i] <= 1.0f)) return fail(c, DVL_ERR_ARG, "ctrl[%u] outside [0, 1]", i);
    std::vector<float> dom(2 * M, NAN);
    if (domain) {
        for (uint32_t m = 0; m < M; ++m) {
            const float lo = domain[m], hi = domain[M + m];
            const bool dflt = std::isnan(lo) && std::isnan(hi);
            if (!dflt && !(std::isfinite(lo) && std::isfinite(hi) && lo < hi))
                return fail(c, DVL_ERR_ARG, "domain must be finite with lo < hi, or NaN/NaN");
            dom[m] = lo;
            dom[M + m] = hi;
        }
    }
    cudaSetDevice(c->device);
    const size_t need = (size_t)M * T;
    if (need > c->tf_cap) {
        CK(dalloc(c->d_tf, need), "alloc TF");
        CK(dalloc(c->d_dom, 2 * DVL_MAX_FIELDS), "alloc TF domain");
        c->tf_cap = need;
    }
    if (K != c->K_ctrl) {
        CK(dalloc(c->d_ctrl, (size_t)M * K), "alloc control points");
        c->K_ctrl = K;
    }
    CK(cudaMemcpyAsync(c->d_ctrl, ctrl, (size_t)M * K * sizeof(float), kind_in(mem_kind), c->stream), "copy ctrl");
    CK(launch_ctrl_table(c->stream, M, K, T, c->d_ctrl, c->d_tf, c->d_err), "control-point tables");
    c->h_dom = dom;
    c->T = T;
    c->tf_set.assign(M, 1);
    c->tf_device = true;
    c->tf_dirty = true;                 // uploads the domains (not the tables) at the next update
    if (mem_kind == DVL_MEM_HOST) CK(cudaStreamSynchronize(c->stream), "synchronize");
    return DVL_OK;
}

int dvl_read_alpha_means(dvl_ctx* c, float* out, int mem_kind)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (!out) return fail(c, DVL_ERR_ARG, "out is NULL");
    if (!c->have_update || !c->last_alpha) return fail(c, DVL_ERR_STATE, "last update had want_alpha = 0");
    if (mem_kind != DVL_MEM_HOST && mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    cudaSetDevice(c->device);
    if (mem_kind == DVL_MEM_HOST) {                   // device outputs stay asynchronous
        int rc = take_device_error(c);
        if (rc) return rc;
    }
    const size_t MW = (size_t)c->M * c->W_last;
    CK(cudaMemcpyAsync(out, c->d_amean, MW * sizeof(float), kind_out(mem_kind), c->stream), "copy alpha means");
    if (mem_kind == DVL_MEM_DEVICE) return DVL_OK;                              // stream-ordered
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return DVL_OK;
}

int dvl_backward(dvl_ctx* c, const float* grad, int mem_in, float* grad_ctrl, int mem_out)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (!grad || !grad_ctrl) return fail(c, DVL_ERR_ARG, "NULL gradient buffer");
    if ((mem_in != DVL_MEM_HOST && mem_in != DVL_MEM_DEVICE) || (mem_out != DVL_MEM_HOST && mem_out != DVL_MEM_DEVICE))
        return fail(c, DVL_ERR_ARG, "bad mem_kind");
    if (!c->have_update || !c->last_alpha) return fail(c, DVL_ERR_STATE, "last update had want_alpha = 0");
    if (!c->tf_device) return fail(c, DVL_ERR_STATE, "transfer functions were not set from control points");
    cudaSetDevice(c->device);
    const uint32_t M = c->M, W = c->W_last, K = c->K_ctrl, T = c->T;
    if ((size_t)M * T > c->gtab_cap) { CK(dalloc(c->d_gtab, (size_t)M * T), "alloc adjoint"); c->gtab_cap = (size_t)M * T; }
    if ((size_t)M * K > c->gout_cap) { CK(dalloc(c->d_gout, (size_t)M * K), "alloc adjoint"); c->gout_cap = (size_t)M * K; }
    const float* g = grad;
    if (mem_in == DVL_MEM_HOST) {
        if ((size_t)M * W > c->gin_cap) { CK(dalloc(c->d_gin, (size_t)M * W), "alloc adjoint"); c->gin_cap = (size_t)M * W; }
        CK(cudaMemcpyAsync(c->d_gin, grad, (size_t)M * W * sizeof(float), cudaMemcpyHostToDevice, c->stream),
           "copy gradient");
        g = c->d_gin;
    }
    CK(cudaMemsetAsync(c->d_gtab, 0, (size_t)M * T * sizeof(double), c->stream), "clear adjoint");
    UpdateArgs a = make_args(c, c->last_prm);
    // the entries of the last update, if they are still the ones it read
    if (c->last_ent && c->ent_valid && c->ent_gen == c->last_ent_gen) a.ent = c->d_ent;
    float* out = mem_out == DVL_MEM_DEVICE ? grad_ctrl : c->d_gout;
    const size_t np = backward_gpart_elems(M, T, c->n, c->W_last);
    if (np > c->gpart_cap) {
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        CK(dalloc(c->d_gpart, np), "alloc adjoint");
        c->gpart_cap = np;
    }
    CK(launch_backward(c->stream, a, g, c->d_gtab, K, out, np ? c->d_gpart : nullptr), "adjoint kernels");
    if (mem_out == DVL_MEM_HOST)
        CK(cudaMemcpyAsync(grad_ctrl, c->d_gout, (size_t)M * K * sizeof(float), cudaMemcpyDeviceToHost, c->stream),
           "copy gradient");
    if (mem_in == DVL_MEM_DEVICE && mem_out == DVL_MEM_DEVICE) return DVL_OK;   // stream-ordered, asynchronous
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return take_device_error(c);
}

int dvl_read_bins(dvl_ctx* c, uint32_t field, const dvl_bins* out)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (!out) return fail(c, DVL_ERR_ARG, "out is NULL");
    if (!c->have_update) return fail(c, DVL_ERR_STATE, "no update has run");
    if (field >= c->M) return fail(c, DVL_ERR_ARG, "field %u out of range", field);
    if (out->mem_kind != DVL_MEM_HOST && out->mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    cudaSetDevice(c->device);
    int rc = take_device_error(c);
    if (rc) return rc;
    const size_t W = c->W_last, off = (size_t)field * W;
    const cudaMemcpyKind k = kind_out(out->mem_kind);
    if (out->mean) CK(cudaMemcpyAsync(out->mean, c->d_mean + off, W * 4, k, c->stream), "copy mean");
    if (out->min) CK(cudaMemcpyAsync(out->min, c->d_vmin + off, W * 4, k, c->stream), "copy min");
    if (out->max) CK(cudaMemcpyAsync(out->max, c->d_vmax + off, W * 4, k, c->stream), "copy max");
    if (out->y) CK(cudaMemcpyAsync(out->y, c->d_y + off, W * 4, k, c->stream), "copy y");
    if (out->sum) CK(cudaMemcpyAsync(out->sum, c->d_sum + off, W * 8, k, c->stream), "copy sum");
    if (out->count) CK(cudaMemcpyAsync(out->count, c->d_count, W * 4, k, c->stream), "copy count");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return DVL_OK;
}

int dvl_read_bins_all(dvl_ctx* c, const dvl_bins* out)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (!out) return fail(c, DVL_ERR_ARG, "out is NULL");
    if (!c->have_update) return fail(c, DVL_ERR_STATE, "no update has run");
    if (out->mem_kind != DVL_MEM_HOST && out->mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    cudaSetDevice(c->device);
    // the per-field rows are adjacent on the device: one copy per array, and
    // the device error word read with them (one synchronisation in all)
    const size_t W = c->W_last, nb = (size_t)c->M * W;
    const cudaMemcpyKind k = kind_out(out->mem_kind);
    if (out->mean) CK(cudaMemcpyAsync(out->mean, c->d_mean, nb * 4, k, c->stream), "copy mean");
    if (out->min) CK(cudaMemcpyAsync(out->min, c->d_vmin, nb * 4, k, c->stream), "copy min");
    if (out->max) CK(cudaMemcpyAsync(out->max, c->d_vmax, nb * 4, k, c->stream), "copy max");
    if (out->y) CK(cudaMemcpyAsync(out->y, c->d_y, nb * 4, k, c->stream), "copy y");
    if (out->sum) CK(cudaMemcpyAsync(out->sum, c->d_sum, nb * 8, k, c->stream), "copy sum");
    if (out->count) CK(cudaMemcpyAsync(out->count, c->d_count, W * 4, k, c->stream), "copy count");
    uint32_t e = 0;
    CK(cudaMemcpyAsync(&e, c->d_err, sizeof e, cudaMemcpyDeviceToHost, c->stream), "read error word");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return e ? take_device_error(c) : DVL_OK;
}

int dvl_get_stats(dvl_ctx* c, dvl_stats* out)
{
    if (!c || !out) return fail(c, DVL_ERR_ARG, "NULL argument");
    c->last_error.clear();
    if (!c->have_update) return fail(c, DVL_ERR_STATE, "no update has run");
    cudaSetDevice(c->device);
    int rc = take_device_error(c);
    if (rc) return rc;
    UpdateConsts u;
    DataMeta meta;
    CK(cudaMemcpyAsync(&u, c->d_consts, sizeof u, cudaMemcpyDeviceToHost, c->stream), "read consts");
    CK(cudaMemcpyAsync(&meta, c->d_meta, sizeof meta, cudaMemcpyDeviceToHost, c->stream), "read meta");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    out->vmax = u.vmax;
    out->inv_vmax = u.inv_vmax;
    out->f_upper = u.f_upper;
    out->Q = u.Q;
    out->i = u.i;
    out->j = u.j;
    out->linear = u.linear;
    out->pow_exact = u.pow_n2 >= 0;
    out->F = u.F;
    out->n_cells = c->n;
    out->n_fields = c->M;
    out->max_level = meta.max_level;
    out->entries = c->last_ent ? 1u : 0u;
    out->pad = 0;
    return DVL_OK;
}

int dvl_read_order(dvl_ctx* c, uint64_t* keys, uint32_t* perm, int mem_kind)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (c->state < 2) return fail(c, DVL_ERR_STATE, "order not built");
    if (mem_kind != DVL_MEM_HOST && mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    cudaSetDevice(c->device);
    if (keys && c->n) CK(cudaMemcpyAsync(keys, c->d_keys, c->n * 8, kind_out(mem_kind), c->stream), "copy keys");
    if (perm && c->n) CK(cudaMemcpyAsync(perm, c->d_perm, c->n * 4, kind_out(mem_kind), c->stream), "copy perm");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return take_device_error(c);
}

int dvl_read_widths(dvl_ctx* c, uint64_t* q, int mem_kind)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (!q && c->n) return fail(c, DVL_ERR_ARG, "q is NULL");
    if (!c->have_update) return fail(c, DVL_ERR_STATE, "no update has run");
    if (mem_kind != DVL_MEM_HOST && mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    cudaSetDevice(c->device);
    if (!c->n) return DVL_OK;
    unsigned long long* dq = nullptr;
    if (mem_kind == DVL_MEM_DEVICE) {
        dq = reinterpret_cast<unsigned long long*>(q);
    } else {
        CK(cudaMalloc(&dq, c->n * 8), "alloc widths");
    }
    UpdateArgs a = make_args(c, c->last_prm);
    cudaError_t e = launch_widths(c->stream, a, dq);
    if (e == cudaSuccess && mem_kind == DVL_MEM_HOST)
        e = cudaMemcpyAsync(q, dq, c->n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (mem_kind == DVL_MEM_HOST) cudaFree(dq);
    if (e != cudaSuccess) return cuda_fail(c, e, "widths");
    return take_device_error(c);
}

// ---- batched updates -----------------------------------------------------------

int dvl_update_batch(dvl_ctx* c, const float* alphas, uint32_t K, uint32_t T, int mem_kind, const float* domain,
                     const dvl_params* p, const uint32_t* pair_tf, const uint32_t* pair_width, uint32_t n_pairs)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (c->state < 2) return fail(c, DVL_ERR_STATE, "order not built");
    if (!alphas || !pair_tf || !pair_width || !p) return fail(c, DVL_ERR_ARG, "NULL argument");
    if (K < 1 || K > DVL_MAX_BATCH_TF) return fail(c, DVL_ERR_ARG, "K must be in [1, %d]", DVL_MAX_BATCH_TF);
    if (n_pairs < 1 || n_pairs > DVL_MAX_BATCH_PAIRS)
        return fail(c, DVL_ERR_ARG, "n_pairs must be in [1, %d]", DVL_MAX_BATCH_PAIRS);
    if (T < 2 || T > DVL_MAX_TF_ENTRIES) return fail(c, DVL_ERR_ARG, "n_entries must be in [2, %d]", DVL_MAX_TF_ENTRIES);
    if (mem_kind != DVL_MEM_HOST && mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    dvl_params prm = *p;
    prm.width = 1;
    int rc = check_params(c, &prm);
    if (rc) return rc;
    if (prm.vmax_mode != DVL_VMAX_APPROX) return fail(c, DVL_ERR_ARG, "batched updates need vmax_mode = APPROX");
    if (prm.want_alpha) return fail(c, DVL_ERR_ARG, "batched updates need want_alpha = 0");
    const uint32_t M = c->M;
    std::vector<float> dom(2 * M, NAN);
    if (domain) {
        for (uint32_t m = 0; m < M; ++m) {
            const float lo = domain[m], hi = domain[M + m];
            const bool dflt = std::isnan(lo) && std::isnan(hi);
            if (!dflt && !(std::isfinite(lo) && std::isfinite(hi) && lo < hi))
                return fail(c, DVL_ERR_ARG, "domain must be finite with lo < hi, or NaN/NaN");
            dom[m] = lo;
            dom[M + m] = hi;
        }
    }
    const size_t nTF = (size_t)K * M * T;
    if (mem_kind == DVL_MEM_HOST)
        for (size_t i = 0; i < nTF; ++i)
            if (!(alphas[i] >= 0.0f && alphas[i] <= 1.0f)) return fail(c, DVL_ERR_ARG, "alpha[%zu] outside [0, 1]", i);
    std::vector<PairDesc> pairs(n_pairs);
    uint64_t bin_off = 0, cnt_off = 0, hs_off = 0;
    uint32_t max_W = 0;
    for (uint32_t q = 0; q < n_pairs; ++q) {
        const uint32_t k = pair_tf[q], W = pair_width[q];
        if (k >= K) return fail(c, DVL_ERR_ARG, "pair %u: TF index %u >= K", q, k);
        if (W < 1 || W > DVL_MAX_WIDTH) return fail(c, DVL_ERR_ARG, "pair %u: width must be in [1, %d]", q, DVL_MAX_WIDTH);
        pairs[q] = PairDesc{k, W, bin_off, cnt_off, hs_off, hs_off, 1u, 0u};
        bin_off += (uint64_t)M * W;
        cnt_off += W;
        hs_off += W + 1;
        max_W = W > max_W ? W : max_W;
    }
    // a pair whose width divides a wider (or equal, earlier) pair's of the same
    // TF reads that pair's pixel bounds instead of computing its own
    std::vector<std::vector<uint32_t>> by_tf(K);
    for (uint32_t q = 0; q < n_pairs; ++q) by_tf[pairs[q].k].push_back(q);
    for (uint32_t q = 0; q < n_pairs; ++q) {
        int best = -1;
        for (uint32_t r : by_tf[pairs[q].k]) {
            if (r == q || pairs[r].W % pairs[q].W) continue;
            if (pairs[r].W == pairs[q].W && r > q) continue;     // equal widths: the first one computes
            if (best < 0 || pairs[r].W > pairs[best].W || (pairs[r].W == pairs[best].W && r < (uint32_t)best))
                best = (int)r;
        }
        if (best >= 0 && pairs[best].W >= pairs[q].W) {
            pairs[q].derived = 1u;
            pairs[q].hstride = pairs[best].W / pairs[q].W;
        }
        pairs[q].src_hs_off = best >= 0 ? (uint64_t)best : (uint64_t)q;   // pair index for now
    }
    for (uint32_t q = 0; q < n_pairs; ++q)
        pairs[q].src_hs_off = pairs[q].derived ? pairs[pairs[q].src_hs_off].hs_off : pairs[q].hs_off;
    if (cnt_off > (1u << 24)) return fail(c, DVL_ERR_ARG, "sum of pair widths above 2^24");
    cudaSetDevice(c->device);

    // device buffers (grown only; a growth drops the captured graph)
    const uint64_t n_tiles = (c->n + TILE - 1) / TILE, n_chunks = n_tiles * WARPS;
    const bool need_grow = nTF > c->btf_cap || K > c->bk_cap || n_pairs > c->pairs_cap || bin_off > c->bbin_cap ||
                           cnt_off > c->bcnt_cap || hs_off > c->bhs_cap || !c->d_bdom;
    if (need_grow) {
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        if (!c->d_bdom) CK(dalloc(c->d_bdom, 2 * DVL_MAX_FIELDS), "alloc batch");
        CK(grow(c->d_btf, c->btf_cap, nTF), "alloc batch TFs");
        if (K > c->bk_cap) {
            CK(dalloc(c->d_bconsts, K), "alloc batch");
            CK(dalloc(c->d_btickets, 2 * K + 1), "alloc batch");
            CK(dalloc(c->d_btile, (size_t)K * n_tiles), "alloc batch scan state");
            CK(dalloc(c->d_bprefix, (size_t)K * n_chunks), "alloc batch scan state");
            CK(dalloc(c->d_bsteps, (size_t)K * n_chunks * STEPS), "alloc batch scan state");
            c->bk_cap = K;
        }
        CK(grow(c->d_pairs, c->pairs_cap, n_pairs), "alloc batch pairs");
        if (bin_off > c->bbin_cap) {
            CK(dalloc(c->d_bsum, bin_off), "alloc batch bins");
            CK(dalloc(c->d_bvmin, bin_off), "alloc batch bins");
            CK(dalloc(c->d_bvmax, bin_off), "alloc batch bins");
            CK(dalloc(c->d_bmean, bin_off), "alloc batch bins");
            CK(dalloc(c->d_by, bin_off), "alloc batch bins");
            c->bbin_cap = bin_off;
        }
        if (cnt_off > c->bcnt_cap) {
            CK(dalloc(c->d_bcount, cnt_off), "alloc batch bins");
            c->bcnt_cap = cnt_off;
        }
        if (hs_off > c->bhs_cap) {
            CK(dalloc(c->d_bH, hs_off), "alloc batch bins");
            CK(dalloc(c->d_bS, hs_off), "alloc batch bins");
            CK(dalloc(c->d_bpsum, hs_off * 2 * M), "alloc batch bins");
            CK(dalloc(c->d_bpmm, hs_off * 2 * M), "alloc batch bins");
            c->bhs_cap = hs_off;
        }
    }
    CK(cudaMemcpyAsync(c->d_btf, alphas, nTF * sizeof(float), kind_in(mem_kind), c->stream), "copy batch TFs");
    // the domains and pair descriptors come from pageable host memory (a copy
    // that may wait on the stream): uploaded only when they changed or the
    // device buffers were reallocated
    if (need_grow || dom.size() != c->b_dom_dev.size() ||
        std::memcmp(dom.data(), c->b_dom_dev.data(), dom.size() * sizeof(float)) != 0) {   // bits: NaN = default
        CK(cudaMemcpyAsync(c->d_bdom, dom.data(), 2 * M * sizeof(float), cudaMemcpyHostToDevice, c->stream),
           "copy batch domain");
        c->b_dom_dev = dom;
    }
    const bool same_pairs = !need_grow && pairs.size() == c->b_pairs.size() &&
                            std::memcmp(pairs.data(), c->b_pairs.data(), pairs.size() * sizeof(PairDesc)) == 0;
    if (!same_pairs)
        CK(cudaMemcpyAsync(c->d_pairs, pairs.data(), n_pairs * sizeof(PairDesc), cudaMemcpyHostToDevice, c->stream),
           "copy batch pairs");
    c->b_pairs = pairs;

    UpdateArgs a = make_args(c, prm);
    a.T = T;                             // the batch's table size (not the single-TF state's)
    a.W = 0;
    a.tf = nullptr;
    a.dom = c->d_bdom;
    a.consts = c->d_bconsts;
    a.tile_status = nullptr;
    a.chunk_prefix = nullptr;
    a.step_sums = nullptr;
    a.H = nullptr;
    a.S = nullptr;
    a.psum = nullptr;
    a.pmm = nullptr;
    int sm = 0;
    CK(cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, c->device), "device attribute");
    BatchArgs b{};
    b.K = K;
    b.tfs = c->d_btf;
    b.consts = c->d_bconsts;
    b.tickets = c->d_btickets;
    b.tile_status = c->d_btile;
    b.chunk_prefix = c->d_bprefix;
    b.step_sums = c->d_bsteps;
    b.n_tiles = n_tiles;
    b.n_chunks = n_chunks;
    b.pairs = c->d_pairs;
    b.n_pairs = n_pairs;
    b.max_W = max_W;
    b.sum = c->d_bsum;
    b.vmin = c->d_bvmin;
    b.vmax = c->d_bvmax;
    b.mean = c->d_bmean;
    b.y = c->d_by;
    b.count = c->d_bcount;
    b.H = c->d_bH;
    b.S = c->d_bS;
    b.psum = c->d_bpsum;
    b.pmm = c->d_bpmm;
    b.sm_count = sm;
    if (!c->d_bstamps) {
        CK(dalloc(c->d_bstamps, 2), "alloc batch stamps");
        CK(cudaMemsetAsync(c->d_bstamps, 0, 2 * sizeof(unsigned long long), c->stream), "clear");
    }
    b.stamps = c->d_bstamps;
    ValueTableArgs v = c->vt;
    v.consts = c->d_bconsts;             // lo / s are the same for every TF of the batch

    const bool build_vt = !c->vt_valid || c->vt_dom.size() != dom.size() ||
                          std::memcmp(c->vt_dom.data(), dom.data(), dom.size() * sizeof(float)) != 0;
    // per-cell TF entries (tables of <= 256 entries), shared with dvl_update:
    // built with the value tables when both are due, else alone
    const bool use_ent = c->use_ent && T <= 256 && c->n > 0;
    bool build_ent = false;
    if (use_ent) {
        if (!c->d_ent) CK(dalloc(c->d_ent, (size_t)(c->M + 1) * c->pitch), "alloc TF entries");
        build_ent = !c->ent_valid || c->ent_T != T || c->ent_dom.size() != dom.size() ||
                    std::memcmp(c->ent_dom.data(), dom.data(), dom.size() * sizeof(float)) != 0;
        a.ent = c->d_ent;
    }
    v.ent = build_ent && build_vt ? c->d_ent : nullptr;
    v.T = T;
    auto mark_built = [&]() {
        if (build_vt) {
            c->vt_valid = true;
            c->vt_dom = dom;
        }
        if (build_ent) {
            c->ent_valid = true;
            c->ent_dom = dom;
            c->ent_T = T;
            ++c->ent_gen;
        }
    };
    const uint32_t P1 = prm.P == 1.0f;
    const std::vector<uint64_t> shape{c->n, M, T, K, P1};
    auto tuned = c->b_tuned.find(shape);
    c->b_replayed = 0;
    if (tuned == c->b_tuned.end()) {
        // autotune: TFs per shared-memory group x resident CTAs per SM, each
        // timed on this data set (all configurations give identical results)
        b.G = K <= 4 ? 4 : 8;
        b.resid = 1;
        CK(enqueue_batch(c, a, b, v, build_vt, nullptr, build_ent), "batch kernels");
        mark_built();
        std::vector<std::pair<int, int>> cand;
        for (uint32_t G : {4u, 8u, 16u}) {        // compiled group sizes
            int blocks = 0;
            CK(passA_batch_occupancy(a, G, &blocks), "occupancy");
            for (int r = 1; r <= blocks && r <= 4; ++r) cand.push_back({(int)G, r});
            if (G >= K) break;                      // a larger group only adds empty slots
        }
        if (cand.empty()) return fail(c, DVL_ERR_UNSUPPORTED, "TF tables too large for shared memory");
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0), "create event");
        CK(cudaEventCreate(&e1), "create event");
        float best = 1e30f;
        std::pair<int, int> pick = cand[0];
        cudaError_t err = cudaSuccess;
        for (auto& gc : cand) {
            b.G = gc.first;
            b.resid = gc.second;
            float t_min = 1e30f;
            for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
                err = cudaEventRecord(e0, c->stream);
                if (err == cudaSuccess) err = enqueue_batch(c, a, b, v, false);
                if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                float t = 0.0f;
                if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
                t_min = t < t_min ? t : t_min;
            }
            if (err != cudaSuccess) break;
            if (t_min < best) {
                best = t_min;
                pick = gc;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (err != cudaSuccess) return cuda_fail(c, err, "batch autotune");
        tuned = c->b_tuned.emplace(shape, pick).first;
    } else if (build_vt || build_ent) {
        b.G = tuned->second.first;
        b.resid = tuned->second.second;
        CK(enqueue_batch(c, a, b, v, build_vt, nullptr, build_ent), "batch kernels");
        mark_built();
    }
    v.ent = nullptr;                                 // the timed and captured runs build nothing
    b.G = tuned->second.first;
    b.resid = tuned->second.second;
    c->b_G = b.G;
    c->b_resid = b.resid;
    if (c->timing) {
        // per-stage events need uncaptured launches (same kernels, no graph)
        std::array<cudaEvent_t, 5> set{};
        for (auto& e : set) CK(cudaEventCreate(&e), "create event");
        c->ev.push_back(set);
        CK(enqueue_batch(c, a, b, v, false, c->ev.back().data()), "batch kernels");
        c->have_batch = true;
        return DVL_OK;
    }
    // one captured graph per launch signature: every value the kernels take
    // by value, and every buffer address
    const std::vector<uint64_t> sig{c->n, M, T, K, P1, b.G, (uint64_t)b.resid, n_pairs, max_W, (uint64_t)sm,
                                    (uint64_t)c->spin_limit,
                                    (uint64_t)__builtin_bit_cast(uint32_t, prm.P),
                                    (uint64_t)__builtin_bit_cast(uint32_t, prm.min_importance),
                                    prm.min_imp_mode, prm.width_mode,
                                    (uint64_t)c->d_val, (uint64_t)c->d_lev, (uint64_t)c->d_meta, (uint64_t)c->d_err,
                                    (uint64_t)c->d_counters, (uint64_t)c->d_btf, (uint64_t)c->d_bdom,
                                    (uint64_t)c->d_bconsts, (uint64_t)c->d_btickets, (uint64_t)c->d_btile, (uint64_t)c->d_bprefix,
                                    (uint64_t)c->d_bsteps, (uint64_t)c->d_pairs, (uint64_t)c->d_bsum,
                                    (uint64_t)c->d_bvmin, (uint64_t)c->d_bvmax, (uint64_t)c->d_bmean,
                                    (uint64_t)c->d_by, (uint64_t)c->d_bcount, (uint64_t)c->d_bH, (uint64_t)c->d_bS,
                                    (uint64_t)c->d_bpsum, (uint64_t)c->d_bpmm, (uint64_t)c->d_bstamps,
                                    (uint64_t)v.loc, (uint64_t)v.blk, (uint64_t)v.raw, (uint64_t)v.pre,
                                    (uint64_t)v.suf, (uint64_t)v.bmm, (uint64_t)v.seg, (uint64_t)a.ent};
    constexpr size_t MAX_GRAPHS = 32;
    auto hit = c->b_graphs.find(sig);
    if (hit == c->b_graphs.end()) {
        if (c->b_graphs.size() >= MAX_GRAPHS) {
            auto lru = c->b_graphs.begin();
            for (auto it = c->b_graphs.begin(); it != c->b_graphs.end(); ++it)
                if (it->second.second < lru->second.second) lru = it;
            cudaGraphExecDestroy(lru->second.first);
            c->b_graphs.erase(lru);
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e1 = enqueue_batch(c, a, b, v, false);
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(c, e1 != cudaSuccess ? e1 : e2, "capture batch");
        }
        cudaGraphExec_t ge = nullptr;
        cudaError_t e3 = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) return cuda_fail(c, e3, "instantiate batch graph");
        hit = c->b_graphs.emplace(sig, std::make_pair(ge, 0ull)).first;
    } else {
        c->b_replayed = 1;
    }
    hit->second.second = ++c->b_graph_clock;
    CK(cudaGraphLaunch(hit->second.first, c->stream), "launch batch graph");
    c->have_batch = true;
    return DVL_OK;
}

int dvl_read_batch_bins(dvl_ctx* c, uint32_t pair, uint32_t field, const dvl_bins* out)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (!out) return fail(c, DVL_ERR_ARG, "out is NULL");
    if (!c->have_batch) return fail(c, DVL_ERR_STATE, "no batched update has run");
    if (pair >= c->b_pairs.size()) return fail(c, DVL_ERR_ARG, "pair %u out of range", pair);
    if (field >= c->M) return fail(c, DVL_ERR_ARG, "field %u out of range", field);
    if (out->mem_kind != DVL_MEM_HOST && out->mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    cudaSetDevice(c->device);
    int rc = take_device_error(c);
    if (rc) return rc;
    const PairDesc& pd = c->b_pairs[pair];
    const size_t W = pd.W, off = pd.bin_off + (size_t)field * W;
    const cudaMemcpyKind k = kind_out(out->mem_kind);
    if (out->mean) CK(cudaMemcpyAsync(out->mean, c->d_bmean + off, W * 4, k, c->stream), "copy mean");
    if (out->min) CK(cudaMemcpyAsync(out->min, c->d_bvmin + off, W * 4, k, c->stream), "copy min");
    if (out->max) CK(cudaMemcpyAsync(out->max, c->d_bvmax + off, W * 4, k, c->stream), "copy max");
    if (out->y) CK(cudaMemcpyAsync(out->y, c->d_by + off, W * 4, k, c->stream), "copy y");
    if (out->sum) CK(cudaMemcpyAsync(out->sum, c->d_bsum + off, W * 8, k, c->stream), "copy sum");
    if (out->count) CK(cudaMemcpyAsync(out->count, c->d_bcount + pd.cnt_off, W * 4, k, c->stream), "copy count");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return DVL_OK;
}

static int read_batch_all(dvl_ctx* c, const dvl_bins* out, bool sync)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (!out) return fail(c, DVL_ERR_ARG, "out is NULL");
    if (!c->have_batch) return fail(c, DVL_ERR_STATE, "no batched update has run");
    if (out->mem_kind != DVL_MEM_HOST && out->mem_kind != DVL_MEM_DEVICE) return fail(c, DVL_ERR_ARG, "bad mem_kind");
    cudaSetDevice(c->device);
    if (sync) {
        int rc = take_device_error(c);
        if (rc) return rc;
    }
    const PairDesc& last = c->b_pairs.back();
    const size_t nb = last.bin_off + (size_t)c->M * last.W, nc = last.cnt_off + last.W;
    const cudaMemcpyKind k = kind_out(out->mem_kind);
    if (out->mean) CK(cudaMemcpyAsync(out->mean, c->d_bmean, nb * 4, k, c->stream), "copy mean");
    if (out->min) CK(cudaMemcpyAsync(out->min, c->d_bvmin, nb * 4, k, c->stream), "copy min");
    if (out->max) CK(cudaMemcpyAsync(out->max, c->d_bvmax, nb * 4, k, c->stream), "copy max");
    if (out->y) CK(cudaMemcpyAsync(out->y, c->d_by, nb * 4, k, c->stream), "copy y");
    if (out->sum) CK(cudaMemcpyAsync(out->sum, c->d_bsum, nb * 8, k, c->stream), "copy sum");
    if (out->count) CK(cudaMemcpyAsync(out->count, c->d_bcount, nc * 4, k, c->stream), "copy count");
    if (sync) CK(cudaStreamSynchronize(c->stream), "synchronize");
    return DVL_OK;
}

int dvl_read_batch_all(dvl_ctx* c, const dvl_bins* out) { return read_batch_all(c, out, true); }

int dvl_read_batch_all_async(dvl_ctx* c, const dvl_bins* out) { return read_batch_all(c, out, false); }

void* dvl_stream(dvl_ctx* c) { return c ? static_cast<void*>(c->stream) : nullptr; }

int dvl_batch_config(dvl_ctx* c, int32_t out[3])
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (!out) return fail(c, DVL_ERR_ARG, "out is NULL");
    if (!c->have_batch) return fail(c, DVL_ERR_STATE, "no batched update has run");
    out[0] = c->b_G;
    out[1] = c->b_resid;
    out[2] = c->b_replayed;
    return DVL_OK;
}

int dvl_get_timings(dvl_ctx* c, double* ms, int n)
{
    if (!c) return DVL_ERR_ARG;
    c->last_error.clear();
    if (!ms || n < 4) return fail(c, DVL_ERR_ARG, "need room for 4 stage times");
    if (c->ev.empty()) return fail(c, DVL_ERR_STATE, "no timed update since the last read");
    cudaSetDevice(c->device);
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    double acc[4] = {0, 0, 0, 0};
    cudaError_t e = cudaSuccess;
    for (auto& set : c->ev)
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
            float t = 0.0f;
            e = cudaEventElapsedTime(&t, set[k], set[k + 1]);
            acc[k] += t;
        }
    const double cnt = (double)c->ev.size();
    for (auto& set : c->ev)
        for (auto ev : set) cudaEventDestroy(ev);
    c->ev.clear();
    if (e != cudaSuccess) return cuda_fail(c, e, "event time");
    for (int k = 0; k < 4; ++k) ms[k] = acc[k] / cnt;
    if (n >= 5) ms[4] = cnt;
    return take_device_error(c);
}

int dvl_sync(dvl_ctx* c)
{
    if (!c) return DVL_ERR_ARG;
    cudaSetDevice(c->device);
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return take_device_error(c);
}

}  // extern "C"
