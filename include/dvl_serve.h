/* Serving loop for DVL transfer-function edits over resident AMR data sets.
 *
 * The paper's interaction model (Sec. 3, Sec. 5) is one analyst editing the
 * alpha transfer functions of one data set and seeing the dynamic volume
 * lines update at once.  A server holds several data sets resident on one GPU
 * (each with its curve order and value tables built once) and answers a
 * stream of edit requests from many clients.  Requests for the same data set
 * that arrive while an earlier batch of that data set is on the GPU wait in
 * its queue and form the next batch (continuous batching); each batch is one
 * dvl_update_batch call on that data set's own stream, so different data
 * sets' batches overlap on the device.  A batch is admitted when an in-flight
 * slot is free and the device memory it would add fits the budget.
 *
 * Every result equals the bins of a plain dvl_update with the request's
 * tables and width on the same data set, bit for bit, whatever else is in the
 * batch or on the GPU (the batched path is exact integer arithmetic).
 *
 * Threading: one scheduler thread per server drives all GPU work; the calls
 * below may come from any host threads.  For low latency the scheduler polls
 * (one host core busy) while batches are in flight and for 0.3 ms after its
 * last activity, then sleeps until a request arrives; dvl_server_wait polls
 * its request for up to 2 ms before it sleeps.  All functions return DVL_OK
 * or a negative dvl_status code (dvl.h). */
#ifndef DVL_SERVE_H
#define DVL_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "dvl.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dvl_server dvl_server;

typedef struct dvl_server_config {
    uint64_t mem_budget;      /* device bytes the server may hold (data sets +
                                 batch buffers); 0 = 90 % of free memory at create */
    uint32_t max_batch;       /* largest batch (TFs) per data set, 1..DVL_MAX_BATCH_TF;
                                 batches are padded to a power of two <= this */
    uint32_t max_inflight;    /* batches on the GPU at once (over all data sets) */
    uint32_t n_entries;       /* alpha-table entries per field of every request */
    uint32_t max_width;       /* largest request width (memory estimate, check) */
    dvl_params params;        /* P, min_importance, min_imp_mode, width_mode of all
                                 requests (vmax_mode APPROX, want_alpha 0) */
} dvl_server_config;

int dvl_server_create(dvl_server** out, int device, const dvl_server_config* cfg);

/* Stops the scheduler after the batches on the GPU have finished; requests
 * still queued fail with DVL_ERR_STATE.  NULL is a no-op. */
void dvl_server_destroy(dvl_server* srv);

/* Loads one data set (host arrays as dvl_load_amr), builds its curve order
 * (sfc as dvl_build_order) and its value tables, and makes it resident.
 * TF domains are the fields' data ranges.  DVL_ERR_NOMEM when its estimated
 * footprint does not fit the budget.  *id receives the data set's index. */
int dvl_server_add_dataset(dvl_server* srv, uint64_t n_cells, const int32_t* lower, const uint8_t* level,
                           uint32_t n_fields, const float* const* fields, int sfc, uint32_t* id);

/* Runs one batch of every size bucket on every data set, so that the launch
 * configurations are tuned and the graphs captured before requests are
 * timed.  Blocking. */
int dvl_server_warmup(dvl_server* srv);

/* Queues one request: host alpha tables (n_fields x n_entries, in [0, 1],
 * copied before return) and the plot width (1..max_width) for data set
 * `dataset`.  *id receives the request id. */
int dvl_server_submit(dvl_server* srv, uint32_t dataset, const float* alpha, uint32_t width, uint64_t* id);

/* Waits up to timeout_s seconds (< 0: forever) for request `id` and copies
 * its bins to host memory: out->mean/min/max/y/sum hold n_fields x width
 * elements (field-major), out->count width (NULL pointers are skipped;
 * mem_kind must be DVL_MEM_HOST).  The request is released on return unless
 * the wait timed out (DVL_ERR_TIMEOUT).  A failed request returns its error. */
int dvl_server_wait(dvl_server* srv, uint64_t id, double timeout_s, const dvl_bins* out);

typedef struct dvl_server_stats {
    uint64_t submitted, completed, failed, batches;
    double mean_batch;        /* real requests per batch */
    double p50_ms, p99_ms, mean_ms, max_ms;   /* submit -> result ready */
    double cells_per_s;       /* sum of served data-set sizes / (last result - first submit) */
    uint64_t mem_used, mem_budget;
    uint64_t slot_bytes;      /* largest estimated batch-buffer bytes per TF slot */
    uint32_t n_datasets, max_batch_seen;
} dvl_server_stats;

/* Statistics since create or the last reset. */
int dvl_server_get_stats(dvl_server* srv, dvl_server_stats* out);
int dvl_server_reset_stats(dvl_server* srv);

/* One finished batch on the device timeline. */
typedef struct dvl_batch_span {
    uint32_t dataset;         /* data-set index */
    uint32_t requests;        /* real requests in the batch */
    double start_ms, end_ms;  /* CUDA events recorded on the data set's stream
                                 before and after the batch's kernels, in ms
                                 from the earliest start of the listed
                                 batches (a start event completes when the
                                 stream reaches it, which may be before its
                                 kernels get SMs) */
    double run_start_ms, run_end_ms;   /* the device clock read by the batch's
                                 first kernel when it starts and by its last
                                 kernel's blocks when they end, in ms from the
                                 earliest such start (end -1: not recorded) */
} dvl_batch_span;

/* The batches finished since create or the last reset (at most 2^20), in
 * order of completion: up to `cap` spans into out, their number into *n
 * (cap = 0 only counts).  Batches of different data sets whose run
 * intervals intersect executed on the device at the same time.  Call it while
 * no dvl_server_reset_stats runs (that recycles the events). */
int dvl_server_timeline(dvl_server* srv, dvl_batch_span* out, uint32_t cap, uint32_t* n);

/* Message of the last failing call on srv (empty if none); never NULL. */
const char* dvl_server_last_error(dvl_server* srv);

/* Scheduling rules, exposed for testing (pure functions, no GPU):
 * dvl_serve_bucket: the power-of-two batch size (<= max_batch) for k queued
 *   requests (0 for k = 0);
 * dvl_serve_admit: how many of `queued` requests a data set whose batch
 *   buffers hold cap_tf TFs may launch now, each further TF slot adding
 *   bytes_per_tf, with mem_used of mem_budget in use: the largest bucket that
 *   fits (buffers only grow), 0 if none does. */
uint32_t dvl_serve_bucket(uint32_t k, uint32_t max_batch);
uint32_t dvl_serve_admit(uint32_t queued, uint32_t max_batch, uint32_t cap_tf, uint64_t bytes_per_tf,
                         uint64_t mem_used, uint64_t mem_budget);

#ifdef __cplusplus
}
#endif
#endif /* DVL_SERVE_H */
