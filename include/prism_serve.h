/* prism_serve.h — many concurrent PRISM filter streams served on one GPU.
 *
 * Each stream is one camera/IMU sequence with its own map, state and
 * anchor (its own prism_config: map size, image size, intrinsics).  A
 * request is one filter step of one stream (Sec. 3.3, App. F: predict from
 * the IMU window, localise, fuse, render the next anchor; the stream's first
 * request only fuses and renders, as prism_step does for frame 1).
 *
 * Serving model (continuous batching)
 *   - Every admitted stream keeps its map, state covariance and anchor
 *     resident on the device between requests.
 *   - Streams are admitted by device-memory budget: prism_serve_open never
 *     waits; a stream whose footprint (prism_serve_stream_bytes) does not fit
 *     the budget or finds no free slot waits in FIFO order until closed
 *     streams release theirs.  Requests submitted meanwhile wait with it.
 *   - A batching thread takes, whenever fewer than max_inflight batches are
 *     on the device, the oldest pending request of every admitted stream and
 *     runs them as one batched step: each kernel of the step is one
 *     persistent launch over the work of all streams in the batch (ray tiles,
 *     pixel blocks, voxel tiles), and the whole step is one CUDA graph.
 *     Requests that arrive while a batch runs join the next one.
 *   - A completion thread timestamps each finished batch and queues one
 *     result per request (prism_serve_poll).
 *   - A stream's result does not depend on which other streams share its
 *     batches: every stream's arithmetic and reduction order are those of a
 *     prism_step on a handle with the same configuration, bit for bit.
 *
 * Ownership
 *   The server owns every stream's device memory.  Frame buffers given to
 *   prism_serve_submit (host or device memory; pinned host memory copies
 *   fastest) and map arrays given to prism_serve_open (device memory) are
 *   read asynchronously: they must stay valid and unchanged until the
 *   request's result (for a map: the stream's first result) has been polled.
 *   All entry points are thread-safe.
 *
 * Errors
 *   Calls return a prism_status (prism.h); prism_serve_last_error describes
 *   the last failure.  A CUDA failure in a server thread puts the server in
 *   a failed state: later calls return PRISM_ECUDA.  A step the device flags
 *   (a matrix that is not positive definite) is rejected as prism_step
 *   rejects it (the stream's state and map stay unchanged) and reported in
 *   its result's status as PRISM_ENOTPD; the stream continues.
 */
#ifndef PRISM_SERVE_H
#define PRISM_SERVE_H

#include <stdint.h>

#include "prism.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PRISM_SERVE_MAX_SLOTS 64

typedef struct prism_server* prism_server_handle;

typedef struct {
    int64_t hbm_budget_bytes; /* device bytes all resident streams may hold together (> 0) */
    int32_t max_slots;        /* streams resident at once, 1 .. PRISM_SERVE_MAX_SLOTS */
    int32_t storage;          /* map storage of every stream: PRISM_STORAGE_F32 or PRISM_STORAGE_BF16 */
    int32_t n_gn;             /* Gauss-Newton passes per step, every stream, 1 .. 62 */
    int32_t max_inflight;     /* batches enqueued on the device at once, 1 .. 4 */
    int32_t use_graph;        /* 1: each batch is one CUDA graph launch; 0: direct kernel launches */
    int32_t device;           /* CUDA device ordinal */
} prism_serve_config;

typedef struct {
    int32_t stream_id;
    int32_t status;           /* PRISM_OK or PRISM_ENOTPD (flag raised on the device by this step) */
    int64_t tag;              /* the tag given to prism_serve_submit */
    int64_t batch;            /* sequence number of the batch that carried the request (from 0) */
    int32_t batch_size;       /* requests in that batch */
    int32_t reserved;
    double submit_s;          /* host monotonic clock at submission, seconds */
    double done_s;            /* host monotonic clock when the batch was seen complete */
    double latency_ms;        /* (done_s - submit_s) in milliseconds */
    prism_state state;        /* the stream's posterior after the step */
} prism_serve_result;

typedef struct {
    int64_t batches;          /* batches launched */
    int64_t frames;           /* requests completed */
    int64_t max_batch;        /* largest batch */
    int64_t bytes_in_use;     /* device bytes held by resident streams */
    int64_t bytes_peak;
    int64_t budget;
    int32_t streams_resident;
    int32_t streams_queued;   /* opened, waiting for admission */
    int32_t streams_open;     /* opened and not yet released */
    int32_t reserved;
    int64_t kernel_launches;  /* kernels run by the batches (a graph launch counts its kernels) */
    int64_t graph_launches;
} prism_serve_stats;

/* Defaults: budget 64 GiB, 32 slots, bf16 maps, 10 Gauss-Newton passes,
 * 2 batches in flight, graphs on, device 0. */
void prism_serve_config_default(prism_serve_config* c);

/* Device bytes one stream with configuration cfg (with cfg->storage
 * replaced by `storage`) holds while resident: map planes, frame staging,
 * anchor, masks, state, reduction scratch.  Host-only; -1 for an invalid
 * configuration. */
int64_t prism_serve_stream_bytes(const prism_config* cfg, int32_t storage);

/* Creates the server, its CUDA stream, device tables and (with use_graph)
 * the captured batched step, and starts its two threads.  PRISM_EINVAL for
 * a bad configuration. */
prism_status prism_serve_create(const prism_serve_config* c, prism_server_handle* out);

/* Stops the threads after the batches already on the device finish, drops
 * pending requests and frees every device buffer. */
prism_status prism_serve_destroy(prism_server_handle s);

/* Opens a stream with configuration cfg (its storage and n_gn are the
 * server's) and first state s1 (NULL: identity pose, zero velocity, 1e-8
 * covariance).  occ, rgb, var_occ, var_rgb: optional initial map in the
 * dense caller layout of prism_map_load (device pointers, each may be NULL:
 * the prior value).  *stream_id receives the new id.  PRISM_ENOMEM if the
 * stream's footprint exceeds the whole budget. */
prism_status prism_serve_open(prism_server_handle s, const prism_config* cfg, const prism_state* s1,
                              const float* occ, const float* rgb, const float* var_occ, const float* var_rgb,
                              int32_t* stream_id);

/* Queues one step of a stream: IMU window imu (n x 7: t, acc xyz, gyro xyz,
 * copied before returning; ignored on the stream's first request), dt, and
 * the frame (depth W x H, rgb W x H x 3 floats; host or device memory).
 * PRISM_ESTATE after prism_serve_close. */
prism_status prism_serve_submit(prism_server_handle s, int32_t stream_id, const double* imu, int32_t n, double dt,
                                const float* depth, const float* rgb, int64_t tag);

/* No more requests for the stream; its pending ones still run, then its
 * memory is released and waiting streams are admitted. */
prism_status prism_serve_close(prism_server_handle s, int32_t stream_id);

/* Moves up to max finished results into out (oldest first), waiting up to
 * timeout_ms (0: do not wait) for the first one.  *n = results written. */
prism_status prism_serve_poll(prism_server_handle s, prism_serve_result* out, int32_t max, int32_t timeout_ms,
                              int32_t* n);

/* Waits until no request is pending or on the device (PRISM_ESTATE on
 * timeout; streams still waiting for admission with requests keep it busy). */
prism_status prism_serve_drain(prism_server_handle s, int32_t timeout_ms);

prism_status prism_serve_get_stats(prism_server_handle s, prism_serve_stats* out);

/* Bounds-check build (libprism_checked.so, see prism_check_status in
 * prism.h): synchronises the server's stream and writes the first index
 * violation of any of its streams' kernels to *word (0 for none); always 0
 * in libprism.so.  PRISM_EINVAL for a NULL argument, PRISM_ECUDA if the
 * read fails. */
prism_status prism_serve_check_status(prism_server_handle s, uint64_t* word);

/* Copies a resident stream's map to the caller's dense device arrays (any
 * may be NULL), after the requests already on the device; returns when the
 * copy is complete.  PRISM_ESTATE if the stream is not resident. */
prism_status prism_serve_map_store(prism_server_handle s, int32_t stream_id, float* occ, float* rgb,
                                   float* var_occ, float* var_rgb);

const char* prism_serve_last_error(prism_server_handle s);

#ifdef __cplusplus
}
#endif

#endif /* PRISM_SERVE_H */
