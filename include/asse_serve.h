/*
 * asse_serve.h -- multi-stream serving loop of the GB300 ASSE library.  The
 * paper has no serving layer: it runs one ATV cube on one traffic stream
 * (Sec. 4.4).  A server holds many independent streams, each with its own
 * pool (own k, g, pool size) on its own CUDA stream, admits streams against a
 * device-memory budget, and runs every stream's ingest and close as captured
 * CUDA graphs, so the work of different streams overlaps on the device while
 * the host only enqueues.
 *
 * Conventions as in asse.h.  A server is driven by one host thread.
 */
#ifndef ASSE_SERVE_H
#define ASSE_SERVE_H

#include "asse.h"
#include "asse_learn.h"

#ifdef __cplusplus
extern "C" {
#endif

#define ASSE_EAGAIN 6 /* nothing ready yet / too much in flight: try again later */

#define ASSE_SERVE_RING 4 /* closes a stream may have in flight */

typedef struct asse_server asse_server;

/* A server with budget_bytes of device memory for its streams. */
ASSE_API int asse_server_create(uint64_t budget_bytes, asse_server **out);

/* Synchronise and free every stream, then the server. */
ASSE_API void asse_server_destroy(asse_server *srv);

/* Device bytes a stream with this pool configuration and batch limit takes
 * from the budget. */
ASSE_API uint64_t asse_server_stream_bytes(const asse_config *cfg, uint64_t max_batch);

/* Device bytes currently taken by open streams. */
ASSE_API uint64_t asse_server_bytes_in_use(const asse_server *srv);

/* Admit a stream: a pool for cfg whose slices close for the window of the
 * latest kp slices, accepting batches of up to max_batch pairs.  Creates its
 * CUDA stream and pool and captures its ingest and close graphs
 * (synchronises).  Returns ASSE_ENOMEM, without side effects, if the stream
 * does not fit the budget next to the open streams: the caller retries after
 * asse_server_close frees memory.  *id receives the stream id.
 * Errors: EINVAL, ENOMEM, ECUDA. */
ASSE_API int asse_server_open(asse_server *srv, const asse_config *cfg, uint32_t kp, uint64_t max_batch,
                              uint32_t *id);

/* Enqueue one batch of n pairs (host or device memory, interleaved aip, bip)
 * for the open slice of stream id, then, if close != 0, the close of that
 * slice.  Returns once the work is enqueued: pinned host or device input must
 * stay unchanged until the stream has consumed it (the next asse_server_poll
 * result of this stream or asse_server_sync); pageable host input is copied
 * before the call returns.  Returns ASSE_EAGAIN without enqueuing anything if
 * close != 0 and ASSE_SERVE_RING closes of this stream are still unreported.
 * Errors: EINVAL (n > max_batch, misalignment), EAGAIN, ECUDA. */
ASSE_API int asse_server_submit(asse_server *srv, uint32_t id, const uint32_t *pairs, uint64_t n, int where,
                                int close);

/* Non-blocking.  If the oldest unreported close of stream id has finished,
 * copy up to cap of its reported super points to out (host memory), set
 * *n_out (the full count), *slice (the closed slice's index) and *latency_ms
 * (device time from the start of the close to its report in host memory) and
 * return ASSE_OK; ASSE_EAGAIN if it has not finished or none is pending.
 * Returns ASSE_ECAPACITY (with *n_out) if the report did not fit cap, the
 * per-close copy limit (restore_cap entries), or the restore's capacity.
 * Errors: EINVAL, EAGAIN, ECAPACITY, ETIMEOUT (a bounded wait of that close's
 * scan gave up; its report is invalid), ECUDA. */
ASSE_API int asse_server_poll(asse_server *srv, uint32_t id, asse_superpoint *out, uint64_t cap, uint64_t *n_out,
                              uint64_t *slice, float *latency_ms);

/* Wait until every stream's enqueued work has finished. */
ASSE_API int asse_server_sync(asse_server *srv);

/* Close stream id: wait for its work, free its pool and memory (returned to
 * the budget).  Unpolled reports are dropped. */
ASSE_API int asse_server_close(asse_server *srv, uint32_t id);

/* Not in the paper: learned per-ATV inference in the serving loop.  Attach
 * the model mlp to stream id: from its next close on, the close graph runs,
 * between the scan and the refresh (which would change the state the
 * features read), the feature rows of every ATV, the tensor-core MLP and the
 * rule of asse_estimate_learned (exp(model) inside [0, max_log_n] and for an
 * unsaturated ATV, else Eq. 2 from its count), then the restore, the refresh
 * and the next slice, so the close-to-report latency includes the inference.
 * The estimates stay in device memory, one buffer per report slot.  The
 * stream must have no close in flight (EAGAIN: poll first); its close graphs
 * are captured again (synchronises).  The feature rows and estimate buffers
 * are charged to the budget (ENOMEM if they do not fit; the stream is then
 * unchanged).  The model is only read and must outlive the stream; one model
 * may serve several streams.  On ECUDA the stream is closed.
 * Errors: EINVAL (kp > 64, a model already attached), EAGAIN, ENOMEM, ECUDA. */
ASSE_API int asse_server_attach_model(asse_server *srv, uint32_t id, asse_mlp *mlp, float max_log_n);

/* Copy the learned estimates of the close that the last successful
 * asse_server_poll of stream id returned into out (host or device, `where`):
 * r*E floats in ATV order (row-major: row i, then the ATV index); *n_fallback
 * (may be NULL) receives how many fell back to Eq. 2.  Available until
 * ASSE_SERVE_RING further closes of the stream have been submitted.
 * Synchronises the stream.  Errors: EINVAL, ESTATE (no model attached or
 * nothing polled yet), ECAPACITY (cap < r*E), ECUDA. */
ASSE_API int asse_server_estimates(asse_server *srv, uint32_t id, float *out, uint64_t cap, int where,
                                   uint32_t *n_fallback);

/* The pool of stream id (for reading its state), or NULL. */
ASSE_API asse_pool *asse_server_pool(asse_server *srv, uint32_t id);

/* Message of the last failing call on srv. */
ASSE_API const char *asse_server_last_error(const asse_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* ASSE_SERVE_H */
