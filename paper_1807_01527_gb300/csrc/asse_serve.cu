// Multi-stream serving loop (include/asse_serve.h).
//
// Every admitted stream owns a pool on its own non-blocking CUDA stream, a
// device staging buffer for batches, and CUDA graphs captured once at
// admission: one for ingest (the kernel reads the batch size from device
// memory, so one graph serves every batch size) and ASSE_SERVE_RING for the
// close (reset, scan with the fused refresh, restore and estimate, advance of
// the device-side slice state, copies of the status and report to pinned host
// memory), one per report slot so up to ASSE_SERVE_RING closes of a stream
// can be in flight.  Streams share the device and overlap freely; admission
// charges each stream's device bytes against the server's budget.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/asse_serve.h"
#include "asse_internal.h"

using namespace asse;

namespace {

struct Slot {
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    Status *status_host = nullptr;          // pinned (in the stream's pinned block)
    asse_superpoint *report_host = nullptr; // pinned, rcap records (same block)
    uint64_t slice = 0;
    // with a model attached: this close's learned estimates (device, r*E)
    // and its count of Eq. 2 fallbacks (device, and its pinned copy)
    float *est = nullptr;
    uint32_t *nfb_dev = nullptr, *nfb_host = nullptr;
};

struct SStream {
    bool open = false;
    asse_config cfg{};
    uint32_t kp = 0;
    uint64_t max_batch = 0, bytes = 0, rcap = 0;
    cudaStream_t s = nullptr;
    asse_pool *pool = nullptr;
    uint32_t *staging = nullptr;
    unsigned long long *n_dev = nullptr;
    cudaGraphExec_t ingest = nullptr;
    // one pinned host block for the status and report copies of every slot:
    // pinning host memory is slow and freeing it may wait for the device, so
    // a stream does each once, when it opens and when it closes
    unsigned char *pinned = nullptr;
    Slot ring[ASSE_SERVE_RING];
    uint32_t head = 0, count = 0;  // in-flight closes: ring[head] is the oldest
    int last_polled = -1;          // slot of the close the last successful poll returned
    // learned inference in the close graphs (asse_server_attach_model)
    asse_mlp *mlp = nullptr;
    float max_log_n = 0.0f;
    uint16_t *x = nullptr;         // feature rows, [r*E][ASSE_FEAT] bf16, shared by the slots
    uint64_t model_bytes = 0;
};

asse_config pool_cfg(const asse_config *cfg)
{
    asse_config c = *cfg;
    c.max_batch = 2;  // the server stages batches itself
    return c;
}

void release(SStream *st)
{
    if (st->s)
        cudaStreamSynchronize(st->s);
    for (Slot &sl : st->ring) {
        if (sl.graph)
            cudaGraphExecDestroy(sl.graph);
        if (sl.start)
            cudaEventDestroy(sl.start);
        if (sl.done)
            cudaEventDestroy(sl.done);
        cudaFree(sl.est);
        cudaFree(sl.nfb_dev);
        if (sl.nfb_host)
            cudaFreeHost(sl.nfb_host);
        sl = Slot{};
    }
    if (st->pinned)
        cudaFreeHost(st->pinned);
    cudaFree(st->x);
    if (st->ingest)
        cudaGraphExecDestroy(st->ingest);
    cudaFree(st->staging);
    cudaFree(st->n_dev);
    asse_destroy(st->pool);
    if (st->s)
        cudaStreamDestroy(st->s);
    *st = SStream{};
}

// Capture what enqueue() puts on stream s into an executable graph.
template <typename Fn>
cudaError_t capture(cudaStream_t s, cudaGraphExec_t *out, Fn &&enqueue, int *rc)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return e;
    *rc = enqueue();
    e = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess && *rc == ASSE_OK)
        e = cudaGraphInstantiate(out, g, 0);
    if (g)
        cudaGraphDestroy(g);
    return e;
}

// Capture the close of one report slot: the fused close (scan with the
// refresh, restore, next slice) or, with a model attached, the scan, the
// learned inference of every ATV, then the restore, the refresh and the next
// slice; then the copies of the status and the report (and the fallback
// count) to the slot's pinned memory.
cudaError_t capture_close(SStream *st, Slot &sl, const PoolBuffers &pb, int *rc)
{
    return capture(st->s, &sl.graph,
                   [&]() {
                       if (st->mlp) {
                           if (int r = pool_enqueue_scan(st->pool, st->kp))
                               return r;
                           std::string why;
                           const FeatureView v = pool_feature_view_device(st->pool, st->kp);
                           if (int r = mlp_enqueue_learned(st->mlp, v, st->max_log_n, st->x, sl.est, sl.nfb_dev,
                                                           &why))
                               return pool_fail(st->pool, r, "learned inference: " + why);
                           if (int r = pool_enqueue_restore_refresh(st->pool))
                               return r;
                           if (cudaMemcpyAsync(sl.nfb_host, sl.nfb_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                               st->s) != cudaSuccess)
                               return (int)ASSE_ECUDA;
                       } else if (int r = pool_enqueue_close(st->pool, st->kp)) {
                           return r;
                       }
                       if (cudaMemcpyAsync(sl.status_host, pb.status, sizeof(Status), cudaMemcpyDeviceToHost,
                                           st->s) != cudaSuccess ||
                           cudaMemcpyAsync(sl.report_host, pb.report, st->rcap * sizeof(asse_superpoint),
                                           cudaMemcpyDeviceToHost, st->s) != cudaSuccess)
                           return (int)ASSE_ECUDA;
                       return (int)ASSE_OK;
                   },
                   rc);
}

}  // namespace

struct asse_server {
    uint64_t budget = 0, in_use = 0;
    std::vector<SStream *> streams;
    std::string err;
};

namespace {

int sfail(asse_server *srv, int code, const std::string &msg)
{
    srv->err = msg;
    return code;
}

SStream *get(asse_server *srv, uint32_t id)
{
    if (!srv || id >= srv->streams.size() || !srv->streams[id]->open)
        return nullptr;
    return srv->streams[id];
}

}  // namespace

extern "C" {

int asse_server_create(uint64_t budget_bytes, asse_server **out)
{
    if (!out)
        return ASSE_EINVAL;
    *out = new (std::nothrow) asse_server();
    if (!*out)
        return ASSE_ENOMEM;
    (*out)->budget = budget_bytes;
    return ASSE_OK;
}

void asse_server_destroy(asse_server *srv)
{
    if (!srv)
        return;
    for (SStream *st : srv->streams) {
        if (st->open)
            release(st);
        delete st;
    }
    delete srv;
}

uint64_t asse_server_stream_bytes(const asse_config *cfg, uint64_t max_batch)
{
    if (!cfg)
        return 0;
    const asse_config c = pool_cfg(cfg);
    return pool_device_bytes(&c) + max_batch * 8 + sizeof(unsigned long long);
}

uint64_t asse_server_bytes_in_use(const asse_server *srv) { return srv ? srv->in_use : 0; }

int asse_server_open(asse_server *srv, const asse_config *cfg, uint32_t kp, uint64_t max_batch, uint32_t *id)
{
    if (!srv || !cfg || !id || max_batch == 0)
        return srv ? sfail(srv, ASSE_EINVAL, "NULL argument or max_batch 0") : ASSE_EINVAL;
    if (kp < 1 || kp > cfg->k)
        return sfail(srv, ASSE_EINVAL, "kp must be in [1, k]");
    const uint64_t bytes = asse_server_stream_bytes(cfg, max_batch);
    if (srv->in_use + bytes > srv->budget)
        return sfail(srv, ASSE_ENOMEM, "stream does not fit the device-memory budget now");
    SStream *st = nullptr;
    uint32_t sid = 0;
    for (; sid < srv->streams.size(); sid++)
        if (!srv->streams[sid]->open)
            break;
    if (sid == srv->streams.size()) {
        st = new (std::nothrow) SStream();
        if (!st)
            return sfail(srv, ASSE_ENOMEM, "host allocation failed");
        srv->streams.push_back(st);
    }
    st = srv->streams[sid];
    st->cfg = *cfg;
    st->kp = kp;
    st->max_batch = max_batch;
    cudaError_t e = cudaStreamCreateWithFlags(&st->s, cudaStreamNonBlocking);
    int rc = ASSE_OK;
    const asse_config pc = pool_cfg(cfg);
    if (e == cudaSuccess) {
        rc = asse_create(&pc, st->s, &st->pool);
        if (rc != ASSE_OK) {
            const std::string why = asse_last_error(nullptr);
            release(st);
            return sfail(srv, rc, "pool: " + why);
        }
    }
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&st->staging, max_batch * 8);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&st->n_dev, sizeof(unsigned long long));
    const PoolBuffers pb = e == cudaSuccess ? pool_buffers(st->pool) : PoolBuffers{};
    st->rcap = pb.cap;
    if (e == cudaSuccess)
        e = capture(st->s, &st->ingest, [&]() { return pool_enqueue_ingest(st->pool, st->staging, st->n_dev); },
                    &rc);
    // per slot: the status, then the report, each part 256-byte aligned
    const size_t status_part = (sizeof(Status) + 255) / 256 * 256;
    const size_t slot_bytes = status_part + (st->rcap * sizeof(asse_superpoint) + 255) / 256 * 256;
    if (e == cudaSuccess && rc == ASSE_OK)
        e = cudaMallocHost((void **)&st->pinned, ASSE_SERVE_RING * slot_bytes);
    for (int i = 0; i < ASSE_SERVE_RING && e == cudaSuccess && rc == ASSE_OK; i++) {
        Slot &sl = st->ring[i];
        sl.status_host = reinterpret_cast<Status *>(st->pinned + i * slot_bytes);
        sl.report_host = reinterpret_cast<asse_superpoint *>(st->pinned + i * slot_bytes + status_part);
        e = cudaEventCreate(&sl.start);
        if (e == cudaSuccess)
            e = cudaEventCreate(&sl.done);
        if (e == cudaSuccess)
            e = capture_close(st, sl, pb, &rc);
    }
    if (e == cudaSuccess && rc == ASSE_OK)
        e = cudaStreamSynchronize(st->s);
    if (e != cudaSuccess || rc != ASSE_OK) {
        const std::string why = e != cudaSuccess ? cudaGetErrorString(e) : asse_last_error(st->pool);
        release(st);
        return sfail(srv, e == cudaErrorMemoryAllocation ? ASSE_ENOMEM : ASSE_ECUDA, "open: " + why);
    }
    st->bytes = bytes;
    st->open = true;
    srv->in_use += bytes;
    *id = sid;
    return ASSE_OK;
}

int asse_server_submit(asse_server *srv, uint32_t id, const uint32_t *pairs, uint64_t n, int where, int close)
{
    SStream *st = get(srv, id);
    if (!st)
        return srv ? sfail(srv, ASSE_EINVAL, "no such open stream") : ASSE_EINVAL;
    if (n > st->max_batch)
        return sfail(srv, ASSE_EINVAL, "batch larger than the stream's max_batch");
    if (n > 0 && !pairs)
        return sfail(srv, ASSE_EINVAL, "pairs is NULL");
    if (close && st->count == ASSE_SERVE_RING)
        return sfail(srv, ASSE_EAGAIN, "report ring full: poll first");
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        // the count comes from pageable memory, so the runtime has copied it
        // before cudaMemcpyAsync returns
        const unsigned long long nn = n;
        e = cudaMemcpyAsync(st->staging, pairs, n * 8,
                            where == ASSE_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st->s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(st->n_dev, &nn, sizeof nn, cudaMemcpyHostToDevice, st->s);
        if (e == cudaSuccess)
            e = cudaGraphLaunch(st->ingest, st->s);
    }
    if (e == cudaSuccess && close) {
        Slot &sl = st->ring[(st->head + st->count) % ASSE_SERVE_RING];
        asse_pool_info info;
        asse_info(st->pool, &info);
        sl.slice = info.slice;
        e = cudaEventRecord(sl.start, st->s);
        if (e == cudaSuccess)
            e = cudaGraphLaunch(sl.graph, st->s);
        if (e == cudaSuccess)
            e = cudaEventRecord(sl.done, st->s);
        if (e == cudaSuccess) {
            pool_after_close(st->pool, st->kp);
            st->count++;
        }
    }
    if (e != cudaSuccess)
        return sfail(srv, ASSE_ECUDA, std::string("submit: ") + cudaGetErrorString(e));
    return ASSE_OK;
}

int asse_server_poll(asse_server *srv, uint32_t id, asse_superpoint *out, uint64_t cap, uint64_t *n_out,
                     uint64_t *slice, float *latency_ms)
{
    SStream *st = get(srv, id);
    if (!st || !n_out)
        return srv ? sfail(srv, ASSE_EINVAL, "no such open stream or NULL argument") : ASSE_EINVAL;
    if (st->count == 0)
        return ASSE_EAGAIN;
    Slot &sl = st->ring[st->head];
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady)
        return ASSE_EAGAIN;
    if (q != cudaSuccess)
        return sfail(srv, ASSE_ECUDA, std::string("poll: ") + cudaGetErrorString(q));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, sl.start, sl.done);
    if (latency_ms)
        *latency_ms = ms;
    if (slice)
        *slice = sl.slice;
    const Status stt = *sl.status_host;
    st->last_polled = (int)st->head;
    st->head = (st->head + 1) % ASSE_SERVE_RING;
    st->count--;
    if (stt.error)
        return sfail(srv, ASSE_ETIMEOUT, "a bounded device wait of the scan gave up");
    if (stt.overflow) {
        *n_out = stt.needed;
        return sfail(srv, ASSE_ECAPACITY, "restore capacity exceeded");
    }
    *n_out = stt.n_report;
    uint64_t m = stt.n_report < cap ? stt.n_report : cap;
    m = m < st->rcap ? m : st->rcap;
    if (m > 0) {
        if (!out)
            return sfail(srv, ASSE_EINVAL, "out is NULL");
        memcpy(out, sl.report_host, m * sizeof(asse_superpoint));
    }
    if (stt.n_report > m)
        return sfail(srv, ASSE_ECAPACITY, "report larger than the output or the per-close copy limit");
    return ASSE_OK;
}

int asse_server_sync(asse_server *srv)
{
    if (!srv)
        return ASSE_EINVAL;
    for (SStream *st : srv->streams)
        if (st->open) {
            const cudaError_t e = cudaStreamSynchronize(st->s);
            if (e != cudaSuccess)
                return sfail(srv, ASSE_ECUDA, std::string("sync: ") + cudaGetErrorString(e));
        }
    return ASSE_OK;
}

int asse_server_close(asse_server *srv, uint32_t id)
{
    SStream *st = get(srv, id);
    if (!st)
        return srv ? sfail(srv, ASSE_EINVAL, "no such open stream") : ASSE_EINVAL;
    srv->in_use -= st->bytes;
    release(st);
    return ASSE_OK;
}

int asse_server_attach_model(asse_server *srv, uint32_t id, asse_mlp *mlp, float max_log_n)
{
    SStream *st = get(srv, id);
    if (!st || !mlp || !(max_log_n >= 0.0f))
        return srv ? sfail(srv, ASSE_EINVAL, "no such open stream, NULL model or negative max_log_n") : ASSE_EINVAL;
    if (st->kp > 64)
        return sfail(srv, ASSE_EINVAL, "learned inference needs k' <= 64");
    if (st->mlp)
        return sfail(srv, ASSE_EINVAL, "a model is already attached to this stream");
    if (st->count != 0)
        return sfail(srv, ASSE_EAGAIN, "closes in flight: poll them first");
    asse_pool_info info;
    asse_info(st->pool, &info);
    const uint64_t rows = (uint64_t)st->cfg.r * info.E;
    const uint64_t bytes = rows * ASSE_FEAT * 2 + ASSE_SERVE_RING * (rows * sizeof(float) + sizeof(uint32_t));
    if (srv->in_use + bytes > srv->budget)
        return sfail(srv, ASSE_ENOMEM, "the model's buffers do not fit the device-memory budget now");
    cudaError_t e = cudaStreamSynchronize(st->s);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&st->x, rows * ASSE_FEAT * 2);
    for (Slot &sl : st->ring) {
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&sl.est, rows * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&sl.nfb_dev, sizeof(uint32_t));
        if (e == cudaSuccess)
            e = cudaMallocHost((void **)&sl.nfb_host, sizeof(uint32_t));
    }
    st->mlp = mlp;
    st->max_log_n = max_log_n;
    const PoolBuffers pb = pool_buffers(st->pool);
    int rc = ASSE_OK;
    for (Slot &sl : st->ring) {
        if (e != cudaSuccess || rc != ASSE_OK)
            break;
        if (sl.graph) {
            cudaGraphExecDestroy(sl.graph);
            sl.graph = nullptr;
        }
        e = capture_close(st, sl, pb, &rc);
    }
    if (e == cudaSuccess && rc == ASSE_OK)
        e = cudaStreamSynchronize(st->s);
    if (e != cudaSuccess || rc != ASSE_OK) {
        // the stream is left unusable; close it to return its memory
        const std::string why = e != cudaSuccess ? cudaGetErrorString(e) : asse_last_error(st->pool);
        srv->in_use -= st->bytes;
        release(st);
        return sfail(srv, e == cudaErrorMemoryAllocation ? ASSE_ENOMEM : ASSE_ECUDA,
                     "attach (the stream was closed): " + why);
    }
    st->model_bytes = bytes;
    st->bytes += bytes;
    srv->in_use += bytes;
    return ASSE_OK;
}

int asse_server_estimates(asse_server *srv, uint32_t id, float *out, uint64_t cap, int where, uint32_t *n_fallback)
{
    SStream *st = get(srv, id);
    if (!st || !out)
        return srv ? sfail(srv, ASSE_EINVAL, "no such open stream or NULL argument") : ASSE_EINVAL;
    if (!st->mlp || st->last_polled < 0)
        return sfail(srv, ASSE_ESTATE, "no model attached or no close polled yet");
    asse_pool_info info;
    asse_info(st->pool, &info);
    const uint64_t rows = (uint64_t)st->cfg.r * info.E;
    if (cap < rows)
        return sfail(srv, ASSE_ECAPACITY, "out holds fewer than r * E estimates");
    const Slot &sl = st->ring[st->last_polled];
    cudaError_t e = cudaMemcpyAsync(out, sl.est, rows * sizeof(float),
                                    where == ASSE_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st->s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st->s);
    if (e != cudaSuccess)
        return sfail(srv, ASSE_ECUDA, std::string("estimates: ") + cudaGetErrorString(e));
    if (n_fallback)
        *n_fallback = *sl.nfb_host;
    return ASSE_OK;
}

asse_pool *asse_server_pool(asse_server *srv, uint32_t id)
{
    SStream *st = get(srv, id);
    return st ? st->pool : nullptr;
}

const char *asse_server_last_error(const asse_server *srv) { return srv ? srv->err.c_str() : ""; }

}  // extern "C"
