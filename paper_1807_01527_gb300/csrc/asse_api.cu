// Host side of the ASSE C ABI (include/asse.h): parameter validation, device
// state, the slice lifecycle and the copies across the process/device
// boundary.  All device work goes through the kernel launchers declared in
// asse_internal.h (asse_ingest.cu, asse_scan.cu, asse_restore.cu, asse_probe.cu).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "asse_internal.h"
#include "asse_pool_access.h"

using namespace asse;

namespace {

thread_local std::string g_create_error;

struct SnapHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    asse_config cfg;
    uint64_t slice;
    uint64_t pool_words;
    uint32_t w, words;
};

}  // namespace

struct asse_pool {
    asse_config cfg{};
    Params P{};
    uint32_t w = 0, F = 0, words_used = 0, blk = 0;
    uint64_t t = 0;
    cudaStream_t stream = nullptr, copy_stream = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
    int sms = 0;
    uint32_t *pool = nullptr;
    uint64_t pool_words = 0;
    uint16_t *cnt = nullptr;
    unsigned long long *aat = nullptr;
    uint32_t *sa_n = nullptr, *sa_x = nullptr, *sa_mask = nullptr;
    Tuple *scratch = nullptr;
    uint32_t cap = 0;
    asse_superpoint *csip = nullptr, *report = nullptr;
    uint64_t out_cap = 0;
    Status *status = nullptr;
    Status *status_host = nullptr;
    // asse_close_slice also copies the status and the head of the report to
    // pinned host memory, so that reading a short report takes one wait
    asse_superpoint *report_host = nullptr;
    uint64_t report_host_cap = 0;
    int report_host_valid = 0;
    cudaEvent_t close_done = nullptr;  // recorded after those copies: a report waits for its close only
    // the copies of a close's status and report to pinned memory run on their
    // own stream, after `closed`, so the next batch's ingest does not wait
    // for them; the next close waits for close_done before it rewrites them
    cudaStream_t d2h_stream = nullptr;
    cudaEvent_t closed = nullptr;
    // asse_set_timing: events around the scan and the restore of each close
    cudaEvent_t tev[3] = {nullptr, nullptr, nullptr};
    int timing = 0, timed = 0;
    SliceCtl *ctl = nullptr;  // device copy of the slice-dependent launch arguments
    uint32_t *stage[2] = {nullptr, nullptr};
    uint64_t stage_pairs = 0;
    uint32_t *q_aips = nullptr;
    asse_superpoint *q_out = nullptr;
    uint64_t q_cap = 0;
    // outputs of windows 1 .. MAX_WINDOWS-1 of a multi-window close (window 0
    // uses the buffers above), allocated on first use
    struct Win {
        uint16_t *cnt = nullptr;
        unsigned long long *aat = nullptr;
        uint32_t *sa_n = nullptr, *sa_x = nullptr, *sa_mask = nullptr;
        Status *status = nullptr;
        asse_superpoint *csip = nullptr, *report = nullptr;
    } win[MAX_WINDOWS - 1];
    uint32_t n_windows = 1, sel = 0;  // windows of the last close, the one the readers return
    int scanned = 0, refreshed = 0, restored = 0, ingested = 0;
    uint32_t scan_kp = 0;
    uint64_t scan_slice = 0;
    uint64_t launches = 0;
    std::string err;
};

namespace {

int fail(asse_pool *p, int code, const std::string &msg)
{
    if (p)
        p->err = msg;
    else
        g_create_error = msg;
    return code;
}

int cuda_fail(asse_pool *p, cudaError_t e, const char *what)
{
    return fail(p, ASSE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(p, call)                                   \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess)                        \
            return cuda_fail((p), e_, #call);         \
    } while (0)

uint64_t inverse_mod(uint64_t a, uint64_t m)
{
    __int128 t0 = 0, t1 = 1, r0 = (__int128)m, r1 = (__int128)a;
    while (r1 != 0) {
        __int128 q = r0 / r1, tmp;
        tmp = r0 - q * r1; r0 = r1; r1 = tmp;
        tmp = t0 - q * t1; t0 = t1; t1 = tmp;
    }
    if (t0 < 0)
        t0 += (__int128)m;
    return (uint64_t)t0;
}

int validate(const asse_config *c, std::string &why)
{
    char buf[256];
    auto bad = [&](const char *m) { why = m; return ASSE_EINVAL; };
    if (!c)
        return bad("cfg is NULL");
    if (c->counter != ASSE_COUNTER_AT && c->counter != ASSE_COUNTER_ACE && c->counter != ASSE_COUNTER_AT_ALIGNED &&
        c->counter != ASSE_COUNTER_AT_HIST)
        return bad("counter must be ASSE_COUNTER_AT, ASSE_COUNTER_ACE, ASSE_COUNTER_AT_ALIGNED or ASSE_COUNTER_AT_HIST");
    if (c->k < 1 || c->k > 127)
        return bad("k must be in [1, 127]");
    if (c->g < 2 * c->k || c->g > 4096)
        return bad("g must be in [2k, 4096]");
    if (c->r < 2 || c->r > 8)
        return bad("r must be in [2, 8]");
    if (c->c < 1 || c->c > 16 || c->u > 8 || c->c + c->u > 24)
        return bad("need 1 <= c <= 16, u <= 8, c + u <= 24");
    const uint32_t W = 32 - c->u;
    if (c->c > W || c->s < 1 || c->s > c->c || c->s * (c->r - 1) >= W) {
        snprintf(buf, sizeof buf, "need c <= 32-u, 1 <= s <= c and s*(r-1) < 32-u (c=%u s=%u r=%u u=%u)", c->c, c->s,
                 c->r, c->u);
        why = buf;
        return ASSE_EINVAL;
    }
    if (c->c + c->s * (c->r - 1) < W)
        return bad("column windows do not cover LBS: need c + s*(r-1) >= 32-u (completeness, Sec. 4.1)");
    if (c->A < 2)
        return bad("A must be in [2, 2^32)");
    if ((c->bh_a & 1) == 0)
        return bad("bh_a must be odd");
    if (c->theta < 1)
        return bad("theta must be >= 1");
    if (c->key_table > ASSE_KEYS_OFF)
        return bad("key_table must be ASSE_KEYS_AUTO, ASSE_KEYS_ON or ASSE_KEYS_OFF");
    if (c->cluster != ASSE_CLUSTER_AUTO && c->cluster != 1 && c->cluster != 2 && c->cluster != 4 && c->cluster != 8)
        return bad("cluster must be ASSE_CLUSTER_AUTO, 1, 2, 4 or 8");
    // the scan holds one ATV in a warp tile of at most 512 words
    const uint32_t w = packed_width(c->counter, c->k);
    if ((c->g + 32 / w - 1) / (32 / w) > 512)
        return bad("an ATV must fit in 512 words: need g <= 512 * floor(32 / w)");
    return ASSE_OK;
}

ScanOut scan_out(asse_pool *p)
{
    ScanOut o;
    o.cnt = p->cnt;
    o.aat = p->aat;
    o.sa_n = p->sa_n;
    o.sa_x = p->sa_x;
    o.sa_mask = p->sa_mask;
    o.status = p->status;
    return o;
}

// Scan outputs, status and lists of window m of the last close.
ScanOut scan_out_w(asse_pool *p, uint32_t m)
{
    if (m == 0)
        return scan_out(p);
    const asse_pool::Win &w = p->win[m - 1];
    ScanOut o;
    o.cnt = w.cnt;
    o.aat = w.aat;
    o.sa_n = w.sa_n;
    o.sa_x = w.sa_x;
    o.sa_mask = w.sa_mask;
    o.status = w.status;
    return o;
}

asse_superpoint *list_w(asse_pool *p, uint32_t m, bool reported)
{
    if (m == 0)
        return reported ? p->report : p->csip;
    return reported ? p->win[m - 1].report : p->win[m - 1].csip;
}

__global__ void init_pool_kernel(uint32_t *pool, uint64_t nwords, uint32_t Wd, uint32_t words_used,
                                 uint32_t full_word, uint32_t last_word)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += stride) {
        const uint32_t q = (uint32_t)(i % Wd);
        pool[i] = q + 1 < words_used ? full_word : (q + 1 == words_used ? last_word : 0u);
    }
}

// Work of the pool's stream that rewrites the status or the report waits
// until the last close's copies of them (on d2h_stream) have read them.  Not
// for captured graphs (their closes copy on their own stream in order).
int wait_close_copies(asse_pool *p)
{
    CK(p, cudaStreamWaitEvent(p->stream, p->close_done, 0));
    return ASSE_OK;
}

int reset_close_state(asse_pool *p)
{
    CK(p, launch_reset(p->aat, p->sa_n, p->cfg.r * p->P.nf, p->status, p->stream, &p->launches));
    return ASSE_OK;
}

int check_kp(asse_pool *p, uint32_t kp)
{
    if (kp < 1 || kp > p->cfg.k)
        return fail(p, ASSE_EINVAL, "kp must be in [1, k]");
    return ASSE_OK;
}

int read_list(asse_pool *p, bool reported, asse_superpoint *out, uint64_t cap, uint64_t *n_out, int where)
{
    if (!p || !n_out)
        return fail(p, ASSE_EINVAL, "NULL argument");
    if (!p->restored)
        return fail(p, ASSE_ESTATE, "no restore since the last scan");
    const bool early = reported && where != ASSE_DEVICE && p->report_host_valid && p->sel == 0;
    if (!early) {
        CK(p, cudaEventSynchronize(p->close_done));  // no close's copy is still writing status_host
        CK(p, cudaMemcpyAsync(p->status_host, scan_out_w(p, p->sel).status, sizeof(Status), cudaMemcpyDeviceToHost,
                              p->stream));
        CK(p, cudaStreamSynchronize(p->stream));
    } else {
        // the close and its copies to pinned memory are done; later work
        // already queued on the stream (the next batch) keeps running
        CK(p, cudaEventSynchronize(p->close_done));
    }
    const Status st = *p->status_host;
    if (st.error)
        return fail(p, ASSE_ETIMEOUT, "a bounded device wait of the scan gave up (bulk copy did not complete)");
    if (st.overflow) {
        *n_out = st.needed;
        char buf[200];
        snprintf(buf, sizeof buf, "restore needed %llu column tuples in one frame, restore_cap is %u",
                 (unsigned long long)st.needed, p->cap);
        return fail(p, ASSE_ECAPACITY, buf);
    }
    const uint64_t n = reported ? st.n_report : st.n_csip;
    *n_out = n;
    const uint64_t m = n < cap ? n : cap;
    if (m > 0 && early && m <= p->report_host_cap) {
        if (!out)
            return fail(p, ASSE_EINVAL, "out is NULL");
        memcpy(out, p->report_host, m * sizeof(asse_superpoint));
    } else if (m > 0) {
        if (!out)
            return fail(p, ASSE_EINVAL, "out is NULL");
        CK(p, cudaMemcpyAsync(out, list_w(p, p->sel, reported), m * sizeof(asse_superpoint),
                              where == ASSE_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
        if (where != ASSE_DEVICE)
            CK(p, cudaStreamSynchronize(p->stream));
    }
    if (n > cap)
        return fail(p, ASSE_ECAPACITY, "output capacity smaller than the list");
    return ASSE_OK;
}

void free_all(asse_pool *p)
{
    cudaFree(p->pool);
    cudaFree(p->cnt);
    cudaFree(p->aat);
    cudaFree(p->sa_n);
    cudaFree(p->sa_x);
    cudaFree(p->sa_mask);
    cudaFree(p->scratch);
    cudaFree(p->csip);
    cudaFree(p->report);
    cudaFree(p->status);
    cudaFree(p->ctl);
    cudaFree(p->P.keys);
    cudaFree(p->P.hist);
    cudaFree(p->P.hsum);
    cudaFree(p->stage[0]);
    cudaFree(p->stage[1]);
    cudaFree(p->q_aips);
    cudaFree(p->q_out);
    for (auto &w : p->win)
        for (void *ptr : {(void *)w.cnt, (void *)w.aat, (void *)w.sa_n, (void *)w.sa_x, (void *)w.sa_mask,
                          (void *)w.status, (void *)w.csip, (void *)w.report})
            cudaFree(ptr);
    if (p->status_host)
        cudaFreeHost(p->status_host);
    if (p->report_host)
        cudaFreeHost(p->report_host);
    if (p->close_done)
        cudaEventDestroy(p->close_done);
    if (p->closed)
        cudaEventDestroy(p->closed);
    if (p->d2h_stream)
        cudaStreamDestroy(p->d2h_stream);
    for (cudaEvent_t ev : p->tev)
        if (ev)
            cudaEventDestroy(ev);
    for (int i = 0; i < 2; i++) {
        if (p->copied[i])
            cudaEventDestroy(p->copied[i]);
        if (p->consumed[i])
            cudaEventDestroy(p->consumed[i]);
    }
    if (p->copy_stream)
        cudaStreamDestroy(p->copy_stream);
}

}  // namespace

namespace asse {

int pool_restore_view(asse_pool *p, RestoreView *v)
{
    if (!p->scanned)
        return fail(p, ASSE_ESTATE, "restore needs a scan of the open slice");
    p->report_host_valid = 0;
    v->P = p->P;
    v->o = scan_out_w(p, p->sel);
    v->stream = p->stream;
    v->launches = &p->launches;
    return ASSE_OK;
}

int pool_fail(asse_pool *p, int code, const std::string &msg) { return fail(p, code, msg); }

int pool_enqueue_close(asse_pool *p, uint32_t kp, bool timed)
{
    if (int rc = reset_close_state(p))
        return rc;
    if (timed)
        CK(p, cudaEventRecord(p->tev[0], p->stream));
    // counts from the slice counts, or from every AT; either way with the
    // refresh for the next slice fused in
    if (p->P.hist)
        CK(p, launch_hist_scan(p->P, p->w, p->pool, kp, true, p->ctl, scan_out(p), p->sms, p->stream, &p->launches));
    else
        CK(p, launch_scan(p->P, p->w, p->pool, kp, true, p->ctl, scan_out(p), p->sms, p->stream, &p->launches));
    if (timed)
        CK(p, cudaEventRecord(p->tev[1], p->stream));
    CK(p, launch_restore(p->P, scan_out(p), p->scratch, p->cap, p->csip, p->report, p->out_cap, p->stream,
                         &p->launches, p->ctl));
    if (timed)
        CK(p, cudaEventRecord(p->tev[2], p->stream));
    return ASSE_OK;
}

int pool_enqueue_scan(asse_pool *p, uint32_t kp)
{
    if (int rc = reset_close_state(p))
        return rc;
    if (p->P.hist)
        CK(p, launch_hist_scan(p->P, p->w, p->pool, kp, false, p->ctl, scan_out(p), p->sms, p->stream,
                               &p->launches));
    else
        CK(p, launch_scan(p->P, p->w, p->pool, kp, false, p->ctl, scan_out(p), p->sms, p->stream, &p->launches));
    return ASSE_OK;
}

int pool_enqueue_restore_refresh(asse_pool *p)
{
    CK(p, launch_restore(p->P, scan_out(p), p->scratch, p->cap, p->csip, p->report, p->out_cap, p->stream,
                         &p->launches));
    CK(p, launch_refresh(p->P, p->w, p->pool, p->ctl, p->sms, p->stream, &p->launches));
    CK(p, launch_advance_ctl(p->P, p->ctl, p->stream, &p->launches));
    return ASSE_OK;
}

FeatureView pool_feature_view_device(asse_pool *p, uint32_t kp)
{
    FeatureView v{};
    v.P = p->P;
    v.w = p->w;
    v.pool = p->pool;
    v.c0 = 0;
    v.kp = kp;
    v.ctl = p->ctl;
    v.aat = p->aat;
    v.cnt = p->cnt;
    v.stream = p->stream;
    v.launches = &p->launches;
    v.sms = p->sms;
    return v;
}

void pool_after_close(asse_pool *p, uint32_t kp)
{
    p->report_host_valid = 0;
    p->n_windows = 1;
    p->sel = 0;
    p->report_host_valid = 0;
    p->scanned = 1;
    p->restored = 1;
    p->refreshed = 1;
    p->ingested = 0;
    p->scan_kp = kp;
    p->scan_slice = p->t;
    p->t += 1;
}

int pool_enqueue_ingest(asse_pool *p, const uint32_t *pairs_dev, const unsigned long long *n_dev)
{
    CK(p, launch_ingest(p->P, p->w, p->pool, pairs_dev, 0, n_dev, p->ctl, p->sms, p->stream, &p->launches));
    p->ingested = 1;
    return ASSE_OK;
}

PoolBuffers pool_buffers(asse_pool *p)
{
    PoolBuffers b;
    b.status = p->status;
    b.report = p->report;
    b.out_cap = p->out_cap;
    b.stream = p->stream;
    b.cap = p->cap;
    return b;
}

// Device bytes asse_create allocates for cfg (the server's admission unit).
uint64_t pool_device_bytes(const asse_config *cfg)
{
    const uint32_t w = packed_width(cfg->counter, cfg->k);
    const uint32_t F = 32 / w;
    const uint64_t Wd = ((cfg->g + F - 1) / F + 7) / 8 * 8;
    const uint64_t n_atv = (uint64_t)cfg->r << (cfg->c + cfg->u);
    const uint64_t nf = 1ull << cfg->u, nseg = cfg->r * nf, mw = (cfg->g + 31) / 32;
    const uint64_t cap = cfg->restore_cap ? cfg->restore_cap : 4096;
    const uint64_t stage = cfg->max_batch ? (cfg->max_batch + 1) / 2 * 2 : (4ull << 20);
    // the key table of asse_create, on the current device
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
        cudaGetLastError();
    const uint32_t klg = key_table_log2(n_atv, n_atv * Wd * 4, (unsigned long long)l2, cfg->key_table);
    const uint64_t hist = cfg->counter == ASSE_COUNTER_AT_HIST ? ((uint64_t)2 * cfg->k + 1) * n_atv * 2 : 0;
    return hist + n_atv * Wd * 4 + n_atv * 2 + nseg * (8 + 4) + n_atv * 4 + n_atv * mw * 4 + nf * 2 * cap * sizeof(Tuple) +
           2 * cap * nf * sizeof(asse_superpoint) + sizeof(Status) + sizeof(SliceCtl) + 2 * stage * 8 +
           (klg ? sizeof(unsigned long long) << klg : 0);
}

uint64_t pool_list_cap(const asse_pool *p) { return p ? p->out_cap : 0; }

int pool_feature_view(asse_pool *p, FeatureView *v)
{
    if (!p->scanned || p->refreshed || p->ingested || p->scan_slice != p->t)
        return fail(p, ASSE_ESTATE, "features need a scan of the open slice and no refresh or ingest since");
    v->P = p->P;
    v->w = p->w;
    v->pool = p->pool;
    v->c0 = (uint32_t)(p->t % (2 * p->cfg.k));
    v->kp = p->scan_kp;
    v->ctl = nullptr;
    v->aat = p->aat;
    v->cnt = p->cnt;
    v->stream = p->stream;
    v->launches = &p->launches;
    v->sms = p->sms;
    return ASSE_OK;
}

}  // namespace asse

extern "C" {

const char *asse_strerror(int status)
{
    switch (status) {
    case ASSE_OK: return "ASSE_OK";
    case ASSE_EINVAL: return "ASSE_EINVAL";
    case ASSE_ENOMEM: return "ASSE_ENOMEM";
    case ASSE_ECAPACITY: return "ASSE_ECAPACITY";
    case ASSE_ECUDA: return "ASSE_ECUDA";
    case ASSE_ESTATE: return "ASSE_ESTATE";
    case 6: return "ASSE_EAGAIN";
    case ASSE_ETIMEOUT: return "ASSE_ETIMEOUT";
    default: return "unknown status";
    }
}

const char *asse_last_error(const asse_pool *pool)
{
    return pool ? pool->err.c_str() : g_create_error.c_str();
}

uint64_t asse_launches(const asse_pool *pool) { return pool ? pool->launches : 0; }

int asse_create(const asse_config *cfg, void *stream, asse_pool **out)
{
    if (!out)
        return fail(nullptr, ASSE_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why;
    if (validate(cfg, why) != ASSE_OK)
        return fail(nullptr, ASSE_EINVAL, why);
    asse_pool *p = new (std::nothrow) asse_pool();
    if (!p)
        return fail(nullptr, ASSE_ENOMEM, "host allocation failed");
    p->cfg = *cfg;
    p->stream = (cudaStream_t)stream;
    const uint32_t k = cfg->k;
    const bool ace = cfg->counter == ASSE_COUNTER_ACE;
    p->w = packed_width(cfg->counter, k);
    p->F = 32 / p->w;
    p->words_used = (cfg->g + p->F - 1) / p->F;
    const uint32_t Wd = (p->words_used + 7) / 8 * 8;
    // the aligned variant is one block of g ATs (every AT has ACT C0)
    p->blk = cfg->counter == ASSE_COUNTER_AT_ALIGNED ? cfg->g : cfg->g / (2 * k);
    Params &P = p->P;
    P.k = k;
    P.k2 = 2 * k;
    P.g = cfg->g;
    P.r = cfg->r;
    P.c = cfg->c;
    P.u = cfg->u;
    P.W = 32 - cfg->u;
    P.E_log2 = cfg->c + cfg->u;
    P.Wd = Wd;
    P.A = cfg->A;
    P.cmask = (1u << cfg->c) - 1;
    P.theta = cfg->theta;
    const double g = (double)cfg->g;
    P.T = (uint32_t)std::ceil(g - g * std::exp(-(double)cfg->theta / g));
    P.ace = ace ? 1 : 0;
    P.nf = 1u << cfg->u;
    P.mw = (cfg->g + 31) / 32;
    P.blk = p->blk;
    P.F = p->F;
    P.blk_magic = ((1ull << 32) + p->blk - 1) / p->blk;
    // timestamps with 2k blocks keep each pair of blocks that one refresh
    // checks side by side (block_slot)
    P.paired = (cfg->counter == ASSE_COUNTER_AT || cfg->counter == ASSE_COUNTER_AT_HIST) ? 1 : 0;
    P.Ainv = inverse_mod(cfg->A, 4294967311ull);
    P.bh_a = cfg->bh_a;
    P.bh_b = cfg->bh_b;
    P.cl = cfg->cluster == ASSE_CLUSTER_AUTO ? 1u : cfg->cluster;
    for (uint32_t i = 0; i < 8; i++)
        P.xshift[i] = i < cfg->r ? 2 * P.W - cfg->c - cfg->s * i : 0;
    p->cap = cfg->restore_cap ? cfg->restore_cap : 4096;
    p->out_cap = (uint64_t)p->cap * P.nf;
    p->stage_pairs = cfg->max_batch ? (cfg->max_batch + 1) / 2 * 2 : (4ull << 20);

    const uint64_t n_atv = (uint64_t)cfg->r << P.E_log2;
    p->pool_words = n_atv * Wd;
    const size_t nseg = (size_t)cfg->r * P.nf;
    const size_t slots = (size_t)cfg->r << P.E_log2;  // super-ATV slots: every ATV of a row-frame
    cudaError_t e = cudaSuccess;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
        delete p;
        return cuda_fail(nullptr, e, "cudaGetDevice/cudaDeviceGetAttribute");
    }
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess)
            e = cudaMalloc(ptr, bytes);
    };
    alloc((void **)&p->pool, p->pool_words * 4);
    alloc((void **)&p->cnt, n_atv * sizeof(uint16_t));
    alloc((void **)&p->aat, nseg * sizeof(unsigned long long));
    alloc((void **)&p->sa_n, nseg * sizeof(uint32_t));
    alloc((void **)&p->sa_x, slots * sizeof(uint32_t));
    alloc((void **)&p->sa_mask, slots * P.mw * sizeof(uint32_t));
    alloc((void **)&p->scratch, (size_t)P.nf * 2 * p->cap * sizeof(Tuple));
    alloc((void **)&p->csip, p->out_cap * sizeof(asse_superpoint));
    alloc((void **)&p->report, p->out_cap * sizeof(asse_superpoint));
    alloc((void **)&p->status, sizeof(Status));
    alloc((void **)&p->ctl, sizeof(SliceCtl));
    int l2 = 0;
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    P.klg = key_table_log2(n_atv, p->pool_words * 4, (unsigned long long)l2, cfg->key_table);
    if (P.klg)
        alloc((void **)&P.keys, sizeof(unsigned long long) << P.klg);
    if (cfg->counter == ASSE_COUNTER_AT_HIST) {
        alloc((void **)&P.hist, (size_t)2 * k * n_atv * sizeof(uint16_t));
        alloc((void **)&P.hsum, (size_t)n_atv * sizeof(uint16_t));
    }
    alloc((void **)&p->stage[0], p->stage_pairs * 8);
    alloc((void **)&p->stage[1], p->stage_pairs * 8);
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&p->status_host, sizeof(Status));
    p->report_host_cap = p->out_cap < 4096 ? p->out_cap : 4096;
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&p->report_host, p->report_host_cap * sizeof(asse_superpoint));
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&p->close_done, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&p->d2h_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&p->closed, cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; i++) {
        e = cudaEventCreateWithFlags(&p->copied[i], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&p->consumed[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        free_all(p);
        delete p;
        return oom ? fail(nullptr, ASSE_ENOMEM, "device allocation failed")
                   : cuda_fail(nullptr, e, "asse_create");
    }
    // InitAT: every field of every ATV at its inactive value (2k, or 0 for
    // aging counters); fields past g and padding words hold 0.
    const uint32_t fill = ace ? 0u : 2 * k;
    uint32_t full_word = 0, last_word = 0;
    for (uint32_t j = 0; j < p->F; j++) {
        full_word |= fill << (j * p->w);
        if ((p->words_used - 1) * p->F + j < cfg->g)
            last_word |= fill << (j * p->w);
    }
    init_pool_kernel<<<p->sms * 4, 256, 0, p->stream>>>(p->pool, p->pool_words, Wd, p->words_used, full_word,
                                                          last_word);
    p->launches++;
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemsetAsync(p->status, 0, sizeof(Status), p->stream);
    if (e == cudaSuccess && P.keys)
        e = cudaMemsetAsync(P.keys, 0xff, sizeof(unsigned long long) << P.klg, p->stream);
    if (e == cudaSuccess && P.hist)
        e = cudaMemsetAsync(P.hist, 0, (size_t)2 * k * n_atv * sizeof(uint16_t), p->stream);
    if (e == cudaSuccess && P.hsum)
        e = cudaMemsetAsync(P.hsum, 0, (size_t)n_atv * sizeof(uint16_t), p->stream);
    const SliceCtl ctl0 = slice_ctl(P, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->ctl, &ctl0, sizeof ctl0, cudaMemcpyHostToDevice, p->stream);

    if (e == cudaSuccess)
        e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        free_all(p);
        delete p;
        return cuda_fail(nullptr, e, "pool initialisation");
    }
    *out = p;
    return ASSE_OK;
}

void asse_destroy(asse_pool *pool)
{
    if (!pool)
        return;
    cudaStreamSynchronize(pool->stream);
    cudaStreamSynchronize(pool->copy_stream);
    cudaStreamSynchronize(pool->d2h_stream);
    free_all(pool);
    delete pool;
}

int asse_set_stream(asse_pool *pool, void *stream)
{
    if (!pool)
        return ASSE_EINVAL;
    pool->stream = (cudaStream_t)stream;
    return ASSE_OK;
}

int asse_ingest(asse_pool *p, const uint32_t *pairs, uint64_t n, int where)
{
    if (!p)
        return fail(nullptr, ASSE_EINVAL, "pool is NULL");
    if (n == 0)
        return ASSE_OK;
    if (!pairs)
        return fail(p, ASSE_EINVAL, "pairs is NULL");
    p->ingested = 1;  // the pool no longer matches the last scan
    if (where == ASSE_DEVICE) {
        if (((uintptr_t)pairs & 15) != 0)
            return fail(p, ASSE_EINVAL, "device pairs must be 16-byte aligned");
        CK(p, launch_ingest(p->P, p->w, p->pool, pairs, n, nullptr, p->ctl, p->sms, p->stream, &p->launches));
        return ASSE_OK;
    }
    if (where != ASSE_HOST)
        return fail(p, ASSE_EINVAL, "where must be ASSE_HOST or ASSE_DEVICE");
    // Double-buffered staging (Sec. 4.4): the copy engines move chunk i+1 on
    // the copy stream while chunk i is ingested on the pool's stream, and the
    // call returns once the last chunk is copied, so the ingest and the close
    // of this slice overlap the caller's next transfer.  (The kernel could
    // read pinned memory in place over the host link, but that keeps the SMs
    // busy for the whole transfer: 19.3 against 23.1 G pairs/s end to end on
    // the link workload with the next batch queued before each report.)
    int last = -1;
    for (uint64_t off = 0, i = 0; off < n; off += p->stage_pairs, i++) {
        const int b = (int)(i & 1);
        const uint64_t m = (n - off) < p->stage_pairs ? (n - off) : p->stage_pairs;
        CK(p, cudaStreamWaitEvent(p->copy_stream, p->consumed[b], 0));
        CK(p, cudaMemcpyAsync(p->stage[b], pairs + 2 * off, m * 8, cudaMemcpyHostToDevice, p->copy_stream));
        CK(p, cudaEventRecord(p->copied[b], p->copy_stream));
        CK(p, cudaStreamWaitEvent(p->stream, p->copied[b], 0));
        CK(p, launch_ingest(p->P, p->w, p->pool, p->stage[b], m, nullptr, p->ctl, p->sms, p->stream,
                            &p->launches));
        CK(p, cudaEventRecord(p->consumed[b], p->stream));
        last = b;
    }
    // the caller may reuse its host buffer once every chunk has been copied
    if (last >= 0)
        CK(p, cudaEventSynchronize(p->copied[last]));
    return ASSE_OK;
}

int asse_scan(asse_pool *p, uint32_t kp)
{
    if (!p)
        return fail(nullptr, ASSE_EINVAL, "pool is NULL");
    if (int rc = check_kp(p, kp))
        return rc;
    if (int rc = wait_close_copies(p))
        return rc;
    if (int rc = pool_enqueue_scan(p, kp))
        return rc;
    p->n_windows = 1;
    p->sel = 0;
    p->report_host_valid = 0;
    p->scanned = 1;
    p->refreshed = 0;
    p->restored = 0;
    p->ingested = 0;
    p->scan_kp = kp;
    p->scan_slice = p->t;
    return ASSE_OK;
}

int asse_restore(asse_pool *p)
{
    if (!p)
        return fail(nullptr, ASSE_EINVAL, "pool is NULL");
    if (!p->scanned)
        return fail(p, ASSE_ESTATE, "restore needs a scan of the open slice");
    p->report_host_valid = 0;
    if (int rc = wait_close_copies(p))
        return rc;
    CK(p, launch_restore(p->P, scan_out(p), p->scratch, p->cap, p->csip, p->report, p->out_cap, p->stream,
                         &p->launches));
    p->restored = 1;
    return ASSE_OK;
}

int asse_advance(asse_pool *p)
{
    if (!p)
        return fail(nullptr, ASSE_EINVAL, "pool is NULL");
    CK(p, launch_refresh(p->P, p->w, p->pool, p->ctl, p->sms, p->stream, &p->launches));
    CK(p, launch_advance_ctl(p->P, p->ctl, p->stream, &p->launches));
    p->t += 1;
    p->refreshed = 1;
    return ASSE_OK;
}

int asse_close_slice(asse_pool *p, uint32_t kp)
{
    if (!p)
        return fail(nullptr, ASSE_EINVAL, "pool is NULL");
    if (int rc = check_kp(p, kp))
        return rc;
    if (int rc = wait_close_copies(p))
        return rc;
    if (int rc = pool_enqueue_close(p, kp, p->timing != 0))
        return rc;
    pool_after_close(p, kp);
    p->timed = p->timing;
    CK(p, cudaEventRecord(p->closed, p->stream));
    CK(p, cudaStreamWaitEvent(p->d2h_stream, p->closed, 0));
    CK(p, cudaMemcpyAsync(p->status_host, p->status, sizeof(Status), cudaMemcpyDeviceToHost, p->d2h_stream));
    CK(p, cudaMemcpyAsync(p->report_host, p->report, p->report_host_cap * sizeof(asse_superpoint),
                          cudaMemcpyDeviceToHost, p->d2h_stream));
    CK(p, cudaEventRecord(p->close_done, p->d2h_stream));
    p->report_host_valid = 1;
    return ASSE_OK;
}

int asse_close_slice_multi(asse_pool *p, const uint32_t *kps, uint32_t n_windows)
{
    if (!p)
        return fail(nullptr, ASSE_EINVAL, "pool is NULL");
    if (!kps || n_windows < 1 || n_windows > (uint32_t)MAX_WINDOWS)
        return fail(p, ASSE_EINVAL, "need kps and 1 <= n_windows <= ASSE_MAX_WINDOWS");
    for (uint32_t m = 0; m < n_windows; m++)
        if (int rc = check_kp(p, kps[m]))
            return rc;
    // outputs of the extra windows, on first use
    const uint64_t n_atv = (uint64_t)p->cfg.r << p->P.E_log2;
    const size_t nseg = (size_t)p->cfg.r * p->P.nf;
    for (uint32_t m = 1; m < n_windows; m++) {
        asse_pool::Win &w = p->win[m - 1];
        if (w.cnt)
            continue;
        cudaError_t e = cudaSuccess;
        auto alloc = [&](void **ptr, size_t bytes) {
            if (e == cudaSuccess)
                e = cudaMalloc(ptr, bytes);
        };
        alloc((void **)&w.cnt, n_atv * sizeof(uint16_t));
        alloc((void **)&w.aat, nseg * sizeof(unsigned long long));
        alloc((void **)&w.sa_n, nseg * sizeof(uint32_t));
        alloc((void **)&w.sa_x, n_atv * sizeof(uint32_t));
        alloc((void **)&w.sa_mask, n_atv * p->P.mw * sizeof(uint32_t));
        alloc((void **)&w.status, sizeof(Status));
        alloc((void **)&w.csip, p->out_cap * sizeof(asse_superpoint));
        alloc((void **)&w.report, p->out_cap * sizeof(asse_superpoint));
        if (e != cudaSuccess) {
            cudaGetLastError();
            for (void *ptr : {(void *)w.cnt, (void *)w.aat, (void *)w.sa_n, (void *)w.sa_x, (void *)w.sa_mask,
                              (void *)w.status, (void *)w.csip, (void *)w.report})
                cudaFree(ptr);
            w = asse_pool::Win();
            return e == cudaErrorMemoryAllocation ? fail(p, ASSE_ENOMEM, "window outputs: device allocation failed")
                                                  : cuda_fail(p, e, "window outputs");
        }
    }
    if (int rc = wait_close_copies(p))
        return rc;
    ScanWindows W{};
    W.n = n_windows;
    for (uint32_t m = 0; m < n_windows; m++) {
        W.kp[m] = kps[m];
        W.o[m] = scan_out_w(p, m);
        CK(p, launch_reset(W.o[m].aat, W.o[m].sa_n, p->cfg.r * p->P.nf, W.o[m].status, p->stream, &p->launches));
    }
    if (p->P.hist) {
        // one count pass per window over the slice counts, then the restores,
        // the refresh (with the zeroing of the next slice's counts) and the next slice
        for (uint32_t m = 0; m < n_windows; m++)
            CK(p, launch_hist_scan(p->P, p->w, p->pool, kps[m], false, p->ctl, W.o[m], p->sms, p->stream,
                                   &p->launches));
        for (uint32_t m = 0; m < n_windows; m++)
            CK(p, launch_restore(p->P, W.o[m], p->scratch, p->cap, list_w(p, m, false), list_w(p, m, true),
                                 p->out_cap, p->stream, &p->launches));
        CK(p, launch_refresh(p->P, p->w, p->pool, p->ctl, p->sms, p->stream, &p->launches));
        CK(p, launch_advance_ctl(p->P, p->ctl, p->stream, &p->launches));
    } else {
        CK(p, launch_scan_windows(p->P, p->w, p->pool, W, p->ctl, p->sms, p->stream, &p->launches));
        for (uint32_t m = 0; m < n_windows; m++)
            CK(p, launch_restore(p->P, W.o[m], p->scratch, p->cap, list_w(p, m, false), list_w(p, m, true),
                                 p->out_cap, p->stream, &p->launches, m + 1 == n_windows ? p->ctl : nullptr));
    }
    pool_after_close(p, kps[0]);
    p->n_windows = n_windows;
    return ASSE_OK;
}

int asse_set_timing(asse_pool *p, int on)
{
    if (!p)
        return fail(nullptr, ASSE_EINVAL, "pool is NULL");
    for (int i = 0; i < 3 && on; i++)
        if (!p->tev[i])
            CK(p, cudaEventCreate(&p->tev[i]));
    p->timing = on ? 1 : 0;
    p->timed = 0;
    return ASSE_OK;
}

int asse_close_timing(asse_pool *p, float *ms)
{
    if (!p || !ms)
        return fail(p, ASSE_EINVAL, "pool and ms must not be NULL");
    if (!p->timed)
        return fail(p, ASSE_ESTATE, "no close since asse_set_timing(pool, 1)");
    CK(p, cudaEventSynchronize(p->tev[2]));
    CK(p, cudaEventElapsedTime(&ms[0], p->tev[0], p->tev[1]));
    CK(p, cudaEventElapsedTime(&ms[1], p->tev[1], p->tev[2]));
    return ASSE_OK;
}

int asse_select_window(asse_pool *p, uint32_t window)
{
    if (!p)
        return fail(nullptr, ASSE_EINVAL, "pool is NULL");
    if (window >= p->n_windows)
        return fail(p, ASSE_EINVAL, "window index beyond the windows of the last close");
    p->sel = window;
    return ASSE_OK;
}

int asse_estimate(asse_pool *p, const uint32_t *aips, uint64_t n, asse_superpoint *out, int where)
{
    if (!p)
        return fail(nullptr, ASSE_EINVAL, "pool is NULL");
    if (!p->scanned || p->refreshed || p->ingested || p->scan_slice != p->t)
        return fail(p, ASSE_ESTATE, "estimate needs a scan of the open slice and no refresh since");
    if (n == 0)
        return ASSE_OK;
    if (!aips || !out)
        return fail(p, ASSE_EINVAL, "NULL argument");
    const uint32_t c0 = (uint32_t)(p->t % (2 * p->cfg.k));
    if (where == ASSE_DEVICE) {
        CK(p, launch_estimate(p->P, p->w, p->pool, c0, p->scan_kp, p->aat, aips, n, out, p->sms, p->stream,
                              &p->launches));
        return ASSE_OK;
    }
    if (n > p->q_cap) {
        cudaFree(p->q_aips);
        cudaFree(p->q_out);
        p->q_aips = nullptr;
        p->q_out = nullptr;
        p->q_cap = 0;
        CK(p, cudaMalloc((void **)&p->q_aips, n * sizeof(uint32_t)));
        CK(p, cudaMalloc((void **)&p->q_out, n * sizeof(asse_superpoint)));
        p->q_cap = n;
    }
    CK(p, cudaMemcpyAsync(p->q_aips, aips, n * sizeof(uint32_t), cudaMemcpyHostToDevice, p->stream));
    CK(p, launch_estimate(p->P, p->w, p->pool, c0, p->scan_kp, p->aat, p->q_aips, n, p->q_out, p->sms, p->stream,
                          &p->launches));
    CK(p, cudaMemcpyAsync(out, p->q_out, n * sizeof(asse_superpoint), cudaMemcpyDeviceToHost, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
    return ASSE_OK;
}

int asse_report(asse_pool *p, asse_superpoint *out, uint64_t cap, uint64_t *n_out, int where)
{
    return read_list(p, true, out, cap, n_out, where);
}

int asse_candidates(asse_pool *p, asse_superpoint *out, uint64_t cap, uint64_t *n_out, int where)
{
    return read_list(p, false, out, cap, n_out, where);
}

int asse_counts(asse_pool *p, uint16_t *out, int where)
{
    if (!p || !out)
        return fail(p, ASSE_EINVAL, "NULL argument");
    if (!p->scanned)
        return fail(p, ASSE_ESTATE, "no scan");
    const size_t bytes = ((size_t)p->cfg.r << p->P.E_log2) * sizeof(uint16_t);
    CK(p, cudaMemcpyAsync(out, scan_out_w(p, p->sel).cnt, bytes,
                          where == ASSE_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
    if (where != ASSE_DEVICE)
        CK(p, cudaStreamSynchronize(p->stream));
    return ASSE_OK;
}

int asse_loads(asse_pool *p, uint64_t *out)
{
    if (!p || !out)
        return fail(p, ASSE_EINVAL, "NULL argument");
    if (!p->scanned)
        return fail(p, ASSE_ESTATE, "no scan");
    CK(p, cudaMemcpyAsync(out, scan_out_w(p, p->sel).aat, (size_t)p->cfg.r * p->P.nf * sizeof(uint64_t),
                          cudaMemcpyDeviceToHost, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
    return ASSE_OK;
}

int asse_info(const asse_pool *p, asse_pool_info *out)
{
    if (!p || !out)
        return ASSE_EINVAL;
    out->w = p->w;
    out->fields = p->F;
    out->words = p->P.Wd;
    out->E = 1u << p->P.E_log2;
    out->threshold = p->P.T;
    out->block = p->blk;
    out->k = p->P.k;
    out->paired = p->P.paired;
    out->slice = p->t;
    out->pool_words = p->pool_words;
    out->pool = p->pool;
    return ASSE_OK;
}

int asse_read_pool(asse_pool *p, uint32_t *out, int where)
{
    if (!p || !out)
        return fail(p, ASSE_EINVAL, "NULL argument");
    CK(p, cudaMemcpyAsync(out, p->pool, p->pool_words * 4,
                          where == ASSE_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
    if (where != ASSE_DEVICE)
        CK(p, cudaStreamSynchronize(p->stream));
    return ASSE_OK;
}

int asse_snapshot(asse_pool *p, void *dst, uint64_t cap, uint64_t *n_out)
{
    if (!p || !n_out)
        return fail(p, ASSE_EINVAL, "NULL argument");
    const uint64_t need = sizeof(SnapHeader) + p->pool_words * 4;
    *n_out = need;
    if (!dst)
        return ASSE_OK;
    if (cap < need)
        return fail(p, ASSE_ECAPACITY, "snapshot buffer too small");
    SnapHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "ASSEPOOL", 8);
    h.version = 1;
    h.header_bytes = sizeof(SnapHeader);
    h.cfg = p->cfg;
    h.slice = p->t;
    h.pool_words = p->pool_words;
    h.w = p->w;
    h.words = p->P.Wd;
    memcpy(dst, &h, sizeof h);
    CK(p, cudaMemcpyAsync((char *)dst + sizeof h, p->pool, p->pool_words * 4, cudaMemcpyDeviceToHost, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
    return ASSE_OK;
}

int asse_probe_random_reads(asse_pool *p, uint64_t n_reads, uint64_t *n_issued)
{
    if (!p)
        return fail(nullptr, ASSE_EINVAL, "pool is NULL");
    if (n_reads > (1ull << 34))
        return fail(p, ASSE_EINVAL, "n_reads must be at most 2^34");
    uint64_t issued = 0;
    if (n_reads > 0)
        CK(p, launch_random_reads(p->pool, p->pool_words, n_reads, p->sms, p->stream, &p->launches, &issued));
    if (n_issued)
        *n_issued = issued;
    return ASSE_OK;
}

int asse_load(asse_pool *p, const void *src, uint64_t n)
{
    if (!p || !src)
        return fail(p, ASSE_EINVAL, "NULL argument");
    p->report_host_valid = 0;
    SnapHeader h;
    if (n < sizeof h)
        return fail(p, ASSE_EINVAL, "image too small");
    memcpy(&h, src, sizeof h);
    if (memcmp(h.magic, "ASSEPOOL", 8) != 0 || h.version != 1 || h.header_bytes != sizeof h)
        return fail(p, ASSE_EINVAL, "not an ASSE pool image");
    const asse_config &a = h.cfg, &b = p->cfg;
    if (a.k != b.k || a.theta != b.theta || a.g != b.g || a.r != b.r || a.c != b.c || a.u != b.u || a.s != b.s ||
        a.A != b.A || a.bh_a != b.bh_a || a.bh_b != b.bh_b || a.counter != b.counter ||
        h.pool_words != p->pool_words || h.w != p->w || h.words != p->P.Wd)
        return fail(p, ASSE_EINVAL, "image was written by a pool with another configuration");
    if (n < sizeof h + p->pool_words * 4)
        return fail(p, ASSE_EINVAL, "image truncated");
    CK(p, cudaMemcpyAsync(p->pool, (const char *)src + sizeof h, p->pool_words * 4, cudaMemcpyHostToDevice,
                          p->stream));
    const SliceCtl c = slice_ctl(p->P, h.slice);
    CK(p, cudaMemcpyAsync(p->ctl, &c, sizeof c, cudaMemcpyHostToDevice, p->stream));
    // the key table describes the replaced state
    if (p->P.keys)
        CK(p, cudaMemsetAsync(p->P.keys, 0xff, sizeof(unsigned long long) << p->P.klg, p->stream));
    // slice counts of a histogram pool, counted again from the loaded words
    if (p->P.hist)
        CK(p, launch_hist_rebuild(p->P, p->w, p->pool, p->ctl, p->sms, p->stream, &p->launches));
    CK(p, cudaStreamSynchronize(p->stream));
    p->t = h.slice;
    p->scanned = p->restored = p->refreshed = 0;
    return ASSE_OK;
}

}  // extern "C"
