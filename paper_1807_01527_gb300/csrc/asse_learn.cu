// Learned per-ATV cardinality model (include/asse_learn.h): feature rows of
// ATV states, synthetic training states, and the MLP (FEAT -> 256 -> 256 -> 1,
// ReLU) with its training step, all in the library's own kernels.
//
// Every matrix product of the training pass runs on the 5th-generation tensor
// cores (tcgen05, BF16 operands, FP32 accumulation in tensor memory) through
// one kernel whose operands are addressed by (row, k) strides
// (launch_tc_gemm, asse_mlp_tc.cu), so the forward products and the
// transposed ones of the weight gradients (split over the batch) are the same
// kernel with a different epilogue: bias + ReLU -> BF16, bias + ReLU + dot
// with w3 (the last layer fused into the second), gradient masked by the
// ReLU -> BF16, or FP32 atomic accumulation.  Inference has its own fused
// tcgen05 kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/asse_learn.h"
#include "asse_device.cuh"
#include "asse_features.cuh"
#include "asse_mlp_tc.h"
#include "asse_pool_access.h"
#include "asse_synth.cuh"

using bf16 = __nv_bfloat16;

namespace asse {

namespace {

constexpr int FEAT = ASSE_FEAT;
constexpr int HID = ASSE_HID;
// offsets of the parameter blocks in the flat fp32 parameter vector
constexpr size_t OFF_W1 = 0;
constexpr size_t OFF_B1 = OFF_W1 + (size_t)HID * FEAT;
constexpr size_t OFF_W2 = OFF_B1 + HID;
constexpr size_t OFF_B2 = OFF_W2 + (size_t)HID * HID;
constexpr size_t OFF_W3 = OFF_B2 + HID;
constexpr size_t OFF_B3 = OFF_W3 + HID;
constexpr size_t NPARAMS = OFF_B3 + 1;
static_assert(NPARAMS == ASSE_MLP_NPARAMS, "parameter layout");

// est[i] = exp(max(y[i], 0)) where the ATV holds an active AT and the model
// is inside its training range (y <= max_log_n, the log of the largest
// cardinality it was trained on; a cardinality is at least 1), else the
// linear-counting estimate of Eq. 2 from the ATV's count: 0 for an empty
// ATV, and a saturated count g taken as g - 1/2.
__global__ void learned_combine_kernel(const float *y, const uint16_t *cnt, uint32_t g, float max_log_n,
                                       uint64_t n, float *est, uint32_t *n_fallback)
{
    uint32_t fb = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float yi = y[i];
        const uint32_t c = cnt[i];
        if (c > 0 && yi <= max_log_n) {
            est[i] = expf(fmaxf(yi, 0.0f));
        } else {
            const double cc = c >= g ? (double)g - 0.5 : (double)c;
            est[i] = (float)(-(double)g * log(((double)g - cc) / (double)g));
            fb++;
        }
    }
    fb = __reduce_add_sync(FULL_MASK, fb);
    if ((threadIdx.x & 31) == 0 && fb)
        atomicAdd(n_fallback, fb);
}

// ---------------------------------------------------------------- learned report

// The host addresses of n candidate records, contiguous for the feature kernel.
__global__ void cand_aips_kernel(const asse_superpoint *c, uint64_t n, uint32_t *aips)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        aips[i] = c[i].aip;
}

// The decision of asse_report_learned for each candidate: inside the model's
// training range its estimate exp(max(y, 0)) and est >= theta, else the
// candidate's Eq. 4 estimate and decision as restored.  The reported records
// are packed into rep, each warp taking its places with one atomic.
__global__ void learned_report_kernel(const asse_superpoint *cand, const float *y, uint64_t n, float max_log_n,
                                      float theta, asse_superpoint *rep, unsigned long long *n_rep)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // one bound per warp, so that every lane takes part in the ballot
    for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
        const uint64_t i = base + lane;
        asse_superpoint sp{};
        bool keep = false;
        if (i < n) {
            sp = cand[i];
            const float yi = y[i];
            if (yi <= max_log_n) {  // false for a NaN output: Eq. 4 stands
                sp.est = expf(fmaxf(yi, 0.0f));
                sp.flags = ASSE_SP_LEARNED | (sp.est >= theta ? ASSE_SP_REPORTED : 0u);
            }
            keep = (sp.flags & ASSE_SP_REPORTED) != 0;
        }
        const unsigned m = __ballot_sync(FULL_MASK, keep);
        unsigned long long at = 0;
        if (lane == 0 && m)
            at = atomicAdd(n_rep, (unsigned long long)__popc(m));
        at = __shfl_sync(FULL_MASK, at, 0);
        if (keep)
            rep[at + __popc(m & ((1u << lane) - 1u))] = sp;
    }
}

// ---------------------------------------------------------------- synthetic states

struct SynthArgs {
    uint64_t seed;
    uint32_t n_max_log2;
    float bg_max;
};

// One block per state: the host's distinct bips and the background set the
// ATs slice by slice (a later slice overwrites), the state is packed exactly
// as ingest would have left it at the end of slice k-1, and its feature row
// is computed from the packed words by atv_features.
template <int WB>
__global__ void __launch_bounds__(256) synth_kernel(Params P, SynthArgs S, uint64_t first, uint64_t n, bf16 *x,
                                                    float *log_n, float *lc)
{
    constexpr uint32_t F = 32 / WB;
    extern __shared__ uint32_t sm[];
    int16_t *last = reinterpret_cast<int16_t *>(sm);                // [g]
    uint32_t *words = sm + (P.g + 1) / 2;                           // [Wd]
    uint32_t *hist_w = words + P.Wd;                                 // [64][32] 16-bit, kept zero between uses
    uint16_t *hist = reinterpret_cast<uint16_t *>(hist_w);
    RangeDesc *desc = reinterpret_cast<RangeDesc *>(hist_w + HIST_WORDS);  // [Wd]
    uint32_t *actw = reinterpret_cast<uint32_t *>(desc + P.Wd);             // [Wd]
    __shared__ uint32_t end[65];
    __shared__ uint32_t card;
    __shared__ float pbg;
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = tid; i < HIST_WORDS; i += blockDim.x)
        hist_w[i] = 0;
    // the states are packed as of the end of slice k - 1 (block 0's ACT (k-1) mod 2k)
    feature_tables<WB>(P, (P.k - 1) % P.k2, P.k, desc, actw);
    __syncthreads();
    for (uint64_t si = blockIdx.x; si < n; si += gridDim.x) {
        const uint64_t key = splitmix(S.seed ^ splitmix(first + si + 0x51ED270B27ull));
        if (tid == 0) {
            const double lnmax = (double)S.n_max_log2 * 0.6931471805599453;
            double c = floor(exp(unit(key, 1) * lnmax));
            card = (uint32_t)(c < 1.0 ? 1.0 : c);
            pbg = (float)(unit(key, 2) * (double)S.bg_max);
            double tot = 0.0, w[64];
            for (uint32_t s = 0; s < P.k; s++) {
                w[s] = -log(unit(key, 16 + s) + 1e-300);
                tot += w[s];
            }
            double cum = 0.0;
            end[0] = 0;
            for (uint32_t s = 0; s < P.k; s++) {
                cum += w[s];
                end[s + 1] = s + 1 == P.k ? card : (uint32_t)floor((double)card * cum / tot);
            }
        }
        for (uint32_t h = tid; h < P.g; h += blockDim.x)
            last[h] = -1;
        __syncthreads();
        const uint32_t base = (uint32_t)(key >> 32);
        for (uint32_t s = 0; s < P.k; s++) {
            for (uint32_t h = tid; h < P.g; h += blockDim.x)
                if (unit(key ^ 0xB5ull, ((uint64_t)s << 32) | h) < (double)pbg)
                    last[h] = (int16_t)s;
            for (uint32_t j = end[s] + tid; j < end[s + 1]; j += blockDim.x)
                last[bip_hash(P, mix32(base + j))] = (int16_t)s;
            __syncthreads();
        }
        // pack: an AT last set in slice s holds that slice's ACT (C0 = s)
        for (uint32_t q = tid; q < P.Wd; q += blockDim.x) {
            uint32_t wd = 0;
            for (uint32_t j = 0; j < F; j++) {
                const uint32_t pos = q * F + j;
                if (pos < P.g) {
                    const uint32_t h = pos_at(P, pos);  // the AT stored there
                    const int s = last[h];
                    const uint32_t v = s < 0 ? P.k2 : act_of(P, (uint32_t)s, act_block(P, h));
                    wd |= v << (j * WB);
                }
            }
            words[q] = wd;
        }
        __syncthreads();
        if (tid < 32) {
            const float pw = 1.0f - powf(1.0f - pbg, (float)P.k);  // background activity over the window
            uint32_t cnt = 0;
            uint32_t wreg[FEAT_MAXM];
            load_atv_words<WB>(P, words, tid, wreg);
            atv_features<WB>(P, wreg, desc, actw, P.k, pw, powf(pw, (float)P.r), pw, hist, x + si * FEAT,
                             tid, &cnt);
            if (tid == 0) {
                log_n[si] = (float)log((double)card);
                const double c = cnt >= P.g ? (double)P.g - 0.5 : (double)cnt;
                lc[si] = (float)(-(double)P.g * log(((double)P.g - c) / (double)P.g));
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- elementwise

__global__ void fill_kernel(float *y, uint64_t n, const float *value)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        y[i] = *value;
}

// Squared error of the log: dy = 2 (y - t) / n, loss += (y - t)^2 / n.
// Squared relative error of the estimate exp(y) against exp(t): with
// e = exp(y - t), loss += (e - 1)^2 / n and dy = 2 (e - 1) e / n (y - t
// clamped at 20 so that e stays finite).
__global__ void loss_kernel(const float *y, const float *t, uint64_t n, int kind, float *dy, float *loss)
{
    float acc = 0.0f;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        if (kind == ASSE_LOSS_REL_MSE) {
            const float e = expf(fminf(d, 20.0f));
            dy[i] = 2.0f * (e - 1.0f) * e / (float)n;
            acc += (e - 1.0f) * (e - 1.0f) / (float)n;
        } else {
            dy[i] = 2.0f * d / (float)n;
            acc += d * d / (float)n;
        }
    }
    acc += __shfl_xor_sync(FULL_MASK, acc, 16);
    acc += __shfl_xor_sync(FULL_MASK, acc, 8);
    acc += __shfl_xor_sync(FULL_MASK, acc, 4);
    acc += __shfl_xor_sync(FULL_MASK, acc, 2);
    acc += __shfl_xor_sync(FULL_MASK, acc, 1);
    if ((threadIdx.x & 31) == 0)
        atomicAdd(loss, acc);
}

// dZ2 = bf16(dy[m] w3[n] [H2 > 0]); dw3[n] += dy[m] H2[m][n]; db2[n] += dZ2;
// db3 += dy.  One block of HID threads per chunk of rows.
__global__ void __launch_bounds__(HID) out_grad_kernel(const float *dy, const bf16 *H2, const float *w3, uint64_t n,
                                                       bf16 *dZ2, float *g_w3, float *g_b2, float *g_b3)
{
    const int col = threadIdx.x;
    float sw = 0.0f, sb = 0.0f, s3 = 0.0f;
    for (uint64_t m = blockIdx.x; m < n; m += gridDim.x) {
        const float d = dy[m];
        const float h = __bfloat162float(H2[m * HID + col]);
        const bf16 z = __float2bfloat16_rn(h > 0.0f ? d * w3[col] : 0.0f);
        dZ2[m * HID + col] = z;
        sw += d * h;
        sb += __bfloat162float(z);
        if (col == 0)
            s3 += d;
    }
    atomicAdd(&g_w3[col], sw);
    atomicAdd(&g_b2[col], sb);
    if (col == 0)
        atomicAdd(g_b3, s3);
}

// g_b[n] += sum over rows of Z[m][n]
__global__ void __launch_bounds__(HID) colsum_kernel(const bf16 *Z, uint64_t n, float *g_b)
{
    const int col = threadIdx.x;
    float s = 0.0f;
    for (uint64_t m = blockIdx.x; m < n; m += gridDim.x)
        s += __bfloat162float(Z[m * HID + col]);
    atomicAdd(&g_b[col], s);
}

// Adam on the fp32 parameters, refreshing the bf16 copies of W1 and W2.
__global__ void adam_kernel(float *p, const float *gr, float *m1, float *m2, uint64_t n, float lr, float b1t,
                            float b2t, bf16 *w1b, bf16 *w2b)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float g = gr[i];
        const float a = 0.9f * m1[i] + 0.1f * g;
        const float b = 0.999f * m2[i] + 0.001f * g * g;
        m1[i] = a;
        m2[i] = b;
        const float v = p[i] - lr * (a / b1t) / (sqrtf(b / b2t) + 1e-8f);
        p[i] = v;
        if (i < OFF_B1)
            w1b[i - OFF_W1] = __float2bfloat16_rn(v);
        else if (i >= OFF_W2 && i < OFF_B2)
            w2b[i - OFF_W2] = __float2bfloat16_rn(v);
    }
}

__global__ void to_bf16_kernel(const float *p, bf16 *w1b, bf16 *w2b)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < NPARAMS;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (i < OFF_B1)
            w1b[i - OFF_W1] = __float2bfloat16_rn(p[i]);
        else if (i >= OFF_W2 && i < OFF_B2)
            w2b[i - OFF_W2] = __float2bfloat16_rn(p[i]);
    }
}

}  // namespace

}  // namespace asse

using namespace asse;

struct asse_mlp {
    cudaStream_t stream = nullptr;
    float *params = nullptr, *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
    bf16 *w1b = nullptr, *w2b = nullptr;
    bf16 *w1p = nullptr, *w2p = nullptr;  // packed operand images of the tensor-core inference
    int *error = nullptr;                 // set by a kernel whose wait gave up
    uint64_t cap = 0;  // rows of the activation workspace
    bf16 *H1 = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    float *y = nullptr, *dy = nullptr, *loss = nullptr;
    uint64_t steps = 0;
    int loss_kind = ASSE_LOSS_LOG_MSE;
    // workspace of asse_report_learned, for rl_cap candidates
    unsigned char *rl = nullptr;
    uint64_t rl_cap = 0;
    uint64_t launches = 0;
    std::string err;
};

namespace {

int mlp_fail(asse_mlp *m, int code, const std::string &msg)
{
    if (m)
        m->err = msg;
    return code;
}

#define MCK(m, call)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return mlp_fail((m), ASSE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int ensure_workspace(asse_mlp *m, uint64_t rows)
{
    if (rows <= m->cap)
        return ASSE_OK;
    cudaStreamSynchronize(m->stream);
    cudaFree(m->H1);
    cudaFree(m->H2);
    cudaFree(m->dZ2);
    cudaFree(m->dZ1);
    cudaFree(m->y);
    cudaFree(m->dy);
    m->H1 = m->H2 = m->dZ2 = m->dZ1 = nullptr;
    m->y = m->dy = nullptr;
    m->cap = 0;
    const size_t act = rows * HID * sizeof(bf16);
    MCK(m, cudaMalloc(&m->H1, act));
    MCK(m, cudaMalloc(&m->H2, act));
    MCK(m, cudaMalloc(&m->dZ2, act));
    MCK(m, cudaMalloc(&m->dZ1, act));
    MCK(m, cudaMalloc(&m->y, rows * sizeof(float)));
    MCK(m, cudaMalloc(&m->dy, rows * sizeof(float)));
    m->cap = rows;
    return ASSE_OK;
}

// Forward pass of n rows into y (and H1, H2 kept for the backward pass).
int forward(asse_mlp *m, const bf16 *x, uint64_t n, float *y, bool keep)
{
    const float *P = m->params;
    MCK(m, cudaGetLastError());
    fill_kernel<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, m->stream>>>(y, n, P + OFF_B3);
    m->launches++;
    MCK(m, launch_tc_gemm(TcOperand{x, FEAT, 1}, TcOperand{m->w1b, FEAT, 1}, (int)n, HID, FEAT, 1,
                          TcEpi{TE_BIAS_RELU, P + OFF_B1, nullptr, nullptr, m->H1, nullptr, nullptr, HID}, m->error,
                          m->stream, &m->launches));
    MCK(m, launch_tc_gemm(TcOperand{m->H1, HID, 1}, TcOperand{m->w2b, HID, 1}, (int)n, HID, HID, 1,
                          TcEpi{TE_BIAS_RELU_DOT, P + OFF_B2, P + OFF_W3, nullptr, keep ? m->H2 : nullptr, nullptr, y,
                                HID},
                          m->error, m->stream, &m->launches));
    return ASSE_OK;
}

int backward(asse_mlp *m, const bf16 *x, const float *t, uint64_t n, float *loss_dev)
{
    if (int rc = ensure_workspace(m, n))
        return rc;
    if (int rc = forward(m, x, n, m->y, true))
        return rc;
    float *G = m->grads;
    MCK(m, cudaMemsetAsync(G, 0, NPARAMS * sizeof(float), m->stream));
    MCK(m, cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream));
    const unsigned eb = (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    loss_kernel<<<eb, 256, 0, m->stream>>>(m->y, t, n, m->loss_kind, m->dy, m->loss);
    const unsigned rb = (unsigned)(n < 2048 ? n : 2048);
    out_grad_kernel<<<rb, HID, 0, m->stream>>>(m->dy, m->H2, m->params + OFF_W3, n, m->dZ2, G + OFF_W3, G + OFF_B2,
                                              G + OFF_B3);
    m->launches += 2;
    MCK(m, cudaGetLastError());
    // the weight-gradient products reduce over the batch: split it so that
    // enough CTAs share the work
    const int splits = (int)((n + 255) / 256);
    // dW2[o][i] = sum_m dZ2[m][o] H1[m][i]
    MCK(m, launch_tc_gemm(TcOperand{m->dZ2, 1, HID}, TcOperand{m->H1, 1, HID}, HID, HID, (int)n, splits,
                          TcEpi{TE_ATOMIC, nullptr, nullptr, nullptr, nullptr, G + OFF_W2, nullptr, HID}, m->error,
                          m->stream, &m->launches));
    // dZ1 = (dZ2 W2) masked by H1 > 0
    MCK(m, launch_tc_gemm(TcOperand{m->dZ2, HID, 1}, TcOperand{m->w2b, 1, HID}, (int)n, HID, HID, 1,
                          TcEpi{TE_RELU_GRAD, nullptr, nullptr, m->H1, m->dZ1, nullptr, nullptr, HID}, m->error,
                          m->stream, &m->launches));
    colsum_kernel<<<rb, HID, 0, m->stream>>>(m->dZ1, n, G + OFF_B1);
    m->launches++;
    // dW1[o][j] = sum_m dZ1[m][o] X[m][j]
    MCK(m, launch_tc_gemm(TcOperand{m->dZ1, 1, HID}, TcOperand{x, 1, FEAT}, HID, FEAT, (int)n, splits,
                          TcEpi{TE_ATOMIC, nullptr, nullptr, nullptr, nullptr, G + OFF_W1, nullptr, FEAT}, m->error,
                          m->stream, &m->launches));
    if (loss_dev)
        MCK(m, cudaMemcpyAsync(loss_dev, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, m->stream));
    return ASSE_OK;
}

}  // namespace

namespace asse {

int mlp_enqueue_learned(asse_mlp *m, const FeatureView &v, float max_log_n, uint16_t *x_dev, float *est_dev,
                        uint32_t *nfb_dev, std::string *why)
{
    cudaError_t e = launch_features(v, x_dev);
    if (e != cudaSuccess) {
        *why = std::string("features launch: ") + cudaGetErrorString(e);
        return ASSE_ECUDA;
    }
    const uint64_t total = (uint64_t)v.P.r << v.P.E_log2;
    // the model's outputs go to est_dev first, then are replaced in place
    const int rc = launch_mlp_forward_tc(reinterpret_cast<const bf16 *>(x_dev), total, m->w1p, m->w2p, m->params,
                                         est_dev, m->error, v.stream, v.launches, why);
    if (rc != 0)
        return rc == 1 ? ASSE_EINVAL : ASSE_ECUDA;
    e = cudaMemsetAsync(nfb_dev, 0, sizeof(uint32_t), v.stream);
    if (e == cudaSuccess) {
        const unsigned grid = (unsigned)v.sms * 4;
        learned_combine_kernel<<<grid, 256, 0, v.stream>>>(est_dev, v.cnt, v.P.g, max_log_n, total, est_dev,
                                                           nfb_dev);
        *v.launches += 1;
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        *why = std::string("learned combine: ") + cudaGetErrorString(e);
        return ASSE_ECUDA;
    }
    return ASSE_OK;
}

}  // namespace asse

using namespace asse;

extern "C" {

int asse_estimate_learned(asse_pool *pool, asse_mlp *mlp, float max_log_n, uint16_t *x_dev, float *est_dev,
                          uint32_t *n_fallback_dev)
{
    if (!pool || !mlp || !x_dev || !est_dev || !n_fallback_dev || !(max_log_n >= 0.0f))
        return pool ? pool_fail(pool, ASSE_EINVAL, "NULL argument or negative max_log_n") : ASSE_EINVAL;
    if ((reinterpret_cast<uintptr_t>(x_dev) & 15u) != 0)
        return pool_fail(pool, ASSE_EINVAL, "x_dev must be 16-byte aligned");
    FeatureView v;
    if (int rc = pool_feature_view(pool, &v))
        return rc;
    if (mlp->stream != v.stream)
        return pool_fail(pool, ASSE_EINVAL, "the model and the pool must use the same stream");
    if (v.kp > 64)
        return pool_fail(pool, ASSE_EINVAL, "features need k' <= 64");
    std::string why;
    if (int rc = mlp_enqueue_learned(mlp, v, max_log_n, x_dev, est_dev, n_fallback_dev, &why))
        return pool_fail(pool, rc, why);
    return ASSE_OK;
}

int asse_report_learned(asse_pool *pool, asse_mlp *m, float max_log_n, asse_superpoint *out, uint64_t cap,
                        uint64_t *n_out, int where)
{
    if (!pool || !m || !n_out || !(max_log_n >= 0.0f) || (where != ASSE_HOST && where != ASSE_DEVICE))
        return pool ? pool_fail(pool, ASSE_EINVAL, "NULL argument, negative max_log_n or unknown where") : ASSE_EINVAL;
    FeatureView v;
    if (int rc = pool_feature_view(pool, &v))
        return rc;
    if (m->stream != v.stream)
        return pool_fail(pool, ASSE_EINVAL, "the model and the pool must use the same stream");
    if (v.kp > 64)
        return pool_fail(pool, ASSE_EINVAL, "features need k' <= 64");
    // workspace, in 256-byte aligned parts of rl_cap records each: feature
    // rows, candidate records, host addresses (then the model's outputs over
    // them), reported records, and the count of reported records
    auto part = [](uint64_t bytes) { return (bytes + 255) / 256 * 256; };
    const uint64_t lcap = pool_list_cap(pool);
    if (lcap > m->rl_cap) {
        cudaFree(m->rl);  // waits for work that may still use the old workspace
        m->rl = nullptr;
        m->rl_cap = 0;
        const uint64_t bytes = part(lcap * FEAT * sizeof(bf16)) + 2 * part(lcap * sizeof(asse_superpoint)) +
                               part(lcap * sizeof(float)) + 256;
        if (cudaMalloc((void **)&m->rl, bytes) != cudaSuccess) {
            cudaGetLastError();
            m->rl = nullptr;
            return pool_fail(pool, ASSE_ENOMEM, "workspace of the learned report");
        }
        m->rl_cap = lcap;
    }
    const uint64_t c = m->rl_cap;
    uint16_t *x = reinterpret_cast<uint16_t *>(m->rl);
    auto *cand = reinterpret_cast<asse_superpoint *>(m->rl + part(c * FEAT * sizeof(bf16)));
    auto *yb = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(cand) + part(c * sizeof(asse_superpoint)));
    auto *rep = reinterpret_cast<asse_superpoint *>(reinterpret_cast<unsigned char *>(yb) + part(c * sizeof(float)));
    auto *n_rep_dev =
        reinterpret_cast<unsigned long long *>(reinterpret_cast<unsigned char *>(rep) + part(c * sizeof(asse_superpoint)));
    // the candidates of the last restore (synchronises; ECAPACITY passes on an overflowed restore)
    uint64_t n = 0;
    if (int rc = asse_candidates(pool, cand, c, &n, ASSE_DEVICE)) {
        *n_out = n;
        return rc;
    }
    *n_out = 0;
    if (n == 0)
        return ASSE_OK;
    const uint64_t blocks = (n + 255) / 256, full = (uint64_t)v.sms * 4;
    const unsigned grid = (unsigned)(blocks < full ? blocks : full);
    uint32_t *aips = reinterpret_cast<uint32_t *>(yb);
    cand_aips_kernel<<<grid, 256, 0, v.stream>>>(cand, n, aips);
    *v.launches += 1;
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess)
        return pool_fail(pool, ASSE_ECUDA, std::string("candidate addresses: ") + cudaGetErrorString(e));
    if (int rc = asse_candidate_features(pool, aips, n, x))
        return rc;
    std::string why;
    if (int rc = launch_mlp_forward_tc(reinterpret_cast<const bf16 *>(x), n, m->w1p, m->w2p, m->params, yb, m->error,
                                       v.stream, v.launches, &why))
        return pool_fail(pool, rc == 1 ? ASSE_EINVAL : ASSE_ECUDA, why);
    unsigned long long n_rep = 0;
    int gave_up = 0;
    cudaError_t e = cudaMemsetAsync(n_rep_dev, 0, sizeof(unsigned long long), v.stream);
    if (e == cudaSuccess) {
        learned_report_kernel<<<grid, 256, 0, v.stream>>>(cand, yb, n, max_log_n, (float)v.P.theta, rep, n_rep_dev);
        *v.launches += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&n_rep, n_rep_dev, sizeof n_rep, cudaMemcpyDeviceToHost, v.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&gave_up, m->error, sizeof gave_up, cudaMemcpyDeviceToHost, v.stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(v.stream);
    if (e != cudaSuccess)
        return pool_fail(pool, ASSE_ECUDA, std::string("learned report: ") + cudaGetErrorString(e));
    if (gave_up)
        return pool_fail(pool, ASSE_ETIMEOUT, "the tensor-core MLP gave up waiting for its pipeline");
    *n_out = n_rep;
    const uint64_t k = n_rep < cap ? n_rep : cap;
    if (k > 0) {
        if (!out)
            return pool_fail(pool, ASSE_EINVAL, "out is NULL");
        e = cudaMemcpyAsync(out, rep, k * sizeof(asse_superpoint),
                            where == ASSE_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, v.stream);
        if (e == cudaSuccess && where != ASSE_DEVICE)
            e = cudaStreamSynchronize(v.stream);
        if (e != cudaSuccess)
            return pool_fail(pool, ASSE_ECUDA, std::string("learned report copy: ") + cudaGetErrorString(e));
    }
    if (n_rep > cap)
        return pool_fail(pool, ASSE_ECAPACITY, "output capacity smaller than the learned report");
    return ASSE_OK;
}

int asse_synth_states(const asse_synth_cfg *cfg, uint64_t first, uint64_t n, uint16_t *x_dev, float *log_n_dev,
                      float *lc_dev, void *stream)
{
    if (!cfg || (n > 0 && (!x_dev || !log_n_dev || !lc_dev)))
        return ASSE_EINVAL;
    if (cfg->k < 1 || cfg->k > 64 || cfg->g < 2 * cfg->k || cfg->g > 4096 || cfg->r < 1 || cfg->n_max_log2 > 24 ||
        (cfg->bh_a & 1) == 0 || !(cfg->bg_max >= 0.0f && cfg->bg_max <= 1.0f))
        return ASSE_EINVAL;
    if (n == 0)
        return ASSE_OK;
    Params P{};
    P.k = cfg->k;
    P.k2 = 2 * cfg->k;
    P.g = cfg->g;
    P.r = cfg->r;
    P.blk = cfg->g / (2 * cfg->k);
    P.blk_magic = ((1ull << 32) + P.blk - 1) / P.blk;
    P.paired = 1;  // the storage order of a timestamp pool's ACT blocks
    P.bh_a = cfg->bh_a;
    P.bh_b = cfg->bh_b;
    const uint32_t w = packed_width(ASSE_COUNTER_AT, cfg->k);
    const uint32_t Fw = 32 / w;
    P.Wd = ((cfg->g + Fw - 1) / Fw + 7) / 8 * 8;
    SynthArgs S{cfg->seed, cfg->n_max_log2, cfg->bg_max};
    const size_t smem = ((cfg->g + 1) / 2 + P.Wd + HIST_WORDS) * sizeof(uint32_t) +
                        (size_t)P.Wd * (sizeof(RangeDesc) + sizeof(uint32_t));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(n < (uint64_t)sms * 8 ? n : (uint64_t)sms * 8);
    cudaError_t e = dispatch_w(w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        synth_kernel<WB><<<grid, 256, smem, (cudaStream_t)stream>>>(P, S, first, n, reinterpret_cast<bf16 *>(x_dev),
                                                                   log_n_dev, lc_dev);
        return cudaGetLastError();
    });
    return e == cudaSuccess ? ASSE_OK : ASSE_ECUDA;
}

int asse_mlp_create(uint64_t seed, void *stream, asse_mlp **out)
{
    if (!out)
        return ASSE_EINVAL;
    *out = nullptr;
    asse_mlp *m = new (std::nothrow) asse_mlp();
    if (!m)
        return ASSE_ENOMEM;
    m->stream = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t b) {
        if (e == cudaSuccess)
            e = cudaMalloc(p, b);
    };
    alloc((void **)&m->params, NPARAMS * sizeof(float));
    alloc((void **)&m->grads, NPARAMS * sizeof(float));
    alloc((void **)&m->m1, NPARAMS * sizeof(float));
    alloc((void **)&m->m2, NPARAMS * sizeof(float));
    alloc((void **)&m->w1b, (size_t)HID * FEAT * sizeof(bf16));
    alloc((void **)&m->w2b, (size_t)HID * HID * sizeof(bf16));
    alloc((void **)&m->loss, sizeof(float));
    alloc((void **)&m->w1p, (size_t)HID * FEAT * sizeof(bf16));
    alloc((void **)&m->w2p, (size_t)HID * HID * sizeof(bf16));
    alloc((void **)&m->error, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemsetAsync(m->error, 0, sizeof(int), m->stream);
    if (e != cudaSuccess) {
        asse_mlp_destroy(m);
        return e == cudaErrorMemoryAllocation ? ASSE_ENOMEM : ASSE_ECUDA;
    }
    // Kaiming-uniform weights (bound sqrt(6 / fan_in)), zero biases, drawn on
    // the host from SplitMix64 of the seed
    std::vector<float> h(NPARAMS, 0.0f);
    uint64_t state = seed * 0x9E3779B97F4A7C15ull + 1;
    auto next = [&]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    const double b1 = std::sqrt(6.0 / 68.0), b2 = std::sqrt(6.0 / HID), b3 = std::sqrt(6.0 / HID);
    for (size_t o = 0; o < (size_t)HID; o++)
        for (size_t j = 0; j < (size_t)FEAT; j++)
            h[OFF_W1 + o * FEAT + j] = j < 68 ? (float)((2 * next() - 1) * b1) : 0.0f;
    for (size_t i = 0; i < (size_t)HID * HID; i++)
        h[OFF_W2 + i] = (float)((2 * next() - 1) * b2);
    for (size_t i = 0; i < (size_t)HID; i++)
        h[OFF_W3 + i] = (float)((2 * next() - 1) * b3);
    int rc = asse_mlp_set_params(m, h.data());
    if (rc == ASSE_OK) {
        cudaMemsetAsync(m->m1, 0, NPARAMS * sizeof(float), m->stream);
        cudaMemsetAsync(m->m2, 0, NPARAMS * sizeof(float), m->stream);
        if (cudaStreamSynchronize(m->stream) != cudaSuccess)
            rc = ASSE_ECUDA;
    }
    if (rc != ASSE_OK) {
        asse_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return ASSE_OK;
}

void asse_mlp_destroy(asse_mlp *m)
{
    if (!m)
        return;
    cudaStreamSynchronize(m->stream);
    for (void *p : {(void *)m->params, (void *)m->grads, (void *)m->m1, (void *)m->m2, (void *)m->w1b, (void *)m->w2b,
                    (void *)m->H1, (void *)m->H2, (void *)m->dZ2, (void *)m->dZ1, (void *)m->y, (void *)m->dy,
                    (void *)m->loss, (void *)m->w1p, (void *)m->w2p, (void *)m->error, (void *)m->rl})
        cudaFree(p);
    delete m;
}

int asse_mlp_set_stream(asse_mlp *m, void *stream)
{
    if (!m)
        return ASSE_EINVAL;
    m->stream = (cudaStream_t)stream;
    return ASSE_OK;
}

int asse_mlp_get_params(asse_mlp *m, float *host)
{
    if (!m || !host)
        return ASSE_EINVAL;
    MCK(m, cudaMemcpyAsync(host, m->params, NPARAMS * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    MCK(m, cudaStreamSynchronize(m->stream));
    return ASSE_OK;
}

int asse_mlp_set_params(asse_mlp *m, const float *host)
{
    if (!m || !host)
        return ASSE_EINVAL;
    MCK(m, cudaMemcpyAsync(m->params, host, NPARAMS * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    to_bf16_kernel<<<64, 256, 0, m->stream>>>(m->params, m->w1b, m->w2b);
    m->launches++;
    MCK(m, cudaGetLastError());
    MCK(m, launch_mlp_pack(m->params, m->w1p, m->w2p, m->stream, &m->launches));
    MCK(m, cudaStreamSynchronize(m->stream));
    return ASSE_OK;
}

int asse_mlp_get_grads(asse_mlp *m, float *host)
{
    if (!m || !host)
        return ASSE_EINVAL;
    MCK(m, cudaMemcpyAsync(host, m->grads, NPARAMS * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    MCK(m, cudaStreamSynchronize(m->stream));
    return ASSE_OK;
}

int asse_mlp_forward(asse_mlp *m, const uint16_t *x_dev, uint64_t n, float *y_dev)
{
    if (!m || (n > 0 && (!x_dev || !y_dev)))
        return ASSE_EINVAL;
    if (n > 0x7fffffffull)
        return mlp_fail(m, ASSE_EINVAL, "at most 2^31-1 rows per call");
    if (n == 0)
        return ASSE_OK;
    std::string why;
    const int rc = launch_mlp_forward_tc(reinterpret_cast<const bf16 *>(x_dev), n, m->w1p, m->w2p, m->params, y_dev,
                                         m->error, m->stream, &m->launches, &why);
    if (rc == 1)
        return mlp_fail(m, ASSE_EINVAL, why);
    if (rc != 0)
        return mlp_fail(m, ASSE_ECUDA, why);
    return ASSE_OK;
}

int asse_mlp_backward(asse_mlp *m, const uint16_t *x_dev, const float *t_dev, uint64_t n, float *loss_dev)
{
    if (!m || n == 0 || !x_dev || !t_dev)
        return ASSE_EINVAL;
    if (n > 0x7fffffffull)
        return mlp_fail(m, ASSE_EINVAL, "at most 2^31-1 rows per call");
    return backward(m, reinterpret_cast<const bf16 *>(x_dev), t_dev, n, loss_dev);
}

int asse_mlp_train_step(asse_mlp *m, const uint16_t *x_dev, const float *t_dev, uint64_t n, float lr,
                        float *loss_dev)
{
    if (int rc = asse_mlp_backward(m, x_dev, t_dev, n, loss_dev))
        return rc;
    m->steps++;
    const float b1t = 1.0f - powf(0.9f, (float)m->steps), b2t = 1.0f - powf(0.999f, (float)m->steps);
    adam_kernel<<<128, 256, 0, m->stream>>>(m->params, m->grads, m->m1, m->m2, NPARAMS, lr, b1t, b2t, m->w1b,
                                           m->w2b);
    m->launches++;
    MCK(m, cudaGetLastError());
    MCK(m, launch_mlp_pack(m->params, m->w1p, m->w2p, m->stream, &m->launches));
    return ASSE_OK;
}

int asse_mlp_set_loss(asse_mlp *m, int kind)
{
    if (!m)
        return ASSE_EINVAL;
    if (kind != ASSE_LOSS_LOG_MSE && kind != ASSE_LOSS_REL_MSE)
        return mlp_fail(m, ASSE_EINVAL, "loss must be ASSE_LOSS_LOG_MSE or ASSE_LOSS_REL_MSE");
    m->loss_kind = kind;
    return ASSE_OK;
}

int asse_mlp_check(asse_mlp *m)
{
    if (!m)
        return ASSE_EINVAL;
    MCK(m, cudaStreamSynchronize(m->stream));
    int flag = 0;
    MCK(m, cudaMemcpy(&flag, m->error, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag)
        return mlp_fail(m, ASSE_ETIMEOUT, "a tensor-core MLP kernel gave up waiting for its pipeline");
    return ASSE_OK;
}

const char *asse_mlp_last_error(const asse_mlp *m) { return m ? m->err.c_str() : ""; }

}  // extern "C"
