// Inference of the learned per-ATV estimator on the 5th-generation tensor
// cores: y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 for every feature row,
// the whole network in one persistent kernel (one CTA per SM).
//
// Per tile of 128 rows:
//   layer 1  acc1[128][256] = X[128][80] W1^T  tcgen05.mma, 5 K-steps of 16
//   epilogue H1 = bf16(relu(acc1 + b1)) written to shared memory
//   layer 2  acc2[128][256] = H1 W2^T           tcgen05.mma, 16 K-steps
//   epilogue y = sum_n bf16(relu(acc2 + b2))[n] w3[n] + b3
// The accumulators live in tensor memory (acc1 in columns 0..255, acc2 in
// 256..511 of a 512-column allocation), W2 stays resident in shared memory
// for the whole kernel (128 KB), and layer 1's operands stream through two
// stages: each K-step brings 16 feature columns of the tile (two TMA tiled
// loads from the row-major feature matrix, out-of-range rows filled with
// zeros) and the matching 16 columns of W1 (one bulk copy, L2-resident).
//
// Warp roles (20 warps): warp 0 issues the copies, warp 1 owns the tensor
// memory and one of its lanes issues every MMA, warps 4..19 are the epilogue
// (four warpgroups; warp w reads accumulator lanes 32 (w mod 4) ..; warpgroup
// h takes columns 64 h .. 64 h + 63 of each accumulator).  The MMA of layer 2
// of one tile and layer 1 of the next run back to back while the epilogue
// drains acc2.
//
// Shared-memory operand layouts (no swizzle, K-major core matrices of 8 rows
// x 16 bytes; LBO = byte distance of core matrices adjacent in K, SBO = in
// M or N):
//   X stage  [k-group 2][row 128][8]         LBO 2048, SBO 128 (TMA box 8 x 128)
//   W1 stage [n-group 32][k-group 2][8][8]    LBO 128,  SBO 256
//   W2       [n-group 32][k-group 32][8][8]   LBO 128,  SBO 4096
//   H1       [m-group 16][k-group 32][8][8]   LBO 128,  SBO 4096
// W1 and W2 are packed into these layouts in global memory (pack_kernel)
// whenever the parameters change.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/asse_learn.h"
#include "asse_device.cuh"
#include "asse_mlp_tc.h"
#include "asse_ptx.cuh"

namespace asse {

namespace {

using bf16 = __nv_bfloat16;

constexpr int FEAT = ASSE_FEAT;
constexpr int HID = ASSE_HID;
constexpr int TM = 128;                         // rows per tile (MMA M)
constexpr int K1_STEPS = FEAT / 16;             // 5
constexpr int K2_STEPS = HID / 16;              // 16
constexpr int EPI_WARP0 = 4;
constexpr int EPI_WARPS = 16;                   // four warpgroups, 64 accumulator columns each
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr int THREADS = (EPI_WARP0 + EPI_WARPS) * 32;
constexpr int EPI_COLS = HID / (EPI_WARPS / 4);  // 64

// parameter offsets (fp32 vector, asse_learn.h order)
constexpr size_t P_B1 = (size_t)HID * FEAT;
constexpr size_t P_B2 = P_B1 + HID + (size_t)HID * HID;
constexpr size_t P_W3 = P_B2 + HID;
constexpr size_t P_B3 = P_W3 + HID;

// shared memory (bytes from a 1024-aligned base)
constexpr uint32_t X_STAGE = 2 * TM * 16;       // 4096
constexpr uint32_t W1_STAGE = 2 * HID * 16;     // 8192
constexpr uint32_t SM_X = 0;                    // 2 stages of X
constexpr uint32_t SM_W1 = SM_X + 2 * X_STAGE;  // 2 stages of W1
constexpr uint32_t SM_H1 = SM_W1 + 2 * W1_STAGE;
constexpr uint32_t SM_W2 = SM_H1 + TM * HID * 2;
constexpr uint32_t SM_BIAS = SM_W2 + HID * HID * 2;  // b1, b2, w3 (fp32)
constexpr uint32_t SM_RED = SM_BIAS + 3 * HID * 4;   // [2][4][128] fp32 partial dots
constexpr uint32_t SM_BAR = SM_RED + 2 * 4 * TM * 4;
constexpr int NBAR = 11;
constexpr uint32_t SM_MISC = SM_BAR + NBAR * 8;      // tmem base, abort flag
constexpr uint32_t SM_TOTAL = SM_MISC + 16;
constexpr uint32_t SMEM_BYTES = SM_TOTAL + 1024;     // slack for the alignment of the base
static_assert(SMEM_BYTES <= 232448, "shared memory of one CTA");
static_assert(SM_W2 % 1024 == 0 && SM_H1 % 1024 == 0, "operand alignment");

// barrier indices
enum {
    B_FULL0 = 0, B_FULL1, B_EMPTY0, B_EMPTY1, B_ACC1_FULL, B_E1_DONE, B_ACC2_FULL, B_ACC2_EMPTY, B_W, B_FINAL, B_RED
};

constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC2_COL = 256;

// ---------------------------------------------------------------- tcgen05

// Shared-memory matrix descriptor: start address, LBO and SBO in 16-byte
// units, descriptor version 1 (bits 46..47), no swizzle (bits 61..63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4..5 = 1), BF16
// A and B (bits 7..9, 10..12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17..22, M >> 4 at bits 24..28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(HID >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
        : "memory");
}

// Arrive on bar once every tcgen05 operation this thread issued so far is done.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 64 consecutive accumulator columns of this thread's lane, waited for.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float *v)
{
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 64; i++)
        v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// A bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile uint32_t *abort_flag)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag)
            return false;
        if (clock64() - t0 > WAIT_CYCLES) {
            *abort_flag = 1u;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}

// ---------------------------------------------------------------- kernels

// fp32 parameters -> the packed BF16 images of W1 and W2 (layouts above).
__global__ void pack_kernel(const float *params, bf16 *w1p, bf16 *w2p)
{
    const uint32_t n1 = HID * FEAT, n2 = HID * HID;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2; i += gridDim.x * blockDim.x) {
        if (i < n1) {
            const uint32_t n = i / FEAT, k = i % FEAT;
            const uint32_t j = k / 16, kg = (k % 16) / 8;
            w1p[j * (HID * 16) + (n / 8) * 128 + kg * 64 + (n % 8) * 8 + (k % 8)] = __float2bfloat16_rn(params[i]);
        } else {
            const uint32_t e = i - n1, n = e / HID, k = e % HID;
            w2p[(n / 8) * (HID * 8) + (k / 8) * 64 + (n % 8) * 8 + (k % 8)] =
                __float2bfloat16_rn(params[P_B1 + HID + e]);
        }
    }
}

__global__ void __launch_bounds__(THREADS, 1)
    mlp_forward_kernel(const __grid_constant__ CUtensorMap xmap, uint32_t n, const bf16 *w1p, const bf16 *w2p,
                       const float *params, float *y, int *error)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + SM_BAR);
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(sm + SM_MISC);
    volatile uint32_t *abort_flag = tmem_slot + 1;
    float *b1s = reinterpret_cast<float *>(sm + SM_BIAS);
    float *b2s = b1s + HID;
    float *w3s = b2s + HID;
    float *red = reinterpret_cast<float *>(sm + SM_RED);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t n_tiles = (n + TM - 1) / TM;

    if (tid == 0) {
        mbar_init(&bar[B_FULL0], 1);
        mbar_init(&bar[B_FULL1], 1);
        mbar_init(&bar[B_EMPTY0], 1);
        mbar_init(&bar[B_EMPTY1], 1);
        mbar_init(&bar[B_ACC1_FULL], 1);
        mbar_init(&bar[B_E1_DONE], EPI_THREADS);
        mbar_init(&bar[B_ACC2_FULL], 1);
        mbar_init(&bar[B_ACC2_EMPTY], EPI_THREADS);
        mbar_init(&bar[B_W], 1);
        mbar_init(&bar[B_FINAL], 1);
        mbar_init(&bar[B_RED], EPI_THREADS - EPI_THREADS / 4);
        tmem_slot[1] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == 1) {
        // 512 columns: with this kernel's shared memory one CTA fits an SM,
        // so the allocation never waits for another CTA
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(const_cast<uint32_t *>(tmem_slot))),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < HID; i += THREADS) {
        b1s[i] = params[P_B1 + i];
        b2s[i] = params[P_B2 + i];
        w3s[i] = params[P_W3 + i];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot[0];
    const float b3 = params[P_B3];

    if (warp == 0) {
        // ------------------------------------------------ copies
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&xmap)) : "memory");
            mbar_expect_tx(&bar[B_W], HID * HID * 2);
            for (int c = 0; c < 8; c++)
                bulk_load(sm + SM_W2 + c * 16384, reinterpret_cast<const uint8_t *>(w2p) + c * 16384, 16384,
                          &bar[B_W]);
            uint32_t step = 0;
            bool ok = true;
            for (uint32_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                for (int j = 0; j < K1_STEPS; j++, step++) {
                    const uint32_t s = step & 1u, use = step >> 1;
                    if (use > 0 && !wait_or_abort(&bar[B_EMPTY0 + s], (use - 1) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&bar[B_FULL0 + s], X_STAGE + W1_STAGE);
                    uint8_t *xs = sm + SM_X + s * X_STAGE;
                    tma_load_2d(xs, &xmap, 16 * j, (int)(tile * TM), &bar[B_FULL0 + s]);
                    tma_load_2d(xs + TM * 16, &xmap, 16 * j + 8, (int)(tile * TM), &bar[B_FULL0 + s]);
                    bulk_load(sm + SM_W1 + s * W1_STAGE, reinterpret_cast<const uint8_t *>(w1p) + j * W1_STAGE,
                              W1_STAGE, &bar[B_FULL0 + s]);
                }
            }
            // let every copy issued above land before the CTA can exit
            for (uint32_t s = 0; s < 2; s++) {
                const uint32_t uses = (step + 1 - s) / 2;
                if (uses > 0 && !mbar_wait(&bar[B_FULL0 + s], (uses - 1) & 1u))
                    tmem_slot[1] = 1u;
            }
            if (!mbar_wait(&bar[B_W], 0))
                tmem_slot[1] = 1u;
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t x_base = smem_addr(sm + SM_X), w1_base = smem_addr(sm + SM_W1);
            const uint32_t h1_base = smem_addr(sm + SM_H1), w2_base = smem_addr(sm + SM_W2);
            uint32_t step = 0, it = 0;
            bool ok = wait_or_abort(&bar[B_W], 0, abort_flag);
            for (uint32_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, it++) {
                // acc1 is free once the epilogue has read the previous tile's
                if (it > 0 && !wait_or_abort(&bar[B_E1_DONE], (it - 1) & 1u, abort_flag))
                    break;
                tc_fence_after();
                for (int j = 0; j < K1_STEPS; j++, step++) {
                    const uint32_t s = step & 1u, use = step >> 1;
                    if (!wait_or_abort(&bar[B_FULL0 + s], use & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    mma_f16(tmem, sdesc(x_base + s * X_STAGE, 2048, 128), sdesc(w1_base + s * W1_STAGE, 128, 256),
                            j > 0);
                    mma_commit(&bar[B_EMPTY0 + s]);
                }
                if (!ok)
                    break;
                mma_commit(&bar[B_ACC1_FULL]);
                // H1 of this tile written; acc2 drained by the previous tile's epilogue
                if (!wait_or_abort(&bar[B_E1_DONE], it & 1u, abort_flag))
                    break;
                if (it > 0 && !wait_or_abort(&bar[B_ACC2_EMPTY], (it - 1) & 1u, abort_flag))
                    break;
                tc_fence_after();
                for (int j = 0; j < K2_STEPS; j++)
                    mma_f16(tmem + ACC2_COL, sdesc(h1_base + j * 256, 128, 4096), sdesc(w2_base + j * 256, 128, 4096),
                            j > 0);
                mma_commit(&bar[B_ACC2_FULL]);
            }
            // every issued MMA completes before the tensor memory is freed
            mma_commit(&bar[B_FINAL]);
            if (!mbar_wait(&bar[B_FINAL], 0))
                tmem_slot[1] = 1u;
        }
    } else if (warp >= EPI_WARP0) {
        // ------------------------------------------------ epilogue
        const int quarter = (warp - EPI_WARP0) >> 2;  // accumulator columns 64 quarter .. + 63
        const int c0 = quarter * EPI_COLS;
        const int row = (warp & 3) * 32 + lane;
        const uint32_t lane_addr = (uint32_t)((warp & 3) * 32) << 16;
        uint8_t *h1 = sm + SM_H1 + (row >> 3) * 4096 + (row & 7) * 16;
        uint32_t it = 0;
        for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, it++) {
            // the tensor-memory loads below are warp-collective: every wait's
            // outcome is made uniform across the warp
            if (!__all_sync(FULL_MASK, wait_or_abort(&bar[B_ACC1_FULL], it & 1u, abort_flag)))
                break;
            tc_fence_after();
            {
                float v[64];
                tmem_ld64(tmem + lane_addr + c0, v);
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const float4 ba = *reinterpret_cast<const float4 *>(b1s + c0 + q * 8);
                    const float4 bb = *reinterpret_cast<const float4 *>(b1s + c0 + q * 8 + 4);
                    uint4 o;
                    o.x = pack_bf16x2(fmaxf(v[q * 8 + 0] + ba.x, 0.0f), fmaxf(v[q * 8 + 1] + ba.y, 0.0f));
                    o.y = pack_bf16x2(fmaxf(v[q * 8 + 2] + ba.z, 0.0f), fmaxf(v[q * 8 + 3] + ba.w, 0.0f));
                    o.z = pack_bf16x2(fmaxf(v[q * 8 + 4] + bb.x, 0.0f), fmaxf(v[q * 8 + 5] + bb.y, 0.0f));
                    o.w = pack_bf16x2(fmaxf(v[q * 8 + 6] + bb.z, 0.0f), fmaxf(v[q * 8 + 7] + bb.w, 0.0f));
                    *reinterpret_cast<uint4 *>(h1 + ((c0 >> 3) + q) * 128) = o;
                }
            }
            fence_async_smem();  // H1 (generic stores) before the MMA reads it
            tc_fence_before();
            mbar_arrive(&bar[B_E1_DONE]);
            if (!__all_sync(FULL_MASK, wait_or_abort(&bar[B_ACC2_FULL], it & 1u, abort_flag)))
                break;
            tc_fence_after();
            float dot = 0.0f;
            {
                float v[64];
                tmem_ld64(tmem + lane_addr + ACC2_COL + c0, v);
                tc_fence_before();
                mbar_arrive(&bar[B_ACC2_EMPTY]);  // acc2 is in registers: the next tile's layer 2 may start
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const float4 bq = *reinterpret_cast<const float4 *>(b2s + c0 + q * 4);
                    const float4 wq = *reinterpret_cast<const float4 *>(w3s + c0 + q * 4);
                    dot = fmaf(__bfloat162float(__float2bfloat16_rn(fmaxf(v[q * 4 + 0] + bq.x, 0.0f))), wq.x, dot);
                    dot = fmaf(__bfloat162float(__float2bfloat16_rn(fmaxf(v[q * 4 + 1] + bq.y, 0.0f))), wq.y, dot);
                    dot = fmaf(__bfloat162float(__float2bfloat16_rn(fmaxf(v[q * 4 + 2] + bq.z, 0.0f))), wq.z, dot);
                    dot = fmaf(__bfloat162float(__float2bfloat16_rn(fmaxf(v[q * 4 + 3] + bq.w, 0.0f))), wq.w, dot);
                }
            }
            // quarters 1..3 hand their partial sums to quarter 0
            float *r = red + (it & 1u) * 4 * TM;
            if (quarter > 0) {
                r[quarter * TM + row] = dot;
                mbar_arrive(&bar[B_RED]);
            } else {
                if (!__all_sync(FULL_MASK, wait_or_abort(&bar[B_RED], it & 1u, abort_flag)))
                    break;
                const uint32_t m = tile * TM + row;
                if (m < n)
                    y[m] = (((dot + r[TM + row]) + r[2 * TM + row]) + r[3 * TM + row]) + b3;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    if (tid == 0 && tmem_slot[1] != 0u)
        atomicExch(error, 1);
}

// ---------------------------------------------------------------- training GEMMs

// C[M][N] = sum_k A(m, k) B(n, k) for the products of the training pass, on
// the tensor cores.  One CTA of four warps computes a 128 x BN tile (BN = 64,
// or N when N is not a multiple of 64; N <= 256, a multiple of 16) over the
// k range of blockIdx.z; A and B are gathered
// from global memory through their (row, k) strides into the K-major
// core-matrix layout in shared memory (the weight-gradient products read
// their operands transposed), 64 k at a time through two stages; one thread
// issues the MMAs (M = 128, N, K = 16) into a tensor-memory accumulator and
// commits each stage to an mbarrier, so the gather of the next stage overlaps
// the MMAs of this one.  The epilogue reads the accumulator with tcgen05.ld
// (warp w: rows 32 w ..) and applies the step's fused operation.
constexpr int TG_THREADS = 128;
constexpr int TG_KC = 64;                               // k per stage
constexpr uint32_t TG_A = 128 * TG_KC * 2;              // 16 KB
constexpr uint32_t TG_B = 256 * TG_KC * 2;              // 32 KB
constexpr uint32_t TG_BAR = 2 * (TG_A + TG_B);          // 2 stage barriers + final barrier + tmem slot, abort
constexpr uint32_t TG_SMEM = TG_BAR + 64 + 1024;        // + alignment slack of the base
constexpr uint32_t TG_TMEM_COLS = 256;

__device__ __forceinline__ void mma_f16_n(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 32 consecutive accumulator columns of this thread's lane, waited for.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; i++)
        v[i] = __uint_as_float(r[i]);
}

// Gather rows [r0, r0 + rows) x k [k0, k0 + 64) of an operand into the
// K-major core-matrix layout: element (row, k) at byte
// (row / 8) * 1024 + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2; outside
// [0, nrows) x [k0, kend) zero.  Rows contiguous in k (sk = 1, 16-byte
// aligned groups) move as one 16-byte load per 8 k; otherwise each thread
// takes consecutive rows so that the warp's loads of one k are contiguous
// when the operand is row-contiguous (si = 1).
__device__ __forceinline__ void tg_gather(uint8_t *dst, TcOperand op, int r0, int rows, int nrows, int k0, int kend)
{
    const bool vec = op.sk == 1 && (op.si % 8) == 0 && (reinterpret_cast<uintptr_t>(op.p) & 15u) == 0;
    for (int e = threadIdx.x; e < rows * (TG_KC / 8); e += TG_THREADS) {
        const int row = vec ? e / (TG_KC / 8) : e % rows;
        const int kg = vec ? e % (TG_KC / 8) : e / rows;
        const int i = r0 + row, k = k0 + kg * 8;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (i < nrows) {
            if (vec && k + 8 <= kend) {
                v = *reinterpret_cast<const uint4 *>(op.p + (long)i * op.si + k);
            } else {
                uint16_t h[8];
#pragma unroll
                for (int j = 0; j < 8; j++)
                    h[j] = k + j < kend ? __bfloat16_as_ushort(op.p[(long)i * op.si + (long)(k + j) * op.sk]) : 0;
                v = make_uint4(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16),
                               h[4] | ((uint32_t)h[5] << 16), h[6] | ((uint32_t)h[7] << 16));
            }
        }
        *reinterpret_cast<uint4 *>(dst + (row >> 3) * 1024 + kg * 128 + (row & 7) * 16) = v;
    }
}

// The CTA at (x, y, z) computes rows 128 x .. and columns BN y .. BN y + BN - 1
// over the z-th k range.
__global__ void __launch_bounds__(TG_THREADS) tc_gemm_kernel(TcOperand A, TcOperand B, int M, int N, int BN, int K,
                                                             int kchunk, TcEpi epi, int *error)
{
    extern __shared__ uint8_t tg_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tg_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + TG_BAR);  // [0], [1] stages, [2] final
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(bar + 3);
    volatile uint32_t *abort_flag = tmem_slot + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    const int nchunks = ke > kb ? (ke - kb + TG_KC - 1) / TG_KC : 0;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        tmem_slot[1] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(const_cast<uint32_t *>(tmem_slot))),
                     "r"(TG_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot[0];
    // FP32 accumulator, BF16 A and B, both K-major, N >> 3, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((128u >> 4) << 24);
    bool ok = true;
    for (int c = 0; c < nchunks && ok; c++) {
        const int s = c & 1;
        // the stage is free once the MMAs of the chunk two back have read it
        if (c >= 2 && !__syncthreads_and(wait_or_abort(&bar[s], ((c - 2) >> 1) & 1, abort_flag))) {
            ok = false;
            break;
        }
        uint8_t *sa = sm + s * (TG_A + TG_B), *sb = sa + TG_A;
        const int k0 = kb + c * TG_KC;
        tg_gather(sa, A, m0, 128, M, k0, ke);
        tg_gather(sb, B, n0, BN, N, k0, ke);
        fence_async_smem();  // the generic stores before the tensor core reads them
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t ab = smem_addr(sa), bb = smem_addr(sb);
#pragma unroll
            for (int kk = 0; kk < TG_KC / 16; kk++)
                mma_f16_n(tmem, sdesc(ab + kk * 256, 128, 1024), sdesc(bb + kk * 256, 128, 1024), idesc,
                          (c > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&bar[s]);
        }
    }
    // every MMA done (or none issued) before the accumulator is read or freed
    if (tid == 0) {
        mma_commit(&bar[2]);
    }
    const bool done = __syncthreads_and(ok && wait_or_abort(&bar[2], 0, abort_flag));
    if (!done && tid == 0)
        mbar_wait(&bar[2], 0);  // bounded: the committed MMAs finish before the free below
    tc_fence_after();
    if (done && nchunks > 0) {
        const int m = m0 + warp * 32 + lane;
        float dot = 0.0f;
        for (int cb = 0; cb < BN; cb += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + cb, v);
            if (m >= M)
                continue;
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const int n = n0 + cb + j;
                if (cb + j >= BN || n >= N)
                    break;
                const float a = v[j];
                if (epi.kind == TE_ATOMIC) {
                    atomicAdd(&epi.outf[(long)m * epi.ld + n], a);
                } else if (epi.kind == TE_RELU_GRAD) {
                    const float act = __bfloat162float(epi.act[(long)m * epi.ld + n]);
                    epi.out[(long)m * epi.ld + n] = __float2bfloat16_rn(act > 0.0f ? a : 0.0f);
                } else {
                    const bf16 h = __float2bfloat16_rn(fmaxf(a + epi.bias[n], 0.0f));
                    if (epi.out)
                        epi.out[(long)m * epi.ld + n] = h;
                    if (epi.kind == TE_BIAS_RELU_DOT)
                        dot = fmaf(__bfloat162float(h), epi.w3[n], dot);
                }
            }
        }
        if (epi.kind == TE_BIAS_RELU_DOT && m < M)
            atomicAdd(&epi.y[m], dot);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TG_TMEM_COLS)
                     : "memory");
    if (tid == 0 && (!done || tmem_slot[1] != 0u))
        atomicExch(error, 1);
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn()
{
    // looked up once per process (the driver's entry point does not change)
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

}  // namespace

cudaError_t launch_tc_gemm(TcOperand A, TcOperand B, int M, int N, int K, int splits, const TcEpi &epi, int *error,
                           cudaStream_t s, uint64_t *launches)
{
    if (N < 16 || N > 256 || N % 16 != 0 || M < 1 || K < 1 || splits < 1)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG_SMEM);
    if (e != cudaSuccess)
        return e;
    // 64-column tiles where N allows, for more CTAs on the small products of a training batch
    const int BN = N % 64 == 0 ? 64 : N;
    const int kchunk = ((K + splits - 1) / splits + TG_KC - 1) / TG_KC * TG_KC;
    const dim3 grid((M + 127) / 128, (N + BN - 1) / BN, (K + kchunk - 1) / kchunk);
    tc_gemm_kernel<<<grid, TG_THREADS, TG_SMEM, s>>>(A, B, M, N, BN, K, kchunk, epi, error);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_mlp_pack(const float *params, bf16 *w1p, bf16 *w2p, cudaStream_t s, uint64_t *launches)
{
    pack_kernel<<<96, 256, 0, s>>>(params, w1p, w2p);
    *launches += 1;
    return cudaGetLastError();
}

int launch_mlp_forward_tc(const bf16 *x, uint64_t n, const bf16 *w1p, const bf16 *w2p, const float *params, float *y,
                          int *error, cudaStream_t s, uint64_t *launches, std::string *why)
{
    if (n == 0)
        return 0;
    if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0) {
        *why = "feature rows must start on a 16-byte boundary";
        return 1;
    }
    EncodeTiled enc = encode_fn();
    if (!enc) {
        *why = "cuTensorMapEncodeTiled is not available from the driver";
        return 2;
    }
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)FEAT, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)FEAT * 2};
    const cuuint32_t box[2] = {8, (cuuint32_t)TM};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(x), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *why = "cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r);
        return 2;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) !=
        cudaSuccess) {
        *why = "cannot reserve shared memory for the tensor-core MLP";
        return 3;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t tiles = (n + TM - 1) / TM;
    const unsigned grid = (unsigned)(tiles < (uint64_t)sms ? tiles : (uint64_t)sms);
    mlp_forward_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(map, (uint32_t)n, w1p, w2p, params, y, error);
    *launches += 1;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *why = std::string("tensor-core MLP launch: ") + cudaGetErrorString(e);
        return 3;
    }
    return 0;
}

}  // namespace asse
