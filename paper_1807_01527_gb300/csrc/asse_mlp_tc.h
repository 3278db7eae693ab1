// Launchers of the tensor-core (tcgen05) inference of the learned estimator.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

namespace asse {

// fp32 parameters (asse_learn.h order) -> the packed BF16 operand images of
// W1 (HID x FEAT) and W2 (HID x HID) that the tensor-core kernel copies into
// shared memory.
cudaError_t launch_mlp_pack(const float *params, __nv_bfloat16 *w1p, __nv_bfloat16 *w2p, cudaStream_t s,
                            uint64_t *launches);

// y[i] = model(x[i]) for n row-major BF16 feature rows (16-byte aligned).
// Returns 0 when launched, else nonzero with the reason in *why.  A wait in
// the kernel that gives up sets *error to 1.
int launch_mlp_forward_tc(const __nv_bfloat16 *x, uint64_t n, const __nv_bfloat16 *w1p, const __nv_bfloat16 *w2p,
                          const float *params, float *y, int *error, cudaStream_t s, uint64_t *launches,
                          std::string *why);

// Products of the training pass on the tensor cores (tcgen05):
// C[M][N] = sum_k A(m, k) B(n, k), operands addressed by strides (element
// (i, k) at p[i * si + k * sk]), N a multiple of 16 up to 256, the k range
// split over `splits` CTAs along z (only with TE_ATOMIC), and a fused
// epilogue:
//   TE_BIAS_RELU      out = bf16(relu(C + bias[n]))
//   TE_BIAS_RELU_DOT  the same (out may be null), and y[m] += sum_n out * w3[n]
//   TE_RELU_GRAD      out = bf16(C) where act > 0, else 0
//   TE_ATOMIC         outf[m][n] += C (FP32 atomics)
// with row stride ld.  A CTA whose bounded wait gave up sets *error to 1.
struct TcOperand {
    const __nv_bfloat16 *p;
    long si, sk;
};
enum { TE_BIAS_RELU = 0, TE_BIAS_RELU_DOT = 1, TE_RELU_GRAD = 2, TE_ATOMIC = 3 };
struct TcEpi {
    int kind;
    const float *bias;
    const float *w3;
    const __nv_bfloat16 *act;
    __nv_bfloat16 *out;
    float *outf;
    float *y;
    int ld;
};
cudaError_t launch_tc_gemm(TcOperand A, TcOperand B, int M, int N, int K, int splits, const TcEpi &epi, int *error,
                           cudaStream_t s, uint64_t *launches);

}  // namespace asse
