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

}  // namespace asse
