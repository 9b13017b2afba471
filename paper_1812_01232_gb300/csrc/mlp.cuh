// Internal interface of the queue-ordering network (mlp.cu) for the batched
// solver: inputs are staged by the caller into the network's BF16 input rows,
// and the forward pass reads its row count from device memory so that it can
// run inside a captured CUDA graph.
#pragma once

#include "gosma_internal.cuh"
#include "tc_gemm.cuh"

namespace gosma {

constexpr int MLP_IN = 16, MLP_HID = 128, MLP_OUT = 16, MLP_SEED = 6;

// Activation buffers for at least `rows` rows (call outside stream capture).
int mlp_reserve(gosma_ctx *ctx, int rows);
bf16 *mlp_input(Mlp *m);         // rows x 16, BF16
const float *mlp_output(Mlp *m);  // rows x 16, FP32
int *mlp_error_flag(Mlp *m);
// Inference over min(*d_rows, max_rows) staged rows; no training outputs.
cudaError_t mlp_forward_rows(gosma_ctx *ctx, int max_rows, const int *d_rows, cudaStream_t st);

}  // namespace gosma
