// Throughput of the pipes the bound kernel runs on, measured on the device:
// scalar FP32 fused multiply-add, packed FP32x2 fused multiply-add, and the
// approximate ex2, sqrt and rcp instructions of the multi-function unit.
// These are the denominators of the bound kernel's roofline (per SM and
// clock cycle), measured instead of taken from tables.
//
// Method: every thread runs eight independent dependency chains of one
// instruction kind (four packed chains for FP32x2) for PR_ITERS rounds, on
// 8 x 256 threads per SM, so that latency is hidden and the pipe saturates.
// CUDA events time the launch; lanes per SM per clock = lane operations /
// (seconds x SMs x the maximum SM clock).  The chains stay bounded
// (a -> a * c + d with |c| < 1, a -> 2^-a on [0, 1], a -> sqrt(a),
// a -> 1 / a) and their results are stored only under a flag that is never
// set, so that the compiler keeps every instruction.
#include "gosma_internal.cuh"
#include "packed.cuh"

namespace gosma {

constexpr int PR_ITERS = 2048;
constexpr int PR_THREADS = 256;
constexpr int PR_BLOCKS_PER_SM = 8;

template <int OP>
__global__ void __launch_bounds__(PR_THREADS) pipe_rate_kernel(float *sink, int store) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 0.5f + 0.01f * (float)k + 1e-6f * (float)(threadIdx.x & 31);
    if (OP == 1) {
        float2 p[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) p[k] = make_float2(a[2 * k], a[2 * k + 1]);
        const float2 c = bc2(0.999f), d = bc2(0.001f);
#pragma unroll 4
        for (int it = 0; it < PR_ITERS; ++it)
#pragma unroll
            for (int k = 0; k < 4; ++k) p[k] = fma2(p[k], c, d);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a[2 * k] = p[k].x;
            a[2 * k + 1] = p[k].y;
        }
    } else {
#pragma unroll 4
        for (int it = 0; it < PR_ITERS; ++it)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (OP == 0) a[k] = fmaf(a[k], 0.999f, 0.001f);
                if (OP == 2) a[k] = ex2a(-a[k]);
                if (OP == 3) a[k] = sqrta(a[k]);
                if (OP == 4) a[k] = rcpa(a[k]);
            }
    }
    if (store) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) s += a[k];
        sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    }
}

int selftest_pipe_rates(gosma_ctx *ctx, double rates[5], double *clock_mhz) {
    cudaSetDevice(ctx->device);
    int khz = 0;
    cudaError_t e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device);
    if (e != cudaSuccess || khz <= 0) return cuda_fail(ctx, e, "clock rate");
    const int grid = ctx->sm_count * PR_BLOCKS_PER_SM;
    float *sink = nullptr;
    e = dev_malloc(ctx, (void **)&sink, sizeof(float) * (size_t)grid * PR_THREADS);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(pipe rates)");
    cudaEvent_t ev[2];
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    void (*kern[5])(float *, int) = {pipe_rate_kernel<0>, pipe_rate_kernel<1>, pipe_rate_kernel<2>,
                                     pipe_rate_kernel<3>, pipe_rate_kernel<4>};
    for (int op = 0; op < 5 && e == cudaSuccess; ++op) {
        float best = 1e30f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
            cudaEventRecord(ev[0], ctx->stream);
            kern[op]<<<grid, PR_THREADS, 0, ctx->stream>>>(sink, 0);
            cudaEventRecord(ev[1], ctx->stream);
            ++ctx->launches;
            e = cudaEventSynchronize(ev[1]);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (rep > 0 && ms < best) best = ms;
        }
        const double lane_ops = (double)grid * PR_THREADS * PR_ITERS * 8.0;
        rates[op] = lane_ops / (best * 1e-3) / ((double)ctx->sm_count * khz * 1e3);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pipe rates");
    *clock_mhz = khz * 1e-3;
    return GOSMA_OK;
}

}  // namespace gosma

extern "C" int gosma_selftest_pipe_rates(gosma_ctx *ctx, double rates[5], double *clock_mhz) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (!rates || !clock_mhz) return gosma::fail(ctx, GOSMA_EINVAL, "selftest_pipe_rates: null output");
    return gosma::selftest_pipe_rates(ctx, rates, clock_mhz);
}
