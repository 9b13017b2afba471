// Throughput of the pipes the bound kernel runs on, measured on the device:
// scalar FP32 fused multiply-add, packed FP32x2 fused multiply-add, and the
// approximate ex2, sqrt, rcp, rsqrt and lg2 instructions of the
// multi-function unit.
// These are the denominators of the bound kernel's roofline (per SM and
// clock cycle), measured instead of taken from tables.
//
// Method: every thread runs eight independent dependency chains of one
// instruction kind (four packed chains for FP32x2) for PR_ITERS rounds, on
// 8 x 256 threads per SM, so that latency is hidden and the pipe saturates.
// CUDA events time the launch; lanes per SM per clock = lane operations /
// (seconds x SMs x the maximum SM clock).  The chains stay bounded
// (a -> a * c + d with |c| < 1, a -> 2^-a on [0, 1], a -> sqrt(a),
// a -> 1 / (a + 0.5), a -> 1 / sqrt(a), a -> lg2(a + 1.5)) and their results are
// stored only under a flag that is never set; the approximate instructions
// are volatile, so that the compiler keeps every one.
#include "bounds_core.cuh"
#include "gosma_internal.cuh"
#include "packed.cuh"

namespace gosma {

// Volatile forms of the approximate instructions: a chain such as
// a -> rcp(a) would otherwise be folded by the compiler.
__device__ __forceinline__ float ex2v(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrtv(float x) {
    float y;
    asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcpv(float x) {
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrtv(float x) {
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2v(float x) {
    float y;
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr int PR_ITERS = 2048;
constexpr int PR_OPS = 7;
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
                if (OP == 2) a[k] = ex2v(-a[k]);
                if (OP == 3) a[k] = sqrtv(a[k]);
                if (OP == 4) a[k] = rcpv(a[k] + 0.5f);  // one FP32 add beside each rcp (rcp(rcp(a)) folds)
                if (OP == 5) a[k] = rsqrtv(a[k]);   // a -> 1/sqrt(a): bounded, 1 is its fixed point
                if (OP == 6) a[k] = lg2v(a[k] + 1.5f);  // one FP32 add beside each lg2
            }
    }
    if (store) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) s += a[k];
        sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    }
}

int selftest_pipe_rates(gosma_ctx *ctx, double rates[PR_OPS], double *clock_mhz) {
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
    void (*kern[PR_OPS])(float *, int) = {pipe_rate_kernel<0>, pipe_rate_kernel<1>, pipe_rate_kernel<2>,
                                          pipe_rate_kernel<3>, pipe_rate_kernel<4>, pipe_rate_kernel<5>,
                                          pipe_rate_kernel<6>};
    for (int op = 0; op < PR_OPS && e == cudaSuccess; ++op) {
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

// The pre-pass's rotation matrices (hi + lo of each entry, in FP64) for n
// rotation vectors, one thread each.
__global__ void rodrigues_probe(int n, const double *__restrict__ r, double *__restrict__ R) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r0[3] = {r[3 * i], r[3 * i + 1], r[3 * i + 2]};
    float h[9], l[9];
    rodrigues_df(r0, h, l);
    for (int k = 0; k < 9; ++k) R[9 * (size_t)i + k] = (double)h[k] + (double)l[k];
}

int selftest_rodrigues(gosma_ctx *ctx, int n, const double *h_r, double *h_R) {
    cudaSetDevice(ctx->device);
    double *d = nullptr;
    cudaError_t e = dev_malloc(ctx, (void **)&d, sizeof(double) * 12 * (size_t)n);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(rodrigues)");
    double *dR = d + 3 * (size_t)n;
    e = cudaMemcpyAsync(d, h_r, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        rodrigues_probe<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, d, dR);
        ++ctx->launches;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_R, dR, sizeof(double) * 9 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    return e == cudaSuccess ? GOSMA_OK : cuda_fail(ctx, e, "rodrigues");
}

}  // namespace gosma

extern "C" int gosma_selftest_rodrigues(gosma_ctx *ctx, int n, const double *r, double *R) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (n < 0 || (n > 0 && (!r || !R))) return gosma::fail(ctx, GOSMA_EINVAL, "selftest_rodrigues: bad arguments");
    if (n == 0) return GOSMA_OK;
    return gosma::selftest_rodrigues(ctx, n, r, R);
}

extern "C" int gosma_selftest_pipe_rates(gosma_ctx *ctx, double rates[7], double *clock_mhz) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (!rates || !clock_mhz) return gosma::fail(ctx, GOSMA_EINVAL, "selftest_pipe_rates: null output");
    return gosma::selftest_pipe_rates(ctx, rates, clock_mhz);
}
