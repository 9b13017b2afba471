// gosma_eval_bounds: Theorem 1 bounds of a batch of sub-cubes.  A
// persistent grid (a few blocks per SM) walks the batch; each block handles
// one cube at a time with the per-cube core of bounds_core.cuh.
#include "bounds_core.cuh"

namespace gosma {

// Pre-pass: one thread per cube.
__global__ void cube_prep_cubes(const gosma_cube *__restrict__ cubes, int n, CubePrep *__restrict__ prep) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) cube_prepare(cubes[c].r0, cubes[c].r_hw, cubes[c].t0, cubes[c].t_hw, prep[c]);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) eval_bounds_kernel(MixDev mx, const gosma_cube *__restrict__ cubes, int n,
                                                            const CubePrep *__restrict__ prep, df zeta2,
                                                            gosma_bound *__restrict__ out, int *__restrict__ counter) {
    extern __shared__ float smem_f[];
    __shared__ CubeShared cs;
    __shared__ CubeSums sums;
    __shared__ int slot;
    SmemArrays sm = carve(smem_f, mx.n1, mx.n2);
    for (int c = next_cube(counter, &slot); c < n; c = next_cube(counter, &slot)) {
        cube_bounds<BLOCK>(mx, prep[c], zeta2, true, cs, sm, sums);
        if (threadIdx.x == 0) {
            gosma_bound o;
            finish_bound(sums, o);
            out[c] = o;
        }
    }
}

size_t bounds_smem_bytes(int n1, int n2) { return bounds_smem_arrays_bytes(n1, n2); }

// Threads per cube: enough to give every thread a few model rows.
int bounds_block_size(int n1, int n2) {
    long long work = (long long)n1 * n2 + (long long)n1 * (n1 - 1) / 2;
    int b;
    if (work <= 1024) b = 32;
    else if (work <= 8192) b = 64;
    else if (n1 <= 256) b = 128;
    else b = 256;
    // Large mixtures leave room for few blocks per SM in shared memory: widen
    // the block (up to one thread per model row, at most 1024) until 32 warps
    // per SM can hide the latencies.
    const long long per_sm = (227LL * 1024) / (long long)(bounds_smem_bytes(n1, n2) + sizeof(CubeShared) + 1024);
    while (b < 1024 && b < n1 && per_sm * b < 1024) b *= 2;
    return b;
}

// The per-cube pre-pass records are followed by the work counter.
static size_t rot_counter_offset(int n) { return sizeof(CubePrep) * (size_t)n; }

template <int BLOCK>
static int launch_t(gosma_ctx *ctx, const gosma_cube *d_cubes, int n, gosma_bound *d_out, const CubePrep *d_rot) {
    size_t smem = bounds_smem_bytes(ctx->n1, ctx->n2);
    auto kern = eval_bounds_kernel<BLOCK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute(bounds)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occupancy(bounds)");
    if (per_sm < 1) return fail(ctx, GOSMA_EINVAL, "mixtures too large for one thread block's shared memory");
    long long grid = (long long)ctx->sm_count * per_sm;
    if (grid > n) grid = n;
    df z2;
    split_double(ctx->zeta * ctx->zeta, z2.h, z2.l);
    int *counter = (int *)((char *)ctx->d_rot + rot_counter_offset(n));
    e = cudaMemsetAsync(counter, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "memset(bounds)");
    kern<<<(int)grid, BLOCK, smem, ctx->stream>>>(ctx->mix, d_cubes, n, d_rot, z2, d_out, counter);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch(bounds)");
    return GOSMA_OK;
}

int launch_bounds(gosma_ctx *ctx, const gosma_cube *d_cubes, int n, gosma_bound *d_out) {
    if (n <= 0) return GOSMA_OK;
    size_t need = rot_counter_offset(n) + 16;
    if (need > ctx->rot_bytes) {
        if (ctx->d_rot) cudaFree(ctx->d_rot);
        ctx->d_rot = nullptr;
        ctx->rot_bytes = 0;
        cudaError_t e = dev_malloc(ctx, &ctx->d_rot, need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(cube pre-pass)");
        ctx->rot_bytes = need;
    }
    CubePrep *rot = (CubePrep *)ctx->d_rot;
    cube_prep_cubes<<<(n + 127) / 128, 128, 0, ctx->stream>>>(d_cubes, n, rot);
    ++ctx->launches;
    switch (bounds_block_size(ctx->n1, ctx->n2)) {
    case 32: return launch_t<32>(ctx, d_cubes, n, d_out, rot);
    case 64: return launch_t<64>(ctx, d_cubes, n, d_out, rot);
    case 128: return launch_t<128>(ctx, d_cubes, n, d_out, rot);
    case 256: return launch_t<256>(ctx, d_cubes, n, d_out, rot);
    case 512: return launch_t<512>(ctx, d_cubes, n, d_out, rot);
    default: return launch_t<1024>(ctx, d_cubes, n, d_out, rot);
    }
}

}  // namespace gosma
