// gosma_eval_bounds: Theorem 1 bounds of a batch of sub-cubes.  A
// persistent grid (a few blocks per SM) walks the batch; each block handles
// one cube at a time with the per-cube core of bounds_core.cuh.
#include "bounds_core.cuh"

namespace gosma {

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) eval_bounds_kernel(MixDev mx, const gosma_cube *__restrict__ cubes, int n,
                                                            gosma_bound *__restrict__ out) {
    extern __shared__ float smem_f[];
    __shared__ CubeShared cs;
    __shared__ CubeSums sums;
    SmemArrays sm = carve(smem_f, mx.n1, mx.n2);
    for (int c = blockIdx.x; c < n; c += gridDim.x) {
        const gosma_cube &q = cubes[c];
        CubeGeom g;
        for (int k = 0; k < 3; ++k) {
            g.r0[k] = q.r0[k];
            g.t0[k] = q.t0[k];
            g.thw[k] = q.t_hw[k];
        }
        g.rhw = q.r_hw;
        cube_bounds<BLOCK>(mx, g, true, cs, sm, sums);
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
    if (work <= 1024) return 32;
    if (work <= 8192) return 64;
    if (n1 <= 256) return 128;
    return 256;
}

template <int BLOCK>
static int launch_t(gosma_ctx *ctx, const gosma_cube *d_cubes, int n, gosma_bound *d_out) {
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
    kern<<<(int)grid, BLOCK, smem, ctx->stream>>>(ctx->mix, d_cubes, n, d_out);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch(bounds)");
    return GOSMA_OK;
}

int launch_bounds(gosma_ctx *ctx, const gosma_cube *d_cubes, int n, gosma_bound *d_out) {
    if (n <= 0) return GOSMA_OK;
    switch (bounds_block_size(ctx->n1, ctx->n2)) {
    case 32: return launch_t<32>(ctx, d_cubes, n, d_out);
    case 64: return launch_t<64>(ctx, d_cubes, n, d_out);
    case 128: return launch_t<128>(ctx, d_cubes, n, d_out);
    default: return launch_t<256>(ctx, d_cubes, n, d_out);
    }
}

}  // namespace gosma
