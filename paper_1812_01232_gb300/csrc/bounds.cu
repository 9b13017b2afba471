// gosma_eval_bounds: Theorem 1 bounds of a batch of sub-cubes.  A
// persistent grid (a few blocks per SM) walks the batch; each block handles
// one cube at a time with the per-cube core of bounds_core.cuh.  Cubes that
// share a translation cuboid share its self sums (computed once, by its
// owner, in a first pass).
#include "bounds_core.cuh"

namespace gosma {

// Pre-pass: one thread per cube.
__global__ void cube_prep_cubes(const gosma_cube *__restrict__ cubes, int n, CubePrep *__restrict__ prep, int point) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n)
        cube_prepare(cubes[c].r0, cubes[c].r_hw, cubes[c].t0, cubes[c].t_hw, prep[c],
                     point ? prep_point(prep, n, c) : nullptr);
}

// The self terms of Theorem 1 depend only on the translation cuboid, so
// within one call they are computed once per distinct cuboid: the cube with
// the smallest index among those sharing it (rotation-feasible ones first)
// owns it.  Cuboids are keyed by a 64-bit hash of their exact double-float
// centre and half-widths in an open-addressing table; a cube whose hash
// matches but whose cuboid differs computes its own self sums.
__device__ __forceinline__ unsigned long long cuboid_hash(const CubePrep &p) {
    unsigned long long h = 0x9e3779b97f4a7c15ULL;
    const float *f = p.th;  // th, tl, wh, wl: 12 consecutive floats
    for (int k = 0; k < 12; ++k) {
        h ^= (unsigned long long)__float_as_uint(f[k]) + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
        h *= 0xbf58476d1ce4e5b9ULL;
        h ^= h >> 31;
    }
    return h ? h : 1ULL;  // 0 marks an empty slot
}
__device__ __forceinline__ bool same_cuboid(const CubePrep &a, const CubePrep &b) {
    const float *fa = a.th, *fb = b.th;  // th, tl, wh, wl: 12 consecutive floats
    for (int k = 0; k < 12; ++k)
        if (__float_as_uint(fa[k]) != __float_as_uint(fb[k])) return false;
    return true;
}

// owner key: the cube index, plus 2^30 when the rotation cube is infeasible
__global__ void cuboid_insert(const CubePrep *__restrict__ prep, int n, unsigned long long *__restrict__ keys,
                              int *__restrict__ owners, int mask) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const unsigned long long h = cuboid_hash(prep[c]);
    const int ok = c + (prep[c].infeasible ? (1 << 30) : 0);
    int s = (int)(h & (unsigned long long)mask);
    for (int probe = 0; probe <= mask; ++probe) {  // the table has at least 2n slots
        const unsigned long long prev = atomicCAS(&keys[s], 0ULL, h);
        if (prev == 0ULL || prev == h) {
            atomicMin(&owners[s], ok);
            return;
        }
        s = (s + 1) & mask;
    }
}

// owner[c]: the cube whose self sums c takes (c itself when it owns them).
__global__ void cuboid_owner(const CubePrep *__restrict__ prep, int n, const unsigned long long *__restrict__ keys,
                             const int *__restrict__ owners, int mask, int *__restrict__ owner) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const unsigned long long h = cuboid_hash(prep[c]);
    int s = (int)(h & (unsigned long long)mask), o = c;
    for (int probe = 0; probe <= mask; ++probe) {
        const unsigned long long k = keys[s];
        if (k == h) {
            const int w = owners[s] & ((1 << 30) - 1);
            o = same_cuboid(prep[w], prep[c]) ? w : c;
            break;
        }
        if (k == 0ULL) break;  // not reached: c inserted its key on this path
        s = (s + 1) & mask;
    }
    owner[c] = o;
}

// pass 0: the cubes that own their self sums (or all cubes when owner is
// null); pass 1: the others, with the owner's self sums.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, bound_min_blocks<BLOCK>()) eval_bounds_kernel(MixDev mx, const gosma_cube *__restrict__ cubes, int n,
                                                            const CubePrep *__restrict__ prep, df zeta2,
                                                            gosma_bound *__restrict__ out, int *__restrict__ counter,
                                                            const int *__restrict__ owner, int pass) {
    extern __shared__ float smem_f[];
    __shared__ CubeShared cs;
    __shared__ CubeSums sums;
    __shared__ int slot;
    SmemArrays sm = carve(smem_f, mx.n1, mx.n2);
    for (int c = next_cube(counter, &slot); c < n; c = next_cube(counter, &slot)) {
        const int o = owner ? owner[c] : c;
        if ((o != c) != (pass == 1)) continue;  // block-uniform
        cube_bounds<BLOCK>(mx, prep[c], prep_point(prep, n, c), zeta2, o == c, cs, sm, sums);
        if (threadIdx.x == 0) {
            if (o != c) {  // written by the owner in pass 0
                sums.self_lb = out[o].self_lb;
                sums.self_c = out[o].self_c;
            }
            gosma_bound r;
            finish_bound(sums, r);
            out[c] = r;
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

// The per-cube pre-pass records (cube records, then the point-dependent
// ones) are followed by the work counter.
static size_t rot_counter_offset(int n) { return 2 * sizeof(CubePrep) * (size_t)n; }

template <int BLOCK>
static int launch_t(gosma_ctx *ctx, const gosma_cube *d_cubes, int n, gosma_bound *d_out, const CubePrep *d_rot,
                    const int *d_owner) {
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
    for (int pass = 0; pass < (d_owner ? 2 : 1); ++pass) {  // owners first, then the cubes sharing their cuboids
        e = cudaMemsetAsync(counter, 0, sizeof(int), ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "memset(bounds)");
        kern<<<(int)grid, BLOCK, smem, ctx->stream>>>(ctx->mix, d_cubes, n, d_rot, z2, d_out, counter, d_owner, pass);
        ++ctx->launches;
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "launch(bounds)");
    }
    return GOSMA_OK;
}

int launch_bounds(gosma_ctx *ctx, const gosma_cube *d_cubes, int n, gosma_bound *d_out) {
    if (n <= 0) return GOSMA_OK;
    // pre-pass records, work counter, then the cuboid table (2^k >= 2n slots:
    // keys, owner keys) and every cube's owner
    int H = 1;
    while (H < 2 * n) H <<= 1;
    const size_t o_keys = (rot_counter_offset(n) + 16 + 255) & ~(size_t)255;
    const size_t o_owners = o_keys + sizeof(unsigned long long) * (size_t)H;
    const size_t o_owner = o_owners + sizeof(int) * (size_t)H;
    size_t need = o_owner + sizeof(int) * (size_t)n;
    if (need > ctx->rot_bytes) {
        if (ctx->d_rot) cudaFree(ctx->d_rot);
        ctx->d_rot = nullptr;
        ctx->rot_bytes = 0;
        cudaError_t e = dev_malloc(ctx, &ctx->d_rot, need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(cube pre-pass)");
        ctx->rot_bytes = need;
    }
    CubePrep *rot = (CubePrep *)ctx->d_rot;
    cube_prep_cubes<<<(n + 127) / 128, 128, 0, ctx->stream>>>(d_cubes, n, rot, ctx->mix.psi_point);
    ++ctx->launches;
    char *base = (char *)ctx->d_rot;
    unsigned long long *keys = (unsigned long long *)(base + o_keys);
    int *owners = (int *)(base + o_owners), *owner = (int *)(base + o_owner);
    cudaError_t e = cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * (size_t)H, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(owners, 0x7f, sizeof(int) * (size_t)H, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "memset(cuboid table)");
    cuboid_insert<<<(n + 255) / 256, 256, 0, ctx->stream>>>(rot, n, keys, owners, H - 1);
    cuboid_owner<<<(n + 255) / 256, 256, 0, ctx->stream>>>(rot, n, keys, owners, H - 1, owner);
    ctx->launches += 2;
    switch (bounds_block_size(ctx->n1, ctx->n2)) {
    case 32: return launch_t<32>(ctx, d_cubes, n, d_out, rot, owner);
    case 64: return launch_t<64>(ctx, d_cubes, n, d_out, rot, owner);
    case 128: return launch_t<128>(ctx, d_cubes, n, d_out, rot, owner);
    case 256: return launch_t<256>(ctx, d_cubes, n, d_out, rot, owner);
    case 512: return launch_t<512>(ctx, d_cubes, n, d_out, rot, owner);
    default: return launch_t<1024>(ctx, d_cubes, n, d_out, rot, owner);
    }
}

}  // namespace gosma
