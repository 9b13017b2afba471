// Mixture generation (Sec. 6) on the device: DP-means over the model's 3D
// points and DP-vMF-means over the image's bearing vectors, then the
// maximum-likelihood GMM / vMFMM fitted to the clusters, the inputs of
// gosma_set_mixtures.
//
// A pass of either algorithm visits the points in index order and a point
// that is farther than lambda from every centre (squared distance; for
// directions: cosine below lambda) opens a new cluster that the later points
// of the pass see.  The device reproduces that order exactly without a
// serial walk: every point first takes its nearest centre of the previous
// pass (one grid-wide step); then, one round per new cluster, the first point
// past the cursor that still exceeds lambda is found by a grid-wide minimum
// over point indices, it opens the cluster, and the points after it compare
// themselves with the new centre.  One cooperative persistent kernel runs all
// passes with grid barriers between the steps.
//
// Exactness: coordinates are rounded to multiples of 2^-32 (points) or 2^-40
// (unit vectors) so that cluster sums are exact 64-bit integer atomics, and
// every decision (nearest centre, a new centre beating the current one,
// opening a cluster) compares distances or cosines formed with explicitly
// rounded FP64 operations (no contraction), so labels and centres equal those
// of a serial FP64 implementation of the same steps bit for bit.  GB300 runs
// FP64 at about 1/64 of its FP32 rate, so the candidates are screened in
// FP32 first: with every coordinate of points and centres at most A in
// magnitude, an FP32 squared distance is within E = 128 u A^2 of the FP64
// one (u = 2^-24; the sum of (|x_k| + |m_k|)^2 is at most 12 A^2 and each
// term carries at most 8u), an FP32 cosine of unit vectors within 8u; only
// centres whose FP32 value is within 2E of the best FP32 value (nearest
// centre) or within E of beating the exact current best (new centre) are
// evaluated in FP64.  The exact winner is always among them.
#include <cooperative_groups.h>
#include <math.h>

#include "gosma_internal.cuh"

namespace gosma {
namespace cg = cooperative_groups;

constexpr int MG_BLOCK = 256;
constexpr int MG_NONE = 0x7fffffff;
constexpr int MG_KMAX = 8192;

// Grid-wide state of the clustering kernel (device memory).
struct MgState {
    int K;           // centres after the last pass
    int next[3];     // first point that opens a cluster in round r: next[r % 3]
    int changed[2];  // labels changed in a pass (by pass parity)
    int passes;      // passes run
    int overflow;    // more than kmax clusters would be needed
};

// Squared distance (DP-means) or cosine (DP-vMF-means), each product and sum
// rounded once: ((a0 b0 + a1 b1) + a2 b2).
template <bool VMF>
__device__ __forceinline__ double mg_score(const double *x, const double *m) {
    if (VMF) return __dadd_rn(__dadd_rn(__dmul_rn(x[0], m[0]), __dmul_rn(x[1], m[1])), __dmul_rn(x[2], m[2]));
    const double d0 = __dsub_rn(x[0], m[0]), d1 = __dsub_rn(x[1], m[1]), d2 = __dsub_rn(x[2], m[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
}
template <bool VMF>
__device__ __forceinline__ bool mg_better(double a, double b) {
    return VMF ? a > b : a < b;
}
template <bool VMF>
__device__ __forceinline__ bool mg_opens(double best, double lam) {
    return VMF ? best < lam : best > lam;
}

// Centre of a cluster from its exact integer coordinate sum S and count n:
// the mean ((double)S / n) 2^-32, or the direction S / |S| (the cluster's
// lowest-index point xf when the sum is exactly zero).
template <bool VMF>
__device__ void mg_centre(const unsigned long long *S, unsigned long long n, const double *xf, double *m) {
    const double s0 = __ll2double_rn((long long)S[0]), s1 = __ll2double_rn((long long)S[1]),
                 s2 = __ll2double_rn((long long)S[2]);
    if (!VMF) {
        const double dn = __ull2double_rn(n);
        m[0] = __dmul_rn(__ddiv_rn(s0, dn), 0x1p-32);
        m[1] = __dmul_rn(__ddiv_rn(s1, dn), 0x1p-32);
        m[2] = __dmul_rn(__ddiv_rn(s2, dn), 0x1p-32);
        return;
    }
    const double nr = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(s0, s0), __dmul_rn(s1, s1)), __dmul_rn(s2, s2)));
    if (nr == 0.0) {
        m[0] = xf[0];
        m[1] = xf[1];
        m[2] = xf[2];
        return;
    }
    m[0] = __ddiv_rn(s0, nr);
    m[1] = __ddiv_rn(s1, nr);
    m[2] = __ddiv_rn(s2, nr);
}

// Quantized coordinates: q = round-to-nearest-even(x 2^s), xq = q 2^-s.
__global__ void mg_quantize(int n3, const double *__restrict__ x, double scale, long long *__restrict__ q,
                            double *__restrict__ xq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const long long v = __double2ll_rn(__dmul_rn(x[i], scale));
    q[i] = v;
    xq[i] = __ddiv_rn(__ll2double_rn(v), scale);
}

// FP32 copies of the quantized points for the screening.
__global__ void mg_pack(int n, const double *__restrict__ xq, float4 *__restrict__ xf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) xf[i] = make_float4((float)xq[3 * i], (float)xq[3 * i + 1], (float)xq[3 * i + 2], 0.f);
}

// FP32 screening value (squared distance or cosine).
template <bool VMF>
__device__ __forceinline__ float mg_score32(float4 x, float4 m) {
    if (VMF) return fmaf(x.z, m.z, fmaf(x.y, m.y, x.x * m.x));
    const float d0 = x.x - m.x, d1 = x.y - m.y, d2 = x.z - m.z;
    return fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
}

__global__ void mg_fill(int count, int value, int *__restrict__ a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) a[i] = value;
}

// Block-wide minimum of an int / sum of a long long (every thread calls;
// thread 0 gets the result).
__device__ __forceinline__ int mg_block_min(int v, int *sred) {
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < MG_BLOCK / 32; ++w) v = min(v, sred[w]);
    __syncthreads();
    return v;
}
__device__ __forceinline__ long long mg_block_sum(long long v, long long *sred) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < MG_BLOCK / 32; ++w) v += sred[w];
    __syncthreads();
    return v;
}

// The clustering passes.  Block b owns the contiguous points [i0, i1).
// best / arg are block-owned; cen, sums, cnt, first, remap and the state are
// shared across blocks (read with __ldcg after a grid barrier).  Every branch
// that leads to a grid barrier depends only on values all blocks read alike,
// so every block runs the same barriers.  All loops are bounded: max_iter
// passes, at most kmax rounds per pass.
template <bool VMF>
__global__ void __launch_bounds__(MG_BLOCK) mg_cluster(int n, const double *__restrict__ xq,
                                                       const long long *__restrict__ q,
                                                       const float4 *__restrict__ xf, float E, double lam, int max_iter,
                                                       int kmax, double *cen, int *lab, double *best, float *bestf,
                                                       int *arg,
                                                       unsigned long long *sums, unsigned long long *cnt, int *first,
                                                       int *remap, MgState *S) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ float4 scf[];  // FP32 copies of the previous pass's centres, kmax
    __shared__ int sred_i[MG_BLOCK / 32];
    __shared__ long long sred_l[MG_BLOCK / 32];
    const int tid = threadIdx.x, b = blockIdx.x, nb = gridDim.x;
    const int chunk = (n + nb - 1) / nb, i0 = min(n, b * chunk), i1 = min(n, i0 + chunk);
    const bool lead = b == 0 && tid == 0;

    // start: one cluster at the mean (mean direction) of all points
    long long s3[3] = {0, 0, 0};
    for (int i = i0 + tid; i < i1; i += MG_BLOCK) {
        lab[i] = 0;
        for (int k = 0; k < 3; ++k) s3[k] += q[3 * i + k];
    }
    for (int k = 0; k < 3; ++k) {
        const long long v = mg_block_sum(s3[k], sred_l);
        if (tid == 0 && i1 > i0) atomicAdd(&sums[k], (unsigned long long)v);
    }
    grid.sync();
    if (lead) {
        unsigned long long s[3] = {__ldcg(&sums[0]), __ldcg(&sums[1]), __ldcg(&sums[2])};
        mg_centre<VMF>(s, (unsigned long long)n, xq, cen);
        sums[0] = sums[1] = sums[2] = 0;
        S->K = 1;
        S->next[0] = S->next[1] = S->next[2] = MG_NONE;
        S->changed[0] = S->changed[1] = 0;
        S->overflow = 0;
    }
    grid.sync();

    int pass = 0;
    for (; pass < max_iter; ++pass) {
        // 1. every point's nearest centre of the previous pass
        const int K0 = __ldcg(&S->K);
        for (int c = tid; c < K0; c += MG_BLOCK)
            scf[c] = make_float4((float)__ldcg(&cen[3 * c]), (float)__ldcg(&cen[3 * c + 1]),
                                 (float)__ldcg(&cen[3 * c + 2]), 0.f);
        __syncthreads();
        for (int i = i0 + tid; i < i1; i += MG_BLOCK) {
            const float4 xv = xf[i];
            float b32 = mg_score32<VMF>(xv, scf[0]);
            for (int c = 1; c < K0; ++c) {
                const float s = mg_score32<VMF>(xv, scf[c]);
                b32 = VMF ? fmaxf(b32, s) : fminf(b32, s);
            }
            // 2E, and E/4 for the rounding of the limit itself
            const float lim = VMF ? b32 - 2.25f * E : b32 + 2.25f * E;
            const double *x = xq + 3 * i;
            double bv = 0.0;
            int a = -1;
            for (int c = 0; c < K0; ++c) {
                const float s32 = mg_score32<VMF>(xv, scf[c]);
                if (VMF ? s32 < lim : s32 > lim) continue;
                const double m[3] = {__ldcg(&cen[3 * c]), __ldcg(&cen[3 * c + 1]), __ldcg(&cen[3 * c + 2])};
                const double s = mg_score<VMF>(x, m);
                if (a < 0 || mg_better<VMF>(s, bv)) {
                    bv = s;
                    a = c;
                }
            }
            best[i] = bv;
            bestf[i] = (float)bv;
            arg[i] = a;
        }
        grid.sync();
        // every block has read changed[(pass + 1) & 1] at the end of the last pass
        if (lead) S->changed[(pass + 1) & 1] = 0;

        // 2. one round per new cluster, in point order
        int cursor = 0, r = 0;
        bool over = false;
        for (;;) {
            int loc = MG_NONE;
            for (int i = max(i0, cursor) + tid; i < i1; i += MG_BLOCK)
                if (mg_opens<VMF>(best[i], lam)) {
                    loc = i;
                    break;
                }
            const int bmin = mg_block_min(loc, sred_i);
            if (tid == 0 && bmin != MG_NONE) atomicMin(&S->next[r % 3], bmin);
            // next[(r + 1) % 3] was last read in round r - 2, before the
            // barrier of round r - 1; its next writers come after this barrier
            if (lead) S->next[(r + 1) % 3] = MG_NONE;
            grid.sync();
            const int istar = __ldcg(&S->next[r % 3]);
            if (istar == MG_NONE) break;
            const int c = K0 + r;
            if (c >= kmax) {
                over = true;
                break;
            }
            if (lead)
                for (int k = 0; k < 3; ++k) cen[3 * c + k] = xq[3 * istar + k];
            const double *m = xq + 3 * istar;
            const float4 mv = xf[istar];
            for (int i = max(i0, istar) + tid; i < i1; i += MG_BLOCK) {
                if (i == istar) {
                    arg[i] = c;
                    continue;
                }
                // cannot beat the current centre: FP32 test with 1.25 E (rounding
                // bestf and the difference each costs less than E / 10)
                const float s32 = mg_score32<VMF>(xf[i], mv), bf = bestf[i];
                if (VMF ? s32 + 1.25f * E <= bf : s32 - 1.25f * E >= bf) continue;
                const double s = mg_score<VMF>(xq + 3 * i, m);
                if (mg_better<VMF>(s, best[i])) {
                    best[i] = s;
                    bestf[i] = (float)s;
                    arg[i] = c;
                }
            }
            __syncthreads();
            cursor = istar + 1;
            ++r;
        }
        if (over) {
            if (lead) S->overflow = 1;
            break;
        }
        const int K = K0 + r;
        // the rounds' reads are done except that of the last buffer, which
        // holds MG_NONE already; the next pass starts from next[0]
        if (lead) S->next[0] = S->next[1] = S->next[2] = MG_NONE;

        // 3. labels, exact cluster sums, counts, lowest members
        long long ch = 0;
        for (int i = i0 + tid; i < i1; i += MG_BLOCK) {
            const int a = arg[i];
            for (int k = 0; k < 3; ++k) atomicAdd(&sums[3 * a + k], (unsigned long long)q[3 * i + k]);
            atomicAdd(&cnt[a], 1ULL);
            atomicMin(&first[a], i);
            ch += a != lab[i];
            lab[i] = a;
        }
        ch = mg_block_sum(ch, sred_l);
        if (tid == 0 && ch) atomicAdd(&S->changed[pass & 1], (int)ch);
        grid.sync();

        // 4. block 0: centres become the means; empty clusters are removed
        if (b == 0) {
            if (tid == 0) {
                int kn = 0;
                for (int c = 0; c < K; ++c) remap[c] = __ldcg(&cnt[c]) ? kn++ : -1;
                S->K = kn;
            }
            __syncthreads();
            for (int c = tid; c < K; c += MG_BLOCK) {
                const int j = __ldcg(&remap[c]);
                if (j < 0) continue;
                unsigned long long s[3] = {__ldcg(&sums[3 * c]), __ldcg(&sums[3 * c + 1]), __ldcg(&sums[3 * c + 2])};
                mg_centre<VMF>(s, __ldcg(&cnt[c]), xq + 3 * __ldcg(&first[c]), cen + 3 * j);
            }
            __syncthreads();
            for (int c = tid; c < K; c += MG_BLOCK) {
                sums[3 * c] = sums[3 * c + 1] = sums[3 * c + 2] = 0;
                cnt[c] = 0;
                first[c] = n;
            }
        }
        grid.sync();
        const int kn = __ldcg(&S->K);
        if (kn < K)
            for (int i = i0 + tid; i < i1; i += MG_BLOCK) lab[i] = __ldcg(&remap[lab[i]]);
        if (__ldcg(&S->changed[pass & 1]) == 0) {
            ++pass;
            break;
        }
    }
    if (lead) S->passes = pass;
}

// Maximum-likelihood fits (reading M3): exact sums, counts and (GMM) the
// squared distances to the centres per final cluster ...
template <bool VMF>
__global__ void mg_fit_sums(int n, const double *__restrict__ xq, const long long *__restrict__ q,
                            const int *__restrict__ lab, const double *__restrict__ cen,
                            unsigned long long *__restrict__ sums, unsigned long long *__restrict__ cnt,
                            double *__restrict__ ss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = lab[i];
    for (int k = 0; k < 3; ++k) atomicAdd(&sums[3 * a + k], (unsigned long long)q[3 * i + k]);
    atomicAdd(&cnt[a], 1ULL);
    if (!VMF) atomicAdd(&ss[a], mg_score<false>(xq + 3 * i, cen + 3 * a));
}

// coth(k) - 1/k: the mean resultant length of a vMF on S^2.
__device__ __forceinline__ double mg_A3(double k) {
    if (k < 1e-3) return k / 3.0 - k * k * k / 45.0;
    return 1.0 / tanh(k) - 1.0 / k;
}

// ... then weights n_k / N and sigma = max(sqrt(ss / 3 n_k), lo) (GMM) or the
// kappa solving coth k - 1/k = |S| / (2^40 n_k), by 200 bisections of log
// kappa on [1e-12, hi] (hi when even that is not enough).
template <bool VMF>
__global__ void mg_fit_final(int K, int n, const unsigned long long *__restrict__ sums,
                             const unsigned long long *__restrict__ cnt, const double *__restrict__ ss, double lo,
                             double hi, double *__restrict__ spread, double *__restrict__ phi) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    const double nc = __ull2double_rn(cnt[c]);
    phi[c] = nc / (double)n;
    if (!VMF) {
        const double s = sqrt(ss[c] / (3.0 * nc));
        spread[c] = s > lo ? s : lo;
        return;
    }
    const double s0 = __ll2double_rn((long long)sums[3 * c]), s1 = __ll2double_rn((long long)sums[3 * c + 1]),
                 s2 = __ll2double_rn((long long)sums[3 * c + 2]);
    const double rbar = sqrt((s0 * s0 + s1 * s1) + s2 * s2) / (0x1p40 * nc);
    if (!(mg_A3(hi) > rbar)) {
        spread[c] = hi;
        return;
    }
    double a = log(1e-12), b = log(hi);
    for (int it = 0; it < 200; ++it) {
        const double m = 0.5 * (a + b);
        if (mg_A3(exp(m)) < rbar) a = m;
        else b = m;
    }
    spread[c] = exp(0.5 * (a + b));
}

template <bool VMF>
static int mg_run(gosma_ctx *ctx, int n, const double *h_x, double lam, int max_iter, int kmax, double lo, double hi,
                  int *k_out, double *mu, double *spread, double *phi, int *labels, int *passes) {
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_x = al(sizeof(double) * 3 * (size_t)n), b_q = al(sizeof(long long) * 3 * (size_t)n),
                 b_xf = al(sizeof(float4) * (size_t)n),
                 b_n = al(sizeof(int) * (size_t)n), b_best = al(sizeof(double) * (size_t)n),
                 b_bestf = al(sizeof(float) * (size_t)n),
                 b_cen = al(sizeof(double) * 3 * (size_t)kmax), b_sums = al(sizeof(unsigned long long) * 3 * (size_t)kmax),
                 b_k = al(sizeof(unsigned long long) * (size_t)kmax), b_ki = al(sizeof(int) * (size_t)kmax),
                 b_kd = al(sizeof(double) * (size_t)kmax), b_st = al(sizeof(MgState));
    // x, xq, q, xf, lab, arg, best, cen, sums, cnt, first, remap, ss, spread, phi, state
    const size_t need = 2 * b_x + b_q + b_xf + 2 * b_n + b_best + b_bestf + b_cen + b_sums + b_k + 2 * b_ki + 3 * b_kd + b_st;
    if (need > ctx->mg_bytes) {
        if (ctx->d_mg) cudaFree(ctx->d_mg);
        ctx->d_mg = nullptr;
        ctx->mg_bytes = 0;
        e = dev_malloc(ctx, &ctx->d_mg, need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(mixture generation)");
        ctx->mg_bytes = need;
    }
    char *p = (char *)ctx->d_mg;
    double *d_x = (double *)p;
    p += b_x;
    double *d_xq = (double *)p;
    p += b_x;
    long long *d_q = (long long *)p;
    p += b_q;
    float4 *d_xf = (float4 *)p;
    p += b_xf;
    int *d_lab = (int *)p;
    p += b_n;
    int *d_arg = (int *)p;
    p += b_n;
    double *d_best = (double *)p;
    p += b_best;
    float *d_bestf = (float *)p;
    p += b_bestf;
    double *d_cen = (double *)p;
    p += b_cen;
    unsigned long long *d_sums = (unsigned long long *)p;
    p += b_sums;
    unsigned long long *d_cnt = (unsigned long long *)p;
    p += b_k;
    int *d_first = (int *)p;
    p += b_ki;
    int *d_remap = (int *)p;
    p += b_ki;
    double *d_ss = (double *)p;
    p += b_kd;
    double *d_spread = (double *)p;
    p += b_kd;
    double *d_phi = (double *)p;
    p += b_kd;
    MgState *d_st = (MgState *)p;

    cudaStream_t st = ctx->stream;
    const double scale = VMF ? 0x1p40 : 0x1p32;
    e = cudaMemcpyAsync(d_x, h_x, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_sums, 0, b_sums, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, b_k, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_st, 0, sizeof(MgState), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mixture generation set-up");
    mg_quantize<<<(3 * n + 255) / 256, 256, 0, st>>>(3 * n, d_x, scale, d_q, d_xq);
    mg_pack<<<(n + 255) / 256, 256, 0, st>>>(n, d_xq, d_xf);
    mg_fill<<<(kmax + 255) / 256, 256, 0, st>>>(kmax, n, d_first);
    ctx->launches += 3;
    // FP32 screening bound (see the top of the file): 128 u A^2, A the
    // largest coordinate magnitude (2^-32 above the input's for the
    // rounding); 8 u for unit vectors
    double A = 0.0;
    for (long long i = 0; i < 3LL * n; ++i) A = fmax(A, fabs(h_x[i]));
    A += 0x1p-32;
    float E = VMF ? (float)(8.0 * 0x1p-24) : (float)(128.0 * 0x1p-24 * A * A);

    auto kern = mg_cluster<VMF>;
    const size_t smem = sizeof(float4) * (size_t)kmax;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute(mixture generation)");
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, MG_BLOCK, smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "occupancy(mixture generation)");
    if (per_sm < 1) return fail(ctx, GOSMA_EINVAL, "mixture generation: kmax too large for one block");
    int grid = ctx->sm_count * per_sm, need_blocks = (n + MG_BLOCK - 1) / MG_BLOCK;
    if (grid > need_blocks) grid = need_blocks;
    void *args[] = {(void *)&n,      (void *)&d_xq,  (void *)&d_q,   (void *)&d_xf,    (void *)&E,
                    (void *)&lam,    (void *)&max_iter,
                    (void *)&kmax,   (void *)&d_cen, (void *)&d_lab, (void *)&d_best,  (void *)&d_bestf,
                    (void *)&d_arg,
                    (void *)&d_sums, (void *)&d_cnt, (void *)&d_first, (void *)&d_remap, (void *)&d_st};
    e = cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(MG_BLOCK), args, smem, st);
    ++ctx->launches;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch(mixture generation)");
    MgState hs;
    e = cudaMemcpyAsync(&hs, d_st, sizeof hs, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mixture generation");
    if (passes) *passes = hs.passes;
    if (hs.overflow) {
        *k_out = -1;
        return fail(ctx, GOSMA_EINVAL, "mixture generation: more than kmax clusters would be needed");
    }
    const int K = hs.K;
    *k_out = K;
    e = cudaMemsetAsync(d_sums, 0, b_sums, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, b_k, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ss, 0, b_kd, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "memset(fit)");
    mg_fit_sums<VMF><<<(n + 255) / 256, 256, 0, st>>>(n, d_xq, d_q, d_lab, d_cen, d_sums, d_cnt, d_ss);
    mg_fit_final<VMF><<<(K + 127) / 128, 128, 0, st>>>(K, n, d_sums, d_cnt, d_ss, lo, hi, d_spread, d_phi);
    ctx->launches += 2;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(mu, d_cen, sizeof(double) * 3 * (size_t)K, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(spread, d_spread, sizeof(double) * (size_t)K, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(phi, d_phi, sizeof(double) * (size_t)K, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && labels)
        e = cudaMemcpyAsync(labels, d_lab, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mixture generation results");
    return GOSMA_OK;
}

}  // namespace gosma

using namespace gosma;

static int mg_check(gosma_ctx *ctx, int n, const double *x, int max_iter, int kmax, int *k, double *mu, double *spread,
                    double *phi) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (n < 1 || !x) return fail(ctx, GOSMA_EINVAL, "mixture generation: need n >= 1 points");
    if (n > (1 << 26)) return fail(ctx, GOSMA_EINVAL, "mixture generation: at most 2^26 points");  // 32-bit indexing
    if (max_iter < 1) return fail(ctx, GOSMA_EINVAL, "mixture generation: max_iter must be >= 1");
    if (kmax < 1 || kmax > MG_KMAX) return fail(ctx, GOSMA_EINVAL, "mixture generation: kmax must be in [1, 8192]");
    if (!k || !mu || !spread || !phi) return fail(ctx, GOSMA_EINVAL, "mixture generation: null output");
    return GOSMA_OK;
}

extern "C" int gosma_dp_means(gosma_ctx *ctx, int n, const double *x, double lambda, int max_iter, int kmax,
                              double sigma_min, int *k, double *mu, double *sigma, double *phi, int *labels,
                              int *passes) {
    int rc = mg_check(ctx, n, x, max_iter, kmax, k, mu, sigma, phi);
    if (rc) return rc;
    if (!(lambda > 0) || !isfinite(lambda)) return fail(ctx, GOSMA_EINVAL, "dp_means: lambda must be > 0");
    if (!(sigma_min > 0)) return fail(ctx, GOSMA_EINVAL, "dp_means: sigma_min must be > 0");
    double amax = 0;
    for (long long i = 0; i < 3LL * n; ++i) {
        if (!isfinite(x[i])) return fail(ctx, GOSMA_EINVAL, "dp_means: non-finite coordinate");
        amax = fmax(amax, fabs(x[i]));
    }
    // exact sums: n |x| 2^32 < 2^62
    if (amax * (double)n >= 0x1p30) return fail(ctx, GOSMA_EINVAL, "dp_means: n * max|x| must be < 2^30");
    return mg_run<false>(ctx, n, x, lambda, max_iter, kmax, sigma_min, 0.0, k, mu, sigma, phi, labels, passes);
}

extern "C" int gosma_dp_vmf_means(gosma_ctx *ctx, int n, const double *x, double lambda, int max_iter, int kmax,
                                  double kappa_max, int *k, double *mu, double *kappa, double *phi, int *labels,
                                  int *passes) {
    int rc = mg_check(ctx, n, x, max_iter, kmax, k, mu, kappa, phi);
    if (rc) return rc;
    if (!isfinite(lambda)) return fail(ctx, GOSMA_EINVAL, "dp_vmf_means: lambda must be finite");
    if (!(kappa_max > 1e-12)) return fail(ctx, GOSMA_EINVAL, "dp_vmf_means: kappa_max must be > 1e-12");
    if (n >= (1 << 22)) return fail(ctx, GOSMA_EINVAL, "dp_vmf_means: at most 2^22 - 1 vectors");
    for (int i = 0; i < n; ++i) {
        const double *v = x + 3 * i;
        const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (!(fabs(r - 1.0) <= 1e-6)) return fail(ctx, GOSMA_EINVAL, "dp_vmf_means: vectors must be unit length");
    }
    return mg_run<true>(ctx, n, x, lambda, max_iter, kmax, 0.0, kappa_max, k, mu, kappa, phi, labels, passes);
}
