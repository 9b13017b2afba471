// The queue-ordering network (an extension of the method, not in the paper):
// a 16 -> 128 -> 128 -> 16 MLP with GELU that scores a sub-cube (output 0, a
// logit) and proposes a seed pose for local refinement (outputs 1..6, an
// offset from the cube centre in half-width units).  Weights and
// activations are BF16, every product runs on the tensor cores (tcgen05,
// tc_gemm.cuh) with FP32 accumulation in tensor memory, and the epilogues
// fuse bias, GELU, its derivative, the transposed copies that the weight
// gradients need and the bias gradients.
//
// Forward   Z1 = X W1^T + b1, H1 = GELU(Z1); Z2 = H1 W2^T + b2, H2 = GELU(Z2);
//           Y = H2 W3^T + b3
// Backward  dZ2 = (dY W3) * GELU'(Z2); dZ1 = (dZ2 W2) * GELU'(Z1);
//           dW3^T = H2^T dY, dW2 = dZ2^T H1, dW1 = dZ1^T X  (split over the
//           batch, FP32 atomics); db = column sums
// Training  logistic loss on Y[:,0] plus a masked squared error on Y[:,1:7],
//           Adam on an FP32 master copy of the parameters.
#include <math.h>
#include <string.h>

#include <vector>

#include "mlp.cuh"

namespace gosma {
// packed parameter layout (FP32): W1 [128 x 16], b1, W2 [128 x 128], b2, W3 [16 x 128], b3
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_HID * MLP_IN, OFF_W2 = OFF_B1 + MLP_HID,
              OFF_B2 = OFF_W2 + MLP_HID * MLP_HID, OFF_W3 = OFF_B2 + MLP_HID, OFF_B3 = OFF_W3 + MLP_OUT * MLP_HID,
              MLP_NPARAM = OFF_B3 + MLP_OUT;
constexpr uint64_t TC_WAIT_NS = 1000000000ull;  // 1 s per wait

enum { EPI_F32 = 0, EPI_GELU = 1, EPI_DGELU = 2 };

struct GemmArgs {
    const bf16 *A;
    long long lda;
    const bf16 *B;
    long long ldb;
    int M;      // rows of D (row-tiled mode): a bound, see Mdev; 128 in split mode
    const int *Mdev;  // if set, the row count is read from device memory (<= M)
    int K;      // contraction length (split mode: a multiple of 128)
    int split;  // contraction split into 128-wide chunks over the CTAs, FP32 atomics
    const float *bias;
    float *outF;  // M x N FP32 (EPI_F32: result; EPI_GELU: pre-activations)
    bf16 *outH;   // M x N BF16
    bf16 *outHT;  // N x ldt BF16 (transposed copy)
    long long ldt;
    const float *zsave;  // M x N pre-activations (EPI_DGELU)
    float *colsum;       // N: column sums of the BF16 result (EPI_DGELU)
    int *err;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Copy a rows x KC tile (rows beyond `valid` zero) into the core-matrix layout.
template <int KC>
__device__ __forceinline__ void tc_stage(unsigned char *dst, const bf16 *src, long long ld, int rows, int valid) {
    const int per_row = KC / 8;
    for (int v = threadIdx.x; v < rows * per_row; v += blockDim.x) {
        const int r = v / per_row, j = v - r * per_row;
        uint4 x = make_uint4(0, 0, 0, 0);
        if (r < valid) x = *reinterpret_cast<const uint4 *>(src + (long long)r * ld + 8 * j);
        *reinterpret_cast<uint4 *>(dst + ((r >> 3) * per_row + j) * 128 + (r & 7) * 16) = x;
    }
}

template <int N, int KC, int EPI>
__global__ void __launch_bounds__(128) tc_gemm_kernel(GemmArgs g) {
    extern __shared__ __align__(128) unsigned char tc_smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase_s;
    constexpr int NCOLS = N < 32 ? 32 : N;
    constexpr uint32_t IDESC = tc_idesc_bf16(128, N);
    constexpr uint32_t SBO = (KC / 8) * 128;
    unsigned char *sA = tc_smem, *sB = tc_smem + 128 * KC * 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) tc_alloc(&tbase_s, NCOLS);
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tbase_s;
    const uint32_t taddr = tbase + ((uint32_t)(32 * warp) << 16);
    uint32_t phase = 0;
    bool ok = true;
    const int Mrows = g.Mdev ? min(*g.Mdev, g.M) : g.M;
    const int nunits = g.split ? g.K / KC : (Mrows + 127) / 128;
    int done_units = 0;
    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        // ---- stage operands (all K in one chunk in row-tiled mode)
        if (g.split) {
            tc_stage<KC>(sA, g.A + (long long)u * KC, g.lda, 128, 128);
            tc_stage<KC>(sB, g.B + (long long)u * KC, g.ldb, N, N);
        } else {
            const int row0 = u * 128;
            tc_stage<KC>(sA, g.A + (long long)row0 * g.lda, g.lda, 128, min(128, Mrows - row0));
            tc_stage<KC>(sB, g.B, g.ldb, N, N);
        }
        tc_fence_proxy();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int s = 0; s < KC / 16; ++s)
                tc_mma(tbase, tc_sdesc(a0 + s * 256, 128, SBO), tc_sdesc(b0 + s * 256, 128, SBO), IDESC,
                       (s > 0 || (g.split && done_units > 0)) ? 1u : 0u);
            tc_commit(&mbar);
        }
        ok = mbar_wait(&mbar, phase, TC_WAIT_NS);
        ok = __syncthreads_and(ok);
        phase ^= 1u;
        ++done_units;
        if (!ok) break;
        tc_fence_after();
        if (g.split) continue;  // keep accumulating; one epilogue at the end
        // ---- row-tiled epilogue: thread = row
        const int row = u * 128 + 32 * warp + lane;
        const bool valid = row < Mrows;
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc_ld16(taddr + c0, v);
            if (EPI == EPI_F32) {
                if (valid) {
                    float *o = g.outF + (long long)row * N + c0;
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        *reinterpret_cast<float4 *>(o + i) =
                            make_float4(v[i] + (g.bias ? g.bias[c0 + i] : 0.f), v[i + 1] + (g.bias ? g.bias[c0 + i + 1] : 0.f),
                                        v[i + 2] + (g.bias ? g.bias[c0 + i + 2] : 0.f),
                                        v[i + 3] + (g.bias ? g.bias[c0 + i + 3] : 0.f));
                }
            } else {
                __align__(16) bf16 hb[16];
                float hv[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float h;
                    if (EPI == EPI_GELU) {
                        const float z = v[i] + g.bias[c0 + i];
                        v[i] = z;
                        h = gelu_f(z);
                    } else {
                        h = valid ? v[i] * gelu_grad_f(g.zsave[(long long)row * N + c0 + i]) : 0.f;
                    }
                    hb[i] = __float2bfloat16_rn(h);
                    hv[i] = valid ? __bfloat162float(hb[i]) : 0.f;
                }
                if (valid) {
                    if (EPI == EPI_GELU && g.outF) {  // pre-activations, kept for training only
                        float *o = g.outF + (long long)row * N + c0;
#pragma unroll
                        for (int i = 0; i < 16; i += 4)
                            *reinterpret_cast<float4 *>(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                    }
                    uint4 *oh = reinterpret_cast<uint4 *>(g.outH + (long long)row * N + c0);
                    oh[0] = reinterpret_cast<const uint4 *>(hb)[0];
                    oh[1] = reinterpret_cast<const uint4 *>(hb)[1];
                    if (g.outHT) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) g.outHT[(long long)(c0 + i) * g.ldt + row] = hb[i];
                    }
                }
                if (EPI == EPI_DGELU && g.colsum) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        float s = hv[i];
                        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
                        if (lane == 0) atomicAdd(g.colsum + c0 + i, s);
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();  // TMEM reads done before the next tile's MMA
    }
    if (ok && g.split && done_units > 0) {
        // split epilogue: FP32 atomics of this CTA's partial sums, thread = row of D
        const int row = 32 * warp + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc_ld16(taddr + c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) atomicAdd(g.outF + (long long)row * N + c0 + i, v[i]);
        }
    }
    if (!ok && threadIdx.x == 0) atomicExch(g.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tbase, NCOLS);
}

template <int N, int KC, int EPI>
static cudaError_t tc_gemm(const GemmArgs &g, int sm_count, cudaStream_t st) {
    auto kern = tc_gemm_kernel<N, KC, EPI>;
    // at least 60 KB so that at most three CTAs share an SM: 3 x 128 TMEM
    // columns fit the SM's 512, so tcgen05.alloc never waits
    const int need = (128 + N) * KC * 2, smem = need > 60 * 1024 ? need : 60 * 1024;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int units = g.split ? g.K / KC : (g.M + 127) / 128;
    if (units <= 0) return cudaSuccess;
    int grid = units < 2 * sm_count ? units : 2 * sm_count;
    kern<<<grid, 128, smem, st>>>(g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- fused inference
// Y = W3 GELU(W2 GELU(W1 x + b1) + b2) + b3 for 128-row tiles in one kernel:
// the BF16 weights are staged once per CTA and stay in shared memory, the
// hidden activations go from TMEM through registers (bias, GELU, BF16) back
// to shared memory as the next layer's A operand, and never reach HBM.
// TMEM columns [0, 128) hold the layer-1 and then the layer-2 accumulator,
// [128, 144) the outputs.
constexpr int INF_X = 128 * MLP_IN * 2, INF_H = 128 * MLP_HID * 2, INF_W1 = MLP_HID * MLP_IN * 2,
              INF_W2 = MLP_HID * MLP_HID * 2, INF_W3 = MLP_OUT * MLP_HID * 2;
constexpr int INF_SMEM = INF_X + INF_H + INF_W1 + INF_W2 + INF_W3;  // 76 KB: at most 2 CTAs (512 TMEM columns) per SM
constexpr int INF_COLS = 256;

// 16 consecutive BF16 values of row r, columns c0..c0+15, into a K = 128
// core-matrix tile.
__device__ __forceinline__ void tc_put16(unsigned char *tile, int r, int c0, const bf16 *v) {
    unsigned char *base = tile + ((r >> 3) * (MLP_HID / 8) + (c0 >> 3)) * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4 *>(base) = reinterpret_cast<const uint4 *>(v)[0];
    *reinterpret_cast<uint4 *>(base + 128) = reinterpret_cast<const uint4 *>(v)[1];
}

__global__ void __launch_bounds__(128)
    mlp_infer_kernel(const bf16 *__restrict__ X, const int *__restrict__ d_rows, int max_rows, const bf16 *__restrict__ W1b,
                     const bf16 *__restrict__ W2b, const bf16 *__restrict__ W3b, const float *__restrict__ P,
                     float *__restrict__ Y, int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char inf_smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase_s;
    unsigned char *sX = inf_smem, *sH = sX + INF_X, *sW1 = sH + INF_H, *sW2 = sW1 + INF_W1, *sW3 = sW2 + INF_W2;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tc_alloc(&tbase_s, INF_COLS);
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_stage<MLP_IN>(sW1, W1b, MLP_IN, MLP_HID, MLP_HID);
    tc_stage<MLP_HID>(sW2, W2b, MLP_HID, MLP_HID, MLP_HID);
    tc_stage<MLP_HID>(sW3, W3b, MLP_HID, MLP_OUT, MLP_OUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tbase_s, taddr = tbase + ((uint32_t)(32 * warp) << 16);
    const int rows = min(*d_rows, max_rows), ntiles = (rows + 127) / 128;
    const float *b1 = P + OFF_B1, *b2 = P + OFF_B2, *b3 = P + OFF_B3;
    uint32_t phase = 0;
    bool ok = true;
    // issue the MMAs of one layer from one thread and wait for them (bounded)
    auto layer = [&](unsigned char *A, uint32_t sboA, unsigned char *B, uint32_t sboB, int ksteps, uint32_t dcol,
                     uint32_t idesc) {
        tc_fence_proxy();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
            for (int s = 0; s < ksteps; ++s)
                tc_mma(tbase + dcol, tc_sdesc(a0 + s * 256, 128, sboA), tc_sdesc(b0 + s * 256, 128, sboB), idesc,
                       s > 0 ? 1u : 0u);
            tc_commit(&mbar);
        }
        bool w = mbar_wait(&mbar, phase, TC_WAIT_NS);
        phase ^= 1u;
        w = __syncthreads_and(w);
        tc_fence_after();
        return w;
    };
    for (int u = blockIdx.x; u < ntiles && ok; u += gridDim.x) {
        const int row0 = u * 128, row = row0 + threadIdx.x;
        tc_stage<MLP_IN>(sX, X + (size_t)row0 * MLP_IN, MLP_IN, 128, min(128, rows - row0));
        ok = layer(sX, 2 * 128, sW1, 2 * 128, 1, 0, tc_idesc_bf16(128, MLP_HID));
        if (!ok) break;
        for (int l = 0; l < 2 && ok; ++l) {  // hidden layer l: TMEM -> bias, GELU -> BF16 tile
            const float *b = l == 0 ? b1 : b2;
#pragma unroll 1
            for (int c0 = 0; c0 < MLP_HID; c0 += 16) {
                float v[16];
                tc_ld16(taddr + c0, v);
                __align__(16) bf16 h[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) h[i] = __float2bfloat16_rn(gelu_f(v[i] + b[c0 + i]));
                tc_put16(sH, threadIdx.x, c0, h);
            }
            if (l == 0) ok = layer(sH, 16 * 128, sW2, 16 * 128, MLP_HID / 16, 0, tc_idesc_bf16(128, MLP_HID));
            else ok = layer(sH, 16 * 128, sW3, 16 * 128, MLP_HID / 16, MLP_HID, tc_idesc_bf16(128, MLP_OUT));
        }
        if (!ok) break;
        float v[16];
        tc_ld16(taddr + MLP_HID, v);
        if (row < rows) {
            float *o = Y + (size_t)row * MLP_OUT;
#pragma unroll
            for (int i = 0; i < 16; i += 4)
                *reinterpret_cast<float4 *>(o + i) =
                    make_float4(v[i] + b3[i], v[i + 1] + b3[i + 1], v[i + 2] + b3[i + 2], v[i + 3] + b3[i + 3]);
        }
        tc_fence_before();
        __syncthreads();  // TMEM reads and the H tile done before the next tile's MMAs
    }
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tbase, INF_COLS);
}

// ---------------------------------------------------------------- small kernels
__global__ void mlp_cast(const float *__restrict__ P, bf16 *W1b, bf16 *W2b, bf16 *W3b, bf16 *W2Tb, bf16 *W3Tb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_HID * MLP_HID; i += gridDim.x * blockDim.x) {
        const int o = i / MLP_HID, c = i % MLP_HID;
        W2b[i] = __float2bfloat16_rn(P[OFF_W2 + i]);
        W2Tb[c * MLP_HID + o] = __float2bfloat16_rn(P[OFF_W2 + i]);
        if (i < MLP_HID * MLP_IN) W1b[i] = __float2bfloat16_rn(P[OFF_W1 + i]);
        if (i < MLP_OUT * MLP_HID) {
            W3b[i] = __float2bfloat16_rn(P[OFF_W3 + i]);
            const int oo = i / MLP_HID, hh = i % MLP_HID;
            W3Tb[hh * MLP_OUT + oo] = __float2bfloat16_rn(P[OFF_W3 + i]);
        }
    }
}

// FP32 rows (n x 16) -> BF16 rows and the transposed copy, zero rows up to npad.
__global__ void mlp_load_x(const float *__restrict__ x, int n, int npad, bf16 *X, bf16 *XT) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad * MLP_IN; i += gridDim.x * blockDim.x) {
        const int r = i / MLP_IN, c = i % MLP_IN;
        const bf16 v = __float2bfloat16_rn(r < n ? x[i] : 0.f);
        X[i] = v;
        XT[(long long)c * npad + r] = v;
    }
}

// Upstream gradient (given, or from the training loss): BF16 rows, the
// transposed copy and the output-bias gradient.  Rows >= n contribute nothing.
__global__ void mlp_dy(const float *__restrict__ Y, const float *__restrict__ dy_in, const float *__restrict__ label,
                       const float *__restrict__ target, float lam, int n, int npad, bf16 *dY, bf16 *dYT,
                       float *db3, float *loss) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < npad; r += gridDim.x * blockDim.x) {
        float d[MLP_OUT];
        for (int c = 0; c < MLP_OUT; ++c) d[c] = 0.f;
        if (r < n) {
            if (dy_in) {
                for (int c = 0; c < MLP_OUT; ++c) d[c] = dy_in[(long long)r * MLP_OUT + c];
            } else {
                const float s = Y[(long long)r * MLP_OUT], l = label[r], inv = 1.f / (float)n;
                // logistic loss log(1 + e^s) - l s, computed stably
                float L = fmaxf(s, 0.f) + log1pf(expf(-fabsf(s))) - l * s;
                d[0] = (1.f / (1.f + expf(-s)) - l) * inv;
                for (int k = 0; k < MLP_SEED; ++k) {
                    const float e = Y[(long long)r * MLP_OUT + 1 + k] - target[(long long)r * MLP_SEED + k];
                    L += lam * l * e * e;
                    d[1 + k] = 2.f * lam * l * e * inv;
                }
                atomicAdd(loss, L * inv);
            }
        }
        for (int c = 0; c < MLP_OUT; ++c) {
            const bf16 b = __float2bfloat16_rn(d[c]);
            dY[(long long)r * MLP_OUT + c] = b;
            dYT[(long long)c * npad + r] = b;
            if (r < n) atomicAdd(db3 + c, __bfloat162float(b));
        }
    }
}

// Adam step on the FP32 master copy; dW3 arrives transposed.  Clears the gradients.
__global__ void mlp_adam(float *P, float *G, float *dW3T, float *Mo, float *Vo, float lr, float b1, float b2, float eps,
                         float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_NPARAM; i += gridDim.x * blockDim.x) {
        float g;
        if (i >= OFF_W3 && i < OFF_B3) {
            const int o = (i - OFF_W3) / MLP_HID, h = (i - OFF_W3) % MLP_HID;
            g = dW3T[h * MLP_OUT + o];
        } else {
            g = G[i];
        }
        const float m = b1 * Mo[i] + (1.f - b1) * g, v = b2 * Vo[i] + (1.f - b2) * g * g;
        Mo[i] = m;
        Vo[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// Gradient in the packed layout (dW3 transposed back).
__global__ void mlp_pack_grad(const float *G, const float *dW3T, float *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_NPARAM; i += gridDim.x * blockDim.x) {
        if (i >= OFF_W3 && i < OFF_B3) {
            const int o = (i - OFF_W3) / MLP_HID, h = (i - OFF_W3) % MLP_HID;
            out[i] = dW3T[h * MLP_OUT + o];
        } else {
            out[i] = G[i];
        }
    }
}

// ---------------------------------------------------------------- state
struct Mlp {
    float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr, *dW3T = nullptr, *loss = nullptr;
    bf16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W2Tb = nullptr, *W3Tb = nullptr;
    int *err = nullptr;
    int step = 0;
    int cap = 0;  // rows (multiple of 128) of the activation buffers
    bf16 *X, *XT, *H1, *H1T, *H2, *H2T, *dY, *dYT, *dZ2, *dZ2T, *dZ1, *dZ1T;
    float *Z1, *Z2, *Y, *gbuf;
    void *act = nullptr;
    void *par = nullptr;
};

void mlp_free(Mlp *m) {
    if (!m) return;
    if (m->act) cudaFree(m->act);
    if (m->par) cudaFree(m->par);
    delete m;
}

static int mlp_params_alloc(gosma_ctx *ctx) {
    if (ctx->mlp) return GOSMA_OK;
    Mlp *m = new Mlp();
    const size_t nf = (size_t)MLP_NPARAM * 4 + MLP_HID * MLP_OUT + 16 + MLP_NPARAM;
    const size_t nb = (size_t)MLP_HID * MLP_IN + 2 * MLP_HID * MLP_HID + 2 * MLP_OUT * MLP_HID;
    cudaError_t e = dev_malloc(ctx, &m->par, nf * 4 + nb * 2 + 256);
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(ctx, e, "cudaMalloc(mlp parameters)");
    }
    float *f = (float *)m->par;
    m->P = f;
    m->G = f + MLP_NPARAM;
    m->Mo = f + 2 * MLP_NPARAM;
    m->Vo = f + 3 * MLP_NPARAM;
    m->dW3T = f + 4 * MLP_NPARAM;
    m->loss = m->dW3T + MLP_HID * MLP_OUT;
    m->gbuf = m->loss + 16;
    m->err = (int *)(m->loss + 8);
    bf16 *b = (bf16 *)(((uintptr_t)(m->gbuf + MLP_NPARAM) + 255) & ~(uintptr_t)255);
    m->W1b = b;
    m->W2b = m->W1b + MLP_HID * MLP_IN;
    m->W2Tb = m->W2b + MLP_HID * MLP_HID;
    m->W3b = m->W2Tb + MLP_HID * MLP_HID;
    m->W3Tb = m->W3b + MLP_OUT * MLP_HID;
    e = cudaMemsetAsync(m->par, 0, nf * 4, ctx->stream);
    if (e != cudaSuccess) {
        mlp_free(m);
        return cuda_fail(ctx, e, "memset(mlp parameters)");
    }
    ctx->mlp = m;
    return GOSMA_OK;
}

static int mlp_act_alloc(gosma_ctx *ctx, int rows) {
    Mlp *m = ctx->mlp;
    const int need = (rows + 127) / 128 * 128;
    if (need <= m->cap) return GOSMA_OK;
    if (m->act) cudaFree(m->act);
    m->act = nullptr;
    m->cap = 0;
    const size_t R = (size_t)need;
    const size_t nb = R * (2 * MLP_IN + 8 * MLP_HID + 2 * MLP_OUT);  // BF16 elements
    const size_t nf = R * (2 * MLP_HID + MLP_OUT);                      // FP32 elements
    cudaError_t e = dev_malloc(ctx, &m->act, nb * 2 + nf * 4 + 1024);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(mlp activations)");
    bf16 *b = (bf16 *)m->act;
    m->X = b;
    m->XT = m->X + R * MLP_IN;
    m->H1 = m->XT + R * MLP_IN;
    m->H1T = m->H1 + R * MLP_HID;
    m->H2 = m->H1T + R * MLP_HID;
    m->H2T = m->H2 + R * MLP_HID;
    m->dZ2 = m->H2T + R * MLP_HID;
    m->dZ2T = m->dZ2 + R * MLP_HID;
    m->dZ1 = m->dZ2T + R * MLP_HID;
    m->dZ1T = m->dZ1 + R * MLP_HID;
    m->dY = m->dZ1T + R * MLP_HID;
    m->dYT = m->dY + R * MLP_OUT;
    float *f = (float *)(((uintptr_t)(m->dYT + R * MLP_OUT) + 255) & ~(uintptr_t)255);
    m->Z1 = f;
    m->Z2 = m->Z1 + R * MLP_HID;
    m->Y = m->Z2 + R * MLP_HID;
    m->cap = need;
    return GOSMA_OK;
}

// Forward pass over npad rows already in m->X / m->XT.
static cudaError_t mlp_forward_dev(gosma_ctx *ctx, Mlp *m, int npad, cudaStream_t st) {
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.err = m->err;
    g.A = m->X, g.lda = MLP_IN, g.B = m->W1b, g.ldb = MLP_IN, g.M = npad, g.K = MLP_IN;
    g.bias = m->P + OFF_B1, g.outF = m->Z1, g.outH = m->H1, g.outHT = m->H1T, g.ldt = npad;
    cudaError_t e = tc_gemm<MLP_HID, MLP_IN, EPI_GELU>(g, ctx->sm_count, st);
    g.A = m->H1, g.lda = MLP_HID, g.B = m->W2b, g.ldb = MLP_HID, g.K = MLP_HID;
    g.bias = m->P + OFF_B2, g.outF = m->Z2, g.outH = m->H2, g.outHT = m->H2T;
    if (e == cudaSuccess) e = tc_gemm<MLP_HID, MLP_HID, EPI_GELU>(g, ctx->sm_count, st);
    g.A = m->H2, g.B = m->W3b, g.ldb = MLP_HID, g.bias = m->P + OFF_B3, g.outF = m->Y;
    g.outH = nullptr, g.outHT = nullptr;
    if (e == cudaSuccess) e = tc_gemm<MLP_OUT, MLP_HID, EPI_F32>(g, ctx->sm_count, st);
    ctx->launches += 3;
    return e;
}

// Backward pass from m->dY / m->dYT (gradients accumulate into m->G, m->dW3T).
static cudaError_t mlp_backward_dev(gosma_ctx *ctx, Mlp *m, int npad, cudaStream_t st) {
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.err = m->err;
    g.A = m->dY, g.lda = MLP_OUT, g.B = m->W3Tb, g.ldb = MLP_OUT, g.M = npad, g.K = MLP_OUT;
    g.zsave = m->Z2, g.outH = m->dZ2, g.outHT = m->dZ2T, g.ldt = npad, g.colsum = m->G + OFF_B2;
    cudaError_t e = tc_gemm<MLP_HID, MLP_OUT, EPI_DGELU>(g, ctx->sm_count, st);
    g.A = m->dZ2, g.lda = MLP_HID, g.B = m->W2Tb, g.ldb = MLP_HID, g.K = MLP_HID;
    g.zsave = m->Z1, g.outH = m->dZ1, g.outHT = m->dZ1T, g.colsum = m->G + OFF_B1;
    if (e == cudaSuccess) e = tc_gemm<MLP_HID, MLP_HID, EPI_DGELU>(g, ctx->sm_count, st);
    // weight gradients: contraction over the batch, split across the CTAs
    GemmArgs w;
    memset(&w, 0, sizeof w);
    w.err = m->err;
    w.split = 1, w.M = 128, w.K = npad;
    w.A = m->H2T, w.lda = npad, w.B = m->dYT, w.ldb = npad, w.outF = m->dW3T;
    if (e == cudaSuccess) e = tc_gemm<MLP_OUT, 128, EPI_F32>(w, ctx->sm_count, st);
    w.A = m->dZ2T, w.B = m->H1T, w.outF = m->G + OFF_W2;
    if (e == cudaSuccess) e = tc_gemm<MLP_HID, 128, EPI_F32>(w, ctx->sm_count, st);
    w.A = m->dZ1T, w.B = m->XT, w.outF = m->G + OFF_W1;
    if (e == cudaSuccess) e = tc_gemm<MLP_OUT, 128, EPI_F32>(w, ctx->sm_count, st);
    ctx->launches += 5;
    return e;
}

static int mlp_check_err(gosma_ctx *ctx, Mlp *m) {
    int herr = 0;
    cudaError_t e = cudaMemcpyAsync(&herr, m->err, sizeof herr, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp");
    if (herr) return fail(ctx, GOSMA_ETIMEOUT, "mlp: a tensor-core wait timed out");
    return GOSMA_OK;
}

static int mlp_stage_x(gosma_ctx *ctx, Mlp *m, int n, const float *h_x, int *npad_out) {
    int rc = mlp_act_alloc(ctx, n);
    if (rc) return rc;
    const int npad = (n + 127) / 128 * 128;
    float *dx = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&dx, sizeof(float) * (size_t)n * MLP_IN, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dx, h_x, sizeof(float) * (size_t)n * MLP_IN, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        mlp_load_x<<<(npad * MLP_IN + 255) / 256, 256, 0, ctx->stream>>>(dx, n, npad, m->X, m->XT);
        ++ctx->launches;
        e = cudaGetLastError();
    }
    if (dx) cudaFreeAsync(dx, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp inputs");
    *npad_out = npad;
    return GOSMA_OK;
}

int mlp_reserve(gosma_ctx *ctx, int rows) {
    if (!ctx->mlp) return fail(ctx, GOSMA_ENOTREADY, "queue-ordering network: no parameters set");
    return mlp_act_alloc(ctx, rows);
}
bf16 *mlp_input(Mlp *m) { return m->X; }
const float *mlp_output(Mlp *m) { return m->Y; }
int *mlp_error_flag(Mlp *m) { return m->err; }

cudaError_t mlp_forward_rows(gosma_ctx *ctx, int max_rows, const int *d_rows, cudaStream_t st) {
    Mlp *m = ctx->mlp;
    cudaError_t e = cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, INF_SMEM);
    if (e != cudaSuccess) return e;
    const int tiles = (max_rows + 127) / 128;
    const int grid = tiles < 2 * ctx->sm_count ? tiles : 2 * ctx->sm_count;
    if (grid <= 0) return cudaSuccess;
    mlp_infer_kernel<<<grid, 128, INF_SMEM, st>>>(m->X, d_rows, max_rows, m->W1b, m->W2b, m->W3b, m->P, m->Y, m->err);
    ++ctx->launches;
    return cudaGetLastError();
}

// Self-test of the bounded waits: one block waits on an mbarrier that nothing
// arrives on, with the given limit; the wait must give up and report it.
__global__ void wait_timeout_selftest(uint64_t limit_ns, int *out) {
    __shared__ uint64_t mbar;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool ok = mbar_wait(&mbar, 0, limit_ns);
    ok = __syncthreads_or(ok);
    if (threadIdx.x == 0) out[0] = ok ? 0 : 1;
}

int selftest_wait_timeout(gosma_ctx *ctx, double limit_s, int *timed_out) {
    int *d = nullptr;
    cudaError_t e = dev_malloc(ctx, (void **)&d, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(selftest)");
    int h = -1;
    wait_timeout_selftest<<<1, 32, 0, ctx->stream>>>((uint64_t)(limit_s * 1e9), d);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "selftest_wait_timeout");
    *timed_out = h;
    return GOSMA_OK;
}

}  // namespace gosma

using namespace gosma;

extern "C" int gosma_mlp_set_params(gosma_ctx *ctx, const float *params) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (!params) return fail(ctx, GOSMA_EINVAL, "mlp_set_params: null parameters");
    cudaSetDevice(ctx->device);
    int rc = mlp_params_alloc(ctx);
    if (rc) return rc;
    Mlp *m = ctx->mlp;
    cudaError_t e = cudaMemcpyAsync(m->P, params, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->Mo, 0, sizeof(float) * 2 * MLP_NPARAM, ctx->stream);
    if (e == cudaSuccess) {
        mlp_cast<<<64, 256, 0, ctx->stream>>>(m->P, m->W1b, m->W2b, m->W3b, m->W2Tb, m->W3Tb);
        ++ctx->launches;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_set_params");
    m->step = 0;
    return GOSMA_OK;
}

extern "C" int gosma_mlp_get_params(gosma_ctx *ctx, float *params) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (!params) return fail(ctx, GOSMA_EINVAL, "mlp_get_params: null output");
    if (!ctx->mlp) return fail(ctx, GOSMA_ENOTREADY, "mlp_get_params: no parameters set");
    cudaError_t e = cudaMemcpyAsync(params, ctx->mlp->P, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_get_params");
    return GOSMA_OK;
}

extern "C" int gosma_mlp_forward(gosma_ctx *ctx, int n, const float *x, float *y) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (n < 0 || (n > 0 && (!x || !y))) return fail(ctx, GOSMA_EINVAL, "mlp_forward: bad arguments");
    if (!ctx->mlp) return fail(ctx, GOSMA_ENOTREADY, "mlp_forward: no parameters set");
    if (n == 0) return GOSMA_OK;
    cudaSetDevice(ctx->device);
    Mlp *m = ctx->mlp;
    int npad = 0;
    int rc = mlp_stage_x(ctx, m, n, x, &npad);
    if (rc) return rc;
    // inference through the fused kernel (row count read from the device)
    int *rows = m->err + 1;
    cudaError_t e = cudaMemsetAsync(m->err, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rows, &n, sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = mlp_forward_rows(ctx, npad, rows, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, m->Y, sizeof(float) * (size_t)n * MLP_OUT, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // the host copy of n must outlive its upload
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_forward");
    return mlp_check_err(ctx, m);
}

extern "C" int gosma_mlp_grad(gosma_ctx *ctx, int n, const float *x, const float *dy, float *grad) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (n < 1 || !x || !dy || !grad) return fail(ctx, GOSMA_EINVAL, "mlp_grad: bad arguments");
    if (!ctx->mlp) return fail(ctx, GOSMA_ENOTREADY, "mlp_grad: no parameters set");
    cudaSetDevice(ctx->device);
    Mlp *m = ctx->mlp;
    int npad = 0;
    int rc = mlp_stage_x(ctx, m, n, x, &npad);
    if (rc) return rc;
    float *ddy = nullptr;
    cudaError_t e = cudaMemsetAsync(m->err, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->G, 0, sizeof(float) * MLP_NPARAM, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->dW3T, 0, sizeof(float) * MLP_HID * MLP_OUT, ctx->stream);
    if (e == cudaSuccess) e = mlp_forward_dev(ctx, m, npad, ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&ddy, sizeof(float) * (size_t)n * MLP_OUT, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ddy, dy, sizeof(float) * (size_t)n * MLP_OUT, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        mlp_dy<<<(npad + 127) / 128, 128, 0, ctx->stream>>>(m->Y, ddy, nullptr, nullptr, 0.f, n, npad, m->dY, m->dYT,
                                                              m->G + OFF_B3, m->loss);
        ++ctx->launches;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = mlp_backward_dev(ctx, m, npad, ctx->stream);
    if (e == cudaSuccess) {
        mlp_pack_grad<<<(MLP_NPARAM + 255) / 256, 256, 0, ctx->stream>>>(m->G, m->dW3T, m->gbuf);
        ++ctx->launches;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, m->gbuf, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, ctx->stream);
    if (ddy) cudaFreeAsync(ddy, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_grad");
    return mlp_check_err(ctx, m);
}

extern "C" int gosma_mlp_train(gosma_ctx *ctx, int n, const float *x, const float *label, const float *target, int batch,
                               int steps, float lr, float lam, float *losses) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (n < 1 || !x || !label || !target || batch < 128 || batch % 128 || n % batch || steps < 0 || !(lr > 0) ||
        !(lam >= 0))
        return fail(ctx, GOSMA_EINVAL, "mlp_train: need n a multiple of batch, batch a multiple of 128, lr > 0");
    if (!ctx->mlp) return fail(ctx, GOSMA_ENOTREADY, "mlp_train: no parameters set");
    cudaSetDevice(ctx->device);
    Mlp *m = ctx->mlp;
    int rc = mlp_act_alloc(ctx, batch);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    // the whole data set stays on the device for the run
    float *dx = nullptr, *dl = nullptr, *dt = nullptr, *dloss = nullptr;
    const size_t bx = sizeof(float) * (size_t)n * MLP_IN, bl = sizeof(float) * (size_t)n,
                 bt = sizeof(float) * (size_t)n * MLP_SEED;
    cudaError_t e = cudaMallocAsync((void **)&dx, bx + bl + bt + sizeof(float) * (size_t)(steps + 1), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(mlp data)");
    dl = (float *)((char *)dx + bx);
    dt = (float *)((char *)dl + bl);
    dloss = (float *)((char *)dt + bt);
    e = cudaMemcpyAsync(dx, x, bx, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dl, label, bl, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dt, target, bt, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dloss, 0, sizeof(float) * (size_t)(steps + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->err, 0, sizeof(int), st);
    const float b1 = 0.9f, b2 = 0.999f;
    for (int s = 0; s < steps && e == cudaSuccess; ++s) {
        const long long r0 = (long long)s * batch % n;
        mlp_load_x<<<(batch * MLP_IN + 255) / 256, 256, 0, st>>>(dx + r0 * MLP_IN, batch, batch, m->X, m->XT);
        ++ctx->launches;
        e = cudaMemsetAsync(m->G, 0, sizeof(float) * MLP_NPARAM, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(m->dW3T, 0, sizeof(float) * MLP_HID * MLP_OUT, st);
        if (e == cudaSuccess) e = mlp_forward_dev(ctx, m, batch, st);
        if (e != cudaSuccess) break;
        mlp_dy<<<(batch + 127) / 128, 128, 0, st>>>(m->Y, nullptr, dl + r0, dt + r0 * MLP_SEED, lam, batch, batch, m->dY,
                                                   m->dYT, m->G + OFF_B3, dloss + s);
        ++ctx->launches;
        e = mlp_backward_dev(ctx, m, batch, st);
        if (e != cudaSuccess) break;
        ++m->step;
        const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
        mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(m->P, m->G, m->dW3T, m->Mo, m->Vo, lr, b1, b2, 1e-8f, c1, c2);
        mlp_cast<<<64, 256, 0, st>>>(m->P, m->W1b, m->W2b, m->W3b, m->W2Tb, m->W3Tb);
        ctx->launches += 2;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && losses && steps > 0)
        e = cudaMemcpyAsync(losses, dloss, sizeof(float) * (size_t)steps, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dx, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp_train");
    return mlp_check_err(ctx, m);
}
