// FP64 device kernels around the bound kernel:
//   - f(R_r, t) and its gradient for local refinement (Lemma 1; SMA, Sec. 5),
//   - set-up constants of the mixtures (C22 and the per-component log terms),
//   - a self-test of the FP32 approximate instructions the bound kernel uses.
#include <math.h>

#include <mutex>

#include "objective_core.cuh"

namespace gosma {

// Poses per launch of the objective kernels (they index poses by gridDim.y).
constexpr int OBJ_MAX_POSES_PER_LAUNCH = 65535;

int objective_grad_device(gosma_ctx *ctx, int count, const double *h_x, double *h_f, double *h_g) {
    if (count <= 0) return GOSMA_OK;
    const int n1 = ctx->n1, n2 = ctx->n2;
    long long total = (long long)n1 * n1 + (long long)n1 * n2;
    int nblk = (int)((total + OBJ_CHUNK - 1) / OBJ_CHUNK);
    size_t bx = sizeof(double) * 6 * count, bi = sizeof(double) * OBJ_STRIDE * (size_t)n1 * count,
           bp = sizeof(double) * 7 * (size_t)nblk * count, bo = sizeof(double) * 7 * count;
    size_t need = bx + bi + bp + bo;
    if (need > ctx->obj_bytes) {
        if (ctx->d_obj) cudaFree(ctx->d_obj);
        ctx->d_obj = nullptr;
        ctx->obj_bytes = 0;
        cudaError_t e = dev_malloc(ctx, &ctx->d_obj, need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(objective)");
        ctx->obj_bytes = need;
    }
    char *base = (char *)ctx->d_obj;
    double *dx = (double *)base, *di = (double *)(base + bx), *dp = (double *)(base + bx + bi),
           *dout = (double *)(base + bx + bi + bp);
    int rc = ensure_pinned(ctx, bx + bo);
    if (rc) return rc;
    double *hp = (double *)ctx->h_pinned;
    memcpy(hp, h_x, bx);
    cudaError_t e = cudaMemcpyAsync(dx, hp, bx, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy poses");
    // poses index gridDim.y, so at most 65,535 of them go into one launch
    for (int p0 = 0; p0 < count; p0 += OBJ_MAX_POSES_PER_LAUNCH) {
        const int m = count - p0 < OBJ_MAX_POSES_PER_LAUNCH ? count - p0 : OBJ_MAX_POSES_PER_LAUNCH;
        const double *xs = dx + 6 * (size_t)p0;
        double *is = di + (size_t)OBJ_STRIDE * n1 * p0, *ps = dp + (size_t)7 * nblk * p0;
        obj_prep<<<dim3((n1 + 127) / 128, m), 128, 0, ctx->stream>>>(OneMix{ctx->mix}, xs, is);
        ++ctx->launches;
        obj_pairs<<<dim3(nblk, m), OBJ_BLOCK, 0, ctx->stream>>>(OneMix{ctx->mix}, xs, is, ps, nblk);
        ++ctx->launches;
        obj_final<<<(m + OBJ_FINAL_WARPS - 1) / OBJ_FINAL_WARPS, 32 * OBJ_FINAL_WARPS, 0, ctx->stream>>>(
            m, xs, ps, nblk, dout + 7 * (size_t)p0);
        ++ctx->launches;
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "launch(objective)");
    }
    double *ho = hp + 6 * count;
    e = cudaMemcpyAsync(ho, dout, bo, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy objective");
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync(objective)");
    for (int p = 0; p < count; ++p) {
        if (h_f) h_f[p] = ho[7 * p];
        if (h_g)
            for (int k = 0; k < 6; ++k) h_g[6 * p + k] = ho[7 * p + 1 + k];
    }
    return GOSMA_OK;
}

// ---------------------------------------------------------------- set-up constants
// Q2_j = phi_2j kappa_2j / (1 - e^{-2 kappa_2j}) (the column factor of the
// linear-form pair terms), FP64 rounded once, and C22 = sum_jj' phi phi
// Z(|k_j mu_j + k_j' mu_j'|)/(Z(k_j) Z(k_j')) (2 pi times the integral of
// p2^2, proof of Lemma 1) as per-block partial sums.
__global__ void setup_image(MixDev mx, double *c22part) {
    float *Q2 = const_cast<float *>(mx.Q2), *mh = const_cast<float *>(mx.mu2h), *ml = const_cast<float *>(mx.mu2l);
    __shared__ double red[8];
    double acc = 0.0;
    const int n2 = mx.n2;
    long long total = (long long)n2 * n2;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        int a = (int)(q / n2), b = (int)(q % n2);
        if (mx.cls2 && mx.cls2[a] != mx.cls2[b]) continue;  // C22 = sum over classes of w_l C22_l
        const double *ma = mx.mu2 + 3 * a, *mb = mx.mu2 + 3 * b;
        double ka = mx.kappa2d[a], kb = mx.kappa2d[b];
        double w0 = ka * ma[0] + kb * mb[0], w1 = ka * ma[1] + kb * mb[1], w2 = ka * ma[2] + kb * mb[2];
        double K = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
        acc += mx.phi2d[a] * mx.phi2d[b] * exp(logZ_d(K) - logZ_d(ka) - logZ_d(kb));
    }
    float *lQc = const_cast<float *>(mx.lQ2c), *lQb = const_cast<float *>(mx.lQ2b);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n2; j += gridDim.x * blockDim.x) {
        double k = mx.kappa2d[j];
        const double q = mx.phi2d[j] * k / -expm1(-2.0 * k);
        Q2[j] = (float)q;
        // log2 Q for the pair terms' exponents; the bound's copy carries the
        // cross pair's slack (20 u) and the rounding of its own size in the
        // exponent's final rounding (u (|log2 Q| + 1)), rounded up
        const float ninf = __int_as_float(0xff800000);
        const double lq = log2(q);
        lQc[j] = q > 0.0 ? (float)lq : ninf;
        lQb[j] = q > 0.0 ? __double2float_ru(lq + (double)GOSMA_CROSS_SLACK + 0x1p-24 * (fabs(lq) + 1.0)) : ninf;
        for (int c = 0; c < 3; ++c) {
            double m = mx.mu2[3 * j + c];
            float h = (float)m;
            mh[3 * j + c] = h;
            ml[3 * j + c] = (float)(m - (double)h);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        c22part[blockIdx.x] = s;
    }
}

__global__ void setup_model(MixDev mx) {
    float *inv_sig2 = const_cast<float *>(mx.inv_sig2), *phi1f = const_cast<float *>(mx.phi1f);
    float *mh = const_cast<float *>(mx.mu1h), *ml = const_cast<float *>(mx.mu1l);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < mx.n1; i += gridDim.x * blockDim.x) {
        double s = mx.sigma1d[i];
        inv_sig2[i] = (float)(1.0 / (s * s));
        phi1f[i] = (float)mx.phi1d[i];
        for (int c = 0; c < 3; ++c) {
            double m = mx.mu1[3 * i + c];
            float h = (float)m;
            mh[3 * i + c] = h;
            ml[3 * i + c] = (float)(m - (double)h);
        }
    }
}

int setup_constants_mix(gosma_ctx *ctx, cudaStream_t st, const MixDev &mx, double *c22_out) {
    const int nb = 64;
    double *dpart = nullptr;
    cudaError_t e = dev_malloc(ctx, (void **)&dpart, sizeof(double) * nb);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(setup)");
    setup_image<<<nb, 256, 0, st>>>(mx, dpart);
    ++ctx->launches;
    setup_model<<<(mx.n1 + 255) / 256, 256, 0, st>>>(mx);
    ++ctx->launches;
    double hp[nb];
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp, dpart, sizeof hp, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dpart);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "setup kernels");
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += hp[k];
    *c22_out = s;
    return GOSMA_OK;
}

int setup_constants(gosma_ctx *ctx, double *c22_out) { return setup_constants_mix(ctx, ctx->stream, ctx->mix, c22_out); }

// ---------------------------------------------------------------- self-test
// Max relative error of ex2, lg2, rcp, rsqrt, sqrt (approximate PTX forms)
// against FP64 over a dense logarithmic sweep of arguments.
__global__ void approx_selftest(unsigned *maxbits) {
    float m[5] = {0, 0, 0, 0, 0};
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < (1LL << 24);
         k += (long long)gridDim.x * blockDim.x) {
        // ex2 on [-120, 120]
        float xe = -120.f + 240.f * (float)k / (float)(1 << 24);
        double re = exp2((double)xe);
        m[0] = fmaxf(m[0], (float)fabs(((double)ex2a(xe) - re) / re));
        // positive arguments spread over 2^-60 .. 2^60
        float xp = exp2f(-60.f + 120.f * (float)k / (float)(1 << 24));
        double rl = log2((double)xp);
        double el = fabs((double)lg2a(xp) - rl);
        // relative for |log2 x| >= 1, absolute below (where the result is small)
        m[1] = fmaxf(m[1], (float)(fabs(rl) >= 1.0 ? el / fabs(rl) : el));
        double rr = 1.0 / (double)xp;
        m[2] = fmaxf(m[2], (float)fabs(((double)rcpa(xp) - rr) / rr));
        double rs = 1.0 / sqrt((double)xp);
        m[3] = fmaxf(m[3], (float)fabs(((double)rsqrta(xp) - rs) / rs));
        double sq = sqrt((double)xp);
        m[4] = fmaxf(m[4], (float)fabs(((double)sqrta(xp) - sq) / sq));
    }
    for (int q = 0; q < 5; ++q) atomicMax(maxbits + q, __float_as_uint(m[q]));
}

int selftest_approx(gosma_ctx *ctx, double measured[5], double assumed[5]) {
    unsigned *d = nullptr;
    cudaError_t e = dev_malloc(ctx, (void **)&d, 5 * sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(selftest)");
    unsigned h[5] = {0, 0, 0, 0, 0};
    e = cudaMemsetAsync(d, 0, sizeof h, ctx->stream);
    if (e == cudaSuccess) {
        approx_selftest<<<4 * ctx->sm_count, 256, 0, ctx->stream>>>(d);
        ++ctx->launches;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "selftest");
    for (int q = 0; q < 5; ++q) {
        float f;
        memcpy(&f, &h[q], sizeof f);
        measured[q] = f;
        assumed[q] = (double)GOSMA_APPROX_REL;
    }
    assumed[1] = (double)GOSMA_LG2_ABS;
    return GOSMA_OK;
}

}  // namespace gosma

namespace gosma {

// ---------------------------------------------------------------- allocation-free objective
// Some callers of this library cannot let it allocate device memory once they
// are running: real-time tracking loops that size every buffer at start-up and
// must not stall on cudaMalloc's implicit device synchronisation, and host
// applications that own the whole device-memory budget and forbid libraries
// from allocating behind their back.  gosma_eval_objective_grad_noalloc serves
// them: the caller passes device buffers for the poses and the results, and the
// kernels' scratch lives in the fixed array below instead of in cudaMalloc'd
// memory.
//
// The array is a file-scope device variable, so every GPU that loads the
// library holds NOALLOC_SCRATCH_BYTES for as long as the library stays loaded.
// All calls on a device share it: two calls whose kernels overlap on the GPU
// (for example on two streams) race on it.  The scratch needs no clearing:
// every byte a call reads was written earlier in the same call.
//
// A call is accepted when its scratch, count * (128 n1 + 56 ceil((n1^2 +
// n1 n2) / 512)) bytes, is at most NOALLOC_LIMIT_BYTES; the array holds 256
// bytes more, so that the partial sums can start on a 256-byte boundary
// without shrinking that limit.
constexpr size_t NOALLOC_LIMIT_BYTES = (size_t)8 << 20;  // 8 MiB
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_LIMIT_BYTES + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, looked up once per device
// (in host code the array's name is only a host-side stand-in, not a device
// address) and kept for the life of the process: a cudaDeviceReset of that
// device between calls would leave it stale.
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[128];

static int noalloc_scratch(gosma_ctx *ctx, void **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (ctx->device < 0 || ctx->device >= 128) return fail(ctx, GOSMA_EINVAL, "device index out of range");
    if (!g_noalloc_ptr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(ctx, e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_ptr[ctx->device] = p;
    }
    *out = g_noalloc_ptr[ctx->device];
    return GOSMA_OK;
}

}  // namespace gosma

extern "C" int gosma_eval_objective_grad_noalloc(gosma_ctx *ctx, int count, const double *d_x, double *d_out) {
    using namespace gosma;
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (!ctx->have_mix) return fail(ctx, GOSMA_ENOTREADY, "eval_objective_grad_noalloc: set mixtures first");
    if (count < 0 || (count > 0 && (!d_x || !d_out)))
        return fail(ctx, GOSMA_EINVAL, "eval_objective_grad_noalloc: bad poses or output");
    if (count == 0) return GOSMA_OK;
    const int n1 = ctx->n1, n2 = ctx->n2;
    long long total = (long long)n1 * n1 + (long long)n1 * n2;
    int nblk = (int)((total + OBJ_CHUNK - 1) / OBJ_CHUNK);
    const size_t bi = sizeof(double) * OBJ_STRIDE * (size_t)n1 * count;
    const size_t bp = sizeof(double) * 7 * (size_t)nblk * count;
    if (bi + bp > NOALLOC_LIMIT_BYTES)
        return fail(ctx, GOSMA_EINVAL,
                    "eval_objective_grad_noalloc: count * (128 n1 + 56 ceil((n1^2 + n1 n2) / 512)) bytes "
                    "exceeds the 8 MiB scratch; use fewer poses per call");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    void *scratch = nullptr;
    int rc = noalloc_scratch(ctx, &scratch);
    if (rc) return rc;
    // partial sums on a 256-byte boundary: at most 255 bytes past the limit, inside the array
    double *di = (double *)scratch, *dp = (double *)((char *)scratch + ((bi + 255) & ~(size_t)255));
    obj_prep<<<dim3((n1 + 127) / 128, count), 128, 0, ctx->stream>>>(OneMix{ctx->mix}, d_x, di);
    ++ctx->launches;
    obj_pairs<<<dim3(nblk, count), OBJ_BLOCK, 0, ctx->stream>>>(OneMix{ctx->mix}, d_x, di, dp, nblk);
    ++ctx->launches;
    obj_final<<<(count + OBJ_FINAL_WARPS - 1) / OBJ_FINAL_WARPS, 32 * OBJ_FINAL_WARPS, 0, ctx->stream>>>(count, d_x, dp, nblk,
                                                                                                   d_out);
    ++ctx->launches;
    e = cudaGetLastError();
    return e == cudaSuccess ? GOSMA_OK : cuda_fail(ctx, e, "launch(objective, no-alloc)");
}

