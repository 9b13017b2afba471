// FP64 device kernels around the bound kernel:
//   - f(R_r, t) and its gradient for local refinement (Lemma 1; SMA, Sec. 5),
//   - set-up constants of the mixtures (C22 and the per-component log terms),
//   - a self-test of the FP32 approximate instructions the bound kernel uses.
#include <math.h>

#include <mutex>

#include "gosma_internal.cuh"

namespace gosma {

// log Z(x) of Eq. (Z) and its derivative coth x - 1/x, FP64.
__device__ __forceinline__ double logZ_d(double x) {
    if (x < 1e-12) return M_LN2;
    return x + log(-expm1(-2.0 * x) / x);
}
__device__ __forceinline__ double dlogZ_d(double x) {
    if (x < 1e-4) return x / 3.0 - x * x * x / 45.0;
    return 1.0 + 2.0 / expm1(2.0 * x) - 1.0 / x;
}

__device__ void rodrigues_dev(const double r[3], double R[9]) {
    double th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], th = sqrt(th2), A, B;
    if (th < 1e-8) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
    } else {
        double s, c;
        sincos(th, &s, &c);
        A = s / th;
        B = (1.0 - c) / th2;
    }
    double x = r[0], y = r[1], z = r[2];
    R[0] = 1.0 - B * (y * y + z * z);
    R[1] = -A * z + B * x * y;
    R[2] = A * y + B * x * z;
    R[3] = A * z + B * x * y;
    R[4] = 1.0 - B * (x * x + z * z);
    R[5] = -A * x + B * y * z;
    R[6] = -A * y + B * x * z;
    R[7] = A * x + B * y * z;
    R[8] = 1.0 - B * (x * x + y * y);
}

// Per (pose, model component) quantities, 16 doubles:
//   v(3) d kappa lZ dlZ Rv(3) dk(3) pad(3)
constexpr int OBJ_STRIDE = 16;
constexpr int OBJ_BLOCK = 256;
constexpr int OBJ_CHUNK = 512;  // pair indices per block

__global__ void obj_prep(MixDev mx, int count, const double *__restrict__ x, double *__restrict__ idata) {
    int p = blockIdx.y;
    __shared__ double R[9];
    if (threadIdx.x == 0) rodrigues_dev(x + 6 * p, R);
    __syncthreads();
    const double *t = x + 6 * p + 3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < mx.n1; i += gridDim.x * blockDim.x) {
        const double *mu = mx.mu1 + 3 * i;
        double m0 = mu[0] - t[0], m1 = mu[1] - t[1], m2 = mu[2] - t[2];
        double d = sqrt(m0 * m0 + m1 * m1 + m2 * m2);
        double v0 = m0 / d, v1 = m1 / d, v2 = m2 / d;
        double s = mx.sigma1d[i];
        double k = d * d / (s * s) + 1.0;  // Eq. (kappa1)
        double *o = idata + ((size_t)p * mx.n1 + i) * OBJ_STRIDE;
        o[0] = v0;
        o[1] = v1;
        o[2] = v2;
        o[3] = d;
        o[4] = k;
        o[5] = logZ_d(k);
        o[6] = dlogZ_d(k);
        o[7] = R[0] * v0 + R[1] * v1 + R[2] * v2;
        o[8] = R[3] * v0 + R[4] * v1 + R[5] * v2;
        o[9] = R[6] * v0 + R[7] * v1 + R[8] * v2;
        double g = -2.0 / (s * s);
        o[10] = g * m0;
        o[11] = g * m1;
        o[12] = g * m2;
    }
}

// f = sum_ij self(i,j) - 2 sum_ij cross(i,j); gradient w.r.t. t and the
// left-perturbation omega of R (d(Rv) = omega x Rv).
__global__ void __launch_bounds__(OBJ_BLOCK) obj_pairs(MixDev mx, int count, const double *__restrict__ x,
                                                       const double *__restrict__ idata, double *__restrict__ part,
                                                       int nblk) {
    int p = blockIdx.y;
    __shared__ double R[9];
    __shared__ double red[7][OBJ_BLOCK / 32];
    if (threadIdx.x == 0) rodrigues_dev(x + 6 * p, R);
    __syncthreads();
    const int n1 = mx.n1, n2 = mx.n2;
    const long long nself = (long long)n1 * n1, total = nself + (long long)n1 * n2;
    const double *I = idata + (size_t)p * n1 * OBJ_STRIDE;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    long long q0 = (long long)blockIdx.x * OBJ_CHUNK;
    long long q1 = q0 + OBJ_CHUNK < total ? q0 + OBJ_CHUNK : total;
    for (long long q = q0 + threadIdx.x; q < q1; q += OBJ_BLOCK) {
        if (q < nself) {
            int i = (int)(q / n1), j = (int)(q % n1);
            const double *A = I + (size_t)i * OBJ_STRIDE, *B = I + (size_t)j * OBJ_STRIDE;
            double w0 = A[4] * A[0] + B[4] * B[0], w1 = A[4] * A[1] + B[4] * B[1], w2 = A[4] * A[2] + B[4] * B[2];
            double K = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
            double T = mx.phi1d[i] * mx.phi1d[j] * exp(logZ_d(K) - A[5] - B[5]);
            acc[0] += T;
            double gK = K > 0 ? dlogZ_d(K) / K : 0.0;
            double vwA = A[0] * w0 + A[1] * w1 + A[2] * w2, vwB = B[0] * w0 + B[1] * w1 + B[2] * w2;
            double ww[3] = {w0, w1, w2};
            for (int c = 0; c < 3; ++c) {
                // dK/dt_c * K = (v_i.w) dk_i + k_i (dv_i/dt)^T w + (same for j)
                double dvA = -(ww[c] - A[c] * vwA) / A[3];
                double dvB = -(ww[c] - B[c] * vwB) / B[3];
                double dKK = vwA * A[10 + c] + A[4] * dvA + vwB * B[10 + c] + B[4] * dvB;
                acc[1 + c] += T * (gK * dKK - A[6] * A[10 + c] - B[6] * B[10 + c]);
            }
        } else {
            long long qq = q - nself;
            int i = (int)(qq / n2), j = (int)(qq % n2);
            const double *A = I + (size_t)i * OBJ_STRIDE;
            const double *mu = mx.mu2 + 3 * j;
            double k2 = mx.kappa2d[j];
            double w0 = A[4] * A[7] + k2 * mu[0], w1 = A[4] * A[8] + k2 * mu[1], w2 = A[4] * A[9] + k2 * mu[2];
            double K = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
            double T = mx.phi1d[i] * mx.phi2d[j] * exp(logZ_d(K) - A[5] - logZ_d(k2));
            acc[0] -= 2.0 * T;
            double gK = K > 0 ? dlogZ_d(K) / K : 0.0;
            // R^T w
            double rw0 = R[0] * w0 + R[3] * w1 + R[6] * w2;
            double rw1 = R[1] * w0 + R[4] * w1 + R[7] * w2;
            double rw2 = R[2] * w0 + R[5] * w1 + R[8] * w2;
            double vw = A[0] * rw0 + A[1] * rw1 + A[2] * rw2;  // = Rv . w
            double rw[3] = {rw0, rw1, rw2};
            for (int c = 0; c < 3; ++c) {
                double dv = -(rw[c] - A[c] * vw) / A[3];
                double dKK = vw * A[10 + c] + A[4] * dv;
                acc[1 + c] += -2.0 * T * (gK * dKK - A[6] * A[10 + c]);
            }
            // dK/domega = k_i (Rv x w) / K
            double c0 = A[8] * w2 - A[9] * w1, c1 = A[9] * w0 - A[7] * w2, c2 = A[7] * w1 - A[8] * w0;
            acc[4] += -2.0 * T * gK * A[4] * c0;
            acc[5] += -2.0 * T * gK * A[4] * c1;
            acc[6] += -2.0 * T * gK * A[4] * c2;
        }
    }
    for (int k = 0; k < 7; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int k = 0; k < 7; ++k) red[k][w] = acc[k];
    __syncthreads();
    if (threadIdx.x < 7) {
        double s = 0.0;
        for (int k = 0; k < OBJ_BLOCK / 32; ++k) s += red[threadIdx.x][k];
        part[((size_t)p * nblk + blockIdx.x) * 7 + threadIdx.x] = s;
    }
}

__global__ void obj_final(int count, const double *__restrict__ x, const double *__restrict__ part, int nblk,
                          double *__restrict__ out) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count) return;
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nblk; ++b)
        for (int k = 0; k < 7; ++k) s[k] += part[((size_t)p * nblk + b) * 7 + k];
    // d/dr = J_l(r)^T d/domega, J_l = I + a [r]x + b [r]x^2 (left Jacobian of SO(3))
    const double *r = x + 6 * p;
    double th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], th = sqrt(th2), a, b;
    if (th < 1e-6) {
        a = 0.5 - th2 / 24.0;
        b = 1.0 / 6.0 - th2 / 120.0;
    } else {
        a = (1.0 - cos(th)) / th2;
        b = (th - sin(th)) / (th2 * th);
    }
    const double *gw = s + 4;
    // [r]x^T g = -r x g ; ([r]x^2)^T g = [r]x^2 g = r (r.g) - |r|^2 g
    double rxg[3] = {r[1] * gw[2] - r[2] * gw[1], r[2] * gw[0] - r[0] * gw[2], r[0] * gw[1] - r[1] * gw[0]};
    double rg = r[0] * gw[0] + r[1] * gw[1] + r[2] * gw[2];
    double *o = out + 7 * p;
    o[0] = s[0];
    for (int c = 0; c < 3; ++c) o[1 + c] = gw[c] - a * rxg[c] + b * (r[c] * rg - th2 * gw[c]);
    for (int c = 0; c < 3; ++c) o[4 + c] = s[1 + c];
}

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
        cudaError_t e = cudaMalloc(&ctx->d_obj, need);
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
    obj_prep<<<dim3((n1 + 127) / 128, count), 128, 0, ctx->stream>>>(ctx->mix, count, dx, di);
    ++ctx->launches;
    obj_pairs<<<dim3(nblk, count), OBJ_BLOCK, 0, ctx->stream>>>(ctx->mix, count, dx, di, dp, nblk);
    ++ctx->launches;
    obj_final<<<(count + 63) / 64, 64, 0, ctx->stream>>>(count, dx, dp, nblk, dout);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch(objective)");
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
        const double *ma = mx.mu2 + 3 * a, *mb = mx.mu2 + 3 * b;
        double ka = mx.kappa2d[a], kb = mx.kappa2d[b];
        double w0 = ka * ma[0] + kb * mb[0], w1 = ka * ma[1] + kb * mb[1], w2 = ka * ma[2] + kb * mb[2];
        double K = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
        acc += mx.phi2d[a] * mx.phi2d[b] * exp(logZ_d(K) - logZ_d(ka) - logZ_d(kb));
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n2; j += gridDim.x * blockDim.x) {
        double k = mx.kappa2d[j];
        Q2[j] = (float)(mx.phi2d[j] * k / -expm1(-2.0 * k));
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

int setup_constants(gosma_ctx *ctx, double *c22_out) {
    const int nb = 64;
    double *dpart = nullptr;
    cudaError_t e = cudaMalloc(&dpart, sizeof(double) * nb);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(setup)");
    setup_image<<<nb, 256, 0, ctx->stream>>>(ctx->mix, dpart);
    ++ctx->launches;
    setup_model<<<(ctx->n1 + 255) / 256, 256, 0, ctx->stream>>>(ctx->mix);
    ++ctx->launches;
    double hp[nb];
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp, dpart, sizeof hp, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(dpart);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "setup kernels");
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += hp[k];
    *c22_out = s;
    return GOSMA_OK;
}

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
    cudaError_t e = cudaMalloc(&d, 5 * sizeof(unsigned));
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
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)8 << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, looked up once per device
// (in host code the array's name is only a host-side stand-in, not a device
// address).
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
    size_t bi = sizeof(double) * OBJ_STRIDE * (size_t)n1 * count;
    size_t bp = sizeof(double) * 7 * (size_t)nblk * count;
    bi = (bi + 255) & ~(size_t)255;
    if (bi + bp > NOALLOC_SCRATCH_BYTES)
        return fail(ctx, GOSMA_EINVAL,
                    "eval_objective_grad_noalloc: count * (128 n1 + 56 ceil((n1^2 + n1 n2) / 512)) bytes "
                    "exceeds the 8 MiB scratch; use fewer poses per call");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    void *scratch = nullptr;
    int rc = noalloc_scratch(ctx, &scratch);
    if (rc) return rc;
    double *di = (double *)scratch, *dp = (double *)((char *)scratch + bi);
    obj_prep<<<dim3((n1 + 127) / 128, count), 128, 0, ctx->stream>>>(ctx->mix, count, d_x, di);
    ++ctx->launches;
    obj_pairs<<<dim3(nblk, count), OBJ_BLOCK, 0, ctx->stream>>>(ctx->mix, count, d_x, di, dp, nblk);
    ++ctx->launches;
    obj_final<<<(count + 63) / 64, 64, 0, ctx->stream>>>(count, d_x, dp, nblk, d_out);
    ++ctx->launches;
    e = cudaGetLastError();
    return e == cudaSuccess ? GOSMA_OK : cuda_fail(ctx, e, "launch(objective, no-alloc)");
}

