// FP64 objective f(R_r, t) of Lemma 1 and its gradient, as kernels over a
// set of poses: per (pose, model component) quantities, per-block partial
// sums over the pairs, and a final reduction that maps the rotation part of
// the gradient to the angle-axis coordinates.  The mixtures are reached
// through a source object so that one set of poses may span several problems
// (batched solving) or share one mixture.
#pragma once

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

__device__ inline void rodrigues_dev(const double r[3], double R[9]) {
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

// All poses share one mixture; pose p's component rows start at p * n1.
struct OneMix {
    MixDev mx;
    __device__ const MixDev &mix(int) const { return mx; }
    __device__ size_t row0(int p) const { return (size_t)p * mx.n1; }
};

// Row i of the per-pose table at pose (R, t).
__device__ __forceinline__ void obj_row(const MixDev &mx, const double R[9], const double t[3], int i, double *o) {
    const double *mu = mx.mu1 + 3 * i;
    double m0 = mu[0] - t[0], m1 = mu[1] - t[1], m2 = mu[2] - t[2];
    double d = sqrt(m0 * m0 + m1 * m1 + m2 * m2);
    double v0 = m0 / d, v1 = m1 / d, v2 = m2 / d;
    double s = mx.sigma1d[i];
    double k = d * d / (s * s) + 1.0;  // Eq. (kappa1)
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

template <class Src>
__global__ void obj_prep(Src src, const double *__restrict__ x, double *__restrict__ idata) {
    const int p = blockIdx.y;
    const MixDev &mx = src.mix(p);
    __shared__ double R[9];
    if (threadIdx.x == 0) rodrigues_dev(x + 6 * p, R);
    __syncthreads();
    const double *t = x + 6 * p + 3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < mx.n1; i += gridDim.x * blockDim.x)
        obj_row(mx, R, t, i, idata + (src.row0(p) + i) * OBJ_STRIDE);
}

// Adds pair q's term to acc: f, df/dt (3), df/domega (3).  Pairs q < n1^2
// are the self pairs (i, j) = (q / n1, q % n1), the rest the cross pairs.
__device__ __forceinline__ void obj_pair(const MixDev &mx, const double *__restrict__ I, const double R[9], long long q,
                                         double acc[7]) {
    const int n1 = mx.n1, n2 = mx.n2;
    const long long nself = (long long)n1 * n1;
    if (q < nself) {
        int i = (int)(q / n1), j = (int)(q % n1);
        if (mx.cls1 && mx.cls1[i] != mx.cls1[j]) return;  // pairs only within a class
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
        if (mx.cls1 && mx.cls1[i] != mx.cls2[j]) return;
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

// f = sum_ij self(i,j) - 2 sum_ij cross(i,j); gradient w.r.t. t and the
// left-perturbation omega of R (d(Rv) = omega x Rv).
template <class Src>
__global__ void __launch_bounds__(OBJ_BLOCK) obj_pairs(Src src, const double *__restrict__ x,
                                                       const double *__restrict__ idata, double *__restrict__ part,
                                                       int nblk) {
    const int p = blockIdx.y;
    const MixDev &mx = src.mix(p);
    __shared__ double R[9];
    __shared__ double red[7][OBJ_BLOCK / 32];
    if (threadIdx.x == 0) rodrigues_dev(x + 6 * p, R);
    __syncthreads();
    const int n1 = mx.n1, n2 = mx.n2;
    const long long nself = (long long)n1 * n1, total = nself + (long long)n1 * n2;
    const double *I = idata + src.row0(p) * OBJ_STRIDE;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    long long q0 = (long long)blockIdx.x * OBJ_CHUNK;
    long long q1 = q0 + OBJ_CHUNK < total ? q0 + OBJ_CHUNK : total;
    for (long long q = q0 + threadIdx.x; q < q1; q += OBJ_BLOCK) obj_pair(mx, I, R, q, acc);
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

// Maps the pair sums s (f, df/dt, df/domega) at angle-axis r to
// o = (f, df/dr, df/dt): d/dr = J_l(r)^T d/domega, with the left Jacobian
// J_l = I + a [r]x + b [r]x^2 of SO(3).
__device__ __forceinline__ void obj_finish(const double r[3], const double s[7], double *o) {
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
    o[0] = s[0];
    for (int c = 0; c < 3; ++c) o[1 + c] = gw[c] - a * rxg[c] + b * (r[c] * rg - th2 * gw[c]);
    for (int c = 0; c < 3; ++c) o[4 + c] = s[1 + c];
}

// One warp per pose (launch OBJ_FINAL_WARPS warps per block): lanes sum
// strided block partials, then a warp reduction in a fixed order.
constexpr int OBJ_FINAL_WARPS = 4;
template <int = 0>
__global__ void obj_final(int count, const double *__restrict__ x, const double *__restrict__ part, int nblk,
                          double *__restrict__ out) {
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (p >= count) return;  // warp-uniform
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = lane; b < nblk; b += 32)
        for (int k = 0; k < 7; ++k) s[k] += part[((size_t)p * nblk + b) * 7 + k];
    for (int k = 0; k < 7; ++k)
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
    if (lane == 0) obj_finish(x + 6 * p, s, out + 7 * p);
}

}  // namespace gosma
