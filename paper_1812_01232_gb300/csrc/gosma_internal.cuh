// Internal definitions shared by the libgosma translation units: the
// context, the device view of the mixtures, and the FP32 math helpers of
// the bound kernel.  Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gosma.h"

namespace gosma {

// ---------------------------------------------------------------- device views
// Mixture arrays in device memory (structure of arrays).  FP64 copies of the
// means feed the per-cube geometry (differences and rotations are taken in
// FP64, rounded once to FP32); the rest is FP32.
struct MixDev {
    int n1, n2;
    const double *mu1;     // n1 x 3
    const float *inv_sig2; // n1: 1 / sigma_1i^2
    const float *lphi1;    // n1: log2(phi_1i), clamped at -200
    const double *sigma1d; // n1: sigma_1i (FP64, objective kernels)
    const double *phi1d;   // n1
    const double *mu2;     // n2 x 3 (unit)
    const float *kappa2;   // n2
    const float *P2;       // n2: log2(phi_2j) - phiZ2(kappa_2j)  (computed in FP64)
    const double *kappa2d; // n2
    const double *phi2d;   // n2
    double zeta;           // point-to-camera limit (Sec. 4.1)
};

// One sub-cube decoded to FP64 geometry.
struct CubeGeom {
    double r0[3], rhw, t0[3], thw[3];
};

// Per-cube outputs of the bound core (FP64 sums).
struct CubeSums {
    double self_lb, cross_ub, self_c, cross_c;
    float psi_r, psi_t_max;
    int feasible, centre_feasible;
};

// ---------------------------------------------------------------- FP32 helpers
// PTX approximate instructions, so that the error model of the bound kernel
// knows exactly what is computed.  Their accuracy is measured against FP64
// by gosma_selftest_approx; the kernel's slack assumes the bounds below.
#define GOSMA_U 5.9604644775390625e-8f   // 2^-24, unit roundoff of FP32
#define GOSMA_LOG2E 1.4426950408889634f
#define GOSMA_LN2 0.69314718055994531f

// Relative error assumed for ex2/rcp/rsqrt/sqrt (2^-21) and the absolute +
// relative error assumed for lg2 (2^-21 each).
#define GOSMA_APPROX_REL (8.0f * GOSMA_U)
#define GOSMA_LG2_ABS (8.0f * GOSMA_U)

__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2a(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcpa(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrta(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrta(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// phiZ2(x) = log2((1 - e^{-2x}) / x) = (log Z(x) - x) / ln 2, the
// decreasing part of log Z in Eq. (Z), for x >= 0.
//   x >= 9    : -log2 x (the dropped log2(1 - e^{-2x}) is in (-2.3e-8, 0])
//   x >= 1/4  : log2(1 - 2^{-2x log2 e}) - log2 x
//   x <  1/4  : series of log(sinh x / x) - x + log 2
__device__ __forceinline__ float phiZ2(float x) {
    if (x >= 9.0f) return -lg2a(x);
    if (x >= 0.25f) return lg2a(1.0f - ex2a(-2.0f * GOSMA_LOG2E * x)) - lg2a(x);
    float x2 = x * x;
    float s = x2 * (1.0f / 6.0f + x2 * (-1.0f / 180.0f + x2 * (1.0f / 2835.0f)));
    return (GOSMA_LN2 - x + s) * GOSMA_LOG2E;
}

// Bound on |phiZ2 computed - phiZ2 exact| for the value v = phiZ2(x)
// (derivation: rounding of the exponent argument, of 1 - e, and the
// assumed lg2/ex2 errors; one-sided 2.3e-8 of the x >= 9 branch included).
__device__ __forceinline__ float phiZ2_err(float x, float v) {
    float c = x >= 9.0f ? 10.0f * GOSMA_U : (x >= 1.0f ? 32.0f * GOSMA_U : 96.0f * GOSMA_U);
    return c + 4.0f * GOSMA_U * fabsf(v);
}

// Compensated FP32 accumulation (TwoSum): s + c carries the running sum
// with an error of at most 2u|sum| plus second-order terms.
struct Acc {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float x) {
        float t = s + x;
        float z = t - s;
        c += (s - (t - z)) + (x - z);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

}  // namespace gosma

// ---------------------------------------------------------------- context
struct gosma_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int sm_count = 0;

    // mixtures
    bool have_mix = false;
    int n1 = 0, n2 = 0;
    std::vector<double> h_mu1, h_sigma1, h_phi1, h_mu2, h_kappa2, h_phi2;
    double c22 = 0.0;
    void *d_mix = nullptr;  // one allocation holding every mixture array
    gosma::MixDev mix{};

    // domain
    bool have_dom = false;
    double t_lo[3] = {0, 0, 0}, t_hi[3] = {0, 0, 0}, zeta = 0.0;

    // staging for host-pointer calls
    void *d_stage = nullptr;
    size_t stage_bytes = 0;
    void *h_pinned = nullptr;
    size_t pinned_bytes = 0;

    // objective scratch
    void *d_obj = nullptr;
    size_t obj_bytes = 0;

    // branch-and-bound state (bnb.cu)
    void *bnb = nullptr;
};

namespace gosma {
int fail(gosma_ctx *ctx, int code, const std::string &msg);
int cuda_fail(gosma_ctx *ctx, cudaError_t e, const char *what);
int ensure_stage(gosma_ctx *ctx, size_t bytes);
int ensure_pinned(gosma_ctx *ctx, size_t bytes);

// bounds.cu
int launch_bounds(gosma_ctx *ctx, const gosma_cube *d_cubes, int n, gosma_bound *d_out);
size_t bounds_smem_bytes(int n1, int n2);
int bounds_block_size(int n1, int n2);

// objective.cu
int objective_grad_device(gosma_ctx *ctx, int count, const double *h_x, double *h_f, double *h_g);
void bnb_release(gosma_ctx *ctx);
}  // namespace gosma
