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
    const float *phi1f;    // n1: phi_1i
    const double *sigma1d; // n1: sigma_1i (FP64, objective kernels)
    const double *phi1d;   // n1
    const double *mu2;     // n2 x 3 (unit)
    const float *kappa2;   // n2
    const float *Q2;       // n2: phi_2j kappa_2j / (1 - e^{-2 kappa_2j})  (computed in FP64)
    const double *kappa2d; // n2
    const double *phi2d;   // n2
    const float *mu1h, *mu1l;  // n1 x 3: mu1 as double-floats (hi, lo)
    const float *mu2h, *mu2l;  // n2 x 3: unit mu2 as double-floats
    // n2: log2 Q2 from FP64: lQ2c rounded to nearest (the centre terms);
    // lQ2b raised by GOSMA_CROSS_SLACK and by u (|log2 Q2| + 1) (the final
    // rounding of a cross bound's exponent, which adds it) and rounded up;
    // -inf for a zero weight
    const float *lQ2c, *lQ2b;
    double zeta;           // point-to-camera limit (Sec. 4.1)
    // Semantic classes (Sec. 4.2); all null for one class.  Pairs interact
    // only within a class: model row i pairs with image columns
    // [rj0[i], rj1[i]) and with model rows below rm1[i]; cls1 / cls2 give
    // each component's class.
    const int *cls1, *cls2;
    const int *rj0, *rj1, *rm1;
    // Rotation uncertainty of the cross pairs (Lemma 2): 0 the point-independent
    // angle sqrt(3) h, 1 the point-dependent angle of each model direction.
    int psi_point;
};

// Feasible translations of a refinement (Sec. 4.1): inside [t_lo, t_hi] and
// at least sqrt(zeta2) from every model mean.
struct SmaBox {
    double t_lo[3], t_hi[3], zeta2;
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
// The cross pair's term slack in log2 units (the error budget in
// bounds_core.cuh): it rides on the log2 of each image column's factor.
#define GOSMA_CROSS_SLACK (20.f * GOSMA_U)
#define GOSMA_LOG2E 1.4426950408889634f

// Relative error assumed for ex2/rcp/rsqrt/sqrt (2^-22) and the absolute +
// relative error assumed for lg2 (2^-22 each).
#define GOSMA_APPROX_REL (4.0f * GOSMA_U)
#define GOSMA_LG2_ABS (4.0f * GOSMA_U)

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
namespace gosma {
struct Mlp;
void mlp_free(Mlp *m);
}  // namespace gosma

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
    unsigned long long mix_hash = 0;  // fingerprint of the staged mixtures (checkpoints)
    void *d_mix = nullptr;  // one allocation holding every mixture array
    gosma::MixDev mix{};

    // rotation uncertainty of the bounds (gosma_set_psi_r_mode): 0 point-independent, 1 point-dependent
    int psi_r_mode = 0;

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

    // batched SMA scratch (sma.cu)
    void *d_sma = nullptr;
    size_t sma_bytes = 0;

    // mixture generation scratch (mixgen.cu)
    void *d_mg = nullptr;
    size_t mg_bytes = 0;

    // per-cube rotation pre-pass (gosma_eval_bounds)
    void *d_rot = nullptr;
    size_t rot_bytes = 0;

    // branch-and-bound state (bnb.cu)
    void *bnb = nullptr;
    // queue-ordering network (mlp.cu)
    gosma::Mlp *mlp = nullptr;
    // error-path testing: the next fail_allocs device allocations fail
    int fail_allocs = 0;
    // kernels may address ordinary host memory (coherent CPU-GPU link with
    // the host page tables): host-buffer calls then skip the staging copies
    bool direct_host = false;

    // number of kernels this context has launched
    long long launches = 0;
};


namespace gosma {
// Device allocations of the library go through here, so that tests can make
// them fail (gosma_debug_fail_allocations) and check the error paths.
inline cudaError_t dev_malloc(gosma_ctx *ctx, void **p, size_t bytes) {
    if (ctx && ctx->fail_allocs > 0) {
        --ctx->fail_allocs;
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}
}  // namespace gosma

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

// sma.cu: FP32-search SMA of count device seeds, seed s on problem d_pid[s]
int sma_refine_many(gosma_ctx *ctx, cudaStream_t st, const MixDev *d_mixes, const SmaBox *d_boxes, const int *d_pid,
                    int max_n1, int max_n2, int count, const double *d_x0, int max_iter, double *d_x, int *d_it,
                    int *d_counter, long long *launches);
void bnb_release(gosma_ctx *ctx);
void bnb_end_run(gosma_ctx *ctx);
}  // namespace gosma
