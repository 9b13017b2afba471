// Branch-and-bound building blocks shared by the single-problem and the
// multi-problem drivers: the 64-byte queue node, cell decoding, branching
// (Sec. 4.1) and the orderable FP32 keys.
#pragma once

#include <stdint.h>
#include <string.h>

#include "bounds_core.cuh"

namespace gosma {

struct Node {
    double lb;
    double self_lb, self_c;  // self sums of the translation cuboid (valid when flags & 1)
    uint32_t r[3], t[3];     // cell coordinates at levels lr, lt
    uint16_t lr, lt;
    float psit;              // max_i psi_t over the cuboid
    uint32_t flags;
    float ubf;               // upper bound at the centre, FP32 (batched solver)
};
static_assert(sizeof(Node) == 64, "node layout");

struct Domain {
    double t_lo[3], t_hi[3];
};

constexpr uint32_t DEAD = 0xFFFFFFFFu;
constexpr int MAX_LEVEL = 30;
constexpr int SEL_BLOCK = 256;
constexpr int SEL_ITEMS = 8;  // keys per thread in the scan kernels
constexpr int SEL_TILE = SEL_BLOCK * SEL_ITEMS;

__host__ __device__ inline uint32_t order_key(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float key_value(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

__host__ __device__ inline double psi_r_level(int lr) {
    double p = sqrt(3.0) * ldexp(M_PI, -lr);
    return p < M_PI ? p : M_PI;
}

// A node's cell as FP64 geometry: the rotation cube (centre, half-width) and
// the translation cuboid (centre, half-widths), each from its own level.
__host__ __device__ inline void decode_rotation(const Node &n, double r0[3], double &rhw) {
    const double rh = ldexp(M_PI, -(int)n.lr);
    rhw = rh;
    for (int k = 0; k < 3; ++k) r0[k] = -M_PI + (2.0 * n.r[k] + 1.0) * rh;
}
__host__ __device__ inline void decode_translation(const Node &n, const Domain &d, double t0[3], double thw[3]) {
    for (int k = 0; k < 3; ++k) {
        const double th = ldexp(d.t_hi[k] - d.t_lo[k], -(int)n.lt - 1);
        thw[k] = th;
        t0[k] = d.t_lo[k] + (2.0 * n.t[k] + 1.0) * th;
    }
}
__host__ __device__ inline void decode(const Node &n, const Domain &d, CubeGeom &g) {
    decode_rotation(n, g.r0, g.rhw);
    decode_translation(n, d, g.t0, g.thw);
}

// The split rule's comparison psi_r(lr) >= psit, taken in FP32: psit is a
// float, so the FP64 comparison holds exactly when psit is at most the
// largest float at or below psi_r(lr).  psi_r(lr) = fl(sqrt(3) pi) 2^-lr for
// lr >= 1 (scaling by 2^-lr is exact) and pi at lr = 0, so that float is
// PSI_R_F 2^-lr, PSI_R_F = fl(sqrt(3) pi) = 5.441398092702653 rounded down to
// a float, and PSI_PI_F at lr = 0.  (FP64 instructions cost the FP64 unit a
// whole warp's time, and every thread of a bound kernel tests its run's
// parent.)
constexpr float PSI_R_F = 0x1.5c3fdcp+2f;
__host__ __device__ inline float psi_r_level_floor(int lr) {
    if (lr == 0) return PSI_PI_F;
    const uint32_t e = (uint32_t)(127 - lr) << 23;  // 2^-lr, 1 <= lr < 127
    float s;
    memcpy(&s, &e, 4);
    return PSI_R_F * s;
}

// Child k of a parent (Sec. 4.1: the split halves the rotation cube or the
// translation cuboid, whichever has the greater angular uncertainty).
__host__ __device__ inline bool split_rotation(const Node &p) {
    if (p.lr >= MAX_LEVEL) return false;
    if (p.lt >= MAX_LEVEL) return true;
    return p.psit <= psi_r_level_floor(p.lr);
}

__host__ __device__ inline Node child_of(const Node &p, int k, bool rot) {
    Node c = p;
    if (rot) {
        c.lr = p.lr + 1;
        for (int a = 0; a < 3; ++a) c.r[a] = 2u * p.r[a] + ((k >> a) & 1u);
    } else {
        c.lt = p.lt + 1;
        for (int a = 0; a < 3; ++a) c.t[a] = 2u * p.t[a] + ((k >> a) & 1u);
        c.flags &= ~1u;  // the cuboid changed: self sums must be recomputed
    }
    return c;
}

}  // namespace gosma
