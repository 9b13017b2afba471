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

__host__ __device__ inline void decode(const Node &n, const Domain &d, CubeGeom &g) {
    double rh = ldexp(M_PI, -(int)n.lr);
    g.rhw = rh;
    for (int k = 0; k < 3; ++k) {
        g.r0[k] = -M_PI + (2.0 * n.r[k] + 1.0) * rh;
        double th = ldexp(d.t_hi[k] - d.t_lo[k], -(int)n.lt - 1);
        g.thw[k] = th;
        g.t0[k] = d.t_lo[k] + (2.0 * n.t[k] + 1.0) * th;
    }
}

// Child k of a parent (Sec. 4.1: the split halves the rotation cube or the
// translation cuboid, whichever has the greater angular uncertainty).
__host__ __device__ inline bool split_rotation(const Node &p) {
    if (p.lr >= MAX_LEVEL) return false;
    if (p.lt >= MAX_LEVEL) return true;
    return psi_r_level(p.lr) >= (double)p.psit;
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
