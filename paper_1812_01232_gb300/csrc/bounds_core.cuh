// Per-cube Theorem 1 bounds: the hot loop of GOSMA (Algorithm 1, "evaluate
// the bounds of the sub-cubes in parallel").
//
// One thread group (a block, part of a block, or half a warp for the
// smallest mixtures) evaluates one sub-cube C_r x C_t at a time:
//   pre-pass (cube_prepare): R_r0 by Rodrigues' formula in double-float
//            arithmetic (hi/lo FP32 pairs), the rotation uncertainty psi_r
//            (Lemma 2) as an outward-rounded half-angle cosine/sine, and the
//            cuboid as double-floats, per cube (the solvers share the parts
//            that siblings have in common);
//   phase 1  per image component j: u_j = R_r0^T mu_2j; per model component
//            i: v_i, kappa_1i(t0), the kappa interval [a_i, b_i] over the
//            cuboid, psi_t(mu_1i) (Lemma 3) -- all in double-float FP32, into
//            shared memory;
//   phase 2  diagonal self terms, all cross pairs (i, j) and all self pairs
//            i < m; threads own model rows and stream the partner arrays
//            from shared memory (broadcast reads within a warp);
//   phase 3  group reduction of the four sums in double-float.
// No FP64 arithmetic runs per component or per pair: FP64 is ~1/64 of the
// FP32 rate on this GPU.
//
// The closed forms follow Theorem 1 with the translation dependence of
// kappa bounded over [a_i, b_i]:
//   K^2 = (k1 - k2)^2 + 4 k1 k2 cos^2(B/2),
//   K - k1 - k2 = -4 k1 k2 sin^2(B/2) / (k1 + k2 + K)     (no cancellation),
//   Z(x) = e^x g(x) / x with g(x) = 1 - e^{-2x}.
// Every rounding that could raise a lower bound is covered, in the direction
// that lowers the cube's lower bound (see the error budget below).
#pragma once

#include "dfloat.cuh"
#include "gosma_internal.cuh"
#include "packed.cuh"

namespace gosma {

// psi_t = pi as a float: the largest float below pi (the nearest float,
// (float)M_PI, lies above it), so that a rotation cube whose angle is capped
// at pi still wins the split rule's tie with a mean inside the cuboid, as in
// the FP64 comparison (ties split rotation).
constexpr float PSI_PI_F = 3.14159250f;

// Per-cube data written by the pre-pass (144 bytes): the rotation and the
// translation cuboid as double-floats.  The terms of the point-dependent
// rotation uncertainty angle are a record of the same size in a second
// array, n records after the first (n = the records of the call), written
// and read only in that mode.
struct CubePrep {
    float Rh[9], Rl[9];  // R_r0 (row-major)
    float th[3], tl[3];  // t0
    float wh[3], wl[3];  // translation half-widths
    float Cr, Sr;        // cos / sin of psi_r / 2 (cosine rounded down, sine up)
    float psi_r;
    int infeasible;      // rotation cube wholly outside the pi-ball
    float pad[2];
};
// point-dependent psi_r (Lemma 2), from the images c_k = J_r(r0) d_k / 2 of
// four vertices d_k = (+-h, +-h, h) of the rotation cube (the other four are
// their negatives): pj[8k .. 8k+2] c_k (hi), pj[8k+3 .. 8k+5] c_k (lo),
// pj[8k+6], pj[8k+7] |c_k|^2 (hi, lo); pj[32] 3 h^2 / 8 and pj[33]
// 64 u^2 max_k |c_k| (both rounded up); pj[34..35] padding
struct CubePrepPoint {
    float pj[36];
};
static_assert(sizeof(CubePrep) == 144 && sizeof(CubePrepPoint) == sizeof(CubePrep), "CubePrep layout");
constexpr int PREP_WORDS = sizeof(CubePrep) / 4;
constexpr int PREP_POINT_WORDS = sizeof(CubePrepPoint) / 4;
// the point-dependent record of cube c of n: the second array
__device__ __forceinline__ CubePrepPoint *prep_point(CubePrep *prep, int n, int c) {
    return reinterpret_cast<CubePrepPoint *>(prep + n) + c;
}
__device__ __forceinline__ const CubePrepPoint *prep_point(const CubePrep *prep, int n, int c) {
    return reinterpret_cast<const CubePrepPoint *>(prep + n) + c;
}

// shared-memory scalars of one cube
struct CubeShared {
    CubePrep rot;
    CubePrepPoint rotp;
    int infeasible;         // no feasible pose in the cube: the rotation cube ...
    int cub_infeasible;     // ... or the translation cuboid (every point within zeta of a mean)
    int centre_infeasible;  // t0 within zeta of a mean
    unsigned spsi_max;      // max over i of sin(psi_t,i / 2), as float bits
    float red[8][32];       // block reduction: 4 double-float sums x warps
};

// Directions are formed as double-floats (hi + lo equals the unit vector to
// ~2^-44); the pair loops read the FP32 parts only and carry the low parts'
// effect as an absolute allowance (GOSMA_HI_ALLOW), and the model rows' low
// parts serve the point-dependent rotation angle.  The pair loops take
// partners two at a time into the two lanes of packed FP32x2 registers, so
// the records are stored in pairs, lanes interleaved: one 16-byte load gives
// two aligned lane pairs.  A missing
// partner of an odd count is a copy of the last one with zero weight.
//   JP (image columns 2p, 2p+1; lanes a, b), 4 float4 per pair:
//     (ux_a, ux_b, uy_a, uy_b) (uz_a, uz_b, k2_a, k2_b) (lqc_a, lqc_b, lqb_a, lqb_b) (lz_a, lz_b, Q_a, Q_b)
//     u = R_r0^T mu_2j (FP32 part), k2 = kappa_2j, lqc and lqb the column
//     factor's log2 for the centre term and for the bound (MixDev::lQ2c,
//     lQ2b); lz, the last low part of u, and Q, the factor itself, unread
//   MP (model rows 2q, 2q+1), 6 float4 per pair:
//     (vx_a, vx_b, vy_a, vy_b) (vz_a, vz_b, a_a, a_b) (lx_a, lx_b, ly_a, ly_b) (lz_a, lz_b, b_a, b_b)
//     (k0_a, k0_b, cp_a, cp_b) (sp_a, sp_b, Aw_a, Aw_b)
//     v = v_i (hi, then lo), [a, b] the kappa interval, k0 = kappa_1i(t0),
//     cp, sp = cos, sin of psi_t,i / 2, Aw the row factor of the self bound
//   UP (model rows 2q, 2q+1): (Uw_a, Uw_b), the row factor of the centre term
struct SmemArrays {
    float4 *JP;
    float4 *MP;
    float2 *UP;
};

__host__ __device__ inline size_t bounds_smem_arrays_bytes(int n1, int n2) {
    const size_t p1 = (size_t)(n1 + 1) / 2, p2 = (size_t)(n2 + 1) / 2;
    return p2 * 4 * sizeof(float4) + p1 * (6 * sizeof(float4) + sizeof(float2)) + 16;
}

__device__ inline SmemArrays carve(float *base, int n1, int n2) {
    SmemArrays s;
    float4 *p = reinterpret_cast<float4 *>(base);
    const int p1 = (n1 + 1) / 2, p2 = (n2 + 1) / 2;
    s.JP = p;
    s.MP = p + 4 * p2;
    s.UP = reinterpret_cast<float2 *>(p + 4 * p2 + 6 * p1);
    return s;
}

// Field f (0..11, in the order of MP above: vx vy vz a lx ly lz b k0 cp sp Aw)
// of model row i.
__device__ __forceinline__ float &mp_at(const SmemArrays &sm, int i, int f) {
    return reinterpret_cast<float *>(sm.MP)[24 * (i >> 1) + 2 * f + (i & 1)];
}
__device__ __forceinline__ float &up_at(const SmemArrays &sm, int i) {
    return reinterpret_cast<float *>(sm.UP)[i];
}
// Field f (0..7: ux uy uz k2 lqc lqb lz Q) of image column j.
__device__ __forceinline__ float &jp_at(const SmemArrays &sm, int j, int f) {
    return reinterpret_cast<float *>(sm.JP)[16 * (j >> 1) + 2 * f + (j & 1)];
}
enum { MP_VX = 0, MP_VY, MP_VZ, MP_A, MP_LX, MP_LY, MP_LZ, MP_B, MP_K0, MP_CP, MP_SP, MP_AW };
enum { JP_UX = 0, JP_UY, JP_UZ, JP_K2, JP_LQC, JP_LQB, JP_LZ, JP_Q };

__device__ inline int pow2ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Rodrigues' formula R = I + A [r]x + B [r]x^2 (A = sin|r| / |r|, B = (1 -
// cos|r|) / |r|^2) in double-float arithmetic, R to ~2^-44 absolute: the
// FP64 form's sincos and divisions cost the FP64 unit (about 1/64 of the
// FP32 rate here) more than all the rest of the pre-pass.  Below |r| = 1e-3
// A and B come from their series (the next terms are below 2^-60).
__device__ inline void rodrigues_df(const double r0[3], float Rh[9], float Rl[9]) {
    df x, y, z;
    split_double(r0[0], x.h, x.l);
    split_double(r0[1], y.h, y.l);
    split_double(r0[2], z.h, z.l);
    const df xx = df_mul(x, x), yy = df_mul(y, y), zz = df_mul(z, z);
    const df th2 = df_add(df_add(xx, yy), zz);
    const df one = {1.f, 0.f};
    df A, B;
    if (th2.h < 1e-6f) {
        A = df_add(one, df_mul(th2, df{fmaf(th2.h, 1.f / 120.f, -1.f / 6.f), 0.f}));
        B = df_add(df{0.5f, 0.f}, df_mul(th2, df{fmaf(th2.h, 1.f / 720.f, -1.f / 24.f), 0.f}));
    } else {
        const df th = df_mul(th2, df_rsqrt(th2, rsqrta(th2.h)));
        df sn, cs;
        df_sincos(th, sn, cs);
        A = df_div(sn, th);
        B = df_div(df_sub(one, cs), th2);
    }
    const df xy = df_mul(x, y), xz = df_mul(x, z), yz = df_mul(y, z);
    const df Ax = df_mul(A, x), Ay = df_mul(A, y), Az = df_mul(A, z);
    const df Bxy = df_mul(B, xy), Bxz = df_mul(B, xz), Byz = df_mul(B, yz);
    const df R[9] = {df_sub(one, df_mul(B, df_add(yy, zz))), df_sub(Bxy, Az), df_add(Bxz, Ay),
                     df_add(Bxy, Az), df_sub(one, df_mul(B, df_add(xx, zz))), df_sub(Byz, Ax),
                     df_sub(Bxz, Ay), df_add(Byz, Ax), df_sub(one, df_mul(B, df_add(xx, yy)))};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        Rh[k] = R[k].h;
        Rl[k] = R[k].l;
    }
}

// Pre-pass for one cube, in three parts that depend on different parts of
// the cube, so that a caller can share them between cubes (the eight children
// of a translation split share their parent's rotation cube, the children of
// any split share a level): Rodrigues' formula (Sec. 4.1) and the
// rotation-cube terms, Lemma 2 read as angle(R_r p, R_r0 p) <= |r - r0| <=
// sqrt(3) r_hw capped at pi, and the translation cuboid split into
// double-floats.
//
// The rotation-cube part: R_r0 (FP64 Rodrigues' formula in the
// point-dependent mode, whose vertex terms reuse its FP64 quantities; else
// the double-float form), whether the cube lies wholly outside the pi-ball,
// and the point-dependent terms when pt is given.
__device__ inline void cube_prepare_rotation(const double r0[3], double rhw, CubePrep &o, CubePrepPoint *pt) {
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double e = fabs(r0[k]) - rhw;
        if (e > 0) d2 += e * e;
    }
    o.infeasible = d2 > M_PI * M_PI ? 1 : 0;
    if (!pt) {
        rodrigues_df(r0, o.Rh, o.Rl);
        return;
    }
    double th2 = r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2];
    double th = sqrt(th2), A, B;
    if (th < 1e-8) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
    } else {
        double s, c;
        sincos(th, &s, &c);
        A = s / th;
        B = (1.0 - c) / th2;
    }
    double x = r0[0], y = r0[1], z = r0[2];
    double R[9] = {1.0 - B * (y * y + z * z), -A * z + B * x * y,        A * y + B * x * z,
                   A * z + B * x * y,         1.0 - B * (x * x + z * z), -A * x + B * y * z,
                   -A * y + B * x * z,        A * x + B * y * z,         1.0 - B * (x * x + y * y)};
    for (int k = 0; k < 9; ++k) split_double(R[k], o.Rh[k], o.Rl[k]);
    // right Jacobian J_r(r0) = I - B [r0]x + C [r0]x^2, C = (|r0| - sin|r0|) / |r0|^3
    // (R_{r0 + d} = R_r0 R_{J_r d} to first order), and the vertex images J_r d / 2
    const double C = th < 1e-6 ? 1.0 / 6.0 - th2 / 120.0 : (th - A * th) / (th2 * th);
    const double S[9] = {0.0, -z, y, z, 0.0, -x, -y, x, 0.0};
    double J[9];
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
            double s2 = S[3 * p] * S[q] + S[3 * p + 1] * S[3 + q] + S[3 * p + 2] * S[6 + q];
            J[3 * p + q] = (p == q ? 1.0 : 0.0) - B * S[3 * p + q] + C * s2;
        }
    double cmax = 0.0;
    for (int k = 0; k < 4; ++k) {
        double d[3] = {rhw, rhw, rhw};
        if (k > 0) d[k - 1] = -rhw;
        double n2 = 0.0;
        for (int p = 0; p < 3; ++p) {
            double c = 0.5 * (J[3 * p] * d[0] + J[3 * p + 1] * d[1] + J[3 * p + 2] * d[2]);
            split_double(c, pt->pj[8 * k + p], pt->pj[8 * k + 3 + p]);
            n2 += c * c;
        }
        split_double(n2, pt->pj[8 * k + 6], pt->pj[8 * k + 7]);
        cmax = fmax(cmax, sqrt(n2));
    }
    pt->pj[32] = __double2float_ru(0.375 * rhw * rhw);
    pt->pj[33] = __double2float_ru(64.0 * 0x1p-48 * cmax);
    pt->pj[34] = pt->pj[35] = 0.f;
}

__device__ inline void cube_prepare_psi_r(double rhw, CubePrep &o) {
    double pr = sqrt(3.0) * rhw;
    if (pr > M_PI) pr = M_PI;
    double sh, ch;
    sincos(0.5 * pr, &sh, &ch);
    o.Sr = __double2float_ru(sh);
    o.Cr = __double2float_rd(ch);
    o.psi_r = (float)pr;
}

__device__ inline void cube_prepare_translation(const double t0[3], const double thw[3], CubePrep &o) {
    for (int k = 0; k < 3; ++k) {
        split_double(t0[k], o.th[k], o.tl[k]);
        split_double(thw[k], o.wh[k], o.wl[k]);
    }
    o.pad[0] = o.pad[1] = 0.f;
}

__device__ inline void cube_prepare(const double r0[3], double rhw, const double t0[3], const double thw[3],
                                    CubePrep &o, CubePrepPoint *pt) {
    cube_prepare_rotation(r0, rhw, o, pt);
    cube_prepare_psi_r(rhw, o);
    cube_prepare_translation(t0, thw, o);
}

// Lemma 2, point-dependent form, for one model direction v (the unit vector
// v_i at t0, as a double-float): with w(r) the vector part of the relative
// quaternion q(r0)^* q(r), sin(angle(R_r v, R_r0 v) / 2) = |w(r) x v|, and
// w(r0 + d) = J_r(r0) d / 2 + rho with |rho| <= |d|^2 / 8 (the second
// derivative of the quaternion exponential along a line is at most |d/2|^2),
// so over the cube sin(psi_r / 2) <= max_k |c_k x v| + 3 h^2 / 8 (the
// first-order term is a norm of a linear map: largest at a vertex).
// |c_k x v|^2 = |c_k|^2 - (c_k . v)^2 is formed in double-float (error at most
// 8 u^2 |c|^2: no cancellation beyond a factor 4, since the largest of the
// four is at least |c|^2 / 4 for any v), its square root by one double-float
// Newton step from the FP32 estimate (relative error below 8 u^2), and the
// sum with 3 h^2 / 8 and the 64 u^2 |c|max allowance is rounded up once: the
// sine is at most one unit in the last place above the exact bound, as the
// point-independent sine.
// The cosine sqrt(1 - s^2) is formed the same way and rounded down (0 where
// it is below 1/16, i.e. psi_r above 172 degrees).  Cr, Sr (the
// point-independent pair) are replaced when the bound is smaller.
__device__ __forceinline__ void point_psi_r(const CubePrepPoint &P, df vx, df vy, df vz, float &Cr, float &Sr) {
    const float U2 = GOSMA_U * GOSMA_U;
    // read at every call: loads hoisted out of the row loop would hold the
    // 36 words in registers across the pair loops
    const volatile float *pj = P.pj;
    df best = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const df c0 = {pj[8 * k], pj[8 * k + 3]}, c1 = {pj[8 * k + 1], pj[8 * k + 4]},
                 c2 = {pj[8 * k + 2], pj[8 * k + 5]};
        const df dot = df_dot3(c0, vx, c1, vy, c2, vz);
        const df n2 = df_sub(df{pj[8 * k + 6], pj[8 * k + 7]}, df_mul(dot, dot));
        if (n2.h > best.h || (n2.h == best.h && n2.l > best.l)) best = n2;
    }
    float lh = 0.f, ll = 0.f;
    if (best.h > 0.f) {
        const float r = sqrta(best.h);
        const df rr = two_prod(r, r);
        const float e = (((best.h - rr.h) - rr.l) + best.l) * (0.5f * rcpa(r));  // best.h - rr.h is exact
        const df lin = fast_two_sum(r, e);
        lh = lin.h;
        ll = lin.l;
    }
    const float s = __fadd_ru(lh, __fadd_ru(ll, __fadd_ru(pj[32], pj[33])));
    if (s < Sr) {
        Sr = s;
        // cos(psi_r / 2) = sqrt(1 - s^2): 1 - s^2 as an exact double-float but
        // for one rounding of its tail (below u^2 / 2)
        const df p = two_prod(s, s);
        const df t = two_sum(1.f, -p.h);
        const df w = two_sum(t.h, t.l - p.l);
        float c = 0.f;
        if (w.h > 0.00390625f) {  // 1/256: cos(psi_r / 2) above 1/16
            const float r = sqrta(w.h);
            const df rr = two_prod(r, r);
            const float e = (((w.h - rr.h) - rr.l) + w.l) * (0.5f * rcpa(r));
            c = __fadd_rd(r, __fmaf_rd(-64.f * U2, r, e));
        }
        Cr = c;
    }
}

// g(x) = 1 - e^{-2x}, so that Z(x) = e^x g(x) / x (Eq. Z).  For x >= 9,
// g(x) > 1 - 2^-25 and rounds to 1 in FP32.
__device__ __forceinline__ float gZ(float x) { return 1.f - ex2a(-2.f * GOSMA_LOG2E * x); }

// Every pair term is written in linear form:
//   Z(K) / (Z(k1) Z(k2)) = e^{K - k1 - k2} * (g(K) / K) * (k1 / g(k1)) * (k2 / g(k2)),
// the last two factors (times the weights phi) being per-row and per-column
// multipliers.  Only K - k1 - k2 goes through the exponential, and
//   K^2 = (k1 - k2)^2 + k1 k2 |v + u|^2,   K - k1 - k2 = -k1 k2 |v - u|^2 / (k1 + k2 + K)
// for unit directions v, u at angle theta (|v -+ u| = 2 sin, 2 cos of theta/2).
//
// Error budget (u = 2^-24; approximate instructions as documented for PTX:
// ex2 2^-22.5, rcp and sqrt 2^-23, rsqrt 2^-22.9 relative, i.e. <= 3u, 2u,
// 2u, 2.2u; gosma_selftest_approx measures them on the device):
//  * |v - u| and |v + u| from the directions' FP32 parts: the differences
//    and sums rounded (u/2 per component), so sin(theta/2), cos(theta/2)
//    carry <= 5.5u relative (squares 3.5u, sqrt 2u), and the missing low
//    parts 0.87u absolute (GOSMA_HI_ALLOW);
//  * the half-angle sine/cosine of s = psi_t + psi_r (row constants, evaluated
//    in double-float, rounded once) carry <= u relative;
//  * hence sin(B/2) = sin(theta/2) cos(s/2) - cos(theta/2) sin(s/2) is off by
//    at most 7.5u (sin(theta/2) + sin(s/2)) + 1.3u =: es; cos(B/2) enters only
//    squared (in K and in cos B = 2 cos^2(B/2) - 1), bounded from the sine
//    bounds as 1 - sin^2 (one rounding of the fused s^2 - 1: no square
//    root);
//  * K: 3.5u (sqrt 2u, K^2 2.5u); the self pair rounds its K bounds outward
//    by 4u and 5u, the cross pair leaves them to the slacks below;
//  * the exponent K - k1 - k2 (log2 units) carries <= 11u relative (15u in
//    the cross pair, whose K and cos^2 are not rounded outward), and
//    rounding the ex2 argument adds 0.5u of it: the argument moves by
//    12u |exponent| (cross pair 16u) in the safe direction;
//  * the factor outside the exponential: ex2 3u, rcp 2u, four products 4u,
//    one sum 1u: 10u relative = 14.4u in log2 units (TERM_SLACK);
//  * row weights, chunk sums (CHUNK-1 terms, plain FP32) and compensated row
//    sums: applied once per row with directed rounding.
#define GOSMA_TERM_SLACK (15.f * GOSMA_U)
// The pair terms take the unit directions' FP32 parts only: |v -+ u| is then
// within sqrt(3) u of its exact value (each low part is at most u/2), so the
// sine and cosine of theta/2 within 0.87u, and a sine built from both
// (sin(theta/2) cos(s/2) -+ cos(theta/2) sin(s/2)) within 0.87u (cos + sin)
// <= 1.23u: an absolute allowance of 1.3u on every half-angle sine.
#define GOSMA_HI_ALLOW (1.3f * GOSMA_U)
// The cross pair's term slack (GOSMA_CROSS_SLACK, 20u): GOSMA_TERM_SLACK and
// the smallest K's rounding without an outward factor (3.5u relative in
// g(K)/K: 5u in log2 units).  It rides on the log2 of the image column's
// factor (MixDev::lQ2b), which enters the exponent instead of multiplying
// the term: lQ2b = log2 Q_j + 20u + u (|log2 Q_j| + 1), rounded up, so that
// the exponent's one rounding (0.5u of |DL| + |lQ2b|) stays covered: its
// |DL| part by the exponent's relative slack, its |lQ2b| part by the last
// term (and the product by Q, one of the four above, is gone).
constexpr int CHUNK = 8;

struct RowCross {
    float vx, vy, vz, wx, wy, wz;  // v_i hi / lo
    float a, b, k0, Cs, Ss, esS, A4;
};

// The row constants of RowCross in both lanes of packed pairs, for
// cross_pair2.  hCs = Cs / 2, nhSs = -Ss / 2, nA4 = -A4 (exact: the halves
// multiply |v - u| and |v + u|, which are 2 sin and 2 cos of theta/2).
struct RowCross2 {
    float2 vx, vy, vz;
    float2 a, b, k0, hCs, nhSs, esS, nA4;
    __device__ __forceinline__ explicit RowCross2(const RowCross &R)
        : vx(bc2(R.vx)), vy(bc2(R.vy)), vz(bc2(R.vz)), a(bc2(R.a)), b(bc2(R.b)), k0(bc2(R.k0)),
          hCs(bc2(0.5f * R.Cs)), nhSs(bc2(-0.5f * R.Ss)), esS(bc2(R.esS)), nA4(bc2(-R.A4)) {}
};

__device__ __forceinline__ float2 sqrt2a(float2 x) { return make_float2(sqrta(x.x), sqrta(x.y)); }
__device__ __forceinline__ float2 rcp2a(float2 x) { return make_float2(rcpa(x.x), rcpa(x.y)); }
__device__ __forceinline__ float2 ex2_2a(float2 x) { return make_float2(ex2a(x.x), ex2a(x.y)); }

// Two cross pairs (i, j) and (i, j') at once, lane x for column j and lane y
// for j' (their JP records P0 .. P2): adds to pl the upper bound of each
// pair's term over the cube (Theorem 1, Eq. K1i2j_ub with B of Eq.
// K1i2j_ub_B) and to pc the term at the centre (Lemma 1), both without the
// row multipliers; the column factor enters each exponent as its log2.
// Every operation is per lane, rounded to nearest as a scalar FP32
// operation would be (the error budget above holds per lane).
//   |v -+ u|^2 from the directions' FP32 parts, the centre term in the linear
//   form above, then the bound: B = max(0, theta - s), s = psi_t,i + psi_r
//   (Cs, Ss = cos, sin of s/2); cos^2(B/2) from the sine bounds as
//   1 - s^2 (one rounding of 1 - s^2, 2u outward); K(a) - a - k2 with the
//   smallest sine and the largest K; the smallest K over kappa_1 in [a, b]
//   (minimiser -k2 cos B, clamped), from below; g(K)/K <= min(1/K, 2).
// Forms chosen for the packed instructions, exact rewritings: 1 - s^2 is
// taken as -(s^2 - 1) (rounding to nearest is symmetric), -k2 cos B as
// -(k2 cos B), and the exponent's relative slack as one fused
// DL (1 - 16u) + slack (DL <= 0: a product of non-negative factors and
// -log2 e; 1 - 16u is a float, and one rounding replaces two).
__device__ __forceinline__ void cross_pair2(const RowCross2 &R, float4 P0, float4 P1, float4 P2, float2 &pl,
                                            float2 &pc) {
    const float U = GOSMA_U;
    const float2 k2 = make_float2(P1.z, P1.w), lqc = make_float2(P2.x, P2.y), lqb = make_float2(P2.z, P2.w);
    const float2 ux = make_float2(P0.x, P0.y), uy = make_float2(P0.z, P0.w), uz = make_float2(P1.x, P1.y);
    // the directions' FP32 parts only (their low parts move sin and cos of
    // theta/2 by at most 0.87u, which the row's allowance esS carries)
    const float2 dx = sub2(R.vx, ux), dy = sub2(R.vy, uy), dz = sub2(R.vz, uz);
    const float2 px = add2(R.vx, ux), py = add2(R.vy, uy), pz = add2(R.vz, uz);
    const float2 x2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));  // |v - u|^2 = 4 sin^2(theta/2)
    const float2 y2 = fma2(px, px, fma2(py, py, mul2(pz, pz)));  // |v + u|^2 = 4 cos^2(theta/2)
    // centre: kappa_1i(t0) = k0, angle theta
    const float2 kk = mul2(R.k0, k2);
    const float2 dk0 = sub2(R.k0, k2);
    const float2 K0 = sqrt2a(fma2(dk0, dk0, mul2(kk, y2)));
    const float2 den0 = add2(add2(R.k0, k2), K0);
    const float2 K0c = max2(K0, 1e-20f);
    const float2 r0 = rcp2a(mul2(den0, K0c));
    float2 w0 = mul2(den0, r0);
    if (K0.x < 9.f) w0.x = K0.x < 1e-3f ? 2.f - 2.f * K0.x : gZ(K0.x) * w0.x;
    if (K0.y < 9.f) w0.y = K0.y < 1e-3f ? 2.f - 2.f * K0.y : gZ(K0.y) * w0.y;
    pc = fma2(ex2_2a(fma2(mul2(mul2(kk, x2), mul2(K0c, r0)), bc2(-GOSMA_LOG2E), lqc)), w0, pc);
    // bound: B = max(0, theta - s)
    // sx, sy = 2 sin, 2 cos of theta/2; the halves sit in the row constants,
    // so sB and es round exactly as from sin(theta/2) and cos(theta/2)
    const float2 sx = sqrt2a(x2), sy = sqrt2a(y2);
    const float2 sB = fma2(sx, R.hCs, mul2(sy, R.nhSs));
    const float2 es = fma2(bc2(3.75f * U), sx, R.esS);
    const float2 slo = max2(sub2(sB, es), 0.f);
    const float2 shi = min2(add2(max2(sB, 0.f), es), 1.f);
    // cos^2(B/2) = 1 - sin^2(B/2) from the sine bounds, as -q with q = s^2 - 1
    // rounded once (q < 0: both sines stay below 1).  No outward factor on
    // the cosines or on K: their roundings (K within 3.5u) are covered by the
    // exponent's relative slack (16u) and the term slack (20u).
    const float2 q1 = fma2(slo, slo, bc2(-1.f)), q2 = fma2(shi, shi, bc2(-1.f));
    const float2 nak4 = mul2(R.nA4, k2);  // -4 a k2
    const float2 dka = sub2(R.a, k2);
    const float2 Khi = sqrt2a(fma2(nak4, q1, mul2(dka, dka)));
    const float2 nkc = mul2(k2, fma2(bc2(2.f), q2, bc2(1.f)));  // -k2 cos B
    const float2 ks = make_float2(fminf(fmaxf(nkc.x, R.a.x), R.b.x), fminf(fmaxf(nkc.y, R.a.y), R.b.y));
    const float2 dks = sub2(ks, k2);
    const float2 Kmin = sqrt2a(fma2(mul2(mul2(bc2(-4.f), ks), k2), q2, mul2(dks, dks)));
    const float2 den = add2(add2(R.a, k2), Khi);
    const float2 Kc = max2(Kmin, 1e-20f);
    const float2 r = rcp2a(mul2(den, Kc));
    const float2 DL = mul2(mul2(mul2(nak4, mul2(slo, slo)), mul2(Kc, r)), bc2(GOSMA_LOG2E));
    const float2 w = min2(mul2(den, r), 2.f);
    const float2 arg = fma2(DL, bc2(1.f - 16.f * U), lqb);
    pl = fma2(ex2_2a(arg), w, pl);
}

struct RowSelf {
    float vx, vy, vz, wx, wy, wz;
    float a, b, k0, cp, sp;
};

// The row constants of RowSelf in both lanes of packed pairs, for self_pair2.
// (the half-angle pair of psi_i/2 halved, hcp = cp / 2, hsp = sp / 2,
// nhsp = -sp / 2, exact: see RowCross2)
struct RowSelf2 {
    float2 vx, vy, vz;
    float2 a, b, k0, hcp, hsp, nhsp;
    __device__ __forceinline__ explicit RowSelf2(const RowSelf &R)
        : vx(bc2(R.vx)), vy(bc2(R.vy)), vz(bc2(R.vz)), a(bc2(R.a)), b(bc2(R.b)), k0(bc2(R.k0)),
          hcp(bc2(0.5f * R.cp)), hsp(bc2(0.5f * R.sp)), nhsp(bc2(-0.5f * R.sp)) {}
};

// Two self pairs (i, m) and (i, m') at once, lane x for partner m and lane y
// for m' (their MP records P0 .. P5 and UP record Um): adds to pl the lower
// bound of each pair's term over the cuboid (Theorem 1, Eq. K1i1j_lb with A
// of Eq. K1i1j_lb_A) and to pc the centre term, both without the row
// multipliers; per lane as a scalar FP32 evaluation would round.
//   The bound: A = min(pi, theta + psi_i + psi_m), the half-angle pair of
//   (psi_i + psi_m)/2 formed here in FP32 (2u each): sin(A/2) carries
//   <= 9.5u (sin(theta/2) + sin(psi/2)), cos(A/2) <= 14u; cos^2(A/2) from
//   the sine bounds as 1 - sin^2 (A/2 <= pi/2; one rounding, 2u outward);
//   K(b_i, b_m) - b_i - b_m with the largest sine
//   and the smallest K; the largest K over the four corners of
//   [a_i, b_i] x [a_m, b_m], from above; g(K)/K from below: >= 2 - 2K for
//   small K, g rounded with <= 64u error otherwise.
// Besides the rewritings of cross_pair2, -sin((psi_i+psi_m)/2) / 2 is formed as
// 0 - hS (exact; hS >= 0, a sum of products of non-negative half-angle
// sines and cosines), and the exponent's slack as DL (1 + 12u) - slack in
// one fused operation (DL <= 0).
__device__ __forceinline__ void self_pair2(const RowSelf2 &R, float4 P0, float4 P1, float4 P2, float4 P3, float4 P4,
                                           float4 P5, float2 Um, float2 &pl, float2 &pc) {
    const float U = GOSMA_U;
    const float2 am = make_float2(P1.z, P1.w), bm = make_float2(P3.z, P3.w), k0m = make_float2(P4.x, P4.y),
                 cpm = make_float2(P4.z, P4.w), spm = make_float2(P5.x, P5.y), Am = make_float2(P5.z, P5.w);
    const float2 ux = make_float2(P0.x, P0.y), uy = make_float2(P0.z, P0.w), uz = make_float2(P1.x, P1.y);
    const float2 dx = sub2(R.vx, ux), dy = sub2(R.vy, uy), dz = sub2(R.vz, uz);  // FP32 parts, as cross_pair2
    const float2 px = add2(R.vx, ux), py = add2(R.vy, uy), pz = add2(R.vz, uz);
    const float2 x2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    const float2 y2 = fma2(px, px, fma2(py, py, mul2(pz, pz)));
    // centre
    const float2 kk = mul2(R.k0, k0m);
    const float2 dk0 = sub2(R.k0, k0m);
    const float2 K0 = sqrt2a(fma2(dk0, dk0, mul2(kk, y2)));
    const float2 den0 = add2(add2(R.k0, k0m), K0);
    const float2 K0c = max2(K0, 1e-20f);
    const float2 r0 = rcp2a(mul2(den0, K0c));
    float2 w0 = mul2(den0, r0);
    if (K0.x < 9.f) w0.x = K0.x < 1e-3f ? 2.f - 2.f * K0.x : gZ(K0.x) * w0.x;
    if (K0.y < 9.f) w0.y = K0.y < 1e-3f ? 2.f - 2.f * K0.y : gZ(K0.y) * w0.y;
    pc = fma2(ex2_2a(mul2(mul2(mul2(kk, x2), mul2(K0c, r0)), bc2(-GOSMA_LOG2E))), mul2(w0, Um), pc);
    // bound: A = min(pi, theta + psi_i + psi_m)
    const float2 sx = sqrt2a(x2), sy = sqrt2a(y2);          // 2 sin, 2 cos of theta/2
    const float2 hC = fma2(R.hcp, cpm, mul2(R.nhsp, spm));  // cos((psi_i + psi_m)/2) / 2
    const float2 hS = fma2(R.hsp, cpm, mul2(R.hcp, spm));   // sin((psi_i + psi_m)/2) / 2
    const float2 cA = fma2(sy, hC, mul2(sx, sub2(bc2(0.f), hS)));
    const float2 sA = fma2(sx, hC, mul2(sy, hS));
    // 10u (sin(theta/2) + sin(psi/2)) as 5u sx + 20u hS (two roundings, at
    // most 2u of it: still above the 9.5u the sine carries)
    const float2 es = fma2(bc2(5.f * U), sx, fma2(bc2(20.f * U), hS, bc2(GOSMA_HI_ALLOW)));
    const float2 t1 = add2(sA, es);
    const float2 shi = make_float2(cA.x <= 16.f * U ? 1.f : fminf(t1.x, 1.f), cA.y <= 16.f * U ? 1.f : fminf(t1.y, 1.f));
    const float2 slo = max2(sub2(sA, es), 0.f);
    // cos^2(A/2) bounds as in cross_pair2
    const float2 q2 = fma2(shi, shi, bc2(-1.f)), q1 = fma2(slo, slo, bc2(-1.f));
    const float2 clo2 = mul2(q2, bc2(-(1.f - 2.f * U))), chi2 = mul2(q1, bc2(-(1.f + 2.f * U)));
    const float2 bb = mul2(R.b, bm);
    const float2 dbb = sub2(R.b, bm);
    const float2 Klo = mul2(sqrt2a(fma2(dbb, dbb, mul2(mul2(bc2(4.f), bb), clo2))), bc2(1.f - 4.f * U));
    const float2 c4 = mul2(bc2(4.f), chi2);
    const float2 q1a = sub2(R.a, am), q2a = sub2(R.a, bm), q3a = sub2(R.b, am);
    const float2 ca = mul2(c4, R.a), cb = mul2(c4, R.b);
    const float2 e1 = fma2(q1a, q1a, mul2(ca, am));
    const float2 e2 = fma2(q2a, q2a, mul2(ca, bm));
    const float2 e3 = fma2(q3a, q3a, mul2(cb, am));
    const float2 e4 = fma2(dbb, dbb, mul2(c4, bb));
    const float2 Kmax = mul2(make_float2(sqrta(fmaxf(fmaxf(e1.x, e2.x), fmaxf(e3.x, e4.x))),
                                         sqrta(fmaxf(fmaxf(e1.y, e2.y), fmaxf(e3.y, e4.y)))),
                             bc2(1.f + 5.f * U));
    const float2 den = add2(add2(R.b, bm), Klo);
    const float2 r = rcp2a(mul2(den, Kmax));
    const float2 DL = mul2(mul2(mul2(bb, mul2(shi, shi)), mul2(Kmax, r)), bc2(-4.f * GOSMA_LOG2E));
    float2 w = mul2(den, r);
    if (Kmax.x < 9.f) w.x = Kmax.x < 0.25f ? fmaxf(2.f - 2.f * Kmax.x, 0.f) : gZ(Kmax.x) * w.x * (1.f - 64.f * U);
    if (Kmax.y < 9.f) w.y = Kmax.y < 0.25f ? fmaxf(2.f - 2.f * Kmax.y, 0.f) : gZ(Kmax.y) * w.y * (1.f - 64.f * U);
    const float2 arg = fma2(DL, bc2(1.f + 12.f * U), bc2(-GOSMA_TERM_SLACK));
    pl = fma2(ex2_2a(arg), mul2(w, Am), pl);
}

// k coth(k) / 2 = Z(2k) / Z(k)^2, the diagonal self term without phi^2
// (relative error <= 12u).
__device__ __forceinline__ float half_kcothk(float k) {
    float e = ex2a(-2.f * GOSMA_LOG2E * k);
    return 0.5f * k * (1.f + e) * rcpa(1.f - e);
}

// A group of GT threads (half a warp, or whole warps) of a BLOCK-thread
// block works on one cube; the block holds BLOCK / GT groups.  gsync is the
// group's barrier: the block barrier when one group is the block, a warp
// barrier over the group's lanes for a half-warp group, else named barrier
// 1 + gid for the group's GT threads.  Half-warp groups serve the smallest
// mixtures (at most 16 model rows), two cubes to a warp.
template <int GT>
__device__ __forceinline__ unsigned group_lanes() {
    if constexpr (GT >= 32) {
        return 0xffffffffu;
    } else {
        return ((1u << GT) - 1u) << ((threadIdx.x & 31) & ~(unsigned)(GT - 1));
    }
}

template <int BLOCK, int GT>
__device__ __forceinline__ void gsync(int gid) {
    static_assert((GT == 16 || GT % 32 == 0) && BLOCK % GT == 0 && BLOCK / GT <= 15, "groups of half or whole warps");
    if constexpr (GT == BLOCK) {
        __syncthreads();
    } else if constexpr (GT < 32) {
        __syncwarp(group_lanes<GT>());
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "n"(GT) : "memory");
    }
}

// Lanes of the group that hold the four sums after group_reduce_df: sum k
// in gtid k * sum_lane_stride<GT>().
template <int GT>
__host__ __device__ constexpr int sum_lane_stride() {
    return GT >= 32 ? 8 : GT / 4;
}

// Warp + group reduction of four double-floats, scattered: on return, the
// group's thread gtid = k sum_lane_stride (k = 0..3; lanes 0, 8, 16, 24 of
// its first warp, or 0, 4, 8, 12 of a half-warp group) holds the group's
// total of v[k].  Within a warp the first two levels halve the sums between
// the lanes (after xor 16, lanes 0-15 carry sums 0 and 1 and lanes 16-31
// sums 2 and 3; after xor 8, lanes 8k .. 8k + 7 carry sum k), and the last
// three reduce within eight lanes: 7 double-float additions per lane instead
// of 20 for four full reductions, and no barrier for a one-warp group.  A
// half-warp group does the same within its 16 lanes (xor 8, 4, then 2, 1).
template <int BLOCK, int GT>
__device__ inline df group_reduce_df(const df v[4], CubeShared &cs, int gid, int gtid) {
    const unsigned mask = group_lanes<GT>();
    auto xshfl = [mask](df x, int o) {
        return df{__shfl_xor_sync(mask, x.h, o), __shfl_xor_sync(mask, x.l, o)};
    };
    if constexpr (GT == 16) {
        const bool h8 = gtid & 8, h4 = gtid & 4;
        const df g0 = df_add(h8 ? v[2] : v[0], xshfl(h8 ? v[0] : v[2], 8));
        const df g1 = df_add(h8 ? v[3] : v[1], xshfl(h8 ? v[1] : v[3], 8));
        df b = df_add(h4 ? g1 : g0, xshfl(h4 ? g0 : g1, 4));
        b = df_add(b, xshfl(b, 2));
        return df_add(b, xshfl(b, 1));
    } else {
        const int lane = gtid & 31, warp = gtid >> 5;
        const bool h16 = lane & 16, h8 = lane & 8;
        const df g0 = df_add(h16 ? v[2] : v[0], xshfl(h16 ? v[0] : v[2], 16));
        const df g1 = df_add(h16 ? v[3] : v[1], xshfl(h16 ? v[1] : v[3], 16));
        df b = df_add(h8 ? g1 : g0, xshfl(h8 ? g0 : g1, 8));
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) b = df_add(b, xshfl(b, o));
        if constexpr (GT > 32) {
            if ((lane & 7) == 0) {
                cs.red[2 * (lane >> 3)][warp] = b.h;
                cs.red[2 * (lane >> 3) + 1][warp] = b.l;
            }
            gsync<BLOCK, GT>(gid);
            if (gtid < 32 && (lane & 7) == 0) {
                const int k = lane >> 3;
                df s = {cs.red[2 * k][0], cs.red[2 * k + 1][0]};
                for (int w = 1; w < GT / 32; ++w) s = df_add(s, {cs.red[2 * k][w], cs.red[2 * k + 1][w]});
                b = s;
            }
        }
        return b;
    }
}

// Blocks per SM the bound kernels ask the compiler to fit.  32- and 64-thread
// blocks work on small mixtures, whose cubes are short and latency-bound, so
// they need every resident warp (32 blocks of one warp, 16 of two: 64
// registers per thread); 128- and 256-thread blocks keep 8 and 3 blocks
// (64 and 85 registers), which is what the pair loops need without spills.
template <int BLOCK>
constexpr int bound_min_blocks() {
    return BLOCK <= 64 ? 1024 / BLOCK : BLOCK == 128 ? 8 : BLOCK == 256 ? 3 : 1;
}

// Work distribution of the persistent bound kernels: cubes are handed out
// one at a time from a device counter that is zero at launch, so that groups
// drawing cheap cubes (infeasible ones, children reusing cached self sums)
// take more of them.  Every thread of the group calls it; the leading barrier
// keeps the group's slot from being overwritten before all its threads have
// read it.
template <int BLOCK, int GT>
__device__ __forceinline__ int next_cube(int *counter, int *slot, int gid, int gtid) {
    gsync<BLOCK, GT>(gid);
    if (gtid == 0) *slot = atomicAdd(counter, 1);
    gsync<BLOCK, GT>(gid);
    return *slot;
}
__device__ __forceinline__ int next_cube(int *counter, int *slot) {
    __syncthreads();
    if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
    __syncthreads();
    return *slot;
}

// The whole per-cube computation.  Every thread of the group (GT threads,
// group gid of the block, gtid its thread) must call it with the same cube,
// its own CubeShared and shared arrays; the sums in out (shared memory) are
// valid for the whole group on return.  need_self = 0 skips the self pairs (the caller reuses cached
// self sums).  reuse_rows = 1 skips the model rows (phase 1b): the group's
// previous call was for a cube of the same mixtures and the same translation
// cuboid (a sibling after a rotation split), and neither call needs its self
// sums; the rows, the cuboid's feasibility flags and psi_t max depend on the
// cuboid alone.
template <int BLOCK, int GT = BLOCK>
__device__ void cube_bounds(const MixDev &mx, const CubePrep &prep, const CubePrepPoint *pt, df zeta2, bool need_self,
                            CubeShared &cs, const SmemArrays &sm, CubeSums &out, int gid = 0,
                            int gtid = threadIdx.x, bool reuse_rows = false) {
    const int tid = gtid;
    const int n1 = mx.n1, n2 = mx.n2;
    const float U = GOSMA_U;
    // Small groups serve small mixtures, whose rows hold few pairs: there one
    // copy of each pair loop, with the edge pairs masked at run time, runs
    // fewer instructions per cube than peeled edge pairs; larger groups peel
    // the masked edge pairs off their long loops.
    constexpr bool COMPACT_LOOPS = GT <= 64;
    for (int k = tid; k < PREP_WORDS; k += GT)
        reinterpret_cast<float *>(&cs.rot)[k] = reinterpret_cast<const float *>(&prep)[k];
    if (mx.psi_point)
        for (int k = tid; k < PREP_POINT_WORDS; k += GT)
            reinterpret_cast<float *>(&cs.rotp)[k] = reinterpret_cast<const float *>(pt)[k];
    if (tid == 0) {
        cs.infeasible = prep.infeasible;
        if (!reuse_rows) {
            cs.cub_infeasible = 0;
            cs.centre_infeasible = 0;
            cs.spsi_max = 0u;
        }
    }
    gsync<BLOCK, GT>(gid);

    // ---------------- phase 1a: image columns u_j = R_r0^T mu_2j (double-float)
    // (an odd count gets a copy of the last column with zero weight as the
    // partner of the last pair)
    for (int j = tid; j < n2 + (n2 & 1); j += GT) {
        const int jj = j < n2 ? j : n2 - 1;
        df m0 = {mx.mu2h[3 * jj], mx.mu2l[3 * jj]}, m1 = {mx.mu2h[3 * jj + 1], mx.mu2l[3 * jj + 1]},
           m2 = {mx.mu2h[3 * jj + 2], mx.mu2l[3 * jj + 2]};
        df u[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            u[c] = df_dot3({cs.rot.Rh[c], cs.rot.Rl[c]}, m0, {cs.rot.Rh[3 + c], cs.rot.Rl[3 + c]}, m1,
                           {cs.rot.Rh[6 + c], cs.rot.Rl[6 + c]}, m2);
        jp_at(sm, j, JP_UX) = u[0].h;
        jp_at(sm, j, JP_UY) = u[1].h;
        jp_at(sm, j, JP_UZ) = u[2].h;
        jp_at(sm, j, JP_K2) = mx.kappa2[jj];
        jp_at(sm, j, JP_LQC) = j < n2 ? mx.lQ2c[jj] : __int_as_float(0xff800000);  // -inf: no term
        jp_at(sm, j, JP_LQB) = j < n2 ? mx.lQ2b[jj] : __int_as_float(0xff800000);
        jp_at(sm, j, JP_LZ) = u[2].l;
        jp_at(sm, j, JP_Q) = j < n2 ? mx.Q2[jj] : 0.f;
    }

    // ---------------- phase 1b: model rows (double-float geometry)
    Acc dsl, dsu;  // diagonal self terms of this thread
    dsl.zero();
    dsu.zero();
    for (int i = reuse_rows ? n1 : tid; i < n1; i += GT) {
        df c[3], w[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c[k] = df_sub({mx.mu1h[3 * i + k], mx.mu1l[3 * i + k]}, {cs.rot.th[k], cs.rot.tl[k]});
            w[k] = {cs.rot.wh[k], cs.rot.wl[k]};
        }
        df d = df_norm2(c[0], c[1], c[2]);
        if (d.h < zeta2.h || (d.h == zeta2.h && d.l < zeta2.l)) atomicOr(&cs.centre_infeasible, 1);
        bool inside = true;
        float e2 = 0.f, f2 = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            df ac = c[k].h < 0.f ? df{-c[k].h, -c[k].l} : c[k];
            df ex = df_sub(ac, w[k]);  // |c_k| - half-width: positive outside the slab
            inside &= ex.h < 0.f || (ex.h == 0.f && ex.l <= 0.f);
            float e = fmaxf(ex.h, 0.f);
            float f = ac.h + w[k].h;
            e2 = fmaf(e, e, e2);
            f2 = fmaf(f, f, f2);
        }
        if (f2 * (1.f + 8.f * U) < zeta2.h) atomicOr(&cs.cub_infeasible, 1);
        float is2 = mx.inv_sig2[i];
        // kappa range over the feasible part of the cuboid (nearest point clamped to
        // zeta); each end carries <= 6u (distance 1u, squares and sums 4u, fma 1u)
        float a = __fmul_rd(fmaf(fmaxf(e2, zeta2.h), is2, 1.f), 1.f - 7.f * U);
        float b = __fmul_ru(fmaf(f2, is2, 1.f), 1.f + 7.f * U);
        float k0 = fmaf(d.h, is2, 1.f);
        // unit direction v_i = c / |c| (double-float)
        df v[3] = {{1.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (d.h > 0.f) {
            df r = df_rsqrt(d, rsqrta(d.h));
#pragma unroll
            for (int k = 0; k < 3; ++k) v[k] = df_mul(c[k], r);
        }
        // Lemma 3: the largest angle between mu - t_vertex and mu - t0, as sin^2(psi/2);
        // pi when mu is in the cuboid or a vertex angle reaches pi/2.  FP32 picks the
        // vertex, double-float evaluates it.
        float sp2 = 1.f;
        if (!inside) {
            const float cx = c[0].h, cy = c[1].h, cz = c[2].h, d2 = d.h;
            const float thx = cs.rot.wh[0], thy = cs.rot.wh[1], thz = cs.rot.wh[2];
            float m1 = -1.f, m2 = -1.f;
            int best = 0;
            bool wide = false;
            for (int vtx = 0; vtx < 8; ++vtx) {
                float ox = (vtx & 1) ? thx : -thx;
                float oy = (vtx & 2) ? thy : -thy;
                float oz = (vtx & 4) ? thz : -thz;
                float ax = cx - ox, ay = cy - oy, az = cz - oz;
                float crx = fmaf(oy, cz, -oz * cy), cry = fmaf(oz, cx, -ox * cz), crz = fmaf(ox, cy, -oy * cx);
                float cr2 = fmaf(crx, crx, fmaf(cry, cry, crz * crz));
                float ac = fmaf(ax, cx, fmaf(ay, cy, az * cz));
                float a2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
                float nn = sqrta(a2 * d2);
                wide |= ac <= 64.f * U * nn;
                // sin^2(psi/2) = sin^2 psi / (2 (1 + cos psi)) = |o x c|^2 / (2 |a||c| (|a||c| + a.c))
                float s2 = cr2 * rcpa(2.f * nn * (nn + ac));
                if (s2 > m1) {
                    m2 = m1;
                    m1 = s2;
                    best = vtx;
                } else {
                    m2 = fmaxf(m2, s2);
                }
            }
            if (!wide) {
                // chord between the unit directions of mu - t_vertex and mu - t0, double-float
                df q[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    df o = ((best >> k) & 1) ? w[k] : df{-w[k].h, -w[k].l};
                    q[k] = df_sub(c[k], o);
                }
                df qn = df_norm2(q[0], q[1], q[2]);
                df rq = df_rsqrt(qn, rsqrta(qn.h));
                float ch2 = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    df qh = df_mul(q[k], rq);
                    float dk = (qh.h - v[k].h) + (qh.l - v[k].l);
                    ch2 = fmaf(dk, dk, ch2);
                }
                // the FP32 runner-up bounds every other vertex (FP32 error <= 24u)
                sp2 = fminf(fmaxf(0.25f * ch2 * (1.f + 8.f * U), m2 * (1.f + 32.f * U)), 1.f);
            }
        }
        float sps = sp2 >= 1.f ? 1.f : fminf(sqrta(sp2) * (1.f + 3.f * U), 1.f);
        float cps = sps >= 1.f ? 0.f : sqrta(fmaxf(fmaf(-sps, sps, 1.f), 0.f)) * (1.f - 3.f * U);
        atomicMax(&cs.spsi_max, __float_as_uint(sps));
        float ph = mx.phi1f[i];
        // phi_i a_i / g(a_i) from below, phi_i k0_i / g(k0_i)
        float Aw = a < 9.f ? ph * a * rcpa(gZ(a)) * (1.f - 12.f * U) : __fmul_rd(ph * a, 1.f - 3.f * U);
        float Uw = k0 < 9.f ? ph * k0 * rcpa(gZ(k0)) : ph * k0;
        // the row's record, and for the last row of an odd count also its copy with
        // zero weights (the partner of the last pair)
        for (int r = i; r <= (i == n1 - 1 && (n1 & 1) ? n1 : i); ++r) {
            mp_at(sm, r, MP_VX) = v[0].h;
            mp_at(sm, r, MP_VY) = v[1].h;
            mp_at(sm, r, MP_VZ) = v[2].h;
            mp_at(sm, r, MP_A) = a;
            mp_at(sm, r, MP_LX) = v[0].l;
            mp_at(sm, r, MP_LY) = v[1].l;
            mp_at(sm, r, MP_LZ) = v[2].l;
            mp_at(sm, r, MP_B) = b;
            mp_at(sm, r, MP_K0) = k0;
            mp_at(sm, r, MP_CP) = cps;
            mp_at(sm, r, MP_SP) = sps;
            mp_at(sm, r, MP_AW) = r == i ? Aw : 0.f;
            up_at(sm, r) = r == i ? Uw : 0.f;
        }
        // diagonal self term phi_i^2 k coth(k) / 2, smallest over [a_i, b_i] at a_i
        dsl.add(ph * ph * half_kcothk(a) * (1.f - 16.f * U));
        dsu.add(ph * ph * half_kcothk(k0));
    }
    gsync<BLOCK, GT>(gid);

    // per-thread sums (double-float): self lb, cross ub, self centre, cross centre
    df T[4] = {fast_two_sum(dsl.s, dsl.c), {0.f, 0.f}, fast_two_sum(dsu.s, dsu.c), {0.f, 0.f}};
    T[0] = df_scale(T[0].h, T[0].l, 1.f - 3.f * U);

    const bool infeasible = cs.infeasible || cs.cub_infeasible;
    if (!infeasible) {
        // ---------------- phase 2a: cross pairs
        const int Ti = n1 >= GT ? GT : pow2ceil(n1);
        const int Tj = GT / Ti;
        const int ti = tid % Ti, tj = tid / Ti;
        for (int i = ti; i < n1; i += Ti) {
            // rotation uncertainty of this row: point-independent, or the
            // point-dependent form of Lemma 2 when the mixtures ask for it
            float Cr = cs.rot.Cr, Sr = cs.rot.Sr;
            RowCross R;
            R.vx = mp_at(sm, i, MP_VX);
            R.vy = mp_at(sm, i, MP_VY);
            R.vz = mp_at(sm, i, MP_VZ);
            R.wx = mp_at(sm, i, MP_LX);
            R.wy = mp_at(sm, i, MP_LY);
            R.wz = mp_at(sm, i, MP_LZ);
            R.a = mp_at(sm, i, MP_A);
            R.b = mp_at(sm, i, MP_B);
            R.k0 = mp_at(sm, i, MP_K0);
            R.A4 = 4.f * R.a;
            if (mx.psi_point) point_psi_r(cs.rotp, df{R.vx, R.wx}, df{R.vy, R.wy}, df{R.vz, R.wz}, Cr, Sr);
            const float cps = mp_at(sm, i, MP_CP), sps = mp_at(sm, i, MP_SP);
            // s = psi_t,i + psi_r as half-angle cosine/sine (double-float, rounded once);
            // s >= pi means B = 0 everywhere
            df cc = two_prod(cps, Cr), ssp = two_prod(sps, Sr), sc = two_prod(sps, Cr), cs2 = two_prod(cps, Sr);
            R.Cs = (cc.h - ssp.h) + (cc.l - ssp.l);
            R.Ss = (sc.h + cs2.h) + (sc.l + cs2.l);
            if (R.Cs <= 0.f) {
                R.Cs = 0.f;
                R.Ss = 1.f;
            }
            R.esS = fmaf(7.5f * U, R.Ss, GOSMA_HI_ALLOW);
            // phi_i b_i / g(b_i) from above (for b >= 9 g rounds to 1, at most 2^-25 high),
            // times the chunk and row-sum allowances
            float Bw = R.b < 9.f ? mx.phi1f[i] * R.b * rcpa(gZ(R.b)) * (1.f + 12.f * U) : mx.phi1f[i] * R.b;
            Bw = __fmul_ru(Bw, 1.f + (float)(CHUNK + 6) * U);
            Acc cl, cu;
            cl.zero();
            cu.zero();
            // the row's columns [j0, j1) in stored pairs p0 .. p1 - 1, pair p to thread
            // p mod Tj; each lane keeps its own FP32 chunk sum of at most CHUNK terms.
            // A pair with a column outside the range (before j0 when j0 is odd, at j1
            // when j1 is odd) runs with that column's weight set to zero (its log2 to -inf).
            const RowCross2 R2(R);
            float2 pl = make_float2(0.f, 0.f), pc = make_float2(0.f, 0.f);
            int cnt = 0;
            const int j0 = mx.rj0 ? mx.rj0[i] : 0, j1 = mx.rj1 ? mx.rj1[i] : n2;
            const int p0 = j0 >> 1, p1 = (j1 + 1) >> 1;
            const int pa = (j0 & 1) ? p0 : -1, pb = (j1 & 1) ? p1 - 1 : -1;
            auto step = [&](int q, bool ma, bool mb) {
                const float4 A = sm.JP[4 * q], B = sm.JP[4 * q + 1];
                float4 C = sm.JP[4 * q + 2];
                if (ma) C.x = C.z = __int_as_float(0xff800000);  // log2 of a zero weight
                if (mb) C.y = C.w = __int_as_float(0xff800000);
                cross_pair2(R2, A, B, C, pl, pc);
                if (++cnt == CHUNK) {
                    cl.add(pl.x);
                    cl.add(pl.y);
                    cu.add(pc.x);
                    cu.add(pc.y);
                    pl = pc = make_float2(0.f, 0.f);
                    cnt = 0;
                }
            };
            int q = p0 + tj;
            if constexpr (COMPACT_LOOPS) {
#pragma unroll 1
                for (; q < p1; q += Tj) step(q, q == pa, q == pb);
            } else {
                if (q == pa) {
                    step(q, true, q == pb);
                    q += Tj;
                }
                const int qend = pb >= 0 ? pb : p1;
#pragma unroll 1
                for (; q < qend; q += Tj) step(q, false, false);
                if (q == pb) step(q, false, true);
            }
            cl.add(pl.x);
            cl.add(pl.y);
            cu.add(pc.x);
            cu.add(pc.y);
            T[1] = df_add(T[1], df_scale(cl.s, cl.c, Bw));
            T[3] = df_add(T[3], df_scale(cu.s, cu.c, up_at(sm, i)));
        }
        // ---------------- phase 2b: self pairs i < m, rows paired (p, n1-2-p) for balance
        if (need_self && n1 > 1) {
            const int NP = n1 / 2;  // ceil((n1 - 1) / 2)
            const int Si = NP >= GT ? GT : pow2ceil(NP);
            const int Sj = GT / Si;
            const int si = tid % Si, sj = tid / Si;
            for (int pp = si; pp < NP; pp += Si) {
                for (int h = 0; h < 2; ++h) {
                    int i = h == 0 ? pp : n1 - 2 - pp;
                    if (h == 1 && i == pp) break;
                    RowSelf R;
                    R.vx = mp_at(sm, i, MP_VX);
                    R.vy = mp_at(sm, i, MP_VY);
                    R.vz = mp_at(sm, i, MP_VZ);
                    R.wx = mp_at(sm, i, MP_LX);
                    R.wy = mp_at(sm, i, MP_LY);
                    R.wz = mp_at(sm, i, MP_LZ);
                    R.a = mp_at(sm, i, MP_A);
                    R.b = mp_at(sm, i, MP_B);
                    R.k0 = mp_at(sm, i, MP_K0);
                    R.cp = mp_at(sm, i, MP_CP);
                    R.sp = mp_at(sm, i, MP_SP);
                    Acc sl, su;
                    sl.zero();
                    su.zero();
                    // partners m in [i + 1, mend) in stored pairs, as the columns above; a
                    // pair holding row i itself (i even) or a row at mend (mend odd) runs
                    // with that row's weights Aw and Uw set to zero
                    const RowSelf2 R2(R);
                    float2 pl = make_float2(0.f, 0.f), pc = make_float2(0.f, 0.f);
                    int cnt = 0;
                    const int mend = mx.rm1 ? mx.rm1[i] : n1;
                    const int q0 = (i + 1) >> 1, q1 = (mend + 1) >> 1;
                    const int qa = ((i + 1) & 1) ? q0 : -1, qb = (mend & 1) ? q1 - 1 : -1;
                    auto step = [&](int q, bool ma, bool mb) {
                        const float4 *P = sm.MP + 6 * q;
                        const float4 A = P[0], B = P[1], C = P[2], D = P[3], E = P[4];
                        float4 F = P[5];
                        float2 Um = sm.UP[q];
                        if (ma) F.z = Um.x = 0.f;
                        if (mb) F.w = Um.y = 0.f;
                        self_pair2(R2, A, B, C, D, E, F, Um, pl, pc);
                        if (++cnt == CHUNK) {
                            sl.add(pl.x);
                            sl.add(pl.y);
                            su.add(pc.x);
                            su.add(pc.y);
                            pl = pc = make_float2(0.f, 0.f);
                            cnt = 0;
                        }
                    };
                    int q = q0 + sj;
                    if constexpr (COMPACT_LOOPS) {
#pragma unroll 1
                        for (; q < q1; q += Sj) step(q, q == qa, q == qb);
                    } else {
                        if (q == qa) {
                            step(q, true, q == qb);
                            q += Sj;
                        }
                        const int qend = qb >= 0 ? qb : q1;
#pragma unroll 1
                        for (; q < qend; q += Sj) step(q, false, false);
                        if (q == qb) step(q, false, true);
                    }
                    sl.add(pl.x);
                    sl.add(pl.y);
                    su.add(pc.x);
                    su.add(pc.y);
                    // both orders (i, m) and (m, i): factor 2, exact
                    float Awi = __fmul_rd(2.f * mp_at(sm, i, MP_AW), 1.f - (float)(CHUNK + 3) * U);
                    T[0] = df_add(T[0], df_scale(sl.s, sl.c, Awi));
                    T[2] = df_add(T[2], df_scale(su.s, su.c, 2.f * up_at(sm, i)));
                }
            }
        }
    }

    // ---------------- phase 3: block reduction (double-float)
    const df tot = group_reduce_df<BLOCK, GT>(T, cs, gid, gtid);
    // The four lanes that hold the sums (lanes 0, 8, 16, 24 of the group's
    // first warp; 0, 4, 8, 12 of a half-warp group) convert them to FP64
    // together: an FP64 instruction costs the FP64 unit a whole warp's time
    // however few lanes run it.
    // (the self sums only when computed: callers that skip them use cached ones)
    constexpr int SL = sum_lane_stride<GT>();
    if (tid < 4 * SL && tid % SL == 0) {
        const int k = tid / SL;
        const double d = (need_self || (k & 1)) ? (double)tot.h + (double)tot.l : 0.0;
        if (k == 0)
            out.self_lb = d;
        else if (k == 1)
            out.cross_ub = d;
        else if (k == 2)
            out.self_c = d;
        else
            out.cross_c = d;
    }
    if (tid == 0) {
        out.psi_r = cs.rot.psi_r;
        float smax = __uint_as_float(cs.spsi_max);
        out.psi_t_max = smax >= 1.f ? PSI_PI_F : fminf(2.f * asinf(smax), PSI_PI_F);
        out.feasible = !infeasible;
        out.centre_feasible = !cs.centre_infeasible;
    }
    gsync<BLOCK, GT>(gid);
}

// Theorem 1's bounds of a cube from its FP64 sums: lb = self_lb - 2 cross_ub
// less 1e-12 (self_lb + 2 cross_ub), the allowance for the double-float
// partial sums (~2^-44), and ub = self_c - 2 cross_c.  Called by lanes 0
// and 1 of a group together (first = lane 0): lane 1 forms ub in the same
// FP64 instructions as lane 0 forms lb (an FP64 instruction costs the FP64
// unit a whole warp's time however few lanes run it); both lanes return
// both.  The sums are finite.
__device__ __forceinline__ void cube_lb_ub(double self_lb, double cross_ub, double self_c, double cross_c, bool first,
                                           double &lb, double &ub) {
    const double x = first ? self_lb : self_c, y = first ? cross_ub : cross_c;
    const double S = x + 2.0 * y;
    const double v = x - 2.0 * y;
    const double w = v - (first ? 1e-12 : 0.0) * S;
    const double o = __shfl_xor_sync(0x3u << ((threadIdx.x & 31) & ~1u), w, 1);
    lb = first ? w : o;
    ub = first ? o : w;
}

// Final per-cube values from the sums (thread 0).
__device__ inline void finish_bound(const CubeSums &s, gosma_bound &o) {
    if (!s.feasible) {
        const double inf = __longlong_as_double(0x7ff0000000000000LL);
        o.lb = o.ub = o.self_lb = o.cross_ub = o.self_c = o.cross_c = inf;
    } else {
        double S = s.self_lb + 2.0 * s.cross_ub;
        // allowance for the double-float additions of the partial sums (~2^-44)
        o.lb = s.self_lb - 2.0 * s.cross_ub - 1e-12 * S;
        o.ub = s.centre_feasible ? s.self_c - 2.0 * s.cross_c : __longlong_as_double(0x7ff0000000000000LL);
        o.self_lb = s.self_lb;
        o.cross_ub = s.cross_ub;
        o.self_c = s.self_c;
        o.cross_c = s.cross_c;
    }
    o.psi_r = s.psi_r;
    o.psi_t_max = s.psi_t_max;
}

}  // namespace gosma
