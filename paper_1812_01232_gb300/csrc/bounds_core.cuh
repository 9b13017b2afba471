// Per-cube Theorem 1 bounds: the hot loop of GOSMA (Algorithm 1, "evaluate
// the bounds of the sub-cubes in parallel").
//
// One thread block evaluates one sub-cube C_r x C_t at a time:
//   pre-pass (cube_prepare): R_r0 by Rodrigues' formula in FP64, split into
//            FP32 hi/lo pairs, the rotation uncertainty psi_r (Lemma 2) as an
//            outward-rounded half-angle cosine/sine, and the cuboid as
//            double-floats, one thread per cube;
//   phase 1  per image component j: u_j = R_r0^T mu_2j; per model component
//            i: v_i, kappa_1i(t0), the kappa interval [a_i, b_i] over the
//            cuboid, psi_t(mu_1i) (Lemma 3) -- all in double-float FP32, into
//            shared memory;
//   phase 2  diagonal self terms, all cross pairs (i, j) and all self pairs
//            i < m; threads own model rows and stream the partner arrays
//            from shared memory (broadcast reads within a warp);
//   phase 3  block reduction of the four sums in double-float.
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

namespace gosma {

// Per-cube data written by the pre-pass (144 bytes): the rotation and the
// translation cuboid as double-floats.
struct CubePrep {
    float Rh[9], Rl[9];  // R_r0 (row-major)
    float th[3], tl[3];  // t0
    float wh[3], wl[3];  // translation half-widths
    float Cr, Sr;        // cos / sin of psi_r / 2 (cosine rounded down, sine up)
    float psi_r;
    int infeasible;      // rotation cube wholly outside the pi-ball
    float pad[2];
};
static_assert(sizeof(CubePrep) == 144, "CubePrep layout");
constexpr int PREP_WORDS = sizeof(CubePrep) / 4;

// shared-memory scalars of one cube
struct CubeShared {
    CubePrep rot;
    int infeasible;         // no feasible pose in the cube
    int centre_infeasible;  // t0 within zeta of a mean
    unsigned spsi_max;      // max over i of sin(psi_t,i / 2), as float bits
    float red[8][32];       // block reduction: 4 double-float sums x warps
};

// Directions are double-floats (hi + lo equals the unit vector to ~2^-44),
// so differences of nearly parallel directions keep full FP32 relative
// accuracy.  Shared-memory records are float4 so that a pair reads its
// partner with two or three 16-byte loads.
struct SmemArrays {
    float4 *M1;  // model rows (n1): v_hi (xyz), a
    float4 *M2;  //                   v_lo (xyz), b
    float4 *M3;  //                   k0, cos(psi_t/2), sin(psi_t/2), A_w
    float *Uw;   //                   U_w
    float4 *J1;  // image columns (n2): u_hi (xyz), kappa_2
    float4 *J2;  //                     u_lo (xyz), Q
};

__host__ __device__ inline size_t bounds_smem_arrays_bytes(int n1, int n2) {
    return (size_t)n1 * (3 * sizeof(float4) + sizeof(float)) + (size_t)n2 * 2 * sizeof(float4) + 16;
}

__device__ inline SmemArrays carve(float *base, int n1, int n2) {
    SmemArrays s;
    float4 *p = reinterpret_cast<float4 *>(base);
    s.M1 = p;
    s.M2 = p + n1;
    s.M3 = p + 2 * n1;
    s.J1 = p + 3 * n1;
    s.J2 = p + 3 * n1 + n2;
    s.Uw = reinterpret_cast<float *>(p + 3 * n1 + 2 * n2);
    return s;
}

__device__ inline int pow2ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Pre-pass for one cube: Rodrigues' formula (Sec. 4.1), Lemma 2 read as
// angle(R_r p, R_r0 p) <= |r - r0| <= sqrt(3) r_hw capped at pi, and the
// translation cuboid split into double-floats.
__device__ inline void cube_prepare(const double r0[3], double rhw, const double t0[3], const double thw[3],
                                    CubePrep &o) {
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
    double pr = sqrt(3.0) * rhw;
    if (pr > M_PI) pr = M_PI;
    double sh, ch;
    sincos(0.5 * pr, &sh, &ch);
    o.Sr = __double2float_ru(sh);
    o.Cr = __double2float_rd(ch);
    o.psi_r = (float)pr;
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double e = fabs(r0[k]) - rhw;
        if (e > 0) d2 += e * e;
    }
    o.infeasible = d2 > M_PI * M_PI ? 1 : 0;
    for (int k = 0; k < 3; ++k) {
        split_double(t0[k], o.th[k], o.tl[k]);
        split_double(thw[k], o.wh[k], o.wl[k]);
    }
    o.pad[0] = o.pad[1] = 0.f;
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
//  * |v - u| and |v + u| from double-float directions: 2u per component, so
//    sin(theta/2), cos(theta/2) carry <= 5.5u relative (squares 3.5u, sqrt 2u);
//  * the half-angle sine/cosine of s = psi_t + psi_r (row constants, evaluated
//    in double-float, rounded once) carry <= u relative;
//  * hence sin(B/2) = sin(theta/2) cos(s/2) - cos(theta/2) sin(s/2) is off by
//    at most 7.5u (sin(theta/2) + sin(s/2)) =: es; cos(B/2) is bounded from
//    the sine bounds as sqrt(1 - sin^2) (one rounding, sqrt 2u: 3u);
//  * K from above/below: 4u (sqrt 2u, K^2 2u);
//  * the exponent K - k1 - k2 (log2 units) carries <= 11u relative, and
//    rounding the ex2 argument adds 0.5u of it: the argument moves by
//    12u |exponent| in the safe direction;
//  * the factor outside the exponential: ex2 3u, rcp 2u, four products 4u,
//    one sum 1u: 10u relative = 14.4u in log2 units (TERM_SLACK);
//  * row weights, chunk sums (CHUNK-1 terms, plain FP32) and compensated row
//    sums: applied once per row with directed rounding.
#define GOSMA_TERM_SLACK (15.f * GOSMA_U)
constexpr int CHUNK = 8;

struct RowCross {
    float vx, vy, vz, wx, wy, wz;  // v_i hi / lo
    float a, b, k0, Cs, Ss, esS, A4;
};

// One cross pair (i, j): adds to pl the upper bound of the pair's term over
// the cube (Theorem 1, Eq. K1i2j_ub with B of Eq. K1i2j_ub_B) and to pc the
// term at the centre (Lemma 1), both without the row multipliers.
__device__ __forceinline__ void cross_pair(const RowCross &R, float4 J1, float4 J2, float &pl, float &pc) {
    const float U = GOSMA_U;
    const float k2 = J1.w, Q = J2.w;
    float dx = (R.vx - J1.x) + (R.wx - J2.x), dy = (R.vy - J1.y) + (R.wy - J2.y), dz = (R.vz - J1.z) + (R.wz - J2.z);
    float px = (R.vx + J1.x) + (R.wx + J2.x), py = (R.vy + J1.y) + (R.wy + J2.y), pz = (R.vz + J1.z) + (R.wz + J2.z);
    float x2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));  // |v - u|^2 = 4 sin^2(theta/2)
    float y2 = fmaf(px, px, fmaf(py, py, pz * pz));  // |v + u|^2 = 4 cos^2(theta/2)
    // centre: kappa_1i(t0) = k0, angle theta
    float kk = R.k0 * k2;
    float dk0 = R.k0 - k2;
    float K0 = sqrta(fmaf(dk0, dk0, kk * y2));
    float den0 = (R.k0 + k2) + K0;
    float K0c = fmaxf(K0, 1e-20f);
    float r0 = rcpa(den0 * K0c);
    float w0 = den0 * r0;  // 1/K0, times g(K0) below (g(K)/K -> 2 as K -> 0)
    if (K0 < 9.f) w0 = K0 < 1e-3f ? 2.f - 2.f * K0 : gZ(K0) * w0;
    pc = fmaf(ex2a(kk * x2 * (K0c * r0) * (-GOSMA_LOG2E)), w0 * Q, pc);
    // bound: B = max(0, theta - s), s = psi_t,i + psi_r (Cs, Ss = cos, sin of s/2)
    float sth = 0.5f * sqrta(x2), cth = 0.5f * sqrta(y2);
    float sB = fmaf(sth, R.Cs, -cth * R.Ss);
    float es = fmaf(7.5f * U, sth, R.esS);
    float slo = fmaxf(sB - es, 0.f);
    float shi = fminf(fmaxf(sB, 0.f) + es, 1.f);
    // cos(B/2) from the sine bounds: sqrt(1 - s^2), one rounding of 1 - s^2, sqrt 2u
    float chi = fminf(sqrta(fmaf(-slo, slo, 1.f)) * (1.f + 3.f * U), 1.f);
    float clo = sqrta(fmaxf(fmaf(-shi, shi, 1.f), 0.f)) * (1.f - 3.f * U);
    // K(a) - a - k2: an upper bound uses the smallest sin and the largest K
    float ak4 = R.A4 * k2;
    float dka = R.a - k2;
    float Khi = sqrta(fmaf(dka, dka, ak4 * (chi * chi))) * (1.f + 4.f * U);
    // smallest K over kappa_1 in [a, b] (minimiser -k2 cos B, clamped), from below
    float cosBlo = fmaf(2.f * clo, clo, -1.f);
    float ks = fminf(fmaxf(-k2 * cosBlo, R.a), R.b);
    float dks = ks - k2;
    float Kmin = sqrta(fmaf(dks, dks, 4.f * ks * k2 * (clo * clo))) * (1.f - 4.f * U);
    float den = (R.a + k2) + Khi;
    float Kc = fmaxf(Kmin, 1e-20f);
    float r = rcpa(den * Kc);
    float DL = ak4 * (slo * slo) * (Kc * r) * (-GOSMA_LOG2E);
    // g(K)/K <= min(1/K, 2): an upper bound without evaluating g
    float w = fminf(den * r, 2.f);
    pl = fmaf(ex2a(fmaf(12.f * U, fabsf(DL), DL + GOSMA_TERM_SLACK)), w * Q, pl);
}

struct RowSelf {
    float vx, vy, vz, wx, wy, wz;
    float a, b, k0, cp, sp;
};

// One self pair (i, m), i != m: adds to pl the lower bound of the pair's term
// over the cuboid (Theorem 1, Eq. K1i1j_lb with A of Eq. K1i1j_lb_A) and to pc
// the centre term, both without the row multipliers.
__device__ __forceinline__ void self_pair(const RowSelf &R, float4 M1, float4 M2, float4 M3, float Um, float &pl,
                                          float &pc) {
    const float U = GOSMA_U;
    const float am = M1.w, bm = M2.w, k0m = M3.x, cpm = M3.y, spm = M3.z, Am = M3.w;
    float dx = (R.vx - M1.x) + (R.wx - M2.x), dy = (R.vy - M1.y) + (R.wy - M2.y), dz = (R.vz - M1.z) + (R.wz - M2.z);
    float px = (R.vx + M1.x) + (R.wx + M2.x), py = (R.vy + M1.y) + (R.wy + M2.y), pz = (R.vz + M1.z) + (R.wz + M2.z);
    float x2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float y2 = fmaf(px, px, fmaf(py, py, pz * pz));
    // centre
    float kk = R.k0 * k0m;
    float dk0 = R.k0 - k0m;
    float K0 = sqrta(fmaf(dk0, dk0, kk * y2));
    float den0 = (R.k0 + k0m) + K0;
    float K0c = fmaxf(K0, 1e-20f);
    float r0 = rcpa(den0 * K0c);
    float w0 = den0 * r0;
    if (K0 < 9.f) w0 = K0 < 1e-3f ? 2.f - 2.f * K0 : gZ(K0) * w0;
    pc = fmaf(ex2a(kk * x2 * (K0c * r0) * (-GOSMA_LOG2E)), w0 * Um, pc);
    // bound: A = min(pi, theta + psi_i + psi_m); the half-angle pair of
    // (psi_i + psi_m)/2 is formed here in FP32 (2u each): sin(A/2) carries
    // <= 9.5u (sin(theta/2) + sin(psi/2)), cos(A/2) <= 14u
    float sth = 0.5f * sqrta(x2), cth = 0.5f * sqrta(y2);
    float C = fmaf(R.cp, cpm, -R.sp * spm);  // cos((psi_i + psi_m)/2)
    float S = fmaf(R.sp, cpm, R.cp * spm);   // sin((psi_i + psi_m)/2)
    float cA = fmaf(cth, C, -sth * S);       // cos(A/2) before the clamp at pi
    float sA = fmaf(sth, C, cth * S);
    float es = 10.f * U * (sth + fabsf(S));
    bool api = cA <= 16.f * U;               // A may reach pi
    float shi = api ? 1.f : fminf(sA + es, 1.f);
    float slo = fmaxf(sA - es, 0.f);
    // cos(A/2) from the sine bounds (A/2 <= pi/2), as in the cross pair
    float clo = sqrta(fmaxf(fmaf(-shi, shi, 1.f), 0.f)) * (1.f - 3.f * U);
    float chi = fminf(sqrta(fmaf(-slo, slo, 1.f)) * (1.f + 3.f * U), 1.f);
    // K(b_i, b_m) - b_i - b_m: a lower bound uses the largest sin and the smallest K
    float bb = R.b * bm;
    float dbb = R.b - bm;
    float Klo = sqrta(fmaf(dbb, dbb, 4.f * bb * (clo * clo))) * (1.f - 4.f * U);
    // largest K over the four corners of [a_i, b_i] x [a_m, b_m], from above
    float c4 = 4.f * (chi * chi);
    float q1 = R.a - am, q2 = R.a - bm, q3 = R.b - am;
    float e1 = fmaf(q1, q1, c4 * R.a * am);
    float e2 = fmaf(q2, q2, c4 * R.a * bm);
    float e3 = fmaf(q3, q3, c4 * R.b * am);
    float e4 = fmaf(dbb, dbb, c4 * bb);
    float Kmax = sqrta(fmaxf(fmaxf(e1, e2), fmaxf(e3, e4))) * (1.f + 5.f * U);
    float den = (R.b + bm) + Klo;
    float r = rcpa(den * Kmax);
    float DL = bb * (shi * shi) * (Kmax * r) * (-4.f * GOSMA_LOG2E);
    // g(K)/K from below: g(K)/K >= 2 - 2K for small K; g rounded with <= 64u error otherwise
    float w = den * r;
    if (Kmax < 9.f) w = Kmax < 0.25f ? fmaxf(2.f - 2.f * Kmax, 0.f) : gZ(Kmax) * w * (1.f - 64.f * U);
    pl = fmaf(ex2a(DL - fmaf(12.f * U, fabsf(DL), GOSMA_TERM_SLACK)), w * Am, pl);
}

// k coth(k) / 2 = Z(2k) / Z(k)^2, the diagonal self term without phi^2
// (relative error <= 12u).
__device__ __forceinline__ float half_kcothk(float k) {
    float e = ex2a(-2.f * GOSMA_LOG2E * k);
    return 0.5f * k * (1.f + e) * rcpa(1.f - e);
}

// Warp + block reduction of four double-floats; the result is valid in thread 0.
template <int BLOCK>
__device__ inline void block_reduce_df(df v[4], CubeShared &cs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) {
            df t = {__shfl_down_sync(0xffffffffu, v[k].h, o), __shfl_down_sync(0xffffffffu, v[k].l, o)};
            v[k] = df_add(v[k], t);
        }
    if (lane == 0)
        for (int k = 0; k < 4; ++k) {
            cs.red[2 * k][warp] = v[k].h;
            cs.red[2 * k + 1][warp] = v[k].l;
        }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) {
            df s = {cs.red[2 * k][0], cs.red[2 * k + 1][0]};
            for (int w = 1; w < BLOCK / 32; ++w) s = df_add(s, {cs.red[2 * k][w], cs.red[2 * k + 1][w]});
            v[k] = s;
        }
}

// Work distribution of the persistent bound kernels: cubes are handed out
// one at a time from a device counter that is zero at launch, so that blocks
// drawing cheap cubes (infeasible ones, children reusing cached self sums)
// take more of them.  Every thread of the block calls it; the leading barrier
// keeps the slot from being overwritten before all threads have read it.
__device__ __forceinline__ int next_cube(int *counter, int *slot) {
    __syncthreads();
    if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
    __syncthreads();
    return *slot;
}

// The whole per-cube computation.  Every thread of the block must call it
// with the same cube; sums are valid in thread 0 on return.  need_self = 0
// skips the self pairs (the caller reuses cached self sums).
template <int BLOCK>
__device__ void cube_bounds(const MixDev &mx, const CubePrep &prep, df zeta2, bool need_self, CubeShared &cs,
                            const SmemArrays &sm, CubeSums &out) {
    const int tid = threadIdx.x;
    const int n1 = mx.n1, n2 = mx.n2;
    const float U = GOSMA_U;
    for (int k = tid; k < PREP_WORDS; k += BLOCK)
        reinterpret_cast<float *>(&cs.rot)[k] = reinterpret_cast<const float *>(&prep)[k];
    if (tid == 0) {
        cs.infeasible = prep.infeasible;
        cs.centre_infeasible = 0;
        cs.spsi_max = 0u;
    }
    __syncthreads();

    // ---------------- phase 1a: image columns u_j = R_r0^T mu_2j (double-float)
    for (int j = tid; j < n2; j += BLOCK) {
        df m0 = {mx.mu2h[3 * j], mx.mu2l[3 * j]}, m1 = {mx.mu2h[3 * j + 1], mx.mu2l[3 * j + 1]},
           m2 = {mx.mu2h[3 * j + 2], mx.mu2l[3 * j + 2]};
        df u[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            u[c] = df_dot3({cs.rot.Rh[c], cs.rot.Rl[c]}, m0, {cs.rot.Rh[3 + c], cs.rot.Rl[3 + c]}, m1,
                           {cs.rot.Rh[6 + c], cs.rot.Rl[6 + c]}, m2);
        sm.J1[j] = make_float4(u[0].h, u[1].h, u[2].h, mx.kappa2[j]);
        sm.J2[j] = make_float4(u[0].l, u[1].l, u[2].l, mx.Q2[j]);
    }

    // ---------------- phase 1b: model rows (double-float geometry)
    Acc dsl, dsu;  // diagonal self terms of this thread
    dsl.zero();
    dsu.zero();
    for (int i = tid; i < n1; i += BLOCK) {
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
        if (f2 * (1.f + 8.f * U) < zeta2.h) atomicOr(&cs.infeasible, 1);
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
        sm.M1[i] = make_float4(v[0].h, v[1].h, v[2].h, a);
        sm.M2[i] = make_float4(v[0].l, v[1].l, v[2].l, b);
        sm.M3[i] = make_float4(k0, cps, sps, Aw);
        sm.Uw[i] = Uw;
        // diagonal self term phi_i^2 k coth(k) / 2, smallest over [a_i, b_i] at a_i
        dsl.add(ph * ph * half_kcothk(a) * (1.f - 16.f * U));
        dsu.add(ph * ph * half_kcothk(k0));
    }
    __syncthreads();

    // per-thread sums (double-float): self lb, cross ub, self centre, cross centre
    df T[4] = {fast_two_sum(dsl.s, dsl.c), {0.f, 0.f}, fast_two_sum(dsu.s, dsu.c), {0.f, 0.f}};
    T[0] = df_scale(T[0].h, T[0].l, 1.f - 3.f * U);

    if (!cs.infeasible) {
        // ---------------- phase 2a: cross pairs
        const int Ti = n1 >= BLOCK ? BLOCK : pow2ceil(n1);
        const int Tj = BLOCK / Ti;
        const int ti = tid % Ti, tj = tid / Ti;
        const float Cr = cs.rot.Cr, Sr = cs.rot.Sr;
        for (int i = ti; i < n1; i += Ti) {
            RowCross R;
            const float4 m1 = sm.M1[i], m2 = sm.M2[i], m3 = sm.M3[i];
            R.vx = m1.x;
            R.vy = m1.y;
            R.vz = m1.z;
            R.wx = m2.x;
            R.wy = m2.y;
            R.wz = m2.z;
            R.a = m1.w;
            R.b = m2.w;
            R.k0 = m3.x;
            R.A4 = 4.f * R.a;
            float cps = m3.y, sps = m3.z;
            // s = psi_t,i + psi_r as half-angle cosine/sine (double-float, rounded once);
            // s >= pi means B = 0 everywhere
            df cc = two_prod(cps, Cr), ssp = two_prod(sps, Sr), sc = two_prod(sps, Cr), cs2 = two_prod(cps, Sr);
            R.Cs = (cc.h - ssp.h) + (cc.l - ssp.l);
            R.Ss = (sc.h + cs2.h) + (sc.l + cs2.l);
            if (R.Cs <= 0.f) {
                R.Cs = 0.f;
                R.Ss = 1.f;
            }
            R.esS = 7.5f * U * R.Ss;
            // phi_i b_i / g(b_i) from above (for b >= 9 g rounds to 1, at most 2^-25 high),
            // times the chunk and row-sum allowances
            float Bw = R.b < 9.f ? mx.phi1f[i] * R.b * rcpa(gZ(R.b)) * (1.f + 12.f * U) : mx.phi1f[i] * R.b;
            Bw = __fmul_ru(Bw, 1.f + (float)(CHUNK + 6) * U);
            Acc cl, cu;
            cl.zero();
            cu.zero();
            float pl = 0.f, pc = 0.f;
            int cnt = 0;
            const int j1 = mx.rj1 ? mx.rj1[i] : n2;
#pragma unroll 1
            for (int j = (mx.rj0 ? mx.rj0[i] : 0) + tj; j < j1; j += Tj) {
                cross_pair(R, sm.J1[j], sm.J2[j], pl, pc);
                if (++cnt == CHUNK) {
                    cl.add(pl);
                    cu.add(pc);
                    pl = pc = 0.f;
                    cnt = 0;
                }
            }
            cl.add(pl);
            cu.add(pc);
            T[1] = df_add(T[1], df_scale(cl.s, cl.c, Bw));
            T[3] = df_add(T[3], df_scale(cu.s, cu.c, sm.Uw[i]));
        }
        // ---------------- phase 2b: self pairs i < m, rows paired (p, n1-2-p) for balance
        if (need_self && n1 > 1) {
            const int NP = n1 / 2;  // ceil((n1 - 1) / 2)
            const int Si = NP >= BLOCK ? BLOCK : pow2ceil(NP);
            const int Sj = BLOCK / Si;
            const int si = tid % Si, sj = tid / Si;
            for (int pp = si; pp < NP; pp += Si) {
                for (int h = 0; h < 2; ++h) {
                    int i = h == 0 ? pp : n1 - 2 - pp;
                    if (h == 1 && i == pp) break;
                    RowSelf R;
                    const float4 m1 = sm.M1[i], m2 = sm.M2[i], m3 = sm.M3[i];
                    R.vx = m1.x;
                    R.vy = m1.y;
                    R.vz = m1.z;
                    R.wx = m2.x;
                    R.wy = m2.y;
                    R.wz = m2.z;
                    R.a = m1.w;
                    R.b = m2.w;
                    R.k0 = m3.x;
                    R.cp = m3.y;
                    R.sp = m3.z;
                    Acc sl, su;
                    sl.zero();
                    su.zero();
                    float pl = 0.f, pc = 0.f;
                    int cnt = 0;
                    const int mend = mx.rm1 ? mx.rm1[i] : n1;
#pragma unroll 1
                    for (int m = i + 1 + sj; m < mend; m += Sj) {
                        self_pair(R, sm.M1[m], sm.M2[m], sm.M3[m], sm.Uw[m], pl, pc);
                        if (++cnt == CHUNK) {
                            sl.add(pl);
                            su.add(pc);
                            pl = pc = 0.f;
                            cnt = 0;
                        }
                    }
                    sl.add(pl);
                    su.add(pc);
                    // both orders (i, m) and (m, i): factor 2, exact
                    float Awi = __fmul_rd(2.f * m3.w, 1.f - (float)(CHUNK + 3) * U);
                    T[0] = df_add(T[0], df_scale(sl.s, sl.c, Awi));
                    T[2] = df_add(T[2], df_scale(su.s, su.c, 2.f * sm.Uw[i]));
                }
            }
        }
    }

    // ---------------- phase 3: block reduction (double-float)
    block_reduce_df<BLOCK>(T, cs);
    if (tid == 0) {
        out.self_lb = (double)T[0].h + (double)T[0].l;
        out.cross_ub = (double)T[1].h + (double)T[1].l;
        out.self_c = (double)T[2].h + (double)T[2].l;
        out.cross_c = (double)T[3].h + (double)T[3].l;
        out.psi_r = cs.rot.psi_r;
        float smax = __uint_as_float(cs.spsi_max);
        out.psi_t_max = smax >= 1.f ? (float)M_PI : 2.f * asinf(smax);
        out.feasible = !cs.infeasible;
        out.centre_feasible = !cs.centre_infeasible;
    }
    __syncthreads();
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
