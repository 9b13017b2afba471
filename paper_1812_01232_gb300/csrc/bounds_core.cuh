// Per-cube Theorem 1 bounds: the hot loop of GOSMA (Algorithm 1, "evaluate
// the bounds of the sub-cubes in parallel").
//
// One thread block evaluates one sub-cube C_r x C_t at a time:
//   phase 1  per image component j: u_j = R_r0^T mu_2j (FP64, rounded once);
//            per model component i: v_i, kappa_1i(t0), the kappa interval
//            [a_i, b_i] over the cuboid, and psi_t(mu_1i) as half-angle
//            cosine/sine (Lemma 3).  Everything goes to shared memory.
//   phase 2  diagonal self terms, all cross pairs (i, j) and all self pairs
//            i < m; each thread owns model rows and walks the partner
//            arrays in shared memory (broadcast reads within a warp).
//   phase 3  block reduction of the four FP64 sums.
//
// Pair terms are computed in FP32.  The closed forms follow Theorem 1 with
// the translation dependence of kappa bounded over [a_i, b_i]:
//   K^2 = (k1 - k2)^2 + 4 k1 k2 cos^2(B/2),
//   K - k1 - k2 = -4 k1 k2 sin^2(B/2) / (k1 + k2 + K)     (no cancellation),
//   Z(x) = e^x g(x) / x with g(x) = 1 - e^{-2x}.
// Every rounding that could raise a lower bound is covered: angle sines and
// cosines are widened by an absolute error bound, kappa intervals by a
// relative one, and the exponent of each term by a bound on its error, in
// the direction that lowers the cube's lower bound.  Cross terms and the
// self terms are accumulated with compensated FP32 sums per model row and
// added in FP64.
#pragma once

#include "gosma_internal.cuh"

namespace gosma {

// shared-memory scalars of one cube
struct CubeShared {
    double R0[9];
    float Cr, Sr;          // cos / sin of psi_r / 2 (sine rounded up, cosine down)
    float psi_r;
    int infeasible;        // no feasible pose in the cube
    int centre_infeasible; // t0 within zeta of a mean
    unsigned spsi_max;     // max over i of sin(psi_t,i / 2), as float bits
    double red[4][32];
};

// Directions are kept as FP32 hi/lo pairs (hi + lo equals the FP64 unit
// vector to ~2^-48), so differences of nearly parallel directions keep full
// FP32 relative accuracy.
struct SmemArrays {
    // model rows (n1)
    float *vx, *vy, *vz, *wx, *wy, *wz;  // v_i hi / lo
    float *a, *b, *k0, *cps, *sps, *Aw, *Uw;
    // image columns (n2)
    float *ux, *uy, *uz, *lx, *ly, *lz;  // u_j hi / lo
    float *k2, *Q;
};

constexpr int MODEL_FLOATS = 13, IMAGE_FLOATS = 8;

__host__ __device__ inline size_t bounds_smem_arrays_bytes(int n1, int n2) {
    return (size_t)(MODEL_FLOATS * n1 + IMAGE_FLOATS * n2) * sizeof(float);
}

__device__ inline SmemArrays carve(float *base, int n1, int n2) {
    SmemArrays s;
    float *p = base;
    float **m[MODEL_FLOATS] = {&s.vx, &s.vy, &s.vz, &s.wx, &s.wy, &s.wz, &s.a, &s.b, &s.k0, &s.cps, &s.sps, &s.Aw, &s.Uw};
    for (int k = 0; k < MODEL_FLOATS; ++k) {
        *m[k] = p;
        p += n1;
    }
    float **q[IMAGE_FLOATS] = {&s.ux, &s.uy, &s.uz, &s.lx, &s.ly, &s.lz, &s.k2, &s.Q};
    for (int k = 0; k < IMAGE_FLOATS; ++k) {
        *q[k] = p;
        p += n2;
    }
    return s;
}

__device__ inline int pow2ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Rodrigues' formula (Sec. 4.1), FP64.
__device__ inline void rodrigues_d(const double r[3], double R[9]) {
    double th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double th = sqrt(th2);
    double A, B;
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

// g(x) = 1 - e^{-2x}, so that Z(x) = e^x g(x) / x (Eq. Z).  For x >= 9,
// g(x) > 1 - 2^-25 and rounds to 1 in FP32.
__device__ __forceinline__ float gZ(float x) { return 1.f - ex2a(-2.f * GOSMA_LOG2E * x); }

// Half-angle sine and cosine of the angle between two unit directions
// given as hi/lo pairs: sin(theta/2) = |v - u|/2, cos(theta/2) = |v + u|/2.
__device__ __forceinline__ void half_angle(float vx, float vy, float vz, float wx, float wy, float wz, float ux,
                                           float uy, float uz, float lx, float ly, float lz, float &sth, float &cth) {
    float dx = (vx - ux) + (wx - lx), dy = (vy - uy) + (wy - ly), dz = (vz - uz) + (wz - lz);
    float px = (vx + ux) + (wx + lx), py = (vy + uy) + (wy + ly), pz = (vz + uz) + (wz + lz);
    float x2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float y2 = fmaf(px, px, fmaf(py, py, pz * pz));
    sth = 0.5f * sqrta(x2);
    cth = 0.5f * sqrta(y2);
}

// Every pair term is written in linear form:
//   Z(K) / (Z(k1) Z(k2)) = e^{K - k1 - k2} * (g(K) / K) * (k1 / g(k1)) * (k2 / g(k2)),
// the last two factors (times the weights phi) being per-row and per-column
// multipliers.  Only K - k1 - k2 goes through the exponential.
//
// Error budget of one term, beyond the directed widening of the angles and
// of K: the factor outside the exponential carries ex2 (4u), rcp (4u) and
// four roundings (4u), 12u relative or 17.3u in log2 units; the exponent
// K - k1 - k2 has a relative error of at most 9u.  The exponent (log2
// units) is therefore moved by 12u |K - k1 - k2| log2 e + TERM_SLACK.
//
// Angles: hi/lo directions make sin(theta/2) and cos(theta/2) accurate to
// 3.5u relative; the uncertainty angles psi_t are widened by 16u relative
// (their sin^2(psi/2) is accurate to 14u), psi_r is rounded outwards; the
// half-angle sine/cosine of B (or A) is then uncertain by at most
// 8u (sin(theta/2) + sin(s/2)), which is added or subtracted ("es").
#define GOSMA_TERM_SLACK (24.f * GOSMA_U)

// One cross pair (i, j): adds the upper bound of the pair's term over the
// cube (Theorem 1, Eq. K1i2j_ub with B of Eq. K1i2j_ub_B), without the row
// multiplier B_i, to cl, and the term at the centre (Lemma 1), without
// U_i, to cu.
__device__ __forceinline__ void cross_pair(float sth, float cth, float a, float b, float k0, float Cs, float Ss,
                                           float k2, float Q, Acc &cl, Acc &cu) {
    const float U = GOSMA_U;
    // centre: kappa_1i(t0) = k0, angle theta
    float kk = k0 * k2;
    float dk0 = k0 - k2;
    float K0 = sqrta(fmaf(dk0, dk0, 4.f * kk * (cth * cth)));
    float den0 = k0 + k2 + K0;
    float K0c = fmaxf(K0, 1e-20f);
    float r0 = rcpa(den0 * K0c);
    float D0 = -4.f * kk * (sth * sth) * (K0c * r0);
    float w0 = den0 * r0;  // 1/K0, times g(K0) below (g(K)/K -> 2 as K -> 0)
    if (K0 < 9.f) w0 = K0 < 1e-3f ? 2.f - 2.f * K0 : gZ(K0) * w0;
    cu.add(ex2a(D0 * GOSMA_LOG2E) * w0 * Q);
    // bound: B = max(0, theta - s), s = psi_t,i + psi_r (Cs, Ss = cos, sin of s/2)
    float sB = fmaf(sth, Cs, -cth * Ss);
    float cB = fmaf(cth, Cs, sth * Ss);
    float es = 8.f * U * (sth + Ss);
    float slo = fmaxf(sB - es, 0.f);
    float cBc = sB <= 0.f ? 1.f : cB;
    float chi = fminf(cBc + es, 1.f);
    float clo = fmaxf(cBc - es, 0.f);
    // K(a) - a - k2: an upper bound uses the smallest sin and the largest K
    float ka = a * k2;
    float dka = a - k2;
    float Khi = sqrta(fmaf(dka, dka, 4.f * ka * (chi * chi))) * (1.f + 8.f * U);
    // smallest K over kappa_1 in [a, b] (minimiser -k2 cos B, clamped), from below
    float cosBlo = fmaf(2.f * clo, clo, -1.f);
    float ks = fminf(fmaxf(-k2 * cosBlo, a), b);
    float dks = ks - k2;
    float Kmin = sqrta(fmaf(dks, dks, 4.f * ks * k2 * (clo * clo))) * (1.f - 8.f * U);
    float den = a + k2 + Khi;
    float Kc = fmaxf(Kmin, 1e-20f);
    float r = rcpa(den * Kc);
    float DL = -4.f * ka * (slo * slo) * (Kc * r) * GOSMA_LOG2E;
    // g(K)/K <= min(1/K, 2): an upper bound without evaluating g
    float w = fminf(den * r, 2.f);
    cl.add(ex2a(fmaf(12.f * U, fabsf(DL), DL + GOSMA_TERM_SLACK)) * w * Q);
}

// One self pair (i, m), i != m: adds the lower bound of the pair's term over
// the cuboid (Theorem 1, Eq. K1i1j_lb with A of Eq. K1i1j_lb_A), without the
// row multiplier A_i, to sl, and the centre term, without U_i, to su.
__device__ __forceinline__ void self_pair(float sth, float cth, float ai, float bi, float k0i, float cpi, float spi,
                                          float am, float bm, float k0m, float cpm, float spm, float Am, float Um,
                                          Acc &sl, Acc &su) {
    const float U = GOSMA_U;
    // centre
    float kk = k0i * k0m;
    float dk0 = k0i - k0m;
    float K0 = sqrta(fmaf(dk0, dk0, 4.f * kk * (cth * cth)));
    float den0 = k0i + k0m + K0;
    float K0c = fmaxf(K0, 1e-20f);
    float r0 = rcpa(den0 * K0c);
    float D0 = -4.f * kk * (sth * sth) * (K0c * r0);
    float w0 = den0 * r0;
    if (K0 < 9.f) w0 = K0 < 1e-3f ? 2.f - 2.f * K0 : gZ(K0) * w0;
    su.add(ex2a(D0 * GOSMA_LOG2E) * w0 * Um);
    // bound: A = min(pi, theta + psi_i + psi_m)
    float C = fmaf(cpi, cpm, -spi * spm);  // cos((psi_i + psi_m)/2)
    float S = fmaf(spi, cpm, cpi * spm);   // sin((psi_i + psi_m)/2)
    float cA = fmaf(cth, C, -sth * S);     // cos(A/2) before the clamp at pi
    float sA = fmaf(sth, C, cth * S);
    float es = 8.f * U * (sth + fabsf(S));
    bool api = cA <= es;
    float clo = api ? 0.f : cA - es;
    float chi = fminf(fmaxf(cA, 0.f) + es, 1.f);
    float shi = api ? 1.f : fminf(sA + es, 1.f);
    // K(b_i, b_m) - b_i - b_m: a lower bound uses the largest sin and the smallest K
    float bb = bi * bm;
    float dbb = bi - bm;
    float Klo = sqrta(fmaf(dbb, dbb, 4.f * bb * (clo * clo))) * (1.f - 8.f * U);
    // largest K over the four corners of [a_i, b_i] x [a_m, b_m], from above
    float c4 = 4.f * (chi * chi);
    float q1 = ai - am, q2 = ai - bm, q3 = bi - am;
    float e1 = fmaf(q1, q1, c4 * ai * am);
    float e2 = fmaf(q2, q2, c4 * ai * bm);
    float e3 = fmaf(q3, q3, c4 * bi * am);
    float e4 = fmaf(dbb, dbb, c4 * bb);
    float Kmax = sqrta(fmaxf(fmaxf(e1, e2), fmaxf(e3, e4))) * (1.f + 8.f * U);
    float den = bi + bm + Klo;
    float r = rcpa(den * Kmax);
    float DL = -4.f * bb * (shi * shi) * (Kmax * r) * GOSMA_LOG2E;
    // g(K)/K from below: g(K)/K >= 2 - 2K for small K; g rounded with <= 64u error otherwise
    float w = den * r;
    if (Kmax < 9.f) w = Kmax < 0.25f ? fmaxf(2.f - 2.f * Kmax, 0.f) : gZ(Kmax) * w * (1.f - 64.f * U);
    sl.add(ex2a(DL - fmaf(12.f * U, fabsf(DL), GOSMA_TERM_SLACK)) * w * Am);
}

// k coth(k) / 2 = Z(2k) / Z(k)^2, the diagonal self term without phi^2.
__device__ __forceinline__ float half_kcothk(float k) {
    float e = ex2a(-2.f * GOSMA_LOG2E * k);
    return 0.5f * k * (1.f + e) * rcpa(1.f - e);
}

// The whole per-cube computation.  Every thread of the block must call it
// with the same cube; sums are valid in thread 0 on return.  need_self = 0
// skips the self pairs (the caller reuses cached self sums).
template <int BLOCK>
__device__ void cube_bounds(const MixDev &mx, const CubeGeom &g, bool need_self, CubeShared &cs, const SmemArrays &sm,
                            CubeSums &out) {
    const int tid = threadIdx.x;
    const int n1 = mx.n1, n2 = mx.n2;
    const float U = GOSMA_U;
    if (tid == 0) {
        rodrigues_d(g.r0, cs.R0);
        // Lemma 2 read as angle(R_r p, R_r0 p) <= |r - r0| <= sqrt(3) r_hw, capped at pi
        double pr = sqrt(3.0) * g.rhw;
        if (pr > M_PI) pr = M_PI;
        double sh, ch;
        sincos(0.5 * pr, &sh, &ch);
        cs.Sr = __double2float_ru(sh);
        cs.Cr = __double2float_rd(ch);
        cs.psi_r = (float)pr;
        // rotation part wholly outside the pi-ball: no rotation there is needed
        double d2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            double e = fabs(g.r0[k]) - g.rhw;
            if (e > 0) d2 += e * e;
        }
        cs.infeasible = sqrt(d2) > M_PI ? 1 : 0;
        cs.centre_infeasible = 0;
        cs.spsi_max = 0u;
    }
    __syncthreads();

    // ---------------- phase 1a: image columns u_j = R_r0^T mu_2j (FP64, split hi/lo)
    for (int j = tid; j < n2; j += BLOCK) {
        const double *m = mx.mu2 + 3 * j;
        double u0 = cs.R0[0] * m[0] + cs.R0[3] * m[1] + cs.R0[6] * m[2];
        double u1 = cs.R0[1] * m[0] + cs.R0[4] * m[1] + cs.R0[7] * m[2];
        double u2 = cs.R0[2] * m[0] + cs.R0[5] * m[1] + cs.R0[8] * m[2];
        float h0 = (float)u0, h1 = (float)u1, h2 = (float)u2;
        sm.ux[j] = h0;
        sm.uy[j] = h1;
        sm.uz[j] = h2;
        sm.lx[j] = (float)(u0 - (double)h0);
        sm.ly[j] = (float)(u1 - (double)h1);
        sm.lz[j] = (float)(u2 - (double)h2);
        sm.k2[j] = mx.kappa2[j];
        sm.Q[j] = mx.Q2[j];
    }

    // ---------------- phase 1b: model rows
    Acc dsl, dsu;  // diagonal self terms of this thread
    dsl.zero();
    dsu.zero();
    const double zeta2d = mx.zeta * mx.zeta;
    const float thx = (float)g.thw[0], thy = (float)g.thw[1], thz = (float)g.thw[2];
    for (int i = tid; i < n1; i += BLOCK) {
        const double *p = mx.mu1 + 3 * i;
        double cxd = p[0] - g.t0[0], cyd = p[1] - g.t0[1], czd = p[2] - g.t0[2];
        double cd2 = cxd * cxd + cyd * cyd + czd * czd;
        if (cd2 < zeta2d) atomicOr(&cs.centre_infeasible, 1);
        bool inside = fabs(cxd) <= g.thw[0] && fabs(cyd) <= g.thw[1] && fabs(czd) <= g.thw[2];
        // squared distances to the cuboid and to its far corner (FP64, rounded once)
        double exd = fmax(fabs(cxd) - g.thw[0], 0.0), eyd = fmax(fabs(cyd) - g.thw[1], 0.0),
               ezd = fmax(fabs(czd) - g.thw[2], 0.0);
        double fxd = fabs(cxd) + g.thw[0], fyd = fabs(cyd) + g.thw[1], fzd = fabs(czd) + g.thw[2];
        double dmin2d = exd * exd + eyd * eyd + ezd * ezd, dmax2d = fxd * fxd + fyd * fyd + fzd * fzd;
        if (dmax2d < zeta2d) atomicOr(&cs.infeasible, 1);
        float cx = (float)cxd, cy = (float)cyd, cz = (float)czd;
        float is2 = mx.inv_sig2[i];
        // kappa range over the feasible part of the cuboid (nearest point clamped to zeta);
        // each end carries at most 3u (rounding of d^2, of 1/sigma^2, and the fma)
        float a = fmaf((float)fmax(dmin2d, zeta2d), is2, 1.f) * (1.f - 4.f * U);
        float b = fmaf((float)dmax2d, is2, 1.f) * (1.f + 4.f * U);
        float d2 = (float)cd2;
        float k0 = fmaf(d2, is2, 1.f);
        // unit direction v_i: FP32 rsqrt refined by one FP64 Newton step, split hi/lo
        float vx = 1.f, vy = 0.f, vz = 0.f, wx = 0.f, wy = 0.f, wz = 0.f;
        if (cd2 > 0.0) {
            double r = (double)rsqrta(d2);
            r = r * (1.5 - 0.5 * cd2 * r * r);
            double v0 = cxd * r, v1 = cyd * r, v2 = czd * r;
            vx = (float)v0;
            vy = (float)v1;
            vz = (float)v2;
            wx = (float)(v0 - (double)vx);
            wy = (float)(v1 - (double)vy);
            wz = (float)(v2 - (double)vz);
        }
        // Lemma 3: largest angle between mu - t_vertex and mu - t0, as sin^2(psi/2);
        // pi when mu is in the cuboid or a vertex angle reaches pi/2
        float sp2 = 1.f;
        if (!inside) {
            float m2 = 0.f;
            bool wide = false;
#pragma unroll
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
                m2 = fmaxf(m2, s2);
            }
            sp2 = wide ? 1.f : fminf(m2, 1.f);
        }
        float sps = sp2 >= 1.f ? 1.f : fminf(sqrta(sp2) * (1.f + 16.f * U), 1.f);
        float cps = sps >= 1.f ? 0.f : sqrta(fmaxf(fmaf(-sps, sps, 1.f), 0.f)) * (1.f - 4.f * U);
        atomicMax(&cs.spsi_max, __float_as_uint(sps));
        float ph = mx.phi1f[i];
        float ga = a < 9.f ? gZ(a) : 1.f, gk = k0 < 9.f ? gZ(k0) : 1.f;
        sm.vx[i] = vx;
        sm.vy[i] = vy;
        sm.vz[i] = vz;
        sm.wx[i] = wx;
        sm.wy[i] = wy;
        sm.wz[i] = wz;
        sm.a[i] = a;
        sm.b[i] = b;
        sm.k0[i] = k0;
        sm.cps[i] = cps;
        sm.sps[i] = sps;
        sm.Aw[i] = ph * a * rcpa(ga) * (1.f - 16.f * U);  // phi_i a_i / g(a_i), from below
        sm.Uw[i] = ph * k0 * rcpa(gk);                    // phi_i k0_i / g(k0_i)
        // diagonal self term phi_i^2 k coth(k) / 2, smallest over [a_i, b_i] at a_i
        dsl.add(ph * ph * half_kcothk(a) * (1.f - 16.f * U));
        dsu.add(ph * ph * half_kcothk(k0));
    }
    __syncthreads();

    double self_lb = dsl.value() * (1.0 - 4.0 * (double)U), self_c = dsu.value();
    double cross_ub = 0.0, cross_c = 0.0;

    if (!cs.infeasible) {
        // ---------------- phase 2a: cross pairs
        const int Ti = n1 >= BLOCK ? BLOCK : pow2ceil(n1);
        const int Tj = BLOCK / Ti;
        const int ti = tid % Ti, tj = tid / Ti;
        const float Cr = cs.Cr, Sr = cs.Sr;
        for (int i = ti; i < n1; i += Ti) {
            float vx = sm.vx[i], vy = sm.vy[i], vz = sm.vz[i], wx = sm.wx[i], wy = sm.wy[i], wz = sm.wz[i];
            float a = sm.a[i], b = sm.b[i], k0 = sm.k0[i];
            float cps = sm.cps[i], sps = sm.sps[i];
            // s = psi_t,i + psi_r as half-angle cosine/sine; s >= pi means B = 0 everywhere
            float Cs = fmaf(cps, Cr, -sps * Sr);
            float Ss = fmaf(sps, Cr, cps * Sr);
            if (Cs <= 0.f) {
                Cs = 0.f;
                Ss = 1.f;
            }
            float gb = b < 9.f ? gZ(b) : 1.f;
            // phi_i b_i / g(b_i) from above (g rounded to 1 for b >= 9 is 2^-25 low at most)
            float Bw = mx.phi1f[i] * b * rcpa(gb) * (1.f + 16.f * U);
            Acc cl, cu;
            cl.zero();
            cu.zero();
            for (int j = tj; j < n2; j += Tj) {
                float sth, cth;
                half_angle(vx, vy, vz, wx, wy, wz, sm.ux[j], sm.uy[j], sm.uz[j], sm.lx[j], sm.ly[j], sm.lz[j], sth, cth);
                cross_pair(sth, cth, a, b, k0, Cs, Ss, sm.k2[j], sm.Q[j], cl, cu);
            }
            cross_ub += cl.value() * (double)Bw * (1.0 + 4.0 * (double)U);
            cross_c += cu.value() * (double)sm.Uw[i];
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
                    float vx = sm.vx[i], vy = sm.vy[i], vz = sm.vz[i], wx = sm.wx[i], wy = sm.wy[i], wz = sm.wz[i];
                    float ai = sm.a[i], bi = sm.b[i], k0i = sm.k0[i], cpi = sm.cps[i], spi = sm.sps[i];
                    Acc sl, su;
                    sl.zero();
                    su.zero();
                    for (int m = i + 1 + sj; m < n1; m += Sj) {
                        float sth, cth;
                        half_angle(vx, vy, vz, wx, wy, wz, sm.vx[m], sm.vy[m], sm.vz[m], sm.wx[m], sm.wy[m], sm.wz[m],
                                   sth, cth);
                        self_pair(sth, cth, ai, bi, k0i, cpi, spi, sm.a[m], sm.b[m], sm.k0[m], sm.cps[m], sm.sps[m],
                                  sm.Aw[m], sm.Uw[m], sl, su);
                    }
                    self_lb += 2.0 * sl.value() * (double)sm.Aw[i] * (1.0 - 4.0 * (double)U);
                    self_c += 2.0 * su.value() * (double)sm.Uw[i];
                }
            }
        }
    }

    // ---------------- phase 3: block reduction (warp shuffles, then shared memory)
    double v[4] = {self_lb, cross_ub, self_c, cross_c};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int warp = tid >> 5, lane = tid & 31;
    constexpr int NW = BLOCK / 32;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) cs.red[k][warp] = v[k];
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < 4; ++k) {
            double s = 0.0;
            for (int w = 0; w < NW; ++w) s += cs.red[k][w];
            v[k] = s;
        }
        out.self_lb = v[0];
        out.cross_ub = v[1];
        out.self_c = v[2];
        out.cross_c = v[3];
        out.psi_r = cs.psi_r;
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
        // allowance for the FP64 additions of the partial sums
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
