/*
 * FP64 CPU oracle for GOSMA (Campbell et al., "The Alignment of the Spheres:
 * Globally-Optimal Spherical Mixture Alignment for Camera Pose Estimation").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library under paper_1812_01232_gb300/) never calls it, and the
 * two share no code.
 *
 * Everything here is plain double precision, written straight from the
 * paper's definitions, with no blocking or fusion:
 *   - Z and the vMF inner product ........ Eq. (Z), Eq. (vMF), proof of Lemma 1
 *   - qPN concentration mapping .......... Eq. (qPN) / Eq. (vMF_PN_map)
 *   - objective f(R,t) ................... Lemma 1, Eq. (objective_function)
 *   - rotation / translation uncertainty . Lemma 2, Lemma 3
 *   - upper and lower bounds ............. Theorem 1
 *   - GOSMA branch-and-bound ............. Algorithm 1, Sec. 5
 *   - SMA local refinement (L-BFGS) ...... Sec. 5
 * Readings taken where the paper is silent (every one is listed in the
 * design notes of the repository):
 *   R1  psi_r: Lemma 2 gives no closed form for the surface maximum; the
 *       oracle uses the provable bound angle(R_r p, R_r0 p) <= |r - r0|,
 *       i.e. psi_r = min(sqrt(3)*half_width, pi).
 *   R2  psi_t: the vertex maximum of Lemma 3 is used only while it is at
 *       most pi/2 (where the cone of directions is convex); beyond that,
 *       and whenever p lies in the cuboid, psi_t = pi.
 *   R3  the translation dependence of kappa_1i inside the min/max of
 *       Theorem 1 (the paper defers it to an appendix that is not in the
 *       text) is bounded term by term over kappa in [a_i, b_i], using that
 *       K - k1 - k2 is non-increasing in each k, phiZ(x) = log Z(x) - x is
 *       decreasing, and K is a norm (convex, minimised along k1 at
 *       -k2 cos B).  [a_i, b_i] comes from the nearest and farthest points
 *       of the cuboid, the nearest clamped to zeta (Sec. 4.1 excludes
 *       |mu - t| < zeta).
 *   R4  self pairs with i == j: K_ii(t) = 2 kappa_i(t) exactly, so the
 *       term is kappa coth(kappa) / 2, increasing in kappa; its minimum
 *       over [a_i, b_i] is taken at a_i.
 *   R5  cubes whose rotation part lies wholly outside the pi-ball, or whose
 *       translation part lies wholly within zeta of one mean, get
 *       lb = ub = +inf (no feasible pose).  A centre within zeta of a mean
 *       gets ub = +inf.
 *   R6  branching compares psi_r with max_i psi_t(mu_1i); ties split
 *       rotation.  Priority is the lower bound, ties broken by greater
 *       depth, then creation order.
 *   R7  epsilon is on the normalised L2 distance f / C22 + 1, where
 *       C22 = sum_jj' phi_2j phi_2j' Z(|k_j mu_j + k_j' mu_j'|)/(Z(k_j)Z(k_j')),
 *       so the raw-f tolerance is eps * C22.
 *   R16 point-dependent psi_r (an option, mode 1 of om_bounds_mode): for
 *       each model direction v_i (at the cuboid centre) a certified bound
 *       of max over the rotation cube of angle(R_r v_i, R_r0 v_i), from the
 *       relative quaternion w(r) = vec(q(r0)^* q(r)), whose norm across v
 *       gives sin(angle / 2) = |w(r) x v| exactly.  Taylor's theorem at r0:
 *       w(r0 + d) = J_r(r0) d / 2 + rho, |rho| <= |d|^2 / 8, since the
 *       second derivative of the quaternion exponential along a line is at
 *       most |d / 2|^2 in norm.  The first-order term is a norm of a linear
 *       map, so its maximum over the cube is at a vertex.  Hence
 *       sin(psi_r,i / 2) <= max_vertices |J_r d x v_i| / 2 + 3 h^2 / 8,
 *       capped by the point-independent sqrt(3) h of R1.  The split rule
 *       (R6) keeps comparing the R1 angle.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#ifndef M_LN2
#define M_LN2 0.69314718055994530942
#endif

/* GMM theta_1 = {mu_1i, sigma_1i, phi_1i} and vMFMM theta_2 = {mu_2j, kappa_2j,
 * phi_2j} (Sec. 4, Eq. GMM and Eq. vMFMM).  mu arrays are n x 3 row-major.
 * sigma1 holds standard deviations (the paper's sigma, variance sigma^2). */
typedef struct {
    int n1;
    const double *mu1, *sigma1, *phi1;
    int n2;
    const double *mu2, *kappa2, *phi2;
} om_mix;

/* Translation domain Omega'_t (a cuboid) and the point-to-camera limit
 * zeta (Sec. 4.1). */
typedef struct {
    double t_lo[3], t_hi[3];
    double zeta;
} om_domain;

/* A 6-orthotope C_r x C_t: rotation cube centre r0 with half-width r_hw,
 * translation cuboid centre t0 with half-widths t_hw. */
enum { CUBE_R0 = 0, CUBE_RHW = 3, CUBE_T0 = 4, CUBE_THW = 7, CUBE_LEN = 10 };

/* ------------------------------------------------------------------ */
/* Eq. (Z): Z(k) = (e^k - e^-k)/k, kept in log form.                     */
/* phiZ(x) = log Z(x) - x = log((1 - e^{-2x}) / x); its limit at 0 is log 2. */
double om_phiZ(double x)
{
    if (x < 1e-12) return M_LN2 - x;
    return log(-expm1(-2.0 * x) / x);
}

double om_logZ(double x) { return x + om_phiZ(x); }

/* Eq. (vMF_PN_map): concentration of the qPN of a Gaussian at distance
 * dist with standard deviation sigma. */
double om_kappa_qpn(double dist, double sigma)
{
    double q = dist / sigma;
    return q * q + 1.0;
}

/* log of Z(|ka ua + kb ub|) / (Z(ka) Z(kb)): the vMF inner product
 * (integral of the product of two vMF densities) times 2 pi, from the
 * proof of Lemma 1. */
double om_pair_log(double ka, const double ua[3], double kb, const double ub[3])
{
    double w[3];
    for (int k = 0; k < 3; ++k) w[k] = ka * ua[k] + kb * ub[k];
    double K = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    return om_logZ(K) - om_logZ(ka) - om_logZ(kb);
}

/* Rodrigues' rotation formula for an angle-axis vector r (Sec. 4.1),
 * R row-major. */
void om_rodrigues(const double r[3], double R[9])
{
    double th = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double A, B;
    if (th < 1e-8) {
        A = 1.0 - th * th / 6.0;
        B = 0.5 - th * th / 24.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / (th * th);
    }
    double x = r[0], y = r[1], z = r[2];
    /* I + A [r]x + B [r]x^2 */
    R[0] = 1.0 + B * (-(y * y + z * z));
    R[1] = -A * z + B * (x * y);
    R[2] = A * y + B * (x * z);
    R[3] = A * z + B * (x * y);
    R[4] = 1.0 + B * (-(x * x + z * z));
    R[5] = -A * x + B * (y * z);
    R[6] = -A * y + B * (x * z);
    R[7] = A * x + B * (y * z);
    R[8] = 1.0 + B * (-(x * x + y * y));
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Angle between two non-zero vectors. */
double om_angle(const double a[3], const double b[3])
{
    double c[3];
    cross3(a, b, c);
    return atan2(norm3(c), dot3(a, b));
}

static void matvec(const double R[9], const double v[3], double o[3])
{
    for (int k = 0; k < 3; ++k) o[k] = R[3 * k] * v[0] + R[3 * k + 1] * v[1] + R[3 * k + 2] * v[2];
}
static void matTvec(const double R[9], const double v[3], double o[3])
{
    for (int k = 0; k < 3; ++k) o[k] = R[k] * v[0] + R[3 + k] * v[1] + R[6 + k] * v[2];
}

/* ------------------------------------------------------------------ */
/* Lemma 1, Eq. (objective_function): f(R, t).  The transformed model is
 * {R (mu_1i - t)} (proof of Lemma 1), so the qPN of component i has mean
 * direction R v_i, v_i = (mu_1i - t)/|mu_1i - t|, and concentration
 * kappa_1i(t) = (|mu_1i - t| / sigma_1i)^2 + 1 (Eq. kappa1).            */
double om_objective(const om_mix *m, const double R[9], const double t[3])
{
    int n1 = m->n1, n2 = m->n2;
    double *v = malloc(sizeof(double) * 3 * n1);
    double *kap = malloc(sizeof(double) * n1);
    for (int i = 0; i < n1; ++i) {
        double c[3] = {m->mu1[3 * i] - t[0], m->mu1[3 * i + 1] - t[1], m->mu1[3 * i + 2] - t[2]};
        double d = norm3(c);
        for (int k = 0; k < 3; ++k) v[3 * i + k] = c[k] / d;
        kap[i] = om_kappa_qpn(d, m->sigma1[i]);
    }
    double self = 0.0, cross = 0.0;
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n1; ++j)
            self += m->phi1[i] * m->phi1[j] * exp(om_pair_log(kap[i], v + 3 * i, kap[j], v + 3 * j));
    for (int i = 0; i < n1; ++i) {
        double Rv[3];
        matvec(R, v + 3 * i, Rv);
        for (int j = 0; j < n2; ++j)
            cross += m->phi1[i] * m->phi2[j] * exp(om_pair_log(kap[i], Rv, m->kappa2[j], m->mu2 + 3 * j));
    }
    free(v);
    free(kap);
    return self - 2.0 * cross;
}

/* Same, with the self and cross sums returned separately. */
void om_objective_parts(const om_mix *m, const double R[9], const double t[3], double *self_out, double *cross_out)
{
    int n1 = m->n1, n2 = m->n2;
    double self = 0.0, cross = 0.0;
    for (int i = 0; i < n1; ++i) {
        double ci[3] = {m->mu1[3 * i] - t[0], m->mu1[3 * i + 1] - t[1], m->mu1[3 * i + 2] - t[2]};
        double di = norm3(ci), vi[3] = {ci[0] / di, ci[1] / di, ci[2] / di};
        double ki = om_kappa_qpn(di, m->sigma1[i]);
        for (int j = 0; j < n1; ++j) {
            double cj[3] = {m->mu1[3 * j] - t[0], m->mu1[3 * j + 1] - t[1], m->mu1[3 * j + 2] - t[2]};
            double dj = norm3(cj), vj[3] = {cj[0] / dj, cj[1] / dj, cj[2] / dj};
            double kj = om_kappa_qpn(dj, m->sigma1[j]);
            self += m->phi1[i] * m->phi1[j] * exp(om_pair_log(ki, vi, kj, vj));
        }
        double Rv[3];
        matvec(R, vi, Rv);
        for (int j = 0; j < n2; ++j)
            cross += m->phi1[i] * m->phi2[j] * exp(om_pair_log(ki, Rv, m->kappa2[j], m->mu2 + 3 * j));
    }
    *self_out = self;
    *cross_out = cross;
}

double om_objective_r(const om_mix *m, const double r[3], const double t[3])
{
    double R[9];
    om_rodrigues(r, R);
    return om_objective(m, R, t);
}

/* C22 = 2 pi * integral of p2^2 (proof of Lemma 1); used to normalise f
 * (reading R7). */
double om_c22(const om_mix *m)
{
    double s = 0.0;
    for (int i = 0; i < m->n2; ++i)
        for (int j = 0; j < m->n2; ++j)
            s += m->phi2[i] * m->phi2[j] *
                 exp(om_pair_log(m->kappa2[i], m->mu2 + 3 * i, m->kappa2[j], m->mu2 + 3 * j));
    return s;
}

/* ------------------------------------------------------------------ */
/* Gradient of f with respect to x = (r, t) for SMA (Sec. 5).  The paper's
 * gradient is in its missing appendix; this one is derived directly:
 *   d log Z(x)/dx = coth x - 1/x,
 *   dK = (w/K) . dw for K = |w|,
 *   d(R v) = [J_l(r) dr]_x R v, with J_l the left Jacobian of SO(3),
 *   d kappa_1i / dt = -2 (mu_1i - t) / sigma_1i^2,
 *   d v_i / dt = -(I - v_i v_i^T) / |mu_1i - t|.                          */
static double dlogZ(double x)
{
    if (x < 1e-4) return x / 3.0 - x * x * x / 45.0;
    return 1.0 + 2.0 / expm1(2.0 * x) - 1.0 / x;
}

static void left_jacobian(const double r[3], double J[9])
{
    double th = norm3(r), a, b;
    if (th < 1e-6) {
        a = 0.5 - th * th / 24.0;
        b = 1.0 / 6.0 - th * th / 120.0;
    } else {
        a = (1.0 - cos(th)) / (th * th);
        b = (th - sin(th)) / (th * th * th);
    }
    double x = r[0], y = r[1], z = r[2];
    double S[9] = {0, -z, y, z, 0, -x, -y, x, 0};
    double S2[9];
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += S[3 * p + k] * S[3 * k + q];
            S2[3 * p + q] = s;
        }
    for (int k = 0; k < 9; ++k) J[k] = (k % 4 == 0 ? 1.0 : 0.0) + a * S[k] + b * S2[k];
}

void om_objective_grad(const om_mix *m, const double x[6], double *f_out, double g[6])
{
    int n1 = m->n1, n2 = m->n2;
    const double *r = x, *t = x + 3;
    double R[9];
    om_rodrigues(r, R);
    double *v = malloc(sizeof(double) * 3 * n1), *kap = malloc(sizeof(double) * n1), *d = malloc(sizeof(double) * n1);
    for (int i = 0; i < n1; ++i) {
        double c[3] = {m->mu1[3 * i] - t[0], m->mu1[3 * i + 1] - t[1], m->mu1[3 * i + 2] - t[2]};
        d[i] = norm3(c);
        for (int k = 0; k < 3; ++k) v[3 * i + k] = c[k] / d[i];
        kap[i] = om_kappa_qpn(d[i], m->sigma1[i]);
    }
    double f = 0.0, gw[3] = {0, 0, 0}, gt[3] = {0, 0, 0};
    /* d kappa_i/dt (3-vector) and d v_i/dt (3x3, column q = d v / d t_q) */
    double *dk = malloc(sizeof(double) * 3 * n1), *dv = malloc(sizeof(double) * 9 * n1);
    for (int i = 0; i < n1; ++i) {
        double s2 = m->sigma1[i] * m->sigma1[i];
        for (int q = 0; q < 3; ++q) dk[3 * i + q] = -2.0 * d[i] * v[3 * i + q] / s2;
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q)
                dv[9 * i + 3 * p + q] = -((p == q ? 1.0 : 0.0) - v[3 * i + p] * v[3 * i + q]) / d[i];
    }
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n1; ++j) {
            double w[3];
            for (int k = 0; k < 3; ++k) w[k] = kap[i] * v[3 * i + k] + kap[j] * v[3 * j + k];
            double K = norm3(w);
            double term = m->phi1[i] * m->phi1[j] * exp(om_logZ(K) - om_logZ(kap[i]) - om_logZ(kap[j]));
            f += term;
            double gK = dlogZ(K), gi = dlogZ(kap[i]), gj = dlogZ(kap[j]);
            for (int q = 0; q < 3; ++q) {
                double dw[3];
                for (int p = 0; p < 3; ++p)
                    dw[p] = dk[3 * i + q] * v[3 * i + p] + kap[i] * dv[9 * i + 3 * p + q] + dk[3 * j + q] * v[3 * j + p] +
                            kap[j] * dv[9 * j + 3 * p + q];
                double dK = (K > 0) ? dot3(w, dw) / K : 0.0;
                gt[q] += term * (gK * dK - gi * dk[3 * i + q] - gj * dk[3 * j + q]);
            }
        }
    for (int i = 0; i < n1; ++i) {
        double Rv[3];
        matvec(R, v + 3 * i, Rv);
        for (int j = 0; j < n2; ++j) {
            const double *u = m->mu2 + 3 * j;
            double k2 = m->kappa2[j];
            double w[3];
            for (int k = 0; k < 3; ++k) w[k] = kap[i] * Rv[k] + k2 * u[k];
            double K = norm3(w);
            double term = m->phi1[i] * m->phi2[j] * exp(om_logZ(K) - om_logZ(kap[i]) - om_logZ(k2));
            f -= 2.0 * term;
            double gK = dlogZ(K), gi = dlogZ(kap[i]);
            /* rotation: dK/domega = kappa_i (R v x w) / K */
            double cr[3];
            cross3(Rv, w, cr);
            for (int q = 0; q < 3; ++q) gw[q] += -2.0 * term * gK * kap[i] * cr[q] / K;
            for (int q = 0; q < 3; ++q) {
                double dvq[3] = {dv[9 * i + q], dv[9 * i + 3 + q], dv[9 * i + 6 + q]};
                double Rdv[3];
                matvec(R, dvq, Rdv);
                double dw[3];
                for (int p = 0; p < 3; ++p) dw[p] = dk[3 * i + q] * Rv[p] + kap[i] * Rdv[p];
                double dK = dot3(w, dw) / K;
                gt[q] += -2.0 * term * (gK * dK - gi * dk[3 * i + q]);
            }
        }
    }
    double J[9];
    left_jacobian(r, J);
    for (int q = 0; q < 3; ++q) g[q] = J[q] * gw[0] + J[3 + q] * gw[1] + J[6 + q] * gw[2];
    for (int q = 0; q < 3; ++q) g[3 + q] = gt[q];
    *f_out = f;
    free(v);
    free(kap);
    free(d);
    free(dk);
    free(dv);
}

/* ------------------------------------------------------------------ */
/* Lemma 2 with reading R1. */
double om_psi_r(double r_hw)
{
    double p = sqrt(3.0) * r_hw;
    return p < M_PI ? p : M_PI;
}

/* Right Jacobian of the exponential map of SO(3) at r:
 * J_r(r) = I - (1 - cos|r|)/|r|^2 [r]x + (|r| - sin|r|)/|r|^3 [r]x^2,
 * so that R_{r + d} = R_r R_{J_r(r) d} to first order in d. */
static void right_jacobian(const double r[3], double J[9])
{
    double th = norm3(r), c1, c2;
    if (th < 1e-6) {
        c1 = 0.5 - th * th / 24.0;
        c2 = 1.0 / 6.0 - th * th / 120.0;
    } else {
        c1 = (1.0 - cos(th)) / (th * th);
        c2 = (th - sin(th)) / (th * th * th);
    }
    double x = r[0], y = r[1], z = r[2];
    double S[9] = {0, -z, y, z, 0, -x, -y, x, 0};
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
            double s2 = 0;
            for (int k = 0; k < 3; ++k) s2 += S[3 * p + k] * S[3 * k + q];
            J[3 * p + q] = (p == q ? 1.0 : 0.0) - c1 * S[3 * p + q] + c2 * s2;
        }
}

/* Lemma 2, point-dependent form (reading R16): an upper bound of the angle
 * between R_r p and R_r0 p over the rotation cube of centre r0 and
 * half-width r_hw, for a unit vector p. */
double om_psi_r_point(const double r0[3], double r_hw, const double p[3])
{
    double J[9];
    right_jacobian(r0, J);
    double lin = 0.0;
    for (int k = 0; k < 4; ++k) { /* the 8 vertices d come in pairs +-d with equal norms */
        double d[3] = {r_hw, r_hw, r_hw}, c[3], x[3];
        if (k > 0) d[k - 1] = -r_hw;
        matvec(J, d, c);
        cross3(c, p, x);
        double nx = 0.5 * norm3(x);
        if (nx > lin) lin = nx;
    }
    double s = lin + 3.0 * r_hw * r_hw / 8.0;
    double psi = s >= 1.0 ? M_PI : 2.0 * asin(s);
    double r1 = om_psi_r(r_hw);
    return psi < r1 ? psi : r1;
}

/* Lemma 3 with reading R2. */
double om_psi_t(const double p[3], const double t0[3], const double thw[3])
{
    int inside = 1;
    for (int k = 0; k < 3; ++k)
        if (p[k] < t0[k] - thw[k] || p[k] > t0[k] + thw[k]) inside = 0;
    if (inside) return M_PI;
    double c[3] = {p[0] - t0[0], p[1] - t0[1], p[2] - t0[2]};
    double mx = 0.0;
    for (int vtx = 0; vtx < 8; ++vtx) {
        double a[3];
        for (int k = 0; k < 3; ++k) a[k] = p[k] - (t0[k] + ((vtx >> k) & 1 ? thw[k] : -thw[k]));
        double ang = om_angle(a, c);
        if (ang > mx) mx = ang;
    }
    return mx <= 0.5 * M_PI ? mx : M_PI;
}

/* Range [a, b] of kappa_1(t) = (|p - t|/sigma)^2 + 1 over the feasible part
 * of the cuboid (reading R3).  Returns 0 when no t in the cuboid is at
 * least zeta from p. */
int om_kappa_interval(const double p[3], double sigma, const double t0[3], const double thw[3], double zeta, double *a,
                      double *b)
{
    double dmin2 = 0.0, dmax2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double lo = t0[k] - thw[k], hi = t0[k] + thw[k];
        double e = 0.0;
        if (p[k] < lo) e = lo - p[k];
        if (p[k] > hi) e = p[k] - hi;
        dmin2 += e * e;
        double f1 = fabs(p[k] - lo), f2 = fabs(p[k] - hi);
        double f = f1 > f2 ? f1 : f2;
        dmax2 += f * f;
    }
    double dmin = sqrt(dmin2), dmax = sqrt(dmax2);
    if (dmax < zeta) return 0;
    if (dmin < zeta) dmin = zeta;
    *a = om_kappa_qpn(dmin, sigma);
    *b = om_kappa_qpn(dmax, sigma);
    return 1;
}

static int rotation_cube_outside_pi_ball(const double r0[3], double r_hw)
{
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double e = fabs(r0[k]) - r_hw;
        if (e > 0) d2 += e * e;
    }
    return sqrt(d2) > M_PI;
}

/* Theorem 1 bound on one self pair (i, j): a lower bound, over the
 * feasible part of C_t, of Z(K_1i1j(t)) / (Z(kappa_1i(t)) Z(kappa_1j(t))),
 * times phi_1i phi_1j.  Eq. (K1i1j_lb), Eq. (K1i1j_lb_A), readings R3, R4. */
static double self_lb_term_pre(const om_mix *m, int i, int j, const double *v, const double *psi, const double *a,
                               const double *b)
{
    double w = m->phi1[i] * m->phi1[j];
    if (i == j) {
        double k = a[i];
        return w * 0.5 * k / tanh(k);
    }
    double A = om_angle(v + 3 * i, v + 3 * j) + psi[i] + psi[j];
    if (A > M_PI) A = M_PI;
    double cA = cos(A);
#define KLB(k1, k2) sqrt((k1) * (k1) + (k2) * (k2) + 2.0 * (k1) * (k2) * cA)
    double Kbb = KLB(b[i], b[j]);
    double Kmax = Kbb;
    double c1 = KLB(a[i], b[j]), c2 = KLB(b[i], a[j]), c3 = KLB(a[i], a[j]);
    if (c1 > Kmax) Kmax = c1;
    if (c2 > Kmax) Kmax = c2;
    if (c3 > Kmax) Kmax = c3;
#undef KLB
    double lg = (Kbb - b[i] - b[j]) + om_phiZ(Kmax) - om_phiZ(a[i]) - om_phiZ(a[j]);
    return w * exp(lg);
}

/* Theorem 1 bound on one cross pair (i, j): an upper bound, over the
 * feasible part of C_r x C_t, of Z(K_1i2j) / (Z(kappa_1i(t)) Z(kappa_2j)),
 * times phi_1i phi_2j.  Eq. (K1i2j_ub), Eq. (K1i2j_ub_B), reading R3. */
static double cross_ub_term_pre(const om_mix *m, int i, int j, const double *v, const double *psi, const double *a,
                                const double *b, const double R0[9], double psir)
{
    /* psir: the rotation uncertainty angle of model direction i (R1, or R16 in mode 1) */
    double w = m->phi1[i] * m->phi2[j];
    double u[3];
    matTvec(R0, m->mu2 + 3 * j, u); /* R_r0^{-1} mu_2j */
    double B = om_angle(v + 3 * i, u) - psi[i] - psir;
    if (B < 0.0) B = 0.0;
    double cB = cos(B), k2 = m->kappa2[j];
#define KUB(k1) sqrt((k1) * (k1) + k2 * k2 + 2.0 * (k1) * k2 * cB)
    double ks = -k2 * cB;
    if (ks < a[i]) ks = a[i];
    if (ks > b[i]) ks = b[i];
    double Ka = KUB(a[i]), Kmin = KUB(ks);
#undef KUB
    double lg = (Ka - a[i] - k2) + om_phiZ(Kmin) - om_phiZ(b[i]) - om_phiZ(k2);
    return w * exp(lg);
}

/* Per-cube quantities shared by all pairs. */
typedef struct {
    double *v, *psi, *a, *b;
    double *psir_i; /* rotation uncertainty angle per model direction (R1, or R16 in mode 1) */
    double R0[9], psir, psit_max;
    int feasible, centre_feasible;
} cube_pre;

/* mode 0: psi_r of reading R1 for every model direction; mode 1: reading R16. */
static void cube_prepare(const om_mix *m, const double cube[CUBE_LEN], double zeta, int mode, cube_pre *cp)
{
    int n1 = m->n1;
    cp->v = malloc(sizeof(double) * 3 * n1);
    cp->psi = malloc(sizeof(double) * n1);
    cp->a = malloc(sizeof(double) * n1);
    cp->b = malloc(sizeof(double) * n1);
    cp->psir_i = malloc(sizeof(double) * n1);
    const double *t0 = cube + CUBE_T0, *thw = cube + CUBE_THW;
    om_rodrigues(cube + CUBE_R0, cp->R0);
    cp->psir = om_psi_r(cube[CUBE_RHW]);
    cp->feasible = !rotation_cube_outside_pi_ball(cube + CUBE_R0, cube[CUBE_RHW]);
    cp->centre_feasible = 1;
    cp->psit_max = 0.0;
    for (int i = 0; i < n1; ++i) {
        const double *p = m->mu1 + 3 * i;
        double c[3] = {p[0] - t0[0], p[1] - t0[1], p[2] - t0[2]};
        double d = norm3(c);
        if (d < zeta) cp->centre_feasible = 0;
        for (int k = 0; k < 3; ++k) cp->v[3 * i + k] = d > 0 ? c[k] / d : 0.0;
        cp->psir_i[i] = mode == 1 ? om_psi_r_point(cube + CUBE_R0, cube[CUBE_RHW], cp->v + 3 * i) : cp->psir;
        cp->psi[i] = om_psi_t(p, t0, thw);
        if (cp->psi[i] > cp->psit_max) cp->psit_max = cp->psi[i];
        if (!om_kappa_interval(p, m->sigma1[i], t0, thw, zeta, cp->a + i, cp->b + i)) cp->feasible = 0;
    }
}

static void cube_release(cube_pre *cp)
{
    free(cp->v);
    free(cp->psi);
    free(cp->a);
    free(cp->b);
    free(cp->psir_i);
}

double om_self_lb_term(const om_mix *m, int i, int j, const double cube[CUBE_LEN], double zeta)
{
    cube_pre cp;
    cube_prepare(m, cube, zeta, 0, &cp);
    double r = cp.feasible ? self_lb_term_pre(m, i, j, cp.v, cp.psi, cp.a, cp.b) : NAN;
    cube_release(&cp);
    return r;
}

double om_cross_ub_term(const om_mix *m, int i, int j, const double cube[CUBE_LEN], double zeta)
{
    cube_pre cp;
    cube_prepare(m, cube, zeta, 0, &cp);
    double r = cp.feasible ? cross_ub_term_pre(m, i, j, cp.v, cp.psi, cp.a, cp.b, cp.R0, cp.psir) : NAN;
    cube_release(&cp);
    return r;
}

/* Theorem 1 for one cube.  out[0] = lower bound, out[1] = upper bound
 * f(R_r0, t0), out[2] = self lower-bound sum, out[3] = cross upper-bound
 * sum (lb = out[2] - 2 out[3]), out[4] = self sum at the centre,
 * out[5] = cross sum at the centre (ub = out[4] - 2 out[5]), out[6] = psi_r,
 * out[7] = max_i psi_t(mu_1i).  Infeasible cubes (R5) get +inf bounds.
 * mode 0: psi_r of reading R1; mode 1: the point-dependent psi_r of
 * reading R16 in the cross pairs (out[6] stays the R1 angle, the one the
 * split rule compares). */
void om_bounds_mode(const om_mix *m, const double cube[CUBE_LEN], double zeta, int mode, double out[8])
{
    cube_pre cp;
    cube_prepare(m, cube, zeta, mode, &cp);
    out[6] = cp.psir;
    out[7] = cp.psit_max;
    if (!cp.feasible) {
        for (int k = 0; k < 6; ++k) out[k] = INFINITY;
        cube_release(&cp);
        return;
    }
    double slb = 0.0, cub = 0.0;
    for (int i = 0; i < m->n1; ++i)
        for (int j = 0; j < m->n1; ++j) slb += self_lb_term_pre(m, i, j, cp.v, cp.psi, cp.a, cp.b);
    for (int i = 0; i < m->n1; ++i)
        for (int j = 0; j < m->n2; ++j)
            cub += cross_ub_term_pre(m, i, j, cp.v, cp.psi, cp.a, cp.b, cp.R0, cp.psir_i[i]);
    out[0] = slb - 2.0 * cub;
    out[2] = slb;
    out[3] = cub;
    double sc = NAN, cc = NAN;
    int centre_defined = 1;
    for (int i = 0; i < m->n1; ++i) {
        const double *p = m->mu1 + 3 * i;
        if (p[0] == cube[CUBE_T0] && p[1] == cube[CUBE_T0 + 1] && p[2] == cube[CUBE_T0 + 2]) centre_defined = 0;
    }
    if (centre_defined) om_objective_parts(m, cp.R0, cube + CUBE_T0, &sc, &cc);
    out[4] = sc;
    out[5] = cc;
    out[1] = cp.centre_feasible ? sc - 2.0 * cc : INFINITY;
    cube_release(&cp);
}

void om_bounds(const om_mix *m, const double cube[CUBE_LEN], double zeta, double out[8])
{
    om_bounds_mode(m, cube, zeta, 0, out);
}

/* Bounds of many cubes, cubes in parallel (nthreads <= 0: library default). */
void om_bounds_batch_mode(const om_mix *m, int n, const double *cubes, double zeta, int mode, double *out, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int c = 0; c < n; ++c) om_bounds_mode(m, cubes + (size_t)CUBE_LEN * c, zeta, mode, out + 8 * (size_t)c);
    (void)nthreads;
}

void om_bounds_batch(const om_mix *m, int n, const double *cubes, double zeta, double *out, int nthreads)
{
    om_bounds_batch_mode(m, n, cubes, zeta, 0, out, nthreads);
}

int om_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* SMA (Sec. 5): L-BFGS on f from a start pose, restricted to feasible
 * translations (inside Omega'_t and at least zeta from every mean).      */
typedef struct {
    int max_iter;   /* outer iterations */
    int memory;     /* L-BFGS history length */
    double gtol;    /* stop when |g|_inf <= gtol */
} om_sma_opts;

static int pose_feasible(const om_mix *m, const om_domain *dom, const double x[6])
{
    for (int k = 0; k < 3; ++k)
        if (x[3 + k] < dom->t_lo[k] || x[3 + k] > dom->t_hi[k]) return 0;
    for (int i = 0; i < m->n1; ++i) {
        double c[3] = {m->mu1[3 * i] - x[3], m->mu1[3 * i + 1] - x[4], m->mu1[3 * i + 2] - x[5]};
        if (norm3(c) < dom->zeta) return 0;
    }
    return 1;
}

int om_sma(const om_mix *m, const om_domain *dom, const om_sma_opts *opt, const double x0[6], double x_out[6],
           double *f_out)
{
    int M = opt->memory > 0 ? opt->memory : 10, maxit = opt->max_iter > 0 ? opt->max_iter : 100;
    double gtol = opt->gtol > 0 ? opt->gtol : 1e-9;
    double x[6], g[6], f;
    memcpy(x, x0, sizeof x);
    if (!pose_feasible(m, dom, x)) {
        memcpy(x_out, x0, sizeof x);
        *f_out = INFINITY;
        return 0;
    }
    om_objective_grad(m, x, &f, g);
    double *S = calloc((size_t)M * 6, sizeof(double)), *Y = calloc((size_t)M * 6, sizeof(double)),
           *rho = calloc(M, sizeof(double));
    int hist = 0, head = 0, evals = 1;
    for (int it = 0; it < maxit; ++it) {
        double gmax = 0;
        for (int k = 0; k < 6; ++k)
            if (fabs(g[k]) > gmax) gmax = fabs(g[k]);
        if (gmax <= gtol) break;
        /* two-loop recursion */
        double q[6], alpha[64], d[6];
        memcpy(q, g, sizeof q);
        for (int h = 0; h < hist; ++h) {
            int idx = (head - 1 - h + M) % M;
            double s = 0;
            for (int k = 0; k < 6; ++k) s += S[6 * idx + k] * q[k];
            alpha[h] = rho[idx] * s;
            for (int k = 0; k < 6; ++k) q[k] -= alpha[h] * Y[6 * idx + k];
        }
        double gamma;
        if (hist > 0) {
            int idx = (head - 1 + M) % M;
            double sy = 0, yy = 0;
            for (int k = 0; k < 6; ++k) {
                sy += S[6 * idx + k] * Y[6 * idx + k];
                yy += Y[6 * idx + k] * Y[6 * idx + k];
            }
            gamma = sy / yy;
        } else {
            gamma = 1e-2 / gmax; /* first step moves the largest coordinate by 0.01 */
        }
        for (int k = 0; k < 6; ++k) q[k] *= gamma;
        for (int h = hist - 1; h >= 0; --h) {
            int idx = (head - 1 - h + M) % M;
            double s = 0;
            for (int k = 0; k < 6; ++k) s += Y[6 * idx + k] * q[k];
            double beta = rho[idx] * s;
            for (int k = 0; k < 6; ++k) q[k] += S[6 * idx + k] * (alpha[h] - beta);
        }
        double gd = 0;
        for (int k = 0; k < 6; ++k) {
            d[k] = -q[k];
            gd += g[k] * d[k];
        }
        if (!(gd < 0)) { /* not a descent direction: restart from steepest descent */
            hist = 0;
            head = 0;
            for (int k = 0; k < 6; ++k) d[k] = -g[k] * 1e-2 / gmax;
            gd = 0;
            for (int k = 0; k < 6; ++k) gd += g[k] * d[k];
        }
        /* backtracking Armijo line search over feasible points */
        double step = 1.0, xn[6], gn[6], fn = INFINITY;
        int ok = 0;
        for (int ls = 0; ls < 40; ++ls) {
            for (int k = 0; k < 6; ++k) xn[k] = x[k] + step * d[k];
            if (pose_feasible(m, dom, xn)) {
                om_objective_grad(m, xn, &fn, gn);
                ++evals;
                if (fn <= f + 1e-4 * step * gd) {
                    ok = 1;
                    break;
                }
            }
            step *= 0.5;
        }
        if (!ok) break;
        double sy = 0;
        for (int k = 0; k < 6; ++k) {
            S[6 * head + k] = xn[k] - x[k];
            Y[6 * head + k] = gn[k] - g[k];
            sy += S[6 * head + k] * Y[6 * head + k];
        }
        if (sy > 1e-300) {
            rho[head] = 1.0 / sy;
            head = (head + 1) % M;
            if (hist < M) ++hist;
        }
        double fprev = f;
        memcpy(x, xn, sizeof x);
        memcpy(g, gn, sizeof g);
        f = fn;
        if (fabs(fprev - f) <= 1e-15 * (1.0 + fabs(f))) break;
    }
    free(S);
    free(Y);
    free(rho);
    memcpy(x_out, x, sizeof x);
    *f_out = f;
    return evals;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 (GOSMA). */
typedef struct {
    double eps;          /* tolerance on the normalised L2 distance (R7) */
    int pop;             /* hypercubes removed from the queue per iteration */
    long long max_nodes; /* evaluated sub-cubes; <= 0: unlimited */
    double max_seconds;  /* <= 0: unlimited */
    int use_sma;         /* run SMA when a sub-cube improves the incumbent */
    int nthreads;        /* OpenMP threads for bound evaluation (<= 0: default) */
    om_sma_opts sma;
    int psi_mode;        /* 0: psi_r of reading R1; 1: point-dependent psi_r (R16) */
} om_bnb_opts;

typedef struct {
    double f;        /* d*, best objective found */
    double lb;       /* global lower bound at termination */
    double f_norm;   /* d* / C22 + 1 */
    double gap_norm; /* (d* - lb) / C22 */
    double c22;
    double r[3], t[3], R[9];
    long long nodes;      /* sub-cubes evaluated */
    long long iterations; /* loop iterations */
    long long sma_calls;
    long long queue_peak;
    double seconds;
    int status; /* 0: eps-optimal, 1: node limit, 2: time limit */
} om_bnb_result;

typedef struct {
    double lb;
    int depth;
    long long id;
    double cube[CUBE_LEN];
    double psir, psit_max;
} node;

static int node_before(const node *x, const node *y)
{
    if (x->lb != y->lb) return x->lb < y->lb;
    if (x->depth != y->depth) return x->depth > y->depth;
    return x->id < y->id;
}

typedef struct {
    node *a;
    long long n, cap;
} heap;

static void heap_push(heap *h, const node *x)
{
    if (h->n == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->a = realloc(h->a, sizeof(node) * h->cap);
    }
    long long k = h->n++;
    h->a[k] = *x;
    while (k > 0) {
        long long p = (k - 1) / 2;
        if (!node_before(&h->a[k], &h->a[p])) break;
        node tmp = h->a[p];
        h->a[p] = h->a[k];
        h->a[k] = tmp;
        k = p;
    }
}

static node heap_pop(heap *h)
{
    node top = h->a[0];
    h->a[0] = h->a[--h->n];
    long long k = 0;
    for (;;) {
        long long l = 2 * k + 1, r = l + 1, s = k;
        if (l < h->n && node_before(&h->a[l], &h->a[s])) s = l;
        if (r < h->n && node_before(&h->a[r], &h->a[s])) s = r;
        if (s == k) break;
        node tmp = h->a[s];
        h->a[s] = h->a[k];
        h->a[k] = tmp;
        k = s;
    }
    return top;
}

static double now_seconds(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

/* Children of a hypercube: split rotation or translation (reading R6),
 * eight sub-cubes either way (Sec. 4.1). */
static void branch(const node *p, node ch[8])
{
    int rot = p->psir >= p->psit_max;
    for (int k = 0; k < 8; ++k) {
        ch[k] = *p;
        ch[k].depth = p->depth + 1;
        double *c = ch[k].cube;
        if (rot) {
            double h = p->cube[CUBE_RHW] * 0.5;
            c[CUBE_RHW] = h;
            for (int a = 0; a < 3; ++a) c[CUBE_R0 + a] = p->cube[CUBE_R0 + a] + (((k >> a) & 1) ? h : -h);
        } else {
            for (int a = 0; a < 3; ++a) {
                double h = p->cube[CUBE_THW + a] * 0.5;
                c[CUBE_THW + a] = h;
                c[CUBE_T0 + a] = p->cube[CUBE_T0 + a] + (((k >> a) & 1) ? h : -h);
            }
        }
    }
}

int om_bnb(const om_mix *m, const om_domain *dom, const om_bnb_opts *opt, om_bnb_result *res)
{
    double t_start = now_seconds();
#ifdef _OPENMP
    if (opt->nthreads > 0) omp_set_num_threads(opt->nthreads);
#endif
    memset(res, 0, sizeof *res);
    double c22 = om_c22(m);
    double eps_f = opt->eps * c22;
    int P = opt->pop > 0 ? opt->pop : 1;
    heap h = {0};
    node root;
    memset(&root, 0, sizeof root);
    root.lb = -INFINITY;
    for (int k = 0; k < 3; ++k) {
        root.cube[CUBE_R0 + k] = 0.0;
        root.cube[CUBE_T0 + k] = 0.5 * (dom->t_lo[k] + dom->t_hi[k]);
        root.cube[CUBE_THW + k] = 0.5 * (dom->t_hi[k] - dom->t_lo[k]);
    }
    root.cube[CUBE_RHW] = M_PI;
    {
        double o[8];
        om_bounds_mode(m, root.cube, dom->zeta, opt->psi_mode, o);
        root.psir = o[6];
        root.psit_max = o[7];
    }
    heap_push(&h, &root);
    long long next_id = 1;
    double dstar = INFINITY, dlb = -INFINITY, best[6] = {0, 0, 0, 0, 0, 0};
    node *par = malloc(sizeof(node) * P);
    node *ch = malloc(sizeof(node) * 8 * (size_t)P);
    double *out = malloc(sizeof(double) * 8 * 8 * (size_t)P);
    res->status = 0;
    for (;;) {
        /* lowest lower bound in the queue */
        dlb = h.n > 0 ? h.a[0].lb : dstar;
        if (dlb > dstar) dlb = dstar;
        int np = 0;
        while (np < P && h.n > 0) par[np++] = heap_pop(&h);
        if (np == 0) break; /* queue exhausted: nothing below d* remains */
        if (dstar - dlb <= eps_f) break;
        if (opt->max_nodes > 0 && res->nodes >= opt->max_nodes) {
            res->status = 1;
            break;
        }
        if (opt->max_seconds > 0 && now_seconds() - t_start > opt->max_seconds) {
            res->status = 2;
            break;
        }
        int nc = 0;
        for (int p = 0; p < np; ++p) {
            branch(&par[p], ch + nc);
            for (int k = 0; k < 8; ++k) ch[nc + k].id = next_id++;
            nc += 8;
        }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
        for (int c = 0; c < nc; ++c) om_bounds_mode(m, ch[c].cube, dom->zeta, opt->psi_mode, out + 8 * c);
        res->nodes += nc;
        res->iterations += 1;
        for (int c = 0; c < nc; ++c) {
            double lb = out[8 * c], ub = out[8 * c + 1];
            ch[c].lb = lb;
            ch[c].psir = out[8 * c + 6];
            ch[c].psit_max = out[8 * c + 7];
            if (ub < dstar) {
                double x0[6], x1[6], f1 = ub;
                for (int k = 0; k < 3; ++k) {
                    x0[k] = ch[c].cube[CUBE_R0 + k];
                    x0[3 + k] = ch[c].cube[CUBE_T0 + k];
                }
                memcpy(x1, x0, sizeof x0);
                if (opt->use_sma) {
                    double fs;
                    om_sma(m, dom, &opt->sma, x0, x1, &fs);
                    res->sma_calls += 1;
                    if (fs < f1) f1 = fs;
                    else memcpy(x1, x0, sizeof x0);
                }
                dstar = f1;
                memcpy(best, x1, sizeof best);
            }
            if (lb < dstar) heap_push(&h, &ch[c]);
        }
        if (h.n > res->queue_peak) res->queue_peak = h.n;
    }
    res->f = dstar;
    res->lb = dlb;
    res->c22 = c22;
    res->f_norm = dstar / c22 + 1.0;
    res->gap_norm = (dstar - dlb) / c22;
    for (int k = 0; k < 3; ++k) {
        res->r[k] = best[k];
        res->t[k] = best[3 + k];
    }
    om_rodrigues(res->r, res->R);
    res->seconds = now_seconds() - t_start;
    free(h.a);
    free(par);
    free(ch);
    free(out);
    return res->status;
}
