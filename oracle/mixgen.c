/*
 * Mixture generation for GOSMA (Campbell et al., Sec. 6): the 3D point set
 * is clustered with DP-means (Kulis and Jordan, "Revisiting k-means: new
 * algorithms via Bayesian nonparametrics", 2012) and the image's bearing
 * vectors with DP-vMF-means (Straub et al., "Small-variance nonparametric
 * clustering on the hypersphere", 2015); a maximum-likelihood mixture is
 * then fitted to the clusters: a GMM (theta_1 = {mu, sigma, phi}) and a
 * vMFMM (theta_2 = {mu, kappa, phi}), the inputs of gosma_set_mixtures.
 *
 * TEST INFRASTRUCTURE ONLY (part of the oracle library): the tests, the
 * smoke check and the benchmark's CPU leg may call it; the CUDA library
 * never does, and the two share no code.
 *
 * Plain serial double precision, compiled without FMA contraction, in the
 * order the algorithms state.  Readings where the cited papers leave a
 * choice (listed in the repository's design notes):
 *   M1  coordinates are first rounded to multiples of 2^-32 (points, in the
 *       input's unit) or 2^-40 (unit bearing vectors), so that a cluster's
 *       coordinate sum is exact in 64-bit integers whatever the order of
 *       summation; a mean is that exact sum divided by the count, i.e.
 *       ((double)S / (double)n) * 2^-32, and a mean direction is the sum
 *       divided by its norm, (double)S_k / sqrt(S0^2 + S1^2 + S2^2).
 *   M2  one pass visits the points in index order.  A point whose squared
 *       distance to every current centre exceeds lambda (DP-means), or whose
 *       cosine with every centre is below lambda (DP-vMF-means), opens a
 *       new cluster centred on itself, which later points of the same pass
 *       see; every other point joins its nearest (most similar) centre, the
 *       lowest index on ties.  After the pass each centre becomes its
 *       cluster's mean (mean direction); empty clusters are removed, the
 *       others keep their order.  A cluster whose direction sum is exactly
 *       zero is centred on its lowest-index point.  Start: one cluster at
 *       the mean (mean direction) of all points.  Stop: a pass that changes
 *       no label, or max_iter passes.
 *   M3  fits: weight n_k / N; GMM: isotropic maximum likelihood
 *       sigma^2 = sum |x - mu|^2 / (3 n_k), floored at sigma_min; vMF: kappa
 *       solving coth(kappa) - 1/kappa = |sum x| / n_k (the maximum-likelihood
 *       equation on the sphere S^2), by bisection on log kappa, capped at
 *       kappa_max.
 * The squared distance is ((dx*dx + dy*dy) + dz*dz) and the cosine
 * ((x0*m0 + x1*m1) + x2*m2), each product and sum rounded once.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MG_SCALE_PTS 4294967296.0       /* 2^32 */
#define MG_SCALE_DIR 1099511627776.0    /* 2^40 */

static double mg_score(int vmf, const double *x, const double *m) {
    if (vmf) return (x[0] * m[0] + x[1] * m[1]) + x[2] * m[2];
    double d0 = x[0] - m[0], d1 = x[1] - m[1], d2 = x[2] - m[2];
    return (d0 * d0 + d1 * d1) + d2 * d2;
}
static int mg_better(int vmf, double a, double b) { return vmf ? a > b : a < b; }
static int mg_opens(int vmf, double best, double lambda) { return vmf ? best < lambda : best > lambda; }

/* Centre of a cluster from its exact integer sum S (3), count n and the
 * quantized coordinates of its lowest-index point xf (M1, M2). */
static void mg_centre(int vmf, const int64_t *S, long long n, const double *xf, double *m) {
    if (!vmf) {
        for (int k = 0; k < 3; ++k) m[k] = ((double)S[k] / (double)n) * (1.0 / MG_SCALE_PTS);
        return;
    }
    double s0 = (double)S[0], s1 = (double)S[1], s2 = (double)S[2];
    double nr = sqrt((s0 * s0 + s1 * s1) + s2 * s2);
    if (nr == 0.0) {
        for (int k = 0; k < 3; ++k) m[k] = xf[k];
        return;
    }
    m[0] = s0 / nr;
    m[1] = s1 / nr;
    m[2] = s2 / nr;
}

/* coth(k) - 1/k, the mean resultant length of a vMF on S^2 with concentration k */
static double mg_A3(double k) {
    if (k < 1e-3) return k / 3.0 - k * k * k / 45.0;
    return 1.0 / tanh(k) - 1.0 / k;
}

/*
 * Cluster n points x (n x 3) and fit the mixture.  vmf = 0: DP-means with
 * penalty lambda (squared distance), fit a GMM (sigma floored at lo);
 * vmf = 1: DP-vMF-means with cosine threshold lambda, fit a vMFMM (kappa
 * capped at hi).  Outputs (kmax-sized): mu (k x 3), spread (sigma or kappa),
 * phi; labels (n); returns the number of clusters k, or -1 when more than
 * kmax clusters would be needed; *passes = passes run.
 */
int om_dp_cluster(int vmf, int n, const double *x, double lambda, int max_iter, int kmax, double lo, double hi,
                  double *mu, double *spread, double *phi, int *labels, int *passes) {
    const double scale = vmf ? MG_SCALE_DIR : MG_SCALE_PTS;
    int64_t *q = malloc(sizeof(int64_t) * 3 * (size_t)n);
    double *xq = malloc(sizeof(double) * 3 * (size_t)n);
    int64_t *S = malloc(sizeof(int64_t) * 3 * (size_t)(kmax + 1));
    long long *cnt = malloc(sizeof(long long) * (size_t)(kmax + 1));
    int *first = malloc(sizeof(int) * (size_t)(kmax + 1));
    int *remap = malloc(sizeof(int) * (size_t)(kmax + 1));
    double *cen = malloc(sizeof(double) * 3 * (size_t)(kmax + 1));
    int K = 1, pass = 0, ok = 1;
    for (int i = 0; i < 3 * n; ++i) {
        q[i] = llrint(x[i] * scale);
        xq[i] = (double)q[i] / scale;
    }
    /* start: one cluster at the mean of all points */
    S[0] = S[1] = S[2] = 0;
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) S[k] += q[3 * i + k];
        labels[i] = 0;
    }
    mg_centre(vmf, S, n, xq, cen);
    for (pass = 0; pass < max_iter; ++pass) {
        int changed = 0;
        for (int i = 0; i < n && ok; ++i) {
            double best = mg_score(vmf, xq + 3 * i, cen);
            int arg = 0;
            for (int c = 1; c < K; ++c) {
                double s = mg_score(vmf, xq + 3 * i, cen + 3 * c);
                if (mg_better(vmf, s, best)) {
                    best = s;
                    arg = c;
                }
            }
            if (mg_opens(vmf, best, lambda)) { /* a new cluster centred on x_i */
                if (K >= kmax) {
                    ok = 0;
                    break;
                }
                memcpy(cen + 3 * K, xq + 3 * i, 3 * sizeof(double));
                arg = K++;
            }
            if (arg != labels[i]) ++changed;
            labels[i] = arg;
        }
        if (!ok) break;
        /* centres become the means; empty clusters are removed */
        memset(S, 0, sizeof(int64_t) * 3 * (size_t)K);
        memset(cnt, 0, sizeof(long long) * (size_t)K);
        for (int c = 0; c < K; ++c) first[c] = n;
        for (int i = 0; i < n; ++i) {
            int c = labels[i];
            for (int k = 0; k < 3; ++k) S[3 * c + k] += q[3 * i + k];
            ++cnt[c];
            if (i < first[c]) first[c] = i;
        }
        int Kn = 0;
        for (int c = 0; c < K; ++c) {
            if (cnt[c] == 0) {
                remap[c] = -1;
                continue;
            }
            remap[c] = Kn;
            mg_centre(vmf, S + 3 * c, cnt[c], xq + 3 * first[c], cen + 3 * Kn);
            ++Kn;
        }
        if (Kn < K)
            for (int i = 0; i < n; ++i) labels[i] = remap[labels[i]];
        K = Kn;
        if (changed == 0) {
            ++pass;
            break;
        }
    }
    *passes = pass;
    if (!ok) {
        free(q), free(xq), free(S), free(cnt), free(first), free(remap), free(cen);
        return -1;
    }
    /* maximum-likelihood fits (M3) */
    double *ss = calloc((size_t)K, sizeof(double));
    memset(S, 0, sizeof(int64_t) * 3 * (size_t)K);
    memset(cnt, 0, sizeof(long long) * (size_t)K);
    for (int i = 0; i < n; ++i) {
        int c = labels[i];
        for (int k = 0; k < 3; ++k) S[3 * c + k] += q[3 * i + k];
        ++cnt[c];
        if (!vmf) ss[c] += mg_score(0, xq + 3 * i, cen + 3 * c);
    }
    for (int c = 0; c < K; ++c) {
        memcpy(mu + 3 * c, cen + 3 * c, 3 * sizeof(double));
        phi[c] = (double)cnt[c] / (double)n;
        if (!vmf) {
            double s = sqrt(ss[c] / (3.0 * (double)cnt[c]));
            spread[c] = s > lo ? s : lo;
        } else {
            double s0 = (double)S[3 * c], s1 = (double)S[3 * c + 1], s2 = (double)S[3 * c + 2];
            double rbar = sqrt((s0 * s0 + s1 * s1) + s2 * s2) / (scale * (double)cnt[c]);
            if (!(mg_A3(hi) > rbar)) {
                spread[c] = hi;
            } else {
                double a = log(1e-12), b = log(hi);
                for (int it = 0; it < 200; ++it) {
                    double m = 0.5 * (a + b);
                    if (mg_A3(exp(m)) < rbar) a = m;
                    else b = m;
                }
                spread[c] = exp(0.5 * (a + b));
            }
        }
    }
    free(ss);
    free(q), free(xq), free(S), free(cnt), free(first), free(remap), free(cen);
    return K;
}
