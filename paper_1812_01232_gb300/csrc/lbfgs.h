// Local refinement of a pose (the SMA step of Sec. 5) as a resumable state
// machine: L-BFGS with memory 8 and a backtracking Armijo line search.  The
// caller evaluates the FP64 objective and gradient wherever the machine asks
// (want() gives the pose, give() returns f and the gradient), so one problem
// can be refined with one evaluation per call, or many problems in lock step
// with one batched evaluation per round.
//
// Trial poses that leave the translation domain or come within zeta of a
// model mean are skipped without evaluation (the step is halved), so the
// result is always a feasible pose whose f was evaluated exactly.
#pragma once

#include <math.h>
#include <string.h>

namespace gosma {

struct Feasibility {
    double t_lo[3], t_hi[3], zeta;
    const double *mu1;  // n1 x 3, host
    int n1;
    bool operator()(const double x[6]) const {
        for (int k = 0; k < 3; ++k)
            if (x[3 + k] < t_lo[k] || x[3 + k] > t_hi[k]) return false;
        const double z2 = zeta * zeta;
        for (int i = 0; i < n1; ++i) {
            double d0 = mu1[3 * i] - x[3], d1 = mu1[3 * i + 1] - x[4], d2 = mu1[3 * i + 2] - x[5];
            if (d0 * d0 + d1 * d1 + d2 * d2 < z2) return false;
        }
        return true;
    }
};

struct Lbfgs {
    static constexpr int M = 8;
    static constexpr int MAX_HALVINGS = 40;
    enum Phase { INIT, TRIAL, DONE };

    Feasibility feas;
    int max_iter = 100;
    Phase phase = DONE;
    double x[6], g[6], fx = 0;  // current iterate and its f, gradient
    double S[M][6], Y[M][6], rho[M];
    int head = 0, used = 0, it = 0;
    double d[6], slope = 0, step = 1, xn[6];
    int ls = 0;
    long long evals = 0;

    void start(const double x0[6], int iters) {
        memcpy(x, x0, sizeof x);
        max_iter = iters;
        head = used = it = 0;
        evals = 0;
        phase = INIT;
    }
    bool done() const { return phase == DONE; }

    // The pose to evaluate next; false once the refinement has finished.
    bool want(double p[6]) const {
        if (phase == INIT) memcpy(p, x, sizeof x);
        else if (phase == TRIAL) memcpy(p, xn, sizeof xn);
        return phase != DONE;
    }

    void give(double f, const double gr[6]) {
        ++evals;
        if (phase == INIT) {
            fx = f;
            memcpy(g, gr, sizeof g);
            begin_iteration();
            return;
        }
        if (phase != TRIAL) return;
        if (!(f <= fx + 1e-4 * step * slope)) {  // Armijo test failed: halve the step
            ++ls;
            step *= 0.5;
            next_trial();
            return;
        }
        double sy = 0;
        for (int k = 0; k < 6; ++k) {
            S[head][k] = xn[k] - x[k];
            Y[head][k] = gr[k] - g[k];
            sy += S[head][k] * Y[head][k];
        }
        if (sy > 0) {  // keep only curvature pairs that keep the inverse Hessian positive definite
            rho[head] = 1.0 / sy;
            head = (head + 1) % M;
            used = used < M ? used + 1 : M;
        }
        const double fprev = fx;
        memcpy(x, xn, sizeof x);
        memcpy(g, gr, sizeof g);
        fx = f;
        ++it;
        if (fabs(fprev - fx) <= 1e-15 * (1.0 + fabs(fx))) {
            phase = DONE;
            return;
        }
        begin_iteration();
    }

  private:
    // Two-loop recursion for the search direction, then the first trial step.
    void begin_iteration() {
        if (it >= max_iter) {
            phase = DONE;
            return;
        }
        double gn = 0;
        for (int k = 0; k < 6; ++k) gn = fmax(gn, fabs(g[k]));
        if (!(gn > 1e-10)) {
            phase = DONE;
            return;
        }
        double al[M];
        for (int k = 0; k < 6; ++k) d[k] = -g[k];
        for (int h = 0; h < used; ++h) {
            int j = (head - 1 - h + M) % M;
            double a = 0;
            for (int k = 0; k < 6; ++k) a += S[j][k] * d[k];
            al[h] = rho[j] * a;
            for (int k = 0; k < 6; ++k) d[k] -= al[h] * Y[j][k];
        }
        double scale = 0.01 / gn;  // first step: 0.01 in the largest coordinate
        if (used) {
            int j = (head - 1 + M) % M;
            double sy = 0, yy = 0;
            for (int k = 0; k < 6; ++k) {
                sy += S[j][k] * Y[j][k];
                yy += Y[j][k] * Y[j][k];
            }
            scale = sy / yy;
        }
        for (int k = 0; k < 6; ++k) d[k] *= scale;
        for (int h = used - 1; h >= 0; --h) {
            int j = (head - 1 - h + M) % M;
            double b = 0;
            for (int k = 0; k < 6; ++k) b += Y[j][k] * d[k];
            b *= rho[j];
            for (int k = 0; k < 6; ++k) d[k] += S[j][k] * (al[h] - b);
        }
        slope = 0;
        for (int k = 0; k < 6; ++k) slope += g[k] * d[k];
        if (!(slope < 0)) {  // lost descent: restart from a scaled gradient step
            used = 0;
            for (int k = 0; k < 6; ++k) d[k] = -g[k] * (0.01 / gn);
            slope = 0;
            for (int k = 0; k < 6; ++k) slope += g[k] * d[k];
        }
        step = 1.0;
        ls = 0;
        next_trial();
    }

    // First feasible pose along d at the current step or a halving of it.
    void next_trial() {
        for (; ls < MAX_HALVINGS; ++ls, step *= 0.5) {
            for (int k = 0; k < 6; ++k) xn[k] = x[k] + step * d[k];
            if (feas(xn)) {
                phase = TRIAL;
                return;
            }
        }
        phase = DONE;
    }
};

}  // namespace gosma
