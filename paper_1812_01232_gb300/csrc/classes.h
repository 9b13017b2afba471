// Semantic classes (Sec. 4.2) on the host: the class layout of a mixture
// pair (components given class by class), checked, with each class's weights
// scaled by sqrt(w_l) so that within-class pair sums give sum_l w_l f_l, the
// class of every component and the within-class pair ranges of every model
// row.  One class of weight 1 leaves the weights unchanged.
#pragma once

#include <math.h>

#include <vector>

namespace gosma {

struct ClassLayout {
    std::vector<double> phi1, phi2;                // scaled weights
    std::vector<int> cls1, cls2, rj0, rj1, rm1;  // class ids; columns [rj0, rj1), rows below rm1
    bool classes = false;                          // more than one class
};

// nclass classes of n1c[l] / n2c[l] components (NULL: one class of all) with
// weights w (NULL: 1).  Returns an error message, or nullptr when valid.
inline const char *class_layout(int nclass, const int *n1c, const int *n2c, const double *w, int n1, int n2,
                                const double *phi1, const double *phi2, ClassLayout &L) {
    if (nclass < 1) return "at least one class";
    L.phi1.assign(phi1, phi1 + n1);
    L.phi2.assign(phi2, phi2 + n2);
    L.cls1.assign(n1, 0);
    L.cls2.assign(n2, 0);
    L.rj0.assign(n1, 0);
    L.rj1.assign(n1, n2);
    L.rm1.assign(n1, n1);
    int i0 = 0, j0 = 0;
    for (int l = 0; l < nclass; ++l) {
        const int a = n1c ? n1c[l] : n1, b = n2c ? n2c[l] : n2;
        const double wl = w ? w[l] : 1.0;
        if (a < 1 || b < 1 || i0 + a > n1 || j0 + b > n2 || !(wl >= 0) || !isfinite(wl))
            return "class sizes must be >= 1 and sum to n1 and n2; class weights >= 0";
        double s1 = 0, s2 = 0;
        for (int i = i0; i < i0 + a; ++i) s1 += L.phi1[i];
        for (int j = j0; j < j0 + b; ++j) s2 += L.phi2[j];
        if (fabs(s1 - 1.0) > 1e-9 || fabs(s2 - 1.0) > 1e-9) return "each class's mixture weights must sum to 1";
        const double sw = sqrt(wl);
        for (int i = i0; i < i0 + a; ++i) {
            L.phi1[i] *= sw;
            L.cls1[i] = l;
            L.rj0[i] = j0;
            L.rj1[i] = j0 + b;
            L.rm1[i] = i0 + a;
        }
        for (int j = j0; j < j0 + b; ++j) {
            L.phi2[j] *= sw;
            L.cls2[j] = l;
        }
        i0 += a;
        j0 += b;
    }
    if (i0 != n1 || j0 != n2) return "class sizes must sum to n1 and n2";
    L.classes = nclass > 1;
    return nullptr;
}

}  // namespace gosma
