// SMA (Sec. 5) from many seed poses at once, entirely on the device.
//
// One thread block refines one seed at a time (a persistent grid takes seeds
// from a work counter): L-BFGS with memory 8 on f of Lemma 1, the two-loop
// recursion and the backtracking Armijo line search kept by thread 0 in shared
// memory, every evaluation of f and its gradient spread over the block.  Trial
// poses that leave the translation domain or come within zeta of a model mean
// are skipped without evaluation (the step is halved), as in the host
// refinement, so every result is a feasible pose.  No host round trip happens
// between iterations.
//
// Two evaluation precisions:
//   64  FP64 throughout (the pair terms of objective_core.cuh).
//   32  the search evaluates f and its gradient in FP32 (GB300 runs FP32 at
//       about 64x its FP64 rate), with the pair exponent and its derivatives
//       in forms that do not cancel (below); it stops when a step gains
//       nothing measurable or the line search runs out of halvings.  The
//       returned f is always the FP64 f of the returned pose, so d* stays an
//       exact objective value.
#include <math.h>

#include "host_rules.h"
#include "objective_core.cuh"

namespace gosma {

// Threads per seed: sma_block_for (host_rules.h), 128 to 1,024.
constexpr int SMA_BLOCK = 128;

constexpr int SMA_M = 8;  // L-BFGS memory

// L-BFGS state of the block's current seed (shared memory; thread 0 writes).
struct SmaState {
    double x[6], g[6], f, fmag;    // iterate, gradient, f, sum of |terms|
    double xn[6], gn[6], fn, fnmag;  // trial pose
    double d[6], slope, step;
    double S[SMA_M][6], Y[SMA_M][6], rho[SMA_M];
    double R[9];
    int head, used, flag;
};

// ---------------------------------------------------------------- FP32 pair terms
// phi_Z(x) = log Z(x) - x = log((1 - e^{-2x}) / x).
__device__ __forceinline__ float phiz32(float x) {
    if (x < 1e-2f) return 0.69314718f - x + x * x * (1.f / 6.f);
    float e = __expf(-2.f * x);
    float l = e < 1e-4f ? -e - 0.5f * e * e : log1pf(-e);
    return l - __logf(x);
}
// coth x - 1.
__device__ __forceinline__ float cothm1_32(float x) {
    if (x < 1e-3f) return __fdividef(1.f, x) - 1.f + x * (1.f / 3.f);
    if (x > 40.f) return 0.f;
    return __fdividef(2.f * __expf(-2.f * x), -expm1f(-2.f * x));
}
// h(x) = d log Z / dx = coth x - 1/x, given gx = coth x - 1.
__device__ __forceinline__ float h32(float x, float gx) {
    if (x < 1e-2f) return x * (1.f / 3.f) - x * x * x * (1.f / 45.f);
    return 1.f + gx - __fdividef(1.f, x);
}

// Rodrigues' formula in FP32, with (1 - cos th)/th^2 = 2 sin^2(th/2)/th^2
// so that small angles do not cancel.
__device__ __forceinline__ void rodrigues32(const double *r, float R[9]) {
    const float x = (float)r[0], y = (float)r[1], z = (float)r[2];
    const float th2 = x * x + y * y + z * z, th = sqrtf(th2);
    float A, B;
    if (th < 1e-4f) {
        A = 1.f - th2 * (1.f / 6.f);
        B = 0.5f - th2 * (1.f / 24.f);
    } else {
        float sh, ch;
        sincosf(0.5f * th, &sh, &ch);
        A = 2.f * sh * ch / th;
        const float sc = sh / (0.5f * th);
        B = 0.5f * sc * sc;
    }
    R[0] = 1.f - B * (y * y + z * z);
    R[1] = -A * z + B * x * y;
    R[2] = A * y + B * x * z;
    R[3] = A * z + B * x * y;
    R[4] = 1.f - B * (x * x + z * z);
    R[5] = -A * x + B * y * z;
    R[6] = -A * y + B * x * z;
    R[7] = A * x + B * y * z;
    R[8] = 1.f - B * (x * x + y * y);
}

// FP32 twin of obj_finish: (f, df/dt, df/domega) -> (f, df/dr, df/dt) with
// the left Jacobian; a = (1 - cos th)/th^2 and b = (th - sin th)/th^3 by
// their series below th = 1/2 (b cancels there).
__device__ __forceinline__ void finish32(const double *rd, double f, const float s[6], double *o) {
    const float r[3] = {(float)rd[0], (float)rd[1], (float)rd[2]};
    const float th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], th = sqrtf(th2);
    float a, b;
    if (th < 0.5f) {
        a = 0.5f - th2 * (1.f / 24.f) + th2 * th2 * (1.f / 720.f) - th2 * th2 * th2 * (1.f / 40320.f);
        b = 1.f / 6.f - th2 * (1.f / 120.f) + th2 * th2 * (1.f / 5040.f) - th2 * th2 * th2 * (1.f / 362880.f);
    } else {
        float sn, cs, sh, ch;
        sincosf(th, &sn, &cs);
        sincosf(0.5f * th, &sh, &ch);
        a = 2.f * sh * sh / th2;
        b = (th - sn) / (th2 * th);
    }
    const float *gw = s + 3;
    const float rxg[3] = {r[1] * gw[2] - r[2] * gw[1], r[2] * gw[0] - r[0] * gw[2], r[0] * gw[1] - r[1] * gw[0]};
    const float rg = r[0] * gw[0] + r[1] * gw[1] + r[2] * gw[2];
    o[0] = f;
    for (int c = 0; c < 3; ++c) o[1 + c] = gw[c] - a * rxg[c] + b * (r[c] * rg - th2 * gw[c]);
    for (int c = 0; c < 3; ++c) o[4 + c] = s[c];
}

// dE/da at fixed b and c = cos of the angle, where E = log Z(K) - log Z(a)
// - log Z(b) and K^2 = a^2 + b^2 + 2abc.  Written as h(K)(a + bc)/K - h(a),
// which cancels for large a, b and aligned vectors; there the same value is
// formed from (h(K) - h(a)) = (K - a)/(aK) + (coth K - coth a) and
// (a + bc)/K - 1 = -b^2 (1 - c^2) / (K (K + a + bc)), q = 1 - c^2.
__device__ __forceinline__ float dE32(float a, float ga, float b, float c, float q, float K, float gK, float hK) {
    const float abc = a + b * c;
    if (K >= 1.f && abc > 0.f) {
        const float Kma = __fdividef(b * (b + 2.f * a * c), K + a);
        return __fdividef(Kma, a * K) + (gK - ga) - __fdividef(hK * b * b * q, K * (K + abc));
    }
    const float hk_k = K > 1e-6f ? __fdividef(hK, K) : (1.f / 3.f);
    return hk_k * abc - h32(a, ga);
}

// E and its partial derivatives for concentrations a, b and unit vectors at
// squared distance s2 = |u - w|^2 (so c = 1 - s2/2).  K - a - b is taken as
// -ab s2 / (K + a + b).
struct Pair32 {
    float E, Ea, Eb, Ec;
};
template <bool NEED_B>
__device__ __forceinline__ Pair32 pair32(float a, float pza, float ga, float b, float pzb, float gb, float s2) {
    Pair32 p;
    const float c = 1.f - 0.5f * s2, q = s2 * (1.f - 0.25f * s2), sum = a + b, ab = a * b;
    const float K = sqrtf(fmaxf(fmaf(-ab, s2, sum * sum), 0.f));
    p.E = __fdividef(-ab * s2, K + sum) + phiz32(K) - pza - pzb;
    const float gK = cothm1_32(K), hK = h32(K, gK);
    p.Ec = K > 1e-6f ? __fdividef(hK * ab, K) : ab * (1.f / 3.f);
    p.Ea = dE32(a, ga, b, c, q, K, gK, hK);
    p.Eb = NEED_B ? dE32(b, gb, a, c, q, K, gK, hK) : 0.f;
    return p;
}

// Shared-memory tables of the FP32 evaluation.
struct Sma32Tab {
    float4 *ma;   // n1: v (3), 1/d            (per pose)
    float4 *mb;   // n1: kappa, phi_Z(kappa), coth kappa - 1, -2 (kappa - 1)/d  (per pose)
    float *phi1;  // n1
    float4 *ja;   // n2: R^T mu_2j (3), kappa_2j (per pose)
    float2 *jb;   // n2: phi_Z(kappa_2j), phi_2j
};

__host__ __device__ inline size_t sma32_smem_bytes(int n1, int n2) {
    return (size_t)n1 * (2 * sizeof(float4) + sizeof(float)) + (size_t)n2 * (sizeof(float4) + sizeof(float2)) + 64;
}

__device__ inline Sma32Tab sma32_carve(void *base, int n1, int n2) {
    Sma32Tab t;
    float4 *p = reinterpret_cast<float4 *>(base);
    t.ma = p;
    t.mb = p + n1;
    t.ja = p + 2 * n1;
    t.jb = reinterpret_cast<float2 *>(p + 2 * n1 + n2);
    t.phi1 = reinterpret_cast<float *>(t.jb + n2);
    return t;
}

// Compensated pair (s, c) for the FP32 sum of f.
__device__ __forceinline__ void two_sum_add(float &s, float &c, float x) {
    float t = s + x, z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
}

// f, df/dr, df/dt at the pose xs (shared) with FP32 terms.  Thread 0 writes
// out (7 doubles: f, df/dr, df/dt) and *mag (sum of |weighted terms|).
// Every thread must call it; it ends with a barrier.
template <int B>
__device__ void sma_eval32(const MixDev &mx, const Sma32Tab &tb, const double *xs, double *out, double *mag,
                           float (*red)[B / 32]) {
    const int tid = threadIdx.x, n1 = mx.n1, n2 = mx.n2;
    float R[9];
    rodrigues32(xs, R);
    // t as a double-float, so that mu - t keeps FP32 relative accuracy
    float th[3], tl[3];
    for (int k = 0; k < 3; ++k) {
        th[k] = (float)xs[3 + k];
        tl[k] = (float)(xs[3 + k] - (double)th[k]);
    }
    for (int i = tid; i < n1; i += B) {
        const float m0 = (mx.mu1h[3 * i] - th[0]) + (mx.mu1l[3 * i] - tl[0]);
        const float m1 = (mx.mu1h[3 * i + 1] - th[1]) + (mx.mu1l[3 * i + 1] - tl[1]);
        const float m2 = (mx.mu1h[3 * i + 2] - th[2]) + (mx.mu1l[3 * i + 2] - tl[2]);
        const float d2 = m0 * m0 + m1 * m1 + m2 * m2, id = rsqrtf(d2);
        const float k = fmaf(d2, mx.inv_sig2[i], 1.f);  // Eq. (kappa1)
        tb.ma[i] = make_float4(m0 * id, m1 * id, m2 * id, id);
        tb.mb[i] = make_float4(k, phiz32(k), cothm1_32(k), -2.f * (k - 1.f) * id);
    }
    for (int j = tid; j < n2; j += B) {
        const float u0 = mx.mu2h[3 * j], u1 = mx.mu2h[3 * j + 1], u2 = mx.mu2h[3 * j + 2];
        tb.ja[j] = make_float4(R[0] * u0 + R[3] * u1 + R[6] * u2, R[1] * u0 + R[4] * u1 + R[7] * u2,
                               R[2] * u0 + R[5] * u1 + R[8] * u2, mx.kappa2[j]);
    }
    __syncthreads();
    float fs = 0.f, fc = 0.f, fa = 0.f, gt0 = 0.f, gt1 = 0.f, gt2 = 0.f, gw0 = 0.f, gw1 = 0.f, gw2 = 0.f;
    // self pairs i <= j (weight 2 off the diagonal) over the flattened square
    {
        const int nn = n1 * n1, si = B / n1, sj = B % n1;
        int i = tid / n1, j = tid % n1;
        for (int q = tid; q < nn; q += B) {
            if (j >= i && !(mx.cls1 && mx.cls1[i] != mx.cls1[j])) {
                const float4 A = tb.ma[i], Ab = tb.mb[i], Bm = tb.ma[j], Bb = tb.mb[j];
                const float e0 = A.x - Bm.x, e1 = A.y - Bm.y, e2 = A.z - Bm.z;
                const float s2 = e0 * e0 + e1 * e1 + e2 * e2;
                const Pair32 p = pair32<true>(Ab.x, Ab.y, Ab.z, Bb.x, Bb.y, Bb.z, s2);
                const float T = (i == j ? 1.f : 2.f) * tb.phi1[i] * tb.phi1[j] * __expf(p.E);
                two_sum_add(fs, fc, T);
                fa += T;
                const float c = 1.f - 0.5f * s2;
                const float ca = T * p.Ea * Ab.w, cb = T * p.Eb * Bb.w, ce = T * p.Ec;
                // dc/dt = -[(v_j - c v_i)/d_i + (v_i - c v_j)/d_j]
                gt0 += ca * A.x + cb * Bm.x - ce * ((Bm.x - c * A.x) * A.w + (A.x - c * Bm.x) * Bm.w);
                gt1 += ca * A.y + cb * Bm.y - ce * ((Bm.y - c * A.y) * A.w + (A.y - c * Bm.y) * Bm.w);
                gt2 += ca * A.z + cb * Bm.z - ce * ((Bm.z - c * A.z) * A.w + (A.z - c * Bm.z) * Bm.w);
            }
            j += sj;
            i += si;
            if (j >= n1) {
                j -= n1;
                ++i;
            }
        }
    }
    // cross pairs in the model frame: u = v_i, w = R^T mu_2j
    {
        const int nn = n1 * n2, si = B / n2, sj = B % n2;
        int i = tid / n2, j = tid % n2;
        for (int q = tid; q < nn; q += B) {
            if (!(mx.cls1 && mx.cls1[i] != mx.cls2[j])) {
                const float4 A = tb.ma[i], Ab = tb.mb[i], W = tb.ja[j];
                const float2 Wb = tb.jb[j];
                const float e0 = A.x - W.x, e1 = A.y - W.y, e2 = A.z - W.z;
                const float s2 = e0 * e0 + e1 * e1 + e2 * e2;
                const Pair32 p = pair32<false>(Ab.x, Ab.y, Ab.z, W.w, Wb.x, 0.f, s2);
                const float T = 2.f * tb.phi1[i] * Wb.y * __expf(p.E);
                two_sum_add(fs, fc, -T);
                fa += T;
                const float c = 1.f - 0.5f * s2;
                const float ca = -T * p.Ea * Ab.w, ce = -T * p.Ec;
                gt0 += ca * A.x - ce * (W.x - c * A.x) * A.w;
                gt1 += ca * A.y - ce * (W.y - c * A.y) * A.w;
                gt2 += ca * A.z - ce * (W.z - c * A.z) * A.w;
                // dc/domega (model frame) = v_i x R^T mu_2j
                gw0 += ce * (A.y * W.z - A.z * W.y);
                gw1 += ce * (A.z * W.x - A.x * W.z);
                gw2 += ce * (A.x * W.y - A.y * W.x);
            }
            j += sj;
            i += si;
            if (j >= n2) {
                j -= n2;
                ++i;
            }
        }
    }
    // block reduction in FP32 (the f sum carries its compensation term)
    float v[9] = {fs, fc, fa, gt0, gt1, gt2, gw0, gw1, gw2};
    for (int o = 16; o > 0; o >>= 1) {
        const float s = __shfl_down_sync(0xffffffffu, v[0], o), c = __shfl_down_sync(0xffffffffu, v[1], o);
        two_sum_add(v[0], v[1], s);
        v[1] += c;
        for (int k = 2; k < 9; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    if ((tid & 31) == 0)
        for (int k = 0; k < 9; ++k) red[k][tid >> 5] = v[k];
    __syncthreads();
    if (tid == 0) {
        float f0 = red[0][0], f1 = red[1][0], fab = red[2][0], g[6];
        for (int k = 0; k < 6; ++k) g[k] = red[3 + k][0];
        for (int w = 1; w < B / 32; ++w) {
            two_sum_add(f0, f1, red[0][w]);
            f1 += red[1][w];
            fab += red[2][w];
            for (int k = 0; k < 6; ++k) g[k] += red[3 + k][w];
        }
        // omega gradient back to the world frame: R (sum of model-frame terms)
        const float gm[3] = {g[3], g[4], g[5]};
        for (int c = 0; c < 3; ++c) g[3 + c] = R[3 * c] * gm[0] + R[3 * c + 1] * gm[1] + R[3 * c + 2] * gm[2];
        finish32(xs, (double)f0 + (double)f1, g, out);
        *mag = fab;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- FP64 evaluation
// Same outputs through the FP64 pair terms; rows is this block's n1 x
// OBJ_STRIDE scratch.
template <int B>
__device__ void sma_eval64(const MixDev &mx, double *rows, double *Rs, const double *xs, double *out, double *mag,
                           double (*red)[B / 32]) {
    const int tid = threadIdx.x, n1 = mx.n1;
    if (tid == 0) rodrigues_dev(xs, Rs);
    __syncthreads();
    for (int i = tid; i < n1; i += B) obj_row(mx, Rs, xs + 3, i, rows + (size_t)i * OBJ_STRIDE);
    __syncthreads();
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const long long total = (long long)n1 * n1 + (long long)n1 * mx.n2;
    for (long long q = tid; q < total; q += B) obj_pair(mx, rows, Rs, q, acc);
    for (int k = 0; k < 7; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    if ((tid & 31) == 0)
        for (int k = 0; k < 7; ++k) red[k][tid >> 5] = acc[k];
    __syncthreads();
    if (tid == 0) {
        double s[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < B / 32; ++w)
            for (int k = 0; k < 7; ++k) s[k] += red[k][w];
        obj_finish(xs, s, out);
        *mag = fabs(s[0]);
    }
    __syncthreads();
}

// ---------------------------------------------------------------- L-BFGS steps (warp 0)
// Lane k < 6 of warp 0 holds coordinate k and lanes 6..31 hold zeros.  Dot
// products and the gradient's max norm are reduced over all 32 lanes, so
// every lane sees the same value and takes the same branch: the shuffles
// below always run with the whole warp.
__device__ __forceinline__ double sum32(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double max32(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Search direction by the two-loop recursion; st.flag = 1 when the gradient
// has vanished.  Called by all of warp 0.
__device__ void lbfgs_direction(SmaState &st) {
    const int k = threadIdx.x;
    const bool on = k < 6;
    const double gk = on ? st.g[k] : 0.0;
    const double gn = max32(fabs(gk));
    const int used = st.used, head = st.head;
    __syncwarp();
    if (!(gn > 1e-10)) {
        if (k == 0) st.flag = 1;
        return;
    }
    double d = -gk, al[SMA_M];
#pragma unroll
    for (int h = 0; h < SMA_M; ++h) {
        if (h < used) {
            const int j = (head - 1 - h + SMA_M) % SMA_M;
            al[h] = st.rho[j] * sum32(on ? st.S[j][k] * d : 0.0);
            if (on) d -= al[h] * st.Y[j][k];
        }
    }
    double scale = 0.01 / gn;  // first step: 0.01 in the largest coordinate
    if (used) {
        const int j = (head - 1 + SMA_M) % SMA_M;
        const double sy = sum32(on ? st.S[j][k] * st.Y[j][k] : 0.0);
        const double yy = sum32(on ? st.Y[j][k] * st.Y[j][k] : 0.0);
        scale = sy / yy;
    }
    d *= scale;
#pragma unroll
    for (int h = SMA_M - 1; h >= 0; --h) {
        if (h < used) {
            const int j = (head - 1 - h + SMA_M) % SMA_M;
            const double b = st.rho[j] * sum32(on ? st.Y[j][k] * d : 0.0);
            if (on) d += st.S[j][k] * (al[h] - b);
        }
    }
    double slope = sum32(gk * d);
    int nused = used;
    if (!(slope < 0.0)) {  // lost descent: restart from a scaled gradient step
        nused = 0;
        d = -gk * (0.01 / gn);
        slope = sum32(gk * d);
    }
    if (on) st.d[k] = d;
    if (k == 0) {
        st.slope = slope;
        st.step = 1.0;
        st.used = nused;
        st.flag = 0;
    }
}

// Takes the accepted trial pose; st.flag = 1 when the decrease was below
// 1e-15 relative (FP64 search) or below u/4 of the terms' magnitude (FP32
// search: nothing measurable).  Called by all of warp 0.
template <bool F64>
__device__ void lbfgs_accept(SmaState &st) {
    const int k = threadIdx.x;
    const bool on = k < 6;
    const int h = st.head, used = st.used;
    const double sk = on ? st.xn[k] - st.x[k] : 0.0, yk = on ? st.gn[k] - st.g[k] : 0.0;
    const double sy = sum32(sk * yk);
    const double fprev = st.f, fn = st.fn, fnmag = st.fnmag;
    __syncwarp();
    if (on) {
        st.S[h][k] = sk;
        st.Y[h][k] = yk;
        st.x[k] = st.xn[k];
        st.g[k] = st.gn[k];
    }
    if (k == 0) {
        if (sy > 0.0) {  // keep only pairs that keep the inverse Hessian positive definite
            st.rho[h] = 1.0 / sy;
            st.head = (h + 1) % SMA_M;
            st.used = used < SMA_M ? used + 1 : SMA_M;
        }
        st.f = fn;
        st.fmag = fnmag;
        st.flag = F64 ? (fabs(fprev - fn) <= 1e-15 * (1.0 + fabs(fn))) : (fprev - fn <= 0x1p-26 * fnmag);
    }
}

template <int B>
__device__ __forceinline__ bool sma_feasible(const MixDev &mx, const SmaBox &box, const double *x) {
    int bad = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k)
            if (x[3 + k] < box.t_lo[k] || x[3 + k] > box.t_hi[k]) bad = 1;
    for (int i = threadIdx.x; i < mx.n1; i += B) {
        const double *mu = mx.mu1 + 3 * i;
        double d0 = mu[0] - x[3], d1 = mu[1] - x[4], d2 = mu[2] - x[5];
        if (d0 * d0 + d1 * d1 + d2 * d2 < box.zeta2) bad = 1;
    }
    return !__syncthreads_or(bad);
}

__device__ __forceinline__ int sma_next(int *counter, int *slot) {
    __syncthreads();
    if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
    __syncthreads();
    return *slot;
}

// Seeds over one mixture and domain.
struct SmaOne {
    MixDev mx;
    SmaBox box;
    __device__ int problem(int) const { return 0; }
    __device__ const MixDev &mix(int) const { return mx; }
    __device__ const SmaBox &dom(int) const { return box; }
};
// Seed s belongs to problem pid[s] with its own mixtures and domain.
struct SmaMany {
    const MixDev *mixes;
    const SmaBox *boxes;
    const int *pid;
    __device__ int problem(int s) const { return pid[s]; }
    __device__ const MixDev &mix(int s) const { return mixes[pid[s]]; }
    __device__ const SmaBox &dom(int s) const { return boxes[pid[s]]; }
};

// iters[s] = L-BFGS iterations taken (-1: infeasible seed, x = seed).
// Every loop is bounded: at most max_iter iterations of at most `halvings`
// trial poses each.  The dynamic shared memory holds the FP32 tables of the
// largest mixture (FP32 search); rows64 one FP64 table per block (FP64).
template <bool F64, class Src, int B>
__global__ void __launch_bounds__(B, F64 || B > SMA_BLOCK ? 1 : 8) sma_kernel(Src src, int count, const double *__restrict__ x0, int max_iter,
                                                        double *__restrict__ xout, int *__restrict__ iters,
                                                        double *__restrict__ rows64, int max_n1, int *__restrict__ counter) {
    extern __shared__ float4 sma_smem[];
    __shared__ SmaState st;
    __shared__ MixDev mx;
    __shared__ SmaBox box;
    __shared__ double fg[7];
    __shared__ int slot;
    __shared__ float red32[9][B / 32];
    __shared__ double red64[7][B / 32];
    const int tid = threadIdx.x;
    constexpr int halvings = F64 ? 40 : 20;
    Sma32Tab tb;
    double *rows = F64 ? rows64 + (size_t)blockIdx.x * max_n1 * OBJ_STRIDE : nullptr;
    int loaded = -1;  // problem whose constant tables are in shared memory
    // f and gradient at st.x (trial = false) or st.xn (trial = true)
    auto eval = [&](bool trial) {
        double mag = 0.0;
        const double *xs = trial ? st.xn : st.x;
        if (F64) sma_eval64<B>(mx, rows, st.R, xs, fg, &mag, red64);
        else sma_eval32<B>(mx, tb, xs, fg, &mag, red32);
        if (tid == 0) {
            if (trial) {
                st.fn = fg[0];
                st.fnmag = mag;
                for (int k = 0; k < 6; ++k) st.gn[k] = fg[1 + k];
            } else {
                st.f = fg[0];
                st.fmag = mag;
                for (int k = 0; k < 6; ++k) st.g[k] = fg[1 + k];
            }
        }
        __syncthreads();
    };
    for (int s = sma_next(counter, &slot); s < count; s = sma_next(counter, &slot)) {
        const int prob = src.problem(s);
        if (prob != loaded) {  // uniform: every thread read the same slot
            if (tid == 0) {
                mx = src.mix(s);
                box = src.dom(s);
            }
            __syncthreads();
            if (!F64) {
                tb = sma32_carve(sma_smem, mx.n1, mx.n2);
                for (int i = tid; i < mx.n1; i += B) tb.phi1[i] = mx.phi1f[i];
                for (int j = tid; j < mx.n2; j += B)
                    tb.jb[j] = make_float2(phiz32((float)mx.kappa2d[j]), (float)mx.phi2d[j]);
            }
            loaded = prob;
        }
        if (tid < 6) st.x[tid] = x0[6 * s + tid];
        if (tid == 0) st.head = st.used = 0;
        __syncthreads();
        if (!sma_feasible<B>(mx, box, st.x)) {
            if (tid < 6) xout[6 * s + tid] = st.x[tid];
            if (tid == 0) iters[s] = -1;
            continue;
        }
        eval(false);
        int it = 0;
        for (; it < max_iter; ++it) {
            __syncthreads();  // every warp has read the previous st.flag
            if (tid < 32) lbfgs_direction(st);
            __syncthreads();
            if (st.flag) break;
            bool accepted = false;
            for (int ls = 0; ls < halvings && !accepted; ++ls) {
                __syncthreads();
                if (tid < 6) st.xn[tid] = st.x[tid] + st.step * st.d[tid];
                __syncthreads();
                if (sma_feasible<B>(mx, box, st.xn)) {
                    eval(true);
                    if (tid == 0) st.flag = st.fn <= st.f + 1e-4 * st.step * st.slope;  // Armijo
                    __syncthreads();
                    accepted = st.flag != 0;
                }
                if (tid == 0 && !accepted) st.step *= 0.5;
            }
            if (!accepted) break;
            __syncthreads();
            if (tid < 32) lbfgs_accept<F64>(st);
            __syncthreads();
            if (st.flag) {
                ++it;
                break;
            }
        }
        if (tid < 6) xout[6 * s + tid] = st.x[tid];
        if (tid == 0) iters[s] = it;
    }
}

// ---------------------------------------------------------------- FP64 f of the results
// f alone, FP64, over the per-pose rows of obj_prep: self pairs i <= j (twice
// off the diagonal) and cross pairs; part[p * nblk + b] is block b's sum.
__global__ void logz_table(MixDev mx, double *__restrict__ lz2) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < mx.n2) lz2[j] = logZ_d(mx.kappa2d[j]);
}

__global__ void __launch_bounds__(OBJ_BLOCK) objf_pairs(MixDev mx, const double *__restrict__ idata,
                                                        const double *__restrict__ lz2, double *__restrict__ part,
                                                        int nblk) {
    const int p = blockIdx.y, n1 = mx.n1, n2 = mx.n2;
    __shared__ double red[OBJ_BLOCK / 32];
    const long long nself = (long long)n1 * n1, total = nself + (long long)n1 * n2;
    const double *I = idata + (size_t)p * n1 * OBJ_STRIDE;
    double acc = 0.0;
    const long long q0 = (long long)blockIdx.x * OBJ_CHUNK, q1 = q0 + OBJ_CHUNK < total ? q0 + OBJ_CHUNK : total;
    for (long long q = q0 + threadIdx.x; q < q1; q += OBJ_BLOCK) {
        if (q < nself) {
            const int i = (int)(q / n1), j = (int)(q % n1);
            if (j < i || (mx.cls1 && mx.cls1[i] != mx.cls1[j])) continue;
            const double *A = I + (size_t)i * OBJ_STRIDE, *B = I + (size_t)j * OBJ_STRIDE;
            const double w0 = A[4] * A[0] + B[4] * B[0], w1 = A[4] * A[1] + B[4] * B[1], w2 = A[4] * A[2] + B[4] * B[2];
            const double K = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
            acc += (i == j ? 1.0 : 2.0) * mx.phi1d[i] * mx.phi1d[j] * exp(logZ_d(K) - A[5] - B[5]);
        } else {
            const long long qq = q - nself;
            const int i = (int)(qq / n2), j = (int)(qq % n2);
            if (mx.cls1 && mx.cls1[i] != mx.cls2[j]) continue;
            const double *A = I + (size_t)i * OBJ_STRIDE, *mu = mx.mu2 + 3 * j;
            const double k2 = mx.kappa2d[j];
            const double w0 = A[4] * A[7] + k2 * mu[0], w1 = A[4] * A[8] + k2 * mu[1], w2 = A[4] * A[9] + k2 * mu[2];
            const double K = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
            acc -= 2.0 * mx.phi1d[i] * mx.phi2d[j] * exp(logZ_d(K) - A[5] - lz2[j]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < OBJ_BLOCK / 32; ++w) s += red[w];
        part[(size_t)p * nblk + blockIdx.x] = s;
    }
}

// One warp per pose: f = sum of the pose's block partials, in a fixed order.
__global__ void objf_reduce(int count, const double *__restrict__ part, int nblk, double *__restrict__ fsum) {
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (p >= count) return;  // warp-uniform
    double v = 0.0;
    for (int b = lane; b < nblk; b += 32) v += part[(size_t)p * nblk + b];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) fsum[p] = v;
}

// Outputs from the FP64 records of the 2 count poses xs = [refined; seeds]:
// per seed the better of the two (the refined pose on a tie), so f never
// exceeds the seed's f; +inf and the seed for infeasible seeds.  The records
// are f alone (fsum, grad == NULL) or f and gradient (rec, 7 per pose).
__global__ void sma_outputs(int count, const int *__restrict__ iters, const double *__restrict__ xs,
                            const double *__restrict__ fsum, const double *__restrict__ rec, double *__restrict__ x,
                            double *__restrict__ f, double *__restrict__ grad) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    const bool ok = iters[s] >= 0;
    const size_t a = s, b = (size_t)count + s;  // refined, seed
    const double fa = rec ? rec[7 * a] : fsum[a], fb = rec ? rec[7 * b] : fsum[b];
    const size_t c = ok && fa <= fb ? a : b;
    for (int k = 0; k < 6; ++k) x[6 * (size_t)s + k] = xs[6 * c + k];
    f[s] = ok ? (c == a ? fa : fb) : INFINITY;
    if (grad)
        for (int k = 0; k < 6; ++k) grad[6 * (size_t)s + k] = ok ? rec[7 * c + 1 + k] : 0.0;
}

// FP64 records of count device poses: f alone into fsum (count) when rec is
// NULL, else f and gradient into rec (count x 7); in chunks that bound the
// per-pose scratch.
static int objective_records(gosma_ctx *ctx, int count, const double *d_x, double *fsum, double *rec,
                             const double *lz2, double *scratch, int chunk) {
    const int n1 = ctx->n1, n2 = ctx->n2;
    const long long total = (long long)n1 * n1 + (long long)n1 * n2;
    const int nblk = (int)((total + OBJ_CHUNK - 1) / OBJ_CHUNK);
    double *di = scratch, *dp = scratch + (size_t)OBJ_STRIDE * n1 * chunk;
    for (int p0 = 0; p0 < count; p0 += chunk) {
        const int c = count - p0 < chunk ? count - p0 : chunk;
        const double *x = d_x + 6 * (size_t)p0;
        obj_prep<<<dim3((n1 + 127) / 128, c), 128, 0, ctx->stream>>>(OneMix{ctx->mix}, x, di);
        if (rec) {
            obj_pairs<<<dim3(nblk, c), OBJ_BLOCK, 0, ctx->stream>>>(OneMix{ctx->mix}, x, di, dp, nblk);
            obj_final<<<(c + OBJ_FINAL_WARPS - 1) / OBJ_FINAL_WARPS, 32 * OBJ_FINAL_WARPS, 0, ctx->stream>>>(
                c, x, dp, nblk, rec + 7 * (size_t)p0);
            ctx->launches += 3;
        } else {
            objf_pairs<<<dim3(nblk, c), OBJ_BLOCK, 0, ctx->stream>>>(ctx->mix, di, lz2, dp, nblk);
            objf_reduce<<<(c + 3) / 4, 128, 0, ctx->stream>>>(c, dp, nblk, fsum + p0);
            ctx->launches += 3;
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GOSMA_OK : cuda_fail(ctx, e, "launch(objective records)");
}

// Dynamic shared memory and persistent grid of the SMA kernel.  Errors are
// recorded on ectx (NULL: not recorded, for calls from a worker thread).
template <bool F64, class Src, int B>
static int sma_config(gosma_ctx *ctx, gosma_ctx *ectx, int max_n1, int max_n2, int count, int *grid, size_t *smem) {
    *smem = F64 ? 0 : sma32_smem_bytes(max_n1, max_n2);
    auto kern = sma_kernel<F64, Src, B>;
    if (*smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ectx, GOSMA_EINVAL, "sma: mixtures too large for one block's shared memory");
        }
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, B, *smem);
    if (e != cudaSuccess) return cuda_fail(ectx, e, "occupancy(sma)");
    if (per_sm < 1) return fail(ectx, GOSMA_EINVAL, "sma: mixtures too large for one block's shared memory");
    long long g = (long long)ctx->sm_count * per_sm;
    *grid = (int)(g < count ? g : count);
    return GOSMA_OK;
}

template <bool F64, class Src, int B>
static int sma_run(gosma_ctx *ectx, cudaStream_t st, const Src &src, int grid, size_t smem, int count,
                   const double *d_x0, int max_iter, double *d_x, int *d_it, double *d_rows, int max_n1,
                   int *d_counter, long long *launches) {
    cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(ectx, e, "memset(sma counter)");
    sma_kernel<F64, Src, B><<<grid, B, smem, st>>>(src, count, d_x0, max_iter, d_x, d_it, d_rows, max_n1,
                                                        d_counter);
    ++*launches;
    e = cudaGetLastError();
    return e == cudaSuccess ? GOSMA_OK : cuda_fail(ectx, e, "launch(sma)");
}

// sma_config / sma_run for the block size b chosen at run time.
template <bool F64, class Src>
static int sma_plan(gosma_ctx *ctx, gosma_ctx *ectx, int b, int max_n1, int max_n2, int count, int *grid,
                    size_t *smem) {
    switch (b) {
    case 128: return sma_config<F64, Src, 128>(ctx, ectx, max_n1, max_n2, count, grid, smem);
    case 256: return sma_config<F64, Src, 256>(ctx, ectx, max_n1, max_n2, count, grid, smem);
    case 512: return sma_config<F64, Src, 512>(ctx, ectx, max_n1, max_n2, count, grid, smem);
    default: return sma_config<F64, Src, (F64 ? 512 : 1024)>(ctx, ectx, max_n1, max_n2, count, grid, smem);
    }
}
template <bool F64, class Src>
static int sma_go(gosma_ctx *ectx, int b, cudaStream_t st, const Src &src, int grid, size_t smem, int count,
                  const double *d_x0, int max_iter, double *d_x, int *d_it, double *d_rows, int max_n1,
                  int *d_counter, long long *launches) {
    switch (b) {
    case 128:
        return sma_run<F64, Src, 128>(ectx, st, src, grid, smem, count, d_x0, max_iter, d_x, d_it, d_rows, max_n1,
                                      d_counter, launches);
    case 256:
        return sma_run<F64, Src, 256>(ectx, st, src, grid, smem, count, d_x0, max_iter, d_x, d_it, d_rows, max_n1,
                                      d_counter, launches);
    case 512:
        return sma_run<F64, Src, 512>(ectx, st, src, grid, smem, count, d_x0, max_iter, d_x, d_it, d_rows, max_n1,
                                      d_counter, launches);
    default:
        return sma_run<F64, Src, (F64 ? 512 : 1024)>(ectx, st, src, grid, smem, count, d_x0, max_iter, d_x, d_it,
                                                     d_rows, max_n1, d_counter, launches);
    }
}

// FP32-search SMA of count seeds, seed s on problem d_pid[s] (the batched
// solver's refinement, run from its worker thread: errors are returned, not
// recorded on the context); asynchronous on st.
int sma_refine_many(gosma_ctx *ctx, cudaStream_t st, const MixDev *d_mixes, const SmaBox *d_boxes, const int *d_pid,
                    int max_n1, int max_n2, int count, const double *d_x0, int max_iter, double *d_x, int *d_it,
                    int *d_counter, long long *launches) {
    if (count <= 0) return GOSMA_OK;
    int grid = 0;
    size_t smem = 0;
    const SmaMany src{d_mixes, d_boxes, d_pid};
    const int b = sma_block_for(count, ctx->sm_count, false, max_n1, max_n2);
    int rc = sma_plan<false, SmaMany>(ctx, nullptr, b, max_n1, max_n2, count, &grid, &smem);
    if (rc) return rc;
    return sma_go<false, SmaMany>(nullptr, b, st, src, grid, smem, count, d_x0, max_iter, d_x, d_it, nullptr, max_n1,
                                  d_counter, launches);
}

}  // namespace gosma

extern "C" int gosma_sma_batch(gosma_ctx *ctx, int count, const double *x0, int max_iter, int precision, double *x,
                               double *f, double *grad, int *iters, int on_device) {
    using namespace gosma;
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (!ctx->have_mix) return fail(ctx, GOSMA_ENOTREADY, "sma_batch: set mixtures first");
    if (!ctx->have_dom) return fail(ctx, GOSMA_ENOTREADY, "sma_batch: set the domain first");
    if (count < 0 || max_iter < 0) return fail(ctx, GOSMA_EINVAL, "sma_batch: count and max_iter must be >= 0");
    if (precision != 32 && precision != 64) return fail(ctx, GOSMA_EINVAL, "sma_batch: precision must be 32 or 64");
    if (count == 0) return GOSMA_OK;
    if (!x0 || !x || !f) return fail(ctx, GOSMA_EINVAL, "sma_batch: null seeds or outputs");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    const bool f64 = precision == 64;
    const int n1 = ctx->n1, n2 = ctx->n2;
    int grid = 0;
    size_t smem = 0;
    const int b = sma_block_for(count, ctx->sm_count, f64, n1, n2);
    int rc = f64 ? sma_plan<true, SmaOne>(ctx, ctx, b, n1, n2, count, &grid, &smem)
                 : sma_plan<false, SmaOne>(ctx, ctx, b, n1, n2, count, &grid, &smem);
    if (rc) return rc;

    // device scratch: seeds and poses (host calls), iterations, counter,
    // FP64 rows (one table per block), objective records (f alone when no
    // gradient is asked for), log Z(kappa_2) and the records' scratch
    const long long total = (long long)n1 * n1 + (long long)n1 * n2;
    const int nblk = (int)((total + OBJ_CHUNK - 1) / OBJ_CHUNK);
    const size_t per_pose = sizeof(double) * ((size_t)OBJ_STRIDE * n1 + 7 * (size_t)nblk);
    int chunk = (int)((64u << 20) / per_pose);
    if (chunk < 1) chunk = 1;
    if (chunk > 2 * count) chunk = 2 * count;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_x0 = on_device ? 0 : al(sizeof(double) * 6 * (size_t)count);
    const size_t b_x = on_device ? 0 : al(sizeof(double) * 6 * (size_t)count);
    const size_t b_f = on_device ? 0 : al(sizeof(double) * (size_t)count);
    const size_t b_g = on_device || !grad ? 0 : al(sizeof(double) * 6 * (size_t)count);
    const size_t b_xs = al(sizeof(double) * 12 * (size_t)count);
    const size_t b_it = al(sizeof(int) * (size_t)count) + 256;
    const size_t b_rows = f64 ? al(sizeof(double) * OBJ_STRIDE * (size_t)n1 * grid) : 0;
    const size_t b_rec = grad ? al(sizeof(double) * 14 * (size_t)count) : 0;
    const size_t b_part = grad ? 0 : al(sizeof(double) * 2 * (size_t)count);
    const size_t b_lz = al(sizeof(double) * (size_t)n2);
    const size_t b_scr = al(per_pose * (size_t)chunk);
    const size_t need = b_x0 + b_x + b_f + b_g + b_xs + b_it + b_rows + b_rec + b_part + b_lz + b_scr;
    if (need > ctx->sma_bytes) {
        if (ctx->d_sma) cudaFree(ctx->d_sma);
        ctx->d_sma = nullptr;
        ctx->sma_bytes = 0;
        e = dev_malloc(ctx, &ctx->d_sma, need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(sma)");
        ctx->sma_bytes = need;
    }
    char *p = (char *)ctx->d_sma;
    double *d_x0 = on_device ? (double *)x0 : (double *)p;
    p += b_x0;
    double *d_x = on_device ? x : (double *)p;
    p += b_x;
    double *d_f = on_device ? f : (double *)p;
    p += b_f;
    double *d_g = on_device ? grad : (grad ? (double *)p : nullptr);
    p += b_g;
    double *d_xs = (double *)p;  // refined poses, then the seeds
    p += b_xs;
    int *d_it = (int *)p;
    int *d_counter = (int *)(p + al(sizeof(int) * (size_t)count));
    p += b_it;
    double *d_rows = (double *)p;
    p += b_rows;
    double *d_rec = grad ? (double *)p : nullptr;
    p += b_rec;
    double *d_fsum = grad ? nullptr : (double *)p;
    p += b_part;
    double *d_lz = (double *)p;
    p += b_lz;
    double *d_scr = (double *)p;

    cudaStream_t st = ctx->stream;
    if (!on_device) {
        e = cudaMemcpyAsync(d_x0, x0, sizeof(double) * 6 * (size_t)count, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy seeds");
    }
    SmaOne one;
    one.mx = ctx->mix;
    for (int k = 0; k < 3; ++k) {
        one.box.t_lo[k] = ctx->t_lo[k];
        one.box.t_hi[k] = ctx->t_hi[k];
    }
    one.box.zeta2 = ctx->zeta * ctx->zeta;
    e = cudaMemcpyAsync(d_xs + 6 * (size_t)count, d_x0, sizeof(double) * 6 * (size_t)count, cudaMemcpyDeviceToDevice,
                        st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy seeds");
    long long *nl = &ctx->launches;
    rc = f64 ? sma_go<true, SmaOne>(ctx, b, st, one, grid, smem, count, d_x0, max_iter, d_xs, d_it, d_rows, n1,
                                    d_counter, nl)
             : sma_go<false, SmaOne>(ctx, b, st, one, grid, smem, count, d_x0, max_iter, d_xs, d_it, d_rows, n1,
                                     d_counter, nl);
    if (rc) return rc;
    if (!grad) {
        logz_table<<<(n2 + 127) / 128, 128, 0, st>>>(ctx->mix, d_lz);
        ++ctx->launches;
    }
    rc = objective_records(ctx, 2 * count, d_xs, d_fsum, d_rec, d_lz, d_scr, chunk);
    if (rc) return rc;
    sma_outputs<<<(count + 127) / 128, 128, 0, st>>>(count, d_it, d_xs, d_fsum, d_rec, d_x, d_f, d_g);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch(sma outputs)");
    if (on_device) {
        if (iters) {
            e = cudaMemcpyAsync(iters, d_it, sizeof(int) * (size_t)count, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "copy iterations");
        }
        return GOSMA_OK;
    }
    e = cudaMemcpyAsync(x, d_x, sizeof(double) * 6 * (size_t)count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d_f, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && grad)
        e = cudaMemcpyAsync(grad, d_g, sizeof(double) * 6 * (size_t)count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && iters)
        e = cudaMemcpyAsync(iters, d_it, sizeof(int) * (size_t)count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sma_batch results");
    return GOSMA_OK;
}
