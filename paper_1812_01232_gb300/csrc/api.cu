// C ABI entry points of libgosma (declared in include/gosma.h): context,
// mixtures, domain, bounds and objective.  Branch-and-bound is in bnb.cu.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <new>

#include "classes.h"
#include "gosma_internal.cuh"
#include "host_rules.h"

namespace gosma {

int fail(gosma_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(gosma_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, GOSMA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int ensure_stage(gosma_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->stage_bytes) return GOSMA_OK;
    if (ctx->d_stage) cudaFree(ctx->d_stage);
    ctx->d_stage = nullptr;
    ctx->stage_bytes = 0;
    cudaError_t e = dev_malloc(ctx, &ctx->d_stage, bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(stage)");
    ctx->stage_bytes = bytes;
    return GOSMA_OK;
}

int ensure_pinned(gosma_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->pinned_bytes) return GOSMA_OK;
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    ctx->h_pinned = nullptr;
    ctx->pinned_bytes = 0;
    cudaError_t e = cudaMallocHost(&ctx->h_pinned, bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMallocHost(stage)");
    ctx->pinned_bytes = bytes;
    return GOSMA_OK;
}

int setup_constants(gosma_ctx *ctx, double *c22_out);
int selftest_approx(gosma_ctx *ctx, double measured[5], double assumed[5]);
int selftest_wait_timeout(gosma_ctx *ctx, double limit_s, int *timed_out);

// (lb, ub) pairs of n records, for the host path: 16 bytes per cube cross the bus.
__global__ void pack_bounds(const gosma_bound *__restrict__ in, int n, double2 *__restrict__ out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = make_double2(in[k].lb, in[k].ub);
}

__global__ void copy_records(const gosma_bound *__restrict__ in, int n, gosma_bound *__restrict__ out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = in[k];
}

__global__ void split_bounds(const gosma_bound *__restrict__ in, int n, double *lb, double *ub) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        if (lb) lb[k] = in[k].lb;
        if (ub) ub[k] = in[k].ub;
    }
}

}  // namespace gosma

using namespace gosma;

extern "C" {

int gosma_create(int device, void *stream, gosma_ctx **out) {
    if (!out) return GOSMA_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return GOSMA_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return GOSMA_ECUDA;
    if (prop.major != 10 || prop.minor != 3) return GOSMA_ECUDA;  // built for sm_103a only
    if (cudaSetDevice(device) != cudaSuccess) return GOSMA_ECUDA;
    gosma_ctx *c = new (std::nothrow) gosma_ctx();
    if (!c) return GOSMA_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    c->sm_count = prop.multiProcessorCount;
    int pageable = 0, host_tables = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device) != cudaSuccess) pageable = 0;
    if (cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, device) != cudaSuccess)
        host_tables = 0;
    const char *staged = getenv("GOSMA_STAGED_HOST_IO");  // force the staged path (tests of both paths)
    c->direct_host = pageable && host_tables && !(staged && staged[0] == '1');
    *out = c;
    return GOSMA_OK;
}

void gosma_destroy(gosma_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    bnb_release(ctx);
    gosma::mlp_free(ctx->mlp);
    if (ctx->d_mix) cudaFree(ctx->d_mix);
    if (ctx->d_stage) cudaFree(ctx->d_stage);
    if (ctx->d_obj) cudaFree(ctx->d_obj);
    if (ctx->d_sma) cudaFree(ctx->d_sma);
    if (ctx->d_mg) cudaFree(ctx->d_mg);
    if (ctx->d_rot) cudaFree(ctx->d_rot);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    delete ctx;
}

const char *gosma_last_error(const gosma_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

long long gosma_kernel_launches(const gosma_ctx *ctx) { return ctx ? ctx->launches : 0; }

// Shared by the single-class and the semantic entry points: nclass classes
// of n1c[l] model and n2c[l] image components (given class by class), class
// weights w (w = NULL: one class of weight 1).  Each class's mixture weights
// sum to 1; they are scaled by sqrt(w_l) so that the within-class pair sums
// give sum_l w_l f_l (Sec. 4.2).
static int set_mixtures_impl(gosma_ctx *ctx, int nclass, const int *n1c, const int *n2c, const double *w, int n1,
                             const double *mu1, const double *sigma1, const double *phi1_in, int n2,
                             const double *mu2, const double *kappa2, const double *phi2_in) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (n1 < 1 || n2 < 1 || !mu1 || !sigma1 || !phi1_in || !mu2 || !kappa2 || !phi2_in)
        return fail(ctx, GOSMA_EINVAL, "set_mixtures: empty mixture or null pointer");
    if (bounds_smem_bytes(n1, n2) > 200 * 1024)
        return fail(ctx, GOSMA_EINVAL, "set_mixtures: 13*n1 + 8*n2 floats exceed the 200 KB shared-memory budget");
    for (int i = 0; i < n1; ++i)
        if (!(sigma1[i] > 0) || !(phi1_in[i] >= 0) || !isfinite(mu1[3 * i]) || !isfinite(mu1[3 * i + 1]) ||
            !isfinite(mu1[3 * i + 2]) || !isfinite(sigma1[i]))
            return fail(ctx, GOSMA_EINVAL, "set_mixtures: sigma1 must be > 0, phi1 >= 0, means finite");
    for (int j = 0; j < n2; ++j) {
        double nn = sqrt(mu2[3 * j] * mu2[3 * j] + mu2[3 * j + 1] * mu2[3 * j + 1] + mu2[3 * j + 2] * mu2[3 * j + 2]);
        if (!(kappa2[j] > 0) || !isfinite(kappa2[j]) || !(phi2_in[j] >= 0) || !(fabs(nn - 1.0) <= 1e-6))
            return fail(ctx, GOSMA_EINVAL, "set_mixtures: kappa2 must be > 0, phi2 >= 0, |mu2_j| = 1");
    }
    // classes: per-class weight sums, class ids, pair ranges; weights scaled by sqrt(w_l)
    ClassLayout CL;
    if (const char *msg = class_layout(nclass, n1c, n2c, w, n1, n2, phi1_in, phi2_in, CL)) {
        std::string m = std::string("set_mixtures: ") + msg;
        return fail(ctx, GOSMA_EINVAL, m.c_str());
    }
    const std::vector<double> &phi1 = CL.phi1, &phi2 = CL.phi2;
    const std::vector<int> &cls1 = CL.cls1, &cls2 = CL.cls2, &rj0 = CL.rj0, &rj1 = CL.rj1, &rm1 = CL.rm1;
    const bool classes = CL.classes;
    cudaSetDevice(ctx->device);
    size_t nd = 3 * (size_t)n1 + 2 * n1 + 3 * (size_t)n2 + 2 * n2;
    size_t nf = 8 * (size_t)n1 + 10 * (size_t)n2;
    const size_t ni = classes ? 5 * (size_t)n1 + (size_t)n2 : 0;  // class ids and pair ranges
    size_t bytes = nd * sizeof(double) + nf * sizeof(float) + ni * sizeof(int) + 256;
    void *d = nullptr;
    cudaError_t e = dev_malloc(ctx, &d, bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(mixtures)");
    double *pd = (double *)d;
    double *dmu1 = pd, *dsig = pd + 3 * n1, *dphi1 = dsig + n1, *dmu2 = dphi1 + n1, *dk2 = dmu2 + 3 * n2,
           *dphi2 = dk2 + n2;
    float *pf = (float *)(dphi2 + n2);
    float *inv_sig2 = pf, *phi1f = pf + n1, *k2f = phi1f + n1, *Q2 = k2f + n2;
    float *mu1h = Q2 + n2, *mu1l = mu1h + 3 * n1, *mu2h = mu1l + 3 * n1, *mu2l = mu2h + 3 * n2;
    float *lQ2c = mu2l + 3 * n2, *lQ2b = lQ2c + n2;
    int *pi = (int *)(lQ2b + n2);
    int *dcls1 = pi, *drj0 = pi + n1, *drj1 = pi + 2 * n1, *drm1 = pi + 3 * n1, *dcls2 = pi + 4 * n1;
    std::vector<float> hk2(n2);
    for (int j = 0; j < n2; ++j) hk2[j] = (float)kappa2[j];
    // image mean directions are used as exact unit vectors: normalise them (FP64)
    std::vector<double> mu2n(mu2, mu2 + 3 * (size_t)n2);
    for (int j = 0; j < n2; ++j) {
        double *m = &mu2n[3 * (size_t)j];
        double nn = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        for (int k = 0; k < 3; ++k) m[k] /= nn;
    }
    struct {
        void *dst;
        const void *src;
        size_t n;
    } cp[] = {{dmu1, mu1, 3 * (size_t)n1 * 8}, {dsig, sigma1, (size_t)n1 * 8}, {dphi1, phi1.data(), (size_t)n1 * 8},
              {dmu2, mu2n.data(), 3 * (size_t)n2 * 8}, {dk2, kappa2, (size_t)n2 * 8},  {dphi2, phi2.data(), (size_t)n2 * 8},
              {k2f, hk2.data(), (size_t)n2 * 4},
              {dcls1, cls1.data(), classes ? (size_t)n1 * 4 : 0}, {drj0, rj0.data(), classes ? (size_t)n1 * 4 : 0},
              {drj1, rj1.data(), classes ? (size_t)n1 * 4 : 0}, {drm1, rm1.data(), classes ? (size_t)n1 * 4 : 0},
              {dcls2, cls2.data(), classes ? (size_t)n2 * 4 : 0}};
    for (auto &c : cp) {
        if (!c.n) continue;
        e = cudaMemcpyAsync(c.dst, c.src, c.n, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) {
            cudaFree(d);
            return cuda_fail(ctx, e, "copy mixtures");
        }
    }
    MixDev mx{};
    mx.n1 = n1;
    mx.n2 = n2;
    mx.mu1 = dmu1;
    mx.inv_sig2 = inv_sig2;
    mx.phi1f = phi1f;
    mx.sigma1d = dsig;
    mx.phi1d = dphi1;
    mx.mu2 = dmu2;
    mx.kappa2 = k2f;
    mx.Q2 = Q2;
    mx.kappa2d = dk2;
    mx.phi2d = dphi2;
    mx.mu1h = mu1h;
    mx.mu1l = mu1l;
    mx.mu2h = mu2h;
    mx.mu2l = mu2l;
    mx.lQ2c = lQ2c;
    mx.lQ2b = lQ2b;
    mx.zeta = ctx->zeta;
    mx.cls1 = classes ? dcls1 : nullptr;
    mx.cls2 = classes ? dcls2 : nullptr;
    mx.rj0 = classes ? drj0 : nullptr;
    mx.rj1 = classes ? drj1 : nullptr;
    mx.rm1 = classes ? drm1 : nullptr;
    mx.psi_point = ctx->psi_r_mode;
    void *old = ctx->d_mix;
    MixDev old_mix = ctx->mix;
    int old_n1 = ctx->n1, old_n2 = ctx->n2;
    ctx->mix = mx;
    ctx->n1 = n1;
    ctx->n2 = n2;
    double c22 = 0;
    int rc = setup_constants(ctx, &c22);
    if (rc) {
        cudaFree(d);
        ctx->mix = old_mix;
        ctx->n1 = old_n1;
        ctx->n2 = old_n2;
        return rc;
    }
    if (old) cudaFree(old);
    ctx->d_mix = d;
    ctx->c22 = c22;
    ctx->h_mu1.assign(mu1, mu1 + 3 * (size_t)n1);
    ctx->h_sigma1.assign(sigma1, sigma1 + n1);
    ctx->h_phi1 = phi1;
    ctx->h_mu2 = mu2n;
    ctx->h_kappa2.assign(kappa2, kappa2 + n2);
    ctx->h_phi2 = phi2;
    ProblemHash ph;
    ph.array(ctx->h_mu1.data(), ctx->h_mu1.size());
    ph.array(ctx->h_sigma1.data(), ctx->h_sigma1.size());
    ph.array(ctx->h_phi1.data(), ctx->h_phi1.size());
    ph.array(ctx->h_mu2.data(), ctx->h_mu2.size());
    ph.array(ctx->h_kappa2.data(), ctx->h_kappa2.size());
    ph.array(ctx->h_phi2.data(), ctx->h_phi2.size());
    ph.array(cls1.data(), classes ? cls1.size() : 0);
    ph.array(cls2.data(), classes ? cls2.size() : 0);
    ctx->mix_hash = ph.h;
    ctx->have_mix = true;
    bnb_end_run(ctx);
    return GOSMA_OK;
}

int gosma_set_psi_r_mode(gosma_ctx *ctx, int mode) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (mode != GOSMA_PSI_R_CUBE && mode != GOSMA_PSI_R_POINT)
        return fail(ctx, GOSMA_EINVAL, "set_psi_r_mode: mode must be GOSMA_PSI_R_CUBE or GOSMA_PSI_R_POINT");
    ctx->psi_r_mode = mode;
    ctx->mix.psi_point = mode;
    return GOSMA_OK;
}

int gosma_set_mixtures(gosma_ctx *ctx, int n1, const double *mu1, const double *sigma1, const double *phi1, int n2,
                       const double *mu2, const double *kappa2, const double *phi2) {
    return set_mixtures_impl(ctx, 1, nullptr, nullptr, nullptr, n1, mu1, sigma1, phi1, n2, mu2, kappa2, phi2);
}

int gosma_set_mixtures_classes(gosma_ctx *ctx, int nclass, const int *n1c, const int *n2c, const double *w,
                               const double *mu1, const double *sigma1, const double *phi1, const double *mu2,
                               const double *kappa2, const double *phi2) {
    if (!ctx) return GOSMA_EINVAL;
    if (nclass < 1 || !n1c || !n2c || !w) return fail(ctx, GOSMA_EINVAL, "set_mixtures_classes: bad class arrays");
    long long n1 = 0, n2 = 0;
    for (int l = 0; l < nclass; ++l) {
        if (n1c[l] < 1 || n2c[l] < 1) return fail(ctx, GOSMA_EINVAL, "set_mixtures_classes: empty class");
        n1 += n1c[l];
        n2 += n2c[l];
    }
    if (n1 > (1 << 20) || n2 > (1 << 20)) return fail(ctx, GOSMA_EINVAL, "set_mixtures_classes: too many components");
    return set_mixtures_impl(ctx, nclass, n1c, n2c, w, (int)n1, mu1, sigma1, phi1, (int)n2, mu2, kappa2, phi2);
}

int gosma_set_domain(gosma_ctx *ctx, const double t_lo[3], const double t_hi[3], double zeta) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (!t_lo || !t_hi || !(zeta >= 0) || !isfinite(zeta)) return fail(ctx, GOSMA_EINVAL, "set_domain: bad arguments");
    for (int k = 0; k < 3; ++k)
        if (!(t_lo[k] < t_hi[k]) || !isfinite(t_lo[k]) || !isfinite(t_hi[k]))
            return fail(ctx, GOSMA_EINVAL, "set_domain: need t_lo < t_hi");
    for (int k = 0; k < 3; ++k) {
        ctx->t_lo[k] = t_lo[k];
        ctx->t_hi[k] = t_hi[k];
    }
    ctx->zeta = zeta;
    ctx->mix.zeta = zeta;
    ctx->have_dom = true;
    bnb_end_run(ctx);
    return GOSMA_OK;
}

static int eval_common(gosma_ctx *ctx, const gosma_cube *cubes, int n, gosma_bound *detail, double *lb, double *ub,
                       int on_device) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (!ctx->have_mix || !ctx->have_dom) return fail(ctx, GOSMA_ENOTREADY, "eval_bounds: set mixtures and domain first");
    if (n < 0 || (n > 0 && !cubes)) return fail(ctx, GOSMA_EINVAL, "eval_bounds: bad cube array");
    if (n == 0) return GOSMA_OK;
    cudaSetDevice(ctx->device);
    size_t bc = sizeof(gosma_cube) * (size_t)n, bo = sizeof(gosma_bound) * (size_t)n;
    cudaError_t e;
    int rc;
    if (on_device) {
        gosma_bound *dout = detail;
        if (!dout) {
            rc = ensure_stage(ctx, bo);
            if (rc) return rc;
            dout = (gosma_bound *)ctx->d_stage;
        }
        rc = launch_bounds(ctx, cubes, n, dout);
        if (rc) return rc;
        if (!detail) {
            split_bounds<<<(n + 255) / 256, 256, 0, ctx->stream>>>(dout, n, lb, ub);
            ++ctx->launches;
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(ctx, e, "launch(split)");
        }
        return GOSMA_OK;
    }
    if (ctx->direct_host) {
        // the kernels read the caller's cubes and write the caller's results in
        // place over the coherent link: no staging copies
        rc = ensure_stage(ctx, bo);
        if (rc) return rc;
        gosma_bound *drec = (gosma_bound *)ctx->d_stage;
        rc = launch_bounds(ctx, cubes, n, drec);
        if (rc) return rc;
        if (detail) copy_records<<<(n + 255) / 256, 256, 0, ctx->stream>>>(drec, n, detail);
        else split_bounds<<<(n + 255) / 256, 256, 0, ctx->stream>>>(drec, n, lb, ub);
        ++ctx->launches;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "bounds (host buffers)");
        return GOSMA_OK;
    }
    // Host buffers: pipelined over chunks, so that staging the next chunk on
    // the host, the copies and the kernels of the current chunk and the
    // unpacking of finished chunks overlap; only the requested results cross
    // the bus (lb and ub: 16 bytes per cube, or the full records).
    const int CH = 16384;
    const int nch = (n + CH - 1) / CH;
    const size_t out_per = detail ? sizeof(gosma_bound) : sizeof(double2);
    rc = ensure_stage(ctx, bc + bo + sizeof(double2) * (size_t)n);
    if (rc) return rc;
    rc = ensure_pinned(ctx, bc + out_per * (size_t)n);
    if (rc) return rc;
    gosma_cube *dc = (gosma_cube *)ctx->d_stage;
    gosma_bound *drec = (gosma_bound *)((char *)ctx->d_stage + bc);
    double2 *dlu = (double2 *)((char *)drec + bo);
    unsigned char *hin = (unsigned char *)ctx->h_pinned, *hout = hin + bc;
    std::vector<cudaEvent_t> ev(nch, nullptr);
    struct EventsFree {
        std::vector<cudaEvent_t> &v;
        ~EventsFree() {
            for (cudaEvent_t x : v)
                if (x) cudaEventDestroy(x);
        }
    } ev_guard{ev};
    for (int c = 0; c < nch; ++c) {
        const int off = c * CH, m = n - off < CH ? n - off : CH;
        e = cudaEventCreateWithFlags(&ev[c], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventCreate");
        memcpy(hin + sizeof(gosma_cube) * (size_t)off, cubes + off, sizeof(gosma_cube) * (size_t)m);
        e = cudaMemcpyAsync(dc + off, hin + sizeof(gosma_cube) * (size_t)off, sizeof(gosma_cube) * (size_t)m,
                            cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy cubes");
        rc = launch_bounds(ctx, dc + off, m, drec + off);
        if (rc) return rc;
        const void *src = drec + off;
        if (!detail) {
            pack_bounds<<<(m + 255) / 256, 256, 0, ctx->stream>>>(drec + off, m, dlu + off);
            ++ctx->launches;
            src = dlu + off;
        }
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hout + out_per * (size_t)off, src, out_per * (size_t)m, cudaMemcpyDeviceToHost,
                                ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[c], ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy bounds");
    }
    for (int c = 0; c < nch; ++c) {
        const int off = c * CH, m = n - off < CH ? n - off : CH;
        e = cudaEventSynchronize(ev[c]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "sync(bounds)");
        if (detail) {
            memcpy(detail + off, hout + out_per * (size_t)off, out_per * (size_t)m);
        } else {
            const double2 *h = (const double2 *)hout + off;
            for (int k = 0; k < m; ++k) {
                if (lb) lb[off + k] = h[k].x;
                if (ub) ub[off + k] = h[k].y;
            }
        }
    }
    return GOSMA_OK;
}

int gosma_eval_bounds(gosma_ctx *ctx, const gosma_cube *cubes, int n, double *lb, double *ub, int on_device) {
    return eval_common(ctx, cubes, n, nullptr, lb, ub, on_device);
}

int gosma_eval_bounds_detail(gosma_ctx *ctx, const gosma_cube *cubes, int n, gosma_bound *out, int on_device) {
    if (!out && n > 0) return fail(ctx, GOSMA_EINVAL, "eval_bounds_detail: null output");
    return eval_common(ctx, cubes, n, out, nullptr, nullptr, on_device);
}

int gosma_eval_objective_grad(gosma_ctx *ctx, int count, const double *x, double *f, double *grad) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (!ctx->have_mix) return fail(ctx, GOSMA_ENOTREADY, "eval_objective: set mixtures first");
    if (count < 0 || (count > 0 && !x)) return fail(ctx, GOSMA_EINVAL, "eval_objective: bad poses");
    cudaSetDevice(ctx->device);
    return objective_grad_device(ctx, count, x, f, grad);
}

int gosma_eval_objective(gosma_ctx *ctx, const double r[3], const double t[3], double *f) {
    if (!r || !t || !f) return fail(ctx, GOSMA_EINVAL, "eval_objective: null pointer");
    double x[6] = {r[0], r[1], r[2], t[0], t[1], t[2]};
    return gosma_eval_objective_grad(ctx, 1, x, f, nullptr);
}

int gosma_selftest_wait_timeout(gosma_ctx *ctx, double limit_seconds) {
    if (!ctx) return GOSMA_EINVAL;
    ctx->err.clear();
    if (!(limit_seconds > 0) || limit_seconds > 10) return fail(ctx, GOSMA_EINVAL, "selftest_wait_timeout: 0 < limit <= 10 s");
    cudaSetDevice(ctx->device);
    int timed_out = 0;
    int rc = selftest_wait_timeout(ctx, limit_seconds, &timed_out);
    if (rc) return rc;
    return timed_out ? fail(ctx, GOSMA_ETIMEOUT, "selftest_wait_timeout: the wait gave up (as designed)") : GOSMA_OK;
}

int gosma_debug_fail_allocations(gosma_ctx *ctx, int n) {
    if (!ctx) return GOSMA_EINVAL;
    if (n < 0) return fail(ctx, GOSMA_EINVAL, "debug_fail_allocations: n >= 0");
    ctx->fail_allocs = n;
    return GOSMA_OK;
}

int gosma_selftest_approx(gosma_ctx *ctx, double measured[5], double assumed[5]) {
    if (!ctx || !measured || !assumed) return GOSMA_EINVAL;
    cudaSetDevice(ctx->device);
    return selftest_approx(ctx, measured, assumed);
}

}  // extern "C"
