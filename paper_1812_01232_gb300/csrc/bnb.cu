// placeholder, replaced below
#include "gosma_internal.cuh"
namespace gosma {
void bnb_release(gosma_ctx *ctx) { (void)ctx; }
}
extern "C" int gosma_bnb_solve(gosma_ctx *ctx, const gosma_opts *opts, gosma_result *out) {
    (void)opts; (void)out;
    return gosma::fail(ctx, GOSMA_ENOTREADY, "not built");
}
