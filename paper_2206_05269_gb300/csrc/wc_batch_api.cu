// Batched counting entry points (filled in with the batched kernels).
#include "../../include/wc.h"
#include "wc_host.h"

wc_status wc_count_batched(wc_ctx *ctx, const uint8_t *, const uint64_t *, const uint64_t *, uint32_t,
                           const uint32_t *, uint32_t, cudaStream_t, wc_batch **out) {
    if (out) *out = nullptr;
    return ctx ? ctx->fail(WC_ERR_UNSUPPORTED, "batched counting not built yet") : WC_ERR_INVALID_ARG;
}
wc_status wc_batch_table(const wc_batch *, int, uint32_t, const wc_table **out) {
    if (out) *out = nullptr;
    return WC_ERR_UNSUPPORTED;
}
wc_status wc_class_ratio_topk(wc_ctx *, const wc_batch *, uint32_t, uint32_t, cudaStream_t, uint64_t *,
                              uint64_t *, uint64_t *, uint32_t *nout) {
    if (nout) *nout = 0;
    return WC_ERR_UNSUPPORTED;
}
void wc_batch_free(wc_batch *) {}
