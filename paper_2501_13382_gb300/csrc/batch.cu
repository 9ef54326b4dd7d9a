// batch.cu -- persistent batched summation (placeholder until implemented).
#include "gbt_internal.h"

extern "C" {
gbt_status gbt_batch_create(const gbt_batch_desc *, void *, gbt_batch_t **out)
{
    if (out) *out = nullptr;
    return GBT_ERR_UNSUPPORTED;
}
gbt_status gbt_batch_submit(gbt_batch_t *, void *) { return GBT_ERR_UNSUPPORTED; }
gbt_status gbt_batch_destroy(gbt_batch_t *) { return GBT_OK; }
}
