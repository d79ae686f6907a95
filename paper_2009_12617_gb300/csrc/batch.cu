// Batched evaluation of many systems in one persistent launch (filled in below).
#include "../../include/pme.h"
#include "plan_internal.h"

using namespace pme;

extern "C" {
pme_status pme_batch_create(int, pme_plan *const *, const int64_t *, void *, pme_batch **out) {
    if (out) *out = nullptr;
    return fail(PME_EUNSUPPORTED, "batched evaluation not built yet");
}
pme_status pme_batch_enqueue(pme_batch *, const float *, const float *, float *, double *) {
    return fail(PME_EUNSUPPORTED, "batched evaluation not built yet");
}
pme_status pme_batch_sync(pme_batch *) { return fail(PME_EUNSUPPORTED, "batched evaluation not built yet"); }
void pme_batch_destroy(pme_batch *) {}
pme_status pme_batch_debug_stall(pme_batch *, int, int64_t) {
    return fail(PME_EUNSUPPORTED, "batched evaluation not built yet");
}
}
