// Continuous-batching request loop (filled in below).
#include "../../include/pme.h"
#include "plan_internal.h"

using namespace pme;

extern "C" {
pme_status pme_server_create(size_t, int, pme_server **out) {
    if (out) *out = nullptr;
    return fail(PME_EUNSUPPORTED, "server not built yet");
}
pme_status pme_submit(pme_server *, pme_plan *, const float *, const float *, int64_t, float *, double *, double *,
                      pme_ticket *) {
    return fail(PME_EUNSUPPORTED, "server not built yet");
}
pme_status pme_poll(pme_server *, pme_ticket, int) { return fail(PME_EUNSUPPORTED, "server not built yet"); }
pme_status pme_server_stats(pme_server *, int64_t *, double *, double *, int64_t *) {
    return fail(PME_EUNSUPPORTED, "server not built yet");
}
void pme_server_destroy(pme_server *) {}
}
