// Ragged batches: placeholder entry points (replaced by the persistent batcher).
#include "sph_internal.h"

using namespace sph;

extern "C" {
int sphericart_batch_plan_create(const sph_batch_set*, int, const sph_launch*, sph_batch_plan** plan) {
    if (plan) *plan = nullptr;
    set_error("batched plans are not available in this build");
    return SPH_EUNSUPPORTED;
}
int sphericart_batch_execute(const sph_batch_plan*, void*) {
    set_error("batched plans are not available in this build");
    return SPH_EUNSUPPORTED;
}
int sphericart_batch_plan_destroy(sph_batch_plan*) { return SPH_OK; }
int sphericart_batch_plan_info(const sph_batch_plan*, int64_t*, int64_t*) {
    set_error("batched plans are not available in this build");
    return SPH_EUNSUPPORTED;
}
}
