// Schedule resolution for CC_ORDER_AUTO.
#include "cc_internal.h"

namespace cc {

cc_status resolve_schedule(cc_graph* g, int* order, int* mode, int* c) {
    (void)g;
    // plain order-2 synchronous schedule, checked every sweep
    *order = 2;
    *mode = CC_SYNC;
    if (*c < 1) *c = 1;
    return CC_OK;
}

}  // namespace cc
