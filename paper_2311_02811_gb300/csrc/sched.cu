// Schedule resolution for CC_ORDER_AUTO.
#include <vector>

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

cc_status batch_resolve_schedule(cc_batch_plan* b, int mode, int c) {
    (void)mode;
    const int32_t G = batch_graph_count(b);
    std::vector<int32_t> h(G, 2), sync(G, 1), cc_(G, c < 1 ? 1 : c);
    batch_set_schedule(b, h.data(), sync.data(), cc_.data());
    return CC_OK;
}

}  // namespace cc
