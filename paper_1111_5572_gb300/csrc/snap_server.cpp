// snap_server.cpp — serving loop (placeholder until the server lands).
#include "snap_internal.h"

using namespace snapgpu;

extern "C" int snap_server_create(const snap_index*, uint64_t, int, snap_server** out) {
    if (out) *out = nullptr;
    set_error("snap_server_create: not available in this build");
    return SNAP_E_INTERNAL;
}
extern "C" int snap_server_submit(snap_server*, const uint8_t*, const uint64_t*, uint64_t,
                                  const snap_params*, uint64_t*) {
    set_error("snap_server_submit: not available in this build");
    return SNAP_E_INTERNAL;
}
extern "C" int snap_server_wait(snap_server*, uint64_t, snap_result*, double*) {
    set_error("snap_server_wait: not available in this build");
    return SNAP_E_INTERNAL;
}
extern "C" int snap_server_destroy(snap_server*) { return SNAP_OK; }
