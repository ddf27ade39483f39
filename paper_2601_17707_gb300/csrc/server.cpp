// server.cpp -- placeholder entry points of the serving loop (replaced by the real loop).
#include "graph.cuh"

using namespace bbc;

extern "C" {
bbc_status bbc_server_create(size_t, const bbc_tuning *, bbc_server **) {
    set_error("serving loop not available in this build");
    return BBC_E_INVALID_ARG;
}
bbc_status bbc_submit(bbc_server *, int32_t, int32_t, int64_t, const int32_t *, const int32_t *,
                      const int8_t *, uint64_t *) { return BBC_E_INVALID_ARG; }
bbc_status bbc_poll(bbc_server *, uint64_t, uint64_t *) { return BBC_E_INVALID_ARG; }
bbc_status bbc_wait(bbc_server *, uint64_t, int64_t, uint64_t *) { return BBC_E_INVALID_ARG; }
bbc_status bbc_server_stats(bbc_server *, uint64_t *, double *, double *, double *) {
    return BBC_E_INVALID_ARG;
}
void bbc_server_destroy(bbc_server *) {}
}
