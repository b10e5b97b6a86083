// Request server (continuous batching).  Placeholder until the batched
// scheduler lands: every call reports that serving is unavailable.
#include "ellsolve.h"
#include "solver.hpp"

using namespace ells;

extern "C" {

ellsolve_status ellsolve_server_create(size_t, int, void *, ellsolve_server_t *out) {
    if (out) *out = nullptr;
    set_last_error("server not available in this build");
    return ELLSOLVE_ERR_ARG;
}

ellsolve_status ellsolve_submit(ellsolve_server_t, const ellsolve_grid *, double, double,
                                const double *, const void *, void *, double, int, uint64_t *) {
    set_last_error("server not available in this build");
    return ELLSOLVE_ERR_ARG;
}

ellsolve_status ellsolve_poll(ellsolve_server_t, uint64_t, int, ellsolve_result *) {
    set_last_error("server not available in this build");
    return ELLSOLVE_ERR_ARG;
}

void ellsolve_server_destroy(ellsolve_server_t) {}

}  // extern "C"
