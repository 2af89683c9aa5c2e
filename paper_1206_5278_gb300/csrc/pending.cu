// Entry points whose kernels are not in this build yet: they fail loudly.
#include "cde_internal.h"
using namespace cde;
extern "C" {
int cde_server_start(cde_ctx*, const cde_server_config*) { return set_error(CDE_EINVAL, "not available"); }
int cde_server_stop(cde_ctx*) { return set_error(CDE_EINVAL, "not available"); }
void cde_server_stop_internal(cde_ctx*) {}
int cde_submit(cde_ctx*, const cde_request*, int64_t*) { return set_error(CDE_EINVAL, "not available"); }
int cde_poll(cde_ctx*, int64_t, int*, int*) { return set_error(CDE_EINVAL, "not available"); }
int cde_wait(cde_ctx*, int64_t, int64_t) { return set_error(CDE_EINVAL, "not available"); }
int cde_cancel(cde_ctx*, int64_t) { return set_error(CDE_EINVAL, "not available"); }
int cde_server_stats_get(cde_ctx*, cde_server_stats*) { return set_error(CDE_EINVAL, "not available"); }
int cde_server_stats_reset(cde_ctx*) { return set_error(CDE_EINVAL, "not available"); }
}
