// Entry points whose kernels are not in this build yet: they fail loudly.
#include "cde_internal.h"
using namespace cde;
extern "C" {
int cde_loo_grad(cde_ctx*, cde_dataset, double, double, double*, int, void*) { return set_error(CDE_EINVAL, "cde_loo_grad: not available"); }
int cde_density(cde_ctx*, cde_dataset, double, double, const float*, int64_t, const float*, int, float*, int, void*) { return set_error(CDE_EINVAL, "cde_density: not available"); }
int cde_loo_loglik_batch(cde_ctx*, int, const cde_dataset*, const double* const*, const int*, const double* const*, const int*, double* const*, double* const*, void*) { return set_error(CDE_EINVAL, "cde_loo_loglik_batch: not available"); }
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
