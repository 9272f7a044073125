// otgs_stubs.cu -- entry points whose device code is not built yet.
#include "otgs_handle.cuh"

using namespace otgs;

namespace otgs {
bool Handle::ensure_screen() { return fail(OTGS_EINVAL, "screening not built"); }
bool Handle::snapshot_at(const double*, bool, const double*, bool, double*, double*, const double*)
{
    return fail(OTGS_EINVAL, "screening not built");
}
bool Handle::eval_screened(const double*, bool, const double*, double*, double*, const double*)
{
    return fail(OTGS_EINVAL, "screening not built");
}
bool Handle::collect_stats() { return true; }
void Handle::reset_device_stats() {}
}  // namespace otgs

extern "C" {
int ot_gs_grad_screened(ot_gs*, const double*, const double*, double*, uint32_t*) { return OTGS_EINVAL; }
int ot_gs_snapshot(ot_gs*, const double*, const double*, int, double*) { return OTGS_EINVAL; }
int ot_gs_get_screen_state(ot_gs*, float*, float*, double*, double*, uint32_t*) { return OTGS_EINVAL; }
int ot_gs_solve(ot_gs*, double, int32_t) { return OTGS_EINVAL; }
int ot_gs_get_solution(ot_gs*, double*, double*, double*, double*, int32_t*) { return OTGS_EINVAL; }
int ot_gs_set_state(ot_gs*, const double*, const double*) { return OTGS_EINVAL; }
}
