// Instantiations of the persistent cell solvers (bucketed rounds and the
// round-free schedule) for one arithmetic mode (MODE_DF), all cell sizes,
// and their launcher.
#include "eik_solver_modes.cuh"

namespace eik {

int solver_shape_df(int k, int num_sms, int n_inst, int sm_cap, int sched, int variant, LaunchShape* out) {
    return solver_shape_mode<MODE_DF>(k, num_sms, n_inst, sm_cap, sched, variant, out);
}

cudaError_t launch_solver_df(int k, int sched, const SolveParams& p, const LaunchShape& s, cudaStream_t st) {
    return launch_solver_mode<MODE_DF>(k, sched, p, s, st);
}

}  // namespace eik
