// Instantiations of the persistent cell solvers (bucketed rounds and the
// round-free schedule) for one arithmetic mode (MODE_F32), all cell sizes,
// and their launcher.
#include "eik_solver_modes.cuh"

namespace eik {

int solver_shape_f32(int k, int num_sms, int n_inst, int sm_cap, int sched, int variant, LaunchShape* out) {
    return solver_shape_mode<MODE_F32>(k, num_sms, n_inst, sm_cap, sched, variant, out);
}

cudaError_t launch_solver_f32(int k, int sched, const SolveParams& p, const LaunchShape& s, cudaStream_t st) {
    return launch_solver_mode<MODE_F32>(k, sched, p, s, st);
}

}  // namespace eik
