// Instantiations of the persistent cell solver for one arithmetic mode
// (MODE_F32), all cell sizes, and their launcher.
#include "eik_solver.cuh"

namespace eik {

template <int K>
static void shape_of(int num_sms, int n_inst, int sm_cap, LaunchShape* s) {
    using C = TileCfg<MODE_F32, K>;
    s->threads = C::WPB * 32;
    s->smem = (size_t)C::WPB * C::WARP_BYTES + 128 + (size_t)inst_state_bytes(n_inst);
    s->blocks = 0;
    s->per_sm = 0;
    if (cudaFuncSetAttribute(k_solve<MODE_F32, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)s->smem) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<MODE_F32, K>, s->threads,
                                                      s->smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    // a single grid: at most two blocks per SM (a round rarely has more cells
    // than that, and every extra block makes each grid barrier slower); a
    // batch keeps every SM full, so it takes the occupancy limit
    int cap = n_inst > 1 ? per_sm : 2;
    if (sm_cap > 0 && sm_cap < cap) cap = sm_cap;  // leave room for other jobs
    s->blocks = (per_sm < cap ? per_sm : cap) * num_sms;
    s->per_sm = per_sm;
}

template <int K>
static cudaError_t launch_one(const SolveParams& p, const LaunchShape& s, cudaStream_t st) {
    void* args[] = {(void*)&p};
    return cudaLaunchCooperativeKernel((const void*)k_solve<MODE_F32, K>, dim3(s.blocks),
                                       dim3(s.threads), args, s.smem, st);
}

int solver_shape_f32(int k, int num_sms, int n_inst, int sm_cap, LaunchShape* out) {
    out->blocks = 0;
    switch (k) {
    case 4: shape_of<4>(num_sms, n_inst, sm_cap, out); break;
    case 8: shape_of<8>(num_sms, n_inst, sm_cap, out); break;
    case 16: shape_of<16>(num_sms, n_inst, sm_cap, out); break;
    case 32: shape_of<32>(num_sms, n_inst, sm_cap, out); break;
    case 64: shape_of<64>(num_sms, n_inst, sm_cap, out); break;
    default: return -1;
    }
    return out->blocks > 0 ? 0 : -1;
}

cudaError_t launch_solver_f32(int k, const SolveParams& p, const LaunchShape& s, cudaStream_t st) {
    switch (k) {
    case 4: return launch_one<4>(p, s, st);
    case 8: return launch_one<8>(p, s, st);
    case 16: return launch_one<16>(p, s, st);
    case 32: return launch_one<32>(p, s, st);
    case 64: return launch_one<64>(p, s, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace eik
