// eik_solver_modes.cuh -- launch shape and launcher of the persistent solver
// kernels for one arithmetic mode; included once by each eik_solver_*.cu.
#pragma once

#include "eik_solver.cuh"

namespace eik {

// The Fast Heap-Cell variant and HCM with locking are built for FP64 only
// (the only mode that offers them); the plain HCM kernels carry none of
// their code.
// sched: SCH_ROUNDS (k_solve), SCH_FIFO or SCH_ORDERED (k_solve_async,
// one cell per warp; the value-ordered form is built for plain HCM only)
template <int MODE, int K, int VAR>
static const void* solver_fn_var(int sched) {
    if constexpr (TileCfg<MODE, K>::CPW == 1) {
        if constexpr (VAR == VAR_HCM)
            if (sched == SCH_ORDERED) return (const void*)k_solve_async<MODE, K, VAR, true>;
        if (sched != SCH_ROUNDS) return (const void*)k_solve_async<MODE, K, VAR, false>;
    }
    return (const void*)k_solve<MODE, K, VAR>;
}

template <int MODE, int K>
static const void* solver_fn(int sched, int variant) {
    if constexpr (MODE == MODE_F64) {
        if (variant == VAR_FHCM) return solver_fn_var<MODE, K, VAR_FHCM>(sched);
        if (variant == VAR_LSM) return solver_fn_var<MODE, K, VAR_LSM>(sched);
    }
    return solver_fn_var<MODE, K, VAR_HCM>(sched);
}

template <int MODE, int K>
static void shape_of(int num_sms, int n_inst, int sm_cap, int sched, int variant, LaunchShape* s) {
    using C = TileCfg<MODE, K>;
    const void* fn = solver_fn<MODE, K>(sched, variant);
    const bool async = sched != SCH_ROUNDS;
    s->threads = C::WPB * 32;
    s->smem = (size_t)C::WPB * C::WARP_BYTES + (size_t)C::lk_area(MODE == MODE_F64 ? variant : VAR_HCM) + 128 +
              (size_t)inst_state_bytes(n_inst);
    s->blocks = 0;
    s->per_sm = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, s->threads, s->smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    // a single grid in rounds: at most two blocks per SM (a round rarely has
    // more cells than that, and every extra block makes each grid barrier
    // slower); a batch keeps every SM full, and the round-free schedule has no
    // barrier and gains from more warps waiting for cells (1025^2: 1.82 ms at
    // three blocks per SM, 1.94 ms at two), so both take the occupancy limit
    int cap = n_inst > 1 || async ? per_sm : 2;
    if (sm_cap > 0 && sm_cap < cap) cap = sm_cap;  // leave room for other jobs
    s->blocks = (per_sm < cap ? per_sm : cap) * num_sms;
    s->per_sm = per_sm;
    block_resources(fn, s->threads, s->smem, s);
}

template <int MODE>
static int solver_shape_mode(int k, int num_sms, int n_inst, int sm_cap, int sched, int variant,
                             LaunchShape* out) {
    out->blocks = 0;
    switch (k) {
    case 4: shape_of<MODE, 4>(num_sms, n_inst, sm_cap, sched, variant, out); break;
    case 8: shape_of<MODE, 8>(num_sms, n_inst, sm_cap, sched, variant, out); break;
    case 16: shape_of<MODE, 16>(num_sms, n_inst, sm_cap, sched, variant, out); break;
    case 32: shape_of<MODE, 32>(num_sms, n_inst, sm_cap, sched, variant, out); break;
    case 64: shape_of<MODE, 64>(num_sms, n_inst, sm_cap, sched, variant, out); break;
    default: return -1;
    }
    return out->blocks > 0 ? 0 : -1;
}

template <int MODE, int K>
static cudaError_t launch_one(int sched, int variant, const SolveParams& p, const LaunchShape& s,
                              cudaStream_t st) {
    void* args[] = {(void*)&p};
    return cudaLaunchCooperativeKernel(solver_fn<MODE, K>(sched, variant), dim3(s.blocks), dim3(s.threads), args,
                                       s.smem, st);
}

template <int MODE>
static cudaError_t launch_solver_mode(int k, int sched, const SolveParams& p, const LaunchShape& s,
                                      cudaStream_t st) {
    switch (k) {
    case 4: return launch_one<MODE, 4>(sched, p.variant, p, s, st);
    case 8: return launch_one<MODE, 8>(sched, p.variant, p, s, st);
    case 16: return launch_one<MODE, 16>(sched, p.variant, p, s, st);
    case 32: return launch_one<MODE, 32>(sched, p.variant, p, s, st);
    case 64: return launch_one<MODE, 64>(sched, p.variant, p, s, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace eik
