// FP64 instantiations of the persistent cell solver and their launcher.
#include "eik_solver.cuh"

namespace eik {

template <typename T, int K>
static void shape_of(int num_sms, LaunchShape* s) {
    using C = TileCfg<T, K>;
    s->threads = C::WPB * 32;
    s->smem = (size_t)C::WPB * C::WARP_BYTES + 128;
    cudaFuncSetAttribute(k_solve<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<T, K>, s->threads, s->smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 0;
    s->blocks = per_sm * num_sms;
}

template <typename T, int K>
static cudaError_t launch_one(const SolveParams<T>& p, const LaunchShape& s, cudaStream_t st) {
    void* args[] = {(void*)&p};
    return cudaLaunchCooperativeKernel((const void*)k_solve<T, K>, dim3(s.blocks), dim3(s.threads),
                                       args, s.smem, st);
}

#define EIK_SHAPE_CASES(T)                       \
    switch (k) {                                 \
    case 4: shape_of<T, 4>(num_sms, out); break;   \
    case 8: shape_of<T, 8>(num_sms, out); break;   \
    case 16: shape_of<T, 16>(num_sms, out); break; \
    case 32: shape_of<T, 32>(num_sms, out); break; \
    case 64: shape_of<T, 64>(num_sms, out); break; \
    default: return -1;                          \
    }

int solver_shape_f64(int k, int num_sms, LaunchShape* out) {
    EIK_SHAPE_CASES(double)
    return out->blocks > 0 ? 0 : -1;
}

cudaError_t launch_solver_f64(int k, const SolveParams<double>& p, const LaunchShape& s,
                              cudaStream_t st) {
    switch (k) {
    case 4: return launch_one<double, 4>(p, s, st);
    case 8: return launch_one<double, 8>(p, s, st);
    case 16: return launch_one<double, 16>(p, s, st);
    case 32: return launch_one<double, 32>(p, s, st);
    case 64: return launch_one<double, 64>(p, s, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace eik
