// eik_common.cuh -- shared declarations of the CUDA solver (device side and
// the host code that launches it).  Nothing here is visible across the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/eik.h"

namespace eik {

// ---------------------------------------------------------------- keys
// Cell values (eq. cell_value) and bucket thresholds are kept as 64-bit
// "ordered keys": an order-preserving map from doubles to unsigned integers so
// that atomicMin on the key is atomicMin on the value.  KEY_UNSET (all ones,
// the image of a positive NaN) means "no cell value yet" and sorts last.
constexpr unsigned long long KEY_UNSET = ~0ull;

__host__ __device__ inline unsigned long long key_from_bits(long long b) {
    return b >= 0 ? ((unsigned long long)b | 0x8000000000000000ull) : ~(unsigned long long)b;
}
__host__ __device__ inline long long bits_from_key(unsigned long long k) {
    return (k & 0x8000000000000000ull) ? (long long)(k & 0x7fffffffffffffffull)
                                       : (long long)~k;
}

#ifdef __CUDACC__
__device__ inline unsigned long long key_of(double v) {
    return key_from_bits(__double_as_longlong(v));
}
__device__ inline double val_of(unsigned long long k) {
    return __longlong_as_double(bits_from_key(k));
}
#endif

// ---------------------------------------------------------------- control block
// One per persistent launch and instance, zeroed (then initialised) before
// every solve.  Lists: three rotating "near" lists (the bucket being released,
// the re-activations for the next round, and the one being recycled) and two
// "far" lists (cells waiting for a later bucket), each of capacity J because a
// cell is queued at most once at a time.
struct Ctl {
    unsigned int bar_count;       // grid barrier arrivals
    unsigned int bar_gen;         // grid barrier generation
    int cnt[3];                   // near-list lengths
    int fcnt[2];                  // far-list lengths
    int cursor[2];                // work cursor of the current round (by parity)
    int status;                   // EIK_* of this launch
    int abort;                    // set on any error: every block stops
    unsigned long long fmin[2];   // min key over a far list (per split parity)
    unsigned long long fmin_f;    // ordered key of min finite h/F (bucket width default)
    // counters (written once per warp at exit)
    unsigned long long visits;    // cell removals
    unsigned long long sweeps;    // sweeps, per cell until its own no-change sweep
    unsigned long long lane_updates;  // node updates executed (incl. lock-step no-ops)
    unsigned long long rounds;
    unsigned long long advances;  // bucket threshold moves
    unsigned long long err_info;  // first failing site (debugging aid)
    // per-phase clock cycles summed over warps, filled only when profiling
    // (EIK_PROFILE=1): 0 split, 1 barrier, 2 list+pop, 3 TMA wait, 4 sweeps,
    // 5 write-back, 6 activation, 7 warp-rounds with work
    unsigned long long prof[8];
};

// ---------------------------------------------------------------- kernel params
// Device layout (per instance):
//   U : (nyp + 2) rows of `upitch` elements; node (i, j) at
//       (j + 1) * upitch + (i + 1).  Row 0, row nyp + 1, column 0 and every
//       column >= nxp + 1 hold +inf forever (the ring of outside neighbours).
//   f : nyp rows of `fpitch` elements, node (i, j) at j * fpitch + i; holds
//       h / F, +inf on obstacles and on padding nodes (i >= nx or j >= ny),
//       and -1 on source nodes (fixed values).
//   nxp = cxn * k, nyp = cyn * k: the grid padded to whole cells.
struct SolveParams {
    CUtensorMap tmU;              // 2-D map over U, box (BW x k+2)
    CUtensorMap tmF;              // 2-D map over f in U's representation, box (k x k)
    void* U;                      // double*, float* or float2* (double-float pairs)
    const void* f;                // f in U's representation
    int upitch, fpitch;
    int nx, ny;
    int cxn, cyn, J;
    unsigned long long* cval;     // ordered cell-value keys
    int* qflag;                   // 1 while the cell sits in a list
    int* visits;                  // removals so far
    const unsigned char* has_src; // cell contains a source node
    int* lists;                   // 5 * J ints: near[3], far[2]
    Ctl* ctl;
    double delta;                 // bucket width; <= 0: k * min f
    long long deadline_ns;        // relative to kernel start
    int profile;                  // accumulate Ctl::prof
};

// ---------------------------------------------------------------- host launchers
// Implemented in eik_solver_f64.cu / eik_solver_f32.cu.
struct LaunchShape {
    int threads;       // per block
    size_t smem;       // dynamic shared memory per block
    int blocks;        // co-resident blocks (cooperative launch)
};

// one per arithmetic mode (eik_solver_f64.cu, eik_solver_f32.cu, eik_solver_df.cu)
int solver_shape_f64(int k, int num_sms, LaunchShape* out);
int solver_shape_f32(int k, int num_sms, LaunchShape* out);
int solver_shape_df(int k, int num_sms, LaunchShape* out);
cudaError_t launch_solver_f64(int k, const SolveParams& p, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_solver_f32(int k, const SolveParams& p, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_solver_df(int k, const SolveParams& p, const LaunchShape& s, cudaStream_t st);

// aux kernels (eik_aux.cu)
// Device arrays of one instance (null where the precision mode has none):
//   FP64 mode:       U64, f64
//   FP32+refinement: U32, f32 (FP32 pass), Udf, fdf (double-float pairs,
//                    refinement pass).  All U arrays share one layout, all f
//                    arrays another (see SolveParams).
struct InitParams {
    const double* F;              // nx*ny row-major speeds (device)
    int nx, ny;
    double h;
    double* f64; float* f32; float2* fdf; int fpitch;
    double* U64; float* U32; float2* Udf; int upitch;
    int nxp, nyp;
    Ctl* ctl;
};
cudaError_t launch_init_grid(const InitParams& p, cudaStream_t st);
cudaError_t launch_fill(double* a, size_t n, double v, cudaStream_t st);
cudaError_t launch_fill32(float* a, size_t n, float v, cudaStream_t st);
cudaError_t launch_fill_df(float2* a, size_t n, cudaStream_t st);  // (+inf, 0)

struct SourceInit {
    const int* node;              // unique source nodes (j*nx + i)
    const double* q;              // their values, shifted by -min q (>= 0)
    int n;
    const int* cell;              // cells holding a source
    const unsigned long long* cell_key;  // key of max q on that cell
    int ncell;
    int nx, k, cxn;
};
cudaError_t launch_init_sources(const InitParams& ip, const SourceInit& s, unsigned long long* cval,
                                int* qflag, unsigned char* has_src, int* far0, cudaStream_t st);

cudaError_t launch_ctl_init(Ctl* ctl, int nfar0, cudaStream_t st);

struct SeedParams {
    const float* U32;
    float2* Udf;
    const float2* fdf;
    int upitch, fpitch;
    int nx, ny, k, cxn, cyn;
    float beta;                   // relative bump (values are >= 0 after the q shift)
    unsigned long long* cval; int* qflag; int* visits; int* far0;
    Ctl* ctl;
};
cudaError_t launch_seed_refine(const SeedParams& p, cudaStream_t st);

struct ResidualOut {              // reduced with atomics on ordered keys
    unsigned long long r_max;     // max |V - T(V)| over non-source nodes
    unsigned long long u_max;     // max finite V
    unsigned long long n_bad;     // finite/infinite mismatches
};
// FP64 residual of the double-float result Udf, with f = h/F recomputed in
// FP64 from the input speeds; sources are the nodes with fdf.x < 0.
cudaError_t launch_residual(const float2* Udf, int upitch, const float2* fdf, int fpitch,
                            const double* F, double h, int nx, int ny, ResidualOut* out,
                            cudaStream_t st);
// dst[j*nx + i] = U[(j+1)*pitch + i+1] + shift (undoes the q shift); exactly
// one of U64 / Udf is non-null
cudaError_t launch_output(const double* U64, const float2* Udf, int upitch, int nx, int ny,
                          double shift, double* dst, cudaStream_t st);

}  // namespace eik
