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
    // set to all ones before every solve (one 2-D memset over the control
    // blocks, CTL_ONES_BYTES of each): keys reduced with atomicMin, unset
    // = KEY_UNSET, and the first start stamp
    unsigned long long fmin[2];   // min key over a far list (per split parity)
    unsigned long long fmin_f;    // ordered key of min finite h/F (bucket width default)
    unsigned long long qdelta;    // value order: ordered key of the launch's bucket width (the smallest
                                  // of its instances')
    unsigned long long t_start;   // launch-wide: first start of the persistent pass (%globaltimer, ns)
    // set to zero before every solve
    unsigned int bar_count;       // grid barrier arrivals
    unsigned int bar_gen;         // grid barrier generation
    int cnt[3];                   // near-list lengths
    int fcnt[2];                  // far-list lengths
    int status;                   // EIK_* of this launch
    int abort;                    // set on any error: every block stops
    int left;                     // per-instance completion: the instance's cells requested or running
    // counters (written once per warp at exit)
    unsigned long long visits;    // cell removals
    unsigned long long sweeps;    // sweeps, per cell until its own no-change sweep
    unsigned long long lane_updates;  // node updates executed (incl. lock-step no-ops)
    unsigned long long rounds;
    unsigned long long advances;  // bucket threshold moves
    unsigned long long err_info;  // first failing site (debugging aid)
    // launch-wide control blocks: last end of the persistent pass
    // (%globaltimer, ns; the start is above), kept where events cannot be
    // (graph replay)
    unsigned long long t_end;
    // FHCM Monotonicity Checks: monotone borders / checks made
    unsigned long long mono_ok, mono_n;
    // value-ordered schedule: front moves, cells handed to idle warps
    unsigned long long fronts, handoffs;
    // value-ordered schedule, profiling only: 0 bucket claims, 1 tickets
    // taken, 2 cells received on a ticket, 3 gives, 4 requests filed again
    // (a front moved meanwhile), 5 bucket puts, 6 cells handed on by rare
    // checks, 7 rare checks by parked warps
    unsigned long long qev[8];
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
//   f : the same layout; holds h / F, +inf on obstacles, on padding nodes
//       (i >= nx or j >= ny) and on the ring, and -1 on source nodes (fixed
//       values).  Its TMA box therefore carries a one-node halo of f too.
//   nxp = cxn * k, nyp = cyn * k: the grid padded to whole cells.
//
// One persistent launch solves n_inst instances (a single solve is a batch of
// one).  Each instance has a descriptor in device memory; its tensor maps live
// there too (64-byte aligned; written by the host before the launch).
struct __align__(64) InstDesc {
    CUtensorMap tmU;              // 2-D map over U, box (BW x k+2)
    CUtensorMap tmF;              // 2-D map over f, same box
    void* U;                      // double*, float* or float2* (double-float pairs)
    const void* f;                // f in U's representation
    unsigned long long* cval;     // ordered cell-value keys
    int* qflag;                   // rounds: 1 while queued; async: bit 0 requested, bit 1 running
    int* visits;                  // removals so far
    int* dflags;                  // FHCM: directional flags (bit d: sweep direction d)
    int* lists;                   // 5 * J ints: near[3], far[2]
    Ctl* ctl;                     // this instance's lists, counters and status
    int upitch;
    int cxn, cyn, J;
    double delta;                 // bucket width; < 0: |delta| k min f (from ctl->fmin_f); 0: 4 k min f
    int cell_base;                // index of this instance's first cell among the job's cells
    unsigned* done;               // per-instance completion: a flag in mapped host memory, set to 1 when
                                  // the instance's last requested cell finishes (null: not reported)
};

constexpr int MAX_BATCH = 2048;   // instances per persistent launch
constexpr size_t CTL_ONES_BYTES = 5 * sizeof(unsigned long long);  // the fields of Ctl set to all ones

// Variants of the persistent cell solver: HCM (Sec. 4.2, every removed cell
// swept to convergence), FHCM (Sec. 4.3, one sweep per flagged direction)
// and HCM whose sweeps update only the unlocked nodes of a cell (Remark
// locking_FSM).  FHCM and locking are built for FP64 only.
enum { VAR_HCM = 0, VAR_FHCM = 1, VAR_LSM = 2 };

struct SolveParams {
    const InstDesc* inst;         // n_inst descriptors (device memory)
    int n_inst;
    Ctl* gctl;                    // grid barrier, abort flag, launch status, rounds
    long long deadline_ns;        // relative to kernel start
    int profile;                  // accumulate gctl->prof
    int variant;                  // VAR_HCM, VAR_FHCM or VAR_LSM
    // round-free schedule: a taken cell requested less than hold_ns ago goes
    // back to the ring's tail, so that requests from several upstream
    // neighbours merge into one visit (req_time: request times, per cell;
    // the value-ordered schedule keeps there, complemented, the lowest value
    // proposed while the cell ran)
    unsigned hold_ns;
    unsigned long long* req_time;
    // asynchronous scheduling only: ring of (sequence << 32 | global cell)
    // words, ring_mask + 1 (a power of two) >= twice the job's cells and the
    // launch's warps; the global
    // cell index of (instance i, cell c) is inst[i].cell_base + c, and
    // cell_pre (n_inst + 1 entries) holds the instances' first indices
    unsigned long long* ring;
    unsigned int ring_mask;
    const int* cell_pre;
    unsigned int* qctl;           // ring head, tail and pending count, 128 bytes apart
    int* hist;                    // 3 x 8192 + 1 ints: counting sort of the initial ring
    // value-ordered round-free schedule only: NBQ bucket rings of cell values
    // (bq: head/tail pairs, counts of queued or running cells, the front;
    // BQ_WORDS words), each ring bq_mask + 1 (a power of two >= the job's
    // cells) words of bq_data; warps take cells from the buckets within
    // bq_window of the front
    unsigned int* bq;
    unsigned long long* bq_data;
    unsigned int bq_mask;
    int bq_window;
    // checks of the failure paths and of the schedule's independence, set
    // from the host (0: off): at most max_passes passes per removal (the
    // cap that reports EIK_ENOTCONVERGED), and a pause of up to jitter_ns
    // before each removal's tile load, drawn per removal
    int max_passes;
    unsigned jitter_ns;
    // round-free schedules: count each instance's requested or running cells
    // and flag the instance done when its count reaches zero (its result is
    // final then, while the launch goes on with the others)
    int inst_done;
};
constexpr int NBQ = 32;           // bucket rings of the value-ordered schedule (one lane of a warp each)
constexpr int BQ_WORDS = 160;     // header words: pairs [0, 64), 64-bit counts [64, 128), front at 128

// ---------------------------------------------------------------- host launchers
// Implemented in eik_solver_f64.cu / eik_solver_f32.cu.
struct LaunchShape {
    int threads;       // per block
    size_t smem;       // dynamic shared memory per block
    int blocks;        // co-resident blocks (cooperative launch)
    int per_sm;        // occupancy limit: blocks of this shape one SM holds
    // what one block takes of an SM: registers (allocated per warp in units
    // of 256) and shared memory (static + dynamic + the 1 KB the SM reserves
    // per block)
    int regs_block;
    size_t smem_block;
};
// per-block resources of kernel fn launched with `threads` threads and
// `dyn_smem` bytes of dynamic shared memory
void block_resources(const void* fn, int threads, size_t dyn_smem, LaunchShape* s);

// Schedules of a persistent pass: bucketed rounds (k_solve), or the
// round-free kernel (k_solve_async, cell sizes >= 8) taking cells first in,
// first out or by value (bucket rings with a moving front; plain HCM).
enum { SCH_ROUNDS = 0, SCH_FIFO = 1, SCH_ORDERED = 2 };
// one per arithmetic mode (eik_solver_f64.cu, eik_solver_f32.cu, eik_solver_df.cu)
int solver_shape_f64(int k, int num_sms, int n_inst, int sm_cap, int sched, int variant, LaunchShape* out);
int solver_shape_f32(int k, int num_sms, int n_inst, int sm_cap, int sched, int variant, LaunchShape* out);
int solver_shape_df(int k, int num_sms, int n_inst, int sm_cap, int sched, int variant, LaunchShape* out);
cudaError_t launch_solver_f64(int k, int sched, const SolveParams& p, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_solver_f32(int k, int sched, const SolveParams& p, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_solver_df(int k, int sched, const SolveParams& p, const LaunchShape& s, cudaStream_t st);

// aux kernels (eik_aux.cu)
// ---------------------------------------------------------------- aux kernels
// Per-instance view for the node-wise kernels (eik_aux.cu), which run once
// over all instances of a job: a block covers 8 rows x 32 columns of one
// instance's padded grid, found from `blk_pre` (prefix sums of blocks per
// instance).  Arrays of the other precision mode are null:
//   FP64 mode:       U64, f64
//   FP32+refinement: U32, f32 (FP32 pass), Udf, fdf (double-float pairs,
//                    refinement pass).  All share the layout of SolveParams.
struct ResidualOut {              // reduced with atomics on ordered keys
    unsigned long long r_max;     // max |V - T(V)| over non-source nodes
    unsigned long long r_rel;     // max |V - T(V)| / f over the same nodes
    unsigned long long u_max;     // max finite V
    unsigned long long n_bad;     // finite/infinite mismatches
    unsigned long long n_left;    // cells still requested or running after the solve (must be 0)
};

// Node-wise kernels (eik_aux.cu) map blocks of AUX_ROWS x AUX_COLS nodes
// onto each instance's padded array; a thread handles AUX_COLS / 32 nodes of
// its row, 32 columns apart.
constexpr int AUX_ROWS = 8, AUX_COLS = 128;
__host__ __device__ inline int aux_blocks(int rows, int cols) {
    return ((rows + AUX_ROWS - 1) / AUX_ROWS) * ((cols + AUX_COLS - 1) / AUX_COLS);
}

struct AuxInst {
    const double* F;              // nx*ny row-major speeds (device)
    double* out;                  // nx*ny result (device; the caller's or staging)
    double h;
    float hx, hy;                 // h as a double-float pair
    double shift;                 // min q: stored values are U - shift
    int nx, ny, nxp, nyp, upitch, k, cxn, cyn;
    double* U64; double* f64;
    float* U32; float* f32;
    float2* Udf; float2* fdf;
    unsigned long long* cval; int* qflag; int* visits; int* far0; int* dflags;
    Ctl* ctl;                     // the instance's control block of the first pass
    Ctl* ctl2;                    // ... of the refinement pass (FP32+refinement)
    ResidualOut* res;
    int J;
    double* Fc;                   // FMSM: coarse speeds, J (cyn x cxn)
    double* Uc;                   // FMSM: coarse values, J
};

// Sources of all instances: node (j*nx + i) and shifted q, with instance id;
// source cells with their key (max q) and instance id.
struct SourceTable {
    const int* node; const double* q; const int* node_inst; int n;
    const int* cell; const unsigned long long* cell_key; const int* cell_inst; int ncell;
};

// A block prefix pre[0..n] is followed in memory by its owner table
// (pre[n + 1 + b] = instance of block b), filled by the host; a job of one
// instance needs none (every block is instance 0's).
// f and U over every element of the padded arrays, validation of F, min h/F
// per instance; then, within the same launch, the sources (U = q, f = -1)
// and the source cells (value max q, queued).  The source table is sorted by
// (instance, node).
cudaError_t launch_init_grid(const AuxInst* a, const int* blk_full, int n, int nblocks, const SourceTable& s,
                             cudaStream_t st);
// FP32 result -> double-float start values, cell keys; then queue the cells
cudaError_t launch_seed_refine(const AuxInst* a, const int* blk_pre, int n, int nblocks,
                               const int* cell_pre, int ncells, float beta, cudaStream_t st);
cudaError_t launch_residual(const AuxInst* a, const int* blk_pre, int n, int nblocks, cudaStream_t st);

// Fast Marching-Sweeping Method (eik_fmsm.cu), FP64, cell sizes >= 8:
// coarse speeds Fc of every cell; then, from the coarse values Uc, each
// cell's sweeps, later neighbours and count of earlier ones, the ready cells
// queued (ring and qctl zeroed before); then the persistent pass.
cudaError_t launch_fmsm_coarse_speed(const AuxInst* a, const int* cell_pre, int n, int ncells, cudaStream_t st);
cudaError_t launch_fmsm_prep(const AuxInst* a, const int* cell_pre, int n, int ncells, unsigned long long* ring,
                             unsigned* qctl, cudaStream_t st);
int fmsm_shape(int k, int num_sms, int n_inst, int sm_cap, LaunchShape* out);
cudaError_t launch_fmsm(int k, const SolveParams& p, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_output(const AuxInst* a, const int* blk_pre, int n, int nblocks, cudaStream_t st);

}  // namespace eik
