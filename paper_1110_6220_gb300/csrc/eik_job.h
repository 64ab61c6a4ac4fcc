// eik_job.h -- a job: n instances solved together (same cell size k and
// precision mode): one launch per kernel for all of them.  Plans (n = 1),
// batches and the no-allocation solve all run through enqueue_job.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "eik_common.cuh"

namespace eik {

struct Layout {
    int nx, ny, k;
    int cxn, cyn, J;
    int nxp, nyp;
    int upitch, urows;  // U and f arrays: urows x upitch elements (ring included)
};

Layout make_layout(int nx, int ny, int k);

// Device arrays of one instance inside a job's arena.
struct InstArrays {
    double* U64; double* f64;   // FP64 mode
    float* U32; float* f32;     // FP32 + refinement: FP32 pass
    float2* Udf; float2* fdf;   //                    refinement pass
    unsigned long long* cval;
    int* qflag;
    int* visits;
    int* dflags;                // FHCM: directional flags per cell
    int* lists;                 // 5 J
    double* Fstage;             // device copy of a host F (null if F is on the device)
    double* Ostage;             // result staging for a host U (null if U is on the device)
};

// Bytes instance arrays need (256-byte aligned pieces).
size_t inst_bytes(const Layout& L, bool fp32, bool stage_F, bool stage_U);
// Assign the arrays of one instance from base (which must have inst_bytes).
InstArrays carve_inst(const Layout& L, bool fp32, bool stage_F, bool stage_U, char* base);

// Control blocks and tables of a job, all in device memory.
struct JobDev {
    int n;                      // instances
    int k;
    bool fp32;
    InstDesc* desc_main;        // n: FP64 pass or refinement pass
    InstDesc* desc_f32;         // n: FP32 pass (fp32 only)
    AuxInst* aux;               // n
    int* blk_pre;               // n + 1: prefix of 8x32 blocks over each padded interior
    int* blk_full;              // n + 1: prefix of 8x32 blocks over each whole array (ring too)
    int* cell_pre;              // n + 1: prefix of cells per instance
    int nblocks, nblocks_full, ncells;
    Ctl* ictl;                  // 2n: [0, n) first pass, [n, 2n) refinement pass
    Ctl* gctl;                  // 2: launch-wide control of each pass
    ResidualOut* res;           // n
    SourceTable src;            // device pointers
    int nsrc_total, ncell_total;
    long long deadline_ns;
    int sm_cap;                 // > 0: at most this many blocks per SM (room for other jobs)
    bool async_first, async_main;  // round-free schedule (k_solve_async) for the FP32 / main pass
    bool one_pass;              // fp32: no FP32 pass; the double-float pass solves from the sources
    int variant;                // main pass: VAR_HCM, VAR_FHCM or VAR_LSM
    bool fmsm;                  // Fast Marching-Sweeping Method (coarse solve, then one visit per cell)
    const JobDev* coarse;       // FMSM: the job of the instances' coarse grids
    unsigned hold_ns;           // round-free: minimum age of a request before its cell runs
    unsigned long long* req_time;  // request times per cell (job-wide index), %globaltimer ns
    unsigned long long* ring;   // async: ring of ring_mask + 1 words
    unsigned ring_mask;
    unsigned* qctl;             // async: head, tail, pending (384 bytes before the ring)
    int* hist;                  // async: 3 x 8192 + 1 ints of counting-sort scratch
    // value-ordered main pass (plain HCM, round-free): bucket rings and their
    // header, and the window in buckets (null bq: first in, first out)
    bool ordered;
    int window;
    unsigned* bq;
    unsigned long long* bq_data;
    unsigned bq_mask;
    // per-instance completion (a round-free main pass in one launch): each
    // instance's done flag is set by the launch, and the node-wise kernel
    // that writes the output runs per instance (finish_instance), not after
    // the pass
    bool inst_done;
    // everything that enqueue_job zeroes before a solve: [zero_base, + zero_bytes)
    void* zero_base;
    size_t zero_bytes;
    // cval / qflag / visits of all instances, contiguous
    unsigned long long* cval_all; size_t ncval;
    int* qflag_all;
    int* visits_all;
};

// Host-side pieces used to fill a JobDev's tables.
bool make_map(CUtensorMap* tm, void* base, bool fp64, int width, int rows, int pitch_elems,
              int box_w, int box_h);
// bw_first / bw_main: bucket width of the FP32 pass and of the FP64 (or
// refinement) pass, > 0 absolute, < 0 relative to k min(h/F), 0 default.
void fill_inst_tables(const Layout& L, const InstArrays& a, bool fp32, double h, double bw_first,
                      double bw_main,
                      Ctl* ictl_first, Ctl* ictl_main, ResidualOut* res, const double* F,
                      double* out, double shift, AuxInst* aux, InstDesc* desc_main, InstDesc* desc_f32,
                      bool* ok);

// Queue the whole solve of a job on st (tables and sources already uploaded).
// ev: null or 4 events around the FP32 pass (FMSM: the coarse solve) [0,1]
// and the main pass [2,3].
int enqueue_job(const JobDev& j, int num_sms, cudaStream_t st, cudaEvent_t* ev, int* launches);

// What the solver launches of a job take of one SM per block (the largest
// over its passes, resource by resource) and the fewest blocks of them one
// SM holds; false if a launch shape cannot be formed (FMSM jobs, whose
// coarse job runs its own launches, report false: they run alone).
struct Footprint {
    int threads = 0, regs = 0, per_sm = 0;
    size_t smem = 0;
};
bool job_footprint(const JobDev& j, int num_sms, Footprint* fp);

// Per-instance completion: the node-wise kernel that certifies and writes
// instance i's output (FP32_REFINE: the residual; FP64: the output), alone,
// on st.  L: the instance's layout.
int finish_instance(const JobDev& j, int i, const Layout& L, cudaStream_t st);
// The same for every instance of the job in one launch (instances finished
// alone before are written again with the same values).
int finish_instances(const JobDev& j, cudaStream_t st);
// A job that only carries the schedule flags, for job_footprint before the
// job is built.
JobDev probe_job(int n, int k, bool fp32, bool one_pass, bool async_first, bool async_main, bool ordered,
                 int variant);

// Fill *st for instance i from the control blocks copied back to the host.
void job_stats(const Layout& L, const eik_plan_desc* d, bool fp32, const Ctl* ictl_first,
               const Ctl* ictl_main, const Ctl* g_first, const Ctl* g_main, const ResidualOut* r,
               double q_min, double bw_main, double ms,
               eik_stats* st);

}  // namespace eik
