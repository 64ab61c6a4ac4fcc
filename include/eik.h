/*
 * eik.h -- C ABI of the GB300-native two-scale Eikonal solver.
 *
 * Problem (Chacon & Vladimirsky, "Fast two-scale methods for Eikonal
 * equations", Sec. 1 eq. Eikonal and Sec. 3): find U on an nx x ny Cartesian
 * grid with spacing h such that, at every node that is not a source, the
 * first-order upwind discretisation of |grad u| F = 1 holds (Sec. 3,
 * eq. Eik_discr):
 *
 *   max(U - min(U_W, U_E), 0)^2 + max(U - min(U_S, U_N), 0)^2 = (h / F)^2,
 *
 * with U = q on the source set Q.  Neighbours outside the grid count as
 * +infinity (the exit-set form of Sec. 3: q = +inf on the boundary outside
 * Q).  F = 0 marks an obstacle: such a node stays +inf unless it is a source.
 *
 * Method: the heap-cell idea of Sec. 4.2 (Alg. generic_LC_cells with the cell
 * values of eq. cell_value and the directional flags of Remark
 * HCM_preferred_sweeps), recast for the GPU -- k x k cells are released from
 * a device-side queue in buckets of cell value instead of one at a time, and
 * each released cell is swept to convergence in shared memory.  By Theorem
 * convergence the result is the exact solution of eq. Eik_discr for any
 * removal order.
 *
 * Layout of every grid array passed in or out: row-major, x fastest, node
 * (i, j) at index j*nx + i, x_i = i*h, y_j = j*h.
 *
 * Pointers: every data pointer (F, sources, U) may be a host pointer or a
 * CUDA device pointer; the library detects which.  Pinned host F and U
 * (cudaMallocHost, cudaHostAlloc, cudaHostRegister) are read and written in
 * place by the kernels across the host link; pageable host buffers are copied
 * through the plan's workspace.  Host source tables are always read by the
 * host.
 * The caller owns all buffers; they must stay valid until the call that uses
 * them has returned (eik_solve, eik_solve_batch) or until eik_poll reports
 * EIK_OK (eik_submit).
 *
 * Errors: every function returns an eik status code (0 = EIK_OK, negative =
 * error); nothing aborts, throws or traps across this boundary.  Device-side
 * waits are bounded by a deadline after which the solve stops with
 * EIK_ETIMEDOUT and the CUDA context stays usable.
 *
 * Threading: an eik_plan may be used by one thread at a time; different plans
 * are independent.  A server (eik_server) is thread-safe.
 */
#ifndef EIK_H
#define EIK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
enum {
    EIK_OK = 0,
    EIK_EINVAL = -1,         /* malformed argument (see each function) */
    EIK_ENOMEM = -2,         /* device or host allocation failed */
    EIK_EBUSY = -3,          /* admission refused: over the memory budget or no slot */
    EIK_EAGAIN = -4,         /* eik_poll: request not finished yet */
    EIK_ETIMEDOUT = -5,      /* device deadline expired; result incomplete */
    EIK_ENOTCONVERGED = -6,  /* sweep cap hit, or the FP32+refinement
                                certificate did not reach the tolerance */
    EIK_ECUDA = -7           /* a CUDA runtime call failed */
};

/* Precision modes.  EIK_FP64: FP64 values; the two-sided increment is
 * evaluated in double-float arithmetic (~1e-14 of it), the sums in FP64.
 * EIK_FP32_REFINE: every update on the FP32 pipe with the cancellation-free
 * quadratic, values carried as double-float pairs -- either one pass from
 * the sources, or an FP32 pass and a refinement pass seeded from it (see
 * autotuning) -- then a residual check whose bound (eik_stats.err_bound)
 * certifies the tolerance. */
enum { EIK_FP64 = 0, EIK_FP32_REFINE = 1 };

/* Methods.  EIK_METHOD_HCM: every removed cell is solved to convergence
 * (Sec. 4.2): the exact solution of eq. Eik_discr.  EIK_METHOD_FHCM: the
 * Fast Heap-Cell Method (Sec. 4.3, Alg. FHCM): a removed cell is swept once
 * in each of its flagged directions, and an activation flags one or two
 * directions by the Monotonicity Check of the cell border; faster, never
 * below the exact solution, but not exact (FP64 only).  EIK_METHOD_FMSM:
 * the Fast Marching-Sweeping Method (Sec. 4.1, Alg. FMSM): Fast Marching on
 * the coarse grid of cell centres (speed F at each centre, as the mean of
 * the nodes nearest to it; the cells holding sources as its exit set, each
 * with its smallest q) orders the cells; each cell is then processed once in
 * that order -- a cell holding a source by Fast Sweeping to convergence, any
 * other by at most four sweeps with sweep-directional updates in the
 * directions set by its neighbours accepted before it (Remark
 * sweeping_in_FMSM, Fig. coarse_sweep_choice).  Never below the exact
 * solution, not exact; FP64 and cell sizes >= 8 only (cell_k 0 picks 8 or
 * more).  EIK_METHOD_HCM_LSM: HCM whose cells are swept by the Locking
 * Sweeping version of Fast Sweeping, as Sec. 4.2 specifies (Remark
 * locking_FSM): a sweep updates only a cell's unlocked nodes, each node it
 * takes is locked, and a node that decreases unlocks its larger neighbours;
 * at a removal the nodes next to a neighbouring cell start unlocked (on the
 * first removal also those next to a source of the cell), and the removal
 * ends when none is unlocked.  The same exact solution as EIK_METHOD_HCM with
 * fewer local updates (eik_stats.updates_per_pt counts the ones computed);
 * FP64 only. */
enum { EIK_METHOD_HCM = 0, EIK_METHOD_FHCM = 1, EIK_METHOD_FMSM = 2, EIK_METHOD_HCM_LSM = 3 };

/* Schedules of the cell solver's persistent passes (the order in which
 * queued cells are removed; Theorem convergence makes the result the same
 * for any order, up to rounding -- only the work and the time differ).
 * EIK_SCHED_AUTO: the tuned or built-in choice (see autotuning).
 * EIK_SCHED_ROUNDS: bucketed rounds -- every queued cell within one bucket
 * width of the smallest cell value is released at once, re-activations run
 * in the next round, a grid-wide barrier ends each round.
 * EIK_SCHED_FIFO: round-free -- each warp takes the next requested cell from
 * a first-in first-out device queue as soon as it is free; cell values are
 * not used.
 * EIK_SCHED_ORDERED: round-free in order of value -- requested cells wait in
 * buckets of the value their activation proposes (eq. cell_value), Dial's
 * buckets of Sec. 2 without rounds; warps take the oldest cell of the lowest
 * bucket within `window` buckets of the lowest one still holding a queued or
 * running cell, which moves up as its last cell finishes.  Cell sizes >= 8;
 * EIK_METHOD_HCM only (the other methods fall back to EIK_SCHED_FIFO). */
enum { EIK_SCHED_AUTO = 0, EIK_SCHED_ROUNDS = 1, EIK_SCHED_FIFO = 2, EIK_SCHED_ORDERED = 3 };

/* Problem-shape description (Sec. 3 problem statement plus the method's
 * cell size).  All fields are read at eik_plan_create. */
typedef struct {
    int32_t nx, ny;        /* grid nodes per side, each >= 2 */
    double h;              /* grid spacing, > 0 */
    int32_t cell_k;        /* cell side k in nodes: 4, 8, 16, 32 or 64; 0 = choose */
    double bucket_width;   /* width Delta of a bucket of cell values (Sec. 2's Dial buckets):
                              > 0: absolute; < 0: |bucket_width| * k * min(h/F);
                              0: the tuned or built-in choice (see autotuning) */
    int32_t precision;     /* EIK_FP64 or EIK_FP32_REFINE */
    double tol;            /* FP32_REFINE: certified max error / max|u|; <= 0: 1e-5 */
    int64_t deadline_ns;   /* device wall-clock limit per solve; <= 0: 20 s */
    int32_t method;        /* EIK_METHOD_HCM, EIK_METHOD_FHCM, EIK_METHOD_FMSM or EIK_METHOD_HCM_LSM */
    int32_t schedule;      /* EIK_SCHED_*: the persistent passes' schedule; 0 = tuned / built in */
    int32_t window;        /* EIK_SCHED_ORDERED: buckets warps take cells from, counting the
                              lowest, 1..32; 0 = tuned / built in */
} eik_plan_desc;

/* One problem instance (Sec. 3: speed F, exit set Q with values q). */
typedef struct {
    const double* F;        /* nx*ny speeds, F >= 0 and finite; 0 = obstacle */
    const int32_t* src_ij;  /* 2*nsrc ints: (i, j) of each source node */
    const double* src_q;    /* nsrc source values q, finite; duplicates keep the min */
    int32_t nsrc;           /* number of sources, >= 0 (0: U is +inf everywhere) */
    double* U;              /* out: nx*ny values; +inf = unreachable */
} eik_instance;

/* Per-solve report.  Counters follow the paper's cost accounting (Sec. 5):
 * avhr = cell removals / cells (AvHR), avs = sweeps / cells (AvS). */
typedef struct {
    double ms;              /* device time from inputs resident to result ready */
    double mpts_per_s;      /* nx*ny / ms / 1000 */
    double updates_per_pt;  /* local updates evaluated / (nx*ny) */
    double avhr;            /* cell visits / number of cells */
    double avs;             /* cell sweeps / number of cells */
    double max_residual;    /* max |V - T(V)| over finite non-source nodes (FP32_REFINE; an
                               upper bound, evaluated in double-float with an allowance) */
    double err_bound;       /* certified max |V - U| / max|U| (FP32_REFINE); 0 for FP64 */
    double bucket_width;    /* bucket width used */
    int64_t cell_visits;    /* total cell removals (all passes) */
    int64_t rounds;         /* grid-wide rounds (barrier-separated bucket releases) */
    int64_t buckets;        /* bucket advances (threshold moves) */
    double pass_ms[2];      /* device time of the persistent FP32 pass (FMSM: the coarse solve) [0]
                               and main pass [1]
                               (events on the launching stream; the kernels' own timers when
                               replayed from a graph; 0 if not run) */
    int32_t launches;       /* kernels this solve launched */
    int32_t cell_k;         /* cell size used */
    int32_t schedule;       /* bit 0: FP32 pass round-free; bit 1: FP64 / double-float pass
                               round-free; bit 2: FP32_REFINE as one double-float pass;
                               bit 3: replayed from a captured CUDA graph; bit 4: FMSM (a
                               coarse solve, then every cell once as its predecessors finish) */
    int32_t status;         /* EIK_OK or the error of this solve */
    double mono_pct;        /* FHCM: Monotonicity Checks that found the border monotone, % */
    int64_t queue_left;     /* cells still requested or running after the solve: 0 whenever the
                               status is EIK_OK (a check of the work queue's bookkeeping) */
} eik_stats;

typedef struct eik_plan_s* eik_plan;

/* Human-readable name of a status code.  Never NULL. */
const char* eik_strerror(int code);

/* Create a plan for one grid shape: validates *d (EIK_EINVAL for nx or ny <
 * 2, h <= 0, a cell_k outside {0,4,8,16,32,64}, an unknown precision), and
 * allocates the device workspace (EIK_ENOMEM on failure).  cuda_stream is a
 * cudaStream_t on which all of the plan's work is queued; NULL makes the plan
 * create its own non-blocking stream.  On success *out owns the workspace. */
int eik_plan_create(eik_plan* out, const eik_plan_desc* d, void* cuda_stream);

/* Release a plan and its device workspace.  NULL is ignored. */
void eik_plan_destroy(eik_plan p);

/* Bytes of device workspace a plan for *d would hold (0 if *d is invalid);
 * for EIK_METHOD_FMSM this includes the coarse grid's solve. */
size_t eik_plan_workspace_bytes(const eik_plan_desc* d);

/* Solve one instance on the plan's grid shape; blocks until U is written.
 * EIK_EINVAL: NULL pointers, nsrc < 0, a source outside the grid or with a
 * non-finite q, an F value that is negative, NaN or infinite.  st may be NULL. */
int eik_solve(eik_plan p, const eik_instance* in, eik_stats* st);

/* Solve n_inst independent instances of (possibly) different shapes together:
 * one persistent launch per pass for all instances of the same cell size and
 * precision, with a device-side work queue per instance (Sec. 4.2's lists,
 * one per grid) and every SM serving cells of any instance.  d[i] describes
 * instance i (nx, ny, h, cell_k, bucket_width, precision, tol); deadline_ns of
 * d[0] applies to each launch.  Up to 2048 instances share a launch; more are
 * run as several launches.  st: NULL or n_inst entries (ms is the device time
 * of the launch that held the instance).  Blocks until every U is written.
 * Returns EIK_OK if every instance succeeded, else the first error; the
 * status of each instance is in st[i].status. */
int eik_solve_batch(const eik_plan_desc* d, const eik_instance* in, int32_t n_inst,
                    eik_stats* st, void* cuda_stream);

/* ------------------------------------------------------- fixed batches
 * A batch solved again and again (the same grids with new speeds, a time
 * loop, a benchmark).  eik_batch_create builds everything eik_solve_batch
 * builds -- layouts, tables, sources, device workspace, the tuned cell size
 * and schedule -- once, and captures each job's launch sequence in a CUDA
 * graph; eik_batch_run replays it.  The instances' sizes, pointers and
 * sources are fixed at creation: their F values may change between runs
 * (speeds in host memory are copied in at each run) and their U buffers
 * receive each run's result.  cuda_stream: NULL, or a stream whose queued
 * work each run waits for.  Where a graph cannot be captured the jobs are
 * queued directly (eik_stats.schedule bit 3 tells which).
 *
 * eik_batch_run blocks until every U is written; st: NULL or n_inst entries
 * (ms is the device time of the job that holds the instance).  Returns
 * EIK_OK if every instance succeeded, else the first error. */
typedef struct eik_batch_s* eik_batch;
int eik_batch_create(eik_batch* out, const eik_plan_desc* d, const eik_instance* in, int32_t n_inst,
                     void* cuda_stream);
int eik_batch_run(eik_batch b, eik_stats* st);
void eik_batch_destroy(eik_batch b);

/* ------------------------------------------------------- autotuning
 * The cell size k (Sec. 4) and the width of the value buckets (Sec. 2's
 * Dial buckets) trade grid-wide rounds against repeated cell visits, and the
 * best choice depends on the grid, its speed field and on whether it runs
 * alone or in a batch.  The library keeps a table of choices per class of
 * job: (precision, one instance or a batch, mean side length rounded to a
 * power of two).  A descriptor that leaves cell_k at 0 gets the table's k;
 * one that leaves bucket_width at 0 gets the table's widths (one for the FP32
 * pass, one for the FP64 or refinement pass).  Classes not in the table use
 * built-in choices measured on GB300.  Plans take the choice at
 * eik_plan_create; batches and served jobs at each call.
 *
 * Each pass runs on one of the schedules above (EIK_SCHED_*).  FP32_REFINE
 * runs either as an FP32 pass followed by a double-float refinement pass
 * seeded from it, or as one double-float pass from the sources; both take
 * every update on the FP32 pipe and end with the same FP64 residual
 * certificate.  Built in: single FP64 grids from about 512^2, and single
 * FP32_REFINE grids from about 4096^2 (cells of 16), run in value order,
 * which keeps the visits per cell low where a first-in first-out queue's grow
 * with the grid; smaller single grids and all batches run first in, first
 * out (batches with cells of 16), where the value order's queue costs more
 * than the visits it saves.
 *
 * eik_tune: time trial solves of the given instances, run as one job like
 * eik_solve_batch (n_inst = 1: like eik_solve), over k in {8, 16, 32}, rounds
 * with relative widths {2, 4, 16, 64, 256}, the round-free schedule, and the
 * value-ordered one with widths {2, 4, 8} and windows of 3 and 4 buckets,
 * timing each pass on its own; record
 * the fastest choice for the job's class (never one slower than the choice
 * in force before) and return it.  Blocks; about forty solves.  Each U
 * receives a valid result.  All descriptors must have one precision and a
 * heap-cell method (EIK_METHOD_FMSM is refused with EIK_EINVAL);
 * their cell_k and bucket_width are ignored.  The table is per process and
 * shared by all threads and devices.  EIK_TUNE_FILE, if set, names a file
 * loaded on first use. */
typedef struct {
    int32_t cell_k;        /* chosen k */
    double bucket_first;   /* relative width of the FP32 pass (FP32_REFINE) */
    double bucket_main;    /* relative width of the FP64 / refinement pass */
    int32_t async_first;   /* 1: the FP32 pass runs round-free (no buckets) */
    int32_t async_main;    /* 1: the FP64 / refinement pass runs round-free */
    int32_t one_pass;      /* FP32_REFINE: 1 = one double-float pass from the sources, 0 = an
                              FP32 pass, then a refinement pass seeded from it */
    int32_t hold_ns;       /* round-free: a taken cell younger than this (since its latest
                              request) goes back to the ring's tail and the warp takes the
                              next, so that several upstream changes merge into one visit */
    double ms;             /* device time of the job with the chosen values */
    double ms_before;      /* device time with the choice in force before */
    int32_t trials;        /* solves run */
    int32_t ordered;       /* 1: the round-free passes run in value order (EIK_SCHED_ORDERED) */
    int32_t window;        /* ... taking cells from this many buckets (eik_plan_desc.window) */
} eik_tune_result;

int eik_tune(const eik_plan_desc* d, const eik_instance* in, int32_t n_inst, void* cuda_stream,
             eik_tune_result* out);
/* Write / merge the table as text ("eik-tune 4" then one line per class).
 * EIK_EINVAL if the file cannot be written / read or is malformed (nothing
 * merged then). */
int eik_tune_save(const char* path);
int eik_tune_load(const char* path);
/* Forget every tuned entry (the built-in choices remain). */
void eik_tune_reset(void);

/* ------------------------------------------------------- serving
 * A request loop that keeps grids and cell queues on the device.  A server
 * thread takes submitted requests in arrival order and launches the oldest
 * ones of one (cell size, precision) class as a batched job (as
 * eik_solve_batch) on one of four job slots, each with its own stream and
 * device workspace.  A request is admitted when its device memory fits
 * hbm_budget_bytes together with the other running jobs, so requests that
 * arrive while jobs run start in a free slot as soon as memory allows, and
 * the jobs share the GPU's SMs (continuous batching): each takes as many
 * blocks per SM as fit, in full, beside the running ones (their registers,
 * threads and shared memory added up against the SM's limits; a job started
 * alone leaves one block per SM for the next).
 * A request completes when its own grid has converged, not when its job's
 * largest one has, wherever the job runs one round-free pass with cells of 8
 * or more (the built-in form of every HCM and HCM_LSM job; not FHCM, FMSM,
 * bucketed rounds or two-pass FP32_REFINE):
 * the kernel flags each finished instance in host memory and the server
 * writes that request's output and completes its ticket while the job goes
 * on.  Other jobs complete all their requests together.
 * Results do not depend on the mix: each instance has its own queue and
 * arrays (Theorem convergence makes the result schedule-independent up to
 * rounding).
 *
 * eik_server_create: max_inflight bounds requests submitted but not yet
 * polled to completion (<= 0: 64).  cuda_stream: NULL, or the stream on
 * which the caller produces request inputs -- each request then waits for the
 * work queued on it before submission.  EIK_EINVAL for a zero budget. */
typedef struct eik_server_s* eik_server;
int eik_server_create(eik_server* out, size_t hbm_budget_bytes, int32_t max_inflight,
                      void* cuda_stream);

/* Queue one request and return at once with a ticket.  The descriptor is
 * copied; the instance's buffers must stay valid until eik_poll returns a
 * final status for the ticket.  EIK_EBUSY: the request alone exceeds the
 * budget, or max_inflight requests are pending.  EIK_EINVAL: bad arguments. */
int eik_submit(eik_server s, const eik_plan_desc* d, const eik_instance* in, uint64_t* ticket);

/* Non-blocking: EIK_EAGAIN while the request is pending; otherwise its final
 * status (st, if not NULL, filled; st->ms is the time from its job's launch
 * to the request's completion: device time of the job where all requests
 * complete together, host clock where each completes on its own).  A ticket
 * is polled to completion once; later polls and unknown tickets return
 * EIK_EINVAL. */
int eik_poll(eik_server s, uint64_t ticket, eik_stats* st);

/* Finish every queued request, then release the server.  NULL is ignored. */
void eik_server_destroy(eik_server s);

/* ------------------------------------------------------- no-allocation solve
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot call cudaMalloc: code that runs where device memory is already owned
 * by another allocator (a framework's caching allocator or a fixed memory
 * budget), or latency-critical loops that cannot afford the implicit device
 * synchronisation of an allocation.
 *
 * eik_solve_noalloc solves one FP64 instance (d->precision must be EIK_FP64,
 * d->method EIK_METHOD_HCM) like eik_plan_create + eik_solve +
 * eik_plan_destroy, but allocates nothing, on the device or on the host: the
 * whole workspace lives in one fixed device array of
 * EIK_NOALLOC_SCRATCH_BYTES inside this library, which every GPU that loads
 * the library holds until the process exits.
 *   - in->F and in->U must be device pointers of the current device
 *     (EIK_EINVAL otherwise); the caller still owns and passes all inputs and
 *     outputs.
 *   - at most EIK_NOALLOC_MAX_SOURCES sources (host or device pointers; device
 *     tables are read in cuda_stream's order).
 *   - a grid whose workspace does not fit the fixed array (about 1000 x 1000
 *     nodes at k = 8) is rejected with EIK_EINVAL.
 *   - it always runs the bucketed-rounds schedule (the round-free schedules'
 *     queues would need more scratch), in one wide bucket unless
 *     d->bucket_width sets one; d->schedule is not used.
 *   - the call copies through stack buffers and waits on its stream, so it
 *     cannot be called while cuda_stream is being captured (EIK_EINVAL).
 *   - the first call on a device looks up that device's copy of the array.
 *   - every call shares the one array: calls that overlap on a GPU (different
 *     streams or threads) race and corrupt each other; serialise them.
 *   - work is queued on cuda_stream (NULL: the legacy default stream); the
 *     call returns when U is written.  st->ms is host wall time of the call. */
#define EIK_NOALLOC_SCRATCH_BYTES (32u << 20)
#define EIK_NOALLOC_MAX_SOURCES 256
int eik_solve_noalloc(const eik_plan_desc* d, const eik_instance* in, eik_stats* st,
                      void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* EIK_H */
