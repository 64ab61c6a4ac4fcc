// eik_plan.h -- host-side structures shared by the single-solve, batch,
// no-allocation and serving entry points.  Internal: not part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "eik_common.cuh"
#include "eik_job.h"

namespace eik {

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct HostSources {
    std::vector<int> node;                     // unique source nodes, j*nx + i
    std::vector<double> q;                     // min q per node, minus q_min
    std::vector<int> cell;                     // cells that hold sources
    std::vector<unsigned long long> cell_key;  // key(max q) per such cell
    double q_min = 0.0;
};

// Cell size and bucket widths of a job.  Widths follow eik_plan_desc's
// convention: > 0 absolute, < 0 relative (|w| * k * min(h/F)).  w_first is
// the FP32 pass of FP32_REFINE, w_main the FP64 or refinement pass.
struct JobParams {
    int k;
    double w_first, w_main;
    bool async_first = false, async_main = false;  // round-free schedule per pass (k >= 8)
    bool one_pass = false;  // FP32_REFINE as one double-float pass from the sources
    unsigned hold_ns = 0;   // round-free: minimum age of a request before its cell runs
    // round-free main pass in value order (bucket rings, a front and a
    // window of `window` buckets above it; plain HCM) instead of first in,
    // first out
    bool ordered = false;
    int window = 31;
};

bool desc_valid(const eik_plan_desc* d);
// Parameters of a job of n instances of one precision (eik_tune.cu): an
// explicit cell_k wins; otherwise the tuned entry of the job's class, else
// the built-in defaults.  Widths: the table's for the chosen k (an instance
// whose bucket_width is set keeps its own, see build_job).
JobParams choose_params(const eik_plan_desc* d, int n);
int default_k(const eik_plan_desc* d);  // choose_params(d, 1).k
int prepare_sources(const Layout& L, const eik_instance* in, HostSources* hs);
// the same from host copies of the n sources (ij: 2n ints, q: n doubles)
int prepare_sources_host(const Layout& L, int n, const int32_t* ij, const double* q, HostSources* hs);
bool is_device_ptr(const void* p);
int grow(DevBuf* b, size_t bytes);
int profiling();

// A job's device arena and the host image of its tables.
struct HostJob {
    DevBuf arena;
    std::vector<char> image;     // tables + source tables, uploaded in one copy
    JobDev j{};
    std::vector<Layout> L;
    std::vector<InstArrays> arr;
    std::vector<double> shift;   // per instance: min q
    std::vector<char> out_host;  // per instance: U is a host pointer
    std::vector<double*> out_user;
    std::vector<double> bw_main;  // per instance: bucket width of the main pass
    char* zero_host = nullptr;   // readback buffer (pinned) of the zero region
    size_t zero_cap = 0;
    char* src_host = nullptr;    // pinned staging of the instances' sources
    size_t src_cap = 0;
    HostJob* coarse = nullptr;   // FMSM: the job of the coarse grids (owned)
    // per-instance completion: device pointer of n done flags in mapped host
    // memory (set by the caller before build_job; null: the job finishes as a whole)
    unsigned* done_dev = nullptr;
};

// Lay out and upload a job of n instances (one k and precision); descs[i]
// gives nx, ny, h of instance i, and its bucket width if set (else P's).
int build_job(HostJob* hj, int n, const eik_plan_desc* descs, const eik_instance* in, const JobParams& P,
              bool fp32, long long deadline_ns, cudaStream_t st);
// Copy results to host buffers, read back control blocks, fill stats (may be
// null).  Synchronises st.
int finish_job(HostJob* hj, const eik_plan_desc* descs, cudaStream_t st, double ms, eik_stats* st_out);
void free_job(HostJob* hj);

// Build, queue and finish one job on st, timed with ev[6] (whole job, FP32
// pass, main pass).  st_out: null or n entries, each with ms = the job's
// device time.  t: null or {job, FP32 pass, main pass} in ms.
int run_job(HostJob* hj, int n, const eik_plan_desc* descs, const eik_instance* in, const JobParams& P,
            bool fp32, long long deadline_ns, int num_sms, cudaStream_t st, cudaEvent_t* ev,
            eik_stats* st_out, float* t);

}  // namespace eik

struct eik_plan_s {
    eik_plan_desc d;
    eik::JobParams P{};
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    eik::HostJob job;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t pev[4] = {nullptr, nullptr, nullptr, nullptr};
};
