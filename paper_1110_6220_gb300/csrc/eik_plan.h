// eik_plan.h -- host-side structures shared by the single-solve, batch and
// serving entry points.  Internal: not part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "eik_common.cuh"

namespace eik {

// Padded device layout of one instance (see SolveParams in eik_common.cuh).
struct Layout {
    int nx, ny, k;
    int cxn, cyn, J;
    int nxp, nyp;
    int upitch, urows;  // U arrays: urows x upitch elements
    int fpitch, frows;  // f arrays: frows x fpitch elements
};

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

// Device workspace of one instance (arrays of the other precision mode null).
struct Workspace {
    Layout L;
    bool fp32;
    double* U64;   // FP64 mode
    double* f64;
    float* U32;    // FP32 + refinement: FP32 pass
    float* f32;
    float2* Udf;   // FP32 + refinement: double-float refinement pass
    float2* fdf;
    double* Fstage;  // device copy of a host F; also the output staging buffer
    unsigned long long* cval;
    int* qflag;
    int* visits;
    unsigned char* has_src;
    int* lists;
    Ctl* ctl;          // [0] FP32 pass, [1] FP64 or refinement pass
    ResidualOut* res;  // follows ctl[1]
    CUtensorMap tmU64, tmF64, tmU32, tmF32, tmUdf, tmFdf;
};

struct HostSources {
    std::vector<int> node;                     // unique source nodes, j*nx + i
    std::vector<double> q;                     // min q per node
    std::vector<int> cell;                     // cells that hold sources
    std::vector<unsigned long long> cell_key;  // key(max q) per such cell
    double q_min = 0.0;
};

struct SrcDev {
    DevBuf buf;
};

// Device copies of the prepared source tables (see HostSources).
struct SrcTables {
    int* node;
    double* q;
    int* cell;
    unsigned long long* cell_key;
    int nsrc, ncell;
};
size_t src_table_bytes(size_t nsrc, size_t ncell);
SrcTables carve_src_tables(void* base, size_t nsrc, size_t ncell);

bool desc_valid(const eik_plan_desc* d);
int default_k(const eik_plan_desc* d);
Layout make_layout(int nx, int ny, int k);
size_t layout_bytes(const Layout& L, bool fp32);
int workspace_alloc(Workspace* w, const Layout& L, bool fp32, cudaStream_t st);
void workspace_free(Workspace* w);
int prepare_sources(const Layout& L, const eik_instance* in, HostSources* hs);
bool is_device_ptr(const void* p);
int grow_staging(DevBuf* b, size_t bytes);
// Pass timing events (may be null): ev[0..1] around the FP32 pass, ev[2..3]
// around the FP64 pass.  *launches counts the kernels queued.
int enqueue_solve(Workspace* w, const eik_plan_desc* d, const double* Fdev, const HostSources& hs,
                  SrcDev* sd, int num_sms, cudaStream_t st, cudaEvent_t* ev, int* launches);
// The same, with the source tables already on the device.
int enqueue_solve_tables(Workspace* w, const eik_plan_desc* d, const double* Fdev, const SrcTables& t,
                         int num_sms, cudaStream_t st, cudaEvent_t* ev, int* launches);
bool make_map(CUtensorMap* tm, void* base, bool fp64, int width, int rows, int pitch_elems,
              int box_w, int box_h);
void finish_stats(const Layout& L, const eik_plan_desc* d, const Ctl* c32, const Ctl* c64,
                  const ResidualOut* r, double q_min, bool fp32, double ms, eik_stats* st);

}  // namespace eik

struct eik_plan_s {
    eik_plan_desc d;
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    eik::Workspace ws{};
    eik::SrcDev src;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t pev[4] = {nullptr, nullptr, nullptr, nullptr};
    void* host_ctl = nullptr;  // pinned copy of ctl[2] + residual
};
