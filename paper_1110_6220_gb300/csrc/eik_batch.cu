// eik_batch.cu -- eik_batch_create / eik_batch_run / eik_batch_destroy: a
// fixed batch of instances solved repeatedly.  Layouts, tables, sources and
// device workspace are built once; the launch sequence of each job (memsets,
// the node-wise kernels and the persistent passes) is captured in a CUDA
// graph on the batch's own stream and replayed by each run, so a run costs
// the device time plus one graph launch and the result read-back.
#include <map>
#include <new>
#include <vector>

#include "eik_common.cuh"
#include "eik_plan.h"

using namespace eik;

namespace {

struct Group {
    std::vector<int> idx;              // positions in the caller's arrays
    std::vector<eik_plan_desc> d;
    std::vector<eik_instance> in;
    JobParams P{};
    bool fp32 = false;
    HostJob job;
    cudaEvent_t ev[2] = {};           // around each run (outside the graph)
    cudaGraphExec_t exec = nullptr;   // null: runs enqueue the job directly
    int launches = 0;
};

}  // namespace

struct eik_batch_s {
    int device = 0;
    int num_sms = 0;
    int n = 0;
    cudaStream_t stream = nullptr;  // own: capture and runs
    cudaStream_t user = nullptr;    // the caller's stream, or null
    cudaEvent_t order = nullptr;    // runs start after the work queued on `user`
    std::vector<Group*> groups;
};

namespace {

void destroy_group(Group* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    free_job(&g->job);
    for (auto& e : g->ev)
        if (e) cudaEventDestroy(e);
    delete g;
}

// Queue one run of the job (the events around it are recorded outside, so
// that a captured graph holds only the work; pass times come from the
// kernels' own timers).
int enqueue_run(eik_batch_s* b, Group* g, int* nl) {
    return enqueue_job(g->job.j, b->num_sms, b->stream, nullptr, nl);
}

// Capture the run into a graph; on any failure the group runs uncaptured.
void capture(eik_batch_s* b, Group* g) {
    cudaGraph_t graph = nullptr;
    int nl = 0;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const int rc = enqueue_run(b, g, &nl);
    const cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
    if (rc || ce != cudaSuccess || !graph) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        return;
    }
    if (cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        g->exec = nullptr;
    }
    cudaGraphDestroy(graph);
    g->launches = nl;
}

}  // namespace

extern "C" int eik_batch_create(eik_batch* out, const eik_plan_desc* d, const eik_instance* in, int32_t n_inst,
                                void* cuda_stream) {
    if (!out) return EIK_EINVAL;
    *out = nullptr;
    if (n_inst < 1 || !d || !in) return EIK_EINVAL;
    for (int i = 0; i < n_inst; ++i)
        if (!desc_valid(&d[i]) || !in[i].F || !in[i].U || in[i].nsrc < 0) return EIK_EINVAL;
    eik_batch_s* b = new (std::nothrow) eik_batch_s();
    if (!b) return EIK_ENOMEM;
    b->n = n_inst;
    b->user = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->order, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        eik_batch_destroy(b);
        return EIK_ECUDA;
    }
    if (b->user) {
        cudaEventRecord(b->order, b->user);
        cudaStreamWaitEvent(b->stream, b->order, 0);
    }
    // groups as eik_solve_batch forms them: (cell_k as given, precision), at
    // most MAX_BATCH instances per job
    std::map<std::pair<int, int>, std::vector<int>> by;
    for (int i = 0; i < n_inst; ++i) by[{d[i].cell_k, d[i].precision + 2 * d[i].method}].push_back(i);
    int rc = EIK_OK;
    for (auto& kv : by) {
        const std::vector<int>& idx = kv.second;
        for (size_t b0 = 0; b0 < idx.size() && !rc; b0 += MAX_BATCH) {
            Group* g = new (std::nothrow) Group();
            if (!g) {
                rc = EIK_ENOMEM;
                break;
            }
            b->groups.push_back(g);
            const size_t m = std::min<size_t>(MAX_BATCH, idx.size() - b0);
            g->idx.assign(idx.begin() + b0, idx.begin() + b0 + m);
            for (int i : g->idx) {
                g->d.push_back(d[i]);
                g->in.push_back(in[i]);
            }
            g->P = choose_params(g->d.data(), (int)m);
            for (auto& x : g->d) x.cell_k = g->P.k;
            g->fp32 = kv.first.second % 2 == EIK_FP32_REFINE;
            for (auto& e : g->ev)
                if (cudaEventCreate(&e) != cudaSuccess) rc = EIK_ECUDA;
            if (!rc)
                rc = build_job(&g->job, (int)m, g->d.data(), g->in.data(), g->P, g->fp32, d[0].deadline_ns,
                               b->stream);
            if (!rc && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = EIK_ECUDA;
            if (!rc) capture(b, g);
        }
        if (rc) break;
    }
    if (rc) {
        cudaGetLastError();
        eik_batch_destroy(b);
        return rc;
    }
    *out = b;
    return EIK_OK;
}

extern "C" int eik_batch_run(eik_batch b, eik_stats* st) {
    if (!b) return EIK_EINVAL;
    cudaSetDevice(b->device);
    if (b->user) {
        cudaEventRecord(b->order, b->user);
        cudaStreamWaitEvent(b->stream, b->order, 0);
    }
    int first_err = EIK_OK;
    std::vector<eik_stats> gs;
    for (Group* g : b->groups) {
        const int m = (int)g->idx.size();
        int rc = EIK_OK;
        // speeds given in host memory are copied in again: their values may change
        for (int e = 0; e < m && !rc; ++e)
            if (g->job.arr[e].Fstage &&
                cudaMemcpyAsync(g->job.arr[e].Fstage, g->in[e].F, (size_t)g->d[e].nx * g->d[e].ny * 8,
                                cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
                rc = EIK_ECUDA;
        int nl = g->launches;
        if (!rc) {
            cudaEventRecord(g->ev[0], b->stream);
            if (g->exec) {
                if (cudaGraphLaunch(g->exec, b->stream) != cudaSuccess) rc = EIK_ECUDA;
            } else {
                rc = enqueue_run(b, g, &nl);
            }
            cudaEventRecord(g->ev[1], b->stream);
        }
        gs.assign(m, eik_stats{});
        if (!rc) rc = finish_job(&g->job, g->d.data(), b->stream, 0.0, gs.data());
        else {
            cudaStreamSynchronize(b->stream);
            cudaGetLastError();
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g->ev[0], g->ev[1]);
        cudaGetLastError();
        for (int e = 0; e < m; ++e) {
            gs[e].ms = ms;
            gs[e].mpts_per_s = ms > 0 ? (double)g->d[e].nx * g->d[e].ny / ms / 1000.0 : 0.0;
            gs[e].launches = nl;
            if (g->exec) gs[e].schedule |= 8;
            if (st) st[g->idx[e]] = gs[e];
        }
        if (rc && !first_err) first_err = rc;
    }
    return first_err;
}

extern "C" void eik_batch_destroy(eik_batch b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (Group* g : b->groups) destroy_group(g);
    if (b->order) cudaEventDestroy(b->order);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}
