// eik_server.cu -- eik_server_create / eik_submit / eik_poll /
// eik_server_destroy: a request loop with HBM admission and continuous
// batching.
//
// A server thread keeps a FIFO of submitted requests and JOB_SLOTS job slots,
// each with its own stream, arena and events.  Whenever a slot is free it
// takes the oldest waiting requests of one (cell size, precision) class that
// fit the memory budget left by the other slots, and launches them as one
// batched job (eik_job.h) with as many blocks per SM as fit beside the jobs
// already running, so that a job built from requests that arrived while
// others run overlaps them on the device.
//
// Completion is per request where the job's persistent pass supports it
// (round-free, cells of 8 or more, one pass): each instance counts its
// requested and running cells, and the cell whose finish brings the count to
// zero sets the instance's flag in mapped host memory.  The loop polls the
// flags and, for each newly finished instance, queues its node-wise output
// kernel, the copy of a host U and the read-back of its counters on the
// slot's second stream; when that work's event has completed the ticket is
// done, while the job's launch may still be running for its other requests.
// A job's blocks leave the co-residency account as soon as its launches end.
// Other jobs (rounds, FMSM, two passes) complete all their requests together
// when the job's last event has completed.  Nothing blocks the loop.
//
// Co-residency: a persistent job's blocks wait for one another, so two of
// them must never hold parts of the SMs the other needs.  Each job's
// per-block resources (threads, registers as allocated per warp, shared
// memory with the SM's per-block reserve) are added up against the SM's
// limits over all running jobs, and a job takes only the blocks per SM that
// fit in full (a job started alone leaves one block per SM free for the next
// one).  A job whose resources are unknown runs alone.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "eik_common.cuh"
#include "eik_plan.h"

using namespace eik;

namespace {

constexpr int JOB_SLOTS = 4;

struct Request {
    uint64_t ticket;
    eik_plan_desc d;
    eik_instance in;
    size_t bytes;       // device workspace estimate
    cudaEvent_t ready = nullptr;  // inputs ready on the caller's stream
    int state = 0;      // 0 waiting, 1 running, 2 done
    eik_stats st{};
    int rc = EIK_EAGAIN;
};

// what a request's finishing work reads back: its instance's control block
// of the main pass, its residual, and the launch-wide control block
constexpr size_t FIN_REC = sizeof(Ctl) * 2 + sizeof(ResidualOut);

struct Slot {
    cudaStream_t stream = nullptr;
    cudaStream_t out = nullptr;  // per-request finishing work, beside the job's launches
    cudaEvent_t ev[6] = {};
    HostJob job;
    std::vector<Request*> reqs;
    std::vector<eik_plan_desc> descs;
    std::vector<eik_instance> insts;
    size_t bytes = 0;   // budget held while running
    bool busy = false;
    bool main_done = false;  // the job's launches have finished
    Footprint fp;       // per-block resources of the job's persistent launches
    int cap = 0;        // blocks per SM it holds; 0: alone at its full occupancy
    // per-instance completion: the job's done flags (mapped host memory), per
    // request 0 running / 1 finishing / 2 complete, the finishing work's event
    unsigned* done_h = nullptr;
    unsigned* done_d = nullptr;
    char* pin = nullptr;  // MAX_BATCH records of FIN_REC bytes (pinned)
    std::vector<int> fin;
    std::vector<cudaEvent_t> fev;
    // the requests still open when the job's launches ended, finished
    // together: their records come from the job's whole read-back
    std::vector<char> in_all;
    cudaEvent_t fev_all = nullptr;
    // the requests in the order their finishing work was queued on `out`:
    // their events complete in that order, so the loop queries only the
    // oldest one still pending
    std::vector<int> fin_order;
    size_t fin_head = 0;
    std::chrono::steady_clock::time_point t0;
};

}  // namespace

struct eik_server_s {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;
    int max_inflight = 64;
    // one SM's limits, for the co-residency of jobs
    int sm_threads = 0, sm_regs = 0, sm_blocks = 0;
    size_t sm_smem = 0;
    cudaStream_t user_stream = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> waiting;
    std::map<uint64_t, Request*> all;
    uint64_t next_ticket = 1;
    int inflight = 0;
    bool stop = false;
    bool blocked = false;  // the head job waits for the other slot to drain
    Slot slots[JOB_SLOTS];
    std::thread worker;
};

namespace {

size_t request_bytes(const eik_plan_desc& d, const eik_instance& in) {
    const bool fp32 = d.precision == EIK_FP32_REFINE;
    const bool sF = !is_device_ptr(in.F), sU = !is_device_ptr(in.U);
    // arrays + staging for host buffers + cell state, lists, rings (the
    // value-ordered schedule's bucket rings: NBQ words per cell, up to twice
    // that once the job's cells round up to a power of two) and tables; a
    // request that leaves the cell size open is charged its largest choice
    size_t most = 0;
    const size_t per_cell = 160 + 2 * NBQ * 8;
    for (int k : {8, 16, 32}) {
        if (d.cell_k && k != d.cell_k) continue;
        const Layout L = make_layout(d.nx, d.ny, k);
        most = std::max(most, inst_bytes(L, fp32, sF, sU) + (size_t)L.J * per_cell);
    }
    if (d.cell_k && !most) {
        const Layout L = make_layout(d.nx, d.ny, d.cell_k);
        most = inst_bytes(L, fp32, sF, sU) + (size_t)L.J * per_cell;
    }
    return most + 4 * sizeof(Ctl) + 4096;
}

// Finish a slot whose job has completed (called with the lock held).
void complete_slot(eik_server_s* s, Slot& sl) {
    std::vector<eik_stats> st(sl.reqs.size());
    int rc = finish_job(&sl.job, sl.descs.data(), sl.stream, 0.0, st.data());
    float ms = 0.f, p0 = 0.f, p1 = 0.f;
    cudaEventElapsedTime(&ms, sl.ev[0], sl.ev[1]);
    cudaEventElapsedTime(&p0, sl.ev[2], sl.ev[3]);
    cudaEventElapsedTime(&p1, sl.ev[4], sl.ev[5]);
    for (size_t e = 0; e < sl.reqs.size(); ++e) {
        Request* r = sl.reqs[e];
        r->st = st[e];
        r->st.ms = ms;
        r->st.mpts_per_s = ms > 0 ? (double)r->d.nx * r->d.ny / ms / 1000.0 : 0.0;
        r->st.pass_ms[0] = sl.descs[e].precision == EIK_FP32_REFINE ? p0 : 0.0;
        r->st.pass_ms[1] = p1;
        r->rc = rc == EIK_ECUDA ? rc : r->st.status;
        r->state = 2;
        --s->inflight;
    }
    sl.reqs.clear();
    sl.busy = false;
    sl.bytes = 0;
}

// Per-instance completion: queue request e's finishing work on the slot's
// second stream -- the node-wise kernel that certifies and writes its
// output, the copy of a host U, and the read-back of its control block and
// residual.  Called only while the job's launches run (requests still open
// when they end are finished together, in advance_slot), so the launch-wide
// block's record stays zero.
void start_finish(Slot& sl, int e) {
    HostJob& hj = sl.job;
    const int n = hj.j.n;
    char* rec = sl.pin + (size_t)e * FIN_REC;
    int rc = finish_instance(hj.j, e, hj.L[e], sl.out);
    if (!rc && hj.out_host[e] &&
        cudaMemcpyAsync(hj.out_user[e], hj.arr[e].Ostage, (size_t)hj.L[e].nx * hj.L[e].ny * 8,
                        cudaMemcpyDeviceToHost, sl.out) != cudaSuccess)
        rc = EIK_ECUDA;
    cudaMemcpyAsync(rec, hj.j.ictl + n + e, sizeof(Ctl), cudaMemcpyDeviceToHost, sl.out);
    cudaMemcpyAsync(rec + sizeof(Ctl), hj.j.res + e, sizeof(ResidualOut), cudaMemcpyDeviceToHost, sl.out);
    std::memset(rec + sizeof(Ctl) + sizeof(ResidualOut), 0, sizeof(Ctl));
    if (rc) cudaGetLastError();
    cudaEventRecord(sl.fev[e], sl.out);
    sl.fin[e] = 1;
    sl.fin_order.push_back(e);
}

// Request e's finishing work is done: its statistics, its ticket.
void complete_request(eik_server_s* s, Slot& sl, int e) {
    HostJob& hj = sl.job;
    const char* rec = sl.pin + (size_t)e * FIN_REC;
    Ctl zero;
    std::memset((void*)&zero, 0, sizeof(zero));
    const Ctl* ic = (const Ctl*)rec;
    const ResidualOut* r = (const ResidualOut*)(rec + sizeof(Ctl));
    const Ctl* g = (const Ctl*)(rec + sizeof(Ctl) + sizeof(ResidualOut));
    if (sl.in_all[e]) {
        // the job's read-back: 2n instance blocks, 2 launch blocks, n residuals
        const int n = hj.j.n;
        const Ctl* base = (const Ctl*)hj.zero_host;
        ic = base + n + e;
        g = base + 2 * n + 1;
        r = (const ResidualOut*)(base + 2 * n + 2) + e;
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - sl.t0).count();
    eik_stats st;
    job_stats(hj.L[e], &sl.descs[e], hj.j.fp32, &zero, ic, &zero, g, r, hj.shift[e], hj.bw_main[e], ms, &st);
    st.schedule = (hj.j.async_main && hj.j.k >= 8 ? 2 : 0) | (hj.j.one_pass ? 4 : 0) |
                  (hj.j.ordered && hj.j.variant == VAR_HCM ? 32 : 0);
    st.pass_ms[0] = 0.0;
    st.pass_ms[1] = ms;
    Request* req = sl.reqs[e];
    req->st = st;
    req->rc = st.status;
    req->state = 2;
    --s->inflight;
    sl.fin[e] = 2;
}

// Advance a busy slot whose job reports per-instance completion; true when
// something happened.  The slot frees once every request is complete.
bool advance_slot(eik_server_s* s, Slot& sl) {
    bool progressed = false;
    if (!sl.main_done && cudaEventQuery(sl.ev[1]) == cudaSuccess) {
        sl.main_done = true;  // its SM blocks are free for other jobs
        progressed = true;
    }
    const int n = (int)sl.reqs.size();
    if (sl.main_done) {
        // the requests not yet finished: one node-wise launch over the job
        // and one read-back of its counters, after the single ones queued
        // before on the same stream
        HostJob& hj = sl.job;
        int open = 0;
        for (int e = 0; e < n; ++e) open += sl.fin[e] == 0;
        if (open) {
            int rc = finish_instances(hj.j, sl.out);
            for (int e = 0; e < n; ++e) {
                if (sl.fin[e] != 0) continue;
                if (!rc && hj.out_host[e] &&
                    cudaMemcpyAsync(hj.out_user[e], hj.arr[e].Ostage, (size_t)hj.L[e].nx * hj.L[e].ny * 8,
                                    cudaMemcpyDeviceToHost, sl.out) != cudaSuccess)
                    rc = EIK_ECUDA;
            }
            cudaMemcpyAsync(hj.zero_host, hj.j.zero_base,
                            (size_t)(2 * n + 2) * sizeof(Ctl) + (size_t)n * sizeof(ResidualOut),
                            cudaMemcpyDeviceToHost, sl.out);
            if (rc) cudaGetLastError();
            cudaEventRecord(sl.fev_all, sl.out);
            for (int e = 0; e < n; ++e)
                if (sl.fin[e] == 0) {
                    sl.fin[e] = 1;
                    sl.in_all[e] = 1;
                    sl.fin_order.push_back(e);
                }
            progressed = true;
        }
    }
    if (!sl.main_done)
        for (int e = 0; e < n; ++e)
            if (sl.fin[e] == 0 && *(volatile unsigned*)(sl.done_h + e)) {
                start_finish(sl, e);
                progressed = true;
            }
    while (sl.fin_head < sl.fin_order.size()) {
        const int e = sl.fin_order[sl.fin_head];
        if (cudaEventQuery(sl.in_all[e] ? sl.fev_all : sl.fev[e]) != cudaSuccess) break;
        complete_request(s, sl, e);
        ++sl.fin_head;
        progressed = true;
    }
    if (sl.fin_head == (size_t)n && sl.main_done) {
        sl.reqs.clear();
        sl.busy = false;
        sl.bytes = 0;
        progressed = true;
    }
    return progressed;
}

// Launch the oldest admissible waiting requests on a free slot (lock held;
// the CUDA calls happen with the lock released by the caller's structure:
// build and enqueue are quick and non-blocking apart from small copies).
bool launch_slot(eik_server_s* s, Slot& sl, size_t held_by_others) {
    if (s->waiting.empty()) return false;
    const Request* head = s->waiting.front();
    const int kreq = head->d.cell_k;  // 0: chosen for the job
    const int prec = head->d.precision;
    // a job lasts about as long as its largest grid: a request joins the
    // head's job unless its grid is more than a size class larger than the
    // head's, so that a small head is not held behind large grids while a
    // large head still takes the small requests along
    auto size_class = [](const eik_plan_desc& d) {
        return (int)std::lround(0.5 * std::log2((double)d.nx * d.ny));
    };
    const int scls = size_class(head->d);
    size_t bytes = 0;
    sl.reqs.clear();
    for (auto it = s->waiting.begin(); it != s->waiting.end() && (int)sl.reqs.size() < MAX_BATCH;) {
        Request* r = *it;
        if (r->d.cell_k == kreq && r->d.precision == prec && r->d.method == head->d.method &&
            size_class(r->d) <= scls + 1) {
            if (held_by_others + bytes + r->bytes > s->budget) break;  // keep FIFO order
            bytes += r->bytes;
            sl.reqs.push_back(r);
            it = s->waiting.erase(it);
        } else {
            ++it;
        }
    }
    if (sl.reqs.empty()) return false;
    sl.descs.resize(sl.reqs.size());
    sl.insts.resize(sl.reqs.size());
    for (size_t e = 0; e < sl.reqs.size(); ++e) {
        sl.descs[e] = sl.reqs[e]->d;
        sl.insts[e] = sl.reqs[e]->in;
        sl.reqs[e]->state = 1;
    }
    const JobParams P = choose_params(sl.descs.data(), (int)sl.descs.size());
    for (auto& dd : sl.descs) dd.cell_k = P.k;
    // blocks per SM for this job beside the running ones (see the top of
    // this file); -1: wait until they finish
    const bool fp32 = prec == EIK_FP32_REFINE;
    const int method = head->d.method;
    const int variant = method == EIK_METHOD_FHCM ? VAR_FHCM : method == EIK_METHOD_HCM_LSM ? VAR_LSM : VAR_HCM;
    Footprint fp;
    const bool known = method != EIK_METHOD_FMSM &&
                       job_footprint(probe_job((int)sl.reqs.size(), P.k, fp32, P.one_pass, P.async_first,
                                               P.async_main, P.ordered && P.async_main && P.k >= 8, variant),
                                     s->num_sms, &fp);
    int used_threads = 0, used_regs = 0, used_blocks = 0;
    size_t used_smem = 0;
    bool any_other = false, other_alone = false;
    for (const Slot& o : s->slots) {
        if (&o == &sl || !o.busy || o.main_done) continue;  // only launches still on the SMs
        any_other = true;
        if (o.cap <= 0) other_alone = true;
        used_threads += o.cap * o.fp.threads;
        used_regs += o.cap * o.fp.regs;
        used_smem += (size_t)o.cap * o.fp.smem;
        used_blocks += o.cap;
    }
    int cap = -1;
    if (!known) {
        cap = any_other ? -1 : 0;
    } else if (!other_alone) {
        int c = fp.per_sm;
        for (; c >= 1; --c)
            if (used_threads + c * fp.threads <= s->sm_threads && used_regs + c * fp.regs <= s->sm_regs &&
                used_smem + (size_t)c * fp.smem <= s->sm_smem && used_blocks + c <= s->sm_blocks)
                break;
        cap = c >= 1 ? c : -1;
        if (cap > 1 && !any_other && cap == fp.per_sm) cap -= 1;  // a block per SM for the next job
    }
    if (cap < 0) {
        // keep the requests at the head of the queue, in order
        for (auto it = sl.reqs.rbegin(); it != sl.reqs.rend(); ++it) {
            (*it)->state = 0;
            s->waiting.push_front(*it);
        }
        sl.reqs.clear();
        s->blocked = true;
        return false;
    }
    for (Request* r : sl.reqs)
        if (r->ready) cudaStreamWaitEvent(sl.stream, r->ready, 0);
    // per-instance completion: fresh flags (no launch of this slot runs now)
    const int n = (int)sl.reqs.size();
    std::memset(sl.done_h, 0, (size_t)n * sizeof(unsigned));
    sl.job.done_dev = sl.done_d;
    sl.fin.assign(n, 0);
    sl.in_all.assign(n, 0);
    sl.fin_order.clear();
    sl.fin_head = 0;
    sl.main_done = false;
    while ((int)sl.fev.size() < n) {
        cudaEvent_t e = nullptr;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        sl.fev.push_back(e);
    }
    sl.t0 = std::chrono::steady_clock::now();
    int rc = build_job(&sl.job, n, sl.descs.data(), sl.insts.data(), P, prec == EIK_FP32_REFINE,
                       head->d.deadline_ns, sl.stream);
    if (!rc) {
        sl.job.j.sm_cap = cap;
        sl.cap = cap;
        sl.fp = fp;
        cudaEventRecord(sl.ev[0], sl.stream);
        int nl = 0;
        rc = enqueue_job(sl.job.j, s->num_sms, sl.stream, sl.ev + 2, &nl);
        cudaEventRecord(sl.ev[1], sl.stream);
    }
    if (rc) {
        cudaStreamSynchronize(sl.stream);
        cudaGetLastError();
        for (Request* r : sl.reqs) {
            r->rc = rc;
            r->st.status = rc;
            r->state = 2;
            --s->inflight;
        }
        sl.reqs.clear();
        return true;
    }
    sl.busy = true;
    sl.bytes = bytes;
    return true;
}

void server_loop(eik_server_s* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        bool progressed = false;
        for (Slot& sl : s->slots) {
            if (!sl.busy) continue;
            if (sl.job.j.inst_done) {
                if (advance_slot(s, sl)) progressed = true;
            } else if (cudaEventQuery(sl.ev[1]) == cudaSuccess) {
                complete_slot(s, sl);
                progressed = true;
            }
        }
        for (int i = 0; i < JOB_SLOTS; ++i) {
            Slot& sl = s->slots[i];
            if (sl.busy || s->waiting.empty() || (s->blocked && !progressed)) continue;
            s->blocked = false;
            size_t others = 0;
            for (int o = 0; o < JOB_SLOTS; ++o)
                if (o != i && s->slots[o].busy) others += s->slots[o].bytes;
            if (launch_slot(s, sl, others)) progressed = true;
        }
        bool any_busy = false;
        for (Slot& sl : s->slots) any_busy |= sl.busy;
        if (s->stop && s->waiting.empty() && !any_busy) break;
        if (!progressed) {
            // poll running jobs every 50 us; sleep until woken when idle
            if (any_busy) s->cv.wait_for(lock, std::chrono::microseconds(50));
            else s->cv.wait_for(lock, std::chrono::milliseconds(50));
        }
    }
}

}  // namespace

extern "C" int eik_server_create(eik_server* out, size_t hbm_budget_bytes, int32_t max_inflight,
                                 void* cuda_stream) {
    if (!out) return EIK_EINVAL;
    *out = nullptr;
    if (hbm_budget_bytes == 0) return EIK_EINVAL;
    eik_server_s* s = new (std::nothrow) eik_server_s();
    if (!s) return EIK_ENOMEM;
    s->budget = hbm_budget_bytes;
    s->max_inflight = max_inflight > 0 ? max_inflight : 64;
    s->user_stream = (cudaStream_t)cuda_stream;
    int smem = 0;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sm_threads, cudaDevAttrMaxThreadsPerMultiProcessor, s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sm_blocks, cudaDevAttrMaxBlocksPerMultiprocessor, s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return EIK_ECUDA;
    }
    s->sm_smem = (size_t)smem;
    for (Slot& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&sl.out, cudaStreamNonBlocking) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.done_h, MAX_BATCH * sizeof(unsigned), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer((void**)&sl.done_d, sl.done_h, 0) != cudaSuccess ||
            cudaMallocHost((void**)&sl.pin, MAX_BATCH * FIN_REC) != cudaSuccess) {
            cudaGetLastError();
            eik_server_destroy(s);
            return EIK_ECUDA;
        }
        for (auto& e : sl.ev) cudaEventCreate(&e);
        cudaEventCreateWithFlags(&sl.fev_all, cudaEventDisableTiming);
    }
    try {
        s->worker = std::thread(server_loop, s);
    } catch (...) {
        eik_server_destroy(s);
        return EIK_ENOMEM;
    }
    *out = s;
    return EIK_OK;
}

extern "C" int eik_submit(eik_server s, const eik_plan_desc* d, const eik_instance* in,
                          uint64_t* ticket) {
    if (!s || !d || !in || !ticket || !desc_valid(d) || !in->F || !in->U || in->nsrc < 0) return EIK_EINVAL;
    Request* r = new (std::nothrow) Request();
    if (!r) return EIK_ENOMEM;
    r->d = *d;
    r->in = *in;
    r->bytes = request_bytes(*d, *in);
    if (r->bytes > s->budget) {
        delete r;
        return EIK_EBUSY;
    }
    if (s->user_stream) {
        // the job that serves this request waits for the caller's stream
        if (cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(r->ready, s->user_stream) != cudaSuccess) {
            cudaGetLastError();
            if (r->ready) cudaEventDestroy(r->ready);
            delete r;
            return EIK_ECUDA;
        }
    }
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) {
            delete r;
            return EIK_EINVAL;
        }
        if (s->inflight >= s->max_inflight) {
            delete r;
            return EIK_EBUSY;
        }
        r->ticket = s->next_ticket++;
        s->all[r->ticket] = r;
        s->waiting.push_back(r);
        ++s->inflight;
        *ticket = r->ticket;
    }
    s->cv.notify_all();
    return EIK_OK;
}

extern "C" int eik_poll(eik_server s, uint64_t ticket, eik_stats* st) {
    if (!s) return EIK_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return EIK_EINVAL;
    Request* r = it->second;
    if (r->state != 2) return EIK_EAGAIN;
    if (st) *st = r->st;
    const int rc = r->rc;
    s->all.erase(it);
    if (r->ready) cudaEventDestroy(r->ready);
    delete r;
    return rc;
}

extern "C" void eik_server_destroy(eik_server s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.out) cudaStreamSynchronize(sl.out);
        free_job(&sl.job);
        for (auto& e : sl.ev)
            if (e) cudaEventDestroy(e);
        for (auto& e : sl.fev)
            if (e) cudaEventDestroy(e);
        if (sl.fev_all) cudaEventDestroy(sl.fev_all);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.out) cudaStreamDestroy(sl.out);
        if (sl.done_h) cudaFreeHost(sl.done_h);
        if (sl.pin) cudaFreeHost(sl.pin);
    }
    for (auto& kv : s->all) {
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
        delete kv.second;
    }
    delete s;
}
