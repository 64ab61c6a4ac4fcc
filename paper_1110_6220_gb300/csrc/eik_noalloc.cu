// eik_noalloc.cu -- eik_solve_noalloc: the FP64 solve of one instance with
// its whole device workspace (padded U and h/F arrays, cell state, work lists,
// control block, source tables) carved out of one fixed file-scope device
// array, so that a call allocates nothing, on the device or on the host.
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <mutex>

#include "eik_common.cuh"
#include "eik_plan.h"

namespace eik {
namespace {

constexpr size_t SCRATCH_BYTES = (size_t)EIK_NOALLOC_SCRATCH_BYTES;
constexpr int MAX_SOURCES = EIK_NOALLOC_MAX_SOURCES;
constexpr int MAX_DEVICES = 64;

// The scratch: one copy per GPU that loads this library, held until exit.
// Every call shares it and it keeps the last call's contents, so each call
// re-initialises everything it reads; calls that overlap on a GPU race.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

std::mutex g_setup_mu;
void* g_scratch_addr[MAX_DEVICES] = {};
int g_num_sms[MAX_DEVICES] = {};

// Once per device, with that device current: the device address of
// g_scratch.  In host code the symbol names a host-side stand-in, never the
// device memory, so kernels and tensor maps get this address instead.
int setup_device(int dev, void** addr, int* sms) {
    if (dev < 0 || dev >= MAX_DEVICES) return EIK_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return EIK_ECUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return EIK_ECUDA;
        }
        g_scratch_addr[dev] = p;
        g_num_sms[dev] = n;
    }
    *addr = g_scratch_addr[dev];
    *sms = g_num_sms[dev];
    return EIK_OK;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Sources on the stack: validate, keep the min q per node, shift by min q,
// and build the per-cell keys of max q (same rules as the plan path).
struct StackSources {
    int node[MAX_SOURCES];
    double q[MAX_SOURCES];
    int cell[MAX_SOURCES];
    unsigned long long key[MAX_SOURCES];
    int n = 0, ncell = 0;
    double q_min = 0.0;
};

int prepare_stack_sources(const Layout& L, const eik_instance* in, cudaStream_t st, StackSources* s) {
    const int n = in->nsrc;
    if (n < 0 || n > MAX_SOURCES) return EIK_EINVAL;
    s->n = s->ncell = 0;
    s->q_min = 0.0;
    if (n == 0) return EIK_OK;
    if (!in->src_ij || !in->src_q) return EIK_EINVAL;
    int32_t ij[2 * MAX_SOURCES];
    double q[MAX_SOURCES];
    // read in the caller's stream order (a table written on that stream just
    // before the call is read after the write), then wait for the copies
    if (cudaMemcpyAsync(ij, in->src_ij, (size_t)n * 8, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemcpyAsync(q, in->src_q, (size_t)n * 8, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return EIK_EINVAL;
    }
    for (int e = 0; e < n; ++e) {
        const int i = ij[2 * e], j = ij[2 * e + 1];
        if (i < 0 || i >= L.nx || j < 0 || j >= L.ny || !std::isfinite(q[e])) return EIK_EINVAL;
        const int node = j * L.nx + i;
        int pos = -1;
        for (int k = 0; k < s->n; ++k)
            if (s->node[k] == node) pos = k;
        if (pos < 0) {
            s->node[s->n] = node;
            s->q[s->n] = q[e];
            ++s->n;
        } else if (q[e] < s->q[pos]) {
            s->q[pos] = q[e];
        }
    }
    // by node, as the device looks them up (insertion sort: at most
    // MAX_SOURCES entries)
    for (int a = 1; a < s->n; ++a) {
        const int nd = s->node[a];
        const double qv = s->q[a];
        int b = a - 1;
        for (; b >= 0 && s->node[b] > nd; --b) {
            s->node[b + 1] = s->node[b];
            s->q[b + 1] = s->q[b];
        }
        s->node[b + 1] = nd;
        s->q[b + 1] = qv;
    }
    s->q_min = std::numeric_limits<double>::infinity();
    for (int k = 0; k < s->n; ++k) s->q_min = std::fmin(s->q_min, s->q[k]);
    double cmax[MAX_SOURCES];
    for (int k = 0; k < s->n; ++k) {
        s->q[k] -= s->q_min;
        const int i = s->node[k] % L.nx, j = s->node[k] / L.nx;
        const int c = (j / L.k) * L.cxn + (i / L.k);
        int pos = -1;
        for (int m = 0; m < s->ncell; ++m)
            if (s->cell[m] == c) pos = m;
        if (pos < 0) {
            s->cell[s->ncell] = c;
            cmax[s->ncell] = s->q[k];
            ++s->ncell;
        } else {
            cmax[pos] = std::fmax(cmax[pos], s->q[k]);
        }
    }
    for (int m = 0; m < s->ncell; ++m) {
        long long b;
        std::memcpy(&b, &cmax[m], 8);
        s->key[m] = key_from_bits(b);
    }
    return EIK_OK;
}

}  // namespace
}  // namespace eik

using namespace eik;

extern "C" int eik_solve_noalloc(const eik_plan_desc* d, const eik_instance* in, eik_stats* st,
                                 void* cuda_stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!desc_valid(d) || !in || !in->F || !in->U) return EIK_EINVAL;
    if (d->precision != EIK_FP64 || d->method != EIK_METHOD_HCM) return EIK_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return EIK_ECUDA;
    }
    // F and U must be device memory of the current device: the scratch
    // used below is that device's copy
    for (const void* ptr : {(const void*)in->F, (const void*)in->U}) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, ptr) != cudaSuccess) {
            cudaGetLastError();
            return EIK_EINVAL;
        }
        if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != dev)
            return EIK_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the call copies through stack buffers and waits on its stream: not a
    // sequence a stream under capture can hold
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return EIK_EINVAL;
    }
    if (cap != cudaStreamCaptureStatusNone) return EIK_EINVAL;
    void* scratch = nullptr;
    int sms = 0;
    int rc = setup_device(dev, &scratch, &sms);
    if (rc) return rc;

    eik_plan_desc dd = *d;
    const JobParams P = choose_params(d, 1);
    dd.cell_k = P.k;
    // always bucketed rounds (the round-free schedules' rings would need
    // more scratch), in one wide bucket unless the descriptor sets a width
    const double bw_main = d->bucket_width != 0.0 ? d->bucket_width : -256.0;
    const Layout L = make_layout(d->nx, d->ny, dd.cell_k);
    StackSources ss;
    rc = prepare_stack_sources(L, in, s, &ss);
    if (rc) return rc;

    // carve the scratch; grids that do not fit are rejected
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align256(off + bytes);
        return (char*)scratch + at;
    };
    struct alignas(64) Tables {
        InstDesc desc;
        AuxInst aux;
        int cell_pre[2];
        double q[MAX_SOURCES];
        unsigned long long key[MAX_SOURCES];
        int node[MAX_SOURCES], node_inst[MAX_SOURCES], cell[MAX_SOURCES], cell_inst[MAX_SOURCES];
    };
    static_assert(sizeof(Tables) < 32 * 1024, "tables live on the stack");
    Tables tb;
    std::memset((void*)&tb, 0, sizeof(tb));
    Tables* tdev = (Tables*)take(sizeof(Tables));
    // block prefixes, each followed by its owner table (filled on the device)
    const int nbi = aux_blocks(L.nyp, L.nxp);
    const int nbf = aux_blocks(L.urows, L.upitch);
    int* blk_pre_dev = (int*)take((size_t)(2 + nbi) * 4);
    int* blk_full_dev = (int*)take((size_t)(2 + nbf) * 4);
    const int blk_pre_h[2] = {0, nbi};
    const int blk_full_h[2] = {0, nbf};
    const size_t z_ctl = align256(4 * sizeof(Ctl) + sizeof(ResidualOut));
    const size_t zero_bytes = z_ctl + 2 * align256((size_t)L.J * 4);
    char* zero = take(zero_bytes);
    unsigned long long* cval = (unsigned long long*)take((size_t)L.J * 8);
    char* inst = take(inst_bytes(L, false, false, false));
    if (off > SCRATCH_BYTES) return EIK_EINVAL;  // grid too large for the fixed scratch

    Ctl* ictl = (Ctl*)zero;  // [0] unused first pass, [1] the FP64 pass
    Ctl* gctl = ictl + 2;
    ResidualOut* res = (ResidualOut*)(gctl + 2);
    InstArrays a = carve_inst(L, false, false, false, inst);
    a.cval = cval;
    a.qflag = (int*)(zero + z_ctl);
    a.visits = (int*)(zero + z_ctl + align256((size_t)L.J * 4));
    const double shift = ss.n ? ss.q_min : 0.0;
    bool ok = true;
    InstDesc unused;
    fill_inst_tables(L, a, false, d->h, bw_main, bw_main, &ictl[0], &ictl[1], res, in->F, in->U, shift,
                     &tb.aux, &tb.desc, &unused, &ok);
    if (!ok) return EIK_ECUDA;
    tb.cell_pre[0] = 0;
    tb.cell_pre[1] = L.J;
    for (int e = 0; e < ss.n; ++e) {
        tb.q[e] = ss.q[e];
        tb.node[e] = ss.node[e];
        tb.node_inst[e] = 0;
    }
    for (int e = 0; e < ss.ncell; ++e) {
        tb.key[e] = ss.key[e];
        tb.cell[e] = ss.cell[e];
        tb.cell_inst[e] = 0;
    }

    // (the scratch holds the previous call's data: the init kernel rewrites
    // every element of the padded arrays, the +inf rings included)
    if (cudaMemcpyAsync(tdev, &tb, sizeof(tb), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(blk_pre_dev, blk_pre_h, 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(blk_full_dev, blk_full_h, 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return EIK_ECUDA;

    JobDev j;
    std::memset((void*)&j, 0, sizeof(j));
    j.n = 1;
    j.k = L.k;
    j.fp32 = false;
    j.desc_main = &tdev->desc;
    j.aux = &tdev->aux;
    j.blk_pre = blk_pre_dev;
    j.blk_full = blk_full_dev;
    j.nblocks_full = nbf;
    j.cell_pre = tdev->cell_pre;
    j.nblocks = nbi;
    j.ncells = L.J;
    j.ictl = ictl;
    j.gctl = gctl;
    j.res = res;
    j.src.q = tdev->q;
    j.src.node = tdev->node;
    j.src.node_inst = tdev->node_inst;
    j.src.n = ss.n;
    j.src.cell_key = tdev->key;
    j.src.cell = tdev->cell;
    j.src.cell_inst = tdev->cell_inst;
    j.src.ncell = ss.ncell;
    j.nsrc_total = ss.n;
    j.ncell_total = ss.ncell;
    j.deadline_ns = d->deadline_ns;
    j.zero_base = zero;
    j.zero_bytes = zero_bytes;
    j.cval_all = cval;
    j.ncval = (size_t)L.J;
    j.qflag_all = a.qflag;
    j.visits_all = a.visits;
    int nl = 0;
    rc = enqueue_job(j, sms, s, nullptr, &nl);
    if (rc) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return rc;
    }
    struct {
        Ctl c[4];
        ResidualOut r;
    } host;
    cudaMemcpyAsync(&host, zero, sizeof(host), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return EIK_ECUDA;
    }
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    eik_stats local;
    job_stats(L, &dd, false, &host.c[0], &host.c[1], &host.c[2], &host.c[3], &host.r, shift, bw_main, ms,
              &local);
    local.launches = nl;
    if (st) *st = local;
    return local.status;
}
