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

int prepare_stack_sources(const Layout& L, const eik_instance* in, StackSources* s) {
    const int n = in->nsrc;
    if (n < 0 || n > MAX_SOURCES) return EIK_EINVAL;
    s->n = s->ncell = 0;
    s->q_min = 0.0;
    if (n == 0) return EIK_OK;
    if (!in->src_ij || !in->src_q) return EIK_EINVAL;
    int32_t ij[2 * MAX_SOURCES];
    double q[MAX_SOURCES];
    if (cudaMemcpy(ij, in->src_ij, (size_t)n * 8, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(q, in->src_q, (size_t)n * 8, cudaMemcpyDefault) != cudaSuccess) {
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
    if (d->precision != EIK_FP64) return EIK_EINVAL;
    if (!is_device_ptr(in->F) || !is_device_ptr(in->U)) return EIK_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return EIK_ECUDA;
    }
    void* scratch = nullptr;
    int sms = 0;
    int rc = setup_device(dev, &scratch, &sms);
    if (rc) return rc;

    eik_plan_desc dd = *d;
    dd.cell_k = default_k(d);
    const Layout L = make_layout(d->nx, d->ny, dd.cell_k);
    StackSources ss;
    rc = prepare_stack_sources(L, in, &ss);
    if (rc) return rc;

    // carve the scratch; grids that do not fit are rejected
    const size_t un = (size_t)L.upitch * L.urows, fn = (size_t)L.fpitch * L.frows;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align256(off + bytes);
        return (char*)scratch + at;
    };
    Workspace w;
    std::memset((void*)&w, 0, sizeof(w));
    w.L = L;
    w.U64 = (double*)take(un * 8);
    w.f64 = (double*)take(fn * 8);
    w.cval = (unsigned long long*)take((size_t)L.J * 8);
    w.qflag = (int*)take((size_t)L.J * 4);
    w.visits = (int*)take((size_t)L.J * 4);
    w.has_src = (unsigned char*)take((size_t)L.J);
    w.lists = (int*)take((size_t)5 * L.J * 4);
    w.ctl = (Ctl*)take(2 * sizeof(Ctl) + sizeof(ResidualOut));
    w.res = (ResidualOut*)(w.ctl + 2);
    void* tables = take(src_table_bytes((size_t)ss.n, (size_t)ss.ncell));
    if (off > SCRATCH_BYTES) return EIK_EINVAL;  // grid too large for the fixed scratch

    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int K = L.k;
    if (!make_map(&w.tmU64, w.U64, true, L.upitch, L.urows, L.upitch, K + 2, K + 2) ||
        !make_map(&w.tmF64, w.f64, true, L.fpitch, L.frows, L.fpitch, K + 2, K + 2))
        return EIK_ECUDA;
    // the scratch holds the previous call's data: rebuild the +inf rings
    if (launch_fill(w.U64, un, std::numeric_limits<double>::infinity(), s) != cudaSuccess ||
        launch_fill(w.f64, fn, std::numeric_limits<double>::infinity(), s) != cudaSuccess)
        return EIK_ECUDA;
    const SrcTables t = carve_src_tables(tables, (size_t)ss.n, (size_t)ss.ncell);
    if (ss.n) {
        cudaMemcpyAsync(t.node, ss.node, (size_t)ss.n * 4, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(t.q, ss.q, (size_t)ss.n * 8, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(t.cell, ss.cell, (size_t)ss.ncell * 4, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(t.cell_key, ss.key, (size_t)ss.ncell * 8, cudaMemcpyHostToDevice, s);
    }
    int nl = 2;
    int launched = 0;
    rc = enqueue_solve_tables(&w, &dd, in->F, t, sms, s, nullptr, &launched);
    if (rc) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return rc;
    }
    nl += launched;
    const double shift = ss.n ? ss.q_min : 0.0;
    if (launch_output(w.U64, nullptr, L.upitch, L.nx, L.ny, shift, in->U, s) != cudaSuccess)
        return EIK_ECUDA;
    ++nl;
    struct {
        Ctl c[2];
        ResidualOut r;
    } host;
    cudaMemcpyAsync(&host, w.ctl, sizeof(host), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return EIK_ECUDA;
    }
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    eik_stats local;
    finish_stats(L, &dd, &host.c[0], &host.c[1], &host.r, shift, false, ms, &local);
    local.launches = nl;
    if (st) *st = local;
    return local.status;
}
