// eik_api.cu -- the C ABI (include/eik.h): plans, single solves.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <new>
#include <vector>

#include "eik_common.cuh"
#include "eik_plan.h"

using namespace eik;

extern "C" const char* eik_strerror(int code) {
    switch (code) {
    case EIK_OK: return "ok";
    case EIK_EINVAL: return "invalid argument";
    case EIK_ENOMEM: return "out of memory";
    case EIK_EBUSY: return "busy: over the memory budget or no free slot";
    case EIK_EAGAIN: return "not finished yet";
    case EIK_ETIMEDOUT: return "device deadline expired";
    case EIK_ENOTCONVERGED: return "not converged / tolerance not certified";
    case EIK_ECUDA: return "CUDA runtime error";
    default: return "unknown eik status";
    }
}

namespace eik {

// ---------------------------------------------------------------- layout
static int round_up(int v, int m) { return (v + m - 1) / m * m; }

bool desc_valid(const eik_plan_desc* d) {
    if (!d) return false;
    if (d->nx < 2 || d->ny < 2) return false;
    if (!(d->h > 0.0) || !std::isfinite(d->h)) return false;
    if (d->cell_k != 0 && d->cell_k != 4 && d->cell_k != 8 && d->cell_k != 16 && d->cell_k != 32 &&
        d->cell_k != 64)
        return false;
    if (d->precision != EIK_FP64 && d->precision != EIK_FP32_REFINE) return false;
    if ((long long)d->nx * d->ny > (1ll << 31) - 1) return false;
    return true;
}

int default_k(const eik_plan_desc* d) {
    if (d->cell_k) return d->cell_k;
    return 8;
}

Layout make_layout(int nx, int ny, int k) {
    Layout L;
    L.nx = nx;
    L.ny = ny;
    L.k = k;
    L.cxn = (nx + k - 1) / k;
    L.cyn = (ny + k - 1) / k;
    L.J = L.cxn * L.cyn;
    L.nxp = L.cxn * k;
    L.nyp = L.cyn * k;
    // room for the FP32 box (k+4 wide from column cx*k) and a multiple of 16 B rows
    L.upitch = round_up(L.nxp + 4, 32);
    L.urows = L.nyp + 2;
    // f shares U's layout (ring included) so that its TMA box carries the halo
    L.fpitch = L.upitch;
    L.frows = L.urows;
    return L;
}

size_t layout_bytes(const Layout& L, bool fp32) {
    size_t b = 0;
    const size_t un = (size_t)L.upitch * L.urows, fn = (size_t)L.fpitch * L.frows;
    if (fp32) b += un * (4 + 8) + fn * (4 + 8);  // U32, Udf, f32, fdf
    else b += un * 8 + fn * 8;                   // U64, f64
    b += (size_t)L.nx * L.ny * 8;                // staging for host F / output
    b += (size_t)L.J * (8 + 4 + 4 + 1);          // cval, qflag, visits, has_src
    b += (size_t)5 * L.J * 4;                    // lists
    b += 2 * sizeof(Ctl) + sizeof(ResidualOut);
    return b;
}

// ---------------------------------------------------------------- tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

bool make_map(CUtensorMap* tm, void* base, bool fp64, int width, int rows, int pitch_elems,
              int box_w, int box_h) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int es = fp64 ? 8 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch_elems * es};
    cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(tm, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------- workspace
static void* dalloc(size_t bytes, int* err) {
    void* p = nullptr;
    if (*err) return nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        *err = EIK_ENOMEM;
        return nullptr;
    }
    return p;
}

int workspace_alloc(Workspace* w, const Layout& L, bool fp32, cudaStream_t st) {
    int err = 0;
    std::memset((void*)w, 0, sizeof(*w));
    w->L = L;
    w->fp32 = fp32;
    const size_t un = (size_t)L.upitch * L.urows, fn = (size_t)L.fpitch * L.frows;
    if (fp32) {
        w->U32 = (float*)dalloc(un * 4, &err);
        w->f32 = (float*)dalloc(fn * 4, &err);
        w->Udf = (float2*)dalloc(un * 8, &err);
        w->fdf = (float2*)dalloc(fn * 8, &err);
    } else {
        w->U64 = (double*)dalloc(un * 8, &err);
        w->f64 = (double*)dalloc(fn * 8, &err);
    }
    w->Fstage = (double*)dalloc((size_t)L.nx * L.ny * 8, &err);
    w->cval = (unsigned long long*)dalloc((size_t)L.J * 8, &err);
    w->qflag = (int*)dalloc((size_t)L.J * 4, &err);
    w->visits = (int*)dalloc((size_t)L.J * 4, &err);
    w->has_src = (unsigned char*)dalloc((size_t)L.J, &err);
    w->lists = (int*)dalloc((size_t)5 * L.J * 4, &err);
    w->ctl = (Ctl*)dalloc(2 * sizeof(Ctl) + sizeof(ResidualOut), &err);
    if (err) {
        workspace_free(w);
        return err;
    }
    w->res = (ResidualOut*)(w->ctl + 2);
    // the +inf ring (and padding columns) never change after this fill
    if (w->U64 && launch_fill(w->U64, un, std::numeric_limits<double>::infinity(), st) != cudaSuccess)
        err = EIK_ECUDA;
    if (w->U32 && launch_fill32(w->U32, un, std::numeric_limits<float>::infinity(), st) != cudaSuccess)
        err = EIK_ECUDA;
    if (w->Udf && launch_fill_df(w->Udf, un, st) != cudaSuccess) err = EIK_ECUDA;
    // f's ring: +inf (obstacles) forever
    if (w->f64 && launch_fill(w->f64, fn, std::numeric_limits<double>::infinity(), st) != cudaSuccess)
        err = EIK_ECUDA;
    if (w->f32 && launch_fill32(w->f32, fn, std::numeric_limits<float>::infinity(), st) != cudaSuccess)
        err = EIK_ECUDA;
    if (w->fdf && launch_fill_df(w->fdf, fn, st) != cudaSuccess) err = EIK_ECUDA;
    const int K = L.k;
    // U maps span the whole pitch, so a box (k+2 or k+4 wide) never leaves the
    // array; 8-byte values (doubles or float pairs) move as FLOAT64 elements
    if (fp32) {
        if (!make_map(&w->tmU32, w->U32, false, L.upitch, L.urows, L.upitch, K + 4, K + 2)) err = EIK_ECUDA;
        if (!make_map(&w->tmF32, w->f32, false, L.fpitch, L.frows, L.fpitch, K + 4, K + 2)) err = EIK_ECUDA;
        if (!make_map(&w->tmUdf, w->Udf, true, L.upitch, L.urows, L.upitch, K + 2, K + 2)) err = EIK_ECUDA;
        if (!make_map(&w->tmFdf, w->fdf, true, L.fpitch, L.frows, L.fpitch, K + 2, K + 2)) err = EIK_ECUDA;
    } else {
        if (!make_map(&w->tmU64, w->U64, true, L.upitch, L.urows, L.upitch, K + 2, K + 2)) err = EIK_ECUDA;
        if (!make_map(&w->tmF64, w->f64, true, L.fpitch, L.frows, L.fpitch, K + 2, K + 2)) err = EIK_ECUDA;
    }
    if (err) workspace_free(w);
    return err;
}

void workspace_free(Workspace* w) {
    void* ptrs[] = {w->U64, w->f64, w->U32, w->f32, w->Udf, w->fdf, w->Fstage,
                    w->cval, w->qflag, w->visits, w->has_src, w->lists, w->ctl};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    std::memset((void*)w, 0, sizeof(*w));
}

// ---------------------------------------------------------------- sources
int prepare_sources(const Layout& L, const eik_instance* in, HostSources* hs) {
    hs->node.clear();
    hs->q.clear();
    hs->cell.clear();
    hs->cell_key.clear();
    hs->q_min = 0.0;
    const int n = in->nsrc;
    if (n < 0) return EIK_EINVAL;
    if (n == 0) return EIK_OK;
    if (!in->src_ij || !in->src_q) return EIK_EINVAL;
    std::vector<int32_t> ij(2 * (size_t)n);
    std::vector<double> q((size_t)n);
    if (cudaMemcpy(ij.data(), in->src_ij, ij.size() * 4, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(q.data(), in->src_q, q.size() * 8, cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        return EIK_EINVAL;
    }
    std::vector<std::pair<int, double>> s((size_t)n);
    for (int e = 0; e < n; ++e) {
        const int i = ij[2 * e], j = ij[2 * e + 1];
        if (i < 0 || i >= L.nx || j < 0 || j >= L.ny || !std::isfinite(q[e])) return EIK_EINVAL;
        s[e] = {j * L.nx + i, q[e]};
    }
    std::sort(s.begin(), s.end());  // by node, then q ascending: first of a run is the min
    hs->q_min = std::numeric_limits<double>::infinity();
    for (size_t e = 0; e < s.size(); ++e) {
        if (e && s[e].first == s[e - 1].first) continue;
        hs->node.push_back(s[e].first);
        hs->q.push_back(s[e].second);
        hs->q_min = std::min(hs->q_min, s[e].second);
    }
    // the device works on q - q_min >= 0 (see the solver: ordered bit patterns)
    for (double& v : hs->q) v -= hs->q_min;
    // cell value of a source cell: max q over its sources (Sec. 4.2, HCM item 1)
    std::vector<std::pair<int, double>> cq;
    for (size_t e = 0; e < hs->node.size(); ++e) {
        const int i = hs->node[e] % L.nx, j = hs->node[e] / L.nx;
        cq.push_back({(j / L.k) * L.cxn + (i / L.k), hs->q[e]});
    }
    std::sort(cq.begin(), cq.end());
    for (size_t e = 0; e < cq.size(); ++e) {
        if (e + 1 < cq.size() && cq[e + 1].first == cq[e].first) continue;  // keep the max
        long long b;
        std::memcpy(&b, &cq[e].second, 8);
        hs->cell.push_back(cq[e].first);
        hs->cell_key.push_back(key_from_bits(b));
    }
    return EIK_OK;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int grow_staging(DevBuf* b, size_t bytes) {
    if (b->cap >= bytes) return EIK_OK;
    if (b->p) cudaFree(b->p);
    b->p = nullptr;
    b->cap = 0;
    const size_t cap = std::max<size_t>(bytes, 4096);
    if (cudaMalloc(&b->p, cap) != cudaSuccess) {
        cudaGetLastError();
        return EIK_ENOMEM;
    }
    b->cap = cap;
    return EIK_OK;
}

// ---------------------------------------------------------------- one solve
// EIK_PROFILE=1 (debugging aid): kernels accumulate per-phase clock cycles and
// each solve prints them to stderr.
int profiling() {
    static int on = -1;
    if (on < 0) {
        const char* e = std::getenv("EIK_PROFILE");
        on = (e && e[0] == '1') ? 1 : 0;
    }
    return on;
}

static void print_profile(const char* what, const Ctl* c) {
    const char* names[8] = {"split", "barrier", "list+pop", "tma", "sweeps", "writeback", "activate",
                            "warp-visits"};
    double tot = 0;
    for (int i = 0; i < 7; ++i) tot += (double)c->prof[i];
    std::fprintf(stderr, "[eik profile %s] rounds=%llu", what, (unsigned long long)c->rounds);
    for (int i = 0; i < 7; ++i)
        std::fprintf(stderr, " %s=%.1f%%", names[i], tot > 0 ? 100.0 * c->prof[i] / tot : 0.0);
    std::fprintf(stderr, " warp-visits=%llu cyc/visit(sweeps)=%.0f cyc/visit(tma)=%.0f cyc/visit(act)=%.0f\n",
                 (unsigned long long)c->prof[7], c->prof[7] ? (double)c->prof[4] / c->prof[7] : 0.0,
                 c->prof[7] ? (double)c->prof[3] / c->prof[7] : 0.0,
                 c->prof[7] ? (double)c->prof[6] / c->prof[7] : 0.0);
}
// Queue the whole solve of one instance on `st` (inputs already validated;
// F on the device).  Reads nothing back.
int enqueue_solve(Workspace* w, const eik_plan_desc* d, const double* Fdev, const HostSources& hs,
                  SrcDev* sd, int num_sms, cudaStream_t st, cudaEvent_t* ev, int* launches) {
    // upload the (small) source tables into the plan's growable buffer
    const size_t nsrc = hs.node.size(), ncell = hs.cell.size();
    int rc = grow_staging(&sd->buf, src_table_bytes(nsrc, ncell));
    if (rc) return rc;
    const SrcTables t = carve_src_tables(sd->buf.p, nsrc, ncell);
    if (nsrc) {
        cudaMemcpyAsync(t.node, hs.node.data(), nsrc * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(t.q, hs.q.data(), nsrc * 8, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(t.cell, hs.cell.data(), ncell * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(t.cell_key, hs.cell_key.data(), ncell * 8, cudaMemcpyHostToDevice, st);
    }
    return enqueue_solve_tables(w, d, Fdev, t, num_sms, st, ev, launches);
}

size_t src_table_bytes(size_t nsrc, size_t ncell) {
    return (nsrc * 4 + 15) / 16 * 16 + nsrc * 8 + (ncell * 4 + 15) / 16 * 16 + ncell * 8 + 64;
}

SrcTables carve_src_tables(void* base_, size_t nsrc, size_t ncell) {
    char* base = (char*)base_;
    SrcTables t;
    t.node = (int*)base;
    t.q = (double*)(base + ((nsrc * 4 + 15) / 16 * 16));
    t.cell = (int*)((char*)t.q + nsrc * 8);
    t.cell_key = (unsigned long long*)((char*)t.cell + ((ncell * 4 + 15) / 16 * 16));
    t.nsrc = (int)nsrc;
    t.ncell = (int)ncell;
    return t;
}

int enqueue_solve_tables(Workspace* w, const eik_plan_desc* d, const double* Fdev, const SrcTables& t,
                         int num_sms, cudaStream_t st, cudaEvent_t* ev, int* launches) {
    int nl = 0;
    const Layout& L = w->L;
    const bool fp32 = d->precision == EIK_FP32_REFINE;
    const size_t nsrc = (size_t)t.nsrc, ncell = (size_t)t.ncell;
    int* d_node = t.node;
    double* d_q = t.q;
    int* d_cell = t.cell;
    unsigned long long* d_ckey = t.cell_key;
    Ctl* ctl32 = w->ctl;
    Ctl* ctl64 = w->ctl + 1;
    cudaMemsetAsync(w->ctl, 0, 2 * sizeof(Ctl) + sizeof(ResidualOut), st);
    cudaMemsetAsync(w->cval, 0xff, (size_t)L.J * 8, st);
    cudaMemsetAsync(w->qflag, 0, (size_t)L.J * 4, st);
    cudaMemsetAsync(w->visits, 0, (size_t)L.J * 4, st);
    cudaMemsetAsync(w->has_src, 0, (size_t)L.J, st);
    Ctl* first_ctl = fp32 ? ctl32 : ctl64;
    if (launch_ctl_init(first_ctl, (int)ncell, st) != cudaSuccess) return EIK_ECUDA;
    ++nl;
    if (fp32) {
        if (launch_ctl_init(ctl64, 0, st) != cudaSuccess) return EIK_ECUDA;
        ++nl;
    }

    InitParams ip{};
    ip.F = Fdev;
    ip.nx = L.nx;
    ip.ny = L.ny;
    ip.h = d->h;
    ip.f64 = w->f64;
    ip.f32 = w->f32;
    ip.fdf = w->fdf;
    ip.fpitch = L.fpitch;
    ip.U64 = w->U64;
    ip.U32 = w->U32;
    ip.Udf = w->Udf;
    ip.upitch = L.upitch;
    ip.nxp = L.nxp;
    ip.nyp = L.nyp;
    ip.ctl = first_ctl;
    if (launch_init_grid(ip, st) != cudaSuccess) return EIK_ECUDA;
    ++nl;
    SourceInit si{d_node, d_q, (int)nsrc, d_cell, d_ckey, (int)ncell, L.nx, L.k, L.cxn};
    if (launch_init_sources(ip, si, w->cval, w->qflag, w->has_src, w->lists + 3 * L.J, st) !=
        cudaSuccess)
        return EIK_ECUDA;
    if (nsrc) ++nl;

    const long long deadline = d->deadline_ns > 0 ? d->deadline_ns : 20000000000ll;
    auto params = [&](const CUtensorMap& tmU, const CUtensorMap& tmF, void* U, const void* f,
                      Ctl* ctl) {
        SolveParams p{};
        p.tmU = tmU;
        p.tmF = tmF;
        p.U = U;
        p.f = f;
        p.upitch = L.upitch;
        p.fpitch = L.fpitch;
        p.nx = L.nx;
        p.ny = L.ny;
        p.cxn = L.cxn;
        p.cyn = L.cyn;
        p.J = L.J;
        p.cval = w->cval;
        p.qflag = w->qflag;
        p.visits = w->visits;
        p.has_src = w->has_src;
        p.lists = w->lists;
        p.ctl = ctl;
        p.delta = d->bucket_width;
        p.deadline_ns = deadline;
        p.profile = profiling();
        return p;
    };
    LaunchShape shape;
    if (fp32) {
        // FP32 cell solves
        if (solver_shape_f32(L.k, num_sms, &shape)) return EIK_ECUDA;
        const SolveParams p32 = params(w->tmU32, w->tmF32, w->U32, w->f32, ctl32);
        if (ev) cudaEventRecord(ev[0], st);
        if (launch_solver_f32(L.k, p32, shape, st) != cudaSuccess) return EIK_ECUDA;
        if (ev) cudaEventRecord(ev[1], st);
        ++nl;
        // refinement pass (double-float) seeded from the FP32 result
        cudaMemsetAsync(w->cval, 0xff, (size_t)L.J * 8, st);
        SeedParams sp{};
        sp.U32 = w->U32;
        sp.Udf = w->Udf;
        sp.fdf = w->fdf;
        sp.upitch = L.upitch;
        sp.fpitch = L.fpitch;
        sp.nx = L.nx;
        sp.ny = L.ny;
        sp.k = L.k;
        sp.cxn = L.cxn;
        sp.cyn = L.cyn;
        sp.beta = 1.0f / 1024.0f;
        sp.cval = w->cval;
        sp.qflag = w->qflag;
        sp.visits = w->visits;
        sp.far0 = w->lists + 3 * L.J;
        sp.ctl = ctl64;
        // the refinement pass needs the bucket-width default too
        cudaMemcpyAsync(&ctl64->fmin_f, &ctl32->fmin_f, 8, cudaMemcpyDeviceToDevice, st);
        if (launch_seed_refine(sp, st) != cudaSuccess) return EIK_ECUDA;
        nl += 2;
        if (solver_shape_df(L.k, num_sms, &shape)) return EIK_ECUDA;
        const SolveParams pd = params(w->tmUdf, w->tmFdf, w->Udf, w->fdf, ctl64);
        if (ev) cudaEventRecord(ev[2], st);
        if (launch_solver_df(L.k, pd, shape, st) != cudaSuccess) return EIK_ECUDA;
        if (ev) cudaEventRecord(ev[3], st);
        ++nl;
        if (launch_residual(w->Udf, L.upitch, w->fdf, L.fpitch, Fdev, d->h, L.nx, L.ny, w->res, st) !=
            cudaSuccess)
            return EIK_ECUDA;
        ++nl;
    } else {
        if (solver_shape_f64(L.k, num_sms, &shape)) return EIK_ECUDA;
        const SolveParams p64 = params(w->tmU64, w->tmF64, w->U64, w->f64, ctl64);
        if (ev) cudaEventRecord(ev[2], st);
        if (launch_solver_f64(L.k, p64, shape, st) != cudaSuccess) return EIK_ECUDA;
        if (ev) cudaEventRecord(ev[3], st);
        ++nl;
    }
    if (launches) *launches = nl;
    return EIK_OK;
}

static double dval(unsigned long long k) {
    long long b = bits_from_key(k);
    double v;
    std::memcpy(&v, &b, 8);
    return v;
}

// Fill *st from the control blocks copied back to the host.
void finish_stats(const Layout& L, const eik_plan_desc* d, const Ctl* c32, const Ctl* c64,
                  const ResidualOut* r, double q_min, bool fp32, double ms, eik_stats* st) {
    eik_stats s;
    std::memset(&s, 0, sizeof(s));
    int status = c64->status;
    if (fp32 && c32->status) status = c32->status;
    unsigned long long visits = c64->visits, sweeps = c64->sweeps, lane = c64->lane_updates;
    long long rounds = (long long)c64->rounds, adv = (long long)c64->advances;
    if (fp32) {
        visits += c32->visits;
        sweeps += c32->sweeps;
        lane += c32->lane_updates;
        rounds += (long long)c32->rounds;
        adv += (long long)c32->advances;
    }
    const double npts = (double)L.nx * L.ny;
    s.ms = ms;
    s.mpts_per_s = ms > 0 ? npts / ms / 1000.0 : 0.0;
    s.updates_per_pt = (double)lane / npts;
    s.avhr = (double)visits / L.J;
    s.avs = (double)sweeps / L.J;
    s.cell_visits = (long long)visits;
    s.rounds = rounds;
    s.buckets = adv;
    s.cell_k = L.k;
    const double fmin = dval(c64->fmin_f);
    s.bucket_width = d->bucket_width > 0 ? d->bucket_width : 4.0 * L.k * fmin;
    if (fp32) {
        // values on the device are U - q_min >= 0
        const double rr = dval(r->r_max), umax = dval(r->u_max);
        s.max_residual = rr;
        // Certificate (comparison principle for the monotone scheme): for
        // lam > 1, lam * (U - q_min) is a strict supersolution with margin
        // (lam - 1) f_min / sqrt 2, and likewise a strict subsolution for
        // lam < 1; so |V - U| <= sqrt 2 * r / f_min * max(U - q_min).
        double bound = 0.0;
        if (r->n_bad) bound = std::numeric_limits<double>::infinity();
        else if (rr > 0 && umax > 0) bound = std::sqrt(2.0) * rr / fmin * umax;
        const double scale = std::max(std::fabs(umax + q_min), std::fabs(q_min));
        s.err_bound = scale > 0 ? bound / scale : bound;
        const double tol = d->tol > 0 ? d->tol : 1e-5;
        if (status == EIK_OK && !(s.err_bound <= tol)) status = EIK_ENOTCONVERGED;
    }
    s.status = status;
    if (st) *st = s;
}

}  // namespace eik

// ================================================================= C ABI
extern "C" size_t eik_plan_workspace_bytes(const eik_plan_desc* d) {
    if (!desc_valid(d)) return 0;
    const Layout L = make_layout(d->nx, d->ny, default_k(d));
    return layout_bytes(L, d->precision == EIK_FP32_REFINE);
}

extern "C" int eik_plan_create(eik_plan* out, const eik_plan_desc* d, void* cuda_stream) {
    if (!out) return EIK_EINVAL;
    *out = nullptr;
    if (!desc_valid(d)) return EIK_EINVAL;
    eik_plan_s* p = new (std::nothrow) eik_plan_s();
    if (!p) return EIK_ENOMEM;
    p->d = *d;
    p->d.cell_k = default_k(d);
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return EIK_ECUDA;
    }
    if (cuda_stream) {
        p->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete p;
            return EIK_ECUDA;
        }
        p->own_stream = true;
    }
    const Layout L = make_layout(d->nx, d->ny, p->d.cell_k);
    int rc = workspace_alloc(&p->ws, L, d->precision == EIK_FP32_REFINE, p->stream);
    if (!rc && (cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess))
        rc = EIK_ECUDA;
    for (int e = 0; e < 4 && !rc; ++e)
        if (cudaEventCreate(&p->pev[e]) != cudaSuccess) rc = EIK_ECUDA;
    if (!rc && cudaMallocHost((void**)&p->host_ctl, 2 * sizeof(Ctl) + sizeof(ResidualOut)) != cudaSuccess)
        rc = EIK_ENOMEM;
    if (!rc && cudaStreamSynchronize(p->stream) != cudaSuccess) rc = EIK_ECUDA;
    if (rc) {
        cudaGetLastError();
        eik_plan_destroy(p);
        return rc;
    }
    *out = p;
    return EIK_OK;
}

extern "C" void eik_plan_destroy(eik_plan p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    workspace_free(&p->ws);
    if (p->src.buf.p) cudaFree(p->src.buf.p);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    for (int e = 0; e < 4; ++e)
        if (p->pev[e]) cudaEventDestroy(p->pev[e]);
    if (p->host_ctl) cudaFreeHost(p->host_ctl);
    if (p->own_stream) cudaStreamDestroy(p->stream);
    delete p;
}

extern "C" int eik_solve(eik_plan p, const eik_instance* in, eik_stats* st) {
    if (!p || !in || !in->F || !in->U || in->nsrc < 0) return EIK_EINVAL;
    cudaSetDevice(p->device);
    Workspace* w = &p->ws;
    const Layout& L = w->L;
    HostSources hs;
    int rc = prepare_sources(L, in, &hs);
    if (rc) return rc;
    cudaStream_t s = p->stream;
    const double* Fdev = in->F;
    if (!is_device_ptr(in->F)) {
        if (cudaMemcpyAsync(w->Fstage, in->F, (size_t)L.nx * L.ny * 8, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return EIK_ECUDA;
        Fdev = w->Fstage;
    }
    cudaEventRecord(p->ev0, s);
    int nl = 0;
    rc = enqueue_solve(w, &p->d, Fdev, hs, &p->src, p->num_sms, s, p->pev, &nl);
    if (rc) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return rc;
    }
    cudaEventRecord(p->ev1, s);
    // result: strip the ring and padding and undo the q shift
    const double shift = hs.node.empty() ? 0.0 : hs.q_min;
    if (is_device_ptr(in->U)) {
        if (launch_output(w->U64, w->Udf, L.upitch, L.nx, L.ny, shift, in->U, s) != cudaSuccess)
            return EIK_ECUDA;
    } else {
        if (launch_output(w->U64, w->Udf, L.upitch, L.nx, L.ny, shift, w->Fstage, s) != cudaSuccess)
            return EIK_ECUDA;
        cudaMemcpyAsync(in->U, w->Fstage, (size_t)L.nx * L.ny * 8, cudaMemcpyDeviceToHost, s);
    }
    ++nl;
    cudaMemcpyAsync(p->host_ctl, w->ctl, 2 * sizeof(Ctl) + sizeof(ResidualOut), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return EIK_ECUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p->ev0, p->ev1);
    const Ctl* c = (const Ctl*)p->host_ctl;
    if (profiling()) {
        if (p->d.precision == EIK_FP32_REFINE) print_profile("fp32 pass", &c[0]);
        print_profile(p->d.precision == EIK_FP32_REFINE ? "refinement pass" : "fp64 pass", &c[1]);
    }
    eik_stats local;
    finish_stats(L, &p->d, &c[0], &c[1], (const ResidualOut*)(c + 2), hs.node.empty() ? 0.0 : hs.q_min,
                 p->d.precision == EIK_FP32_REFINE, ms, &local);
    if (p->d.precision == EIK_FP32_REFINE) cudaEventElapsedTime(&ms, p->pev[0], p->pev[1]), local.pass_ms[0] = ms;
    cudaEventElapsedTime(&ms, p->pev[2], p->pev[3]);
    local.pass_ms[1] = ms;
    local.launches = nl;
    if (st) *st = local;
    return local.status;
}
