// eik_job.cu -- layouts, per-instance tables and the launch sequence of a job.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>

#include "eik_job.h"

namespace eik {

static int round_up(int v, int m) { return (v + m - 1) / m * m; }
static size_t a256(size_t b) { return (b + 255) / 256 * 256; }

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
    // room for the FP32 box (k+4 wide from column cx*k) and rows that are a
    // multiple of 16 bytes; f shares the layout so its box carries the halo
    L.upitch = round_up(L.nxp + 4, 32);
    L.urows = L.nyp + 2;
    return L;
}

size_t inst_bytes(const Layout& L, bool fp32, bool stage_F, bool stage_U) {
    const size_t un = (size_t)L.upitch * L.urows;
    size_t b = 0;
    if (fp32) b += a256(un * 4) * 2 + a256(un * 8) * 2;
    else b += a256(un * 8) * 2;
    b += a256((size_t)5 * L.J * 4);
    if (stage_F) b += a256((size_t)L.nx * L.ny * 8);
    if (stage_U) b += a256((size_t)L.nx * L.ny * 8);
    return b;
}

InstArrays carve_inst(const Layout& L, bool fp32, bool stage_F, bool stage_U, char* base) {
    InstArrays a;
    std::memset((void*)&a, 0, sizeof(a));
    const size_t un = (size_t)L.upitch * L.urows;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base + off;
        off += a256(bytes);
        return p;
    };
    if (fp32) {
        a.U32 = (float*)take(un * 4);
        a.f32 = (float*)take(un * 4);
        a.Udf = (float2*)take(un * 8);
        a.fdf = (float2*)take(un * 8);
    } else {
        a.U64 = (double*)take(un * 8);
        a.f64 = (double*)take(un * 8);
    }
    a.lists = (int*)take((size_t)5 * L.J * 4);
    if (stage_F) a.Fstage = (double*)take((size_t)L.nx * L.ny * 8);
    if (stage_U) a.Ostage = (double*)take((size_t)L.nx * L.ny * 8);
    return a;
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

static void fill_desc(InstDesc* d, const Layout& L, void* U, const void* f, bool fp64_maps,
                      int box_w, const InstArrays& a, Ctl* ctl, double bucket_width, bool* ok) {
    std::memset((void*)d, 0, sizeof(*d));
    // the maps span the whole pitch, so a box never leaves the array
    *ok = *ok && make_map(&d->tmU, U, fp64_maps, L.upitch, L.urows, L.upitch, box_w, L.k + 2);
    *ok = *ok && make_map(&d->tmF, const_cast<void*>(f), fp64_maps, L.upitch, L.urows, L.upitch, box_w,
                          L.k + 2);
    d->U = U;
    d->f = f;
    d->cval = a.cval;
    d->qflag = a.qflag;
    d->visits = a.visits;
    d->dflags = a.dflags;
    d->lists = a.lists;
    d->ctl = ctl;
    d->upitch = L.upitch;
    d->cxn = L.cxn;
    d->cyn = L.cyn;
    d->J = L.J;
    d->delta = bucket_width;
}

void fill_inst_tables(const Layout& L, const InstArrays& a, bool fp32, double h, double bw_first,
                      double bw_main,
                      Ctl* ictl_first, Ctl* ictl_main, ResidualOut* res, const double* F,
                      double* out, double shift, AuxInst* aux, InstDesc* desc_main, InstDesc* desc_f32,
                      bool* ok) {
    const int K = L.k;
    if (fp32) {
        // 4-byte values: a box row of k+2 floats is not a multiple of 16
        // bytes, so the FP32 box is k+4 wide; pairs are 8-byte elements
        fill_desc(desc_f32, L, a.U32, a.f32, false, K + 4, a, ictl_first, bw_first, ok);
        fill_desc(desc_main, L, a.Udf, a.fdf, true, K + 2, a, ictl_main, bw_main, ok);
    } else {
        fill_desc(desc_main, L, a.U64, a.f64, true, K + 2, a, ictl_main, bw_main, ok);
    }
    std::memset((void*)aux, 0, sizeof(*aux));
    aux->F = F;
    aux->out = out;
    aux->h = h;
    aux->hx = (float)h;
    aux->hy = (float)(h - (double)aux->hx);
    aux->shift = shift;
    aux->nx = L.nx;
    aux->ny = L.ny;
    aux->nxp = L.nxp;
    aux->nyp = L.nyp;
    aux->upitch = L.upitch;
    aux->k = K;
    aux->cxn = L.cxn;
    aux->cyn = L.cyn;
    aux->U64 = a.U64;
    aux->f64 = a.f64;
    aux->U32 = a.U32;
    aux->f32 = a.f32;
    aux->Udf = a.Udf;
    aux->fdf = a.fdf;
    aux->cval = a.cval;
    aux->qflag = a.qflag;
    aux->visits = a.visits;
    aux->dflags = a.dflags;
    aux->far0 = a.lists + 3 * L.J;
    aux->ctl = fp32 ? ictl_first : ictl_main;
    aux->ctl2 = fp32 ? ictl_main : nullptr;
    aux->res = res;
    aux->J = L.J;
}

// ---------------------------------------------------------------- launches
int profiling() {
    static int on = -1;
    if (on < 0) {
        const char* e = std::getenv("EIK_PROFILE");
        on = (e && e[0] == '1') ? 1 : 0;
    }
    return on;
}

int enqueue_job(const JobDev& j, int num_sms, cudaStream_t st, cudaEvent_t* ev, int* launches) {
    int nl = 0;
    const int n = j.n;
    cudaMemsetAsync(j.zero_base, 0, j.zero_bytes, st);
    cudaMemsetAsync(j.cval_all, 0xff, j.ncval * 8, st);
    // the fields of the instances' control blocks and of the two launch-wide
    // ones behind them that start at all ones
    if (cudaMemset2DAsync(j.ictl, sizeof(Ctl), 0xff, CTL_ONES_BYTES, (size_t)(2 * n + 2), st) != cudaSuccess)
        return EIK_ECUDA;
    // f, U, the sources and the source cells, in one launch
    if (launch_init_grid(j.aux, j.blk_full, n, j.nblocks_full, j.src, st) != cudaSuccess) return EIK_ECUDA;
    ++nl;
    SolveParams p{};
    p.n_inst = n;
    p.deadline_ns = j.deadline_ns > 0 ? j.deadline_ns : 20000000000ll;
    p.profile = profiling();
    p.variant = j.variant;
    p.hold_ns = j.hold_ns;
    p.req_time = j.req_time;
    p.ring = j.ring;
    p.ring_mask = j.ring_mask;
    p.cell_pre = j.cell_pre;
    p.qctl = j.qctl;
    p.hist = j.hist;
    p.bq = j.bq;
    p.bq_data = j.bq_data;
    p.bq_mask = j.bq_mask;
    p.bq_window = j.window < 0 ? 0 : j.window > NBQ - 1 ? NBQ - 1 : j.window;
    p.inst_done = j.inst_done ? 1 : 0;
    // host-set checks (0 / unset: off): EIK_MAX_PASSES caps the passes of a
    // removal (a cap it hits reports EIK_ENOTCONVERGED), EIK_JITTER_NS
    // pauses each removal by up to that many ns before its tile load
    if (const char* e = std::getenv("EIK_MAX_PASSES")) p.max_passes = (int)std::strtol(e, nullptr, 10);
    if (const char* e = std::getenv("EIK_JITTER_NS")) {
        const long v = std::strtol(e, nullptr, 10);
        p.jitter_ns = v > 0 ? (unsigned)(v < 1000000 ? v : 1000000) : 0u;
    }
    const bool af = j.async_first && j.ring && j.k >= 8, am = j.async_main && j.ring && j.k >= 8;
    // the main pass's schedule (the value-ordered form for plain HCM only)
    const int sm = !am ? SCH_ROUNDS
                   : j.ordered && j.bq && j.variant == VAR_HCM ? SCH_ORDERED
                                                                    : SCH_FIFO;
    const int sf = !af ? SCH_ROUNDS : j.ordered && j.bq ? SCH_ORDERED : SCH_FIFO;
    LaunchShape shape;
    if (j.fp32 && j.one_pass) {
        // FP32_REFINE in one double-float pass from the sources (every
        // update on the FP32 pipe), certified like the two-pass form
        if (ev) cudaEventRecord(ev[0], st), cudaEventRecord(ev[1], st);
        if (solver_shape_df(j.k, num_sms, n, j.sm_cap, sm, VAR_HCM, &shape)) return EIK_ECUDA;
        p.inst = j.desc_main;
        p.gctl = j.gctl + 1;
        if (ev) cudaEventRecord(ev[2], st);
        if (launch_solver_df(j.k, sm, p, shape, st) != cudaSuccess) return EIK_ECUDA;
        if (ev) cudaEventRecord(ev[3], st);
        ++nl;
        if (!j.inst_done) {
            if (launch_residual(j.aux, j.blk_pre, n, j.nblocks, st) != cudaSuccess) return EIK_ECUDA;
            ++nl;
        }
    } else if (j.fp32) {
        if (solver_shape_f32(j.k, num_sms, n, j.sm_cap, sf, VAR_HCM, &shape)) return EIK_ECUDA;
        p.inst = j.desc_f32;
        p.gctl = j.gctl;
        if (ev) cudaEventRecord(ev[0], st);
        if (launch_solver_f32(j.k, sf, p, shape, st) != cudaSuccess) return EIK_ECUDA;
        if (ev) cudaEventRecord(ev[1], st);
        ++nl;
        // refinement pass (double-float) seeded from the FP32 result
        cudaMemsetAsync(j.cval_all, 0xff, j.ncval * 8, st);
        if (launch_seed_refine(j.aux, j.blk_pre, n, j.nblocks, j.cell_pre, j.ncells, 1.0f / 1024.0f, st) !=
            cudaSuccess)
            return EIK_ECUDA;
        nl += 2;
        if (solver_shape_df(j.k, num_sms, n, j.sm_cap, sm, VAR_HCM, &shape)) return EIK_ECUDA;
        p.inst = j.desc_main;
        p.gctl = j.gctl + 1;
        if (ev) cudaEventRecord(ev[2], st);
        if (launch_solver_df(j.k, sm, p, shape, st) != cudaSuccess) return EIK_ECUDA;
        if (ev) cudaEventRecord(ev[3], st);
        ++nl;
        if (launch_residual(j.aux, j.blk_pre, n, j.nblocks, st) != cudaSuccess) return EIK_ECUDA;
        ++nl;
    } else if (j.fmsm) {
        // Fast Marching-Sweeping: the coarse speeds, the coarse grids solved
        // by their own job (Part I), the order and the ready cells, then
        // every cell once (Part II)
        if (!j.coarse) return EIK_EINVAL;
        if (launch_fmsm_coarse_speed(j.aux, j.cell_pre, n, j.ncells, st) != cudaSuccess) return EIK_ECUDA;
        ++nl;
        int nlc = 0;
        if (ev) cudaEventRecord(ev[0], st);
        const int rc = enqueue_job(*j.coarse, num_sms, st, nullptr, &nlc);
        if (rc) return rc;
        if (ev) cudaEventRecord(ev[1], st);
        nl += nlc;
        if (cudaMemsetAsync(j.qctl, 0, 384, st) != cudaSuccess ||
            cudaMemsetAsync(j.ring, 0, ((size_t)j.ring_mask + 1) * 8, st) != cudaSuccess)
            return EIK_ECUDA;
        if (launch_fmsm_prep(j.aux, j.cell_pre, n, j.ncells, j.ring, j.qctl, st) != cudaSuccess)
            return EIK_ECUDA;
        ++nl;
        if (fmsm_shape(j.k, num_sms, n, j.sm_cap, &shape)) return EIK_ECUDA;
        p.inst = j.desc_main;
        p.gctl = j.gctl + 1;
        if (ev) cudaEventRecord(ev[2], st);
        if (launch_fmsm(j.k, p, shape, st) != cudaSuccess) return EIK_ECUDA;
        if (ev) cudaEventRecord(ev[3], st);
        ++nl;
    } else {
        if (solver_shape_f64(j.k, num_sms, n, j.sm_cap, sm, j.variant, &shape)) return EIK_ECUDA;
        p.inst = j.desc_main;
        p.gctl = j.gctl + 1;
        if (ev) cudaEventRecord(ev[2], st);
        if (launch_solver_f64(j.k, sm, p, shape, st) != cudaSuccess) return EIK_ECUDA;
        if (ev) cudaEventRecord(ev[3], st);
        ++nl;
    }
    if (!j.fp32 && !j.inst_done) {  // the pair modes' residual kernel writes the output
        if (launch_output(j.aux, j.blk_pre, n, j.nblocks, st) != cudaSuccess) return EIK_ECUDA;
        ++nl;
    }
    if (launches) *launches = nl;
    return EIK_OK;
}

int finish_instance(const JobDev& j, int i, const Layout& L, cudaStream_t st) {
    // a launch over one instance: its aux entry as entry 0, and the job's
    // block prefix, whose first element is 0 (a single instance reads no
    // owner table)
    const int nb = aux_blocks(L.nyp, L.nxp);
    const cudaError_t e = j.fp32 ? launch_residual(j.aux + i, j.blk_pre, 1, nb, st)
                                 : launch_output(j.aux + i, j.blk_pre, 1, nb, st);
    return e == cudaSuccess ? EIK_OK : EIK_ECUDA;
}

int finish_instances(const JobDev& j, cudaStream_t st) {
    const cudaError_t e = j.fp32 ? launch_residual(j.aux, j.blk_pre, j.n, j.nblocks, st)
                                 : launch_output(j.aux, j.blk_pre, j.n, j.nblocks, st);
    return e == cudaSuccess ? EIK_OK : EIK_ECUDA;
}

void block_resources(const void* fn, int threads, size_t dyn_smem, LaunchShape* s) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        s->regs_block = 1 << 30;  // unknown: never shares an SM
        s->smem_block = (size_t)1 << 40;
        return;
    }
    const int warps = (threads + 31) / 32;
    const int per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    s->regs_block = warps * per_warp;
    s->smem_block = fa.sharedSizeBytes + dyn_smem + 1024;
}

JobDev probe_job(int n, int k, bool fp32, bool one_pass, bool async_first, bool async_main, bool ordered,
                 int variant) {
    static unsigned long long dummy_ring[1];
    static unsigned dummy_bq[1];
    JobDev j{};
    j.n = n;
    j.k = k;
    j.fp32 = fp32;
    j.one_pass = fp32 && one_pass;
    j.async_first = async_first;
    j.async_main = async_main;
    j.ordered = ordered;
    j.variant = variant;
    j.ring = dummy_ring;  // the shapes only ask whether a ring exists
    j.bq = ordered ? dummy_bq : nullptr;
    return j;
}

bool job_footprint(const JobDev& j, int num_sms, Footprint* fp) {
    if (j.fmsm) return false;
    const bool am = j.async_main && j.ring && j.k >= 8;
    const int sm = !am ? SCH_ROUNDS
                   : j.ordered && j.bq && j.variant == VAR_HCM ? SCH_ORDERED
                                                               : SCH_FIFO;
    const int sf = !(j.async_first && j.ring && j.k >= 8) ? SCH_ROUNDS
                   : j.ordered && j.bq                    ? SCH_ORDERED
                                                          : SCH_FIFO;
    LaunchShape sh[2];
    int m = 0;
    if (j.fp32 && j.one_pass) {
        if (solver_shape_df(j.k, num_sms, j.n, 1, sm, VAR_HCM, &sh[m++])) return false;
    } else if (j.fp32) {
        if (solver_shape_f32(j.k, num_sms, j.n, 1, sf, VAR_HCM, &sh[m++]) ||
            solver_shape_df(j.k, num_sms, j.n, 1, sm, VAR_HCM, &sh[m++]))
            return false;
    } else {
        if (solver_shape_f64(j.k, num_sms, j.n, 1, sm, j.variant, &sh[m++])) return false;
    }
    Footprint f;
    f.per_sm = 1 << 30;
    for (int e = 0; e < m; ++e) {
        f.threads = std::max(f.threads, sh[e].threads);
        f.regs = std::max(f.regs, sh[e].regs_block);
        f.smem = std::max(f.smem, sh[e].smem_block);
        f.per_sm = std::min(f.per_sm, sh[e].per_sm);
    }
    if (f.per_sm < 1) return false;
    *fp = f;
    return true;
}

// ---------------------------------------------------------------- statistics
static double dval(unsigned long long k) {
    long long b = bits_from_key(k);
    double v;
    std::memcpy(&v, &b, 8);
    return v;
}

static void print_profile(const char* what, const Ctl* c) {
    const char* names[7] = {"split", "barrier", "list+pop", "tma", "sweeps", "writeback", "activate"};
    double tot = 0;
    for (int i = 0; i < 7; ++i) tot += (double)c->prof[i];
    std::fprintf(stderr, "[eik profile %s] rounds=%llu", what, (unsigned long long)c->rounds);
    for (int i = 0; i < 7; ++i)
        std::fprintf(stderr, " %s=%.1f%%", names[i], tot > 0 ? 100.0 * c->prof[i] / tot : 0.0);
    const double v = (double)c->prof[7];
    std::fprintf(stderr, " warp-visits=%.0f cyc/visit: sweeps=%.0f tma=%.0f act=%.0f pop=%.0f finish=%.0f\n", v,
                 v ? c->prof[4] / v : 0.0, v ? c->prof[3] / v : 0.0, v ? c->prof[6] / v : 0.0,
                 v ? c->prof[2] / v : 0.0, v ? c->prof[0] / v : 0.0);
    if (c->fronts || c->qev[1])
        std::fprintf(stderr,
                     "[eik queue %s] fronts=%llu handoffs=%llu claims=%llu tickets=%llu received=%llu gives=%llu "
                     "gone-skips=%llu puts=%llu given-back=%llu rare-checks=%llu\n",
                     what, (unsigned long long)c->fronts, (unsigned long long)c->handoffs,
                     (unsigned long long)c->qev[0], (unsigned long long)c->qev[1], (unsigned long long)c->qev[2],
                     (unsigned long long)c->qev[3], (unsigned long long)c->qev[4], (unsigned long long)c->qev[5],
                     (unsigned long long)c->qev[6], (unsigned long long)c->qev[7]);
}

void job_stats(const Layout& L, const eik_plan_desc* d, bool fp32, const Ctl* ictl_first,
               const Ctl* ictl_main, const Ctl* g_first, const Ctl* g_main, const ResidualOut* r,
               double q_min, double bw_main, double ms,
               eik_stats* st) {
    eik_stats s;
    std::memset(&s, 0, sizeof(s));
    int status = g_main->status ? g_main->status : ictl_main->status;
    if (fp32) {
        if (g_first->status) status = g_first->status;
        else if (ictl_first->status) status = ictl_first->status;
    }
    unsigned long long visits = ictl_main->visits, sweeps = ictl_main->sweeps, lane = ictl_main->lane_updates;
    long long rounds = (long long)g_main->rounds, adv = (long long)(ictl_main->advances + g_main->fronts);
    if (fp32) {
        visits += ictl_first->visits;
        sweeps += ictl_first->sweeps;
        lane += ictl_first->lane_updates;
        rounds += (long long)g_first->rounds;
        adv += (long long)ictl_first->advances;
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
    // pass times from the kernels' own timers (callers with events on the
    // launching stream replace them)
    auto span = [](const Ctl* g) {
        return g->t_end > g->t_start && g->t_start != ~0ull ? (double)(g->t_end - g->t_start) * 1e-6 : 0.0;
    };
    s.pass_ms[0] = fp32 ? span(g_first) : 0.0;
    s.pass_ms[1] = span(g_main);
    s.mono_pct = g_main->mono_n ? 100.0 * (double)g_main->mono_ok / (double)g_main->mono_n : 0.0;
    s.queue_left = (int64_t)r->n_left;
    const double fmin = dval(ictl_main->fmin_f);
    s.bucket_width = bw_main > 0 ? bw_main : (bw_main < 0 ? -bw_main : 4.0) * L.k * fmin;
    if (fp32) {
        // values on the device are U - q_min >= 0
        const double rr = dval(r->r_max), rrel = dval(r->r_rel), umax = dval(r->u_max);
        s.max_residual = rr;
        // Certificate (comparison principle for the monotone scheme): for
        // lam > 1, lam * (U - q_min) is a strict supersolution whose margin
        // at node x is (lam - 1) f(x) / sqrt 2, and likewise a strict
        // subsolution for lam < 1; a residual r(x) <= that margin at every x
        // keeps V between them, so
        //   |V - U| <= sqrt 2 * max_x (r(x) / f(x)) * max(U - q_min).
        double bound = 0.0;
        if (r->n_bad) bound = std::numeric_limits<double>::infinity();
        else if (rrel > 0 && umax > 0) bound = std::sqrt(2.0) * rrel * umax;
        const double scale = std::max(std::fabs(umax + q_min), std::fabs(q_min));
        s.err_bound = scale > 0 ? bound / scale : bound;
        const double tol = d->tol > 0 ? d->tol : 1e-5;
        if (status == EIK_OK && !(s.err_bound <= tol)) status = EIK_ENOTCONVERGED;
    }
    s.status = status;
    if (profiling()) {
        if (fp32) print_profile("fp32 pass", g_first);
        print_profile(fp32 ? "refinement pass" : "fp64 pass", g_main);
    }
    if (st) *st = s;
}

}  // namespace eik
