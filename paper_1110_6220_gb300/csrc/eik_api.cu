// eik_api.cu -- the C ABI (include/eik.h): plans, single solves and batches,
// all run as jobs (eik_job.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
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

static size_t a256(size_t b) { return (b + 255) / 256 * 256; }

bool desc_valid(const eik_plan_desc* d) {
    if (!d) return false;
    if (d->nx < 2 || d->ny < 2) return false;
    if (!(d->h > 0.0) || !std::isfinite(d->h)) return false;
    if (d->cell_k != 0 && d->cell_k != 4 && d->cell_k != 8 && d->cell_k != 16 && d->cell_k != 32 &&
        d->cell_k != 64)
        return false;
    if (d->precision != EIK_FP64 && d->precision != EIK_FP32_REFINE) return false;
    if (d->method != EIK_METHOD_HCM && d->method != EIK_METHOD_FHCM && d->method != EIK_METHOD_FMSM &&
        d->method != EIK_METHOD_HCM_LSM)
        return false;
    if (d->method != EIK_METHOD_HCM && d->precision != EIK_FP64) return false;
    if (d->method == EIK_METHOD_FMSM && d->cell_k != 0 && d->cell_k < 8) return false;
    if ((long long)d->nx * d->ny > (1ll << 31) - 1) return false;
    if (d->schedule < EIK_SCHED_AUTO || d->schedule > EIK_SCHED_ORDERED) return false;
    if (d->window < 0 || d->window > NBQ) return false;
    return true;
}

int default_k(const eik_plan_desc* d) { return choose_params(d, 1).k; }

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A host buffer the kernels can address in place -- pinned memory
// (cudaMallocHost, cudaHostAlloc, cudaHostRegister) -- has a device address
// for the current device: the init kernel then reads F, and the output kernel
// writes U, across the host link with no staging copy.  Null for device and
// pageable memory.
const void* host_mapped(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// EIK_ALLOC_LIMIT (bytes; unset: none): every workspace need above it fails
// as cudaMalloc would on a device that small, whether or not a buffer kept
// from an earlier call could serve it -- a host-side way to drive the
// EIK_ENOMEM paths without exhausting the device.
static size_t alloc_limit() {
    const char* e = std::getenv("EIK_ALLOC_LIMIT");
    return e && e[0] ? (size_t)std::strtoull(e, nullptr, 10) : ~(size_t)0;
}

int grow(DevBuf* b, size_t bytes) {
    if (bytes > alloc_limit()) return EIK_ENOMEM;
    if (b->cap >= bytes) return EIK_OK;
    if (b->p) cudaFree(b->p);
    b->p = nullptr;
    b->cap = 0;
    const size_t cap = std::max<size_t>(bytes + bytes / 8, 1 << 20);
    if (cudaMalloc(&b->p, cap) != cudaSuccess) {
        cudaGetLastError();
        return EIK_ENOMEM;
    }
    b->cap = cap;
    return EIK_OK;
}

// ---------------------------------------------------------------- sources
int prepare_sources(const Layout& L, const eik_instance* in, HostSources* hs) {
    const int n = in->nsrc;
    if (n < 0) return EIK_EINVAL;
    if (n > 0 && (!in->src_ij || !in->src_q)) return EIK_EINVAL;
    std::vector<int32_t> ij(2 * (size_t)n);
    std::vector<double> q((size_t)n);
    if (n > 0 && (cudaMemcpy(ij.data(), in->src_ij, ij.size() * 4, cudaMemcpyDefault) != cudaSuccess ||
                  cudaMemcpy(q.data(), in->src_q, q.size() * 8, cudaMemcpyDefault) != cudaSuccess)) {
        cudaGetLastError();
        return EIK_EINVAL;
    }
    return prepare_sources_host(L, n, ij.data(), q.data(), hs);
}

int prepare_sources_host(const Layout& L, int n, const int32_t* ij, const double* q, HostSources* hs) {
    hs->node.clear();
    hs->q.clear();
    hs->cell.clear();
    hs->cell_key.clear();
    hs->q_min = 0.0;
    if (n <= 0) return n < 0 ? EIK_EINVAL : EIK_OK;
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

// ---------------------------------------------------------------- jobs
int build_job(HostJob* hj, int n, const eik_plan_desc* descs, const eik_instance* in, const JobParams& P,
              bool fp32, long long deadline_ns, cudaStream_t st) {
    if (n < 1 || n > MAX_BATCH) return EIK_EINVAL;
    const int k = P.k;
    hj->bw_main.resize(n);
    std::vector<HostSources> hs((size_t)n);
    std::vector<char> stageF((size_t)n);
    std::vector<const double*> mapF((size_t)n, nullptr);  // pinned host F, U: their device addresses
    std::vector<double*> mapU((size_t)n, nullptr);
    hj->L.resize(n);
    hj->arr.resize(n);
    hj->shift.resize(n);
    hj->out_host.resize(n);
    hj->out_user.resize(n);
    size_t nsrc = 0, ncs = 0, Jtot = 0, ibytes = 0;
    std::vector<size_t> inst_off((size_t)n);
    // ---- the sources of every instance into one pinned staging buffer:
    // one asynchronous copy per array that lives on the device, one wait
    size_t sbytes = 0;
    std::vector<size_t> soff((size_t)n);
    for (int i = 0; i < n; ++i) {
        if (!in[i].F || !in[i].U || in[i].nsrc < 0) return EIK_EINVAL;
        if (in[i].nsrc > 0 && (!in[i].src_ij || !in[i].src_q)) return EIK_EINVAL;
        soff[i] = sbytes;
        sbytes += (size_t)in[i].nsrc * 16;  // 2 ints + 1 double per source
    }
    if (hj->src_cap < sbytes) {
        if (hj->src_host) cudaFreeHost(hj->src_host);
        hj->src_host = nullptr;
        hj->src_cap = 0;
        if (cudaMallocHost((void**)&hj->src_host, sbytes) != cudaSuccess) {
            cudaGetLastError();
            return EIK_ENOMEM;
        }
        hj->src_cap = sbytes;
    }
    bool waited = true;
    for (int i = 0; i < n; ++i) {
        const size_t m = (size_t)in[i].nsrc;
        if (!m) continue;
        char* dst = hj->src_host + soff[i];
        const bool dij = is_device_ptr(in[i].src_ij), dq = is_device_ptr(in[i].src_q);
        if (dij) {
            if (cudaMemcpyAsync(dst, in[i].src_ij, m * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
                cudaGetLastError();
                return EIK_EINVAL;
            }
            waited = false;
        } else {
            std::memcpy(dst, in[i].src_ij, m * 8);
        }
        if (dq) {
            if (cudaMemcpyAsync(dst + m * 8, in[i].src_q, m * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
                cudaGetLastError();
                return EIK_EINVAL;
            }
            waited = false;
        } else {
            std::memcpy(dst + m * 8, in[i].src_q, m * 8);
        }
    }
    if (!waited && cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return EIK_ECUDA;
    }
    for (int i = 0; i < n; ++i) {
        hj->L[i] = make_layout(descs[i].nx, descs[i].ny, k);
        const char* sp = hj->src_host + soff[i];
        const int rc = prepare_sources_host(hj->L[i], in[i].nsrc, (const int32_t*)sp,
                                            (const double*)(sp + (size_t)in[i].nsrc * 8), &hs[i]);
        if (rc) return rc;
        const bool dF = is_device_ptr(in[i].F), dU = is_device_ptr(in[i].U);
        mapF[i] = dF ? nullptr : (const double*)host_mapped(in[i].F);
        mapU[i] = dU ? nullptr : (double*)host_mapped(in[i].U);
        stageF[i] = !dF && !mapF[i];
        hj->out_host[i] = !dU && !mapU[i];
        hj->out_user[i] = in[i].U;
        hj->shift[i] = hs[i].node.empty() ? 0.0 : hs[i].q_min;
        nsrc += hs[i].node.size();
        ncs += hs[i].cell.size();
        Jtot += (size_t)hj->L[i].J;
        inst_off[i] = ibytes;
        ibytes += inst_bytes(hj->L[i], fp32, stageF[i], hj->out_host[i]);
    }
    // ---- arena: [tables | sources] [zero region] [cval] [instances]
    const size_t t_desc = a256((size_t)n * sizeof(InstDesc));
    const size_t t_aux = a256((size_t)n * sizeof(AuxInst));
    const size_t t_pre = a256((size_t)(n + 1) * 4);
    // block prefixes carry their owner tables (one int per block) behind them
    size_t nb_int = 0, nb_full = 0;
    for (int i = 0; i < n; ++i) {
        nb_int += (size_t)aux_blocks(hj->L[i].nyp, hj->L[i].nxp);
        nb_full += (size_t)aux_blocks(hj->L[i].urows, hj->L[i].upitch);
    }
    const size_t t_own_int = a256((size_t)(n + 1) * 4 + nb_int * 4);
    const size_t t_own_full = a256((size_t)(n + 1) * 4 + nb_full * 4);
    const size_t ns4 = a256(std::max(nsrc, ncs) * 4 + 4);
    const size_t t_src = a256(nsrc * 8 + 8) + a256(ncs * 8 + 8) + 4 * ns4;
    const size_t image_bytes = 2 * t_desc + t_aux + t_own_int + t_pre + t_own_full + t_src;
    const size_t z_ctl = a256((size_t)(2 * n + 2) * sizeof(Ctl) + (size_t)n * sizeof(ResidualOut));
    const size_t zero_bytes = z_ctl + a256(Jtot * 4) * 3 + a256(Jtot * 8);  // qflag, visits, FHCM flags, request times
    // ring of the round-free schedule: a power of two >= 16 times the job's
    // cells (a launch rarely pushes more, so pushes seldom wait for a slot)
    // and the warps of a launch, behind its three counters
    size_t Q = 8192;
    while (Q < 16 * Jtot) Q <<= 1;
    const size_t hist_bytes = a256((3 * 8192 + 1) * 4);
    // the value-ordered schedule's bucket rings: NBQ rings of a power of two
    // >= the job's cells (a cell sits in at most one ring at a time), behind
    // their header
    size_t BQ = 1024;
    while (BQ < Jtot) BQ <<= 1;
    const bool ordered = P.ordered && P.async_main && k >= 8 && Jtot < ((size_t)1 << 26);
    const size_t bq_bytes = ordered ? a256((size_t)BQ_WORDS * 4) + (size_t)NBQ * BQ * 8 : 0;
    const size_t ring_bytes = a256(384 + hist_bytes + Q * 8) + bq_bytes;
    // FMSM: coarse speeds and coarse values, one of each per cell
    const bool fmsm = descs[0].method == EIK_METHOD_FMSM;
    const size_t fm_bytes = fmsm ? 2 * a256(Jtot * 8) : 0;
    const size_t total = image_bytes + zero_bytes + a256(Jtot * 8) + ring_bytes + fm_bytes + ibytes + 256;
    int rc = grow(&hj->arena, total);
    if (rc) return rc;
    char* base = (char*)hj->arena.p;
    char* img_dev = base;
    char* zero_dev = base + image_bytes;
    char* cval_dev = zero_dev + zero_bytes;
    char* ring_dev = cval_dev + a256(Jtot * 8);
    char* fm_dev = ring_dev + ring_bytes;
    char* inst_dev = fm_dev + fm_bytes;

    hj->image.assign(image_bytes, 0);
    char* img = hj->image.data();
    InstDesc* desc_main_h = (InstDesc*)img;
    InstDesc* desc_f32_h = (InstDesc*)(img + t_desc);
    AuxInst* aux_h = (AuxInst*)(img + 2 * t_desc);
    const size_t o_blk = 2 * t_desc + t_aux, o_cpre = o_blk + t_own_int, o_full = o_cpre + t_pre;
    const size_t o_src = o_full + t_own_full;
    int* blk_pre_h = (int*)(img + o_blk);
    int* cell_pre_h = (int*)(img + o_cpre);
    int* blk_full_h = (int*)(img + o_full);
    char* src_h = img + o_src;
    const size_t o_q = 0, o_key = a256(nsrc * 8 + 8), o_node = o_key + a256(ncs * 8 + 8);
    const size_t o_ninst = o_node + ns4, o_cell = o_ninst + ns4, o_cinst = o_cell + ns4;

    Ctl* ictl_dev = (Ctl*)zero_dev;
    Ctl* gctl_dev = ictl_dev + 2 * n;
    ResidualOut* res_dev = (ResidualOut*)(gctl_dev + 2);
    int* qflag_all = (int*)(zero_dev + z_ctl);
    int* visits_all = (int*)(zero_dev + z_ctl + a256(Jtot * 4));
    int* dflags_all = (int*)(zero_dev + z_ctl + 2 * a256(Jtot * 4));
    unsigned long long* req_all = (unsigned long long*)(zero_dev + z_ctl + 3 * a256(Jtot * 4));
    unsigned long long* cval_all = (unsigned long long*)cval_dev;

    bool ok = true;
    size_t coff = 0, so = 0, co = 0;
    int boff = 0, bfull = 0;
    for (int i = 0; i < n; ++i) {
        const Layout& L = hj->L[i];
        InstArrays a = carve_inst(L, fp32, stageF[i], hj->out_host[i], inst_dev + inst_off[i]);
        a.cval = cval_all + coff;
        a.qflag = qflag_all + coff;
        a.visits = visits_all + coff;
        a.dflags = dflags_all + coff;
        hj->arr[i] = a;
        const double* F = stageF[i] ? a.Fstage : mapF[i] ? mapF[i] : in[i].F;
        double* out = hj->out_host[i] ? a.Ostage : mapU[i] ? mapU[i] : in[i].U;
        const double bw = descs[i].bucket_width;
        hj->bw_main[i] = bw != 0.0 ? bw : P.w_main;
        fill_inst_tables(L, a, fp32, descs[i].h, bw != 0.0 ? bw : P.w_first, hj->bw_main[i], &ictl_dev[i],
                         &ictl_dev[n + i],
                         &res_dev[i], F, out, hj->shift[i], &aux_h[i], &desc_main_h[i], &desc_f32_h[i], &ok);
        if (fp32 && P.one_pass) {
            // the source cells are queued for the double-float pass itself,
            // and nothing reads the FP32 pass's arrays
            aux_h[i].ctl = &ictl_dev[n + i];
            aux_h[i].ctl2 = nullptr;
            aux_h[i].f32 = nullptr;
            aux_h[i].U32 = nullptr;
        }
        aux_h[i].Fc = fmsm ? (double*)fm_dev + coff : nullptr;
        aux_h[i].Uc = fmsm ? (double*)(fm_dev + a256(Jtot * 8)) + coff : nullptr;
        desc_main_h[i].cell_base = (int)coff;
        desc_main_h[i].done = hj->done_dev ? hj->done_dev + i : nullptr;
        if (fp32) desc_f32_h[i].cell_base = (int)coff;
        blk_pre_h[i] = boff;
        boff += aux_blocks(L.nyp, L.nxp);
        blk_full_h[i] = bfull;
        bfull += aux_blocks(L.urows, L.upitch);
        // the owner tables behind the prefixes (instance of each block); a
        // job of one instance reads none
        if (n > 1) {
            for (int b = blk_pre_h[i]; b < boff; ++b) blk_pre_h[n + 1 + b] = i;
            for (int b = blk_full_h[i]; b < bfull; ++b) blk_full_h[n + 1 + b] = i;
        }
        cell_pre_h[i] = (int)coff;
        coff += (size_t)L.J;
        for (size_t e = 0; e < hs[i].node.size(); ++e, ++so) {
            ((double*)(src_h + o_q))[so] = hs[i].q[e];
            ((int*)(src_h + o_node))[so] = hs[i].node[e];
            ((int*)(src_h + o_ninst))[so] = i;
        }
        for (size_t e = 0; e < hs[i].cell.size(); ++e, ++co) {
            ((unsigned long long*)(src_h + o_key))[co] = hs[i].cell_key[e];
            ((int*)(src_h + o_cell))[co] = hs[i].cell[e];
            ((int*)(src_h + o_cinst))[co] = i;
        }
    }
    blk_pre_h[n] = boff;
    blk_full_h[n] = bfull;
    cell_pre_h[n] = (int)coff;
    if (!ok) return EIK_ECUDA;
    if (cudaMemcpyAsync(img_dev, img, image_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return EIK_ECUDA;
    for (int i = 0; i < n; ++i)
        if (stageF[i] && cudaMemcpyAsync(hj->arr[i].Fstage, in[i].F, (size_t)descs[i].nx * descs[i].ny * 8,
                                         cudaMemcpyHostToDevice, st) != cudaSuccess)
            return EIK_ECUDA;

    JobDev& j = hj->j;
    j.n = n;
    j.k = k;
    j.fp32 = fp32;
    j.desc_main = (InstDesc*)img_dev;
    j.desc_f32 = (InstDesc*)(img_dev + t_desc);
    j.aux = (AuxInst*)(img_dev + 2 * t_desc);
    j.blk_pre = (int*)(img_dev + o_blk);
    j.cell_pre = (int*)(img_dev + o_cpre);
    j.blk_full = (int*)(img_dev + o_full);
    j.nblocks = boff;
    j.nblocks_full = bfull;
    j.ncells = (int)coff;
    j.ictl = ictl_dev;
    j.gctl = gctl_dev;
    j.res = res_dev;
    char* src_dev = img_dev + o_src;
    j.src.q = (const double*)(src_dev + o_q);
    j.src.node = (const int*)(src_dev + o_node);
    j.src.node_inst = (const int*)(src_dev + o_ninst);
    j.src.n = (int)nsrc;
    j.src.cell_key = (const unsigned long long*)(src_dev + o_key);
    j.src.cell = (const int*)(src_dev + o_cell);
    j.src.cell_inst = (const int*)(src_dev + o_cinst);
    j.src.ncell = (int)ncs;
    j.nsrc_total = (int)nsrc;
    j.ncell_total = (int)ncs;
    j.deadline_ns = deadline_ns;
    j.sm_cap = 0;
    j.one_pass = fp32 && P.one_pass;
    j.variant = descs[0].method == EIK_METHOD_FHCM      ? VAR_FHCM
                : descs[0].method == EIK_METHOD_HCM_LSM ? VAR_LSM
                                                        : VAR_HCM;
    j.fmsm = fmsm;
    j.coarse = nullptr;
    j.hold_ns = P.hold_ns;
    j.req_time = req_all;
    j.async_first = P.async_first;
    j.async_main = P.async_main;
    j.qctl = (unsigned*)ring_dev;
    j.hist = (int*)(ring_dev + 384);
    j.ring = (unsigned long long*)(ring_dev + 384 + hist_bytes);
    j.ring_mask = (unsigned)(Q - 1);
    j.ordered = ordered;
    // per-instance completion needs the main pass round-free in one launch:
    // the one-pass FP32_REFINE form or FP64 HCM-family methods, cells >= 8
    j.inst_done = hj->done_dev && P.async_main && k >= 8 && !fmsm && (!fp32 || P.one_pass);
    j.window = P.window;
    j.bq = ordered ? (unsigned*)(ring_dev + a256(384 + hist_bytes + Q * 8)) : nullptr;
    j.bq_data = ordered ? (unsigned long long*)((char*)j.bq + a256((size_t)BQ_WORDS * 4)) : nullptr;
    j.bq_mask = ordered ? (unsigned)(BQ - 1) : 0u;
    j.zero_base = zero_dev;
    j.zero_bytes = zero_bytes;
    j.cval_all = cval_all;
    j.ncval = Jtot;
    j.qflag_all = qflag_all;
    j.visits_all = visits_all;
    // pinned readback buffer for the control blocks
    if (hj->zero_cap < z_ctl) {
        if (hj->zero_host) cudaFreeHost(hj->zero_host);
        hj->zero_host = nullptr;
        hj->zero_cap = 0;
        if (cudaMallocHost((void**)&hj->zero_host, z_ctl) != cudaSuccess) {
            cudaGetLastError();
            return EIK_ENOMEM;
        }
        hj->zero_cap = z_ctl;
    }
    if (fmsm) {
        // Part I's problem: per instance the grid of cell centres (spacing
        // k h, speeds from k_fmsm_coarse_speed), with the cells that hold
        // sources as its exit set at their sources' q (the job keeps the
        // smallest per node); solved exactly, its values land in Uc
        if (!hj->coarse) hj->coarse = new (std::nothrow) HostJob();
        if (!hj->coarse) return EIK_ENOMEM;
        std::vector<eik_plan_desc> cd((size_t)n);
        std::vector<eik_instance> ci((size_t)n);
        std::vector<std::vector<int32_t>> cij((size_t)n);
        for (int i = 0; i < n; ++i) {
            const Layout& L = hj->L[i];
            cd[i] = descs[i];
            cd[i].nx = L.cxn;
            cd[i].ny = L.cyn;
            cd[i].h = descs[i].h * k;
            cd[i].cell_k = 0;
            cd[i].bucket_width = 0.0;
            cd[i].precision = EIK_FP64;
            cd[i].method = EIK_METHOD_HCM;
            const int m = in[i].nsrc;
            const int32_t* ij = (const int32_t*)(hj->src_host + soff[i]);
            cij[i].resize((size_t)2 * m + 2);
            for (int s = 0; s < 2 * m; ++s) cij[i][s] = ij[s] / k;
            ci[i] = in[i];
            ci[i].F = aux_h[i].Fc;
            ci[i].U = aux_h[i].Uc;
            ci[i].src_ij = cij[i].data();
            ci[i].src_q = (const double*)(hj->src_host + soff[i] + (size_t)m * 8);
        }
        // the coarse sources' q are read from this job's staging buffer
        // (pinned host memory) while the coarse job copies them into its own
        const JobParams Pc = choose_params(cd.data(), n);
        rc = build_job(hj->coarse, n, cd.data(), ci.data(), Pc, false, deadline_ns, st);
        if (rc) return rc;
        j.coarse = &hj->coarse->j;
    }
    return EIK_OK;
}

int finish_job(HostJob* hj, const eik_plan_desc* descs, cudaStream_t st, double ms, eik_stats* st_out) {
    const JobDev& j = hj->j;
    const int n = j.n;
    for (int i = 0; i < n; ++i)
        if (hj->out_host[i])
            cudaMemcpyAsync(hj->out_user[i], hj->arr[i].Ostage, (size_t)hj->L[i].nx * hj->L[i].ny * 8,
                            cudaMemcpyDeviceToHost, st);
    const size_t rb = (size_t)(2 * n + 2) * sizeof(Ctl) + (size_t)n * sizeof(ResidualOut);
    cudaMemcpyAsync(hj->zero_host, j.zero_base, rb, cudaMemcpyDeviceToHost, st);
    const bool fmsm = j.fmsm && hj->coarse;
    if (fmsm) cudaMemcpyAsync(hj->coarse->zero_host, hj->coarse->j.zero_base, rb, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return EIK_ECUDA;
    }
    const Ctl* ic = (const Ctl*)hj->zero_host;
    const Ctl* g = ic + 2 * n;
    const ResidualOut* r = (const ResidualOut*)(g + 2);
    int first_err = EIK_OK;
    for (int i = 0; i < n; ++i) {
        eik_stats s;
        job_stats(hj->L[i], &descs[i], j.fp32, &ic[i], &ic[n + i], &g[0], &g[1], &r[i], hj->shift[i],
                  hj->bw_main[i], ms, &s);
        s.schedule = (j.fp32 && !j.one_pass && j.async_first && j.k >= 8 ? 1 : 0) |
                     (j.async_main && j.k >= 8 && !j.fmsm ? 2 : 0) | (j.one_pass ? 4 : 0) | (j.fmsm ? 16 : 0) |
                     (j.ordered && j.variant == VAR_HCM && !j.fmsm ? 32 : 0);
        if (fmsm && !s.status) {
            // a failed coarse solve fails the instance
            const Ctl* cc = (const Ctl*)hj->coarse->zero_host;
            const int cs = cc[2 * n + 1].status ? cc[2 * n + 1].status : cc[n + i].status;
            if (cs) s.status = cs;
        }
        if (st_out) st_out[i] = s;
        if (s.status && !first_err) first_err = s.status;
    }
    return first_err;
}

void free_job(HostJob* hj) {
    if (hj->coarse) {
        free_job(hj->coarse);
        delete hj->coarse;
        hj->coarse = nullptr;
    }
    if (hj->arena.p) cudaFree(hj->arena.p);
    hj->arena.p = nullptr;
    hj->arena.cap = 0;
    if (hj->zero_host) cudaFreeHost(hj->zero_host);
    hj->zero_host = nullptr;
    hj->zero_cap = 0;
    if (hj->src_host) cudaFreeHost(hj->src_host);
    hj->src_host = nullptr;
    hj->src_cap = 0;
}

int run_job(HostJob* hj, int n, const eik_plan_desc* descs, const eik_instance* in, const JobParams& P,
            bool fp32, long long deadline_ns, int num_sms, cudaStream_t s, cudaEvent_t* ev,
            eik_stats* st_out, float* t) {
    int rc = build_job(hj, n, descs, in, P, fp32, deadline_ns, s);
    int nl = 0;
    if (!rc) {
        cudaEventRecord(ev[0], s);
        rc = enqueue_job(hj->j, num_sms, s, ev + 2, &nl);
        cudaEventRecord(ev[1], s);
    }
    if (rc) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return rc;
    }
    rc = finish_job(hj, descs, s, 0.0, st_out);
    float ms = 0.f, p0 = 0.f, p1 = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (fp32 || hj->j.fmsm) cudaEventElapsedTime(&p0, ev[2], ev[3]);
    cudaEventElapsedTime(&p1, ev[4], ev[5]);
    if (st_out)
        for (int e = 0; e < n; ++e) {
            st_out[e].ms = ms;  // the whole job (all of its instances)
            st_out[e].mpts_per_s = ms > 0 ? (double)descs[e].nx * descs[e].ny / ms / 1000.0 : 0.0;
            st_out[e].pass_ms[0] = p0;
            st_out[e].pass_ms[1] = p1;
            st_out[e].launches = nl;
        }
    if (t) t[0] = ms, t[1] = p0, t[2] = p1;
    return rc;
}

}  // namespace eik

// ================================================================= plans
namespace {
// Arena bytes of a one-instance job for *d (build_job's layout, rounded up)
size_t job_bytes(const eik_plan_desc* d) {
    const Layout L = make_layout(d->nx, d->ny, default_k(d));
    const bool fp32 = d->precision == EIK_FP32_REFINE;
    size_t Q = 8192;
    while (Q < 16 * (size_t)L.J) Q <<= 1;
    size_t BQ = 1024;
    while (BQ < (size_t)L.J) BQ <<= 1;
    size_t b = inst_bytes(L, fp32, true, true) + (size_t)L.J * 16 + Q * 8 + 128 * 1024;
    const JobParams P = choose_params(d, 1);
    if (P.ordered && P.async_main && P.k >= 8) b += (size_t)NBQ * BQ * 8 + 1024;
    if (d->method == EIK_METHOD_FMSM) b += (size_t)L.J * 16 + 512;  // coarse speeds and values
    return b;
}
// FMSM: the descriptor of the coarse grid's job (as build_job forms it)
eik_plan_desc coarse_desc(const eik_plan_desc* d) {
    const int k = default_k(d);
    const Layout L = make_layout(d->nx, d->ny, k);
    eik_plan_desc c = *d;
    c.nx = L.cxn;
    c.ny = L.cyn;
    c.h = d->h * k;
    c.cell_k = 0;
    c.bucket_width = 0.0;
    c.precision = EIK_FP64;
    c.method = EIK_METHOD_HCM;
    return c;
}
}  // namespace

extern "C" size_t eik_plan_workspace_bytes(const eik_plan_desc* d) {
    if (!desc_valid(d)) return 0;
    size_t b = job_bytes(d);
    if (d->method == EIK_METHOD_FMSM) {
        const eik_plan_desc c = coarse_desc(d);
        b += job_bytes(&c);
    }
    return b;
}

extern "C" int eik_plan_create(eik_plan* out, const eik_plan_desc* d, void* cuda_stream) {
    if (!out) return EIK_EINVAL;
    *out = nullptr;
    if (!desc_valid(d)) return EIK_EINVAL;
    eik_plan_s* p = new (std::nothrow) eik_plan_s();
    if (!p) return EIK_ENOMEM;
    p->d = *d;
    p->P = choose_params(d, 1);
    p->d.cell_k = p->P.k;
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
            cudaGetLastError();
            delete p;
            return EIK_ECUDA;
        }
        p->own_stream = true;
    }
    int rc = EIK_OK;
    if (cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess) rc = EIK_ECUDA;
    for (int e = 0; e < 4 && !rc; ++e)
        if (cudaEventCreate(&p->pev[e]) != cudaSuccess) rc = EIK_ECUDA;
    // reserve the workspace now, so that solves do not allocate (FMSM: the
    // coarse grid's job too)
    if (!rc) rc = grow(&p->job.arena, job_bytes(&p->d));
    if (!rc && p->d.method == EIK_METHOD_FMSM) {
        p->job.coarse = new (std::nothrow) HostJob();
        const eik_plan_desc c = coarse_desc(&p->d);
        rc = p->job.coarse ? grow(&p->job.coarse->arena, job_bytes(&c)) : EIK_ENOMEM;
    }
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
    free_job(&p->job);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    for (int e = 0; e < 4; ++e)
        if (p->pev[e]) cudaEventDestroy(p->pev[e]);
    if (p->own_stream) cudaStreamDestroy(p->stream);
    delete p;
}

extern "C" int eik_solve(eik_plan p, const eik_instance* in, eik_stats* st) {
    if (!p || !in || !in->F || !in->U || in->nsrc < 0) return EIK_EINVAL;
    cudaSetDevice(p->device);
    cudaStream_t s = p->stream;
    const bool fp32 = p->d.precision == EIK_FP32_REFINE;
    int rc = build_job(&p->job, 1, &p->d, in, p->P, fp32, p->d.deadline_ns, s);
    if (rc) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return rc;
    }
    cudaEventRecord(p->ev0, s);
    int nl = 0;
    rc = enqueue_job(p->job.j, p->num_sms, s, p->pev, &nl);
    if (rc) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return rc;
    }
    cudaEventRecord(p->ev1, s);
    eik_stats local;
    finish_job(&p->job, &p->d, s, 0.0, &local);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p->ev0, p->ev1);
    local.ms = ms;
    local.mpts_per_s = ms > 0 ? (double)p->d.nx * p->d.ny / ms / 1000.0 : 0.0;
    if (fp32 || p->job.j.fmsm) cudaEventElapsedTime(&ms, p->pev[0], p->pev[1]), local.pass_ms[0] = ms;
    cudaEventElapsedTime(&ms, p->pev[2], p->pev[3]);
    local.pass_ms[1] = ms;
    local.launches = nl;
    if (st) *st = local;
    return local.status;
}

// ================================================================= batches
namespace {
struct BatchCtx {
    std::mutex mu;
    HostJob job;
    cudaEvent_t ev[6] = {};
    int num_sms = 0;
};
std::mutex g_batch_mu;
std::map<int, BatchCtx*> g_batch;

BatchCtx* batch_ctx(int dev) {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    auto it = g_batch.find(dev);
    if (it != g_batch.end()) return it->second;
    BatchCtx* c = new (std::nothrow) BatchCtx();
    if (!c) return nullptr;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    for (auto& e : c->ev) cudaEventCreate(&e);
    g_batch[dev] = c;
    return c;
}
}  // namespace

extern "C" int eik_solve_batch(const eik_plan_desc* d, const eik_instance* in, int32_t n_inst,
                               eik_stats* st, void* cuda_stream) {
    if (n_inst < 0 || (n_inst > 0 && (!d || !in))) return EIK_EINVAL;
    if (n_inst == 0) return EIK_OK;
    for (int i = 0; i < n_inst; ++i)
        if (!desc_valid(&d[i])) return EIK_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return EIK_ECUDA;
    }
    BatchCtx* ctx = batch_ctx(dev);
    if (!ctx) return EIK_ENOMEM;
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // group the instances by (cell_k as given, precision): instances that
    // leave cell_k at 0 are grouped together and get the tuned choice for
    // the group; each group runs as jobs of at most MAX_BATCH instances, one
    // persistent launch per pass
    std::map<std::pair<int, int>, std::vector<int>> groups;
    for (int i = 0; i < n_inst; ++i)
        groups[{d[i].cell_k, d[i].precision + 2 * d[i].method}].push_back(i);
    int first_err = EIK_OK;
    std::vector<eik_plan_desc> gd;
    std::vector<eik_instance> gi;
    std::vector<eik_stats> gs;
    for (auto& kv : groups) {
        const bool fp32 = kv.first.second % 2 == EIK_FP32_REFINE;
        const std::vector<int>& idx = kv.second;
        for (size_t b0 = 0; b0 < idx.size(); b0 += MAX_BATCH) {
            const int m = (int)std::min<size_t>(MAX_BATCH, idx.size() - b0);
            gd.resize(m);
            gi.resize(m);
            gs.resize(m);
            for (int e = 0; e < m; ++e) {
                gd[e] = d[idx[b0 + e]];
                gi[e] = in[idx[b0 + e]];
            }
            const JobParams P = choose_params(gd.data(), m);
            for (int e = 0; e < m; ++e) gd[e].cell_k = P.k;
            int rc = run_job(&ctx->job, m, gd.data(), gi.data(), P, fp32, d[0].deadline_ns, ctx->num_sms, s,
                             ctx->ev, gs.data(), nullptr);
            if (st)
                for (int e = 0; e < m; ++e) st[idx[b0 + e]] = gs[e];
            if (rc && !first_err) first_err = rc;
        }
    }
    return first_err;
}
