// eik_solver.cuh -- the persistent, bucketed cell solver (templated on the
// value type T and the cell size K).  Included by eik_solver_f64.cu and
// eik_solver_f32.cu, which instantiate it.
//
// What one launch computes (Chacon & Vladimirsky, Sec. 4.2):
//   Alg. generic_LC_cells with the HCM refinements -- cells carry cell values
//   (eq. cell_value) and four directional flags (Remark HCM_preferred_sweeps);
//   a removed cell is swept to convergence with its preferred directions first
//   and the Alg. FSM_order cycle afterwards; a changed boundary value V_i with
//   V_i < V_j (x_j across the boundary, not in Q) activates the neighbour.
// GPU recast: instead of popping the single smallest cell from a heap, every
// queued cell whose value lies within `delta` of the smallest one is released
// at once (one "bucket"), and the bucket's cells are processed concurrently
// by all warps.  Re-activations that fall inside the current bucket are
// processed in the next round; the others wait in a far list.  Theorem
// convergence (any removal order, exact per-cell solves) makes the result the
// exact solution of eq. Eik_discr regardless of this schedule.
#pragma once

#include "eik_common.cuh"

namespace eik {

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// 2-D tiled TMA load (no multicast) of one box into shared memory, completing
// on the mbarrier `bar`.  x must be a multiple of 16 bytes / sizeof(T).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"((unsigned long long)tm), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ int ld_cg(const int* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ld_cg(const unsigned long long* p) {
    return __ldcg(p);
}
__device__ __forceinline__ int ld_vol(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ unsigned ld_vol(const unsigned* p) {
    return *(const volatile unsigned*)p;
}

template <typename T> __device__ __forceinline__ T inf_of();
template <> __device__ __forceinline__ double inf_of<double>() {
    return __longlong_as_double(0x7ff0000000000000LL);
}
template <> __device__ __forceinline__ float inf_of<float>() {
    return __int_as_float(0x7f800000);
}

// ---------------------------------------------------------------- local update
// The update at one node from its four neighbours, using the relevant-quadrant
// shortcut of Remark regular_FSM_update: a = min(U_W, U_E), b = min(U_S, U_N).
// If |a - b| < f the two-sided root of (U-a)^2 + (U-b)^2 = f^2
// (eq. two_sided_update), else the one-sided min(a, b) + f
// (eq. one_sided_update).  Callers skip sources and obstacles (f < 0 or
// f = +inf), so f is finite and positive here.
__device__ __forceinline__ double local_update(double W, double E, double S, double N,
                                               double f) {
    const double a = fmin(W, E), b = fmin(S, N);
    const double lo = fmin(a, b);
    const double d = a - b;  // NaN only when a = b = +inf, then the one-sided branch
    const double one = lo + f;
    const double two = (a + b + sqrt(fma(-d, d, 2.0 * f * f))) * 0.5;
    return fabs(d) < f ? two : one;
}
// FP32: the same root in the cancellation-free form
//   max(a,b) + (f^2 - d^2) / (d + sqrt(2 f^2 - d^2)),  d = |a - b|,
// where the small increment carries all the rounding; the quotient and root
// only need a few correct bits relative to f, far below ulp(U).
__device__ __forceinline__ float local_update(float W, float E, float S, float N, float f) {
    const float a = fminf(W, E), b = fminf(S, N);
    const float lo = fminf(a, b), hi = fmaxf(a, b);
    const float d = hi - lo;
    const float one = lo + f;
    const float root = __fsqrt_rn(fmaf(-d, d, 2.0f * f * f));
    const float two = hi + __fdividef((f - d) * (f + d), d + root);
    return d < f ? two : one;
}

// ---------------------------------------------------------------- tile config
template <typename T, int K>
struct TileCfg {
    static constexpr int LPC = K >= 32 ? 32 : K;        // lanes per cell
    static constexpr int CPW = 32 / LPC;                // cells per warp (lock-step)
    static constexpr int RPL = K > 32 ? K / 32 : 1;     // rows per lane
    // U box: rows k+2; width k+2 for FP64 (multiple of 16 B since k is even),
    // k+4 for FP32 (k+2 floats is not a multiple of 16 B for k = 4m).
    static constexpr int BW = sizeof(T) == 8 ? K + 2 : K + 4;
    static constexpr int BH = K + 2;
    static constexpr int UBYTES = BW * BH * (int)sizeof(T);
    static constexpr int FBYTES = K * K * (int)sizeof(T);
    static constexpr int UBYTES_AL = (UBYTES + 127) / 128 * 128;
    static constexpr int FBYTES_AL = (FBYTES + 127) / 128 * 128;
    static constexpr int GROUP_BYTES = UBYTES_AL + FBYTES_AL;
    static constexpr int MASK_OFF = CPW * GROUP_BYTES;
    static constexpr int BAR_OFF = MASK_OFF + CPW * K * 8;
    static constexpr int WARP_BYTES = (BAR_OFF + 16 + 127) / 128 * 128;
    static constexpr int WPB_SMEM = (200 * 1024) / WARP_BYTES;
    static constexpr int WPB = WPB_SMEM >= 8 ? 8 : (WPB_SMEM < 1 ? 1 : WPB_SMEM);
    static constexpr int MAX_SWEEPS = 4 * K * K + 8;
};

// ---------------------------------------------------------------- grid barrier
// Sense-counting barrier across all (co-resident) blocks.  Every wait is
// bounded by the launch deadline and by the abort flag; on expiry the block
// records EIK_ETIMEDOUT, raises abort and returns false.
__device__ __forceinline__ bool grid_sync(Ctl* ctl, unsigned long long deadline, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = ld_vol(&ctl->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            unsigned spins = 0;
            while (ld_vol(&ctl->bar_gen) == gen) {
                if ((++spins & 63u) == 0) {
                    if (ld_vol(&ctl->abort)) break;
                    if (gtimer() > deadline) {
                        atomicCAS(&ctl->status, 0, EIK_ETIMEDOUT);
                        atomicExch(&ctl->abort, 1);
                        break;
                    }
                }
            }
        }
        __threadfence();
        *s_flag = ld_vol(&ctl->abort);
    }
    __syncthreads();
    return *s_flag == 0;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

__device__ __forceinline__ void fail(Ctl* ctl, int code, unsigned long long info) {
    if (atomicCAS(&ctl->status, 0, code) == 0) ctl->err_info = info;
    atomicExch(&ctl->abort, 1);
}

// warp-aggregated append of `val` (where pred) to a list of capacity cap
__device__ __forceinline__ void warp_push(int* list, int* count, bool pred, int val, int cap,
                                          Ctl* ctl) {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) {
        const int pos = base + __popc(m & ((1u << lane) - 1u));
        if (pos < cap) list[pos] = val;
        else fail(ctl, EIK_ECUDA, 0x1000000ull + (unsigned)pos);
    }
}

__device__ __forceinline__ void lane_push(int* list, int* count, int val, int cap, Ctl* ctl) {
    const int pos = atomicAdd(count, 1);
    if (pos < cap) list[pos] = val;
    else fail(ctl, EIK_ECUDA, 0x2000000ull + (unsigned)pos);
}

// ---------------------------------------------------------------- the kernel
template <typename T, int K>
__global__ void __launch_bounds__(TileCfg<T, K>::WPB * 32)
    k_solve(const __grid_constant__ SolveParams<T> p) {
    using C = TileCfg<T, K>;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_flag;
    // TMA destinations must be 128-byte aligned: the host asks for 128 spare bytes
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char* wbase = smem + warp * C::WARP_BYTES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(wbase + C::BAR_OFF);
    unsigned long long* masks = reinterpret_cast<unsigned long long*>(wbase + C::MASK_OFF);
    const int g = lane / C::LPC;   // which of the warp's cells this lane works on
    const int r0 = lane % C::LPC;  // first tile row of this lane
    T* tU = reinterpret_cast<T*>(wbase + g * C::GROUP_BYTES);
    T* tF = reinterpret_cast<T*>(wbase + g * C::GROUP_BYTES + C::UBYTES_AL);
    const unsigned gmask = C::LPC == 32 ? FULL : (((1u << C::LPC) - 1u) << (g * C::LPC));

    Ctl* ctl = p.ctl;
    const unsigned long long deadline = gtimer() + (unsigned long long)p.deadline_ns;
    const T INF = inf_of<T>();

    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;

    // bucket width: given, else k times the smallest h/F
    double delta = p.delta;
    if (!(delta > 0.0)) delta = (double)K * val_of(ld_cg(&ctl->fmin_f));
    if (!(delta > 0.0) || !(delta < inf_of<double>())) delta = inf_of<double>();
    const double fmin_glob = val_of(ld_cg(&ctl->fmin_f));

    const int J = p.J;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gthreads = gridDim.x * blockDim.x;

    unsigned long long st_visits = 0, st_sweeps = 0, st_lane = 0, st_rounds = 0, st_adv = 0;
    int ns = 0, fs = 0, round = 0;
    unsigned long long theta = 0;
    bool ok = true;

    for (;;) {
        int n_near = min(ld_cg(&ctl->cnt[ns]), J);  // a list never exceeds J entries
        if (n_near == 0) {
            const int nfar = min(ld_cg(&ctl->fcnt[fs]), J);
            if (nfar == 0) break;  // every list empty: converged
            // --- release the next bucket: min key over the far list ...
            const int* far = p.lists + (3 + fs) * J;
            unsigned long long mn = KEY_UNSET;
            for (int e = gtid; e < nfar; e += gthreads) {
                const unsigned long long kk = ld_cg(&p.cval[ld_cg(&far[e])]);
                mn = kk < mn ? kk : mn;
            }
            mn = warp_min_u64(mn);
            if (lane == 0 && mn != KEY_UNSET) atomicMin(&ctl->fmin[fs], mn);
            if (!(ok = grid_sync(ctl, deadline, &s_flag))) break;
            const unsigned long long fm = ld_cg(&ctl->fmin[fs]);
            theta = fm == KEY_UNSET ? KEY_UNSET : key_of(val_of(fm) + delta);
            // ... then move every far cell with key <= theta to the near list
            int* far2 = p.lists + (3 + (fs ^ 1)) * J;
            int* nearL = p.lists + ns * J;
            for (int e0 = gtid - lane; e0 < nfar; e0 += gthreads) {
                const int e = e0 + lane;
                int c = -1;
                bool to_near = false;
                if (e < nfar) {
                    c = ld_cg(&far[e]);
                    to_near = ld_cg(&p.cval[c]) <= theta;
                }
                warp_push(nearL, &ctl->cnt[ns], c >= 0 && to_near, c, J, ctl);
                warp_push(far2, &ctl->fcnt[fs ^ 1], c >= 0 && !to_near, c, J, ctl);
            }
            if (!(ok = grid_sync(ctl, deadline, &s_flag))) break;
            if (gtid == 0) {
                ctl->fcnt[fs] = 0;
                ctl->fmin[fs] = KEY_UNSET;
            }
            fs ^= 1;
            ++st_adv;
            n_near = min(ld_cg(&ctl->cnt[ns]), J);
        }

        // --- one round: process every cell of the near list
        const int nx_slot = ns == 2 ? 0 : ns + 1;
        // deadline, grid-uniformly: raised here, seen by all at this round's barrier
        if (gtid == 0 && gtimer() > deadline) fail(ctl, EIK_ETIMEDOUT, 0x5000000ull);
        if (gtid == 0) {
            ctl->cnt[nx_slot == 2 ? 0 : nx_slot + 1] = 0;  // the list consumed last round
            ctl->cursor[(round + 1) & 1] = 0;
        }
        const int* nearL = p.lists + ns * J;
        int* nextL = p.lists + nx_slot * J;
        int* farL = p.lists + (3 + fs) * J;
        int* next_cnt = &ctl->cnt[nx_slot];
        int* far_cnt = &ctl->fcnt[fs];

        for (;;) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&ctl->cursor[round & 1], C::CPW);
            base = __shfl_sync(FULL, base, 0);
            if (base >= n_near) break;
            const int idx = base + g;
            const int c = idx < n_near ? ld_cg(&nearL[idx]) : -1;
            int cg[C::CPW];
#pragma unroll
            for (int gg = 0; gg < C::CPW; ++gg) cg[gg] = __shfl_sync(FULL, c, gg * C::LPC);

            // ---- remove the cell from the list: clear its flag BEFORE reading
            // its halo, so that a neighbour that improves the halo while we
            // work re-queues it (Alg. generic_LC_cells, activation test)
            int dm = 0, first = 0;
            if (r0 == 0 && c >= 0) {
                atomicExch(&p.qflag[c], 0);
                dm = atomicExch(&p.dirmask[c], 0);
                first = atomicAdd(&p.visits[c], 1) == 0;
            }
            dm = __shfl_sync(FULL, dm, g * C::LPC);
            first = __shfl_sync(FULL, first, g * C::LPC);
            __threadfence();
            fence_proxy_async_global();
            fence_proxy_async_shared();
            __syncwarp();

            // ---- TMA: (k+2) x BW box of U (cell + halo) and k x k box of f
            if (lane == 0) {
                int nvalid = 0;
#pragma unroll
                for (int gg = 0; gg < C::CPW; ++gg) nvalid += cg[gg] >= 0;
                mbar_arrive_expect_tx(bar, (uint32_t)(nvalid * (C::UBYTES + C::FBYTES)));
#pragma unroll
                for (int gg = 0; gg < C::CPW; ++gg) {
                    if (cg[gg] >= 0) {
                        const int cx = cg[gg] % p.cxn, cy = cg[gg] / p.cxn;
                        unsigned char* gb = wbase + gg * C::GROUP_BYTES;
                        tma_load_2d(gb, &p.tmU, cx * K, cy * K, bar);
                        tma_load_2d(gb + C::UBYTES_AL, &p.tmF, cx * K, cy * K, bar);
                    }
                }
            }
            {
                bool got = false;
                unsigned spins = 0;
                for (;;) {
                    if (mbar_try_wait(bar, phase)) { got = true; break; }
                    if ((++spins & 255u) == 0 && gtimer() > deadline) break;
                }
                if (!got) {
                    fail(ctl, EIK_ETIMEDOUT, 0x3000000ull);
                    // let our own copies land before the block leaves (bounded)
                    const unsigned long long d2 = gtimer() + 1000000000ull;
                    while (!mbar_try_wait(bar, phase) && gtimer() < d2) {
                    }
                    ok = false;
                    break;
                }
            }
            phase ^= 1u;

            // ---- sweep order: preferred (flagged) directions first, then the
            // rest, then the Alg. FSM_order cycle (dir = sweep mod 4).
            int ord = 0, pos = 0;
#pragma unroll
            for (int d = 0; d < 4; ++d)
                if (dm & (1 << d)) { ord |= d << (2 * pos); ++pos; }
#pragma unroll
            for (int d = 0; d < 4; ++d)
                if (!(dm & (1 << d))) { ord |= d << (2 * pos); ++pos; }

            unsigned long long chg[C::RPL];
#pragma unroll
            for (int m = 0; m < C::RPL; ++m) chg[m] = 0ull;
            int gsweeps = 0;
            bool gdone = c < 0;
            int s = 0;
            for (; s < C::MAX_SWEEPS; ++s) {
                const int dir = s < 4 ? (ord >> (2 * s)) & 3 : (s & 3);
                const bool sx = dir <= 1;                 // i increasing
                const bool sy = (dir == 0) || (dir == 3); // j increasing
                bool changed = false;
                for (int t = 0; t < 2 * K - 1; ++t) {
#pragma unroll
                    for (int m = 0; m < C::RPL; ++m) {
                        const int j = r0 + 32 * m;
                        const int jj = sy ? j : K - 1 - j;
                        const int ii = t - jj;
                        if (c >= 0 && ii >= 0 && ii < K) {
                            const int i = sx ? ii : K - 1 - ii;
                            const T fv = tF[j * K + i];
                            if (fv >= (T)0 && fv < INF) {
                                const int q = (j + 1) * C::BW + (i + 1);
                                const T old = tU[q];
                                const T cand =
                                    local_update(tU[q - 1], tU[q + 1], tU[q - C::BW], tU[q + C::BW], fv);
                                if (cand < old) {
                                    tU[q] = cand;
                                    chg[m] |= 1ull << i;
                                    changed = true;
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
                const unsigned any = __ballot_sync(FULL, changed);
                if (!gdone) {
                    ++gsweeps;
                    if (!(any & gmask)) gdone = true;
                }
                if (!any) break;
                if ((s & 31) == 31) {
                    // values only decrease, so stopping early leaves valid upper
                    // bounds; the expired deadline aborts the launch
                    const unsigned long long now = __shfl_sync(FULL, gtimer(), 0);
                    if (now > deadline) {
                        if (lane == 0) fail(ctl, EIK_ETIMEDOUT, 0x4000000ull);
                        s = C::MAX_SWEEPS + 1;
                        break;
                    }
                }
            }
            if (s == C::MAX_SWEEPS && r0 == 0 && c >= 0) fail(ctl, EIK_ENOTCONVERGED, (unsigned)c);
            if (lane == 0)
                st_lane += (unsigned long long)(s < C::MAX_SWEEPS ? s + 1 : C::MAX_SWEEPS) * C::CPW * K * K;
            if (r0 == 0 && c >= 0) {
                ++st_visits;
                st_sweeps += gsweeps;
            }

            // ---- write back the nodes that changed (coalesced across lanes)
#pragma unroll
            for (int m = 0; m < C::RPL; ++m) masks[g * K + r0 + 32 * m] = chg[m];
            __syncwarp();
            for (int e = lane; e < C::CPW * K * K; e += 32) {
                const int gg = e / (K * K);
                const int rem = e - gg * K * K;
                const int j = rem / K, i = rem - j * K;
                int cc = cg[0];
#pragma unroll
                for (int q = 1; q < C::CPW; ++q)
                    if (gg == q) cc = cg[q];
                if (cc >= 0 && ((masks[gg * K + j] >> i) & 1ull)) {
                    const int cx = cc % p.cxn, cy = cc / p.cxn;
                    const T* gU = reinterpret_cast<const T*>(wbase + gg * C::GROUP_BYTES);
                    p.U[(size_t)(cy * K + j + 1) * p.upitch + (size_t)(cx * K + i + 1)] =
                        gU[(j + 1) * C::BW + (i + 1)];
                }
            }
            __threadfence();  // release the new values before any activation
            fence_proxy_async_global();
            __syncwarp();

            // ---- activation of the neighbours (Alg. generic_LC_cells) and
            // their cell values (eq. cell_value).  Side s: 0 W, 1 E, 2 S, 3 N.
            const int cx = c >= 0 ? c % p.cxn : 0, cy = c >= 0 ? c / p.cxn : 0;
#pragma unroll
            for (int sd = 0; sd < 4; ++sd) {
                int nc = -1;
                if (c >= 0) {
                    if (sd == 0 && cx > 0) nc = c - 1;
                    if (sd == 1 && cx + 1 < p.cxn) nc = c + 1;
                    if (sd == 2 && cy > 0) nc = c - p.cxn;
                    if (sd == 3 && cy + 1 < p.cyn) nc = c + p.cxn;
                }
                const bool nsrc = nc >= 0 && p.has_src[nc];
                bool cond = false;
                double vmax = -inf_of<double>();
                int bmax = -1;
#pragma unroll
                for (int m = 0; m < C::RPL; ++m) {
                    const int b = r0 + 32 * m;
                    int bi, bj, ai, aj;
                    if (sd == 0) { bi = 0; bj = b; ai = -1; aj = b; }
                    else if (sd == 1) { bi = K - 1; bj = b; ai = K; aj = b; }
                    else if (sd == 2) { bi = b; bj = 0; ai = b; aj = -1; }
                    else { bi = b; bj = K - 1; ai = b; aj = K; }
                    if (nc >= 0) {
                        const T vb = tU[(bj + 1) * C::BW + (bi + 1)];
                        const T va = tU[(aj + 1) * C::BW + (ai + 1)];
                        const bool ch = (masks[g * K + bj] >> bi) & 1ull;
                        const bool isrc = tF[bj * K + bi] < (T)0;
                        bool cnd = (ch || (first && isrc)) && vb < va;
                        if (cnd && nsrc) {
                            const T fa = __ldg(&p.f[(size_t)(cy * K + aj) * p.fpitch + (cx * K + ai)]);
                            if (fa < (T)0) cnd = false;  // x_j in Q: no activation
                        }
                        cond = cond || cnd;
                        if (vb < INF && (double)vb > vmax) { vmax = (double)vb; bmax = b; }
                    }
                }
                const bool act = (__ballot_sync(FULL, cond) & gmask) != 0u;
                // max boundary value on this side, and where (argmax)
#pragma unroll
                for (int o = C::LPC / 2; o > 0; o >>= 1) {
                    const double ov = __shfl_xor_sync(FULL, vmax, o);
                    const int ob = __shfl_xor_sync(FULL, bmax, o);
                    if (ov > vmax || (ov == vmax && ob > bmax)) { vmax = ov; bmax = ob; }
                }
                if (nc >= 0 && r0 == sd) {
                    double vt = inf_of<double>();
                    if (bmax >= 0) {
                        // y_i: (h + h^c)/2 = (k+1)h/2 from x_i into the
                        // neighbour; F(y_i) read at the node (k+1)/2 deep
                        const int dep = (K + 1) / 2;
                        int yi, yj, ai, aj;
                        if (sd == 0) { yi = cx * K - dep; yj = cy * K + bmax; ai = cx * K - 1; aj = yj; }
                        else if (sd == 1) { yi = cx * K + K - 1 + dep; yj = cy * K + bmax; ai = cx * K + K; aj = yj; }
                        else if (sd == 2) { yi = cx * K + bmax; yj = cy * K - dep; ai = yi; aj = cy * K - 1; }
                        else { yi = cx * K + bmax; yj = cy * K + K - 1 + dep; ai = yi; aj = cy * K + K; }
                        double fy = (double)__ldg(&p.f[(size_t)yj * p.fpitch + yi]);
                        if (!(fy >= 0.0 && fy < inf_of<double>()))
                            fy = (double)__ldg(&p.f[(size_t)aj * p.fpitch + ai]);
                        if (!(fy >= 0.0 && fy < inf_of<double>())) fy = fmin_glob;
                        vt = vmax + (double)(K + 1) * 0.5 * fy;
                    }
                    unsigned long long cur;
                    if (vt < inf_of<double>()) {
                        const unsigned long long kk = key_of(vt);
                        const unsigned long long old = atomicMin(&p.cval[nc], kk);
                        cur = old < kk ? old : kk;
                    } else {
                        cur = ld_cg(&p.cval[nc]);
                    }
                    if (act) {
                        // flags of the directions the influence travels in
                        const int bits = sd == 0 ? 0xC : sd == 1 ? 0x3 : sd == 2 ? 0x6 : 0x9;
                        atomicOr(&p.dirmask[nc], bits);
                        if (atomicExch(&p.qflag[nc], 1) == 0) {
                            if (cur <= theta) lane_push(nextL, next_cnt, nc, J, ctl);
                            else lane_push(farL, far_cnt, nc, J, ctl);
                        }
                    }
                }
            }
            __syncwarp();
        }
        // a warp that gave up (abort raised) still reaches the barrier, which
        // then reports the abort to every block
        ++st_rounds;
        if (!(ok = grid_sync(ctl, deadline, &s_flag))) break;
        ns = nx_slot;
        ++round;
    }

    if (lane == 0) {
        atomicAdd(&ctl->lane_updates, st_lane);
    }
    // per-group counters live on the group leaders
    if (r0 == 0) {
        atomicAdd(&ctl->visits, st_visits);
        atomicAdd(&ctl->sweeps, st_sweeps);
    }
    if (gtid == 0) {
        ctl->rounds = st_rounds;
        ctl->advances = st_adv;
    }
}

}  // namespace eik
