// eik_fmsm.cu -- the Fast Marching-Sweeping Method (Sec. 4.1, Alg. FMSM,
// Remark sweeping_in_FMSM, Fig. coarse_sweep_choice) on the GPU, FP64.
//
// Part I, Fast Marching on the coarse grid of cell centres, is needed only
// for its acceptance order, and Fast Marching accepts its exit set first and
// then every node after its upwind neighbours, i.e. in the order of the
// coarse values.  So the coarse grid is solved by the library's exact cell
// solver (a job of its own, queued before these kernels, on speeds written by
// k_fmsm_coarse_speed), and the acceptance order is that of the keys
// (exit-set cell first, coarse value, cell index): equal values go by index.
// Cells the coarse grid never reaches (+inf) come last, by index.
//
// Part II processes every cell once, in that order.  What a cell computes
// depends only on which of its four neighbours ran before it -- their values
// are its halo -- so the loop need not run one cell at a time: a cell waits
// only for its earlier neighbours, counted down in visits[c], and cells whose
// earlier neighbours are done run at once on separate warps.  The result is
// the serial loop's.  Per cell, dflags[c] (written by k_fmsm_prep) holds
//   bits 0-3  the sweep directions (numbered as in Alg. FSM_order): those
//             both of whose sides border earlier cells, or, when none has
//             both, those with one such side;
//   bit 4     an exit-set cell: Alg. FSM with the full local update until a
//             sweep changes nothing;
//   bits 5-8  the sides W, E, S, N whose neighbour comes later (released
//             when this cell is done).
#include "eik_solver.cuh"

namespace eik {

namespace {

constexpr int FMSM_FSM = 16;    // dflags: exit-set cell
constexpr int FMSM_LATER = 5;   // dflags: first bit of the later sides

// Coarse speed of every cell: F at its centre, as the mean of the (one, two
// or four) nodes nearest to it, clamped to the grid; exact for a bilinear F.
__global__ void k_fmsm_coarse_speed(const AuxInst* A, const int* cell_pre, int n, int ncells) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ncells) return;
    const int ii = find_inst(cell_pre, n, e);
    const AuxInst& a = A[ii];
    const int c = e - cell_pre[ii];
    const int cx = c % a.cxn, cy = c / a.cxn, k = a.k;
    const int i0 = min(cx * k + (k - 1) / 2, a.nx - 1), i1 = min(cx * k + k / 2, a.nx - 1);
    const int j0 = min(cy * k + (k - 1) / 2, a.ny - 1), j1 = min(cy * k + k / 2, a.ny - 1);
    const double f00 = a.F[(size_t)j0 * a.nx + i0], f01 = a.F[(size_t)j0 * a.nx + i1];
    const double f10 = a.F[(size_t)j1 * a.nx + i0], f11 = a.F[(size_t)j1 * a.nx + i1];
    a.Fc[c] = 0.25 * (((f00 + f01) + f10) + f11);
}

// The acceptance order, locally: which neighbours of each cell come before
// it; its sweep directions and later sides; its count of earlier neighbours;
// and the cells with none, queued.  Source cells carry qflag 1 (set when the
// sources were placed).
__global__ void k_fmsm_prep(const AuxInst* A, const int* cell_pre, int n, int ncells,
                            unsigned long long* ring, unsigned* qctl) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ncells) return;
    const int ii = find_inst(cell_pre, n, e);
    const AuxInst& a = A[ii];
    const int c = e - cell_pre[ii];
    const int cx = c % a.cxn, cy = c / a.cxn;
    const bool src = a.qflag[c] == 1;
    const double u = a.Uc[c];
    auto before = [&](int c2) -> bool {  // is cell c2 accepted before c?
        const bool s2 = a.qflag[c2] == 1;
        if (s2 != src) return s2;
        const double u2 = a.Uc[c2];
        if (u2 != u) return u2 < u;
        return c2 < c;
    };
    int earlier = 0, later = 0;
    if (cx > 0) (before(c - 1) ? earlier : later) |= 1;
    if (cx + 1 < a.cxn) (before(c + 1) ? earlier : later) |= 2;
    if (cy > 0) (before(c - a.cxn) ? earlier : later) |= 4;
    if (cy + 1 < a.cyn) (before(c + a.cxn) ? earlier : later) |= 8;
    const bool w = earlier & 1, ea = earlier & 2, s = earlier & 4, no = earlier & 8;
    // direction d starts from a corner: 0 SW (behind it W, S), 1 NW (W, N),
    // 2 NE (E, N), 3 SE (E, S)
    int dirs = (w && s ? 1 : 0) | (w && no ? 2 : 0) | (ea && no ? 4 : 0) | (ea && s ? 8 : 0);
    if (!dirs) dirs = (w || s ? 1 : 0) | (w || no ? 2 : 0) | (ea || no ? 4 : 0) | (ea || s ? 8 : 0);
    a.dflags[c] = (src ? FMSM_FSM : dirs) | (later << FMSM_LATER);
    a.visits[c] = __popc(earlier);
    if (!earlier) {
        const unsigned t = atomicAdd(&qctl[Q_TAIL], 1u);
        ring[t] = ((unsigned long long)(t + 1u) << 32) | (unsigned)e;
    }
    if (e == 0) qctl[Q_PENDING] = (unsigned)ncells;
}

// One Gauss-Seidel sweep of the tile in direction dir as an anti-diagonal
// wavefront: lane l owns the rows l, l + 32, ... (in sweep order); at step t
// it updates the node t - row of each, whose neighbours behind the sweep are
// on step t - 1 and whose neighbours ahead are untouched this sweep -- the
// serial sweep's values.  FULL: the full local update (Alg. FSM); else the
// sweep-directional update from the two neighbours behind the sweep
// (Remark sweeping_in_FMSM, item 3).  True if a value changed.
template <int K, bool FULL>
__device__ __forceinline__ bool fmsm_sweep(double* tU, const double* tF, const float2* tG, int lane, int dir) {
    using C = TileCfg<MODE_F64, K>;
    constexpr int RPL = (K + 31) / 32;
    const bool sx = dir <= 1, sy = dir == 0 || dir == 3;
    const double INF = inf_of<double>();
    bool changed = false;
    for (int t = 0; t < 2 * K - 1; ++t) {
#pragma unroll
        for (int m = 0; m < RPL; ++m) {
            const int r = lane + 32 * m;
            const int c2 = t - r;
            if (r < K && c2 >= 0 && c2 < K) {
                const int i = sx ? c2 : K - 1 - c2, j = sy ? r : K - 1 - r;
                const int q = (j + 1) * C::BW + (i + 1);
                const double fv = tF[q];
                if (updatable(fv)) {
                    double cand;
                    if constexpr (FULL) {
                        cand = update_f64(tU[q - 1], tU[q + 1], tU[q - C::BW], tU[q + C::BW], fv, tG[j * K + i]);
                    } else {
                        const double ux = sx ? tU[q - 1] : tU[q + 1];
                        const double uy = sy ? tU[q - C::BW] : tU[q + C::BW];
                        cand = update_f64(ux, INF, uy, INF, fv, tG[j * K + i]);
                    }
                    if (lt(cand, tU[q])) {
                        tU[q] = cand;
                        changed = true;
                    }
                }
            }
        }
        __syncwarp();
    }
    return changed;
}

// Part II.  Each warp takes a ready cell from the ring, loads its tile and
// halo, sweeps it, writes it back and counts down its later neighbours; of
// those whose count reaches zero it keeps one to run next and queues the
// rest.  `pending` counts the cells not yet done; a waiting warp that sees it
// at zero leaves.  Every wait is bounded by the launch deadline.
template <int K>
__global__ void __launch_bounds__(TileCfg<MODE_F64, K>::WPB * 32)
    k_solve_fmsm(const __grid_constant__ SolveParams p) {
    using C = TileCfg<MODE_F64, K>;
    static_assert(C::CPW == 1, "one cell per warp");
    constexpr unsigned FULLM = 0xffffffffu;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    WarpState<MODE_F64, K> w;
    w.init(smem);
    __syncwarp();
    const int lane = w.lane;
    Ctl* gctl = p.gctl;
    const InstDesc* inst = p.inst;
    const int NI = p.n_inst;
    const unsigned long long deadline = gtimer() + (unsigned long long)p.deadline_ns;
    if (threadIdx.x == 0) atomicMin(&gctl->t_start, gtimer());
    double* tU = w.tU;
    const double* tF = w.tF;
    float2* tG = reinterpret_cast<float2*>(const_cast<double*>(w.tG));
    constexpr int MAX_SWEEPS = 4 * (K * K + 8);
    const int prof_on = p.profile;  // per-phase cycles into gctl->prof (profiling only)
    unsigned long long pacc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long pt = clock64();

    int next = -1;  // a cell this warp released itself and runs next
    for (;;) {
        int e = next;
        if (e < 0) {
            if (lane == 0) e = ring_pop(p, gctl, deadline);
            e = __shfl_sync(FULLM, e, 0);
            if (e < 0) break;
        }
        next = -1;
        const int ii = find_inst(p.cell_pre, NI, e);
        const InstDesc& d = inst[ii];
        const int c = e - d.cell_base;
        const int cx = c % d.cxn, cy = c / d.cxn;
        int fl = 0;
        if (lane == 0) fl = ld_cg(&d.dflags[c]);
        fl = __shfl_sync(FULLM, fl, 0);
        // the earlier neighbours' values were released before this cell was
        // queued; acquire them for the halo load
        fence_acq_rel_gpu();
        fence_proxy_async_global();
        fence_proxy_async_shared();
        __syncwarp();
        PROF_MARK(2);
        pacc[7] += 1;
        if (lane == 0) {
            mbar_arrive_expect_tx(w.bar, (uint32_t)C::TX_BYTES);
            tma_load_2d(tU, &d.tmU, cx * K, cy * K, w.bar);
            tma_load_2d(const_cast<double*>(tF), &d.tmF, cx * K, cy * K, w.bar);
        }
        {
            bool got = false;
            unsigned spins = 0;
            for (;;) {
                if (mbar_try_wait(w.bar, w.phase)) { got = true; break; }
                if ((++spins & 255u) == 0 && gtimer() > deadline) break;
            }
            if (!got) {
                if (lane == 0) fail(gctl, EIK_ETIMEDOUT, 0x3000000ull);
                const unsigned long long d2 = gtimer() + 1000000000ull;
                while (!mbar_try_wait(w.bar, w.phase) && gtimer() < d2) {
                }
                break;
            }
        }
        w.phase ^= 1u;
        for (int r = lane; r < K * K; r += 32) {
            const int jj = r / K, i2 = r - jj * K;
            tG[r] = f64_pair(tF[(jj + 1) * C::BW + i2 + 1]);
        }
        __syncwarp();
        PROF_MARK(3);

        int nsw = 0;
        bool timed_out = false;
        if (fl & FMSM_FSM) {
            // Alg. FSM on the cell: the directions in turn until a sweep
            // changes nothing
            for (int s = 0;; ++s) {
                const bool ch = fmsm_sweep<K, true>(tU, tF, tG, lane, s & 3);
                ++nsw;
                if (!__ballot_sync(FULLM, ch)) break;
                if (nsw >= MAX_SWEEPS) {
                    if (lane == 0) {
                        atomicCAS(&d.ctl->status, 0, EIK_ENOTCONVERGED);
                        fail(gctl, EIK_ENOTCONVERGED, (unsigned)c);
                    }
                    break;
                }
                if ((s & 15) == 15 && __shfl_sync(FULLM, gtimer(), 0) > deadline) {
                    if (lane == 0) fail(gctl, EIK_ETIMEDOUT, 0x4000000ull);
                    timed_out = true;
                    break;
                }
            }
        } else {
#pragma unroll 1
            for (int dd = 0; dd < 4; ++dd)
                if ((fl >> dd) & 1) {
                    fmsm_sweep<K, false>(tU, tF, tG, lane, dd);
                    ++nsw;
                }
        }
        PROF_MARK(4);
        // ---- write back the cell (padding nodes keep their +inf)
        for (int r = lane; r < K * K; r += 32) {
            const int j = r / K, i = r - j * K;
            reinterpret_cast<double*>(d.U)[(size_t)(cy * K + j + 1) * d.upitch + (size_t)(cx * K + i + 1)] =
                tU[(j + 1) * C::BW + (i + 1)];
        }
        fence_acq_rel_gpu();  // release the cell before its later neighbours run
        fence_proxy_async_global();
        __syncwarp();
        PROF_MARK(5);
        // ---- count down the later neighbours (lane s: side s).  Of those
        // that become ready, this warp keeps the first and runs it next (no
        // round trip through the ring on the chain of dependent cells); the
        // others are queued.
        bool ready = false;
        int nc = -1;
        if (lane < 4 && ((fl >> (FMSM_LATER + lane)) & 1)) {
            nc = lane == 0 ? c - 1 : lane == 1 ? c + 1 : lane == 2 ? c - d.cxn : c + d.cxn;
            ready = atomicSub(&d.visits[nc], 1) == 1;
        }
        const unsigned rmask = __ballot_sync(FULLM, ready);
        if (rmask) {
            const int keep = __ffs(rmask) - 1;
            if (ready && lane != keep) {
                fence_acq_rel_gpu();  // pass on what this neighbour's other predecessors released
                ring_push(p, gctl, (unsigned)(d.cell_base + nc), deadline);
            }
            next = __shfl_sync(FULLM, d.cell_base + nc, keep);
        }
        __syncwarp();
        if (lane == 0) {
            if (ii != w.acc_inst) {
                flush_counters(inst, w.acc_inst, w.acc_visits, w.acc_sweeps, w.acc_lane);
                w.acc_inst = ii;
            }
            w.acc_visits += 1;
            w.acc_sweeps += (unsigned long long)nsw;
            w.acc_lane += (unsigned long long)nsw * K * K;
            atomicSub(&p.qctl[Q_PENDING], 1u);
        }
        __syncwarp();
        PROF_MARK(6);
        if (timed_out) break;
    }
    if (lane == 0) {
        flush_counters(inst, w.acc_inst, w.acc_visits, w.acc_sweeps, w.acc_lane);
        atomicMax(&gctl->t_end, gtimer());
        if (prof_on)
            for (int i = 0; i < 8; ++i) atomicAdd(&gctl->prof[i], pacc[i]);
    }
}

// One grid: a block per SM.  Only about a hundred cells are ready at a time,
// and the waiting warps' polling slowed the working ones (1025^2 sin20 at
// k = 8: 3.46 ms at the occupancy limit, 3.30 ms at two blocks per SM, 3.27
// ms at one).  A batch keeps the occupancy limit.
template <int K>
void shape_fmsm(int num_sms, int n_inst, int sm_cap, LaunchShape* s) {
    using C = TileCfg<MODE_F64, K>;
    const void* fn = (const void*)k_solve_fmsm<K>;
    s->threads = C::WPB * 32;
    s->smem = (size_t)C::WPB * C::WARP_BYTES + 128;
    s->blocks = 0;
    s->per_sm = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, s->threads, s->smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    int cap = n_inst > 1 || per_sm < 1 ? per_sm : 1;
    if (sm_cap > 0 && sm_cap < cap) cap = sm_cap;
    s->blocks = cap * num_sms;
    s->per_sm = per_sm;
    block_resources(fn, s->threads, s->smem, s);
}

}  // namespace

cudaError_t launch_fmsm_coarse_speed(const AuxInst* a, const int* cell_pre, int n, int ncells, cudaStream_t st) {
    k_fmsm_coarse_speed<<<(ncells + 255) / 256, 256, 0, st>>>(a, cell_pre, n, ncells);
    return cudaGetLastError();
}

cudaError_t launch_fmsm_prep(const AuxInst* a, const int* cell_pre, int n, int ncells, unsigned long long* ring,
                             unsigned* qctl, cudaStream_t st) {
    k_fmsm_prep<<<(ncells + 255) / 256, 256, 0, st>>>(a, cell_pre, n, ncells, ring, qctl);
    return cudaGetLastError();
}

int fmsm_shape(int k, int num_sms, int n_inst, int sm_cap, LaunchShape* out) {
    out->blocks = 0;
    switch (k) {
    case 8: shape_fmsm<8>(num_sms, n_inst, sm_cap, out); break;
    case 16: shape_fmsm<16>(num_sms, n_inst, sm_cap, out); break;
    case 32: shape_fmsm<32>(num_sms, n_inst, sm_cap, out); break;
    case 64: shape_fmsm<64>(num_sms, n_inst, sm_cap, out); break;
    default: return -1;
    }
    return out->blocks > 0 ? 0 : -1;
}

cudaError_t launch_fmsm(int k, const SolveParams& p, const LaunchShape& s, cudaStream_t st) {
    const void* fn = nullptr;
    switch (k) {
    case 8: fn = (const void*)k_solve_fmsm<8>; break;
    case 16: fn = (const void*)k_solve_fmsm<16>; break;
    case 32: fn = (const void*)k_solve_fmsm<32>; break;
    case 64: fn = (const void*)k_solve_fmsm<64>; break;
    default: return cudaErrorInvalidValue;
    }
    void* args[] = {(void*)&p};
    return cudaLaunchKernel(fn, dim3(s.blocks), dim3(s.threads), args, s.smem, st);
}

}  // namespace eik
