// eik_aux.cu -- the node-wise kernels around the persistent solver, each
// launched once for all instances of a job: per-solve initialisation, the
// FP32 -> double-float refinement seed, the residual that certifies the
// FP32+refinement result (with the output copy of the pair modes), and the
// output copy of the FP64 mode.
#include "eik_solver.cuh"

namespace eik {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int ROWS = AUX_ROWS;      // rows per block (256 threads = 8 rows x 32 lanes)
constexpr int SPAN = AUX_COLS / 32;  // nodes per thread, 32 columns apart

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(FULL, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// a double as a normalised double-float pair (hi = nearest float)
__device__ __forceinline__ float2 df_of(double v) {
    const float hi = __double2float_rn(v);
    if (!(hi < inf_of<float>()) && !(hi > -inf_of<float>())) return make_float2(hi, 0.0f);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}

// h / F for the pair modes: a double-float quotient from the split F, or the
// FP64 quotient where F cannot be split
__device__ __forceinline__ float2 f_pair(float hx, float hy, double h, double F) {
    float2 Fp;
    if (split_pos(F, &Fp)) return df_div(make_float2(hx, hy), Fp);
    return df_of(h / F);
}

// The instance and the (row, first column) of this thread's nodes in its
// padded grid: columns i, i + 32, ..., i + 32 (SPAN - 1).
struct Where {
    int inst, i, j;
};
__device__ __forceinline__ Where locate(const AuxInst* a, const int* blk_pre, int n) {
    const int b = blockIdx.x;
    // blk_pre[n + 1 + b] holds the instance of block b (written by the host;
    // a single instance has no table)
    const int lo = n == 1 ? 0 : blk_pre[n + 1 + b];
    const int local = b - blk_pre[lo];
    const int tx = (a[lo].nxp + AUX_COLS - 1) / AUX_COLS;
    Where w;
    w.inst = lo;
    w.i = (local % tx) * AUX_COLS + (threadIdx.x & 31);
    w.j = (local / tx) * ROWS + (threadIdx.x >> 5);
    return w;
}

// Tests of a speed on its bit pattern (the integer pipe; GB300 runs double
// comparisons on its FP64 pipe).  valid: 0 <= F < +inf (either zero, no NaN);
// positive: 0 < F < +inf.
__device__ __forceinline__ bool speed_valid(double F) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(F);
    return b < 0x7ff0000000000000ull || b == 0x8000000000000000ull;
}
__device__ __forceinline__ bool speed_positive(double F) {
    const long long b = __double_as_longlong(F);
    return b > 0 && b < 0x7ff0000000000000ll;
}

// Every element of the padded arrays (ring included): f = h/F on grid nodes,
// +inf on obstacles, padding nodes and the ring; U = +inf.  Rejects F < 0,
// NaN, +inf; reduces the smallest finite h/F into the instance's control
// blocks.  Blocks map onto whole padded arrays (blk_full), 8 rows x 32 columns.
__device__ void init_sources_of_block(const AuxInst& p, int lo, int rb, int cb, const SourceTable& s);
__device__ void init_source_cells(const AuxInst* A, const SourceTable& s);

__global__ void k_init_grid(const AuxInst* A, const int* blk_full, int n, const SourceTable s) {
    const int b = blockIdx.x;
    const int lo = n == 1 ? 0 : blk_full[n + 1 + b];
    const AuxInst& p = A[lo];
    const int local = b - blk_full[lo];
    const int tx = (p.upitch + AUX_COLS - 1) / AUX_COLS;
    const int c0 = (local % tx) * AUX_COLS + (threadIdx.x & 31);  // first column in the padded array
    const int r = (local / tx) * ROWS + (threadIdx.x >> 5);        // row in the padded array
    const int j = r - 1;                                            // grid row (ring: outside)
    const double INF = inf_of<double>();
    const float FINF = inf_of<float>();
    // the speeds first, all at once
    double F[SPAN];
#pragma unroll
    for (int s = 0; s < SPAN; ++s) {
        const int i = c0 + 32 * s - 1;
        F[s] = (i >= 0 && j >= 0 && i < p.nx && j < p.ny) ? p.F[(size_t)j * p.nx + i] : 0.0;
    }
    bool bad = false;
    unsigned long long kmin = KEY_UNSET;
    unsigned mmin = 0xffffffffu;
#pragma unroll
    for (int s = 0; s < SPAN; ++s) {
        const int c = c0 + 32 * s;
        const bool in = c < p.upitch && r < p.nyp + 2;
        if (!speed_valid(F[s])) bad = true;
        const bool finite_f = speed_positive(F[s]);  // a grid node with a positive speed
        const size_t q = (size_t)r * p.upitch + c;
        if (p.f64) {
            // FP64 mode: f = h/F in FP64
            const double fv = finite_f ? p.h / F[s] : INF;
            if (in) {
                p.f64[q] = fv;
                p.U64[q] = INF;
            }
            if (fv < INF) kmin = min(kmin, key_of(fv));
        } else {
            // pair modes: f = h/F as a double-float quotient on the FP32
            // pipe; beyond 1e18 the FP32 quadratic would overflow: an obstacle
            float2 fp = make_float2(FINF, 0.0f);
            if (finite_f) {
                fp = f_pair(p.hx, p.hy, p.h, F[s]);
                if (!(fp.x < 1e18f)) fp = make_float2(FINF, 0.0f);
            }
            if (in) {
                p.fdf[q] = fp;
                p.Udf[q] = make_float2(FINF, 0.0f);
                if (p.f32) p.f32[q] = fp.x;
                if (p.U32) p.U32[q] = FINF;
            }
            if (fp.x < FINF) mmin = min(mmin, __float_as_uint(fp.x));
        }
    }
    // the smallest f of the warp's row, one atomic per warp (pair modes: a
    // lower bound of it, from the leading float)
    if (p.f64) {
        kmin = warp_min_u64(kmin);
        if ((threadIdx.x & 31) == 0 && kmin != KEY_UNSET) atomicMin(&p.ctl->fmin_f, kmin);
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mmin = min(mmin, __shfl_xor_sync(FULL, mmin, o));
        if ((threadIdx.x & 31) == 0 && mmin != 0xffffffffu) {
            const unsigned long long k = key_of(widen(__uint_as_float(mmin)) * (1.0 - 0x1p-20));
            atomicMin(&p.ctl->fmin_f, k);
            if (p.ctl2) atomicMin(&p.ctl2->fmin_f, k);
        }
    }
    if (bad) atomicCAS(&p.ctl->status, 0, EIK_EINVAL);
    // the sources that fall in this block's nodes, once its f and U are
    // written; the source cells' queueing spread over the whole launch
    if (s.n) {
        __syncthreads();
        init_sources_of_block(p, lo, (local / tx) * ROWS, (local % tx) * AUX_COLS, s);
    }
    if (s.ncell) init_source_cells(A, s);
}

// Sources: U = q (shifted) and f = -1 (fixed node).  The block of the
// padded array at rows rb.., columns cb.. of instance lo finds the sources
// of its rows by a binary search of the table (sorted by instance, then
// node j nx + i) and writes the ones of its columns.
__device__ void init_sources_of_block(const AuxInst& p, int lo, int rb, int cb, const SourceTable& s) {
    __shared__ int s_first;
    const int jlo = max(rb - 1, 0), jhi = min(rb - 1 + ROWS, p.ny);  // grid rows of the block
    if (jlo >= jhi) return;
    const long long key_lo = (long long)jlo * p.nx, key_hi = (long long)jhi * p.nx;
    if (threadIdx.x == 0) {
        int a = 0, z = s.n;  // first entry >= (lo, key_lo)
        while (a < z) {
            const int m = (a + z) >> 1;
            const int mi = s.node_inst[m];
            if (mi < lo || (mi == lo && (long long)s.node[m] < key_lo)) a = m + 1;
            else z = m;
        }
        s_first = a;
    }
    __syncthreads();
    for (int e = s_first + threadIdx.x; e < s.n; e += blockDim.x) {
        if (s.node_inst[e] != lo || (long long)s.node[e] >= key_hi) break;
        const int node = s.node[e];
        const int i = node % p.nx, j = node / p.nx;
        if (i + 1 < cb || i + 1 >= cb + AUX_COLS) continue;
        const double q = s.q[e];
        const size_t u = (size_t)(j + 1) * p.upitch + (i + 1);
        if (p.f64) p.f64[u] = -1.0;
        if (p.f32) p.f32[u] = -1.0f;
        if (p.fdf) p.fdf[u] = make_float2(-1.0f, 0.0f);
        if (p.U64) p.U64[u] = q;
        if (p.U32) p.U32[u] = (float)q;
        if (p.Udf) p.Udf[u] = df_of(q);
    }
}
// Source cells get the cell value max q (Sec. 4.2, HCM item 1) and start
// queued, one thread of the launch each (they touch only the cell arrays,
// which nothing else of the launch writes).
__device__ void init_source_cells(const AuxInst* A, const SourceTable& s) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < s.ncell; e += gridDim.x * blockDim.x) {
        const AuxInst& p = A[s.cell_inst[e]];
        const int c = s.cell[e];
        p.cval[c] = s.cell_key[e];
        p.qflag[c] = 1;
        if (p.dflags) p.dflags[c] = 15;  // FHCM: source cells sweep in all four directions
        const int pos = atomicAdd(&p.ctl->fcnt[0], 1);
        if (pos < p.J) p.far0[pos] = c;
    }
}


// Refinement start: V0 = (1 + beta) u32 just above the FP32 result (a
// supersolution when the FP32 error is below beta; values are >= 0 after the
// q shift), +inf where the FP32 pass found nothing.  Every cell with a finite
// start value is queued with key = its smallest start value.
__global__ void k_seed(const AuxInst* A, const int* blk_pre, int n, float beta) {
    const Where w = locate(A, blk_pre, n);
    const AuxInst& p = A[w.inst];
    const int j = w.j;
#pragma unroll
    for (int s = 0; s < SPAN; ++s) {
        const int i = w.i + 32 * s;
        const bool in = i < p.nx && j < p.ny;
        unsigned long long k = KEY_UNSET;
        if (in) {
            const size_t q = (size_t)(j + 1) * p.upitch + (i + 1);
            const float2 fv = p.fdf[q];
            float2 v;
            if (fv.x < 0.0f) {
                v = p.Udf[q];  // source: keeps q
            } else {
                const float u = p.U32[q];
                v = (fv.x < inf_of<float>() && u < inf_of<float>()) ? make_float2(u * (1.0f + beta), 0.0f)
                                                                     : make_float2(inf_of<float>(), 0.0f);
                p.Udf[q] = v;
            }
            if (v.x < inf_of<float>()) k = key_of((double)v.x + (double)v.y);
        }
        // min over the k-wide segment of the row that lies in one cell
        for (int o = 1; o < p.k && o < 32; o <<= 1) {
            const unsigned long long x = __shfl_xor_sync(FULL, k, o);
            k = x < k ? x : k;
        }
        if (in && (i % (p.k < 32 ? p.k : 32)) == 0 && k != KEY_UNSET) {
            const int c = (j / p.k) * p.cxn + (i / p.k);
            atomicMin(&p.cval[c], k);
        }
    }
}

__global__ void k_seed_cells(const AuxInst* A, const int* cell_pre, int n, int ncells) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ncells) return;
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cell_pre[mid] <= e) lo = mid;
        else hi = mid;
    }
    const AuxInst& p = A[lo];
    const int c = e - cell_pre[lo];
    // the FP32 pass may leave flags behind (its removal marks): a cell not
    // queued here starts idle
    p.qflag[c] = p.cval[c] != KEY_UNSET ? 1 : 0;
    if (p.cval[c] != KEY_UNSET) {
        p.visits[c] = 0;
        const int pos = atomicAdd(&p.ctl2->fcnt[0], 1);
        if (pos < p.J) p.far0[pos] = c;
    }
}

// Certificate data of the pair modes, and the output.  At every non-source
// node, an upper bound of r = |V - T(V)|: T the exact local update (eqs.
// one_sided_update / two_sided_update with the relevant-quadrant shortcut)
// with f = h/F as k_init_grid stored it: the double-float quotient of h by
// the split F (the solvers never write f except on sources, which this
// skips).  T(V) - V is evaluated relative to V in
// double-float arithmetic on the FP32 pipe -- the upwind offsets, 2 f^2 - d^2,
// its root and the quotient of the cancellation-free form all carry ~46 bits
// -- and an allowance of 2^-40 (V + min(a, b) + 4 f) covers every rounding of
// that evaluation and of f (over a hundred times the worst case of the dozen
// pair operations involved).  +inf against a finite value counts as an
// infinite residual.  Also the max finite V, and out = V + min q.
// After a solve no cell may still be requested or running (every schedule
// clears bits 0 and 1 of a cell's flag when it removes the cell and when
// the removal ends): 1 if node (i, j) is its cell's first node and the cell
// is flagged so.  FMSM marks its source cells for good and is left out.
__device__ __forceinline__ unsigned queued_at(const AuxInst& p, int i, int j) {
    if (!p.qflag || p.Fc || ((i | j) & (p.k - 1))) return 0u;
    return (p.qflag[(j / p.k) * p.cxn + i / p.k] & 3) != 0;
}

__global__ void k_residual(const AuxInst* A, const int* blk_pre, int n) {
    const Where w = locate(A, blk_pre, n);
    const AuxInst& p = A[w.inst];
    const int j = w.j;
    const int up = p.upitch;
    const float FINF = inf_of<float>();
    float r = 0.0f, rrel = 0.0f, umax = 0.0f;
    unsigned long long bad = 0, left = 0;
    const bool shifted = __double_as_longlong(p.shift) != 0;  // min q != 0: add it back
#pragma unroll
    for (int s = 0; s < SPAN; ++s) {
        const int i = w.i + 32 * s;
        if (i >= p.nx || j >= p.ny) continue;
        const size_t q = (size_t)(j + 1) * up + (i + 1);
        left += queued_at(p, i, j);
        // U through L2: with per-instance completion this kernel runs while
        // the persistent pass still works on other instances
        const float2 V = __ldcg(p.Udf + q);
        const float2 fs = p.fdf[q];
        const float2 W = __ldcg(p.Udf + q - 1), E = __ldcg(p.Udf + q + 1), S = __ldcg(p.Udf + q - up),
                     N = __ldcg(p.Udf + q + up);
        const bool vfin = V.x < FINF;
        if (vfin) umax = fmaxf(umax, V.x);
        double o = inf_of<double>();
        if (vfin) {
            o = widen(V.x) + widen(V.y);
            if (shifted) o += p.shift;
        }
        p.out[(size_t)j * p.nx + i] = o;
        if (fs.x < 0.0f) continue;  // a source
        const float2 f = fs;  // +inf on obstacles
        const float2 a = lt(E, W) ? E : W, b = lt(N, S) ? N : S;
        const bool ab = lt(a, b);
        const float2 lo = ab ? a : b, hi = ab ? b : a;
        const bool tfin = f.x < FINF && lo.x < FINF;
        if (vfin && tfin) {
            const float2 d = hi.x < FINF ? df_sub(hi, lo) : make_float2(FINF, 0.0f);
            float2 R;  // T(V) - V
            if (lt(d, f)) {
                const float2 x = df_sub(df_add(df_mul(f, f), df_mul(f, f)), df_mul(d, d));
                const float2 inc = df_div(df_mul(df_sub(f, d), df_add(f, d)), df_add(d, df_sqrt(x)));
                R = df_add(df_sub(hi, V), inc);
            } else {
                R = df_add(df_sub(lo, V), f);
            }
            const float allow = 0x1p-40f * (V.x + lo.x + 4.0f * f.x);
            const float rn = (fabsf(R.x) + fabsf(R.y) + allow) * (1.0f + 0x1p-20f);
            r = fmaxf(r, rn);
            // relative to this node's f, rounded up (f.y < ulp(f.x)): the fast
            // quotient is within 2 ulps for divisors in [2^-100, 1e18], and the
            // factor adds 8; tinier f take the directed-rounding quotient
            const float fd = f.x * (1.0f - 0x1p-22f);
            rrel = fmaxf(rrel, fd >= 0x1p-100f ? __fdividef(rn, fd) * (1.0f + 0x1p-20f) : __fdiv_ru(rn, fd));
        } else if (vfin || tfin) {
            r = rrel = FINF;
            bad += 1;
        }
    }
    // maxima of the warp on the float images (all >= 0), one atomic per warp
    unsigned rb = __float_as_uint(r), ub = __float_as_uint(umax), eb = __float_as_uint(rrel);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rb = max(rb, __shfl_xor_sync(FULL, rb, o));
        eb = max(eb, __shfl_xor_sync(FULL, eb, o));
        ub = max(ub, __shfl_xor_sync(FULL, ub, o));
        bad += __shfl_xor_sync(FULL, bad, o);
        left += __shfl_xor_sync(FULL, left, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (left) atomicAdd(&p.res->n_left, left);
        const float rf = __uint_as_float(rb), ef = __uint_as_float(eb);
        atomicMax(&p.res->r_max, key_of(rf < FINF ? widen(rf) : inf_of<double>()));
        atomicMax(&p.res->r_rel, key_of(ef < FINF ? widen(ef) : inf_of<double>()));
        // V.y < ulp(V.x): a bound of max V
        atomicMax(&p.res->u_max, key_of(widen(__uint_as_float(ub)) * (1.0 + 0x1p-20)));
        if (bad) atomicAdd(&p.res->n_bad, bad);
    }
}

__global__ void k_output(const AuxInst* A, const int* blk_pre, int n) {
    const Where w = locate(A, blk_pre, n);
    const AuxInst& p = A[w.inst];
    const int j = w.j;
    unsigned long long left = 0;
#pragma unroll
    for (int s = 0; s < SPAN; ++s) {
        const int i = w.i + 32 * s;
        if (i < p.nx && j < p.ny) {
            left += queued_at(p, i, j);
            const size_t q = (size_t)(j + 1) * p.upitch + (i + 1);
            double v;
            if (p.U64) {
                v = __ldcg(p.U64 + q);
            } else {
                const float2 a = __ldcg(p.Udf + q);
                v = a.x < inf_of<float>() ? widen(a.x) + widen(a.y) : inf_of<double>();
            }
            p.out[(size_t)j * p.nx + i] = v + p.shift;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) left += __shfl_xor_sync(FULL, left, o);
    if ((threadIdx.x & 31) == 0 && left) atomicAdd(&p.res->n_left, left);
}

}  // namespace

cudaError_t launch_init_grid(const AuxInst* a, const int* blk_full, int n, int nblocks, const SourceTable& s,
                             cudaStream_t st) {
    k_init_grid<<<nblocks, 32 * ROWS, 0, st>>>(a, blk_full, n, s);
    return cudaGetLastError();
}

cudaError_t launch_seed_refine(const AuxInst* a, const int* blk_pre, int n, int nblocks,
                               const int* cell_pre, int ncells, float beta, cudaStream_t st) {
    k_seed<<<nblocks, 32 * ROWS, 0, st>>>(a, blk_pre, n, beta);
    k_seed_cells<<<(ncells + 255) / 256, 256, 0, st>>>(a, cell_pre, n, ncells);
    return cudaGetLastError();
}

cudaError_t launch_residual(const AuxInst* a, const int* blk_pre, int n, int nblocks, cudaStream_t st) {
    k_residual<<<nblocks, 32 * ROWS, 0, st>>>(a, blk_pre, n);
    return cudaGetLastError();
}

cudaError_t launch_output(const AuxInst* a, const int* blk_pre, int n, int nblocks, cudaStream_t st) {
    k_output<<<nblocks, 32 * ROWS, 0, st>>>(a, blk_pre, n);
    return cudaGetLastError();
}

}  // namespace eik
