// eik_aux.cu -- the node-wise kernels around the persistent solver, each
// launched once for all instances of a job: per-solve initialisation, the
// FP32 -> double-float refinement seed, the FP64 residual that certifies the
// FP32+refinement result, and the output copy.
#include "eik_solver.cuh"

namespace eik {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int ROWS = 8;  // rows per block (256 threads = 8 rows x 32 columns)

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

// The instance and the (row, column) of this thread's node in its padded grid.
struct Where {
    int inst, i, j;
};
__device__ __forceinline__ Where locate(const AuxInst* a, const int* blk_pre, int n) {
    const int b = blockIdx.x;
    // blk_pre[n + 1 + b] holds the instance of block b (see k_block_owner)
    const int lo = blk_pre[n + 1 + b];
    const int local = b - blk_pre[lo];
    const int tx = (a[lo].nxp + 31) / 32;
    Where w;
    w.inst = lo;
    w.i = (local % tx) * 32 + (threadIdx.x & 31);
    w.j = (local / tx) * ROWS + (threadIdx.x >> 5);
    return w;
}

// owner[b] = instance of block b, for the prefix pre[0..n]: one block per
// instance fills its range
__global__ void k_block_owner(const int* pre, int n, int* owner) {
    const int i = blockIdx.x;
    if (i >= n) return;
    for (int b = pre[i] + threadIdx.x; b < pre[i + 1]; b += blockDim.x) owner[b] = i;
}

// Every element of the padded arrays (ring included): f = h/F on grid nodes,
// +inf on obstacles, padding nodes and the ring; U = +inf.  Rejects F < 0,
// NaN, +inf; reduces the smallest finite h/F into the instance's control
// blocks.  Blocks map onto whole padded arrays (blk_full), 8 rows x 32 columns.
__global__ void k_init_grid(const AuxInst* A, const int* blk_full, int n) {
    const int b = blockIdx.x;
    const int lo = blk_full[n + 1 + b];
    const AuxInst& p = A[lo];
    const int local = b - blk_full[lo];
    const int tx = (p.upitch + 31) / 32;
    const int c = (local % tx) * 32 + (threadIdx.x & 31);   // column in the padded array
    const int r = (local / tx) * ROWS + (threadIdx.x >> 5); // row in the padded array
    const int i = c - 1, j = r - 1;                          // grid node (ring: outside)
    const bool in = c < p.upitch && r < p.nyp + 2;
    const double INF = inf_of<double>();
    double fv = INF;
    bool bad = false;
    if (in && i >= 0 && j >= 0 && i < p.nx && j < p.ny) {
        const double F = p.F[(size_t)j * p.nx + i];
        if (!(F >= 0.0) || F == INF) bad = true;
        else fv = F == 0.0 ? INF : p.h / F;
    }
    if (in) {
        const size_t q = (size_t)r * p.upitch + c;
        if (p.f64) p.f64[q] = fv;
        // beyond 1e18 the FP32 quadratic would overflow: an obstacle for the
        // FP32 pass; the refinement pass (48-bit pairs) restores the node
        if (p.f32) p.f32[q] = fv < 1e18 ? (float)fv : inf_of<float>();
        if (p.fdf) p.fdf[q] = fv < 1e18 ? df_of(fv) : make_float2(inf_of<float>(), 0.0f);
        if (p.U64) p.U64[q] = INF;
        if (p.U32) p.U32[q] = inf_of<float>();
        if (p.Udf) p.Udf[q] = make_float2(inf_of<float>(), 0.0f);
    }
    if (bad) atomicCAS(&p.ctl->status, 0, EIK_EINVAL);
    unsigned long long k = (fv < INF) ? key_of(fv) : KEY_UNSET;
    k = warp_min_u64(k);  // a warp lies in one row of one instance
    if ((threadIdx.x & 31) == 0 && k != KEY_UNSET) {
        atomicMin(&p.ctl->fmin_f, k);
        if (p.ctl2) atomicMin(&p.ctl2->fmin_f, k);
    }
}

__global__ void k_fill(double* a, size_t n, double v) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        a[e] = v;
}
__global__ void k_fill32(float* a, size_t n, float v) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        a[e] = v;
}
__global__ void k_fill_df(float2* a, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        a[e] = make_float2(inf_of<float>(), 0.0f);
}

// Sources: U = q (shifted) and f = -1 (fixed node); source cells get the cell
// value max q (Sec. 4.2, HCM item 1) and start queued.
__global__ void k_init_sources(const AuxInst* A, const SourceTable s) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < s.n) {
        const AuxInst& p = A[s.node_inst[e]];
        const int node = s.node[e];
        const int i = node % p.nx, j = node / p.nx;
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
// one thread per instance: queue its source cells (their number per instance
// is small; the far list is filled in order)
__global__ void k_init_source_cells(const AuxInst* A, const SourceTable s) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < s.ncell) {
        const AuxInst& p = A[s.cell_inst[e]];
        const int c = s.cell[e];
        p.cval[c] = s.cell_key[e];
        p.qflag[c] = 1;
        const int pos = atomicAdd(&p.ctl->fcnt[0], 1);
        if (pos < p.J) p.far0[pos] = c;
    }
}

__global__ void k_ctl_init(Ctl* ctl, int count) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) {
        ctl[e].fmin[0] = KEY_UNSET;
        ctl[e].fmin[1] = KEY_UNSET;
        ctl[e].fmin_f = KEY_UNSET;
    }
}

// Refinement start: V0 = (1 + beta) u32 just above the FP32 result (a
// supersolution when the FP32 error is below beta; values are >= 0 after the
// q shift), +inf where the FP32 pass found nothing.  Every cell with a finite
// start value is queued with key = its smallest start value.
__global__ void k_seed(const AuxInst* A, const int* blk_pre, int n, float beta) {
    const Where w = locate(A, blk_pre, n);
    const AuxInst& p = A[w.inst];
    const int i = w.i, j = w.j;
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
    if (p.cval[c] != KEY_UNSET) {
        p.qflag[c] = 1;
        p.visits[c] = 0;
        const int pos = atomicAdd(&p.ctl2->fcnt[0], 1);
        if (pos < p.J) p.far0[pos] = c;
    }
}

// r = |V - T(V)| at every non-source node, with T the FP64 local update and
// f = h/F recomputed in FP64 from F (+inf against a finite value counts as an
// infinite residual), and max finite V.
__global__ void k_residual(const AuxInst* A, const int* blk_pre, int n) {
    const Where w = locate(A, blk_pre, n);
    const AuxInst& p = A[w.inst];
    const int i = w.i, j = w.j;
    const double INF = inf_of<double>();
    double r = 0.0, umax = 0.0;
    unsigned long long bad = 0;
    if (i < p.nx && j < p.ny) {
        const size_t q = (size_t)(j + 1) * p.upitch + (i + 1);
        const int up = p.upitch;
        auto val = [&](size_t e) {
            const float2 a = p.Udf[e];
            return a.x < inf_of<float>() ? (double)a.x + (double)a.y : INF;
        };
        const double v = val(q);
        if (v < INF) umax = v;
        if (!(p.fdf[q].x < 0.0f)) {
            const double Fv = p.F[(size_t)j * p.nx + i];
            const double fv = Fv > 0.0 ? p.h / Fv : INF;
            const double t = fv < INF ? update_f64(val(q - 1), val(q + 1), val(q - up), val(q + up), fv,
                                                   2.0 * fv * fv)
                                      : INF;
            if (v < INF && t < INF) r = fabs(v - t);
            else if (v < INF || t < INF) { r = INF; bad = 1; }
        }
    }
    const unsigned long long kr = warp_max_u64(key_of(r));
    const unsigned long long ku = warp_max_u64(key_of(umax));
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(FULL, bad, o);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&p.res->r_max, kr);
        atomicMax(&p.res->u_max, ku);
        if (bad) atomicAdd(&p.res->n_bad, bad);
    }
}

__global__ void k_output(const AuxInst* A, const int* blk_pre, int n) {
    const Where w = locate(A, blk_pre, n);
    const AuxInst& p = A[w.inst];
    const int i = w.i, j = w.j;
    if (i < p.nx && j < p.ny) {
        const size_t q = (size_t)(j + 1) * p.upitch + (i + 1);
        double v;
        if (p.U64) {
            v = p.U64[q];
        } else {
            const float2 a = p.Udf[q];
            v = a.x < inf_of<float>() ? (double)a.x + (double)a.y : inf_of<double>();
        }
        p.out[(size_t)j * p.nx + i] = v + p.shift;
    }
}

}  // namespace

cudaError_t launch_fill(double* a, size_t n, double v, cudaStream_t st) {
    k_fill<<<1024, 256, 0, st>>>(a, n, v);
    return cudaGetLastError();
}
cudaError_t launch_fill32(float* a, size_t n, float v, cudaStream_t st) {
    k_fill32<<<1024, 256, 0, st>>>(a, n, v);
    return cudaGetLastError();
}
cudaError_t launch_fill_df(float2* a, size_t n, cudaStream_t st) {
    k_fill_df<<<1024, 256, 0, st>>>(a, n);
    return cudaGetLastError();
}

cudaError_t launch_ctl_init(Ctl* ctl, int count, cudaStream_t st) {
    k_ctl_init<<<(count + 255) / 256, 256, 0, st>>>(ctl, count);
    return cudaGetLastError();
}

cudaError_t launch_block_owner(const int* pre, int n, cudaStream_t st) {
    k_block_owner<<<n, 256, 0, st>>>(pre, n, const_cast<int*>(pre) + n + 1);
    return cudaGetLastError();
}

cudaError_t launch_init_grid(const AuxInst* a, const int* blk_pre, int n, int nblocks, cudaStream_t st) {
    k_init_grid<<<nblocks, 32 * ROWS, 0, st>>>(a, blk_pre, n);
    return cudaGetLastError();
}

cudaError_t launch_init_sources(const AuxInst* a, const SourceTable& s, cudaStream_t st) {
    if (s.n > 0) k_init_sources<<<(s.n + 255) / 256, 256, 0, st>>>(a, s);
    if (s.ncell > 0) k_init_source_cells<<<(s.ncell + 255) / 256, 256, 0, st>>>(a, s);
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
