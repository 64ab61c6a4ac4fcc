// eik_aux.cu -- per-solve initialisation, the FP32 -> double-float refinement
// seed, the FP64 residual that certifies the FP32+refinement result, and the
// output copy.
#include "eik_solver.cuh"

namespace eik {

namespace {

constexpr unsigned FULL = 0xffffffffu;

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

// f = h/F on every node of the padded grid (+inf on obstacles and padding),
// U = +inf on every node of the padded interior; rejects F < 0, NaN, +inf;
// reduces the smallest finite h/F into ctl->fmin_f.
__global__ void k_init_grid(const InitParams p) {
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int j = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const bool in = i < p.nxp && j < p.nyp;
    const double INF = inf_of<double>();
    double fv = INF;
    bool bad = false;
    if (in && i < p.nx && j < p.ny) {
        const double F = p.F[(size_t)j * p.nx + i];
        if (!(F >= 0.0) || F == INF) bad = true;
        else fv = F == 0.0 ? INF : p.h / F;
    }
    if (in) {
        const size_t fi = (size_t)(j + 1) * p.fpitch + (i + 1);
        const size_t ui = (size_t)(j + 1) * p.upitch + (i + 1);
        if (p.f64) p.f64[fi] = fv;
        // beyond 1e18 the FP32 quadratic would overflow: an obstacle for the
        // FP32 pass; the refinement pass (48-bit pairs) restores the node
        if (p.f32) p.f32[fi] = fv < 1e18 ? (float)fv : inf_of<float>();
        if (p.fdf) p.fdf[fi] = fv < 1e18 ? df_of(fv) : make_float2(inf_of<float>(), 0.0f);
        if (p.U64) p.U64[ui] = INF;
        if (p.U32) p.U32[ui] = inf_of<float>();
        if (p.Udf) p.Udf[ui] = make_float2(inf_of<float>(), 0.0f);
    }
    if (bad) atomicCAS(&p.ctl->status, 0, EIK_EINVAL);
    unsigned long long k = (fv < INF) ? key_of(fv) : KEY_UNSET;
    k = warp_min_u64(k);
    if ((threadIdx.x & 31) == 0 && k != KEY_UNSET) atomicMin(&p.ctl->fmin_f, k);
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
__global__ void k_init_sources(const InitParams p, const SourceInit s, unsigned long long* cval,
                               int* qflag, unsigned char* has_src, int* far0) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < s.n) {
        const int node = s.node[e];
        const int i = node % s.nx, j = node / s.nx;
        const double q = s.q[e];
        const size_t fi = (size_t)(j + 1) * p.fpitch + (i + 1);
        const size_t ui = (size_t)(j + 1) * p.upitch + (i + 1);
        if (p.f64) p.f64[fi] = -1.0;
        if (p.f32) p.f32[fi] = -1.0f;
        if (p.fdf) p.fdf[fi] = make_float2(-1.0f, 0.0f);
        if (p.U64) p.U64[ui] = q;
        if (p.U32) p.U32[ui] = (float)q;
        if (p.Udf) p.Udf[ui] = df_of(q);
    }
    if (e < s.ncell) {
        const int c = s.cell[e];
        cval[c] = s.cell_key[e];
        has_src[c] = 1;
        qflag[c] = 1;
        far0[e] = c;
    }
}

__global__ void k_ctl_init(Ctl* ctl, int nfar0) {
    ctl->fmin[0] = KEY_UNSET;
    ctl->fmin[1] = KEY_UNSET;
    ctl->fmin_f = KEY_UNSET;
    ctl->fcnt[0] = nfar0;
}

// Refinement start: V0 = (1 + beta) u32 just above the FP32 result (a
// supersolution when the FP32 error is below beta; values are >= 0 after the
// q shift), +inf where the FP32 pass found nothing.  Every cell with a finite
// start value is queued with key = its smallest start value.
__global__ void k_seed(const SeedParams p) {
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int j = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const bool in = i < p.nx && j < p.ny;
    unsigned long long k = KEY_UNSET;
    if (in) {
        const float2 fv = p.fdf[(size_t)(j + 1) * p.fpitch + (i + 1)];
        float2* dst = &p.Udf[(size_t)(j + 1) * p.upitch + (i + 1)];
        float2 v;
        if (fv.x < 0.0f) {
            v = *dst;  // source: keeps q
        } else {
            const float u = p.U32[(size_t)(j + 1) * p.upitch + (i + 1)];
            v = (fv.x < inf_of<float>() && u < inf_of<float>())
                    ? make_float2(u * (1.0f + p.beta), 0.0f)
                    : make_float2(inf_of<float>(), 0.0f);
            *dst = v;
        }
        if (v.x < inf_of<float>()) k = key_of((double)v.x + (double)v.y);
    }
    // min over the k-wide segment of the row that lies in one cell
    for (int o = 1; o < p.k && o < 32; o <<= 1) {
        const unsigned long long w = __shfl_xor_sync(FULL, k, o);
        k = w < k ? w : k;
    }
    if (in && (i % (p.k < 32 ? p.k : 32)) == 0 && k != KEY_UNSET) {
        const int c = (j / p.k) * p.cxn + (i / p.k);
        atomicMin(&p.cval[c], k);
    }
}

__global__ void k_seed_cells(const SeedParams p, int J) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const bool queued = c < J && p.cval[c] != KEY_UNSET;
    const unsigned m = __ballot_sync(FULL, queued);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&p.ctl->fcnt[0], __popc(m));
    base = __shfl_sync(FULL, base, leader);
    if (queued) {
        p.qflag[c] = 1;
        p.visits[c] = 0;
        p.far0[base + __popc(m & ((1u << lane) - 1u))] = c;
    }
}

// r = |V - T(V)| at every non-source node, with T the FP64 local update and
// f = h/F recomputed in FP64 (+inf against a finite value counts as an
// infinite residual), and max finite V.
__global__ void k_residual(const float2* U, int up, const float2* fdf, int fp, const double* F,
                           double h, int nx, int ny, ResidualOut* out) {
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int j = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const double INF = inf_of<double>();
    double r = 0.0, umax = 0.0;
    unsigned long long bad = 0;
    if (i < nx && j < ny) {
        const size_t q = (size_t)(j + 1) * up + (i + 1);
        auto val = [&](size_t e) {
            const float2 a = U[e];
            return a.x < inf_of<float>() ? (double)a.x + (double)a.y : INF;
        };
        const double v = val(q);
        if (v < INF) umax = v;
        if (!(fdf[(size_t)(j + 1) * fp + (i + 1)].x < 0.0f)) {
            const double Fv = F[(size_t)j * nx + i];
            const double fv = Fv > 0.0 ? h / Fv : INF;
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
        atomicMax(&out->r_max, kr);
        atomicMax(&out->u_max, ku);
        if (bad) atomicAdd(&out->n_bad, bad);
    }
}

__global__ void k_output(const double* U64, const float2* Udf, int up, int nx, int ny, double shift,
                         double* dst) {
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int j = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i < nx && j < ny) {
        const size_t q = (size_t)(j + 1) * up + (i + 1);
        double v;
        if (U64) {
            v = U64[q];
        } else {
            const float2 a = Udf[q];
            v = a.x < inf_of<float>() ? (double)a.x + (double)a.y : inf_of<double>();
        }
        dst[(size_t)j * nx + i] = v + shift;
    }
}

inline dim3 grid2d(int nx, int ny, int rows_per_block) {
    return dim3((unsigned)((nx + 31) / 32), (unsigned)((ny + rows_per_block - 1) / rows_per_block));
}

}  // namespace

cudaError_t launch_init_grid(const InitParams& p, cudaStream_t st) {
    k_init_grid<<<grid2d(p.nxp, p.nyp, 8), 256, 0, st>>>(p);
    return cudaGetLastError();
}

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

cudaError_t launch_init_sources(const InitParams& ip, const SourceInit& s, unsigned long long* cval,
                                int* qflag, unsigned char* has_src, int* far0, cudaStream_t st) {
    const int n = s.n > s.ncell ? s.n : s.ncell;
    if (n == 0) return cudaSuccess;
    k_init_sources<<<(n + 255) / 256, 256, 0, st>>>(ip, s, cval, qflag, has_src, far0);
    return cudaGetLastError();
}

cudaError_t launch_ctl_init(Ctl* ctl, int nfar0, cudaStream_t st) {
    k_ctl_init<<<1, 1, 0, st>>>(ctl, nfar0);
    return cudaGetLastError();
}

cudaError_t launch_seed_refine(const SeedParams& p, cudaStream_t st) {
    k_seed<<<grid2d(p.nx, p.ny, 8), 256, 0, st>>>(p);
    const int J = p.cxn * p.cyn;
    k_seed_cells<<<(J + 255) / 256, 256, 0, st>>>(p, J);
    return cudaGetLastError();
}

cudaError_t launch_output(const double* U64, const float2* Udf, int upitch, int nx, int ny,
                          double shift, double* dst, cudaStream_t st) {
    k_output<<<grid2d(nx, ny, 8), 256, 0, st>>>(U64, Udf, upitch, nx, ny, shift, dst);
    return cudaGetLastError();
}

cudaError_t launch_residual(const float2* Udf, int upitch, const float2* fdf, int fpitch,
                            const double* F, double h, int nx, int ny, ResidualOut* out,
                            cudaStream_t st) {
    k_residual<<<grid2d(nx, ny, 8), 256, 0, st>>>(Udf, upitch, fdf, fpitch, F, h, nx, ny, out);
    return cudaGetLastError();
}

}  // namespace eik
