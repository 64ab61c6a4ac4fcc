// eik_aux.cu -- per-solve initialisation, the FP32 -> FP64 refinement seed and
// the FP64 residual that certifies the FP32+refinement result.
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
        if (p.f64) p.f64[(size_t)j * p.f64pitch + i] = fv;
        if (p.f32) {
            // beyond 1e18 the FP32 quadratic would overflow: treat as an
            // obstacle in the FP32 pass; the FP64 refinement restores it
            p.f32[(size_t)j * p.f32pitch + i] = fv < 1e18 ? (float)fv : inf_of<float>();
        }
        if (p.U64) p.U64[(size_t)(j + 1) * p.u64pitch + (i + 1)] = INF;
        if (p.U32) p.U32[(size_t)(j + 1) * p.u32pitch + (i + 1)] = inf_of<float>();
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

// Sources: U = q and f = -1 (fixed node); source cells get the cell value
// max q (Sec. 4.2, HCM item 1), all four directional flags, and start queued.
__global__ void k_init_sources(const InitParams p, const SourceInit s, unsigned long long* cval,
                               int* qflag, int* dirmask, unsigned char* has_src, int* far0) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < s.n) {
        const int node = s.node[e];
        const int i = node % s.nx, j = node / s.nx;
        const double q = s.q[e];
        if (p.f64) p.f64[(size_t)j * p.f64pitch + i] = -1.0;
        if (p.f32) p.f32[(size_t)j * p.f32pitch + i] = -1.0f;
        if (p.U64) p.U64[(size_t)(j + 1) * p.u64pitch + (i + 1)] = q;
        if (p.U32) p.U32[(size_t)(j + 1) * p.u32pitch + (i + 1)] = (float)q;
    }
    if (e < s.ncell) {
        const int c = s.cell[e];
        cval[c] = s.cell_key[e];
        has_src[c] = 1;
        dirmask[c] = 0xF;
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

// FP64 refinement start: V0 = u32 + beta (u32 - q_min) above the FP32 result
// (a supersolution when the FP32 error is below beta), +inf where the FP32
// pass found nothing; every cell with a finite start value is queued with key
// = its smallest start value.
__global__ void k_seed(const SeedParams p) {
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int j = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const bool in = i < p.nx && j < p.ny;
    const double INF = inf_of<double>();
    unsigned long long k = KEY_UNSET;
    if (in) {
        const double fv = p.f64[(size_t)j * p.f64pitch + i];
        double* dst = &p.U64[(size_t)(j + 1) * p.u64pitch + (i + 1)];
        double v;
        if (fv < 0.0) {
            v = *dst;  // source: keeps q
        } else {
            const float u = p.U32[(size_t)(j + 1) * p.u32pitch + (i + 1)];
            v = (fv < INF && u < inf_of<float>()) ? (double)u + p.beta * ((double)u - p.q_min) : INF;
            *dst = v;
        }
        if (v < INF) k = key_of(v);
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
        p.dirmask[c] = 0;
        p.visits[c] = 0;
        p.far0[base + __popc(m & ((1u << lane) - 1u))] = c;
    }
}

// r = |V - T(V)| at every non-source node (T = the FP64 local update; +inf
// against a finite value counts as an infinite residual), and max finite V.
__global__ void k_residual(const double* U, int up, const double* f, int fp, int nx, int ny,
                           ResidualOut* out) {
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int j = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const double INF = inf_of<double>();
    double r = 0.0, umax = -INF;
    unsigned long long bad = 0;
    if (i < nx && j < ny) {
        const size_t q = (size_t)(j + 1) * up + (i + 1);
        const double v = U[q];
        const double fv = f[(size_t)j * fp + i];
        if (v < INF) umax = v;
        if (fv >= 0.0) {
            const double t = fv < INF ? local_update(U[q - 1], U[q + 1], U[q - up], U[q + up], fv) : INF;
            if (v < INF && t < INF) r = fabs(v - t);
            else if (v < INF || t < INF) { r = INF; bad = 1; }
        }
    }
    unsigned long long kr = warp_max_u64(key_of(r));
    unsigned long long ku = warp_max_u64(key_of(umax));
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(FULL, bad, o);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out->r_max, kr);
        atomicMax(&out->u_max, ku);
        if (bad) atomicAdd(&out->n_bad, bad);
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

cudaError_t launch_init_sources(const InitParams& ip, const SourceInit& s, unsigned long long* cval,
                                int* qflag, int* dirmask, unsigned char* has_src, int* far0,
                                cudaStream_t st) {
    const int n = s.n > s.ncell ? s.n : s.ncell;
    if (n == 0) return cudaSuccess;
    k_init_sources<<<(n + 255) / 256, 256, 0, st>>>(ip, s, cval, qflag, dirmask, has_src, far0);
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

cudaError_t launch_residual(const double* U64, int u64pitch, const double* f64, int f64pitch,
                            int nx, int ny, ResidualOut* out, cudaStream_t st) {
    k_residual<<<grid2d(nx, ny, 8), 256, 0, st>>>(U64, u64pitch, f64, f64pitch, nx, ny, out);
    return cudaGetLastError();
}

}  // namespace eik
