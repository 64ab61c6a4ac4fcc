// eik_solver.cuh -- the persistent cell solvers, templated on the arithmetic
// mode and the cell size K.  Instantiated by eik_solver_*.cu.
//
// What one launch computes (Chacon & Vladimirsky, Sec. 4.2):
//   Alg. generic_LC_cells with the HCM refinements -- cells carry cell values
//   (eq. cell_value); a removed cell is swept to convergence in the four
//   directions of Alg. FSM_order (here all four at once, one warp per cell);
//   a changed boundary value V_i with V_i < V_j (x_j across the boundary, not
//   in Q) activates the neighbour.
// GPU recast: no heap.  Three orders of removal, each exact by Theorem
// convergence (any removal order, exact per-cell solves):
//   - k_solve, bucketed rounds: every queued cell whose value lies within
//     `delta` of the smallest is released at once and processed by all
//     warps; re-activations run in the next round, after a grid barrier;
//   - k_solve_async, first in first out: each warp takes the next requested
//     cell from a device ring as soon as it is free;
//   - k_solve_async with ORD, value order: Dial's buckets without rounds
//     (bucket rings, a front that moves up as its bucket empties, a window
//     of buckets above it that warps take cells from).
//
// All stored values are >= +0 (the host shifts q by its minimum), so the
// bit patterns of doubles and floats order like the values: min and compare
// run on the integer pipe, which on this part is far faster than FP64.
#pragma once

#include <type_traits>

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
// on the mbarrier `bar`.  x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"((unsigned long long)tm), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
// Release / acquire at GPU scope.  Every hand-off of tile values between
// warps goes through read-modify-writes of the receiving cell's flag, which
// are totally ordered: the writer's fence orders its value stores before its
// flag update, the reader's fence orders its flag update before its loads,
// so whichever update comes second sees the other side's work.  No
// sequentially consistent fence is needed.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
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

// ---------------------------------------------------------------- ordered bits
// For values in [+0, +inf] the signed integer image orders like the value.
__device__ __forceinline__ long long ob(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ int ob(float x) { return __float_as_int(x); }
__device__ __forceinline__ double from_ob(long long b) { return __longlong_as_double(b); }
__device__ __forceinline__ float from_ob(int b) { return __int_as_float(b); }
constexpr long long INF_BITS64 = 0x7ff0000000000000LL;
constexpr int INF_BITS32 = 0x7f800000;
// f in [+0, +inf): a node that is neither a source (f = -1) nor an obstacle
__device__ __forceinline__ bool updatable(double f) {
    return (unsigned long long)__double_as_longlong(f) < (unsigned long long)INF_BITS64;
}
__device__ __forceinline__ bool updatable(float f) {
    return (unsigned)__float_as_int(f) < (unsigned)INF_BITS32;
}

// ---------------------------------------------------------------- local update
// The update at one node from its four neighbours with the relevant-quadrant
// shortcut of Remark regular_FSM_update: a = min(U_W, U_E), b = min(U_S, U_N);
// if |a - b| < f = h/F the two-sided root of (U-a)^2 + (U-b)^2 = f^2
// (eq. two_sided_update), else the one-sided min(a, b) + f
// (eq. one_sided_update).  Neighbours are >= 0 (possibly +inf); f is finite.

// FP32, with the quadratic in the cancellation-free form
//   hi + (f^2 - d^2) / (d + sqrt(2 f^2 - d^2))
// whose small increment carries all the rounding; its quotient and root need
// only a few correct bits relative to f, far below ulp(U).
__device__ __forceinline__ float increment_f32(float d, float f) {
    const float x = fmaf(-d, d, 2.0f * f * f);  // 2 f^2 - d^2 >= f^2 > 0
    const float root = x * rsqrtf(x);
    return __fdividef((f - d) * (f + d), d + root);
}
__device__ __forceinline__ float update_f32(float W, float E, float S, float N, float f) {
    const int a = min(ob(W), ob(E)), b = min(ob(S), ob(N));
    const int lob = min(a, b), hib = max(a, b);
    const float lo = from_ob(lob), hi = from_ob(hib);
    const float one = lo + f;
    const float d = hi - lo;
    const bool two_sided = hib < INF_BITS32 && ob(d) < ob(f);
    const float two = hi + increment_f32(two_sided ? d : 0.0f, f);
    return two_sided ? two : one;
}

// ---------------------------------------------------------------- double-float
// Refinement arithmetic entirely on the FP32 pipe: a value is an unevaluated
// pair hi + lo of floats with |lo| <= ulp(hi)/2 (48 significant bits), kept
// in a float2 (x = hi, y = lo).  Sums use Knuth's TwoSum and Dekker's
// Fast2Sum; the quadratic's increment is the FP32 safe form above, computed
// from the pair difference d.  Its error, a few FP32 ulps of f per update, is
// far below what the FP64 residual certificate has to certify.
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return make_float2(s, b - (s - a));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float2 s = two_sum(a.x, b.x);
    s.y += a.y + b.y;
    return fast_two_sum(s.x, s.y);
}
__device__ __forceinline__ float2 df_add_f(float2 a, float b) {
    float2 s = two_sum(a.x, b);
    s.y += a.y;
    return fast_two_sum(s.x, s.y);
}

// Products, quotients and square roots of pairs (the refinement's residual
// and its start values).  two_prod is exact (Dekker's product through one
// fused multiply-add); df_mul keeps the cross terms; df_div and df_sqrt take
// the FP32 quotient / root and add one Newton correction computed from the
// exact residual of that first approximation (Markstein's and Heron's
// correction steps).  Each is accurate to a few units of 2^-46 relative to
// its operands.
__device__ __forceinline__ float2 two_prod(float a, float b) {
    const float p = a * b;
    return make_float2(p, fmaf(a, b, -p));
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_sub(float2 a, float2 b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    float2 p = two_prod(a.x, b.x);
    p.y = fmaf(a.x, b.y, fmaf(a.y, b.x, p.y));
    return fast_two_sum(p.x, p.y);
}
// The first approximations come from the fast reciprocal / inverse-root
// units (a couple of ulps); the correction squares that error away.
__device__ __forceinline__ float2 df_div(float2 a, float2 b) {  // 0 < b < 2^126
    const float q0 = __fdividef(a.x, b.x);
    const float2 p = two_prod(q0, b.x);  // q0 b.x exactly
    // a - q0 b: a.x - p.x is exact (the two agree to within a few roundings)
    const float r = ((a.x - p.x) - p.y) + fmaf(-q0, b.y, a.y);
    return fast_two_sum(q0, __fdividef(r, b.x));
}
__device__ __forceinline__ float2 df_sqrt(float2 a) {  // 0 <= a < 2^126
    if (!(a.x > 0.0f)) return make_float2(0.0f, 0.0f);
    const float ri = rsqrtf(a.x);
    const float y0 = a.x * ri;
    const float2 p = two_prod(y0, y0);
    const float r = ((a.x - p.x) - p.y) + a.y;  // a - y0^2
    return fast_two_sum(y0, 0.5f * r * ri);
}

// order, finiteness and conversion of a stored value, for each representation
// (normalised pairs with hi >= 0 order lexicographically)
__device__ __forceinline__ bool lt(float2 a, float2 b) { return a.x < b.x || (a.x == b.x && a.y < b.y); }
__device__ __forceinline__ bool lt(double a, double b) { return ob(a) < ob(b); }
__device__ __forceinline__ bool lt(float a, float b) { return ob(a) < ob(b); }
__device__ __forceinline__ bool is_finite_v(float2 a) { return a.x < inf_of<float>(); }
__device__ __forceinline__ bool is_finite_v(double a) { return ob(a) < INF_BITS64; }
__device__ __forceinline__ bool is_finite_v(float a) { return ob(a) < INF_BITS32; }
__device__ __forceinline__ double to_d(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ double to_d(double a) { return a; }
__device__ __forceinline__ double to_d(float a) { return (double)a; }
__device__ __forceinline__ bool updatable(float2 f) { return updatable(f.x); }
__device__ __forceinline__ bool is_src(float2 f) { return f.x < 0.0f; }
__device__ __forceinline__ bool is_src(double f) { return f < 0.0; }
__device__ __forceinline__ bool is_src(float f) { return f < 0.0f; }
__device__ __forceinline__ float2 shfl_xor(float2 v, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
template <typename T> __device__ __forceinline__ T zero_v();
template <> __device__ __forceinline__ double zero_v<double>() { return 0.0; }
template <> __device__ __forceinline__ float zero_v<float>() { return 0.0f; }
template <> __device__ __forceinline__ float2 zero_v<float2>() { return make_float2(0.0f, 0.0f); }

__device__ __forceinline__ float2 update_df(float2 W, float2 E, float2 S, float2 N, float2 f) {
    const float2 a = lt(E, W) ? E : W, b = lt(N, S) ? N : S;
    const bool ab = lt(a, b);
    const float2 lo = ab ? a : b, hi = ab ? b : a;
    const float INF = inf_of<float>();
    const float d = (hi.x - lo.x) + (hi.y - lo.y);
    const bool two_sided = hi.x < INF && d < f.x;
    // one pair sum for both branches: hi + increment (two-sided), lo + f
    // (one-sided); adding a pair whose low part is 0 equals df_add_f
    const float inc = increment_f32(two_sided ? d : 0.0f, f.x);
    const float2 r = df_add(two_sided ? hi : lo, two_sided ? make_float2(inc, 0.0f) : f);
    return lo.x < INF ? r : make_float2(INF, 0.0f);
}

// Exact conversions without the FP64 pipe (GB300 runs conversions there).
// split_pos: a positive double as a pair -- hi keeps the leading 24
// significand bits (exact in a float), lo the next 24 of the remaining 29
// (rounded, 2^-53 relative); false outside [2^-74, 2^126).  widen: a float as
// a double, exactly, from its bits alone (exponent rebias; a subnormal is
// normalised by its leading-zero count).
__device__ __forceinline__ bool split_pos(double v, float2* out) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 1023 - 74 || e > 1023 + 125) return false;
    const float hi = __uint_as_float(((unsigned)(e - 1023 + 127) << 23) | (unsigned)((b >> 29) & 0x7fffff));
    const float lo = __int2float_rn((int)(b & 0x1fffffffull)) * __uint_as_float((unsigned)(e - 1075 + 127) << 23);
    *out = make_float2(hi, lo);
    return true;
}
__device__ __forceinline__ double widen(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned long long b;
    if (e == 255u) {
        b = 0x7ff0000000000000ull | ((unsigned long long)m << 29);  // inf, NaN
    } else if (e != 0u) {
        b = ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    } else if (m == 0u) {
        b = 0ull;  // zero
    } else {
        // m 2^-149: the leading one moved to bit 23, exponent 2^(23 - lz - 149)
        const int lz = __clz(m) - 8;
        b = ((unsigned long long)(897 - lz) << 52) | ((unsigned long long)((m << lz) & 0x7fffffu) << 29);
    }
    return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) | b));
}

// The two-sided increment (f^2 - d^2) / (d + sqrt(2 f^2 - d^2)) in
// double-float arithmetic, 0 <= d < f.
__device__ __forceinline__ float2 df_increment(float2 d, float2 f) {
    const float2 f2 = df_mul(f, f);
    const float2 x = df_sub(df_add(f2, f2), df_mul(d, d));  // >= f^2 > 0
    return df_div(df_mul(df_sub(f, d), df_add(f, d)), df_add(d, df_sqrt(x)));
}

// FP64: U = hi + increment, with the increment -- at most sqrt 2 f, so a
// few units of 2^-46 relative to it are ~1e-14 f -- in double-float
// arithmetic on the FP32 pipe.  Only the difference d = hi - lo and the
// sums run on the FP64 pipe (three adds, no square root or division; one
// final add serves both branches), which on GB300 runs at 1/64 of the FP32
// rate.  fp: f as a pair, (0, 0)
// where f lies outside [2^-40, 2^40] (the pair products would leave the
// float range): the update then takes the FP64 root.
__device__ __forceinline__ double update_f64(double W, double E, double S, double N, double f, float2 fp) {
    const long long a = min(ob(W), ob(E)), b = min(ob(S), ob(N));
    const long long lob = min(a, b), hib = max(a, b);
    const double lo = from_ob(lob), hi = from_ob(hib);
    const double d = hi - lo;  // finite whenever hi is
    const bool two_sided = hib < INF_BITS64 && ob(d) < ob(f);
    float2 dp;
    if (!split_pos(d, &dp)) dp = make_float2(0.0f, 0.0f);  // d < 2^-74 (or not two-sided)
    const float2 inc = df_increment(dp, fp);
    if (two_sided && fp.x == 0.0f) {
        const double s = sqrt(fma(-d, d, 2.0 * f * f));
        return fma(0.5, s - d, hi);
    }
    // hi + increment (two-sided), lo + f (one-sided)
    return (two_sided ? hi : lo) + (two_sided ? widen(inc.x) + widen(inc.y) : f);
}
// f as the pair update_f64 takes
__device__ __forceinline__ float2 f64_pair(double f) {
    float2 r;
    if (f >= 0x1p-40 && f <= 0x1p40 && split_pos(f, &r)) return r;
    return make_float2(0.0f, 0.0f);
}

// ---------------------------------------------------------------- modes
enum { MODE_F64 = 0, MODE_F32 = 1, MODE_DF = 2 };

template <int MODE> struct ModeTypes;
template <> struct ModeTypes<MODE_F64> { using T = double; using FT = double; };
template <> struct ModeTypes<MODE_F32> { using T = float; using FT = float; };
template <> struct ModeTypes<MODE_DF> { using T = float2; using FT = float2; };

// One warp works on one cell (two cells for k = 4).  Its lanes sweep the four
// directions of Alg. FSM_order at the same time, LPD lanes per direction.  At
// wavefront step t the lanes of a direction update the nodes of anti-diagonal
// t of that direction.  For k <= 8 each lane owns one row of the tile (and
// keeps that row's changed-node mask in a register); for k >= 16 lane u takes
// the diagonal's nodes u, u + LPD, ...: every direction's diagonal t has the
// same length, so a slot no lane needs is skipped by the whole warp (k = 16:
// 46 slots a pass instead of 62), and changed nodes are marked by a byte
// each.  Lanes that reach the same node in one step read the same inputs and
// write the same value, so a pass of 2k-1 steps is four Gauss-Seidel sweeps,
// race free.
template <int MODE, int K>
struct TileCfg {
    using T = typename ModeTypes<MODE>::T;    // a value of U
    using FT = typename ModeTypes<MODE>::FT;  // f = h/F
    static constexpr int ES = (int)sizeof(T);
    static constexpr int LPD = K < 8 ? K : 8;        // lanes per direction
    static constexpr int LPC = 4 * LPD;              // lanes per cell
    static constexpr int CPW = 32 / LPC;             // cells per warp (lock-step)
    static constexpr int RPL = K / LPD;              // rows per lane
    // U box: k+2 rows; k+2 wide for 8-byte values, k+4 for floats (a row of
    // a TMA box must be a multiple of 16 bytes)
    static constexpr int BW = ES == 8 ? K + 2 : K + 4;
    static constexpr int BH = K + 2;
    static constexpr int UBYTES = BW * BH * ES;
    static constexpr int FBYTES = BW * BH * (int)sizeof(FT);        // f box incl. halo (TMA)
    static constexpr int XBYTES = MODE == MODE_F64 ? K * K * 8 : 0;  // f as pairs (computed)
    static constexpr int TX_BYTES = UBYTES + FBYTES;
    static constexpr int A128(int b) { return (b + 127) / 128 * 128; }
    static constexpr int F_OFF = A128(UBYTES);
    static constexpr int X_OFF = F_OFF + A128(FBYTES);
    static constexpr int FL_OFF = X_OFF + A128(XBYTES);               // k >= 16: a changed flag per node
    static constexpr int GROUP_BYTES = FL_OFF + A128(RPL > 1 ? K * K : 0);
    static constexpr int MASK_OFF = CPW * GROUP_BYTES;
    static constexpr int BAR_OFF = MASK_OFF + CPW * K * 8;
    static constexpr int WARP_BYTES = A128(BAR_OFF + 16);
    static constexpr int WPB_SMEM = (200 * 1024) / WARP_BYTES;
    static constexpr int WPB = WPB_SMEM >= 8 ? 8 : (WPB_SMEM < 1 ? 1 : WPB_SMEM);
    static constexpr int MAX_PASSES = K * K + 8;
    // HCM with locking: a lock byte per node of the warp's cells, after all
    // warps' areas (the other variants leave it out)
    static constexpr int LK_BYTES = A128(CPW * K * K);
    static constexpr int lk_area(int var) { return var == VAR_LSM ? WPB * LK_BYTES : 0; }
};

// ---------------------------------------------------------------- one node
// Candidate value of tile node (i, j) from its four tile neighbours (tU holds
// the cell plus its halo, row stride BW); false for sources and obstacles.
template <int MODE, int K>
__device__ __forceinline__ bool node_candidate(const typename TileCfg<MODE, K>::T* tU,
                                               const typename TileCfg<MODE, K>::FT* tF,
                                               const double* tG, int i, int j,
                                               typename TileCfg<MODE, K>::T& cand,
                                               typename TileCfg<MODE, K>::T& old) {
    using C = TileCfg<MODE, K>;
    const int q = (j + 1) * C::BW + (i + 1);
    const auto fv = tF[q];
    if (!updatable(fv)) return false;
    old = tU[q];
    if constexpr (MODE == MODE_F64)
        cand = update_f64(tU[q - 1], tU[q + 1], tU[q - C::BW], tU[q + C::BW], fv,
                          reinterpret_cast<const float2*>(tG)[j * K + i]);
    else if constexpr (MODE == MODE_F32)
        cand = update_f32(tU[q - 1], tU[q + 1], tU[q - C::BW], tU[q + C::BW], fv);
    else
        cand = update_df(tU[q - 1], tU[q + 1], tU[q - C::BW], tU[q + C::BW], fv);
    return true;
}

// The same, for a lane that may have nothing to update (act false): every
// input is loaded before anything is decided (the loads go out together,
// and no update waits for f to come back first).  On the FP32 pipe the
// update then runs without a branch -- a node that is not updated (a
// source, an obstacle, the padding, an inactive lane) computes a value the
// result masks; FP64 updates, at 1/64 of the FP32 rate on this part, are
// skipped by a branch when the lane has none to make.
template <int MODE, int K>
__device__ __forceinline__ bool node_eval(const typename TileCfg<MODE, K>::T* tU,
                                          const typename TileCfg<MODE, K>::FT* tF, const double* tG, int i,
                                          int j, bool act, typename TileCfg<MODE, K>::T& cand,
                                          typename TileCfg<MODE, K>::T& old) {
    using C = TileCfg<MODE, K>;
    const int q = (j + 1) * C::BW + (i + 1);
    const auto fv = tF[q];
    old = tU[q];
    const auto W = tU[q - 1], E = tU[q + 1], S = tU[q - C::BW], N = tU[q + C::BW];
    const bool upd = act && updatable(fv);
    if constexpr (MODE == MODE_F64) {
        const float2 fp = reinterpret_cast<const float2*>(tG)[j * K + i];
        cand = old;
        if (upd) cand = update_f64(W, E, S, N, fv, fp);
    } else if constexpr (MODE == MODE_F32) {
        cand = update_f32(W, E, S, N, fv);
    } else {
        cand = update_df(W, E, S, N, fv);
    }
    return upd;
}

// Linear addressing of the anti-diagonal slots (k >= 16, FP32 and
// double-float modes).  In sweep coordinates node u of diagonal t2 is
// (jj, ii2) = (u, t2 - u) for t2 < k and (t2 - (k-1) + u, k-1-u) after; its
// tile index (j+1) BW + i + 1 and flag index j k + i are therefore a base per
// half plus u times a per-direction delta plus t2 times a per-half delta.
// Computed once per visit, they leave an add per slot on the step's
// dependent chain instead of the index arithmetic a fresh step would redo
// after each warp barrier (a step of a 16-node cell alone: 468 -> 359 cycles
// for a warp, 925 -> 824 with three blocks per SM; the 4097^2 pass 10.47 ->
// 9.59 ms, its sweeps ~29 K -> ~19 K cycles per visit; with the loops of a
// fixed slot count below, the 512-grid batch's pass 11.6 -> 11.1 ms).
struct DiagLin {
    int qz0, qz1, fz0, fz1;  // node u = 0 at t2 = 0 of each half (the second extrapolated)
    int dq0, dq1, df0, df1;  // per step, each half
    int dqu, dfu;            // per unit of u
    int qrl, frl, qsl, fsl;  // this lane's first slot (u = rl) and the slot stride (u += LPD)
};
template <int K, int BW>
__device__ __forceinline__ DiagLin diag_lin(bool sx, bool sy, int rl = 0, int lpd = 8) {
    DiagLin L;
    const int sgx = sx ? 1 : -1, sgy = sy ? 1 : -1;
    const int j0 = sy ? 0 : K - 1, i0 = sx ? 0 : K - 1;
    L.qz0 = (j0 + 1) * BW + (i0 + 1);
    L.fz0 = j0 * K + i0;
    const int j1 = sy ? -(K - 1) : 2 * K - 2, i1 = sx ? K - 1 : 0;
    L.qz1 = (j1 + 1) * BW + (i1 + 1);
    L.fz1 = j1 * K + i1;
    L.dq0 = sgx;
    L.df0 = sgx;
    L.dq1 = sgy * BW;
    L.df1 = sgy * K;
    L.dqu = sgy * BW - sgx;
    L.dfu = sgy * K - sgx;
    L.qrl = rl * L.dqu;
    L.frl = rl * L.dfu;
    L.qsl = lpd * L.dqu;
    L.fsl = lpd * L.dfu;
    return L;
}
// One step with linear addresses: this lane's NS slots of diagonal t2 (len
// nodes), loads first, then the branch-free updates, then the stores.
template <int MODE, int K, int NS>
__device__ __forceinline__ bool diag_step_lin(typename TileCfg<MODE, K>::T* tU,
                                              const typename TileCfg<MODE, K>::FT* tF, unsigned char* flags, int t2,
                                              int len, int rl, const DiagLin& L, bool on) {
    using C = TileCfg<MODE, K>;
    typename C::T cand[NS], old[NS];
    bool ok[NS];
    int qq[NS], ff[NS];
    const bool first = t2 < K;
    const int qb = first ? L.qz0 + L.dq0 * t2 : L.qz1 + L.dq1 * t2;
    const int fb = first ? L.fz0 + L.df0 * t2 : L.fz1 + L.df1 * t2;
#pragma unroll
    for (int m = 0; m < NS; ++m) {
        const int u = rl + C::LPD * m;
        const bool a = on && u < len;
        // an idle slot reads the diagonal's first node
        const int q = a ? qb + L.qrl + m * L.qsl : qb;
        qq[m] = q;
        ff[m] = a ? fb + L.frl + m * L.fsl : fb;
        const auto fv = tF[q];
        old[m] = tU[q];
        const auto W = tU[q - 1], E = tU[q + 1], S = tU[q - C::BW], N = tU[q + C::BW];
        ok[m] = a && updatable(fv);
        if constexpr (MODE == MODE_F32) cand[m] = update_f32(W, E, S, N, fv);
        else cand[m] = update_df(W, E, S, N, fv);
    }
    bool changed = false;
#pragma unroll
    for (int m = 0; m < NS; ++m) {
        if (ok[m] && lt(cand[m], old[m])) {
            tU[qq[m]] = cand[m];
            flags[ff[m]] = 1;
            changed = true;
        }
    }
    return changed;
}
// A whole pass (2k-1 steps) as loops of a fixed slot count: diagonal t2
// holds len = t2 + 1 nodes while rising and 2k-1-t2 after, so ns =
// ceil(len / LPD) steps up from 1 to RPL over t2 < LPD (RPL - 1) and back
// down over the last LPD (RPL - 1) steps; each loop's steps compile without
// a dispatch on ns (a 16-node cell's step alone: 429 -> 359 cycles for a
// warp, 703 -> 645 at two blocks per SM; the 4097^2 pass: 9.59 -> 9.56 ms,
// whose visits now spend ~19 K of ~33 K cycles in sweeps).
template <int MODE, int K, int NS = 1>
__device__ __forceinline__ bool diag_pass_lin(typename TileCfg<MODE, K>::T* tU,
                                              const typename TileCfg<MODE, K>::FT* tF, unsigned char* flags, int rl,
                                              const DiagLin& L, bool on) {
    using C = TileCfg<MODE, K>;
    constexpr int P = C::LPD;
    bool changed = false;
    if constexpr (NS < C::RPL) {
        // rising: t2 in [P (NS - 1), P NS); then the phases above; then falling
        for (int t2 = P * (NS - 1); t2 < P * NS; ++t2) {
            changed |= diag_step_lin<MODE, K, NS>(tU, tF, flags, t2, t2 + 1, rl, L, on);
            __syncwarp();
        }
        changed |= diag_pass_lin<MODE, K, NS + 1>(tU, tF, flags, rl, L, on);
        for (int t2 = 2 * K - 1 - P * NS; t2 < 2 * K - 1 - P * (NS - 1); ++t2) {
            changed |= diag_step_lin<MODE, K, NS>(tU, tF, flags, t2, 2 * K - 1 - t2, rl, L, on);
            __syncwarp();
        }
    } else {
        // the middle: every diagonal of RPL slots
        for (int t2 = P * (NS - 1); t2 < 2 * K - 1 - P * (NS - 1); ++t2) {
            const int len = t2 < K ? t2 + 1 : 2 * K - 1 - t2;
            changed |= diag_step_lin<MODE, K, NS>(tU, tF, flags, t2, len, rl, L, on);
            __syncwarp();
        }
    }
    return changed;
}

// Fixed-point check of a whole tile (this lane's share): true if some node
// would still decrease.  It is equivalent to asking whether another pass
// would change anything -- a pass changes nothing exactly when no node can
// decrease -- but all nodes are evaluated at once instead of along 2k-1
// wavefront steps.
template <int MODE, int K>
__device__ __forceinline__ bool tile_improvable(const typename TileCfg<MODE, K>::T* tU,
                                                const typename TileCfg<MODE, K>::FT* tF,
                                                const double* tG, int dl) {
    using C = TileCfg<MODE, K>;
    bool imp = false;
#pragma unroll 4
    for (int e = dl; e < K * K; e += C::LPC) {
        const int j = e / K, i = e - j * K;
        typename C::T cand, old;
        const bool upd = node_eval<MODE, K>(tU, tF, tG, i, j, true, cand, old);
        imp |= upd && lt(cand, old);
    }
    return imp;
}

// Locking (Remark locking_FSM): node (i, j) of the tile has just decreased;
// unlock each neighbour inside the cell whose value is larger -- the only
// ones whose local update can use the new value.
template <int MODE, int K>
__device__ __forceinline__ void unlock_larger(const typename TileCfg<MODE, K>::T* tU, unsigned char* lk, int i,
                                              int j) {
    using C = TileCfg<MODE, K>;
    const int q = (j + 1) * C::BW + (i + 1);
    const auto v = tU[q];
    if (i > 0 && lt(v, tU[q - 1])) lk[j * K + i - 1] = 1;
    if (i < K - 1 && lt(v, tU[q + 1])) lk[j * K + i + 1] = 1;
    if (j > 0 && lt(v, tU[q - C::BW])) lk[(j - 1) * K + i] = 1;
    if (j < K - 1 && lt(v, tU[q + C::BW])) lk[(j + 1) * K + i] = 1;
}

// ---------------------------------------------------------------- grid barrier
// Counting barrier across all (co-resident) blocks.  Every wait is bounded by
// the launch deadline and by the abort flag; on expiry the block records
// EIK_ETIMEDOUT, raises abort and returns false.
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
                __nanosleep(40);
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

__device__ __forceinline__ void lane_push(int* list, int* count, int val, int cap, Ctl* ctl) {
    const int pos = atomicAdd(count, 1);
    if (pos < cap) list[pos] = val;
    else fail(ctl, EIK_ECUDA, 0x2000000ull + (unsigned)pos);
}

// ---------------------------------------------------------------- block scan
// Exclusive prefix sums of in[0..n) into out[0..n], out[n] = total; every
// thread of the block must call it (uses `scratch`, >= 33 ints).
__device__ __forceinline__ int block_exclusive_scan(const int* in, int* out, int n, int* scratch) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = (nt + 31) >> 5;
    const int per = (n + nt - 1) / nt;
    const int lo = min(tid * per, n), hi = min(lo + per, n);
    int s = 0;
    for (int e = lo; e < hi; ++e) s += in[e];
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) scratch[wid] = incl;
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int w = 0; w < nw; ++w) {
            const int v = scratch[w];
            scratch[w] = run;
            run += v;
        }
        scratch[32] = run;
    }
    __syncthreads();
    int run = scratch[wid] + incl - s;
    for (int e = lo; e < hi; ++e) {
        out[e] = run;
        run += in[e];
    }
    const int total = scratch[32];
    if (tid == 0) out[n] = total;
    __syncthreads();
    return total;
}

// index of the instance whose [pre[i], pre[i+1]) range holds e (pre ascending)
__device__ __forceinline__ int find_inst(const int* pre, int n, int e) {
    int lo = 0, hi = n;  // pre[lo] <= e < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

// per-instance state kept (identically) in every block's shared memory
struct InstState {
    unsigned long long* theta;  // current bucket's upper key
    int* pre;                   // prefix sums (n + 1)
    int* nn;                    // near-list length this round
    int* nf;                    // far-list length this round
    unsigned char* ns;          // near-list slot (0..2)
    unsigned char* fs;          // far-list slot (0..1)
    int* scan_scratch;          // 33 ints
};
__host__ __device__ constexpr int inst_state_bytes(int n) {
    return n * 8 + (n + 1) * 4 + n * 4 + n * 4 + n + n + 33 * 4 + 64;
}

__device__ __forceinline__ void flush_counters(const InstDesc* inst, int i, unsigned long long& v,
                                               unsigned long long& sw, unsigned long long& l) {
    if (i >= 0 && v) {
        Ctl* c = inst[i].ctl;
        atomicAdd(&c->visits, v);
        atomicAdd(&c->sweeps, sw);
        atomicAdd(&c->lane_updates, l);
    }
    v = sw = l = 0;
}

// ---------------------------------------------------------------- one visit
// PROF_MARK(i): add the cycles since the last mark to phase i (profiling only)
#define PROF_MARK(i)                                    \
    do {                                                \
        if (prof_on) {                                  \
            const long long now_ = clock64();           \
            pacc[i] += (unsigned long long)(now_ - pt); \
            pt = now_;                                  \
        }                                               \
    } while (0)

// Per-warp state of the solver kernels: the warp's tile buffers in shared
// memory, its lane roles and its counters.
template <int MODE, int K>
struct WarpState {
    using C = TileCfg<MODE, K>;
    using T = typename C::T;
    using FT = typename C::FT;
    int lane, g, dl, dir, rl;
    bool sx, sy;
    unsigned char* wbase;
    uint64_t* bar;
    unsigned long long* masks;
    T* tU;
    const FT* tF;
    const double* tG;
    unsigned char* lk;  // HCM with locking: the lock bytes of this lane's cell
    unsigned gmask;
    uint32_t phase;
    // counters gather per lane while the instance stays the same (one flush
    // per instance change instead of three atomics per visit on one address)
    int acc_inst;
    unsigned long long acc_visits, acc_sweeps, acc_lane, st_lane;
    unsigned long long mono_ok, mono_n;  // FHCM Monotonicity Checks
    int cap;  // passes per removal before EIK_ENOTCONVERGED

    __device__ __forceinline__ void init(unsigned char* smem, int max_passes = 0) {
        cap = max_passes > 0 && max_passes < C::MAX_PASSES ? max_passes : C::MAX_PASSES;
        lane = threadIdx.x & 31;
        const int warp = threadIdx.x >> 5;
        wbase = smem + warp * C::WARP_BYTES;
        bar = reinterpret_cast<uint64_t*>(wbase + C::BAR_OFF);
        masks = reinterpret_cast<unsigned long long*>(wbase + C::MASK_OFF);
        g = lane / C::LPC;    // which of the warp's cells this lane works on
        dl = lane % C::LPC;   // lane within the cell
        dir = dl / C::LPD;    // sweep direction of this lane (Alg. FSM_order)
        rl = dl % C::LPD;     // first tile row of this lane
        sx = dir <= 1;                  // i increasing
        sy = (dir == 0) || (dir == 3);  // j increasing
        unsigned char* gbase = wbase + g * C::GROUP_BYTES;
        tU = reinterpret_cast<T*>(gbase);
        tF = reinterpret_cast<const FT*>(gbase + C::F_OFF);
        tG = reinterpret_cast<const double*>(gbase + C::X_OFF);
        gmask = C::LPC == 32 ? 0xffffffffu : (((1u << C::LPC) - 1u) << (g * C::LPC));
        lk = smem + C::WPB * C::WARP_BYTES + warp * C::LK_BYTES + g * K * K;  // used by VAR_LSM only
        phase = 0;
        acc_inst = -1;
        acc_visits = acc_sweeps = acc_lane = st_lane = 0;
        mono_ok = mono_n = 0;
        if (lane == 0) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
    }
};

// A pause of up to jitter_ns before a removal's tile load (0: none), drawn
// from the cell, the removal's start time and the warp: a host-set
// perturbation of the schedule, whose result must not change (Theorem
// convergence).  Bounded: __nanosleep's pause is at most about twice its
// argument.
__device__ __forceinline__ void jitter(unsigned jitter_ns, unsigned cell) {
    if (!jitter_ns) return;
    unsigned x = cell * 0x9E3779B1u ^ (unsigned)gtimer() ^ (threadIdx.x >> 5) * 0x85EBCA6Bu;
    x ^= x >> 15;
    x *= 0x2C1B3C6Du;
    x ^= x >> 12;
    __nanosleep(x % (jitter_ns + 1u));
}

// Solve the warp's cells cg[0..CPW) of instances ig[] (cell -1: none), which
// the caller has already claimed (flag cleared, fences issued): TMA load of
// each tile with its halo, passes of four concurrent directional sweeps to
// the fixed point, write-back of the changed nodes, then the activation test
// of every side (Alg. generic_LC_cells) with the neighbour's cell value
// (eq. cell_value, min-updated here when CVAL: the bucketed schedule orders
// by it, the round-free one does not need it).  For each side with a neighbour, one
// lane calls act(d, nc, key, old, activate): key/old the proposed and the
// previous cell value of neighbour cell nc of instance d, activate the
// outcome of the test -- the scheduler's part.  c, ii, first: this lane's
// cell, its instance and whether this is the cell's first removal.  VAR:
// VAR_HCM, VAR_FHCM (one pass of the flagged directions) or VAR_LSM (HCM
// whose passes update only unlocked nodes).  Returns false when the TMA wait
// gave up (abort raised).
template <int MODE, int K, bool CVAL, int VAR, class Act>
__device__ __forceinline__ bool visit_cells(WarpState<MODE, K>& w, const InstDesc* inst, Ctl* gctl,
                                            unsigned long long deadline, int c, int ii, int first,
                                            const int* cg, const int* ig, int prof_on,
                                            unsigned long long* pacc, long long& pt, Act&& act) {
    using C = TileCfg<MODE, K>;
    using T = typename C::T;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr bool FAST = VAR == VAR_FHCM, LSM = VAR == VAR_LSM;
    const int lane = w.lane, g = w.g, dl = w.dl, dir = w.dir, rl = w.rl;
    const bool sx = w.sx, sy = w.sy;
    T* tU = w.tU;
    const auto* tF = w.tF;
    const double* tG = w.tG;
    unsigned char* wbase = w.wbase;
    unsigned long long* masks = w.masks;
    const InstDesc& d = inst[ii];
    Ctl* ictl = d.ctl;
    const int cxn = d.cxn, cyn = d.cyn;

    // ---- TMA: U box (cell + halo) and f box (+ halo) into shared memory
    if (lane == 0) {
        int nvalid = 0;
#pragma unroll
        for (int gg = 0; gg < C::CPW; ++gg) nvalid += cg[gg] >= 0;
        mbar_arrive_expect_tx(w.bar, (uint32_t)(nvalid * C::TX_BYTES));
#pragma unroll
        for (int gg = 0; gg < C::CPW; ++gg) {
            if (cg[gg] >= 0) {
                const InstDesc& dg = inst[ig[gg]];
                const int cxg = cg[gg] % dg.cxn, cyg = cg[gg] / dg.cxn;
                unsigned char* gb = wbase + gg * C::GROUP_BYTES;
                tma_load_2d(gb, &dg.tmU, cxg * K, cyg * K, w.bar);
                tma_load_2d(gb + C::F_OFF, &dg.tmF, cxg * K, cyg * K, w.bar);
            }
        }
    }
    {
        bool got = false;
        unsigned spins = 0;
        for (;;) {
            if (mbar_try_wait(w.bar, w.phase)) { got = true; break; }
            if ((++spins & 255u) == 0 && gtimer() > deadline) break;
        }
        if (!got) {
            fail(gctl, EIK_ETIMEDOUT, 0x3000000ull);
            // let our own copies land before the block leaves (bounded)
            const unsigned long long d2 = gtimer() + 1000000000ull;
            while (!mbar_try_wait(w.bar, w.phase) && gtimer() < d2) {
            }
            return false;
        }
    }
    w.phase ^= 1u;
    PROF_MARK(3);
    if constexpr (MODE == MODE_F64) {
        // f as a pair per node, once per visit (the update's increment)
        for (int e = lane; e < C::CPW * K * K; e += 32) {
            const int gg = e / (K * K), r = e - gg * (K * K);
            const int jj = r / K, i2 = r - jj * K;
            unsigned char* gb = wbase + gg * C::GROUP_BYTES;
            const double fv = reinterpret_cast<const double*>(gb + C::F_OFF)[(jj + 1) * C::BW + i2 + 1];
            reinterpret_cast<float2*>(gb + C::X_OFF)[r] = f64_pair(fv);
        }
        __syncwarp();
    }

    // ---- FHCM (Alg. FHCM): the cell's directional flags, taken and cleared
    // now (after the claim); only the flagged directions sweep, once
    int fl = 15;
    if constexpr (FAST) {
        int mine = 0;
        if (dl == 0 && c >= 0) mine = atomicExch(&d.dflags[c], 0);
        fl = __shfl_sync(FULL, mine, g * C::LPC);
        if (fl == 0) fl = 15;  // a cell queued without flags: sweep all four
    }
    const bool dir_on = (fl >> dir) & 1;

    // ---- passes of four concurrent directional sweeps until a pass
    // changes nothing or the fixed-point check finds nothing to improve
    // (FHCM: one pass of the flagged directions)
    // k <= 8: this lane's row mask of changed nodes; k >= 16: a byte per node
    // of this visit, 1 once the node has changed (lanes of several directions
    // that change one node in one step all store 1)
    constexpr bool DIAG = C::RPL > 1;
    unsigned chg = 0u;  // k <= 8: bit i of this lane's row
    // k <= 8: this lane's row, in sweep order (live at steps jr .. jr + K - 1)
    const int jr = sy ? rl : K - 1 - rl;
    const bool lane_on = c >= 0 && (!FAST || dir_on);
    unsigned char* flags = wbase + g * C::GROUP_BYTES + C::FL_OFF;
    if constexpr (DIAG) {
        for (int e = 4 * dl; e < K * K; e += 4 * C::LPC) *reinterpret_cast<unsigned*>(flags + e) = 0u;
        __syncwarp();
    }
    // HCM with locking (Sec. 4.2 sweeps a removed cell by the Locking
    // Sweeping version, Remark locking_FSM): the cell was left at its fixed
    // point by its last removal, so only the nodes next to a neighbouring
    // cell, whose boundary data may have changed since, start unlocked --
    // and on the first removal also the nodes next to a source of the cell.
    // A pass updates only unlocked nodes; each node it takes is locked as it
    // is taken, and a decrease unlocks the node's larger neighbours in the
    // cell.  Within a step only locks are written before the barrier and
    // only unlocks after it, so a node that read a neighbour's old value in
    // the step the neighbour changed is unlocked again.  (Lanes of two
    // directions that reach one node in one step: the one that finds it
    // already locked skips it, and the other computes the same update.)  The
    // visit ends when no node is unlocked.
    unsigned char* lk = w.lk;
    int nev = 0;  // local updates this lane computed
    if constexpr (LSM) {
        if (c >= 0) {
            const int cx = c % cxn, cy = c / cxn;
            for (int e = dl; e < K * K; e += C::LPC) {
                const int j = e / K, i = e - j * K;
                const int q = (j + 1) * C::BW + (i + 1);
                bool u = false;
                if (updatable(tF[q])) {
                    u = (i == 0 && cx > 0) || (i == K - 1 && cx + 1 < cxn) || (j == 0 && cy > 0) ||
                        (j == K - 1 && cy + 1 < cyn);
                    if (!u && first)
                        u = (i > 0 && is_src(tF[q - 1])) || (i < K - 1 && is_src(tF[q + 1])) ||
                            (j > 0 && is_src(tF[q - C::BW])) || (j < K - 1 && is_src(tF[q + C::BW]));
                }
                lk[e] = u ? 1 : 0;
            }
        }
        __syncwarp();
    }
    int gsweeps = 0;
    bool gdone = c < 0;
    int s = 0;
    const int cap = w.cap;
    [[maybe_unused]] const DiagLin dlin = diag_lin<K, C::BW>(sx, sy, rl, C::LPD);
    for (; s < cap && __ballot_sync(FULL, !gdone) != 0u; ++s) {
        bool changed = false;
        // FP32 and double-float passes with k >= 16: loops of a fixed slot
        // count with linear addresses (the t2 loop below then runs no step)
        constexpr bool PHASED = DIAG && !LSM && MODE != MODE_F64;
        if constexpr (PHASED)
            changed = diag_pass_lin<MODE, K>(tU, tF, flags, rl, dlin, c >= 0 && (!FAST || dir_on));
        for (int t2 = 0; t2 < (PHASED ? 0 : 2 * K - 1); ++t2) {
            if constexpr (LSM) {
                if constexpr (!DIAG) {
                    const unsigned ii2 = (unsigned)(t2 - jr);
                    const int j = rl, i = sx ? (int)ii2 : K - 1 - (int)ii2;
                    bool dec = false;
                    if (lane_on && ii2 < (unsigned)K && lk[j * K + i]) {
                        lk[j * K + i] = 0;
                        T cand, old;
                        if (node_candidate<MODE, K>(tU, tF, tG, i, j, cand, old)) {
                            ++nev;
                            if (lt(cand, old)) {
                                tU[(j + 1) * C::BW + (i + 1)] = cand;
                                chg |= 1u << i;
                                changed = true;
                                dec = true;
                            }
                        }
                    }
                    __syncwarp();
                    if (dec) unlock_larger<MODE, K>(tU, lk, i, j);
                } else {
                    const int lo = t2 < K ? 0 : t2 - (K - 1);
                    const int len = (t2 < K ? t2 : K - 1) - lo + 1;
                    unsigned dec = 0u;
                    auto node = [&](int m, int& i, int& j) {
                        const int jj = lo + rl + C::LPD * m, ii2 = t2 - jj;
                        j = sy ? jj : K - 1 - jj;
                        i = sx ? ii2 : K - 1 - ii2;
                    };
#pragma unroll
                    for (int m = 0; m < C::RPL; ++m) {
                        if (m * C::LPD < len && rl + C::LPD * m < len && c >= 0) {
                            int i, j;
                            node(m, i, j);
                            if (lk[j * K + i]) {
                                lk[j * K + i] = 0;
                                T cand, old;
                                if (node_candidate<MODE, K>(tU, tF, tG, i, j, cand, old)) {
                                    ++nev;
                                    if (lt(cand, old)) {
                                        tU[(j + 1) * C::BW + (i + 1)] = cand;
                                        flags[j * K + i] = 1;
                                        changed = true;
                                        dec |= 1u << m;
                                    }
                                }
                            }
                        }
                    }
                    __syncwarp();
#pragma unroll
                    for (int m = 0; m < C::RPL; ++m)
                        if ((dec >> m) & 1u) {
                            int i, j;
                            node(m, i, j);
                            unlock_larger<MODE, K>(tU, lk, i, j);
                        }
                }
            } else if constexpr (!DIAG) {
                // this lane's row (node ii2 of it at this step, when in range):
                // evaluated without a branch, stored when in range and lower
                const unsigned ii2 = (unsigned)(t2 - jr);
                const bool a = lane_on && ii2 < (unsigned)K;
                const int ic = a ? (int)ii2 : 0;
                const int j = rl, i = sx ? ic : K - 1 - ic;
                T cand, old;
                if (node_eval<MODE, K>(tU, tF, tG, i, j, a, cand, old) && lt(cand, old)) {
                    tU[(j + 1) * C::BW + (i + 1)] = cand;
                    chg |= 1u << i;
                    changed = true;
                }
            } else if constexpr (MODE == MODE_F64) {
                // FP64: the slots one after another (its updates are bound by
                // the FP64 pipe, not by the chain's latency, and the straight-
                // line block measured slower: k = 32 11.4 against 8.2 ms on
                // the 1025^2 sin20 grid)
                const int len = t2 < K ? t2 + 1 : 2 * K - 1 - t2;
                const bool first = t2 < K;  // linear addresses, as above
                const int qb = first ? dlin.qz0 + dlin.dq0 * t2 : dlin.qz1 + dlin.dq1 * t2;
                const int fb = first ? dlin.fz0 + dlin.df0 * t2 : dlin.fz1 + dlin.df1 * t2;
#pragma unroll
                for (int m = 0; m < C::RPL; ++m) {
                    if (m * C::LPD < len) {  // the same for every lane
                        const int u = rl + C::LPD * m;
                        if (u < len && c >= 0 && (!FAST || dir_on)) {
                            const int q = qb + u * dlin.dqu, fi = fb + u * dlin.dfu;
                            const auto fv = tF[q];
                            if (updatable(fv)) {
                                const T old = tU[q];
                                const T cand = update_f64(tU[q - 1], tU[q + 1], tU[q - C::BW], tU[q + C::BW], fv,
                                                          reinterpret_cast<const float2*>(tG)[fi]);
                                if (lt(cand, old)) {
                                    tU[q] = cand;
                                    flags[fi] = 1;
                                    changed = true;
                                }
                            }
                        }
                    }
                }
            }
            __syncwarp();
        }
        if constexpr (LSM) {
            // done when every node of the cell is locked
            bool left = false;
            if (c >= 0)
                for (int e = 4 * dl; e < K * K; e += 4 * C::LPC)
                    left |= *reinterpret_cast<const unsigned*>(lk + e) != 0u;
            const unsigned anyl = __ballot_sync(FULL, left);
            if (!gdone) {
                gsweeps += 4;
                if (!(anyl & w.gmask)) gdone = true;
            }
        } else {
            const unsigned any = __ballot_sync(FULL, changed);
            if constexpr (FAST) {
                if (!gdone) gsweeps += __popc(fl);
                gdone = true;
            }
            if (!gdone) {
                gsweeps += 4;
                if (!(any & w.gmask)) gdone = true;
            }
            bool imp = false;
            if (!gdone) imp = tile_improvable<MODE, K>(tU, tF, tG, dl);
            const unsigned anyi = __ballot_sync(FULL, imp);
            if (!gdone && !(anyi & w.gmask)) {
                gdone = true;
                ++gsweeps;  // counted like the confirming sweep it replaces
            }
        }
        if (__ballot_sync(FULL, !gdone) == 0u) break;
        if ((s & 15) == 15) {
            // values only decrease, so stopping early leaves valid upper
            // bounds; the expired deadline aborts the launch
            const unsigned long long now = __shfl_sync(FULL, gtimer(), 0);
            if (now > deadline) {
                if (lane == 0) fail(gctl, EIK_ETIMEDOUT, 0x4000000ull);
                s = cap + 1;
                break;
            }
        }
    }
    if (s == cap && !gdone && dl == 0 && c >= 0) {
        atomicCAS(&ictl->status, 0, EIK_ENOTCONVERGED);
        fail(gctl, EIK_ENOTCONVERGED, (unsigned)c);
    }
    if constexpr (LSM) {  // the cell's lanes' local updates
#pragma unroll
        for (int o = C::LPC / 2; o > 0; o >>= 1) nev += __shfl_xor_sync(FULL, nev, o);
    }
    if (dl == 0 && c >= 0) {
        // node evaluations executed for this cell (lock-step passes included;
        // with locking the local updates computed)
        const unsigned long long ev =
            LSM ? (unsigned long long)nev : (unsigned long long)(s < cap ? s + 1 : cap) * 4 * K * K;
        if (ii != w.acc_inst) {
            flush_counters(inst, w.acc_inst, w.acc_visits, w.acc_sweeps, w.acc_lane);
            w.acc_inst = ii;
        }
        w.acc_visits += 1;
        w.acc_sweeps += (unsigned long long)gsweeps;
        w.acc_lane += ev;
        w.st_lane += ev;
    }
    PROF_MARK(4);

    // ---- changed-node masks per row: union over the four directions
    if constexpr (!DIAG) {
        // the four directions' lanes of a row hold its masks
        unsigned v = chg;
        v |= __shfl_xor_sync(FULL, v, C::LPD);
        v |= __shfl_xor_sync(FULL, v, 2 * C::LPD);
        if (dir == 0) masks[g * K + rl] = v;
    } else {
        // from the flag bytes (0 or 1 each): eight bytes folded into their
        // low eight bits by OR-ing shifted copies
        for (int j = dl; j < K; j += C::LPC) {
            unsigned long long v = 0ull;
#pragma unroll
            for (int i0 = 0; i0 < K; i0 += 8) {
                unsigned long long x = *reinterpret_cast<const unsigned long long*>(flags + j * K + i0);
                x |= x >> 7;
                x |= x >> 14;
                x |= x >> 28;
                v |= (x & 0xffull) << i0;
            }
            masks[g * K + j] = v;
        }
    }
    __syncwarp();
    // ---- write back the nodes that changed (coalesced across lanes).  One
    // cell per warp: the descriptor is read and the cell's origin formed once,
    // before the stores (which the compiler must assume may alias it).
    if constexpr (C::CPW == 1) {
        if (cg[0] >= 0) {
            const InstDesc& dc = inst[ig[0]];
            const int cxn0 = dc.cxn;
            const size_t up = dc.upitch;
            T* const gbase = reinterpret_cast<T*>(dc.U) + (size_t)((cg[0] / cxn0) * K + 1) * up +
                             (size_t)((cg[0] % cxn0) * K + 1);
            const T* gU = reinterpret_cast<const T*>(wbase);
#pragma unroll 8
            for (int e = lane; e < K * K; e += 32) {
                const int j = e / K, i = e - (e / K) * K;
                if ((masks[j] >> i) & 1ull) gbase[(size_t)j * up + i] = gU[(j + 1) * C::BW + (i + 1)];
            }
        }
    } else
    for (int e = lane; e < C::CPW * K * K; e += 32) {
        const int gg = e / (K * K);
        const int rem = e - gg * K * K;
        const int j = rem / K, i = rem - j * K;
        int cc = cg[0], ic = ig[0];
#pragma unroll
        for (int q = 1; q < C::CPW; ++q)
            if (gg == q) { cc = cg[q]; ic = ig[q]; }
        if (cc >= 0 && ((masks[gg * K + j] >> i) & 1ull)) {
            const InstDesc& dc = inst[ic];
            const int cx = cc % dc.cxn, cy = cc / dc.cxn;
            const T* gU = reinterpret_cast<const T*>(wbase + gg * C::GROUP_BYTES);
            reinterpret_cast<T*>(dc.U)[(size_t)(cy * K + j + 1) * dc.upitch + (size_t)(cx * K + i + 1)] =
                gU[(j + 1) * C::BW + (i + 1)];
        }
    }
    fence_acq_rel_gpu();  // release the new values before any activation
    fence_proxy_async_global();
    __syncwarp();
    PROF_MARK(5);

    // ---- activation of the neighbours (Alg. generic_LC_cells) and their
    // cell values (eq. cell_value).  Side sd: 0 W, 1 E, 2 S, 3 N.  The lanes
    // of sweep direction d take side d: LPD lanes per side, each owning
    // k/LPD boundary nodes; the first lane of each side then issues that
    // side's atomics, all four sides at once.  Everything the test needs
    // (values, changed flags, and f across the boundary, whose sign marks
    // sources) is in shared memory.
    {
        const int sd = dir;
        const int cx = c >= 0 ? c % cxn : 0, cy = c >= 0 ? c / cxn : 0;
        bool has_nb = false;
        if (c >= 0) has_nb = sd == 0 ? cx > 0 : sd == 1 ? cx + 1 < cxn : sd == 2 ? cy > 0 : cy + 1 < cyn;
        bool cond = false;
        T vmax = zero_v<T>();
        int bmax = -1;
#pragma unroll
        for (int m = 0; m < C::RPL; ++m) {
            const int b = rl + C::LPD * m;
            int bi, bj, ai, aj;
            if (sd == 0) { bi = 0; bj = b; ai = -1; aj = b; }
            else if (sd == 1) { bi = K - 1; bj = b; ai = K; aj = b; }
            else if (sd == 2) { bi = b; bj = 0; ai = b; aj = -1; }
            else { bi = b; bj = K - 1; ai = b; aj = K; }
            if (has_nb) {
                const int qb = (bj + 1) * C::BW + (bi + 1), qa = (aj + 1) * C::BW + (ai + 1);
                const T vb = tU[qb], va = tU[qa];
                const bool ch = (masks[g * K + bj] >> bi) & 1ull;
                // V_i changed (or x_i in Q on the first removal),
                // V_i < V_j, and x_j not in Q
                cond = cond || ((ch || (first && is_src(tF[qb]))) && lt(vb, va) && !is_src(tF[qa]));
                if (is_finite_v(vb) && (bmax < 0 || lt(vmax, vb))) { vmax = vb; bmax = b; }
            }
        }
        const unsigned smask = ((1u << C::LPD) - 1u) << (g * C::LPC + sd * C::LPD);
        const bool activate = (__ballot_sync(FULL, cond) & smask) != 0u;
        // max finite boundary value on this side, and where (argmax)
#pragma unroll
        for (int o = C::LPD / 2; o > 0; o >>= 1) {
            const T ov = shfl_xor(vmax, o);
            const int obm = __shfl_xor_sync(FULL, bmax, o);
            if (obm >= 0 && (bmax < 0 || lt(vmax, ov) || (!lt(ov, vmax) && obm > bmax))) {
                vmax = ov;
                bmax = obm;
            }
        }
        // FHCM: the neighbour's flags, from the Monotonicity Check of this
        // border (its values along the border coordinate: non-increasing ->
        // the sweep that runs against it, non-decreasing -> the one that runs
        // with it, neither -> both), released before the activation
        if (FAST && rl == 0 && has_nb && activate) {
            bool nondec = true, noninc = true;
            T prev = zero_v<T>();
            for (int b = 0; b < K; ++b) {
                const int bi = sd == 0 ? 0 : sd == 1 ? K - 1 : b;
                const int bj = sd == 2 ? 0 : sd == 3 ? K - 1 : b;
                const T v = tU[(bj + 1) * C::BW + (bi + 1)];
                if (b > 0) {
                    if (lt(v, prev)) nondec = false;
                    if (lt(prev, v)) noninc = false;
                }
                prev = v;
            }
            // neighbour W: i down; E: i up; S: j down; N: j up
            const int up = sd == 0 ? 3 : sd == 1 ? 0 : sd == 2 ? 1 : 0;
            const int down = sd == 0 ? 2 : sd == 1 ? 1 : sd == 2 ? 2 : 3;
            const int bits = noninc ? 1 << down : nondec ? 1 << up : (1 << up) | (1 << down);
            w.mono_n += 1;
            w.mono_ok += (noninc || nondec) ? 1 : 0;
            const int nc = sd == 0 ? c - 1 : sd == 1 ? c + 1 : sd == 2 ? c - cxn : c + cxn;
            atomicOr(&d.dflags[nc], bits);
            fence_acq_rel_gpu();
        }
        if (rl == 0 && has_nb) {
            const int nc = sd == 0 ? c - 1 : sd == 1 ? c + 1 : sd == 2 ? c - cxn : c + cxn;
            double vt = inf_of<double>();
            if (CVAL && bmax >= 0) {
                // eq. cell_value: V_i + ((h + h^c)/2) / F(y_i) with
                // (h + h^c)/2 = (k+1) h/2; h/F(y_i) read at the node across
                // the boundary from x_i (the box in shared memory carries a
                // one-node halo of f)
                int ai, aj;
                if (sd == 0) { ai = -1; aj = bmax; }
                else if (sd == 1) { ai = K; aj = bmax; }
                else if (sd == 2) { ai = bmax; aj = -1; }
                else { ai = bmax; aj = K; }
                double fy = to_d(tF[(aj + 1) * C::BW + (ai + 1)]);
                if (!(fy >= 0.0 && fy < inf_of<double>())) fy = val_of(ld_cg(&ictl->fmin_f));
                vt = to_d(vmax) + (double)(K + 1) * 0.5 * fy;
            }
            // HCM: update the neighbour's cell value whether or not it is
            // activated
            unsigned long long old = KEY_UNSET, kk = KEY_UNSET;
            if (CVAL && vt < inf_of<double>()) {
                kk = key_of(vt);
                old = atomicMin(&d.cval[nc], kk);
            }
            act(d, nc, kk, old, activate);
        }
    }
    __syncwarp();
    PROF_MARK(6);
    return true;
}

// ---------------------------------------------------------------- rounds
// The bucketed schedule: every round releases the near lists of all
// instances, the warps process them, re-activations go to the next near list
// (key <= theta) or to the far list, and a grid barrier ends the round; when
// an instance's near list runs dry its next bucket is split off the far list.
template <int MODE, int K, int VAR>
__global__ void __launch_bounds__(TileCfg<MODE, K>::WPB * 32, 2)
    k_solve(const __grid_constant__ SolveParams p) {
    using C = TileCfg<MODE, K>;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr bool FAST = VAR == VAR_FHCM;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_flag;
    // TMA destinations must be 128-byte aligned: the host asks for 128 spare bytes
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);

    const int NI = p.n_inst;
    InstState S;
    {
        unsigned char* sp = smem + C::WPB * C::WARP_BYTES + C::lk_area(VAR);
        S.theta = reinterpret_cast<unsigned long long*>(sp);
        sp += NI * 8;
        S.pre = reinterpret_cast<int*>(sp);
        sp += (NI + 1) * 4;
        S.nn = reinterpret_cast<int*>(sp);
        sp += NI * 4;
        S.nf = reinterpret_cast<int*>(sp);
        sp += NI * 4;
        S.scan_scratch = reinterpret_cast<int*>(sp);
        sp += 33 * 4;
        S.ns = sp;
        sp += NI;
        S.fs = sp;
    }

    WarpState<MODE, K> w;
    w.init(smem, p.max_passes);
    const int lane = w.lane, g = w.g, dl = w.dl;
    const int warp = threadIdx.x >> 5;
    const int prof_on = p.profile;

    Ctl* gctl = p.gctl;
    const InstDesc* inst = p.inst;
    const unsigned long long deadline = gtimer() + (unsigned long long)p.deadline_ns;
    if (threadIdx.x == 0) atomicMin(&gctl->t_start, gtimer());

    for (int i = threadIdx.x; i < NI; i += blockDim.x) {
        S.theta[i] = 0;
        S.ns[i] = 0;
        S.fs[i] = 0;
    }
    __syncthreads();

    const int nb = gridDim.x;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gthreads = gridDim.x * blockDim.x;
    // static assignment of list entries: consecutive entries go to different
    // blocks (SMs) first, then to different warps, then to a warp's cells
    const int slot = g * C::WPB + warp;
    constexpr int SLOTS = C::WPB * C::CPW;

    unsigned long long st_rounds = 0;
    unsigned long long pacc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long pt = clock64();

    for (;;) {
        // ---- every instance's list lengths (the same in every block)
        int my_split = 0, my_work = 0;
        for (int i = threadIdx.x; i < NI; i += blockDim.x) {
            const Ctl* c = inst[i].ctl;
            const int J = inst[i].J;
            const int a = min(ld_cg(&c->cnt[S.ns[i]]), J), b = min(ld_cg(&c->fcnt[S.fs[i]]), J);
            S.nn[i] = a;
            S.nf[i] = b;
            my_split |= (a == 0 && b > 0);
            my_work |= (a > 0 || b > 0);
        }
        const int any_split = __syncthreads_or(my_split);
        const int any_work = __syncthreads_or(my_work);
        if (!any_work) break;  // every list of every instance empty: converged

        if (any_split) {
            // ---- release the next bucket of every instance whose near list
            // is empty: min key over its far list ...
            // far-list lengths of the splitting instances (0 for the others),
            // prefix-summed into pre: the concatenated index space of this phase
            for (int i = threadIdx.x; i < NI; i += blockDim.x)
                if (S.nn[i] != 0) S.nf[i] = 0;
            __syncthreads();
            const int total = block_exclusive_scan(S.nf, S.pre, NI, S.scan_scratch);
            for (int e = gtid; e < total; e += gthreads) {
                const int i = find_inst(S.pre, NI, e);
                const InstDesc& d = inst[i];
                const int* far = d.lists + (3 + S.fs[i]) * d.J;
                const unsigned long long kk = ld_cg(&d.cval[ld_cg(&far[e - S.pre[i]])]);
                if (kk != KEY_UNSET) atomicMin(&d.ctl->fmin[S.fs[i]], kk);
            }
            PROF_MARK(0);
            if (!grid_sync(gctl, deadline, &s_flag)) break;
            PROF_MARK(1);
            for (int i = threadIdx.x; i < NI; i += blockDim.x) {
                if (S.nn[i] == 0 && S.pre[i + 1] > S.pre[i]) {
                    const InstDesc& d = inst[i];
                    double delta = d.delta;
                    if (!(delta > 0.0)) {
                        // relative width: |delta| (default 4) cells' worth of the fastest crossing
                        const double m = delta < 0.0 ? -delta : 4.0;
                        delta = m * (double)K * val_of(ld_cg(&d.ctl->fmin_f));
                    }
                    if (!(delta > 0.0) || !(delta < inf_of<double>())) delta = inf_of<double>();
                    const unsigned long long fm = ld_cg(&d.ctl->fmin[S.fs[i]]);
                    S.theta[i] = fm == KEY_UNSET ? KEY_UNSET : key_of(val_of(fm) + delta);
                }
            }
            __syncthreads();
            // ... then move every far cell with key <= theta to the near list
            for (int e0 = gtid - lane; e0 < total; e0 += gthreads) {
                const int e = e0 + lane;
                if (e < total) {
                    const int i = find_inst(S.pre, NI, e);
                    const InstDesc& d = inst[i];
                    const int c = ld_cg(&d.lists[(3 + S.fs[i]) * d.J + (e - S.pre[i])]);
                    if (ld_cg(&d.cval[c]) <= S.theta[i])
                        lane_push(d.lists + S.ns[i] * d.J, &d.ctl->cnt[S.ns[i]], c, d.J, gctl);
                    else
                        lane_push(d.lists + (3 + (S.fs[i] ^ 1)) * d.J, &d.ctl->fcnt[S.fs[i] ^ 1], c, d.J, gctl);
                }
            }
            PROF_MARK(0);
            if (!grid_sync(gctl, deadline, &s_flag)) break;
            PROF_MARK(1);
            for (int i = threadIdx.x; i < NI; i += blockDim.x) {
                if (S.nn[i] == 0 && S.pre[i + 1] > S.pre[i]) {
                    const InstDesc& d = inst[i];
                    if (blockIdx.x == 0) {
                        d.ctl->fcnt[S.fs[i]] = 0;
                        d.ctl->fmin[S.fs[i]] = KEY_UNSET;
                        d.ctl->advances += 1;
                    }
                    S.fs[i] ^= 1;
                    S.nn[i] = min(ld_cg(&d.ctl->cnt[S.ns[i]]), d.J);
                }
            }
            __syncthreads();
        }

        // ---- one round: process the near lists of all instances
        const int total = block_exclusive_scan(S.nn, S.pre, NI, S.scan_scratch);
        // deadline, grid-uniformly: raised here, seen by all at this round's barrier
        if (gtid == 0 && gtimer() > deadline) fail(gctl, EIK_ETIMEDOUT, 0x5000000ull);
        if (blockIdx.x == 0)
            for (int i = threadIdx.x; i < NI; i += blockDim.x) {
                const int nsl = S.ns[i];
                inst[i].ctl->cnt[nsl == 0 ? 2 : nsl - 1] = 0;  // the list consumed last round
            }

        for (int t = 0;; ++t) {
            const int first_idx = blockIdx.x + nb * (warp + SLOTS * t);  // cell slot 0's entry
            if (first_idx >= total) break;
            const int idx = blockIdx.x + nb * (slot + SLOTS * t);
            int c = -1, ii_ = 0;
            if (idx < total) {
                ii_ = find_inst(S.pre, NI, idx);
                const InstDesc& d0 = inst[ii_];
                c = ld_cg(&d0.lists[S.ns[ii_] * d0.J + (idx - S.pre[ii_])]);
            }
            const InstDesc& d = inst[ii_];
            int cg[C::CPW], ig[C::CPW];
#pragma unroll
            for (int gg = 0; gg < C::CPW; ++gg) {
                cg[gg] = __shfl_sync(FULL, c, gg * C::LPC);
                ig[gg] = __shfl_sync(FULL, ii_, gg * C::LPC);
            }

            // ---- remove the cell from the list: clear its flag BEFORE reading
            // its halo, so that a neighbour that improves the halo while we
            // work re-queues it (Alg. generic_LC_cells, activation test)
            int first = 0;
            if (dl == 0 && c >= 0) {
                atomicExch(&d.qflag[c], 0);
                first = atomicAdd(&d.visits[c], 1) == 0;
            }
            first = __shfl_sync(FULL, first, g * C::LPC);
            fence_acq_rel_gpu();
            fence_proxy_async_global();
            fence_proxy_async_shared();
            jitter(p.jitter_ns, (unsigned)c);
            __syncwarp();
            PROF_MARK(2);
            pacc[7] += 1;

            const bool ok = visit_cells<MODE, K, true, VAR>(
                w, inst, gctl, deadline, c, ii_, first, cg, ig, prof_on, pacc, pt,
                [&](const InstDesc& dn, int nc, unsigned long long kk, unsigned long long old, bool activate) {
                    const int was = activate ? atomicExch(&dn.qflag[nc], 1) : 1;
                    if (!was) {
                        unsigned long long cur = old < kk ? old : kk;
                        if (kk == KEY_UNSET) cur = ld_cg(&dn.cval[nc]);
                        const int nsl = S.ns[ii_];
                        const int J = dn.J;
                        if (cur <= S.theta[ii_])
                            lane_push(dn.lists + (nsl == 2 ? 0 : nsl + 1) * J,
                                      &dn.ctl->cnt[nsl == 2 ? 0 : nsl + 1], nc, J, gctl);
                        else
                            lane_push(dn.lists + (3 + S.fs[ii_]) * J, &dn.ctl->fcnt[S.fs[ii_]], nc, J, gctl);
                    }
                });
            if (!ok) break;  // the round's barrier reports the abort to every block
        }
        // a warp that gave up (abort raised) still reaches the barrier, which
        // then reports the abort to every block
        ++st_rounds;
        PROF_MARK(2);
        if (!grid_sync(gctl, deadline, &s_flag)) break;
        PROF_MARK(1);
        for (int i = threadIdx.x; i < NI; i += blockDim.x) S.ns[i] = S.ns[i] == 2 ? 0 : S.ns[i] + 1;
        __syncthreads();
    }

    flush_counters(inst, w.acc_inst, w.acc_visits, w.acc_sweeps, w.acc_lane);
    if (w.st_lane) atomicAdd(&gctl->lane_updates, w.st_lane);
    if (FAST && w.mono_n) {
        atomicAdd(&gctl->mono_n, w.mono_n);
        atomicAdd(&gctl->mono_ok, w.mono_ok);
    }
    if (p.profile && lane == 0)
        for (int i = 0; i < 8; ++i) atomicAdd(&gctl->prof[i], pacc[i]);
    if (gtid == 0) gctl->rounds = st_rounds;
    if (lane == 0) atomicMax(&gctl->t_end, gtimer());
}

// ---------------------------------------------------------------- async
// The round-free schedule.  The job's cells share one ring (a bounded
// multi-producer multi-consumer queue of global cell indices: each 64-bit
// word holds a sequence number over the index).  Producers and consumers
// both take tickets with one atomicAdd: a producer waits for the consumer of
// the slot's previous lap, a consumer for the producer of its own ticket, so
// an idle warp holds a ticket and watches only its own slot, and every push
// goes straight to the warp that has waited longest.  Each cell's flag has
// two bits: requested (bit 0) and running (bit 1); bit 2 records that the
// cell was removed before.
//   activate: set bit 0; the caller that set it on an idle cell pushes it.
//   claim:    flag := running (the request is consumed) before the halo load.
//   finish:   clear bit 1; if bit 0 came back meanwhile, push the cell again.
// So a cell sits in the ring at most once and never runs on two warps, and a
// neighbour that changed the halo after the load always makes the cell run
// again.  `pending` counts cells requested or running; a waiting warp that
// sees it at 0 is done (a running cell's activations are counted before its
// own finish, so it cannot reach 0 early).  There are no rounds: a cell runs
// as soon as a warp is free.  The order is the ring's, first in first out --
// label correcting without buckets, exact by Theorem convergence like any
// removal order.  head, tail and pending live on separate 128-byte lines.
__device__ __forceinline__ unsigned long long ld_vol64(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}
__device__ __forceinline__ void st_vol64(unsigned long long* p, unsigned long long v) {
    *(volatile unsigned long long*)p = v;
}
constexpr int Q_HEAD = 0, Q_TAIL = 32, Q_PENDING = 64;  // qctl word offsets (128 B apart)
constexpr int SORT_MIN = 2048;      // initial cells above which the ring is seeded in value order
constexpr int SORT_BUCKETS = 8192;  // counting-sort bins (p.hist holds 3 x SORT_BUCKETS + 1 ints)

__device__ __forceinline__ bool ring_push(const SolveParams& p, Ctl* gctl, unsigned e,
                                          unsigned long long deadline) {
    const unsigned t = atomicAdd(&p.qctl[Q_TAIL], 1u);
    unsigned long long* sl = p.ring + (t & p.ring_mask);
    unsigned spins = 0;
    // the first lap finds every slot free (seeded so); later laps wait for
    // the previous lap's consumer to have read the slot
    while (t > p.ring_mask && (unsigned)(ld_vol64(sl) >> 32) != t) {
        if ((++spins & 255u) == 0 && (gtimer() > deadline || ld_vol(&gctl->abort))) {
            fail(gctl, EIK_ETIMEDOUT, 0x6000000ull);
            return false;
        }
    }
    st_vol64(sl, ((unsigned long long)(t + 1u) << 32) | e);
    return true;
}
// Take the next ticket and wait for its cell: >= 0 the cell, -1 converged
// (nothing requested or running), -2 gave up (abort raised or deadline).
__device__ __forceinline__ int ring_pop(const SolveParams& p, Ctl* gctl, unsigned long long deadline) {
    const unsigned h = atomicAdd(&p.qctl[Q_HEAD], 1u);
    unsigned long long* sl = p.ring + (h & p.ring_mask);
    unsigned long long v;
    unsigned spins = 0, ns = 16;
    while ((unsigned)((v = ld_vol64(sl)) >> 32) != h + 1u) {
        if ((++spins & 31u) == 0) {
            if (ld_vol(reinterpret_cast<const int*>(&p.qctl[Q_PENDING])) == 0) return -1;
            if (ld_vol(&gctl->abort)) return -2;
            if (gtimer() > deadline) {
                fail(gctl, EIK_ETIMEDOUT, 0x7000000ull);
                return -2;
            }
        }
        __nanosleep(ns);
        ns = ns < 256 ? 2 * ns : 256;
    }
    st_vol64(sl, ((unsigned long long)(h + p.ring_mask + 1u) << 32) | 0xffffffffull);
    return (int)(unsigned)v;
}

// ---------------------------------------------------------------- value order
// The value-ordered round-free schedule: Dial's buckets (Sec. 2) without
// rounds.  A requested cell goes into the bucket ring of the value its
// activation proposes (eq. cell_value) -- bucket a = floor(value / delta),
// rings indexed by a mod NBQ, values below the front raised to it and values
// more than NBQ - 1 buckets above it lowered to the last one.  Each ring has
// a count word: the cells requested or running that are filed under its
// bucket, the bucket's lap (a / NBQ) and a closed flag.  The front is the
// lowest bucket still counted; the warp whose finish empties it closes it
// (a compare-and-swap from "this lap, open, 0"), moves the front one up and
// reopens the ring for the bucket NBQ higher -- no barrier.  A request whose
// count lands on a closed ring or another lap takes it back and files the
// cell under the new front, so a counted cell never sits below the front.
// A warp takes the oldest cell of the lowest non-empty bucket within
// bq_window buckets of the front (a compare-and-swap on that ring's head);
// cells above the window wait until the front comes within reach, which
// keeps cells from running long before their upstream neighbours settle --
// the revisits the first-in first-out ring pays for.  A warp that finds
// nothing to take parks on a ticket of the first-in first-out ring (as in
// the round-free schedule above); a cell requested within the window while
// warps are parked is handed to one of them directly, and when the front
// moves, the bucket that enters the window is handed to parked warps in
// batches.  Parked warps look at the buckets only rarely (thousands of them
// polling the same lines would queue every atomic of the working warps):
// then they move the front if its last cell finished unseen and hand on any
// cells left within the window.  Any removal order is exact (Theorem
// convergence), so the order only changes the work; `pending` (cells
// requested or running) still ends the pass.
//
// A ring entry carries the cell and the ring it is counted under: cell |
// ring << 26, below 2^31 (the job's cells < 2^26, which the host checks), so
// it reads as a non-negative int and never as the ring markers 0xffffffff.
constexpr int BQ_CW = 64, BQ_FRONT = 128;  // header word offsets (count words are 64-bit)
constexpr int CELL_BITS = 26;
constexpr unsigned CELL_MASK = (1u << CELL_BITS) - 1u;
constexpr unsigned long long CW_CLOSED = 1ull << 32, CW_LAP = 1ull << 33;
__device__ __forceinline__ unsigned long long slot_free(unsigned t) {
    return ((unsigned long long)t << 32) | 0xffffffffull;
}
__device__ __forceinline__ unsigned long long slot_full(unsigned t, unsigned v) {
    return ((unsigned long long)(t + 1u) << 32) | v;
}
__device__ __forceinline__ unsigned long long* bq_cw(const SolveParams& p, unsigned s) {
    return reinterpret_cast<unsigned long long*>(p.bq + BQ_CW) + s;
}
// parked warps: consumer tickets handed out beyond the producers'
__device__ __forceinline__ int ring_waiters(const SolveParams& p) {
    return (int)(ld_vol(&p.qctl[Q_HEAD]) - ld_vol(&p.qctl[Q_TAIL]));
}
#define QEV(i)                                              \
    do {                                                    \
        if (p.profile) atomicAdd(&gctl->qev[i], 1ull);      \
    } while (0)
// Put entry v into the first-in first-out ring's slot of ticket t (waiting
// for the previous lap's consumer to release it).
__device__ __forceinline__ bool ring_fill(const SolveParams& p, Ctl* gctl, unsigned t, unsigned v,
                                          unsigned long long deadline) {
    unsigned long long* sl = p.ring + (t & p.ring_mask);
    unsigned spins = 0;
    while (t > p.ring_mask && (unsigned)(ld_vol64(sl) >> 32) != t) {
        if ((++spins & 255u) == 0 && (gtimer() > deadline || ld_vol(&gctl->abort))) {
            fail(gctl, EIK_ETIMEDOUT, 0x6100000ull);
            return false;
        }
    }
    st_vol64(sl, slot_full(t, v));
    return true;
}
__device__ __forceinline__ bool give(const SolveParams& p, Ctl* gctl, unsigned v, unsigned long long deadline) {
    QEV(3);
    return ring_fill(p, gctl, atomicAdd(&p.qctl[Q_TAIL], 1u), v, deadline);
}
// File entry v in bucket ring s.
__device__ __forceinline__ bool bq_put(const SolveParams& p, Ctl* gctl, unsigned s, unsigned v,
                                       unsigned long long deadline) {
    QEV(5);
    const unsigned t = atomicAdd(&p.bq[2 * s + 1], 1u);
    unsigned long long* sl = p.bq_data + (size_t)s * (p.bq_mask + 1u) + (t & p.bq_mask);
    unsigned spins = 0;
    // later laps wait for the previous lap's consumer to release the slot
    while (t > p.bq_mask && (unsigned)(ld_vol64(sl) >> 32) != t) {
        if ((++spins & 255u) == 0 && (gtimer() > deadline || ld_vol(&gctl->abort))) {
            fail(gctl, EIK_ETIMEDOUT, 0x6200000ull);
            return false;
        }
    }
    st_vol64(sl, slot_full(t, v));
    return true;
}
// The entry of ticket h of bucket ring s (already claimed), given the slot's
// first reading w: wait for its producer, release the slot.  -2: gave up.
__device__ __forceinline__ int bq_take(const SolveParams& p, Ctl* gctl, unsigned s, unsigned h,
                                       unsigned long long w, unsigned long long deadline) {
    unsigned long long* sl = p.bq_data + (size_t)s * (p.bq_mask + 1u) + (h & p.bq_mask);
    unsigned spins = 0;
    while ((unsigned)(w >> 32) != h + 1u) {
        if ((++spins & 255u) == 0 && (gtimer() > deadline || ld_vol(&gctl->abort))) {
            fail(gctl, EIK_ETIMEDOUT, 0x6300000ull);
            return -2;
        }
        w = ld_vol64(sl);
    }
    st_vol64(sl, slot_free(h + p.bq_mask + 1u));
    return (int)(unsigned)w;
}
__device__ __forceinline__ int bq_read(const SolveParams& p, Ctl* gctl, unsigned s, unsigned h,
                                       unsigned long long deadline) {
    return bq_take(p, gctl, s, h, ld_vol64(p.bq_data + (size_t)s * (p.bq_mask + 1u) + (h & p.bq_mask)), deadline);
}
// Request a cell (global index e) whose activation proposes cell-value key
// `key`: count it under its bucket, then hand it to a parked warp (within
// the window) or file it.  f and waiters: the front and the parked warps as
// the caller read them, before its own atomics (their loads then overlap the
// caller's round trips; a stale front only sends the count round once more).
// A cell handed on takes its ticket of the parking ring together with its
// count: a cell within the window stays within it when the front moves up,
// since its bucket rises to the new front at most.
__device__ __forceinline__ bool bq_request(const SolveParams& p, Ctl* gctl, unsigned e, unsigned long long key,
                                           double inv_delta, unsigned long long deadline, unsigned f, int waiters) {
    const double v = key == KEY_UNSET ? inf_of<double>() : val_of(key) * inv_delta;
    const unsigned a0 = v < 1073741824.0 ? (unsigned)v : 1073741824u;
    unsigned a = a0 < f ? f : a0;
    a = a > f + NBQ - 1 ? f + NBQ - 1 : a;
    const bool hand = a <= f + (unsigned)p.bq_window && waiters > 0;
    unsigned t = 0;
    if (hand) {
        QEV(3);
        t = atomicAdd(&p.qctl[Q_TAIL], 1u);
    }
    unsigned s = a & (NBQ - 1);
    unsigned long long old = atomicAdd(bq_cw(p, s), 1ull);
    bool moved = false;
    for (unsigned tries = 1; (old & CW_CLOSED) != 0 || (old >> 33) != (unsigned long long)(a / NBQ); ++tries) {
        // the front moved past this bucket: file the cell under the new front
        atomicAdd(bq_cw(p, s), ~0ull);
        QEV(4);
        if ((tries & 255u) == 0 && (gtimer() > deadline || ld_vol(&gctl->abort))) {
            fail(gctl, EIK_ETIMEDOUT, 0x6500000ull);
            return false;
        }
        moved = true;
        f = ld_vol(&p.bq[BQ_FRONT]);
        a = a0 < f ? f : a0;
        a = a > f + NBQ - 1 ? f + NBQ - 1 : a;
        s = a & (NBQ - 1);
        old = atomicAdd(bq_cw(p, s), 1ull);
    }
    const unsigned ent = e | (s << CELL_BITS);
    if (hand) return ring_fill(p, gctl, t, ent, deadline);
    if (moved && a <= f + (unsigned)p.bq_window && ring_waiters(p) > 0) return give(p, gctl, ent, deadline);
    return bq_put(p, gctl, s, ent, deadline);
}
__device__ __forceinline__ bool bq_request(const SolveParams& p, Ctl* gctl, unsigned e, unsigned long long key,
                                           double inv_delta, unsigned long long deadline) {
    return bq_request(p, gctl, e, key, inv_delta, deadline, ld_vol(&p.bq[BQ_FRONT]), ring_waiters(p));
}
// Warp-wide scan of the bucket rings in one round trip (lane L reads ring
// L's head and tail, lane 0 the front too): the mask of rings, rotated so
// that bit i is bucket front + i, that hold cells within the window.
struct BqScan {
    unsigned f, rm, hd, n;
};
__device__ __forceinline__ BqScan bq_scan(const SolveParams& p, int lane) {
    const unsigned f0 = lane == 0 ? ld_vol(&p.bq[BQ_FRONT]) : 0u;
    const unsigned long long ht = ld_vol64(reinterpret_cast<const unsigned long long*>(p.bq) + lane);
    BqScan r;
    r.f = __shfl_sync(0xffffffffu, f0, 0);
    r.hd = (unsigned)ht;
    const int n = (int)((unsigned)(ht >> 32) - r.hd);
    r.n = n > 0 ? (unsigned)n : 0u;
    const unsigned rel = ((unsigned)lane - r.f) & (NBQ - 1);
    const unsigned m = __ballot_sync(0xffffffffu, rel <= (unsigned)p.bq_window && n > 0);
    r.rm = __funnelshift_r(m, m, r.f & (NBQ - 1));
    return r;
}
// Warp-wide: claim the oldest cell of the lowest non-empty bucket within the
// window.  >= 0 the entry, -3 nothing to claim (or the race for it lost
// three times: the warp then parks rather than join a herd of warps retrying
// on one ring's head), -2 gave up.
__device__ __forceinline__ int bq_claim(const SolveParams& p, Ctl* gctl, unsigned long long deadline, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    for (int tries = 0; tries < 3; ++tries) {
        const BqScan sc = bq_scan(p, lane);
        if (!sc.rm) return -3;
        const int L0 = (int)((sc.f + (unsigned)(__ffs(sc.rm) - 1)) & (NBQ - 1));
        int r = -4;
        if (lane == L0 && atomicCAS(&p.bq[2 * L0], sc.hd, sc.hd + 1u) == sc.hd) {
            QEV(0);
            r = bq_read(p, gctl, (unsigned)L0, sc.hd, deadline);
        }
        r = __shfl_sync(FULL, r, L0);
        if (r != -4) return r;
    }
    return -3;
}
// Warp-wide: hand up to `most` cells of bucket ring s to parked warps (up to
// one per parked warp), HB cells a lane at a time: the ring's head moves
// once per batch, the producers' slots are read together, and one ticket
// draw covers the batch.  Returns the cells handed on.
constexpr int HB = 4;
__device__ __forceinline__ unsigned bq_handoff(const SolveParams& p, Ctl* gctl, unsigned s, unsigned most,
                                               unsigned long long deadline, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    unsigned total = 0;
    for (int round = 0; round < 16 && total < most; ++round) {
        unsigned hd = 0, n = 0;
        if (lane == 0) {
            const unsigned long long ht = ld_vol64(reinterpret_cast<const unsigned long long*>(p.bq) + s);
            hd = (unsigned)ht;
            const int avail = (int)((unsigned)(ht >> 32) - hd), wait = ring_waiters(p);
            int want = avail < wait ? avail : wait;
            want = want < 32 * HB ? want : 32 * HB;
            want = (unsigned)want < most - total ? want : (int)(most - total);
            if (want > 0) n = atomicCAS(&p.bq[2 * s], hd, hd + (unsigned)want) == hd ? (unsigned)want : ~0u;
        }
        n = __shfl_sync(FULL, n, 0);
        if (n == 0u) break;
        if (n == ~0u) continue;  // lost the race for the head: look again
        hd = __shfl_sync(FULL, hd, 0);
        unsigned long long* base = p.bq_data + (size_t)s * (p.bq_mask + 1u);
        unsigned long long w[HB];
        int v[HB];
#pragma unroll
        for (int q = 0; q < HB; ++q) {
            const unsigned j = (unsigned)lane + 32u * q;
            w[q] = j < n ? ld_vol64(base + ((hd + j) & p.bq_mask)) : 0ull;
        }
#pragma unroll
        for (int q = 0; q < HB; ++q) {
            const unsigned j = (unsigned)lane + 32u * q;
            v[q] = j < n ? bq_take(p, gctl, s, hd + j, w[q], deadline) : -1;
        }
        unsigned t0 = lane == 0 ? atomicAdd(&p.qctl[Q_TAIL], n) : 0u;
        t0 = __shfl_sync(FULL, t0, 0);
#pragma unroll
        for (int q = 0; q < HB; ++q) {
            const unsigned j = (unsigned)lane + 32u * q;
            if (j < n && v[q] >= 0) ring_fill(p, gctl, t0 + j, (unsigned)v[q], deadline);
        }
        if (lane == 0) atomicAdd(&gctl->handoffs, (unsigned long long)n);
        total += n;
        __syncwarp();
        if (ld_vol(&gctl->abort)) break;
    }
    return total;
}
// Warp-wide: while cells remain, close the front's bucket if it counts no
// cell, move the front one up, reopen the ring for the bucket NBQ higher,
// and hand the cells of the bucket that enters the window to parked warps.
__device__ __forceinline__ void bq_advance(const SolveParams& p, Ctl* gctl, unsigned long long deadline, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    for (int step = 0; step < NBQ; ++step) {
        int moved = 0;
        unsigned f = 0;
        if (lane == 0) {
            f = ld_vol(&p.bq[BQ_FRONT]);
            const unsigned s0 = f & (NBQ - 1);
            const unsigned long long open0 = (unsigned long long)(f / NBQ) * CW_LAP;
            if (ld_vol(reinterpret_cast<const int*>(&p.qctl[Q_PENDING])) != 0 &&
                atomicCAS(bq_cw(p, s0), open0, open0 | CW_CLOSED) == open0) {
                atomicMax(&p.bq[BQ_FRONT], f + 1u);
                // the ring now serves bucket f + NBQ: next lap, open (counts of
                // requests that took the closed bucket are taken back by them)
                atomicAdd(bq_cw(p, s0), CW_LAP - CW_CLOSED);
                atomicAdd(&gctl->fronts, 1ull);
                moved = 1;
            }
        }
        moved = __shfl_sync(FULL, moved, 0);
        if (!moved) return;
        f = __shfl_sync(FULL, f, 0);
        bq_handoff(p, gctl, (f + 1u + (unsigned)p.bq_window) & (NBQ - 1), ~0u, deadline, lane);
        if (ld_vol(&gctl->abort)) return;
    }
}
// Warp-wide: a cell to run -- claimed from the buckets, or received on a
// parked ticket.  >= 0 the entry, -1 converged, -2 gave up.
__device__ __forceinline__ int bq_next(const SolveParams& p, Ctl* gctl, unsigned long long deadline, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    const int r = bq_claim(p, gctl, deadline, lane);
    if (r != -3) return r;
    unsigned x = 0;
    if (lane == 0) {
        QEV(1);
        x = atomicAdd(&p.qctl[Q_HEAD], 1u);
    }
    x = __shfl_sync(FULL, x, 0);
    unsigned long long* sl = p.ring + (x & p.ring_mask);
    unsigned spins = 0, ns = 16;
    for (;;) {
        int got = -3;
        if (lane == 0) {
            const unsigned long long w = ld_vol64(sl);
            if ((unsigned)(w >> 32) == x + 1u) {
                st_vol64(sl, slot_free(x + p.ring_mask + 1u));
                got = (int)(unsigned)w;
                QEV(2);
            }
        }
        got = __shfl_sync(FULL, got, 0);
        if (got >= 0) return got;
        if ((++spins & 31u) == 0) {
            int st = 0;
            if (lane == 0) {
                if (ld_vol(reinterpret_cast<const int*>(&p.qctl[Q_PENDING])) == 0) st = -1;
                else if (ld_vol(&gctl->abort)) st = -2;
                else if (gtimer() > deadline) {
                    fail(gctl, EIK_ETIMEDOUT, 0x7100000ull);
                    st = -2;
                }
            }
            st = __shfl_sync(FULL, st, 0);
            if (st) return st;
        }
        // Rarely (every 512 waits, ~0.1 ms): a front whose last cell
        // finished unseen, and cells left within the window while the warps
        // waited (filed when none was parked), handed on to parked warps --
        // this one among them, which keeps its ticket.
        if ((spins & 511u) == 0) {
            if (lane == 0) QEV(7);
            bq_advance(p, gctl, deadline, lane);
            const BqScan sc = bq_scan(p, lane);
            unsigned rm = sc.rm;
            while (rm) {
                const int i = __ffs(rm) - 1;
                rm &= rm - 1u;
                const unsigned sr = (sc.f + (unsigned)i) & (NBQ - 1);
                const unsigned n = bq_handoff(p, gctl, sr, ~0u, deadline, lane);
                if (lane == 0 && n) atomicAdd(&gctl->qev[6], (unsigned long long)n);
            }
        }
        __nanosleep(ns);
        ns = ns < 256 ? 2 * ns : 256;
    }
}

// Per-instance completion: the instance's last requested cell has finished,
// so its values are final -- publish them, then flag it in host memory.
__device__ __forceinline__ void instance_done(const InstDesc& d) {
    __threadfence_system();
    *(volatile unsigned*)d.done = 1u;
}

// The double-float kernels at k = 8 and 16 are held to three blocks per SM:
// left alone, the compiler fits them into 64 registers (four blocks) with
// spills, which measured slower (1025^2: 1.86 against 1.73 ms per pass; the
// 512-grid batch 14.1 against 13.9 ms).  0 leaves the others to the compiler.
// ORD: the value-ordered schedule (bucket rings, a front, a window) instead
// of first-in first-out.  Left to itself the compiler squeezes several of
// these kernels into 48-72 registers with spills; they are held to two
// blocks per SM (up to 128 registers).  The first-in first-out double-float
// kernels at k = 8 and 16 keep three (their whole warp budget waits on the
// ring at once), the ordered one at k = 16 takes two and keeps the two
// slots of each anti-diagonal step in registers (at three it spills).
template <int MODE, int K, int VAR, bool ORD>
__global__ void __launch_bounds__(TileCfg<MODE, K>::WPB * 32,
                                  (MODE == MODE_DF && (K == 8 || (K == 16 && !ORD))) ? 3 : 2)
    k_solve_async(const __grid_constant__ SolveParams p) {
    using C = TileCfg<MODE, K>;
    static_assert(C::CPW == 1, "one cell per warp");
    constexpr unsigned FULL = 0xffffffffu;
    constexpr bool FAST = VAR == VAR_FHCM;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_flag;
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);

    const int NI = p.n_inst;
    int* s_cnt = reinterpret_cast<int*>(smem + C::WPB * C::WARP_BYTES + C::lk_area(VAR));
    int* s_pre = s_cnt + NI;
    int* s_scr = s_pre + NI + 1;

    WarpState<MODE, K> w;
    w.init(smem, p.max_passes);
    const int lane = w.lane;
    const int prof_on = p.profile;
    Ctl* gctl = p.gctl;
    const InstDesc* inst = p.inst;
    const unsigned long long deadline = gtimer() + (unsigned long long)p.deadline_ns;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gthreads = gridDim.x * blockDim.x;
    unsigned long long pacc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long pt = clock64();
    if (threadIdx.x == 0) atomicMin(&gctl->t_start, gtimer());

    // ---- seed the ring with every instance's initially queued cells (their
    // flags are already 1: requested).  When many cells start queued (the
    // refinement pass queues them all) they enter the ring in order of cell
    // value, by a counting sort on the value in units of one cell crossing at
    // the highest speed, k min(h/F): cells then mostly run after their
    // upstream neighbours, as the bucketed schedule would order them.
    for (int i = threadIdx.x; i < NI; i += blockDim.x) s_cnt[i] = min(ld_cg(&inst[i].ctl->fcnt[0]), inst[i].J);
    __syncthreads();
    if (p.inst_done && blockIdx.x == 0)  // (before the prologue's grid barriers)
        for (int i = threadIdx.x; i < NI; i += blockDim.x) {
            inst[i].ctl->left = s_cnt[i];
            if (s_cnt[i] == 0) instance_done(inst[i]);  // no source: final as it is
        }
    const int total = block_exclusive_scan(s_cnt, s_pre, NI, s_scr);
    const unsigned Q = p.ring_mask + 1u;
    double inv_delta = 0.0;  // ORD: 1 / bucket width
    if constexpr (ORD) {
        // empty rings (slot j of every ring free for ticket j), the front at
        // bucket 0, and the launch's bucket width: the smallest of its
        // instances' (relative widths in units of k min(h/F), default 4)
        const unsigned BQ = p.bq_mask + 1u;
        for (unsigned e = gtid; e < Q; e += gthreads) p.ring[e] = slot_free(e);
        for (size_t e = gtid; e < (size_t)NBQ * BQ; e += gthreads) p.bq_data[e] = slot_free((unsigned)(e & p.bq_mask));
        for (int e = gtid; e < BQ_WORDS; e += gthreads) p.bq[e] = 0u;
        for (int i = gtid; i < NI; i += gthreads) {
            double delta = inst[i].delta;
            if (!(delta > 0.0)) delta = (delta < 0.0 ? -delta : 4.0) * (double)K * val_of(ld_cg(&inst[i].ctl->fmin_f));
            if (delta > 0.0 && delta < inf_of<double>()) atomicMin(&gctl->qdelta, key_of(delta));
        }
        if (gtid == 0) {
            p.qctl[Q_HEAD] = 0;
            p.qctl[Q_TAIL] = 0;
            p.qctl[Q_PENDING] = (unsigned)total;
        }
        if (!grid_sync(gctl, deadline, &s_flag)) return;
        const unsigned long long dk = ld_cg(&gctl->qdelta);
        inv_delta = dk == KEY_UNSET ? 0.0 : 1.0 / val_of(dk);
        for (int e = gtid; e < total; e += gthreads) {
            const int i = find_inst(s_pre, NI, e);
            const InstDesc& d = inst[i];
            const int c = ld_cg(&d.lists[3 * d.J + (e - s_pre[i])]);
            bq_request(p, gctl, (unsigned)(d.cell_base + c), ld_cg(&d.cval[c]), inv_delta, deadline);
        }
        if (!grid_sync(gctl, deadline, &s_flag)) return;
    }
    const bool sorted = !ORD && total > SORT_MIN;
    auto seed_cell = [&](int e, int& gcell) -> int {  // initial entry e: global cell, bucket
        const int i = find_inst(s_pre, NI, e);
        const InstDesc& d = inst[i];
        const int c = ld_cg(&d.lists[3 * d.J + (e - s_pre[i])]);
        gcell = d.cell_base + c;
        if (!sorted) return 0;
        const double unit = (double)K * val_of(ld_cg(&d.ctl->fmin_f));
        const double v = val_of(ld_cg(&d.cval[c]));
        const double b = unit > 0.0 ? v / unit : 0.0;
        return b >= 0.0 && b < (double)(SORT_BUCKETS - 1) ? (int)b : SORT_BUCKETS - 1;
    };
    if (sorted) {
        // p.hist: counts [0, B), exclusive prefix [B, 2B], cursors [2B + 1, 3B + 1)
        for (int e = gtid; e < 3 * SORT_BUCKETS + 1; e += gthreads) p.hist[e] = 0;
        if (!grid_sync(gctl, deadline, &s_flag)) return;
        for (int e = gtid; e < total; e += gthreads) {
            int gc;
            atomicAdd(&p.hist[seed_cell(e, gc)], 1);
        }
        if (!grid_sync(gctl, deadline, &s_flag)) return;
        if (blockIdx.x == 0) block_exclusive_scan(p.hist, p.hist + SORT_BUCKETS, SORT_BUCKETS, s_scr);
        if (!grid_sync(gctl, deadline, &s_flag)) return;
    }
    if constexpr (!ORD) {
        for (unsigned e = gtid; e < Q; e += gthreads) {
            if ((int)e < total) {
                int gc;
                const int b = seed_cell((int)e, gc);
                const unsigned pos =
                    sorted ? (unsigned)(ld_cg(&p.hist[SORT_BUCKETS + b]) + atomicAdd(&p.hist[2 * SORT_BUCKETS + 1 + b], 1))
                           : e;
                p.ring[pos] = ((unsigned long long)(pos + 1u) << 32) | (unsigned)gc;
            } else {
                p.ring[e] = ((unsigned long long)e << 32) | 0xffffffffull;
            }
        }
        if (gtid == 0) {
            p.qctl[Q_HEAD] = 0;
            p.qctl[Q_TAIL] = (unsigned)total;
            p.qctl[Q_PENDING] = (unsigned)total;
        }
        if (!grid_sync(gctl, deadline, &s_flag)) return;
    }

    // ---- each warp: take a cell, solve it, hand on its activations.  (A
    // warp that kept one of the neighbours it requested and ran it next,
    // skipping the ring, was measured slower: running ahead depth first
    // reaches cells before their other upstream neighbours settle, and the
    // revisits outweigh the saved round trips.  First in, first out keeps the
    // wave together.)
    for (;;) {
        int e = 0;
        unsigned my_ring = 0;  // ORD: the bucket ring this cell is counted under
        if constexpr (ORD) {
            e = bq_next(p, gctl, deadline, lane);
            if (e < 0) break;
            my_ring = (unsigned)e >> CELL_BITS;
            e &= (int)CELL_MASK;
        } else {
            if (lane == 0) e = ring_pop(p, gctl, deadline);
            e = __shfl_sync(FULL, e, 0);
            if (e < 0) break;
        }
        if (!ORD && p.hold_ns) {
            // a cell requested less than hold_ns ago (0: no time recorded)
            // goes back to the ring's tail, still requested, and the warp
            // takes the next one: requests from several upstream neighbours
            // merge into one visit without the warp idling
            int young = 0;
            if (lane == 0) {
                const unsigned long long t = __ldcg(&p.req_time[e]), now = gtimer();
                young = t != 0ull && now < t + p.hold_ns && t + p.hold_ns - now <= p.hold_ns;
                if (young) ring_push(p, gctl, (unsigned)e, deadline);
            }
            if (__shfl_sync(FULL, young, 0)) continue;
        }
        __syncwarp();
        const int ii = find_inst(p.cell_pre, NI, e);
        const InstDesc& d = inst[ii];
        const int c = e - d.cell_base;
        // ---- claim: running, the request consumed, before the halo load;
        // bit 2 marks a cell removed before (its first removal activates
        // across source boundaries)
        int first = 0;
        if (lane == 0) first = (atomicExch(&d.qflag[c], 6) & 4) == 0;
        first = __shfl_sync(FULL, first, 0);
        fence_acq_rel_gpu();
        fence_proxy_async_global();
        fence_proxy_async_shared();
        jitter(p.jitter_ns, (unsigned)e);
        __syncwarp();
        PROF_MARK(2);
        pacc[7] += 1;
        const int cg[1] = {c}, ig[1] = {ii};
        const bool ok = visit_cells<MODE, K, ORD, VAR>(
            w, inst, gctl, deadline, c, ii, first, cg, ig, prof_on, pacc, pt,
            [&](const InstDesc& dn, int nc, unsigned long long kk, unsigned long long old, bool activate) {
                if (!activate) return;
                // ORD: the front and the parked warps, read while the flag's
                // atomic is on its way
                unsigned f_pre = 0u;
                int w_pre = 0;
                if constexpr (ORD) {
                    f_pre = ld_vol(&p.bq[BQ_FRONT]);
                    w_pre = ring_waiters(p);
                }
                const int was = atomicOr(&dn.qflag[nc], 1) & 3;
                if (was == 0) {
                    atomicAdd(&p.qctl[Q_PENDING], 1u);
                    if (p.inst_done) atomicAdd(&dn.ctl->left, 1);
                    if constexpr (ORD) {
                        // filed by the value this side proposes (eq. cell_value):
                        // the cell's own value, lowered by every earlier proposal,
                        // would rank a cell visited before at its old value
                        // (an activation always has a finite side, so a proposal)
                        bq_request(p, gctl, (unsigned)(dn.cell_base + nc), kk, inv_delta, deadline, f_pre, w_pre);
                    } else {
                        if (p.hold_ns) p.req_time[dn.cell_base + nc] = gtimer();
                        ring_push(p, gctl, (unsigned)(dn.cell_base + nc), deadline);
                    }
                } else if (ORD && (was & 2) && kk != KEY_UNSET) {
                    // requested while it runs: its finish files it again, by
                    // the lowest value proposed meanwhile (kept complemented,
                    // 0 = none)
                    atomicMax(&p.req_time[dn.cell_base + nc], ~kk);
                }
            });
        // ---- finish: push again if a neighbour asked meanwhile
        int adv = 0;
        if (p.inst_done && lane == 0)  // the instance's counters in place before it can be flagged done
            flush_counters(inst, w.acc_inst, w.acc_visits, w.acc_sweeps, w.acc_lane);
        if (lane == 0) {
            const int old = atomicAnd(&d.qflag[c], ~2);
            const bool last = !(old & 1) && p.inst_done && atomicSub(&d.ctl->left, 1) == 1;
            if constexpr (ORD) {
                if (old & 1) {
                    // requested again while it ran: filed by the lowest value
                    // proposed meanwhile (its reads all in flight at once)
                    const unsigned f_pre = ld_vol(&p.bq[BQ_FRONT]);
                    const int w_pre = ring_waiters(p);
                    const unsigned long long cv = ld_cg(&d.cval[c]);
                    const unsigned long long rk = atomicExch(&p.req_time[e], 0ull);
                    bq_request(p, gctl, (unsigned)e, rk ? ~rk : cv, inv_delta, deadline, f_pre, w_pre);
                } else {
                    atomicSub(&p.qctl[Q_PENDING], 1u);
                }
                // the last cell of the front's bucket moves the front
                const unsigned long long was = atomicAdd(bq_cw(p, my_ring), ~0ull);
                adv = (was & 0xffffffffull) == 1ull && (ld_vol(&p.bq[BQ_FRONT]) & (NBQ - 1)) == my_ring;
            } else {
                if (old & 1) ring_push(p, gctl, (unsigned)e, deadline);
                else atomicSub(&p.qctl[Q_PENDING], 1u);
            }
            if (last) instance_done(d);
        }
        if constexpr (ORD) {
            if (__shfl_sync(FULL, adv, 0)) bq_advance(p, gctl, deadline, lane);
            PROF_MARK(0);  // finish and front moves (profiles: "split")
        }
        __syncwarp();
        if (!ok) break;
    }

    flush_counters(inst, w.acc_inst, w.acc_visits, w.acc_sweeps, w.acc_lane);
    if (w.st_lane) atomicAdd(&gctl->lane_updates, w.st_lane);
    if (FAST && w.mono_n) {
        atomicAdd(&gctl->mono_n, w.mono_n);
        atomicAdd(&gctl->mono_ok, w.mono_ok);
    }
    if (p.profile && lane == 0)
        for (int i = 0; i < 8; ++i) atomicAdd(&gctl->prof[i], pacc[i]);
    if (lane == 0) atomicMax(&gctl->t_end, gtimer());
}

}  // namespace eik
