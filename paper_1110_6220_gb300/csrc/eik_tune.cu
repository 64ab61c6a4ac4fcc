// eik_tune.cu -- the cell size k, the schedule and bucket width of each pass
// (and the value order's window), per class of job, and the autotuner that
// fills that table by timing trial solves (eik_tune / eik_tune_save /
// eik_tune_load / eik_tune_reset).
//
// The paper leaves k to the user (Sec. 4's HCM/FHCM tables sweep it) and the
// bucket width of Dial's method (Sec. 2) is a free parameter of the bucketed
// release.  On the GPU both trade rounds (each ends in a grid barrier, so a
// round costs a few microseconds however little it does) against repeated
// cell visits.  The two passes of FP32_REFINE want different widths: the FP32
// pass is round-bound and gains from wide buckets, the double-float
// refinement pass repeats expensive visits when too many cells are released
// at once.  A class of jobs is (precision, single or batch, the job's mean
// side length rounded to a power of two).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "eik_common.cuh"
#include "eik_plan.h"

namespace eik {
namespace {

struct Key {
    int prec, batch, side;
    bool operator<(const Key& o) const {
        return std::tie(prec, batch, side) < std::tie(o.prec, o.batch, o.side);
    }
};

struct Entry {
    int k;
    double m_first, m_main;  // relative widths: bucket = m * k * min(h/F)
    double ms;               // device time measured when tuned (0: built in)
    bool async_first = false, async_main = false;  // round-free schedule per pass
    bool one_pass = false;  // FP32_REFINE as one double-float pass
    unsigned hold_ns = 0;   // round-free: minimum request age before a cell runs
    bool ordered = false;   // round-free main pass in value order (bucket rings)
    int window = 31;        // ... taking cells from this many buckets above the front
};

std::mutex g_mu;
std::map<Key, Entry> g_table;
bool g_env_loaded = false;

int side_class(const eik_plan_desc* d, int n) {
    double pts = 0.0;
    for (int i = 0; i < n; ++i) pts += (double)d[i].nx * d[i].ny;
    pts /= std::max(n, 1);
    return (int)std::lround(0.5 * std::log2(std::max(pts, 1.0)));
}

// Built-in choices, from sweeps on GB300 over k in {8, 16, 32}, relative
// widths 2..256 and the three schedules (single 1025^2 sin-product grids in
// both precisions, 4097^2 checkerboard + maze, 8193^2 and larger sin20
// grids, 512 uneven grids).  The measurements that set each one stand beside
// it in builtin() below; the history, in brief:
//  - FP32 + refinement runs as one double-float pass from the sources: 2.10
//    ms on the 1025^2 grid against 4.89 ms for an FP32 pass plus a
//    refinement pass, 8.2 against 21.6 ms on a 2049^2 checkerboard + maze,
//    28.7 against 56.6 ms on the batch.  A double-float visit costs about a
//    quarter of an FP64 one (the FP64 pipe is slow), and a pass from the
//    sources visits each cell a few times where a refinement pass seeded
//    everywhere revisits it on every upstream change.
//  - Bucketed rounds pay a grid barrier per round (~19 us however few cells
//    it holds); the first-in first-out ring pays revisits that grow with the
//    grid side (21 visits per cell at 1025^2, 38 at 8193^2, 159 at 32769^2
//    on sin20).  The value-ordered schedule keeps the buckets and drops the
//    rounds, and wins for single grids from ~512^2 in FP64 and ~4096^2 in
//    FP32_REFINE; below that (and on every batch, where its queue costs more
//    than the visits it saves) first in, first out stays.
//  - A hold on the first-in first-out ring (a cell requested less than the
//    hold ago goes back to the ring, so the requests of several upstream
//    neighbours merge into one visit) pays at ~2048^2 only.
//  - The tuner (eik_tune) on each class moved some choices: FP64 batches run
//    round-free (46.2 ms instead of 75.8 ms on the 512-grid mix in rounds),
//    small FP64 grids too (129^2: 0.32 ms instead of 0.37 ms), ~2048^2
//    grids hold for 4 us (2049^2 maze: 6.3 ms for 6.8 ms).
Entry builtin(int prec, bool batch, int side, bool fhcm) {
    // the value-ordered round-free schedule (bucket rings of the proposed
    // cell value, a front without barriers, a window of `w` buckets above it)
    auto ordered = [](Entry e, double m, int w) {
        e.async_first = e.async_main = true;
        e.ordered = true;
        e.m_first = e.m_main = m;
        e.window = w;
        e.hold_ns = 0;
        return e;
    };
    if (prec == EIK_FP32_REFINE) {
        // cells of 16 from ~4096^2 (4097^2 sin20: 18.3 vs 29.1 ms at k = 8;
        // checkerboard+maze 23.6 vs 25.3 ms); at ~2048^2 k = 8 and 16 split
        Entry e{batch || side >= 12 ? 16 : 8, 256.0, 16.0, 0.0, false, true};
        e.one_pass = true;
        // holds (a young cell goes back to the ring): 2049^2 4 us
        if (!batch) e.hold_ns = side == 11 ? 4000 : 0;
        // single grids from ~4096^2 run in value order: buckets of 4 cell
        // crossings, cells taken from the front's bucket and the w above it.
        // 4097^2 checkerboard + maze 12.96 ms at w = 3 against 18.5 ms first
        // in, first out (visits per cell 5.9 against 17.6), sin20 9.5-10.9 ms
        // against 13.1-13.4; 8193^2 (w = 2) sin20 33.4 / maze 31.0 ms
        // against 46 / 62 ms in rounds, 16385^2 116 / 100 against 120 / 192
        if (!batch && side == 12) e = ordered(e, 4.0, 3);
        if (!batch && side >= 13) e = ordered(e, 4.0, 2);
        return e;
    }
    // FP64 batches: first in, first out at k = 16 (the 512-grid mix 36.8 ms
    // against 50.2 ms at k = 8; the 128-request serving mix, sides up to
    // 2003, 60.0 against 74.1 ms; value order at k = 16 72-86 ms: its one
    // bucket width, the finest instance's, is too narrow for the others)
    if (batch && !fhcm) return Entry{16, 4.0, 4.0, 0.0, false, true};
    if (batch || side <= 8) return Entry{8, 4.0, 4.0, 0.0, false, true};
    // FHCM's one-sweep visits gain less from merged requests: rounds
    // (1025^2 sin20 2.72 ms, against 2.92 ms round-free with a 4 us hold);
    // it has no value-ordered form
    if (fhcm) return Entry{8, 256.0, 256.0, 0.0};
    // one FP64 grid from ~512^2: value order, buckets of 4 crossings (FP64
    // visits are the costly ones, so fewer of them pay most): 513^2 sin20 /
    // maze 1.45 / 3.58 ms (w = 3) against 1.85 / 4.59 in rounds; 1025^2
    // sin20 2.87 ms (w = 2) against 3.20 first in, first out with a 4 us
    // hold; 2049^2 8.2 / 9.5 against 8.9 / 13.4; 4097^2 maze 24.0 against
    // 41.1; 8193^2 at k = 16 46.6 / 55.5 against 55.1 / 158 in rounds
    Entry e{side >= 13 ? 16 : 8, 4.0, 4.0, 0.0};
    return ordered(e, 4.0, side <= 9 ? 3 : 2);
}

int load_file(const char* path) {
    FILE* f = std::fopen(path, "r");
    if (!f) return EIK_EINVAL;
    char line[256];
    int rc = EIK_OK;
    // version 5 adds the value-ordered schedule and its window to each line;
    // version 4 lines (no such fields) read as first in, first out
    int version = 0;
    if (std::fgets(line, sizeof line, f) && std::strncmp(line, "eik-tune 5", 10) == 0) version = 5;
    else if (std::strncmp(line, "eik-tune 4", 10) == 0) version = 4;
    if (!version) {
        rc = EIK_EINVAL;
    } else {
        std::map<Key, Entry> t;
        while (std::fgets(line, sizeof line, f)) {
            Key key;
            Entry e;
            int af = 0, am = 0, op = 0, ord = 0, win = 31;
            unsigned hold = 0;
            const int want = version == 5 ? 13 : 11;
            if (std::sscanf(line, "%d %d %d %d %lf %lf %d %d %d %u %lf %d %d", &key.prec, &key.batch, &key.side,
                            &e.k, &e.m_first, &e.m_main, &af, &am, &op, &hold, &e.ms, &ord, &win) != want ||
                (e.k != 4 && e.k != 8 && e.k != 16 && e.k != 32 && e.k != 64) || !(e.m_first > 0) ||
                !(e.m_main > 0) || (af != 0 && af != 1) || (am != 0 && am != 1) || (op != 0 && op != 1) ||
                (ord != 0 && ord != 1) || win < 0 || win > NBQ - 1) {
                rc = EIK_EINVAL;
                break;
            }
            e.async_first = af;
            e.async_main = am;
            e.one_pass = op;
            e.hold_ns = hold;
            e.ordered = ord;
            e.window = win;
            t[key] = e;
        }
        if (!rc)
            for (auto& kv : t) g_table[kv.first] = kv.second;
    }
    std::fclose(f);
    return rc;
}

void maybe_load_env() {  // g_mu held
    if (g_env_loaded) return;
    g_env_loaded = true;
    const char* p = std::getenv("EIK_TUNE_FILE");
    if (p && p[0]) load_file(p);
}

}  // namespace

JobParams choose_params(const eik_plan_desc* d, int n) {
    const int prec = d[0].precision;
    const bool batch = n > 1;
    const int side = side_class(d, n);
    Entry e = builtin(prec, batch, side, d[0].method == EIK_METHOD_FHCM);
    {
        std::lock_guard<std::mutex> lock(g_mu);
        maybe_load_env();
        auto it = g_table.find(Key{prec, batch ? 1 : 0, side});
        if (it != g_table.end()) e = it->second;
    }
    JobParams P;
    P.k = d[0].cell_k ? d[0].cell_k : e.k;
    if (d[0].method == EIK_METHOD_FMSM && P.k < 8) P.k = 8;  // one cell per warp
    P.w_first = -e.m_first;
    P.w_main = -e.m_main;
    P.async_first = e.async_first;
    P.async_main = e.async_main;
    // EIK_SCHED="<first>,<main>" with r (rounds) or a (async) overrides the
    // schedule of each pass (for measurements)
    const char* sched = std::getenv("EIK_SCHED");
    if (sched && std::strlen(sched) >= 3) {
        P.async_first = sched[0] == 'a';
        P.async_main = sched[2] == 'a';
    }
    P.one_pass = e.one_pass;
    P.hold_ns = e.hold_ns;
    P.ordered = e.ordered;
    P.window = e.window;
    // a schedule named in the descriptor wins for every persistent pass
    if (d[0].schedule == EIK_SCHED_ROUNDS) {
        P.async_first = P.async_main = P.ordered = false;
    } else if (d[0].schedule == EIK_SCHED_FIFO || d[0].schedule == EIK_SCHED_ORDERED) {
        P.async_first = P.async_main = true;
        P.ordered = d[0].schedule == EIK_SCHED_ORDERED;
        P.hold_ns = 0;
    }
    if (d[0].window > 0) P.window = d[0].window - 1;
    const char* hold = std::getenv("EIK_HOLD_NS");  // measurements: overrides the table
    if (hold && hold[0]) P.hold_ns = (unsigned)std::strtoul(hold, nullptr, 10);
    const char* onep = std::getenv("EIK_ONE_PASS");
    if (onep && onep[0]) P.one_pass = onep[0] == '1';
    return P;
}

}  // namespace eik

using namespace eik;

extern "C" int eik_tune(const eik_plan_desc* d, const eik_instance* in, int32_t n_inst, void* cuda_stream,
                        eik_tune_result* out) {
    if (!d || !in || n_inst < 1 || n_inst > MAX_BATCH) return EIK_EINVAL;
    for (int i = 0; i < n_inst; ++i)
        if (!desc_valid(&d[i]) || d[i].precision != d[0].precision || d[i].method == EIK_METHOD_FMSM)
            return EIK_EINVAL;  // the table holds the cell solver's schedules
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return EIK_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool fp32 = d[0].precision == EIK_FP32_REFINE;
    // trials leave k and the widths to the tuner
    std::vector<eik_plan_desc> dd(d, d + n_inst);
    for (auto& x : dd) x.bucket_width = 0.0, x.cell_k = 0;
    const JobParams before = choose_params(dd.data(), n_inst);

    HostJob job;
    cudaEvent_t ev[6] = {};
    int rc = EIK_OK;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) rc = EIK_ECUDA;
    int trials = 0;
    auto trial = [&](const JobParams& P, float* t) -> int {
        for (auto& x : dd) x.cell_k = P.k;
        ++trials;
        return run_job(&job, n_inst, dd.data(), in, P, fp32, d[0].deadline_ns, sms, s, ev, nullptr, t);
    };
    float t_before[3] = {0, 0, 0};
    if (!rc) {
        float warm[3];
        trial(before, warm);  // first launches load the kernels
        rc = trial(before, t_before);
    }
    const double widths[] = {2.0, 4.0, 16.0, 64.0, 256.0};
    struct Best {
        int k = 0;
        double mf = 0, mm = 0, est = 1e300;
        bool af = false, am = false, op = false;
        bool ord = false;
        int win = 31;
    } best;
    if (!rc) {
        for (int k : {8, 16, 32}) {
            float t[3];
            if (trial(JobParams{k, -4.0, -4.0}, t)) continue;  // warm-up of this k
            // bucketed rounds at every width: each pass keeps its best width
            double bf = 1e300, bm = 1e300, mf = 4.0, mm = 4.0;
            bool af = false, am = false;
            std::vector<double> over;
            for (double m : widths) {
                if (trial(JobParams{k, -m, -m}, t)) continue;
                if (fp32 && t[1] < bf) bf = t[1], mf = m;
                if (t[2] < bm) bm = t[2], mm = m;
                over.push_back(t[0] - t[1] - t[2]);
            }
            // the round-free schedule for both passes (k >= 8)
            JobParams A{k, -mf, -mm};
            A.async_first = A.async_main = true;
            if (trial(A, t) == EIK_OK) {
                if (fp32 && t[1] < bf) bf = t[1], af = true;
                if (t[2] < bm) bm = t[2], am = true;
                over.push_back(t[0] - t[1] - t[2]);
            }
            if (over.empty()) continue;
            std::sort(over.begin(), over.end());
            const double ov = over[over.size() / 2];
            const double est = (fp32 ? bf : 0.0) + bm + ov;
            if (!fp32) mf = mm, af = am;
            if (est < best.est) best = Best{k, mf, mm, est, af, am, false};
            // the value-ordered schedule (FP32_REFINE as one double-float
            // pass): buckets of 2, 4 and 8 cell crossings, windows of 2 and 3
            // buckets above the front; whole-job times
            for (double m : {2.0, 4.0, 8.0})
                for (int w : {2, 3}) {
                    JobParams O{k, -m, -m};
                    O.async_first = O.async_main = true;
                    O.ordered = true;
                    O.window = w;
                    O.one_pass = fp32;
                    if (trial(O, t)) continue;
                    if (t[0] < best.est) {
                        best = Best{k, m, m, t[0], true, true, fp32};
                        best.ord = true;
                        best.win = w;
                    }
                }
            if (!fp32) continue;
            // FP32 + refinement as one double-float pass: rounds at every
            // width, then round-free
            for (int m = 0; m <= 5; ++m) {
                JobParams O{k, -mf, m < 5 ? -widths[m] : -mm};
                O.one_pass = true;
                O.async_main = m == 5;
                if (trial(O, t)) continue;
                const double e1 = t[2] + (t[0] - t[2] < ov ? t[0] - t[2] : ov);
                if (e1 < best.est) best = Best{k, mf, -O.w_main, e1, false, O.async_main, true};
            }
        }
    }
    Entry chosen{before.k, -before.w_first, -before.w_main, t_before[0], before.async_first, before.async_main};
    chosen.one_pass = before.one_pass;
    chosen.hold_ns = before.hold_ns;
    chosen.ordered = before.ordered;
    chosen.window = before.window;
    float t_new[3] = {0, 0, 0};
    JobParams B{best.k, -best.mf, -best.mm};
    B.async_first = best.af;
    B.async_main = best.am;
    B.one_pass = best.op;
    B.ordered = best.ord;
    B.window = best.win;
    if (!rc && best.k && trial(B, t_new) == EIK_OK && t_new[0] < t_before[0]) {
        chosen = Entry{best.k, best.mf, best.mm, t_new[0], best.af, best.am};
        chosen.one_pass = best.op;
        chosen.ordered = best.ord;
        chosen.window = best.win;
    }
    // a first-in first-out main pass: also try holding cells after their requests
    if (!rc && chosen.async_main && !chosen.ordered) {
        JobParams H{chosen.k, -chosen.m_first, -chosen.m_main};
        H.async_first = chosen.async_first;
        H.async_main = true;
        H.one_pass = chosen.one_pass;
        for (unsigned hold : {4000u, 8000u, 16000u, 24000u}) {
            H.hold_ns = hold;
            float t[3];
            if (trial(H, t) == EIK_OK && t[0] < chosen.ms) {
                chosen.ms = t[0];
                chosen.hold_ns = hold;
            }
        }
    }
    if (!rc) {
        std::lock_guard<std::mutex> lock(g_mu);
        maybe_load_env();
        g_table[Key{d[0].precision, n_inst > 1 ? 1 : 0, side_class(dd.data(), n_inst)}] = chosen;
    }
    free_job(&job);
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (rc) return rc;
    if (out) {
        out->cell_k = chosen.k;
        out->bucket_first = chosen.m_first;
        out->bucket_main = chosen.m_main;
        out->async_first = chosen.async_first;
        out->async_main = chosen.async_main;
        out->one_pass = chosen.one_pass;
        out->hold_ns = (int32_t)chosen.hold_ns;
        out->ordered = chosen.ordered;
        out->window = chosen.ordered ? chosen.window + 1 : 0;
        out->ms = chosen.ms;
        out->ms_before = t_before[0];
        out->trials = trials;
    }
    return EIK_OK;
}

extern "C" int eik_tune_save(const char* path) {
    if (!path) return EIK_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    FILE* f = std::fopen(path, "w");
    if (!f) return EIK_EINVAL;
    std::fprintf(f, "eik-tune 5\n");
    for (auto& kv : g_table)
        std::fprintf(f, "%d %d %d %d %.17g %.17g %d %d %d %u %.17g %d %d\n", kv.first.prec, kv.first.batch,
                     kv.first.side, kv.second.k, kv.second.m_first, kv.second.m_main, (int)kv.second.async_first,
                     (int)kv.second.async_main, (int)kv.second.one_pass, kv.second.hold_ns, kv.second.ms,
                     (int)kv.second.ordered, kv.second.window);
    return std::fclose(f) == 0 ? EIK_OK : EIK_EINVAL;
}

extern "C" int eik_tune_load(const char* path) {
    if (!path) return EIK_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    g_env_loaded = true;
    return load_file(path);
}

extern "C" void eik_tune_reset(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table.clear();
    g_env_loaded = true;
}
