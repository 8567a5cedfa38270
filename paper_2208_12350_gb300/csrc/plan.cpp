// Host planning of the persistent kernel: lane-group widths and warp shares.
// Groups have at least 2 lanes (kMinLog2G): the kernel's per-group staging
// buffers are sized for at most 16 groups per warp.
//
// A pair aligned by a group of G lanes with R rows per lane takes
// ceil(n / (G R)) strips of (m + G - 1) wavefront steps (rounded up to the
// kernel's 4-step blocks); its reverse pass is estimated at a quarter of
// that.  Narrow groups waste the fewest cells on padding and fill but make
// a pair's serial sweep long, so a batch with a long tail finishes late.
// The planner therefore keeps a narrow width Gn for the bulk and sends each
// pair whose sweep under Gn exceeds a cap (a fraction of the mean load per
// group) to the narrowest wider class that fits.  Warps start on classes in
// proportion to class work and then walk the classes cyclically.  Among a
// few (Gn, cap) candidates the planner keeps the one whose simulated
// longest-first schedule (each group taking the next pair when free)
// finishes first.
#include <algorithm>
#include <cmath>
#include <queue>
#include <tuple>

#include "sw_internal.h"

namespace swgb {

int64_t sweep_steps(int n, int m, int G) {
    if (n <= 0 || m <= 0) return 4;
    const int64_t strips = (n + (int64_t)G * kRows - 1) / ((int64_t)G * kRows);
    const int64_t cols = ((int64_t)m + G - 1 + 3) / 4 * 4;
    return strips * cols;
}

static double est_cost(const PlanPair &p, int G) {
    return 1.25 * (double)sweep_steps(p.n, p.m, G);
}

namespace {

struct Candidate {
    std::vector<PlannedClass> classes;
    double makespan = 0;
};

// Longest-first schedule of every class on its warps' groups; returns the
// time the last warp finishes (in wavefront steps).
double simulate(const std::vector<PlanPair> &pairs, const std::vector<PlannedClass> &cls,
                int n_warps, const std::vector<int> &sample_ids) {
    const int nc = (int)cls.size();
    if (nc == 0) return 0;
    // per class: sampled costs (largest first) and a scaled warp count
    const double scale = pairs.empty() ? 1.0 : (double)sample_ids.size() / (double)pairs.size();
    std::vector<std::vector<double>> q(nc);
    std::vector<int> idx_of(pairs.size(), -1);
    for (size_t k = 0; k < sample_ids.size(); ++k) idx_of[sample_ids[k]] = 1;
    for (int c = 0; c < nc; ++c) {
        const int G = 1 << cls[c].log2g;
        for (int32_t id : cls[c].pairs)
            if (idx_of[id] > 0) q[c].push_back(est_cost(pairs[id], G));
    }
    int sw = std::max(1, (int)std::lround(n_warps * scale));
    std::vector<int> start;
    {
        int tot = 0;
        for (int c = 0; c < nc; ++c) tot += cls[c].warps;
        for (int c = 0; c < nc; ++c) {
            int k = tot > 0 ? (int)std::lround((double)cls[c].warps * sw / tot) : 0;
            if (cls[c].warps > 0 && k == 0) k = 1;
            for (int w = 0; w < k; ++w) start.push_back(c);
        }
        if (start.empty()) start.push_back(0);
    }
    sw = (int)start.size();
    using Ev = std::tuple<double, int, int>;  // time, warp, class visit index
    std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> ev;
    std::vector<int> pos(nc, 0), visit(sw, 0), busy(sw, 0);
    std::vector<double> wend(sw, 0.0);
    for (int w = 0; w < sw; ++w) {
        const int P = 32 >> cls[start[w]].log2g;
        busy[w] = P;
        for (int g = 0; g < P; ++g) ev.emplace(0.0, w, 0);
    }
    double makespan = 0;
    while (!ev.empty()) {
        auto [t, w, v] = ev.top();
        ev.pop();
        if (v != visit[w]) continue;
        const int c = (start[w] + v) % nc;
        if (pos[c] < (int)q[c].size()) {
            ev.emplace(t + q[c][pos[c]++], w, v);
            continue;
        }
        wend[w] = std::max(wend[w], t);
        if (--busy[w] == 0) {
            makespan = std::max(makespan, wend[w]);
            if (++visit[w] < nc) {
                const int c2 = (start[w] + visit[w]) % nc;
                const int P = 32 >> cls[c2].log2g;
                busy[w] = P;
                for (int g = 0; g < P; ++g) ev.emplace(wend[w], w, visit[w]);
            }
        }
    }
    return makespan;
}

std::vector<PlannedClass> build(const std::vector<PlanPair> &pairs, int n_warps, int gn,
                                double frac) {
    const int Gn = 1 << gn;
    double total = 0;
    for (const auto &p : pairs) total += est_cost(p, Gn);
    const double groups = (double)n_warps * (32 >> gn);
    const double cap = frac * total / std::max(1.0, groups);
    std::vector<std::vector<int32_t>> by(6);
    for (const auto &p : pairs) {
        int lg = gn;
        if (est_cost(p, Gn) > cap) {
            for (lg = gn + 1; lg < 5; ++lg)
                if (est_cost(p, 1 << lg) <= cap) break;
        }
        by[lg].push_back(p.id);
    }
    std::vector<PlannedClass> cls;
    double work_total = 0;
    std::vector<double> work(6, 0.0);
    for (int lg = 5; lg >= 0; --lg) {
        if (by[lg].empty()) continue;
        std::sort(by[lg].begin(), by[lg].end(), [&](int32_t a, int32_t b) {
            const double ca = est_cost(pairs[a], 1 << lg), cb = est_cost(pairs[b], 1 << lg);
            if (ca != cb) return ca > cb;
            return a < b;
        });
        for (int32_t id : by[lg]) work[lg] += est_cost(pairs[id], 1 << lg) / (32 >> lg);
        work_total += work[lg];
        cls.push_back({lg, std::move(by[lg]), 0});
    }
    int assigned = 0;
    for (auto &c : cls) {
        c.warps = (int)std::floor(n_warps * work[c.log2g] / std::max(work_total, 1e-9));
        if (c.warps == 0 && n_warps >= (int)cls.size()) c.warps = 1;
        assigned += c.warps;
    }
    // hand out the rounding remainder to the largest class, take back excess
    size_t big = 0;
    for (size_t k = 1; k < cls.size(); ++k)
        if (work[cls[k].log2g] > work[cls[big].log2g]) big = k;
    if (!cls.empty()) cls[big].warps += n_warps - assigned;
    if (!cls.empty() && cls[big].warps < 0) cls[big].warps = 0;
    return cls;
}

}  // namespace

std::vector<PlannedClass> plan_classes(const std::vector<PlanPair> &pairs, int n_warps,
                                       int narrow_log2g_hint, double cap_fraction_hint) {
    if (pairs.empty()) return {};
    n_warps = std::max(1, n_warps);
    if (narrow_log2g_hint >= 0)
        return build(pairs, n_warps, std::max(narrow_log2g_hint, kMinLog2G), cap_fraction_hint);
    // a deterministic sample for the simulation
    std::vector<int> sample;
    const size_t step = std::max<size_t>(1, pairs.size() / 8192);
    for (size_t k = 0; k < pairs.size(); k += step) sample.push_back((int)k);
    Candidate best;
    bool have = false;
    for (int gn = kMinLog2G; gn <= 3; ++gn) {
        for (double frac : {0.25, 0.5, 1.0}) {
            Candidate c;
            c.classes = build(pairs, n_warps, gn, frac);
            c.makespan = simulate(pairs, c.classes, n_warps, sample);
            if (!have || c.makespan < best.makespan) {
                best = std::move(c);
                have = true;
            }
        }
    }
    return best.classes;
}

}  // namespace swgb
