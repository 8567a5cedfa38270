// Host planning of the persistent kernel: lane-group widths and warp shares.
// Groups have at least 2 lanes (kMinLog2G): the kernel's per-group staging
// buffers are sized for at most 16 groups per warp.
//
// A pair aligned by a group of G lanes with R rows per lane takes
// ceil(n / (G R)) strips of (m + G - 1) wavefront steps (rounded up to the
// kernel's 4-step blocks); its reverse pass is estimated at a quarter of
// that.  Each strip start also stalls the group's whole warp (its 32 / G
// groups) while the warp builds the strip's query profile, so a strip is
// charged a fixed number of steps times 32 / G besides its columns (the
// charge is set in host_plan.cpp: 18 steps; measured on 100k DNA pairs with
// the host-only plan preview, every value from 4 to 20 made the planner's
// own choice the measured best, bulk groups of 8 lanes with half-width
// tails, against the all-2-lane plan it chose without the charge, and from
// 24 up it sends 20k protein pairs to wider groups, measured slower).
// Narrow groups waste the fewest cells on padding and fill but make
// a pair's serial sweep long, so a batch with a long tail finishes late.
// The planner therefore keeps a narrow width Gn for the bulk and sends each
// pair whose sweep under Gn exceeds a cap (a fraction of the mean load per
// group) to the narrowest wider class that fits.  With half_tails (the
// packed form with 32-bit profile words) each bulk pair whose last strip under Gn would be at most
// half used (n mod Gn R in (0, Gn R / 2]) goes to Gn / 2, which computes
// fewer padded rows for more strips: measured +1.5 % and +2.3 % on 100k and
// 200k DNA pairs (the autotuner then preferring Gn = 8 over 4), but -23 % on
// 20k protein pairs in the int32 form and -2.3 % in the packed form with the
// byte profile (2,006 against 2,054 GCUPS, twice each, the autotuner's
// choice in both), so the plan asks for it with 32-bit profile words only.
// Warps start on classes in
// proportion to class work and then walk the classes cyclically.  Among a
// few (Gn, cap) candidates the planner keeps the one whose simulated
// longest-first schedule (each group taking the next pair when free)
// finishes first.  The bulk widths run up to 32 lanes: a batch too small to
// fill the GPU finishes with its longest pairs' serial sweeps, which wide
// groups shorten (1,000 pairs of 100-150 x 200-300 residues: 32 lanes,
// 0.099 ms against 0.109 at 8; 4,000: 16 lanes, 0.148 against 0.207).
#include <algorithm>
#include <cmath>
#include <queue>
#include <tuple>

#include "sw_internal.h"

namespace swgb {

int64_t sweep_steps(int n, int m, int G, int rows) {
    if (n <= 0 || m <= 0) return 4;
    const int64_t strips = (n + (int64_t)G * rows - 1) / ((int64_t)G * rows);
    const int64_t cols = ((int64_t)m + G - 1 + 3) / 4 * 4;
    return strips * cols;
}

namespace {

// est_cost[lg][i]: estimated time of pair i under lane-group width 2^lg, in
// wavefront steps (forward sweep plus a quarter for the reverse pass).
struct Costs {
    std::vector<double> at[6];
    double operator()(int lg, int32_t id) const { return at[lg][(size_t)id]; }
};

Costs compute_costs(const std::vector<PlanPair> &pairs, int rows, double strip_overhead) {
    Costs c;
    for (int lg = kMinLog2G; lg <= 5; ++lg) {
        const int G = 1 << lg;
        c.at[lg].resize(pairs.size());
        for (size_t i = 0; i < pairs.size(); ++i) {
            const PlanPair &p = pairs[i];
            const int64_t strips =
                (p.n > 0 && p.m > 0) ? (p.n + (int64_t)G * rows - 1) / ((int64_t)G * rows) : 0;
            // a strip start stalls the whole warp (its 32 / G groups) for the
            // profile build: charged to the pair as group steps
            c.at[lg][i] = 1.25 * ((double)sweep_steps(p.n, p.m, G, rows) +
                                  (double)strips * strip_overhead * (double)(32 >> lg));
        }
    }
    return c;
}


// The sampled pairs in descending order of their estimated cost under each
// lane-group width: sorted once per width and shared by every candidate.
struct SampleOrder {
    std::vector<int32_t> at[6];
};
SampleOrder sample_order(const Costs &cost, const std::vector<char> &sampled) {
    SampleOrder o;
    std::vector<int32_t> ids;
    for (size_t i = 0; i < sampled.size(); ++i)
        if (sampled[i]) ids.push_back((int32_t)i);
    for (int lg = kMinLog2G; lg <= 5; ++lg) {
        o.at[lg] = ids;
        std::sort(o.at[lg].begin(), o.at[lg].end(),
                  [&](int32_t a, int32_t b) { return cost(lg, a) > cost(lg, b); });
    }
    return o;
}

// A candidate's schedule before it is simulated: each class's queue of
// sampled pair costs, longest first; the class each simulated warp starts
// on; and a lower bound on the makespan: no group finishes before the
// longest pair it runs, and a pair of cost x in a class of width G keeps
// G / 32 of a warp busy for x, so the W simulated warps need at least
// sum(x G / 32) / W.
struct SimSetup {
    std::vector<std::vector<double>> q;
    std::vector<int> start;
    double lower = 0;
};
SimSetup sim_setup(const Costs &cost, const std::vector<PlannedClass> &cls, int n_warps,
                   const SampleOrder &order, size_t n_pairs, double scale) {
    SimSetup S;
    const int nc = (int)cls.size();
    if (nc == 0) return S;
    std::vector<int8_t> cls_of(n_pairs, -1);
    for (int c = 0; c < nc; ++c)
        for (int32_t id : cls[c].pairs) cls_of[(size_t)id] = (int8_t)c;
    S.q.resize(nc);
    double warp_time = 0, longest = 0;
    for (int c = 0; c < nc; ++c) {
        const int lg = cls[c].log2g;
        for (int32_t id : order.at[lg])
            if (cls_of[(size_t)id] == c) S.q[c].push_back(cost(lg, id));
        double sum = 0;
        for (double v : S.q[c]) sum += v;
        warp_time += sum * (double)(1 << lg) / 32.0;
        if (!S.q[c].empty()) longest = std::max(longest, S.q[c].front());
    }
    const int sw = std::max(1, (int)std::lround(n_warps * scale));
    int tot = 0;
    for (int c = 0; c < nc; ++c) tot += cls[c].warps;
    for (int c = 0; c < nc; ++c) {
        int k = tot > 0 ? (int)std::lround((double)cls[c].warps * sw / tot) : 0;
        if (cls[c].warps > 0 && k == 0) k = 1;
        for (int w = 0; w < k; ++w) S.start.push_back(c);
    }
    if (S.start.empty()) S.start.push_back(0);
    // the average load per warp, less a margin for rounding
    S.lower = std::max(longest, warp_time / (double)S.start.size() * (1.0 - 1e-9));
    return S;
}

// Longest-first schedule of every class on its warps' groups, over a sample
// of the pairs (with the warp count scaled by the same factor); returns the
// time the last warp finishes (in wavefront steps).
double simulate(const SimSetup &S, const std::vector<PlannedClass> &cls) {
    const int nc = (int)cls.size();
    if (nc == 0) return 0;
    const std::vector<std::vector<double>> &q = S.q;
    const std::vector<int> &start = S.start;
    const int sw = (int)start.size();
    // An event is k idle groups of warp w, free from time t, on the warp's
    // v-th class visit: one entry stands for all of a warp's groups that
    // fall idle together, so a warp costs one entry, not one per group.
    // The heap is a vector ordered by std::greater (earliest time first,
    // then warp, visit, groups).
    using Ev = std::tuple<double, int, int, int>;  // time, warp, visit, groups
    std::vector<Ev> heap;
    heap.reserve((size_t)sw + 64);
    const std::greater<Ev> later;
    auto push = [&](double t, int w, int v, int k) {
        heap.emplace_back(t, w, v, k);
        std::push_heap(heap.begin(), heap.end(), later);
    };
    std::vector<int> pos(nc, 0), visit(sw, 0), busy(sw, 0);
    std::vector<double> wend(sw, 0.0);
    size_t left = 0;  // sampled pairs not yet handed out
    for (int c = 0; c < nc; ++c) left += q[c].size();
    for (int w = 0; w < sw; ++w) {
        busy[w] = 32 >> cls[start[w]].log2g;
        heap.emplace_back(0.0, w, 0, busy[w]);
    }
    std::make_heap(heap.begin(), heap.end(), later);
    double makespan = 0;
    while (!heap.empty()) {
        if (left == 0) {
            // every queue is empty: the remaining events only walk idle
            // groups through the classes, and each warp then ends at the
            // latest of its wend and its pending events' times
            for (int w = 0; w < sw; ++w) makespan = std::max(makespan, wend[w]);
            for (const Ev &e : heap)
                if (std::get<2>(e) == visit[std::get<1>(e)]) makespan = std::max(makespan, std::get<0>(e));
            break;
        }
        std::pop_heap(heap.begin(), heap.end(), later);
        auto [t, w, v, k] = heap.back();
        heap.pop_back();
        if (v != visit[w]) continue;
        const int c = (start[w] + v) % nc;
        // the warp's idle groups take pairs one after another: each time the
        // rest of them would be the next event popped (every other pending
        // event is later in the heap order and costs are positive)
        while (k > 0 && pos[c] < (int)q[c].size()) {
            push(t + q[c][pos[c]++], w, v, 1);
            --left;
            --k;
        }
        if (k == 0) continue;
        if (left == 0) {
            push(t, w, v, k);
            continue;
        }
        wend[w] = std::max(wend[w], t);
        busy[w] -= k;
        if (busy[w] == 0) {
            makespan = std::max(makespan, wend[w]);
            if (++visit[w] < nc) {
                const int c2 = (start[w] + visit[w]) % nc;
                busy[w] = 32 >> cls[c2].log2g;
                push(wend[w], w, visit[w], busy[w]);
            }
        }
    }
    return makespan;
}

// Classes of candidate (Gn = 2^gn, cap = frac x mean load per group) with
// warp shares in proportion to class work; pairs within a class unsorted.
std::vector<PlannedClass> build(const std::vector<PlanPair> &pairs, const Costs &cost,
                                int n_warps, int gn, double frac, bool half_tails, int rows) {
    double total = 0;
    for (const auto &p : pairs) total += cost(gn, p.id);
    const double groups = (double)n_warps * (32 >> gn);
    const double cap = frac * total / std::max(1.0, groups);
    std::vector<std::vector<int32_t>> by(6);
    std::vector<double> work(6, 0.0);
    for (const auto &p : pairs) {
        // the narrowest width from gn up whose cost stays under the cap, else
        // the widest (32 lanes)
        int lg = gn;
        while (lg < 5 && cost(lg, p.id) > cap) ++lg;
        // a bulk pair whose last strip would be at most half used takes
        // half-width groups: same strips' worth of rows or fewer, less padding
        if (half_tails && lg == gn && gn > kMinLog2G) {
            const int64_t h = (int64_t)rows << gn;
            if ((p.n + h / 2 - 1) / (h / 2) * (h / 2) < (p.n + h - 1) / h * h) lg = gn - 1;
        }
        by[lg].push_back(p.id);
        work[lg] += cost(lg, p.id) / (32 >> lg);
    }
    std::vector<PlannedClass> cls;
    double work_total = 0;
    for (int lg = 5; lg >= 0; --lg) {
        if (by[lg].empty()) continue;
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

// Longest first within each class (ties by pair id), as the kernel's
// queues hand pairs out in order.
void sort_classes(std::vector<PlannedClass> &cls, const Costs &cost) {
    std::vector<std::pair<double, int32_t>> key;
    for (auto &c : cls) {
        key.clear();
        key.reserve(c.pairs.size());
        for (int32_t id : c.pairs) key.emplace_back(-cost(c.log2g, id), id);
        std::sort(key.begin(), key.end());
        for (size_t k = 0; k < key.size(); ++k) c.pairs[k] = key[k].second;
    }
}

}  // namespace

std::vector<PlannedClass> plan_classes(const std::vector<PlanPair> &pairs, int n_warps,
                                       int narrow_log2g_hint, double cap_fraction_hint,
                                       int sample_cap, bool half_tails, int rows,
                                       double strip_overhead) {
    if (pairs.empty()) return {};
    n_warps = std::max(1, n_warps);
    const Costs cost = compute_costs(pairs, rows, strip_overhead);
    if (narrow_log2g_hint >= 0) {
        auto cls = build(pairs, cost, n_warps, std::max(narrow_log2g_hint, kMinLog2G),
                         cap_fraction_hint, half_tails, rows);
        sort_classes(cls, cost);
        return cls;
    }
    // a deterministic sample for the simulation
    std::vector<char> sampled(pairs.size(), 0);
    const size_t step = std::max<size_t>(1, pairs.size() / (size_t)std::max(64, sample_cap));
    size_t n_sampled = 0;
    for (size_t k = 0; k < pairs.size(); k += step, ++n_sampled) sampled[k] = 1;
    const double scale = (double)n_sampled / (double)pairs.size();
    const SampleOrder order = sample_order(cost, sampled);
    // Candidates in a fixed order; the plan is the one with the smallest
    // simulated makespan, the earliest in that order among equals.  They
    // are simulated in order of their lower bounds, and one whose bound
    // already exceeds the best makespan found (or equals it, coming later
    // in the order) is not simulated: it could not be chosen.
    struct Cand {
        std::vector<PlannedClass> classes;
        SimSetup setup;
        int idx;
    };
    std::vector<Cand> cands;
    for (int gn = kMinLog2G; gn <= 5; ++gn)
        for (double frac : {0.25, 0.5, 1.0}) {
            Cand c;
            c.classes = build(pairs, cost, n_warps, gn, frac, half_tails, rows);
            c.setup = sim_setup(cost, c.classes, n_warps, order, pairs.size(), scale);
            c.idx = (int)cands.size();
            cands.push_back(std::move(c));
        }
    std::vector<int> by_bound(cands.size());
    for (size_t k = 0; k < cands.size(); ++k) by_bound[k] = (int)k;
    std::sort(by_bound.begin(), by_bound.end(), [&](int a, int b) {
        return cands[a].setup.lower < cands[b].setup.lower ||
               (cands[a].setup.lower == cands[b].setup.lower && a < b);
    });
    int best = -1;
    double best_ms = 0;
    for (int k : by_bound) {
        const Cand &c = cands[k];
        if (best >= 0 && (c.setup.lower > best_ms || (c.setup.lower == best_ms && c.idx > best)))
            continue;
        const double ms = simulate(c.setup, c.classes);
        if (best < 0 || ms < best_ms || (ms == best_ms && c.idx < best)) {
            best = c.idx;
            best_ms = ms;
        }
    }
    std::vector<PlannedClass> chosen = std::move(cands[(size_t)best].classes);
    sort_classes(chosen, cost);
    return chosen;
}

}  // namespace swgb
