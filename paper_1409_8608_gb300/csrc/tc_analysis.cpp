// Cache analysis of Section 3 ("Performance Prediction"), host integer
// work: access distances (Section 3.2), setup lists with remote regions and
// their truncation at 5/4 of the cache (Section 3.2), line sharing /
// prefetch (Section 3.3), prefetch failures (Section 3.4), first iterations
// (Section 3.5) and the invocation count of every case (weighted sum).
//
// The analysis runs on a loop nest around one "kernel": at the paper's
// granularity the loops are the algorithm's sliced loops and the kernel is
// one BLAS call; at the device granularity the loops are the device-wide
// phases (contracted loops enclosing a free loop) and the kernel is one
// phase launch, whose operands are the A, B and C slices of that phase.
//
// Readings where the paper is silent: a remote region that would be
// negative is dropped; equal distances keep the order of the plain access
// distances (larger first), then C, A, B; a truncated operand becomes a
// remote region of the size left; misses are counted as the iterations
// 1 .. n-1 of the innermost loop that start a new line.
#include <algorithm>
#include <cstring>
#include <vector>

#include "tc_analysis.h"

namespace tc {

NestView nest_view(const Plan &p, const Algorithm &alg, int granularity) {
    NestView v;
    v.kernel.assign(p.nidx, false);
    if (granularity == 0) {
        for (int pos = 0; pos < alg.nloops; ++pos) v.loops.push_back(alg.loops[pos]);
        for (int r = 0; r < alg.nk; ++r) v.kernel[alg.kidx[r]] = true;
    } else {
        // device phases: contracted loops up to the last one enclosing a
        // free loop; everything else is inside the phase launch
        std::vector<bool> in_loop(p.nidx, false);
        for (int pos = 0; pos <= alg.q && pos < alg.nloops; ++pos) {
            int id = alg.loops[pos];
            if (p.cls[id] == CLS_CONTRACTED) {
                v.loops.push_back(id);
                in_loop[id] = true;
            }
        }
        for (int id = 0; id < p.nidx; ++id) v.kernel[id] = !in_loop[id];
    }
    return v;
}

int64_t region_elems(const Plan &p, const NestView &v, int op, const std::vector<bool> &joined) {
    int64_t n = 1;
    const Layout &L = p.op[op];
    for (int m = 0; m < L.n; ++m) {
        int id = L.idx[m];
        if (v.kernel[id] || joined[id]) n *= p.ext[id];
    }
    return n;
}

// Section 3.2 walk.  start_depth < 0 starts at the kernel; start_depth = d
// starts at loop d (first iteration, Section 3.5) with every kernel region
// already joined along loops d .. n-1.
int64_t access_distance(const Plan &p, const NestView &v, int op, int start_depth, int64_t elem) {
    const int n = (int)v.loops.size();
    std::vector<bool> joined(p.nidx, false);
    bool have_m = false;
    int level;
    if (start_depth < 0) {
        level = n - 1;
    } else {
        for (int d = start_depth; d < n; ++d) joined[v.loops[d]] = true;
        have_m = true;
        level = start_depth - 1;
    }
    for (; level >= 0; --level) {
        const int l = v.loops[level];
        if (!p.op[op].has(l)) break;  // case 1: invariant across this loop
        joined[l] = true;             // case 2: varies; join every operand
        have_m = true;
    }
    if (!have_m) return 0;
    int64_t dist = 0;
    for (int x = 0; x < 3; ++x) dist += region_elems(p, v, x, joined) * elem;
    return dist;
}

namespace {

struct Entry {
    int op;
    int64_t size, dist, tie0, tie1;
};

std::vector<SetupItem> build_setup(std::vector<Entry> e) {
    std::stable_sort(e.begin(), e.end(), [](const Entry &a, const Entry &b) {
        if (a.dist != b.dist) return a.dist > b.dist;
        if (a.tie0 != b.tie0) return a.tie0 < b.tie0;
        return a.tie1 < b.tie1;
    });
    std::vector<SetupItem> rev;
    int64_t tail = 0;
    for (int i = (int)e.size() - 1; i >= 0; --i) {
        int64_t remote = std::max<int64_t>(e[i].dist - tail, 0);
        if (remote > 0) rev.push_back({1, -1, remote});
        rev.push_back({0, e[i].op, e[i].size});
        tail += remote + e[i].size;
    }
    std::reverse(rev.begin(), rev.end());
    return rev;
}

std::vector<SetupItem> truncate(const std::vector<SetupItem> &s, int64_t limit) {
    std::vector<SetupItem> kept;
    int64_t total = 0;
    for (int i = (int)s.size() - 1; i >= 0; --i) {
        if (total + s[i].size <= limit) {
            kept.push_back(s[i]);
            total += s[i].size;
            continue;
        }
        int64_t left = limit - total;
        if (left > 0) kept.push_back({1, -1, left});
        break;
    }
    std::reverse(kept.begin(), kept.end());
    return kept;
}

// C, A, B: the order the paper's worked example lists equal distances in
const int kOrder[3] = {OP_C, OP_A, OP_B};

int order_rank(int op) {
    for (int r = 0; r < 3; ++r)
        if (kOrder[r] == op) return r;
    return 3;
}

}  // namespace

// Section 3.3: 0 = not prefetched, 1 = the innermost loop indexes the
// operand's first dimension (line sharing, fails once per line), 2 = its
// second dimension while the first is covered by the slice or fits a line.
int prefetch_kind(const Plan &p, const NestView &v, int op, int64_t line_elems) {
    if (v.loops.empty()) return 0;
    const int l = v.loops.back();
    const Layout &L = p.op[op];
    if (!L.has(l) || L.n == 0) return 0;
    if (L.idx[0] == l) return 1;
    if (L.n > 1 && L.idx[1] == l) {
        const int d0 = L.idx[0];
        if (v.kernel[d0] || p.ext[d0] <= line_elems) return 2;
    }
    return 0;
}

int64_t prefetch_elems(const Plan &p, const NestView &v, int op, int64_t line_elems) {
    const Layout &L = p.op[op];
    int64_t n = 1;
    for (int m = 0; m < L.n; ++m) {
        int id = L.idx[m];
        if (!v.kernel[id]) continue;
        n *= m == 0 ? std::min<int64_t>(p.ext[id], line_elems) : p.ext[id];
    }
    return n;
}

std::vector<Case> analyse(const Plan &p, const Algorithm &alg, int granularity, int64_t elem,
                          int64_t cache_bytes, int64_t line_bytes) {
    NestView v = nest_view(p, alg, granularity);
    const int n = (int)v.loops.size();
    const int64_t limit = cache_bytes * 5 / 4;
    const int64_t line_elems = std::max<int64_t>(1, line_bytes / std::max<int64_t>(1, elem));
    std::vector<Case> cases;

    int64_t plain[3], size[3];
    int kinds[3];
    bool any_first_dim = false;
    for (int o = 0; o < 3; ++o) {
        plain[o] = access_distance(p, v, o, -1, elem);
        std::vector<bool> none(p.nidx, false);
        size[o] = region_elems(p, v, o, none) * elem;
        kinds[o] = granularity == 0 ? prefetch_kind(p, v, o, line_elems) : 0;
        any_first_dim |= kinds[o] == 1;
    }
    auto entries = [&](bool with_prefetch) {
        std::vector<Entry> e;
        for (int r = 0; r < 3; ++r) {
            const int o = kOrder[r];
            if (with_prefetch && kinds[o] != 0)
                e.push_back({o, prefetch_elems(p, v, o, line_elems) * elem, 0, -plain[o], r});
            else
                e.push_back({o, size[o], plain[o], -plain[o], r});
        }
        return e;
    };

    // invocation counts: entered[d] = product of the extents of loops 0..d-1
    std::vector<int64_t> entered(n + 1, 1);
    for (int d = 0; d < n; ++d) entered[d + 1] = entered[d] * p.ext[v.loops[d]];
    const int64_t total = entered[n];

    Case hit;
    hit.kind = CASE_STEADY;
    hit.depth = -1;
    hit.setup = truncate(build_setup(entries(true)), limit);
    hit.omit = std::all_of(hit.setup.begin(), hit.setup.end(), [](const SetupItem &s) { return s.kind == 0; });
    if (n == 0) {
        hit.count = 1;
        cases.push_back(hit);
        return cases;
    }
    int64_t misses = 0;
    if (any_first_dim) misses = entered[n - 1] * ((p.ext[v.loops[n - 1]] - 1) / line_elems);
    hit.count = total - entered[n - 1] - misses;
    cases.push_back(hit);
    if (any_first_dim) {
        Case miss;
        miss.kind = CASE_MISS;
        miss.depth = -1;
        miss.count = misses;
        miss.setup = truncate(build_setup(entries(false)), limit);
        miss.omit = false;
        cases.push_back(miss);
    }
    // Section 3.5: the innermost loop, and every loop entered more than 1 %
    // as often as the kernel runs (loops entered once per contraction run
    // are the outermost ones: their first iteration is the run's first)
    int64_t prev = 0;
    for (int d = 0; d < n; ++d) {
        if (!(d == n - 1 || entered[d] * 100 > total)) continue;
        Case f;
        f.kind = CASE_FIRST;
        f.depth = d;
        f.count = entered[d] - prev;
        prev = entered[d];
        std::vector<Entry> e;
        for (int r = 0; r < 3; ++r) {
            const int o = kOrder[r];
            int64_t dist = access_distance(p, v, o, d, elem);
            e.push_back({o, size[o], dist, -dist, r});
        }
        f.setup = truncate(build_setup(e), limit);
        f.omit = false;
        cases.push_back(f);
    }
    return cases;
}

}  // namespace tc
