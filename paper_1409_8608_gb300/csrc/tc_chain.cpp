// Contraction chains: D = X Y Z as a tree of two contraction kernels
// (Section 3.2: the access-distance method holds for any combination of
// loops and several kernels in the tree).  A variant contracts one pair of
// operands into an intermediate T and T with the third operand into D, each
// step a plan of this library with its own algorithm; a sliced variant
// wraps both kernels in a loop over one index of D that the pair carries and
// the third operand does not, so that T holds a single slice.  The
// prediction of a variant is the sum of its two steps' micro-benchmark
// predictions (tc_predict), times the slices.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "tc_internal.h"

namespace {

struct Step {
    std::string spec;
    std::vector<int64_t> ext, strides;
    tc_plan plan = nullptr;
};

struct Variant {
    int p = 0, q = 1, r = 2;   // (p, q) first, then r
    char sliced = 0;           // index looped around both steps
    int64_t slices = 1;
    int64_t off_p = 0, off_q = 0, off_d = 0;  // element stride of the sliced index in X_p, X_q, D
    std::string t_modes;       // the intermediate's modes (one slice)
    int64_t t_elems = 1;
    double flops = 0;
    Step s1, s2;
    double predicted = -1;
};

// dense (first index fastest) strides of `modes`, keyed by letter
std::vector<int64_t> dense_strides(const std::string &modes, const int64_t *ext_of_letter) {
    std::vector<int64_t> s;
    int64_t st = 1;
    for (char m : modes) {
        s.push_back(st);
        st *= ext_of_letter[m - 'a'];
    }
    return s;
}

int64_t stride_in(const std::string &modes, char m, const int64_t *ext) {
    int64_t st = 1;
    for (char x : modes) {
        if (x == m) return st;
        st *= ext[x - 'a'];
    }
    return 0;
}

bool has(const std::string &s, char c) { return s.find(c) != std::string::npos; }

std::string without(const std::string &s, char c) {
    std::string o;
    for (char x : s)
        if (x != c) o.push_back(x);
    return o;
}

// extents of a step spec "C=A,B" in order of first appearance
std::vector<int64_t> step_extents(const std::string &c, const std::string &a, const std::string &b,
                                  const int64_t *ext) {
    std::vector<int64_t> e;
    std::string seen;
    for (char m : c + a + b)
        if (!has(seen, m)) {
            seen.push_back(m);
            e.push_back(ext[m - 'a']);
        }
    return e;
}

}  // namespace

struct tc_chain_s {
    std::string d, op[3];
    tc_dtype dtype = TC_F64;
    int64_t ext[26] = {};
    std::vector<Variant> vars;
    int selected = -1;
    int64_t ws_limit = -1;
    void *T = nullptr;
    size_t t_bytes = 0;
    int device = -1;
};

namespace {

void destroy_variants(tc_chain_s &c) {
    for (auto &v : c.vars) {
        if (v.s1.plan) tc_plan_destroy(v.s1.plan);
        if (v.s2.plan) tc_plan_destroy(v.s2.plan);
    }
    c.vars.clear();
}

// Builds variant (p, q | r), sliced over `s` (0: not sliced); false when a
// step would contract nothing or a plan rejects it.
bool build_variant(tc_chain_s &c, int p, int q, char s, Variant &v) {
    const int r = 3 - p - q;
    const std::string &P = c.op[p], &Q = c.op[q], &R = c.op[r], &D = c.d;
    // T: the pair's indices still needed (in D or in R), D's order first,
    // then R's
    std::string t;
    for (char m : D)
        if ((has(P, m) || has(Q, m)) && !has(t, m)) t.push_back(m);
    for (char m : R)
        if ((has(P, m) || has(Q, m)) && !has(D, m) && !has(t, m)) t.push_back(m);
    // every step contracts at least one index
    bool k1 = false, k2 = false;
    for (char m : P)
        if (has(Q, m) && !has(t, m)) k1 = true;
    for (char m : t)
        if (has(R, m) && !has(D, m)) k2 = true;
    if (!k1 || !k2) return false;
    if (s) {
        if (!has(D, s) || !has(t, s) || has(R, s)) return false;
    }
    const int64_t *e = c.ext;
    v.p = p, v.q = q, v.r = r;
    v.sliced = s;
    v.slices = s ? e[s - 'a'] : 1;
    v.off_p = s ? stride_in(P, s, e) : 0;
    v.off_q = s ? stride_in(Q, s, e) : 0;
    v.off_d = s ? stride_in(D, s, e) : 0;
    const std::string ts = s ? without(t, s) : t, Ps = s ? without(P, s) : P, Qs = s ? without(Q, s) : Q,
                      Ds = s ? without(D, s) : D;
    v.t_modes = ts;
    v.t_elems = 1;
    for (char m : ts) v.t_elems *= e[m - 'a'];
    // step 1: T = P Q (P, Q with their full strides); step 2: D = T R
    auto full = [&](const std::string &modes, const std::string &all) {
        std::vector<int64_t> o;
        for (char m : modes) o.push_back(stride_in(all, m, e));
        return o;
    };
    v.s1.spec = ts + "=" + Ps + "," + Qs;
    v.s1.ext = step_extents(ts, Ps, Qs, e);
    std::vector<int64_t> st = dense_strides(ts, e), sp = full(Ps, P), sq = full(Qs, Q);
    v.s1.strides = st;
    v.s1.strides.insert(v.s1.strides.end(), sp.begin(), sp.end());
    v.s1.strides.insert(v.s1.strides.end(), sq.begin(), sq.end());
    v.s2.spec = Ds + "=" + ts + "," + R;
    v.s2.ext = step_extents(Ds, ts, R, e);
    std::vector<int64_t> sd = full(Ds, D), sr = dense_strides(R, e);
    v.s2.strides = sd;
    v.s2.strides.insert(v.s2.strides.end(), st.begin(), st.end());
    v.s2.strides.insert(v.s2.strides.end(), sr.begin(), sr.end());
    if (ts.empty() || Ds.empty()) return false;  // a scalar step: not a plan
    if (tc_plan_create(&v.s1.plan, v.s1.spec.c_str(), v.s1.ext.data(), v.s1.strides.data(), c.dtype) != TC_SUCCESS)
        return false;
    if (tc_plan_create(&v.s2.plan, v.s2.spec.c_str(), v.s2.ext.data(), v.s2.strides.data(), c.dtype) != TC_SUCCESS) {
        tc_plan_destroy(v.s1.plan);
        v.s1.plan = nullptr;
        return false;
    }
    double f1 = 0, f2 = 0;
    tc_plan_flops(v.s1.plan, &f1);
    tc_plan_flops(v.s2.plan, &f2);
    v.flops = (f1 + f2) * (double)v.slices;
    return true;
}

size_t t_bytes_of(const tc_chain_s &c, const Variant &v) {
    return (size_t)v.t_elems * tc::elem_bytes_c(c.dtype);
}

bool within_limit(const tc_chain_s &c, const Variant &v) {
    return c.ws_limit < 0 || (int64_t)t_bytes_of(c, v) <= c.ws_limit;
}

}  // namespace

using namespace tc;

extern "C" {

tc_status tc_chain_create(tc_chain *out, const char *spec, const int64_t *extents, tc_dtype dtype) {
    if (!out) return fail(TC_ERROR_INVALID_ARGUMENT, "out is NULL");
    *out = nullptr;
    if (!spec || !extents) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    if (dtype != TC_F64 && dtype != TC_F32 && dtype != TC_TF32 && dtype != TC_BF16X3 && dtype != TC_TF32X3)
        return fail(TC_ERROR_UNSUPPORTED_DTYPE, "chains run with FP64, FP32 or FP32-input tensor-core dtypes");
    std::string s;
    for (const char *x = spec; *x; ++x)
        if (*x != ' ') s.push_back(*x);
    const size_t eq = s.find('=');
    if (eq == std::string::npos) return fail(TC_ERROR_INVALID_SPEC, "spec must read \"D=X,Y,Z\"");
    std::string rhs = s.substr(eq + 1), parts[3];
    int n = 0;
    for (char ch : rhs) {
        if (ch == ',') {
            if (++n > 2) return fail(TC_ERROR_INVALID_SPEC, "spec must read \"D=X,Y,Z\"");
        } else {
            parts[n].push_back(ch);
        }
    }
    if (n != 2) return fail(TC_ERROR_INVALID_SPEC, "spec must read \"D=X,Y,Z\"");
    tc_chain_s *c = new (std::nothrow) tc_chain_s();
    if (!c) return fail(TC_ERROR_OUT_OF_MEMORY, "host allocation failed");
    c->d = s.substr(0, eq);
    for (int i = 0; i < 3; ++i) c->op[i] = parts[i];
    c->dtype = dtype;
    std::string seen;
    auto reject = [&](const std::string &msg) {
        delete c;
        return fail(TC_ERROR_INVALID_SPEC, msg);
    };
    for (const std::string *m : {&c->d, &c->op[0], &c->op[1], &c->op[2]}) {
        if (m != &c->d && m->empty()) return reject("every operand needs an index");
        for (size_t x = 0; x < m->size(); ++x) {
            const char ch = (*m)[x];
            if (ch < 'a' || ch > 'z') return reject("indices must be letters a-z");
            if (m->find(ch, x + 1) != std::string::npos) return reject(std::string("index repeated within an operand: ") + ch);
            if (!has(seen, ch)) seen.push_back(ch);
        }
    }
    for (char ch : seen) {
        const int in = has(c->op[0], ch) + has(c->op[1], ch) + has(c->op[2], ch);
        if (!has(c->d, ch) && in < 2) return reject(std::string("index in one operand only and not in D: ") + ch);
        if (has(c->d, ch) && in == 0) return reject(std::string("index of D in no operand: ") + ch);
    }
    for (size_t x = 0; x < seen.size(); ++x) {
        if (extents[x] < 1) {
            delete c;
            return fail(TC_ERROR_INVALID_EXTENT, std::string("extent < 1 for index ") + seen[x]);
        }
        c->ext[seen[x] - 'a'] = extents[x];
    }
    const int pairs[3][2] = {{0, 1}, {1, 2}, {0, 2}};
    for (auto &pq : pairs) {
        Variant v;
        if (build_variant(*c, pq[0], pq[1], 0, v)) c->vars.push_back(v);
        for (char sl : c->d) {  // sliced forms
            Variant w;
            if (build_variant(*c, pq[0], pq[1], sl, w)) c->vars.push_back(w);
        }
    }
    if (c->vars.empty()) return reject("no order contracts an index in both steps");
    tc_chain_select(c, -1);
    *out = c;
    return TC_SUCCESS;
}

tc_status tc_chain_destroy(tc_chain chain) {
    if (!chain) return TC_SUCCESS;
    destroy_variants(*chain);
    if (chain->T) cudaFree(chain->T);
    delete chain;
    return TC_SUCCESS;
}

tc_status tc_chain_variants(tc_chain chain, tc_chain_variant *buf, int32_t capacity, int32_t *count) {
    if (!chain || (capacity > 0 && !buf) || capacity < 0) return fail(TC_ERROR_INVALID_ARGUMENT, "bad arguments");
    if (count) *count = (int32_t)chain->vars.size();
    for (int32_t i = 0; i < capacity && i < (int32_t)chain->vars.size(); ++i) {
        const Variant &v = chain->vars[i];
        tc_chain_variant &o = buf[i];
        std::memset(&o, 0, sizeof(o));
        o.first[0] = v.p;
        o.first[1] = v.q;
        o.third = v.r;
        o.sliced = v.sliced;
        o.slices = v.slices;
        o.workspace_bytes = (int64_t)t_bytes_of(*chain, v);
        o.flops = v.flops;
        tc_plan_selected(v.s1.plan, &o.algorithm[0]);
        tc_plan_selected(v.s2.plan, &o.algorithm[1]);
        o.predicted_seconds = v.predicted;
    }
    return TC_SUCCESS;
}

tc_status tc_chain_set_workspace_limit(tc_chain chain, int64_t bytes) {
    if (!chain) return fail(TC_ERROR_INVALID_ARGUMENT, "chain is NULL");
    chain->ws_limit = bytes < 0 ? -1 : bytes;
    return TC_SUCCESS;
}

tc_status tc_chain_predict(tc_chain chain, int32_t all_algorithms, void *stream) {
    if (!chain) return fail(TC_ERROR_INVALID_ARGUMENT, "chain is NULL");
    for (auto &v : chain->vars) {
        double t[2] = {0, 0};
        Step *steps[2] = {&v.s1, &v.s2};
        for (int k = 0; k < 2; ++k) {
            tc_plan pl = steps[k]->plan;
            int32_t nalg = 1;
            if (all_algorithms) {
                tc_status s = tc_enumerate_algorithms(pl, nullptr, 0, &nalg);
                if (s != TC_SUCCESS) return s;
            }
            std::vector<int32_t> ids(nalg);
            for (int32_t x = 0; x < nalg; ++x) ids[x] = x;
            std::vector<double> sec(nalg, -1);
            tc_status s = tc_predict(pl, ids.data(), nalg, nullptr, nullptr, nullptr, sec.data(), stream);
            if (s != TC_SUCCESS) return s;
            int32_t best = -1;
            s = tc_plan_select_best(pl, &best);
            if (s != TC_SUCCESS) return s;
            t[k] = sec[best];
        }
        v.predicted = (t[0] + t[1]) * (double)v.slices;
    }
    return tc_chain_select(chain, -1);
}

tc_status tc_chain_select(tc_chain chain, int32_t variant) {
    if (!chain) return fail(TC_ERROR_INVALID_ARGUMENT, "chain is NULL");
    const int32_t n = (int32_t)chain->vars.size();
    if (variant >= n || variant < -1) return fail(TC_ERROR_INVALID_ARGUMENT, "variant out of range");
    if (variant >= 0) {
        if (!within_limit(*chain, chain->vars[variant]))
            return fail(TC_ERROR_INVALID_ARGUMENT, "the variant's intermediate exceeds the workspace limit");
        chain->selected = variant;
        return TC_SUCCESS;
    }
    // the smallest prediction where every variant has one, else the fewest
    // flops (then the fewest slices: launches); only variants within the limit
    bool all_pred = true;
    for (auto &v : chain->vars) all_pred = all_pred && v.predicted > 0;
    int32_t best = -1;
    for (int32_t i = 0; i < n; ++i) {
        const Variant &v = chain->vars[i];
        if (!within_limit(*chain, v)) continue;
        if (best < 0) {
            best = i;
            continue;
        }
        const Variant &b = chain->vars[best];
        const bool better = all_pred ? v.predicted < b.predicted
                                     : (v.flops < b.flops || (v.flops == b.flops && v.slices < b.slices));
        if (better) best = i;
    }
    if (best < 0) return fail(TC_ERROR_INVALID_ARGUMENT, "no variant fits the workspace limit");
    chain->selected = best;
    return TC_SUCCESS;
}

tc_status tc_chain_selected(tc_chain chain, int32_t *variant) {
    if (!chain || !variant) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    *variant = chain->selected;
    return TC_SUCCESS;
}

tc_status tc_chain_execute(tc_chain chain, const void *alpha, const void *X, const void *Y, const void *Z,
                           const void *beta, void *D, void *stream) {
    if (!chain || !alpha || !beta || !X || !Y || !Z || !D) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    tc_chain_s &c = *chain;
    if (c.selected < 0) return fail(TC_ERROR_INVALID_ARGUMENT, "no variant selected");
    const Variant &v = c.vars[c.selected];
    int dev = 0;
    cudaGetDevice(&dev);
    if (c.device >= 0 && c.device != dev) return fail(TC_ERROR_INVALID_ARGUMENT, "chain used on another device");
    c.device = dev;
    const size_t need = t_bytes_of(c, v);
    if (need > c.t_bytes) {
        if (c.T) {
            cudaStreamSynchronize((cudaStream_t)stream);  // the old intermediate may still be in use
            cudaFree(c.T);
        }
        c.T = nullptr;
        c.t_bytes = 0;
        cudaError_t e = cudaMalloc(&c.T, need);
        if (e != cudaSuccess) return fail(TC_ERROR_OUT_OF_MEMORY, cudaGetErrorString(e));
        c.t_bytes = need;
    }
    const void *ops[3] = {X, Y, Z};
    const size_t esz = elem_bytes_ab(c.dtype), dsz = elem_bytes_c(c.dtype);
    const double one = 1.0, zero = 0.0;
    const float onef = 1.0f, zerof = 0.0f;
    const void *a1 = c.dtype == TC_F64 ? (const void *)&one : (const void *)&onef;
    const void *b1 = c.dtype == TC_F64 ? (const void *)&zero : (const void *)&zerof;
    for (int64_t sv = 0; sv < v.slices; ++sv) {
        const char *P = (const char *)ops[v.p] + (size_t)(sv * v.off_p) * esz;
        const char *Q = (const char *)ops[v.q] + (size_t)(sv * v.off_q) * esz;
        char *Dp = (char *)D + (size_t)(sv * v.off_d) * dsz;
        tc_status s = tc_execute(v.s1.plan, a1, P, Q, b1, c.T, stream);
        if (s != TC_SUCCESS) return s;
        s = tc_execute(v.s2.plan, alpha, c.T, ops[v.r], beta, Dp, stream);
        if (s != TC_SUCCESS) return s;
    }
    return TC_SUCCESS;
}

tc_status tc_chain_device_status(tc_chain chain) {
    if (!chain) return fail(TC_ERROR_INVALID_ARGUMENT, "chain is NULL");
    if (chain->selected < 0) return TC_SUCCESS;
    const Variant &v = chain->vars[chain->selected];
    tc_status s = tc_plan_device_status(v.s1.plan);
    if (s != TC_SUCCESS) return s;
    return tc_plan_device_status(v.s2.plan);
}

}  // extern "C"
