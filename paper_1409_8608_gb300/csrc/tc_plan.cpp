// Host planner: spec parsing, index classification, validation and the
// algorithm generator of Section 2 (slicing rules of Table 1, all loop
// permutations, copy insertion, naming), plus the plan-level C ABI.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "tc_internal.h"

namespace tc {

static thread_local std::string g_last_error;

tc_status fail(tc_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

size_t elem_bytes_ab(tc_dtype dt) {
    switch (dt) {
    case TC_F64: return 8;
    case TC_BF16:
    case TC_F16: return 2;
    default: return 4;
    }
}

size_t elem_bytes_c(tc_dtype dt) { return dt == TC_F64 ? 8 : 4; }

namespace {

bool parse_operand(const std::string &s, std::string &out) {
    out.clear();
    for (char ch : s) {
        if (ch == ' ') continue;
        if (ch < 'a' || ch > 'z') return false;
        out.push_back(ch);
    }
    return true;
}

// Table 1: the admissible kernel-index tuples of one kernel, in
// enumeration order (free index of A outermost, then of B, then the
// contracted index).
std::vector<std::vector<int>> kernel_choices(int kernel, const Plan &p) {
    std::vector<std::vector<int>> out;
    switch (kernel) {
    case TC_KERNEL_DOT:
        for (int k : p.contracted) out.push_back({k});
        break;
    case TC_KERNEL_AXPY:
        for (int f : p.freeA) out.push_back({f});
        for (int f : p.freeB) out.push_back({f});
        break;
    case TC_KERNEL_GEMV: {
        std::vector<int> fr(p.freeA);
        fr.insert(fr.end(), p.freeB.begin(), p.freeB.end());
        for (int f : fr)
            for (int k : p.contracted) out.push_back({f, k});
        break;
    }
    case TC_KERNEL_GER:
        for (int fa : p.freeA)
            for (int fb : p.freeB) out.push_back({fa, fb});
        break;
    case TC_KERNEL_GEMM:
        for (int fa : p.freeA)
            for (int fb : p.freeB)
                for (int k : p.contracted) out.push_back({fa, fb, k});
        break;
    }
    return out;
}

const char *kKernelNames[] = {"dot", "axpy", "gemv", "ger", "gemm", "gett"};

void finish_algorithm(const Plan &p, Algorithm &a) {
    // copies: a matrix slice (two kernel modes) without a unit-stride mode
    for (int o = 0; o < 3; ++o) {
        const Layout &L = p.op[o];
        int nkm = 0;
        bool unit = false;
        for (int m = 0; m < L.n; ++m) {
            for (int r = 0; r < a.nk; ++r)
                if (L.idx[m] == a.kidx[r]) {
                    ++nkm;
                    if (L.stride[m] == 1) unit = true;
                }
        }
        if (nkm != 2 || unit) continue;
        int level = -1;
        for (int pos = 0; pos < a.nloops; ++pos)
            if (L.has(a.loops[pos])) level = pos;
        a.copy_level[o] = level;
    }
    // name: loops, an apostrophe after the loop holding each copy
    std::string name;
    for (int o = 0; o < 3; ++o)
        if (a.copy_level[o] == -1) name.push_back('\'');
    for (int pos = 0; pos < a.nloops; ++pos) {
        name.push_back(p.letter[a.loops[pos]]);
        for (int o = 0; o < 3; ++o)
            if (a.copy_level[o] == pos) name.push_back('\'');
    }
    name += "-";
    name += kKernelNames[a.kernel];
    // phases: contracted loops that enclose a free loop run device-wide in
    // sequence; everything else runs concurrently or inside a task
    a.q = -1;
    for (int pos = 0; pos < a.nloops; ++pos) {
        if (p.cls[a.loops[pos]] != CLS_CONTRACTED) continue;
        for (int inner = pos + 1; inner < a.nloops; ++inner)
            if (p.cls[a.loops[inner]] != CLS_CONTRACTED) { a.q = pos; break; }
    }
    int64_t phases = 1;
    for (int pos = 0; pos <= a.q; ++pos)
        if (p.cls[a.loops[pos]] == CLS_CONTRACTED) phases *= p.ext[a.loops[pos]];

    tc_algorithm &pub = a.pub;
    std::memset(&pub, 0, sizeof(pub));
    pub.id = 0;
    std::snprintf(pub.name, sizeof(pub.name), "%s", name.c_str());
    pub.kernel = a.kernel;
    pub.n_loops = a.nloops;
    for (int pos = 0; pos < a.nloops && pos < 8; ++pos) pub.loops[pos] = p.letter[a.loops[pos]];
    pub.n_kernel_indices = a.nk;
    for (int r = 0; r < a.nk; ++r) pub.kernel_indices[r] = p.letter[a.kidx[r]];
    pub.copy_mask = 0;
    for (int o = 0; o < 3; ++o) {
        pub.copy_level[o] = a.copy_level[o];
        if (a.copy_level[o] != -2) pub.copy_mask |= 1u << o;
    }
    pub.n_phases = (int32_t)std::min<int64_t>(phases, INT32_MAX);
}

}  // namespace

// enumerate = false: spec, index classes, layouts and the fused GETT only
// (no Section 2 algorithms), for callers that only run the GETT.
tc_status build_plan(Plan &p, const char *spec, const int64_t *extents, const int64_t *strides, tc_dtype dtype,
                     bool enumerate) {
    if (!spec) return fail(TC_ERROR_INVALID_ARGUMENT, "spec is NULL");
    if (!extents) return fail(TC_ERROR_INVALID_ARGUMENT, "extents is NULL");
    if (dtype < TC_F64 || dtype > TC_E4M3)
        return fail(TC_ERROR_UNSUPPORTED_DTYPE, "unknown dtype");
    std::string s(spec);
    size_t eq = s.find('='), comma = s.find(',');
    if (eq == std::string::npos || comma == std::string::npos || comma < eq ||
        s.find('=', eq + 1) != std::string::npos ||
        s.find(',', comma + 1) != std::string::npos)
        return fail(TC_ERROR_INVALID_SPEC, "spec must read \"C=A,B\"");
    std::string c, a, b;
    if (!parse_operand(s.substr(0, eq), c) ||
        !parse_operand(s.substr(eq + 1, comma - eq - 1), a) ||
        !parse_operand(s.substr(comma + 1), b))
        return fail(TC_ERROR_INVALID_SPEC, "indices must be letters a-z");
    if (a.empty() || b.empty())
        return fail(TC_ERROR_INVALID_SPEC, "both inputs need at least one index");
    const std::string *mode_str[3] = {&a, &b, &c};
    for (int o = 0; o < 3; ++o) {
        const std::string &m = *mode_str[o];
        if ((int)m.size() > kMaxModes)
            return fail(TC_ERROR_INVALID_SPEC, "more than 8 modes in one operand");
        for (size_t x = 0; x < m.size(); ++x)
            if (m.find(m[x], x + 1) != std::string::npos)
                return fail(TC_ERROR_INVALID_SPEC,
                            std::string("index repeated within an operand: ") + m[x]);
    }
    // distinct indices in order of first appearance: C, then A, then B
    p.nidx = 0;
    for (char ch : c + a + b) {
        bool seen = false;
        for (int x = 0; x < p.nidx; ++x) seen |= p.letter[x] == ch;
        if (!seen) {
            if (p.nidx == kMaxIdx) return fail(TC_ERROR_INVALID_SPEC, "too many indices");
            p.letter[p.nidx++] = ch;
        }
    }
    auto id_of = [&](char ch) {
        for (int x = 0; x < p.nidx; ++x)
            if (p.letter[x] == ch) return x;
        return -1;
    };
    // Section 1: contracted = in A and B, not in C; free = in one input and
    // C.  Beyond the paper: an index in A, B and C is a batch (Hadamard)
    // index -- free, and carried by both inputs.
    for (int x = 0; x < p.nidx; ++x) {
        char ch = p.letter[x];
        bool inA = a.find(ch) != std::string::npos;
        bool inB = b.find(ch) != std::string::npos;
        bool inC = c.find(ch) != std::string::npos;
        if (inA && inB && inC) p.cls[x] = CLS_BATCH;
        else if (inA && inB) p.cls[x] = CLS_CONTRACTED;
        else if (inA && inC) p.cls[x] = CLS_FREE_A;
        else if (inB && inC) p.cls[x] = CLS_FREE_B;
        else
            return fail(TC_ERROR_INVALID_SPEC,
                        std::string("index must be contracted (A and B) or free (one input and C): ") + ch);
    }
    for (int x = 0; x < p.nidx; ++x) {
        if (extents[x] < 1)
            return fail(TC_ERROR_INVALID_EXTENT, std::string("extent < 1 for index ") + p.letter[x]);
        p.ext[x] = extents[x];
    }
    // total iteration space must fit comfortably in int64
    {
        double t = 1;
        for (int x = 0; x < p.nidx; ++x) t *= (double)p.ext[x];
        if (t > 4.0e18) return fail(TC_ERROR_INVALID_EXTENT, "iteration space overflows int64");
    }
    int off = 0;
    const int order[3] = {OP_C, OP_A, OP_B};  // stride array order: C, A, B
    for (int oi = 0; oi < 3; ++oi) {
        int o = order[oi];
        const std::string &m = *mode_str[o];
        Layout &L = p.op[o];
        L.n = (int)m.size();
        int64_t dense = 1;
        for (int k = 0; k < L.n; ++k) {
            L.idx[k] = id_of(m[k]);
            if (strides) {
                if (strides[off + k] < 1)
                    return fail(TC_ERROR_INVALID_STRIDE, "strides must be >= 1");
                L.stride[k] = strides[off + k];
            } else {
                L.stride[k] = dense;
            }
            dense *= p.ext[L.idx[k]];
        }
        off += L.n;
    }
    // C must not alias itself: sorted by stride, each stride must step over
    // the whole span of the smaller modes (modes of extent 1 ignored)
    {
        const Layout &L = p.op[OP_C];
        std::vector<std::pair<int64_t, int64_t>> sm;
        for (int k = 0; k < L.n; ++k)
            if (p.ext[L.idx[k]] > 1) sm.push_back({L.stride[k], p.ext[L.idx[k]]});
        std::sort(sm.begin(), sm.end());
        int64_t span = 1;
        for (auto &e : sm) {
            if (e.first < span)
                return fail(TC_ERROR_INVALID_STRIDE, "C strides let two elements share an address");
            span = e.first * e.second;
        }
    }
    for (int x = 0; x < p.nidx; ++x) {
        if (p.cls[x] == CLS_CONTRACTED) p.contracted.push_back(x);
        else if (p.cls[x] == CLS_FREE_A) p.freeA.push_back(x);
        else if (p.cls[x] == CLS_FREE_B) p.freeB.push_back(x);
        else p.batch.push_back(x);
    }
    p.spec = s;
    p.dtype = dtype;

    // algorithm 0: the fused GETT (whole contraction in one kernel)
    {
        Algorithm g;
        g.kernel = TC_KERNEL_GETT;
        std::memset(&g.pub, 0, sizeof(g.pub));
        std::snprintf(g.pub.name, sizeof(g.pub.name), "gett");
        g.pub.kernel = TC_KERNEL_GETT;
        for (int o = 0; o < 3; ++o) g.pub.copy_level[o] = -2;
        g.pub.n_phases = 1;
        p.algs.push_back(g);
    }
    // Section 2: every kernel, every admissible kernel-index choice, every
    // permutation of the sliced loops
    for (int kernel = TC_KERNEL_DOT; kernel <= TC_KERNEL_GEMM && enumerate; ++kernel) {
        for (const auto &kc : kernel_choices(kernel, p)) {
            std::vector<int> sliced;
            for (int x = 0; x < p.nidx; ++x)
                if (std::find(kc.begin(), kc.end(), x) == kc.end()) sliced.push_back(x);
            // ids are already in first-appearance order, so sorted ids give
            // the lexicographically first permutation
            do {
                Algorithm alg;
                alg.kernel = kernel;
                alg.nk = (int)kc.size();
                for (int r = 0; r < alg.nk; ++r) alg.kidx[r] = kc[r];
                alg.nloops = (int)sliced.size();
                for (int pos = 0; pos < alg.nloops; ++pos) alg.loops[pos] = sliced[pos];
                finish_algorithm(p, alg);
                p.algs.push_back(alg);
            } while (std::next_permutation(sliced.begin(), sliced.end()));
        }
    }
    for (size_t i = 0; i < p.algs.size(); ++i) p.algs[i].pub.id = (int32_t)i;
    p.selected = 0;
    return TC_SUCCESS;
}

}  // namespace tc

using namespace tc;

extern "C" {

const char *tc_status_string(tc_status st) {
    switch (st) {
    case TC_SUCCESS: return "success";
    case TC_ERROR_INVALID_SPEC: return "invalid contraction spec";
    case TC_ERROR_INVALID_EXTENT: return "invalid extent";
    case TC_ERROR_INVALID_STRIDE: return "invalid stride";
    case TC_ERROR_UNSUPPORTED_DTYPE: return "unsupported dtype for this algorithm";
    case TC_ERROR_INVALID_ALGORITHM: return "invalid algorithm id";
    case TC_ERROR_OUT_OF_MEMORY: return "out of device memory";
    case TC_ERROR_CUDA: return "CUDA runtime error";
    case TC_ERROR_TIMEOUT: return "device wait timed out";
    case TC_ERROR_INVALID_ARGUMENT: return "invalid argument";
    case TC_ERROR_ADMISSION: return "request exceeds the admission budget";
    }
    return "unknown status";
}

const char *tc_last_error(void) { return g_last_error.c_str(); }

tc_status tc_plan_create(tc_plan *out, const char *spec, const int64_t *extents,
                         const int64_t *strides, tc_dtype dtype) {
    if (!out) return fail(TC_ERROR_INVALID_ARGUMENT, "out is NULL");
    *out = nullptr;
    tc_plan_s *h = new (std::nothrow) tc_plan_s();
    if (!h) return fail(TC_ERROR_OUT_OF_MEMORY, "host allocation failed");
    tc_status st = build_plan(h->p, spec, extents, strides, dtype, true);
    if (st != TC_SUCCESS) {
        delete h;
        return st;
    }
    *out = h;
    return TC_SUCCESS;
}

tc_status tc_plan_destroy(tc_plan plan) {
    if (!plan) return TC_SUCCESS;
    Plan &p = plan->p;
    if (p.device >= 0) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(p.device);
        gett_release(p);
        if (p.workspace) cudaFree(p.workspace);
        if (p.dev_status) cudaFree(p.dev_status);
        if (p.flush_buf) cudaFree(p.flush_buf);
        if (p.qbuf) cudaFree(p.qbuf);
        if (p.busy_event) cudaEventDestroy((cudaEvent_t)p.busy_event);
        for (void *d : p.host_dev)
            if (d) cudaFree(d);
        cudaSetDevice(cur);
    }
    delete plan;
    return TC_SUCCESS;
}

tc_status tc_algorithm_count(tc_plan plan, int32_t *count) {
    if (!plan || !count) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    *count = (int32_t)plan->p.algs.size();
    return TC_SUCCESS;
}

tc_status tc_enumerate_algorithms(tc_plan plan, tc_algorithm *out,
                                  int32_t capacity, int32_t *count) {
    if (!plan || !count) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    if (capacity < 0 || (capacity > 0 && !out))
        return fail(TC_ERROR_INVALID_ARGUMENT, "bad output buffer");
    const Plan &p = plan->p;
    *count = (int32_t)p.algs.size();
    for (int32_t i = 0; i < capacity && i < *count; ++i) out[i] = p.algs[i].pub;
    return TC_SUCCESS;
}

tc_status tc_plan_select(tc_plan plan, int32_t alg_id) {
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    if (alg_id < 0 || alg_id >= (int32_t)plan->p.algs.size())
        return fail(TC_ERROR_INVALID_ALGORITHM, "algorithm id out of range");
    plan->p.selected = alg_id;
    return TC_SUCCESS;
}

tc_status tc_plan_selected(tc_plan plan, int32_t *alg_id) {
    if (!plan || !alg_id) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    *alg_id = plan->p.selected;
    return TC_SUCCESS;
}

tc_status tc_algorithm_workspace(tc_plan plan, int32_t alg_id, size_t *bytes) {
    if (!plan || !bytes) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    const Plan &p = plan->p;
    if (alg_id < 0 || alg_id >= (int32_t)p.algs.size())
        return fail(TC_ERROR_INVALID_ALGORITHM, "algorithm id out of range");
    *bytes = alg_id == 0 ? gett_workspace_bytes(p) : nest_workspace_bytes(p, p.algs[alg_id]);
    return TC_SUCCESS;
}

tc_status tc_plan_set_split(tc_plan plan, int32_t products) {
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    if (products != 3 && products != 6 && products != 9)
        return fail(TC_ERROR_INVALID_ARGUMENT, "split products must be 3, 6 or 9");
    plan->p.split_products = products;
    return TC_SUCCESS;
}

tc_status tc_plan_set_gett_tile(tc_plan plan, int32_t width) {
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    if (width != 0 && width != 128 && width != 256)
        return fail(TC_ERROR_INVALID_ARGUMENT, "GETT tile width must be 0, 128 or 256");
    plan->p.gett_bn = width;
    return TC_SUCCESS;
}

tc_status tc_plan_set_gett_tma(tc_plan plan, int32_t enable) {
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    if (enable != 0 && enable != 1) return fail(TC_ERROR_INVALID_ARGUMENT, "enable must be 0 or 1");
    plan->p.gett_tma = enable;
    return TC_SUCCESS;
}

tc_status tc_plan_set_gett_pack(tc_plan plan, int32_t mode) {
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    if (mode < 0 || mode > 3) return fail(TC_ERROR_INVALID_ARGUMENT, "pack mode must be 0, 1, 2 or 3");
    plan->p.gett_pack = mode;
    return TC_SUCCESS;
}

tc_status tc_plan_set_gett_pair(tc_plan plan, int32_t enable) {
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    if (enable != 0 && enable != 1) return fail(TC_ERROR_INVALID_ARGUMENT, "enable must be 0 or 1");
    plan->p.gett_pair = enable;
    return TC_SUCCESS;
}

tc_status tc_plan_set_split_accumulators(tc_plan plan, int32_t enable) {
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    if (enable < -1 || enable > 1) return fail(TC_ERROR_INVALID_ARGUMENT, "enable must be -1, 0 or 1");
    plan->p.gett_split = enable;
    return TC_SUCCESS;
}

tc_status tc_plan_set_compensation(tc_plan plan, int32_t chunk) {
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    if (chunk < -1 || (chunk > 0 && chunk % 32 != 0))
        return fail(TC_ERROR_INVALID_ARGUMENT, "compensation chunk must be -1, 0 or a positive multiple of 32");
    plan->p.comp_chunk = chunk;
    return TC_SUCCESS;
}

tc_status tc_plan_flops(tc_plan plan, double *flops) {
    if (!plan || !flops) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    double f = 2.0;
    for (int x = 0; x < plan->p.nidx; ++x) f *= (double)plan->p.ext[x];
    *flops = f;
    return TC_SUCCESS;
}

tc_status tc_execute(tc_plan plan, const void *alpha, const void *A, const void *B,
                     const void *beta, void *C, void *stream) {
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    if (!alpha || !beta) return fail(TC_ERROR_INVALID_ARGUMENT, "alpha/beta is NULL");
    if (!A || !B || !C) return fail(TC_ERROR_INVALID_ARGUMENT, "operand pointer is NULL");
    Plan &p = plan->p;
    // One plan runs on one stream at a time: its workspace and status word
    // serve one execute.  An execute on another stream while the previous
    // one is still in flight is refused.  Work captured into a graph is
    // not checked (the graph and its caller order the replays).
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing((cudaStream_t)stream, &cs);
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, std::string("stream query: ") + cudaGetErrorString(e));
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    if (!capturing && p.busy_event && stream != p.last_stream) {
        e = cudaEventQuery((cudaEvent_t)p.busy_event);
        if (e == cudaErrorNotReady)
            return fail(TC_ERROR_INVALID_ARGUMENT,
                        "the plan's previous execute is still running on another stream; "
                        "give each stream its own plan, or wait for that stream first");
        if (e != cudaSuccess) return fail(TC_ERROR_CUDA, std::string("event query: ") + cudaGetErrorString(e));
    }
    const Algorithm &alg = p.algs[p.selected];
    tc_status s = alg.kernel == TC_KERNEL_GETT ? exec_gett(p, alpha, A, B, beta, C, stream)
                                               : exec_nest(p, alg, alpha, A, B, beta, C, stream);
    if (s != TC_SUCCESS || capturing) return s;
    if (!p.busy_event) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(TC_ERROR_CUDA, std::string("event create: ") + cudaGetErrorString(e));
        p.busy_event = ev;
    }
    e = cudaEventRecord((cudaEvent_t)p.busy_event, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, std::string("event record: ") + cudaGetErrorString(e));
    return TC_SUCCESS;
}

// Elements an operand's strided layout spans: 1 + sum (extent - 1) * stride.
static size_t operand_span_bytes(const Plan &p, int o) {
    int64_t span = 1;
    for (int m = 0; m < p.op[o].n; ++m) span += (p.ext[p.op[o].idx[m]] - 1) * p.op[o].stride[m];
    return (size_t)span * (o == OP_C ? elem_bytes_c(p.dtype) : elem_bytes_ab(p.dtype));
}

tc_status tc_execute_host(tc_plan plan, const void *alpha, const void *hA, const void *hB, const void *beta,
                          void *hC, void *stream) {
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    if (!alpha || !beta) return fail(TC_ERROR_INVALID_ARGUMENT, "alpha/beta is NULL");
    if (!hA || !hB || !hC) return fail(TC_ERROR_INVALID_ARGUMENT, "operand pointer is NULL");
    Plan &p = plan->p;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    if (p.device >= 0 && p.device != dev)
        return fail(TC_ERROR_INVALID_ARGUMENT, "plan used on a different device than its first execute");
    // device copies of the three operands, allocated once (outside any
    // graph capture) and kept with the plan
    const size_t bytes[3] = {operand_span_bytes(p, OP_A), operand_span_bytes(p, OP_B), operand_span_bytes(p, OP_C)};
    for (int o = 0; o < 3; ++o) {
        if (p.host_dev[o] && p.host_dev_bytes[o] >= bytes[o]) continue;
        if (p.host_dev[o]) cudaFree(p.host_dev[o]);
        p.host_dev[o] = nullptr;
        p.host_dev_bytes[o] = 0;
        e = cudaMalloc(&p.host_dev[o], bytes[o]);
        if (e != cudaSuccess) {
            p.host_dev[o] = nullptr;
            return fail(TC_ERROR_OUT_OF_MEMORY, std::string("device copy of an operand: ") + cudaGetErrorString(e));
        }
        p.host_dev_bytes[o] = bytes[o];
    }
    const bool beta_zero = p.dtype == TC_F64 ? *(const double *)beta == 0.0 : *(const float *)beta == 0.0f;
    cudaStream_t st = (cudaStream_t)stream;
    // the same stream rule as tc_execute, checked before any copy is queued
    if (p.busy_event && stream != p.last_stream) {
        e = cudaEventQuery((cudaEvent_t)p.busy_event);
        if (e == cudaErrorNotReady)
            return fail(TC_ERROR_INVALID_ARGUMENT, "the plan's previous execute is still running on another stream");
    }
    const void *src[3] = {hA, hB, hC};
    for (int o = 0; o < 3; ++o) {
        if (o == OP_C && beta_zero) continue;
        e = cudaMemcpyAsync(p.host_dev[o], src[o], bytes[o], cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(TC_ERROR_CUDA, std::string("host to device copy: ") + cudaGetErrorString(e));
    }
    tc_status s = tc_execute(plan, alpha, p.host_dev[OP_A], p.host_dev[OP_B], beta, p.host_dev[OP_C], stream);
    if (s != TC_SUCCESS) return s;
    e = cudaMemcpyAsync(hC, p.host_dev[OP_C], bytes[OP_C], cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, std::string("device to host copy: ") + cudaGetErrorString(e));
    return TC_SUCCESS;
}

tc_status tc_plan_device_status(tc_plan plan) {
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    Plan &p = plan->p;
    if (!p.dev_status) return TC_SUCCESS;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p.device);
    cudaStreamSynchronize((cudaStream_t)p.last_stream);
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, p.dev_status, sizeof(int), cudaMemcpyDeviceToHost);
    int zero = 0;
    if (e == cudaSuccess) e = cudaMemcpy(p.dev_status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    cudaSetDevice(cur);
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    return h == 0 ? TC_SUCCESS : fail(TC_ERROR_TIMEOUT, "a bounded device wait gave up");
}

}  // extern "C"
