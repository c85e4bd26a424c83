// Internal declarations shared by the host planner (tc_plan.cpp) and the
// device executors (*.cu).  Not part of the public ABI (include/tc.h).
#pragma once

#include <cstdint>
#include <cstddef>
#include <map>
#include <string>
#include <vector>

#include "tc.h"

namespace tc {

constexpr int kMaxModes = 8;    // modes per operand
constexpr int kMaxIdx = 24;     // distinct indices per spec

enum OperandId { OP_A = 0, OP_B = 1, OP_C = 2 };

// CLS_BATCH: an index in A, B and C (a batch or Hadamard index, outside the
// paper's notation): never a kernel index, always a sliced (free) loop.
enum IndexClass { CLS_FREE_A = 0, CLS_FREE_B = 1, CLS_CONTRACTED = 2, CLS_BATCH = 3 };

struct Layout {
    int n = 0;                    // number of modes
    int idx[kMaxModes] = {};      // index id of each mode, storage order
    int64_t stride[kMaxModes] = {};
    bool has(int id) const {
        for (int m = 0; m < n; ++m)
            if (idx[m] == id) return true;
        return false;
    }
    int64_t stride_of(int id) const {
        for (int m = 0; m < n; ++m)
            if (idx[m] == id) return stride[m];
        return 0;
    }
};

struct Algorithm {
    tc_algorithm pub{};
    int kernel = 0;                 // tc_kernel
    int nk = 0;
    int kidx[3] = {-1, -1, -1};     // kernel indices by role
    int nloops = 0;
    int loops[kMaxIdx] = {};        // sliced index ids, outermost first
    int copy_level[3] = {-2, -2, -2};
    int q = -1;                     // deepest contracted loop enclosing a free loop
};

struct Plan {
    std::string spec;
    tc_dtype dtype = TC_F64;
    int nidx = 0;
    char letter[kMaxIdx] = {};
    int64_t ext[kMaxIdx] = {};
    int cls[kMaxIdx] = {};
    Layout op[3];                   // A, B, C
    std::vector<int> contracted, freeA, freeB, batch;  // first-appearance order
    std::vector<Algorithm> algs;    // algs[0] is the fused GETT
    int selected = 0;
    int split_products = 6;         // TC_BF16X3: 3, 6 or 9 slice products
    int gett_bn = 0;                // tensor-core GETT tile width (0: by N)
    int gett_tma = 1;               // tensor-core GETT: TMA staging where legal
    int gett_pack = 1;              // tensor-core GETT: pre-convert the small input (0 never, 1 auto, 2 always)
    int comp_chunk = -1;            // TC_BF16X3: compensated K chunk (-1 default, 0 off)
    int gett_pair = 0;              // tensor-core GETT: CTA pairs (cta_group::2) where legal
    int gett_split = -1;            // TC_BF16X3: (0,0) products in their own accumulator (-1 auto)
    // device resources, created lazily by the first execute
    int device = -1;
    void *workspace = nullptr;
    size_t workspace_bytes = 0;
    int *dev_status = nullptr;      // bounded-wait status word
    void *last_stream = nullptr;
    void *busy_event = nullptr;     // recorded after each tc_execute (cudaEvent_t)
    void *host_dev[3] = {nullptr, nullptr, nullptr};  // tc_execute_host: device copies of A, B, C
    size_t host_dev_bytes[3] = {0, 0, 0};
    void *gett_state = nullptr;     // owned by the GETT executor
    void *qbuf = nullptr;           // TC_E4M3: the inputs' maxima and scales (16 bytes)
    void *flush_buf = nullptr;      // predictor: remote regions / L2 flush
    size_t flush_bytes = 0;
    std::vector<double> predicted;  // last tc_predict result per algorithm (< 0: none)
};

// A micro-benchmark run of one algorithm (Section 3 restated for the
// device): a nest runs one phase -- its copies and its kernel -- given by
// the values of the phase loops, over `fraction` of the phase's work; the
// GETT runs `fraction` of its tiles.
struct Probe {
    std::vector<int64_t> phase;  // phase-loop values, outermost first
    bool first = true;           // the contraction's first phase (C from beta)
    int changed_from = 0;        // outermost phase loop that advanced
    double fraction = 1.0;
};

// error reporting (thread-local message)
tc_status fail(tc_status st, const std::string &msg);

// Parses and validates a spec into p; with enumerate = false only the
// fused GETT (algorithm 0) is listed (tc_plan.cpp).
tc_status build_plan(Plan &p, const char *spec, const int64_t *extents, const int64_t *strides, tc_dtype dtype,
                     bool enumerate);

// element size of A/B and of C for a dtype
size_t elem_bytes_ab(tc_dtype dt);
size_t elem_bytes_c(tc_dtype dt);

// device-side executors (tc_exec.cu, tc_gett.cu)
tc_status exec_nest(Plan &p, const Algorithm &alg, const void *alpha,
                    const void *A, const void *B, const void *beta, void *C,
                    void *stream, const Probe *probe = nullptr);
size_t nest_workspace_bytes(const Plan &p, const Algorithm &alg);
int64_t nest_phase_items(const Plan &p, const Algorithm &alg, bool *tiled);
int64_t gett_items(const Plan &p);
tc_status exec_gett(Plan &p, const void *alpha, const void *A, const void *B,
                    const void *beta, void *C, void *stream, const Probe *probe = nullptr);
tc_status exec_gett_simt(Plan &p, const void *alpha, const void *A, const void *B,
                         const void *beta, void *C, void *stream, const Probe *probe = nullptr);
size_t gett_workspace_bytes(const Plan &p);
void gett_release(Plan &p);
tc_status ensure_device_resources(Plan &p, size_t workspace_bytes);

// One phase of a gemm loop nest on the tensor cores (tensor dtypes): the
// kernel's free index of A (m: sA, sC) and of B (n: sB, sC), its K modes
// (the in-task contracted loops outermost first, the kernel's contracted
// index last: sA, sB), and the concurrent free loops as tasks (t: sA, sB,
// sC, first fastest).  init 2: C = alpha*acc; 1: C = alpha*acc + beta*C.
struct NestGemmMode {
    int64_t ext, sA, sB, sC;
};
struct NestGemm {
    NestGemmMode m, n;
    int nk;
    NestGemmMode k[kMaxModes];
    int nt;
    NestGemmMode t[kMaxModes];
    const void *A;
    const void *B;
    void *C;
    float alpha, beta;
    int init;
};
tc_status gett_launch_nest(Plan &p, const NestGemm &g, double frac, void *stream);

// Batched SIMT GETT (FP64 / FP32; the serving form's batches): one
// descriptor per problem (simt_desc_bytes each) holding its modes, strides
// and operands with alpha = 1, beta = 0; simt_fill_desc returns the
// problem's tile count, tile0 is its first tile in the batch's list.  The
// launch runs tile t of the list in CTA t (dtile_prob[t] = its problem).
size_t simt_desc_bytes();
int64_t simt_fill_desc(const Plan &p, const void *A, const void *B, void *C, int64_t tile0, void *out);
tc_status simt_launch_batch(tc_dtype dt, const void *ddescs, const int32_t *dtile_prob, int64_t ntiles,
                            void *stream);

// One problem of the batched form: a strided GEMM over the merged free
// modes of A (m), of B (n) and the merged contracted modes (k).
struct BatchProblem {
    int64_t M, N, K;
    int64_t sAm, sAk, sBk, sBn, sCm, sCn;
    const void *A;
    const void *B;
    void *C;
    int64_t tile0;    // first tile of this problem in the flattened list
    int32_t shape;    // SIMT tiles (8 << shape) x (512 >> shape), shape 0..4
    int32_t tiles_m;
    int32_t bk;       // SIMT K chunk per pipeline stage (8, 16 or 32)
    int32_t flags;    // SIMT copy paths (kBatchVecA | kBatchVecB | kBatchStagedC)
};
constexpr int32_t kBatchVecA = 1;     // A copied in 16-byte pieces (m contiguous, aligned)
constexpr int32_t kBatchVecB = 2;     // B copied in 16-byte pieces (k contiguous, aligned)
constexpr int32_t kBatchStagedC = 4;  // a tile's C is one contiguous run (staged epilogue)

// Batched split-BF16 on the tensor-core GETT kernel: one device descriptor
// per problem (gett_desc_bytes each, filled by gett_fill_batch_desc for
// 128 x bn tiles), then one launch over tiles [t_begin, t_end).
// Split-BF16 stream kernel of the batched form (tc_stream.cu): problems
// with A, B and C dense along m, k and m, K a multiple of 4 up to 32, M up
// to 128, 16-byte aligned A and B; one tile per 128 columns n.
bool stream_eligible(const BatchProblem &P);
int64_t stream_tiles(const BatchProblem &P);
tc_status stream_launch_batch(const BatchProblem *dprobs, const int32_t *dtile_prob, int64_t t_begin, int64_t t_end,
                              float alpha, float beta, int nprod, int *dstatus, void *stream);

// Process-wide tuning cache (tc_tuning_cache_save / _load): named integer
// choices per key.
bool tuning_get(const std::string &key, std::map<std::string, int> &out);
void tuning_put(const std::string &key, const std::map<std::string, int> &v);

size_t gett_desc_bytes();
void gett_fill_batch_desc(const BatchProblem &P, int bn, void *out);
// one_stage: every problem's K fits one 32-element stage (the converter
// groups then take alternate tiles).
// split: the (0,0) slice products in their own accumulator (every problem).
tc_status gett_launch_batch(const void *ddescs, const int32_t *dtile_prob, int64_t t_begin, int64_t t_end, int bn,
                            float alpha, float beta, int nprod, int *dstatus, int one_stage, int split,
                            void *stream);
// A general problem (any modes and strides the plan describes, global-load
// inputs, 128 x bn tiles) as one descriptor of the batched tensor-core
// GETT; returns its tile count (-1 if the GETT cannot describe it).
int64_t gett_fill_plan_desc(const Plan &p, int bn, const void *A, const void *B, void *C, int64_t tile0, void *out);

}  // namespace tc

struct tc_plan_s {
    tc::Plan p;
};
