// Cache analysis of Section 3 (host, integer); see tc_analysis.cpp.
#pragma once

#include <cstdint>
#include <vector>

#include "tc_internal.h"

namespace tc {

enum CaseKind { CASE_STEADY = 0, CASE_MISS = 1, CASE_FIRST = 2 };

struct NestView {
    std::vector<int> loops;    // index ids of the analysed loops, outermost first
    std::vector<bool> kernel;  // per index id: a mode of the kernel's operand slices
};

struct SetupItem {
    int kind;     // 0: touch an operand slice, 1: remote region
    int op;       // OP_A, OP_B, OP_C (kind 0)
    int64_t size; // bytes (or elements when elem == 1)
};

struct Case {
    int kind;     // CaseKind
    int depth;    // loop of a first-iteration case, else -1
    int64_t count;
    bool omit;    // setup touches operands only: it can be left out
    std::vector<SetupItem> setup;
};

// granularity 0: the paper's loop nest around one BLAS call;
// granularity 1: the device phases around one phase launch
NestView nest_view(const Plan &p, const Algorithm &alg, int granularity);
int64_t region_elems(const Plan &p, const NestView &v, int op, const std::vector<bool> &joined);
int64_t access_distance(const Plan &p, const NestView &v, int op, int start_depth, int64_t elem);
int prefetch_kind(const Plan &p, const NestView &v, int op, int64_t line_elems);
std::vector<Case> analyse(const Plan &p, const Algorithm &alg, int granularity, int64_t elem,
                          int64_t cache_bytes, int64_t line_bytes);

}  // namespace tc
