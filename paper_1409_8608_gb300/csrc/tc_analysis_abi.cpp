// C ABI of the cache analysis (Section 3): access distances, prediction
// cases and setup lists, at the paper's or the device's granularity.
#include <cstring>

#include "tc_analysis.h"

using namespace tc;

namespace {

tc_status check(tc_plan plan, int32_t alg_id, int32_t granularity, int64_t elem) {
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    if (alg_id < 1 || alg_id >= (int32_t)plan->p.algs.size())
        return fail(TC_ERROR_INVALID_ALGORITHM, "the analysis covers the loop-nest algorithms (ids >= 1)");
    if (granularity != 0 && granularity != 1) return fail(TC_ERROR_INVALID_ARGUMENT, "granularity is 0 or 1");
    if (elem < 1) return fail(TC_ERROR_INVALID_ARGUMENT, "elem_size must be >= 1");
    return TC_SUCCESS;
}

}  // namespace

extern "C" {

tc_status tc_access_distances(tc_plan plan, int32_t alg_id, int32_t granularity, int64_t elem_size,
                              int64_t *dist) {
    tc_status s = check(plan, alg_id, granularity, elem_size);
    if (s != TC_SUCCESS) return s;
    if (!dist) return fail(TC_ERROR_INVALID_ARGUMENT, "dist is NULL");
    const Plan &p = plan->p;
    NestView v = nest_view(p, p.algs[alg_id], granularity);
    for (int o = 0; o < 3; ++o) dist[o] = access_distance(p, v, o, -1, elem_size);
    return TC_SUCCESS;
}

tc_status tc_prediction_cases(tc_plan plan, int32_t alg_id, int32_t granularity, int64_t elem_size,
                              int64_t cache_size, int64_t line_size, tc_pred_case *out, int32_t capacity,
                              int32_t *count) {
    tc_status s = check(plan, alg_id, granularity, elem_size);
    if (s != TC_SUCCESS) return s;
    if (!count || capacity < 0 || (capacity > 0 && !out) || cache_size < 1 || line_size < 1)
        return fail(TC_ERROR_INVALID_ARGUMENT, "bad output buffer or sizes");
    std::vector<Case> cs = analyse(plan->p, plan->p.algs[alg_id], granularity, elem_size, cache_size, line_size);
    *count = (int32_t)cs.size();
    for (int32_t i = 0; i < capacity && i < *count; ++i) {
        out[i].kind = cs[i].kind;
        out[i].depth = cs[i].depth;
        out[i].count = cs[i].count;
        out[i].omit = cs[i].omit ? 1 : 0;
        out[i].n_items = (int32_t)cs[i].setup.size();
    }
    return TC_SUCCESS;
}

tc_status tc_setup_list(tc_plan plan, int32_t alg_id, int32_t granularity, int32_t case_index,
                        int64_t elem_size, int64_t cache_size, int64_t line_size, tc_setup_item *out,
                        int32_t capacity, int32_t *count) {
    tc_status s = check(plan, alg_id, granularity, elem_size);
    if (s != TC_SUCCESS) return s;
    if (!count || capacity < 0 || (capacity > 0 && !out) || cache_size < 1 || line_size < 1)
        return fail(TC_ERROR_INVALID_ARGUMENT, "bad output buffer or sizes");
    std::vector<Case> cs = analyse(plan->p, plan->p.algs[alg_id], granularity, elem_size, cache_size, line_size);
    if (case_index < 0 || case_index >= (int32_t)cs.size())
        return fail(TC_ERROR_INVALID_ARGUMENT, "case index out of range");
    const auto &list = cs[case_index].setup;
    *count = (int32_t)list.size();
    for (int32_t i = 0; i < capacity && i < *count; ++i) {
        out[i].kind = list[i].kind;
        out[i].operand = list[i].kind == 0 ? list[i].op : -1;
        out[i].size = list[i].size;
    }
    return TC_SUCCESS;
}

}  // extern "C"
