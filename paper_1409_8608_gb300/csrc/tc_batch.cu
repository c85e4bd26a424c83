// Batched form: thousands of independent contractions of one spec with
// their own extents in one persistent launch (no paper counterpart; the
// project's batching addition).
//
// Every problem is a GETT whose free indices of A, free indices of B and
// contracted indices each merge into one strided mode (they appear in the
// same order and are contiguous in the operands that carry them), i.e. a
// strided GEMM  C[m*sCm + n*sCn] = alpha * sum_k A[m*sAm + k*sAk] *
// B[k*sBk + n*sBn] + beta*C.  The problems' tiles are flattened into one
// list ordered by problem size (largest first); the persistent kernel walks
// it with a grid stride and finds each tile's problem in a tile-to-problem
// table built on the host.  Tile shapes (64x64, 32x128, 16x256) hold
// 4096 outputs each and are chosen per problem to waste the fewest padded
// rows ("tuned"), or fixed at 64x64 ("untuned").  The workload is bound by
// HBM (C dominates), so the arithmetic runs on the FP32 / FP64 pipes with
// the same FMA chain as the loop nests.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "tc_internal.h"

namespace tc {

namespace {

constexpr int kBK = 32;  // the whole K of the batched workloads in one round
constexpr int kThreadsB = 256;
constexpr int kShapeM[3] = {64, 32, 16};
constexpr int kShapeN[3] = {64, 128, 256};

template <typename T>
__device__ __forceinline__ T fma_b(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_b<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_b<float>(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T, int TM, int TN>
__device__ __forceinline__ void batch_tile(const BatchProblem &P, int64_t lt, T alpha, T beta, int init,
                                           T (*As)[64], T (*Bs)[256]) {
    constexpr int TX = TM / 4;  // threads along M; TX * (TN / 4) == 256
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int64_t m0 = (lt % P.tiles_m) * TM, n0 = (lt / P.tiles_m) * TN;
    // tile-local 32-bit offsets (the host checked every span fits)
    const int mlim = (int)(P.M - m0 < TM ? P.M - m0 : TM), nlim = (int)(P.N - n0 < TN ? P.N - n0 : TN);
    const int sAm = (int)P.sAm, sAk = (int)P.sAk, sBk = (int)P.sBk, sBn = (int)P.sBn;
    const int sCm = (int)P.sCm, sCn = (int)P.sCn;
    const T *__restrict__ A = (const T *)P.A + m0 * P.sAm;
    const T *__restrict__ B = (const T *)P.B + n0 * P.sBn;
    T *__restrict__ C = (T *)P.C + m0 * P.sCm + n0 * P.sCn;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    if (init != 2) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = tx + i * TX;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = ty + j * (TN / 4);
                if (m < mlim && n < nlim) {
                    T v = C[m * sCm + n * sCn];
                    acc[i][j] = init == 1 ? beta * v : v;
                }
            }
        }
    }
    for (int k0 = 0; k0 < (int)P.K; k0 += kBK) {
        const int kk = (int)P.K - k0 < kBK ? (int)P.K - k0 : kBK;  // K positions in this round
        const bool pow2 = (kk & (kk - 1)) == 0;
        const int ksh = __ffs(kk) - 1;
        const T *Ak = A + k0 * sAk;
        const T *Bk = B + k0 * sBk;
        for (int e = tid; e < TM * kk; e += kThreadsB) {
            const int m = e % TM, k = e / TM;  // TM: compile-time power of two
            T v = T(0);
            if (m < mlim) {
                v = Ak[m * sAm + k * sAk];
                if (alpha != T(1)) v = alpha * v;
            }
            As[k][m] = v;
        }
        for (int e = tid; e < TN * kk; e += kThreadsB) {
            // K fastest across lanes: B is contiguous along K in the workloads
            const int k = pow2 ? (e & (kk - 1)) : e % kk;
            const int n = pow2 ? (e >> ksh) : e / kk;
            Bs[k][n] = n < nlim ? Bk[k * sBk + n * sBn] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kk; ++k) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][tx + i * TX];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][ty + j * (TN / 4)];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma_b<T>(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = tx + i * TX;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = ty + j * (TN / 4);
            if (m < mlim && n < nlim) C[m * sCm + n * sCn] = acc[i][j];
        }
    }
}

// Tiles [t_begin, t_end) of the flattened list, grid-strided.
template <typename T>
__global__ void __launch_bounds__(kThreadsB, 4) batch_kernel(const BatchProblem *__restrict__ probs,
                                                          const int32_t *__restrict__ tile_prob,
                                                          int64_t t_begin, int64_t t_end, T alpha, T beta,
                                                          int init) {
    extern __shared__ __align__(16) unsigned char bsm[];
    T(*As)[64] = (T(*)[64])bsm;
    T(*Bs)[256] = (T(*)[256])(bsm + sizeof(T) * kBK * 64);
    __shared__ BatchProblem P;
    constexpr int kWords = sizeof(BatchProblem) / 8;
    static_assert(sizeof(BatchProblem) % 8 == 0, "problem record in 8-byte words");
    for (int64_t t = t_begin + blockIdx.x; t < t_end; t += gridDim.x) {
        const int q = tile_prob[t];
        if (threadIdx.x < kWords)
            ((int64_t *)&P)[threadIdx.x] = ((const int64_t *)(probs + q))[threadIdx.x];
        __syncthreads();
        const int64_t lt = t - P.tile0;
        if (P.shape == 0) batch_tile<T, 64, 64>(P, lt, alpha, beta, init, As, Bs);
        else if (P.shape == 1) batch_tile<T, 32, 128>(P, lt, alpha, beta, init, As, Bs);
        else batch_tile<T, 16, 256>(P, lt, alpha, beta, init, As, Bs);
        __syncthreads();  // P is rewritten for the next tile
    }
}

int g_bsms = 0;

}  // namespace

struct BatchImpl {
    std::string spec;
    tc_dtype dtype = TC_F32;
    int count = 0;
    std::vector<BatchProblem> probs;  // problem order: largest first
    std::vector<int> order;           // caller index of each slot
    int64_t total_tiles = 0;
    int policy = 1;                   // 1: shape per problem, 0: fixed 64x64
    BatchProblem *dprobs = nullptr;
    int32_t *dtile_prob = nullptr;    // problem slot of every tile
    int64_t dtile_cap = 0;
    // split-BF16 (tensor-core GETT tiles of 128 x bn)
    int bn = 128;
    int nprod = 6;
    void *ddescs = nullptr;           // one kernel descriptor per problem slot
    int *dstatus = nullptr;           // bounded-wait status word
    void *last_stream = nullptr;
    bool dirty = true;
    int device = -1;
    double flops = 0;
};

namespace {

// merged strided modes of one problem; false when a mode group does not merge
bool merge_group(const Layout &L1, const Layout &L2, const std::vector<int> &ids, const int64_t *ext,
                 int64_t &e, int64_t &s1, int64_t &s2) {
    // the group's modes must appear consecutively and in the same order in
    // both operands, each stride chaining onto the previous
    e = 1;
    s1 = s2 = 0;
    if (ids.empty()) return true;
    auto order_in = [&](const Layout &L) {
        std::vector<int> o;
        for (int m = 0; m < L.n; ++m)
            if (std::find(ids.begin(), ids.end(), L.idx[m]) != ids.end()) o.push_back(L.idx[m]);
        return o;
    };
    std::vector<int> o1 = order_in(L1), o2 = order_in(L2);
    if (o1 != o2) return false;
    for (const Layout *L : {&L1, &L2}) {
        int64_t expect = -1;
        for (size_t x = 0; x < o1.size(); ++x) {
            int64_t st = L->stride_of(o1[x]);
            if (x > 0 && st != expect) return false;
            expect = st * ext[o1[x]];
        }
    }
    for (int id : o1) e *= ext[id];
    s1 = L1.stride_of(o1[0]);
    s2 = L2.stride_of(o1[0]);
    return true;
}

int shape_for(int64_t M, int policy) {
    if (policy == 0) return 0;
    if (M <= 16) return 2;
    if (M <= 32) return 1;
    return 0;
}

void assign_tiles(BatchImpl &b) {
    int64_t t = 0;
    if (b.dtype == TC_BF16X3) {
        // 128 x bn tensor-core tiles, one width for the launch: per problem
        // (policy 1) the width with the fewest padded columns plus a fixed
        // per-tile cost of 64 columns, or 256 (policy 0)
        int bn = 256;
        if (b.policy == 1) {
            double best = 0;
            for (int w : {128, 256}) {
                double cost = 0;
                for (const auto &P : b.probs) cost += (double)((P.N + w - 1) / w) * (w + 64);
                if (w == 128 || cost < best) {
                    best = cost;
                    bn = w;
                }
            }
        }
        b.bn = bn;
        for (auto &P : b.probs) {
            P.shape = 0;
            P.tiles_m = (int32_t)((P.M + 127) / 128);
            P.tile0 = t;
            t += (int64_t)P.tiles_m * ((P.N + bn - 1) / bn);
        }
        b.total_tiles = t;
        b.dirty = true;
        return;
    }
    for (auto &P : b.probs) {
        P.shape = shape_for(P.M, b.policy);
        const int tm = kShapeM[P.shape], tn = kShapeN[P.shape];
        P.tiles_m = (int32_t)((P.M + tm - 1) / tm);
        P.tile0 = t;
        t += (int64_t)P.tiles_m * ((P.N + tn - 1) / tn);
    }
    b.total_tiles = t;
    b.dirty = true;
}

}  // namespace
}  // namespace tc

using namespace tc;

struct tc_batch_s {
    BatchImpl b;
};

extern "C" {

tc_status tc_batch_create(tc_batch *out, const char *spec, int32_t count, const int64_t *extents,
                          tc_dtype dtype) {
    if (!out) return fail(TC_ERROR_INVALID_ARGUMENT, "out is NULL");
    *out = nullptr;
    if (!spec || !extents || count < 1) return fail(TC_ERROR_INVALID_ARGUMENT, "bad batch arguments");
    if (dtype != TC_F32 && dtype != TC_F64 && dtype != TC_BF16X3)
        return fail(TC_ERROR_UNSUPPORTED_DTYPE, "the batched form runs in FP32, FP64 or split-BF16");
    tc_batch_s *h = new (std::nothrow) tc_batch_s();
    if (!h) return fail(TC_ERROR_OUT_OF_MEMORY, "host allocation failed");
    BatchImpl &b = h->b;
    b.spec = spec;
    b.dtype = dtype;
    b.count = count;
    // classify once (the classes do not depend on the extents)
    tc_plan plan = nullptr;
    tc_status s = tc_plan_create(&plan, spec, extents, nullptr, dtype == TC_BF16X3 ? TC_F32 : dtype);
    if (s != TC_SUCCESS) {
        delete h;
        return s;
    }
    const int nidx = plan->p.nidx;
    std::vector<BatchProblem> probs(count);
    std::vector<int64_t> work(count);
    for (int32_t q = 0; q < count; ++q) {
        const int64_t *e = extents + (int64_t)q * nidx;
        for (int x = 0; x < nidx; ++x)
            if (e[x] < 1) {
                tc_plan_destroy(plan);
                delete h;
                return fail(TC_ERROR_INVALID_EXTENT, "extent < 1 in problem " + std::to_string(q));
            }
        // dense strides for this problem's extents
        Layout L[3];
        for (int o = 0; o < 3; ++o) {
            L[o] = plan->p.op[o];
            int64_t st = 1;
            for (int m = 0; m < L[o].n; ++m) {
                L[o].stride[m] = st;
                st *= e[L[o].idx[m]];
            }
        }
        BatchProblem &P = probs[q];
        std::memset(&P, 0, sizeof(P));
        int64_t dummy;
        bool ok = merge_group(L[OP_A], L[OP_C], plan->p.freeA, e, P.M, P.sAm, P.sCm) &&
                  merge_group(L[OP_B], L[OP_C], plan->p.freeB, e, P.N, P.sBn, P.sCn) &&
                  merge_group(L[OP_A], L[OP_B], plan->p.contracted, e, P.K, P.sAk, P.sBk);
        (void)dummy;
        if (!ok) {
            tc_plan_destroy(plan);
            delete h;
            return fail(TC_ERROR_INVALID_SPEC,
                        "batched form needs the free indices of A, of B and the contracted indices to merge "
                        "into single strided modes");
        }
        // tile-local offsets are 32-bit: every operand's span must fit
        const int64_t spanA = (P.M - 1) * P.sAm + (P.K - 1) * P.sAk, spanB = (P.K - 1) * P.sBk + (P.N - 1) * P.sBn;
        const int64_t spanC = (P.M - 1) * P.sCm + (P.N - 1) * P.sCn;
        if (std::max(spanA, std::max(spanB, spanC)) >= ((int64_t)1 << 31) || P.K >= ((int64_t)1 << 31)) {
            tc_plan_destroy(plan);
            delete h;
            return fail(TC_ERROR_INVALID_EXTENT, "batched problem " + std::to_string(q) + " spans 2^31 elements or more");
        }
        work[q] = P.M * P.N * P.K;
        b.flops += 2.0 * (double)P.M * (double)P.N * (double)P.K;
    }
    tc_plan_destroy(plan);
    b.order.resize(count);
    std::iota(b.order.begin(), b.order.end(), 0);
    std::stable_sort(b.order.begin(), b.order.end(), [&](int x, int y) { return work[x] > work[y]; });
    b.probs.resize(count);
    for (int32_t slot = 0; slot < count; ++slot) b.probs[slot] = probs[b.order[slot]];
    assign_tiles(b);
    *out = h;
    return TC_SUCCESS;
}

tc_status tc_batch_destroy(tc_batch batch) {
    if (!batch) return TC_SUCCESS;
    if (batch->b.dprobs) cudaFree(batch->b.dprobs);
    if (batch->b.dtile_prob) cudaFree(batch->b.dtile_prob);
    if (batch->b.ddescs) cudaFree(batch->b.ddescs);
    if (batch->b.dstatus) cudaFree(batch->b.dstatus);
    delete batch;
    return TC_SUCCESS;
}

tc_status tc_batch_set_tiles(tc_batch batch, int32_t policy) {
    if (!batch) return fail(TC_ERROR_INVALID_ARGUMENT, "batch is NULL");
    if (policy != 0 && policy != 1) return fail(TC_ERROR_INVALID_ARGUMENT, "policy is 0 (fixed) or 1 (per problem)");
    batch->b.policy = policy;
    assign_tiles(batch->b);
    return TC_SUCCESS;
}

tc_status tc_batch_set_operands(tc_batch batch, void *const *A, void *const *B, void *const *C) {
    if (!batch || !A || !B || !C) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    BatchImpl &b = batch->b;
    for (int slot = 0; slot < b.count; ++slot) {
        const int q = b.order[slot];
        if (!A[q] || !B[q] || !C[q]) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL operand pointer");
        b.probs[slot].A = A[q];
        b.probs[slot].B = B[q];
        b.probs[slot].C = C[q];
    }
    b.dirty = true;
    return TC_SUCCESS;
}

tc_status tc_batch_prepare(tc_batch batch) {
    if (!batch) return fail(TC_ERROR_INVALID_ARGUMENT, "batch is NULL");
    BatchImpl &b = batch->b;
    for (const auto &P : b.probs)
        if (!P.A) return fail(TC_ERROR_INVALID_ARGUMENT, "call tc_batch_set_operands first");
    int dev = 0;
    cudaGetDevice(&dev);
    if (b.device >= 0 && b.device != dev) return fail(TC_ERROR_INVALID_ARGUMENT, "batch used on another device");
    b.device = dev;
    if (!b.dprobs) {
        cudaError_t e = cudaMalloc(&b.dprobs, sizeof(BatchProblem) * b.count);
        if (e != cudaSuccess) {
            b.dprobs = nullptr;
            return fail(TC_ERROR_OUT_OF_MEMORY, cudaGetErrorString(e));
        }
        b.dirty = true;
    }
    if (b.total_tiles > b.dtile_cap) {
        if (b.dtile_prob) cudaFree(b.dtile_prob);
        b.dtile_prob = nullptr;
        b.dtile_cap = 0;
        cudaError_t e = cudaMalloc(&b.dtile_prob, sizeof(int32_t) * b.total_tiles);
        if (e != cudaSuccess) {
            b.dtile_prob = nullptr;
            return fail(TC_ERROR_OUT_OF_MEMORY, cudaGetErrorString(e));
        }
        b.dtile_cap = b.total_tiles;
        b.dirty = true;
    }
    if (b.dtype == TC_BF16X3 && (!b.ddescs || !b.dstatus)) {
        cudaError_t e = cudaSuccess;
        if (!b.ddescs) e = cudaMalloc(&b.ddescs, gett_desc_bytes() * b.count);
        if (e == cudaSuccess && !b.dstatus) e = cudaMalloc(&b.dstatus, 16);
        if (e == cudaSuccess) e = cudaMemset(b.dstatus, 0, 16);
        if (e != cudaSuccess) return fail(TC_ERROR_OUT_OF_MEMORY, cudaGetErrorString(e));
        b.dirty = true;
    }
    if (b.dirty) {
        cudaError_t e = cudaMemcpy(b.dprobs, b.probs.data(), sizeof(BatchProblem) * b.count, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
        if (b.dtype == TC_BF16X3) {
            const size_t db = gett_desc_bytes();
            std::vector<unsigned char> hd(db * b.count);
            for (int slot = 0; slot < b.count; ++slot) gett_fill_batch_desc(b.probs[slot], b.bn, hd.data() + db * slot);
            e = cudaMemcpy(b.ddescs, hd.data(), hd.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
        }
        std::vector<int32_t> tp(b.total_tiles);
        for (int slot = 0; slot < b.count; ++slot) {
            const int64_t t1 = slot + 1 < b.count ? b.probs[slot + 1].tile0 : b.total_tiles;
            for (int64_t t = b.probs[slot].tile0; t < t1; ++t) tp[t] = slot;
        }
        e = cudaMemcpy(b.dtile_prob, tp.data(), sizeof(int32_t) * b.total_tiles, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
        b.dirty = false;
    }
    return TC_SUCCESS;
}

tc_status tc_batch_execute(tc_batch batch, const void *alpha, const void *beta, int32_t one_launch_per_problem,
                           void *stream) {
    if (!batch || !alpha || !beta) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    BatchImpl &b = batch->b;
    if (b.dirty || !b.dprobs) {
        tc_status s = tc_batch_prepare(batch);
        if (s != TC_SUCCESS) return s;
    }
    if (g_bsms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_bsms, cudaDevAttrMultiProcessorCount, dev);
        if (g_bsms <= 0) g_bsms = 1;
    }
    cudaStream_t st = (cudaStream_t)stream;
    b.last_stream = stream;
    if (b.dtype == TC_BF16X3) {
        const float a = *(const float *)alpha, be = *(const float *)beta;
        int one_stage = 1;
        for (const auto &P : b.probs)
            if (P.K > 32) one_stage = 0;
        auto run = [&](int64_t t0, int64_t t1) {
            return gett_launch_batch(b.ddescs, b.dtile_prob, t0, t1, b.bn, a, be, b.nprod, b.dstatus, one_stage, 0,
                                     stream);
        };
        if (one_launch_per_problem) {
            for (int slot = 0; slot < b.count; ++slot) {
                const int64_t t0 = b.probs[slot].tile0;
                const int64_t t1 = slot + 1 < b.count ? b.probs[slot + 1].tile0 : b.total_tiles;
                tc_status s = run(t0, t1);
                if (s != TC_SUCCESS) return s;
            }
            return TC_SUCCESS;
        }
        return run(0, b.total_tiles);
    }
    // persistent grid: exactly the CTAs that fit at once
    int per_sm = 1;
    if (b.dtype == TC_F64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<double>, kThreadsB,
                                                      (int)(sizeof(double) * kBK * (64 + 256)));
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<float>, kThreadsB,
                                                      (int)(sizeof(float) * kBK * (64 + 256)));
    const int64_t resident = (int64_t)g_bsms * std::max(1, per_sm);
    const int smem_f = (int)(sizeof(float) * kBK * (64 + 256)), smem_d = (int)(sizeof(double) * kBK * (64 + 256));
    cudaFuncSetAttribute(batch_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_d);
    cudaFuncSetAttribute(batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_f);
    auto launch = [&](int64_t t0, int64_t t1) {
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(t1 - t0, resident));
        if (b.dtype == TC_F64) {
            const double a = *(const double *)alpha, be = *(const double *)beta;
            batch_kernel<double><<<(unsigned)grid, kThreadsB, smem_d, st>>>(b.dprobs, b.dtile_prob, t0, t1, a, be,
                                                                       be == 0.0 ? 2 : (be == 1.0 ? 0 : 1));
        } else {
            const float a = *(const float *)alpha, be = *(const float *)beta;
            batch_kernel<float><<<(unsigned)grid, kThreadsB, smem_f, st>>>(b.dprobs, b.dtile_prob, t0, t1, a, be,
                                                                      be == 0.0f ? 2 : (be == 1.0f ? 0 : 1));
        }
    };
    if (one_launch_per_problem) {
        for (int slot = 0; slot < b.count; ++slot) {
            const int64_t t0 = b.probs[slot].tile0;
            const int64_t t1 = slot + 1 < b.count ? b.probs[slot + 1].tile0 : b.total_tiles;
            launch(t0, t1);
        }
    } else {
        launch(0, b.total_tiles);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TC_SUCCESS : fail(TC_ERROR_CUDA, cudaGetErrorString(e));
}

tc_status tc_batch_info(tc_batch batch, double *flops, int64_t *tiles, int64_t *bytes) {
    if (!batch) return fail(TC_ERROR_INVALID_ARGUMENT, "batch is NULL");
    const BatchImpl &b = batch->b;
    if (flops) *flops = b.flops;
    if (tiles) *tiles = b.total_tiles;
    if (bytes) {
        const int64_t es = b.dtype == TC_F64 ? 8 : 4;  // split-BF16: FP32 I/O
        int64_t t = 0;
        for (const auto &P : b.probs) t += (P.M * P.K + P.K * P.N + P.M * P.N) * es;
        *bytes = t;
    }
    return TC_SUCCESS;
}

tc_status tc_batch_device_status(tc_batch batch) {
    if (!batch) return fail(TC_ERROR_INVALID_ARGUMENT, "batch is NULL");
    BatchImpl &b = batch->b;
    if (!b.dstatus) return TC_SUCCESS;
    int v = 0;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)b.last_stream);
    if (e == cudaSuccess) e = cudaMemcpy(&v, b.dstatus, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v != 0) e = cudaMemset(b.dstatus, 0, sizeof(int));
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    if (v != 0) return fail((tc_status)v, "a bounded wait in the batched kernel ran out");
    return TC_SUCCESS;
}

}  // extern "C"
