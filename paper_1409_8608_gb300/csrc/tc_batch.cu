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
// table built on the host.
//
// FP32 / FP64 (SIMT FMA): every tile holds 4096 outputs, (8 << s) x
// (512 >> s) for s = 0..4, and a problem's K runs in chunks of bk (8, 16 or
// 32).  A block's sequence of (tile, K chunk) stages is software-pipelined:
// cp.async copies of stage s+1 (16-byte pieces where the layout allows)
// overlap the FMAs of stage s.  Each thread owns 4 rows x 4 columns; A is
// staged k-major and B n-major with a pitch that keeps the 16-byte reads of
// both conflict-free.  Where a tile's C is one contiguous run (one column
// tile covers M, C dense along m) the epilogue stages it in shared memory
// and writes it with aligned 16-byte stores.  The tile shape and K chunk
// are chosen per problem: fixed (64 x 64, bk 16), by rule (the smallest
// tile height that covers M), or by the autotuner, which times every
// candidate on each shape class's problems (tc_batch_autotune).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "tc_internal.h"

namespace tc {

namespace {

constexpr int kThreadsB = 256;
constexpr int kShapes = 5;           // tiles (8 << s) x (512 >> s)
constexpr int kStageElems = 6400;    // one stage: A chunk (bk x TM) + B chunk (TN x pitch)
constexpr int kOutElems = 4096 + 4;  // staged epilogue (in a stage buffer) + 16-byte alignment shift

// n-major B pitch for a K chunk of kk: a multiple of 4 elements whose
// quarter is odd, so that 16-byte reads at rows ty, ty+1, ... fall in
// distinct bank groups
__host__ __device__ __forceinline__ int b_pitch(int kk) { return 4 * (((kk + 3) >> 2) | 1); }

__host__ __device__ constexpr int shape_rows(int s) { return 8 << s; }
__host__ __device__ constexpr int shape_cols(int s) { return 512 >> s; }

bool stage_fits(int s, int bk) { return bk * shape_rows(s) + shape_cols(s) * b_pitch(bk) <= kStageElems; }

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src) {
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T>
__device__ __forceinline__ T fma_b(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_b<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_b<float>(float a, float b, float c) { return fmaf(a, b, c); }

// four consecutive elements from shared memory (16-byte aligned)
template <typename T>
__device__ __forceinline__ void lds4(const T *p, T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 x = *(const float4 *)p;
        v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
    } else {
        const double2 x = *(const double2 *)p, y = *(const double2 *)(p + 2);
        v[0] = x.x, v[1] = x.y, v[2] = y.x, v[3] = y.y;
    }
}

// Geometry of one pipeline stage, worked out once by the producer and read
// by every thread from shared memory.
struct StageMeta {
    int q;                  // problem slot
    int chunk;              // K chunk of the tile
    int m0, n0, mlim, nlim; // tile origin and valid rows / columns
    int kk;                 // K positions in this chunk
    int last;               // the tile's last chunk
};

// Fills the stage record for tile lt of problem P, K chunk `chunk`.
__device__ __forceinline__ void stage_meta(const BatchProblem *__restrict__ P, int q, int lt, int chunk,
                                           StageMeta &m) {
    const int shape = P->shape, tm = P->tiles_m, bk = P->bk;
    const int mt = tm == 1 ? 0 : lt % tm, nt = tm == 1 ? lt : lt / tm;
    m.q = q;
    m.chunk = chunk;
    m.m0 = mt * shape_rows(shape);
    m.n0 = nt * shape_cols(shape);
    m.mlim = (int)min((int64_t)shape_rows(shape), P->M - m.m0);
    m.nlim = (int)min((int64_t)shape_cols(shape), P->N - m.n0);
    const int64_t rest = P->K - (int64_t)chunk * bk;
    m.kk = (int)min((int64_t)bk, rest);
    m.last = rest <= bk;
}

// Issues the copies of one stage into S: A as [k][m] (pitch TM), B as
// [n][k] (pitch b_pitch(kk)); the K padding up to a multiple of 4 is zeroed
// in both.  Rows past M and columns past N are left as they are: they only
// reach outputs that are never stored.
template <typename T>
__device__ __forceinline__ void batch_produce(T *S, const BatchProblem *__restrict__ P, const StageMeta &g) {
    constexpr int V = 16 / sizeof(T), lgV = sizeof(T) == 4 ? 2 : 1;
    const int shape = P->shape, TM = shape_rows(shape), lgTM = 3 + shape;
    const int bk = P->bk, flags = P->flags;
    const int kk = g.kk, kk4 = (kk + 3) & ~3, KP = b_pitch(kk), mlim = g.mlim, nlim = g.nlim;
    // tile-local offsets are 32-bit (the host checked every span fits)
    const int sAm = (int)P->sAm, sAk = (int)P->sAk, sBk = (int)P->sBk, sBn = (int)P->sBn;
    const int64_t k0 = (int64_t)g.chunk * bk;
    const T *A = (const T *)P->A + g.m0 * P->sAm + k0 * P->sAk;
    const T *B = (const T *)P->B + g.n0 * P->sBn + k0 * P->sBk;
    T *As = S, *Bs = S + bk * TM;
    if (flags & kBatchVecA) {  // sAm == 1: 16-byte pieces of V rows
        const int lgp = lgTM - lgV, units = kk << lgp;
        for (int u = threadIdx.x; u < units; u += kThreadsB) {
            const int k = u >> lgp, m = (u & ((1 << lgp) - 1)) * V;
            T *dst = As + k * TM + m;
            const T *src = A + m + k * sAk;
            if (m + V <= mlim)
                cp_async16(dst, src);
            else
                for (int x = 0; x < V && m + x < mlim; ++x) cp_async_elem(dst + x, src + x);
        }
    } else {
        for (int e = threadIdx.x; e < kk * TM; e += kThreadsB) {
            const int m = e & (TM - 1), k = e >> lgTM;
            if (m < mlim) cp_async_elem(As + e, A + m * sAm + k * sAk);
        }
    }
    if (flags & kBatchVecB) {  // sBk == 1, kk % V == 0: 16-byte pieces along k
        const int ku = kk / V, units = nlim * ku;
        if ((ku & (ku - 1)) == 0) {
            const int lg = __ffs(ku) - 1;
            for (int u = threadIdx.x; u < units; u += kThreadsB) {
                const int n = u >> lg, kq = u & (ku - 1);
                cp_async16(Bs + n * KP + kq * V, B + n * sBn + kq * V);
            }
        } else {
            for (int u = threadIdx.x; u < units; u += kThreadsB) {
                const int n = u / ku, kq = u - n * ku;
                cp_async16(Bs + n * KP + kq * V, B + n * sBn + kq * V);
            }
        }
    } else {
        for (int e = threadIdx.x; e < nlim * kk; e += kThreadsB) {
            const int n = e / kk, k = e - n * kk;
            cp_async_elem(Bs + n * KP + k, B + n * sBn + k * sBk);
        }
    }
    if (kk4 != kk) {  // zero K padding: 0 * (anything finite) would not be enough
        const int pad = kk4 - kk;
        for (int e = threadIdx.x; e < pad * TM; e += kThreadsB) As[kk * TM + e] = T(0);
        for (int e = threadIdx.x; e < pad * nlim; e += kThreadsB) {
            const int n = e / pad;
            Bs[n * KP + kk + (e - n * pad)] = T(0);
        }
    }
    (void)lgV;
}

// FMAs of one staged K chunk: thread (tx, ty) owns rows 4tx..4tx+3 and
// columns ty + j*TY, j = 0..3; K runs in increasing order.
template <typename T, int SHAPE>
__device__ __forceinline__ void batch_compute(const T *S, int bk, int kk4, int KP, T (&acc)[4][4]) {
    constexpr int TM = shape_rows(SHAPE), TX = TM / 4, TY = kThreadsB / TX;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const T *As = S + 4 * tx;
    const T *Bs = S + bk * TM + ty * KP;
    for (int k4 = 0; k4 < kk4; k4 += 4) {
        T b[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) lds4(Bs + j * TY * KP + k4, b[j]);
#pragma unroll
        for (int kq = 0; kq < 4; ++kq) {
            T a[4];
            lds4(As + (k4 + kq) * TM, a);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma_b<T>(a[i], b[j][kq], acc[i][j]);
        }
    }
}

template <typename T>
__device__ __forceinline__ T blend(T acc, T alpha, T beta, int init, const T *c) {
    return init == 2 ? alpha * acc : fma_b<T>(beta, *c, alpha * acc);
}

// C = alpha * acc (+ beta * C) for one tile.  Cs: the stage buffer just
// consumed (free once every thread has passed the barrier below).
template <typename T, int SHAPE>
__device__ __forceinline__ void batch_epilogue(const BatchProblem *__restrict__ P, const StageMeta &g,
                                               T (&acc)[4][4], T alpha, T beta, int init, T *Cs) {
    constexpr int TM = shape_rows(SHAPE), TX = TM / 4, TY = kThreadsB / TX;
    constexpr int V = 16 / sizeof(T);
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int mlim = g.mlim, nlim = g.nlim;
    T *C = (T *)P->C;
    if (P->flags & kBatchStagedC) {
        // the tile's C is nlim * M contiguous elements from C + n0 * M
        const int M = mlim;
        T *Cg = C + (int64_t)g.n0 * M;
        const int shift = (int)(((uintptr_t)Cg / sizeof(T)) & (V - 1));
        __syncthreads();  // every thread is done reading the stage
        T *cs = Cs + shift + 4 * tx;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = ty + j * TY;
            if (n < nlim) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (4 * tx + i < M) cs[n * M + i] = acc[i][j];
            }
        }
        __syncthreads();
        const int total = nlim * M + shift;
        T *Ca = Cg - shift;  // 16-byte aligned
        for (int u = threadIdx.x * V; u < total; u += kThreadsB * V) {
            if (u >= shift && u + V <= total) {
                if constexpr (sizeof(T) == 4) {
                    float4 v = *(const float4 *)(Cs + u);
                    if (init == 2) {
                        v.x *= alpha, v.y *= alpha, v.z *= alpha, v.w *= alpha;
                    } else {
                        const float4 o = *(const float4 *)(Ca + u);
                        v.x = fmaf(beta, o.x, alpha * v.x), v.y = fmaf(beta, o.y, alpha * v.y);
                        v.z = fmaf(beta, o.z, alpha * v.z), v.w = fmaf(beta, o.w, alpha * v.w);
                    }
                    *(float4 *)(Ca + u) = v;
                } else {
                    double2 v = *(const double2 *)(Cs + u);
                    if (init == 2) {
                        v.x *= alpha, v.y *= alpha;
                    } else {
                        const double2 o = *(const double2 *)(Ca + u);
                        v.x = fma(beta, o.x, alpha * v.x), v.y = fma(beta, o.y, alpha * v.y);
                    }
                    *(double2 *)(Ca + u) = v;
                }
            } else {
                for (int x = 0; x < V; ++x) {
                    const int s = u + x;
                    if (s >= shift && s < total) Ca[s] = blend<T>(Cs[s], alpha, beta, init, Ca + s);
                }
            }
        }
        return;
    }
    const int sCm = (int)P->sCm, sCn = (int)P->sCn;
    T *Ct = C + g.m0 * P->sCm + g.n0 * P->sCn;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = 4 * tx + i, n = ty + j * TY;
            if (m < mlim && n < nlim) {
                T *c = Ct + m * sCm + n * sCn;
                *c = blend<T>(acc[i][j], alpha, beta, init, c);
            }
        }
}

// Tiles [t_begin, t_end) of the flattened list (fewer than 2^31 tiles),
// grid-strided; each block runs its tiles' K chunks as one pipelined
// sequence of stages.
template <typename T, int STAGES>
__global__ void __launch_bounds__(kThreadsB) batch_kernel(const BatchProblem *__restrict__ probs,
                                                          const int32_t *__restrict__ tile_prob,
                                                          int64_t t_begin, int64_t t_end, T alpha, T beta,
                                                          int init) {
    static_assert(kOutElems <= kStageElems, "the staged epilogue reuses a stage buffer");
    extern __shared__ __align__(16) unsigned char bsm[];
    T *stages = (T *)bsm;
    __shared__ StageMeta meta[STAGES];
    int64_t pt = t_begin + blockIdx.x;  // producer cursor: tile and K chunk
    int pc = 0;
    auto produce = [&](int slot) {
        if (pt >= t_end) return;
        const int q = tile_prob[pt];
        const BatchProblem *__restrict__ P = probs + q;
        StageMeta g;
        stage_meta(P, q, (int)(pt - P->tile0), pc, g);
        batch_produce<T>(stages + slot * kStageElems, P, g);
        if (threadIdx.x == 0) meta[slot] = g;
        if (g.last) {
            pc = 0;
            pt += gridDim.x;
        } else {
            ++pc;
        }
    };
#pragma unroll
    for (int p = 0; p < STAGES - 1; ++p) {
        produce(p);
        cp_async_commit();
    }
    T acc[4][4];
    int s = 0;
    for (int64_t ct = t_begin + blockIdx.x; ct < t_end; ++s) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();  // stage s landed for every thread; stage s-1's buffer is free
        produce((s + STAGES - 1) % STAGES);
        cp_async_commit();
        const int slot = s % STAGES;
        const StageMeta g = meta[slot];
        const BatchProblem *__restrict__ P = probs + g.q;
        const int shape = P->shape, bk = P->bk;
        const int kk4 = (g.kk + 3) & ~3, KP = b_pitch(g.kk);
        if (g.chunk == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
        }
        T *S = stages + slot * kStageElems;
        switch (shape) {
            case 0: batch_compute<T, 0>(S, bk, kk4, KP, acc); break;
            case 1: batch_compute<T, 1>(S, bk, kk4, KP, acc); break;
            case 2: batch_compute<T, 2>(S, bk, kk4, KP, acc); break;
            case 3: batch_compute<T, 3>(S, bk, kk4, KP, acc); break;
            default: batch_compute<T, 4>(S, bk, kk4, KP, acc); break;
        }
        if (g.last) {
            switch (shape) {
                case 0: batch_epilogue<T, 0>(P, g, acc, alpha, beta, init, S); break;
                case 1: batch_epilogue<T, 1>(P, g, acc, alpha, beta, init, S); break;
                case 2: batch_epilogue<T, 2>(P, g, acc, alpha, beta, init, S); break;
                case 3: batch_epilogue<T, 3>(P, g, acc, alpha, beta, init, S); break;
                default: batch_epilogue<T, 4>(P, g, acc, alpha, beta, init, S); break;
            }
            ct += gridDim.x;
        }
    }
    cp_async_wait<0>();
}

template <typename T, int STAGES>
constexpr int batch_smem() {
    return (int)(sizeof(T) * STAGES * kStageElems);
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
    int policy = 1;                   // 0 fixed, 1 rule, 2 autotuned
    BatchProblem *dprobs = nullptr;
    int32_t *dtile_prob = nullptr;    // problem slot of every tile
    int64_t dtile_cap = 0;
    // SIMT: pipeline stages of the launch, and the autotuner's choice per
    // shape class (tile shape, K chunk)
    int stages = 2;
    int tuned_stages = 2;
    std::map<std::tuple<int, int, int>, std::pair<int, int>> tuned;
    bool has_tuning = false;
    // split-BF16: the stream kernel (one tile per 128 columns) or the
    // tensor-core GETT tiles of 128 x bn
    int bf_stream = 0;
    int bn = 128;
    int tuned_bn = 0;
    int tuned_stream = 0;
    bool stream_layout = false;  // every problem's strides, M and K suit the stream kernel
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

int ceil_log2(int64_t x) {
    int l = 0;
    while (((int64_t)1 << l) < x) ++l;
    return l;
}

// shape class of a problem: ceil(log2 M), ceil(log2 K) and an N bucket
std::tuple<int, int, int> class_of(const BatchProblem &P) {
    return {std::min(ceil_log2(P.M), 8), std::min(ceil_log2(P.K), 7), P.N <= 256 ? 0 : (P.N <= 2048 ? 1 : 2)};
}

// K chunks that differ for K up to kmax: 8 always, 16 and 32 only where
// they cut the number of chunks
bool chunk_useful(int bk, int64_t kmax) { return bk == 8 || kmax > bk / 2; }

// rule: the smallest tile height that covers M, the largest K chunk
std::pair<int, int> rule_choice(int64_t M, int64_t kmax) {
    const int s = std::max(0, std::min(kShapes - 1, ceil_log2(M) - 3));
    int bk = 32;
    while (bk > 8 && (!stage_fits(s, bk) || !chunk_useful(bk, kmax))) bk /= 2;
    return {s, bk};
}

std::pair<int, int> fixed_choice(int64_t kmax) { return {3, chunk_useful(16, kmax) ? 16 : 8}; }

void set_tiles_of(BatchProblem &P, int shape, int bk, int64_t &t) {
    P.shape = shape;
    P.bk = bk;
    P.tiles_m = (int32_t)((P.M + shape_rows(shape) - 1) / shape_rows(shape));
    P.tile0 = t;
    t += (int64_t)P.tiles_m * ((P.N + shape_cols(shape) - 1) / shape_cols(shape));
}

// copy paths that the problem's strides and pointers allow
int32_t flags_for(const BatchProblem &P, size_t esz) {
    const int64_t V = 16 / (int64_t)esz;
    int32_t f = 0;
    if (P.sAm == 1 && P.sAk % V == 0 && ((uintptr_t)P.A & 15) == 0) f |= kBatchVecA;
    if (P.sBk == 1 && P.sBn % V == 0 && P.K % V == 0 && ((uintptr_t)P.B & 15) == 0) f |= kBatchVecB;
    if (P.sCm == 1 && P.sCn == P.M && P.tiles_m == 1) f |= kBatchStagedC;
    return f;
}

void assign_tiles(BatchImpl &b) {
    int64_t t = 0;
    if (b.dtype == TC_BF16X3) {
        // the stream kernel (rule, where every problem suits it), or
        // 128 x bn tensor-core GETT tiles with one width for the launch: the
        // width with the fewest padded columns plus a fixed per-tile cost of
        // 64 columns (rule otherwise), 256 (fixed); or the autotuner's choice
        b.bf_stream = b.policy == 2 ? b.tuned_stream : (b.policy == 1 && b.stream_layout);
        if (b.bf_stream) {
            for (auto &P : b.probs) {
                P.shape = 0;
                P.bk = 32;
                P.tiles_m = 1;
                P.tile0 = t;
                t += stream_tiles(P);
            }
            b.total_tiles = t;
            b.dirty = true;
            return;
        }
        int bn = 256;
        if (b.policy == 2) {
            bn = b.tuned_bn;
        } else if (b.policy == 1) {
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
            P.bk = 32;
            P.tiles_m = (int32_t)((P.M + 127) / 128);
            P.tile0 = t;
            t += (int64_t)P.tiles_m * ((P.N + bn - 1) / bn);
        }
        b.total_tiles = t;
        b.dirty = true;
        return;
    }
    b.stages = b.policy == 2 ? b.tuned_stages : 2;
    for (auto &P : b.probs) {
        std::pair<int, int> c;
        if (b.policy == 0) {
            c = fixed_choice(P.K);
        } else if (b.policy == 1) {
            c = rule_choice(P.M, P.K);
        } else {
            auto it = b.tuned.find(class_of(P));
            c = it != b.tuned.end() ? it->second : rule_choice(P.M, P.K);
        }
        set_tiles_of(P, c.first, c.second, t);
    }
    b.total_tiles = t;
    b.dirty = true;
}

int sm_count() {
    if (g_bsms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_bsms, cudaDevAttrMultiProcessorCount, dev);
        if (g_bsms <= 0) g_bsms = 1;
    }
    return g_bsms;
}

template <typename T, int ST>
void launch_simt_t(const BatchProblem *dp, const int32_t *dt, int64_t t0, int64_t t1, T a, T be, cudaStream_t st) {
    constexpr int smem = batch_smem<T, ST>();
    static int per_sm = 0;  // resident blocks per SM of this instantiation
    if (per_sm == 0) {
        cudaFuncSetAttribute(batch_kernel<T, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, batch_kernel<T, ST>, kThreadsB, smem);
        per_sm = std::max(1, v);
    }
    // persistent grid: exactly the blocks that fit at once
    const int64_t grid = std::min<int64_t>(t1 - t0, (int64_t)sm_count() * per_sm);
    batch_kernel<T, ST><<<(unsigned)grid, kThreadsB, smem, st>>>(dp, dt, t0, t1, a, be,
                                                                 be == T(0) ? 2 : (be == T(1) ? 0 : 1));
}

// one SIMT launch over tiles [t0, t1) of the table dp / dt
tc_status launch_simt(tc_dtype dtype, int stages, const BatchProblem *dp, const int32_t *dt, int64_t t0, int64_t t1,
                      const void *alpha, const void *beta, cudaStream_t st) {
    if (t1 <= t0) return TC_SUCCESS;
    if (dtype == TC_F64) {
        const double a = *(const double *)alpha, be = *(const double *)beta;
        if (stages == 3) launch_simt_t<double, 3>(dp, dt, t0, t1, a, be, st);
        else launch_simt_t<double, 2>(dp, dt, t0, t1, a, be, st);
    } else {
        const float a = *(const float *)alpha, be = *(const float *)beta;
        if (stages == 3) launch_simt_t<float, 3>(dp, dt, t0, t1, a, be, st);
        else launch_simt_t<float, 2>(dp, dt, t0, t1, a, be, st);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TC_SUCCESS : fail(TC_ERROR_CUDA, cudaGetErrorString(e));
}

std::vector<int32_t> tile_table(const std::vector<BatchProblem> &ps, int64_t total) {
    std::vector<int32_t> tp(total);
    for (size_t slot = 0; slot < ps.size(); ++slot) {
        const int64_t t1 = slot + 1 < ps.size() ? ps[slot + 1].tile0 : total;
        for (int64_t t = ps[slot].tile0; t < t1; ++t) tp[t] = (int32_t)slot;
    }
    return tp;
}

// device scratch for the autotuner's problem subsets
struct TuneScratch {
    BatchProblem *dp = nullptr;
    int32_t *dt = nullptr;
    int64_t tcap = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~TuneScratch() {
        if (dp) cudaFree(dp);
        if (dt) cudaFree(dt);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Median seconds of `reps` launches (after one warm-up) over the problems
// ps (their tile fields already set; alpha 1, beta 0: C = A.B).
tc_status time_subset(const BatchImpl &b, std::vector<BatchProblem> &ps, int stages, int reps, TuneScratch &sc,
                      cudaStream_t st, double *sec) {
    const size_t esz = b.dtype == TC_F64 ? 8 : 4;
    int64_t total = 0;
    for (auto &P : ps) {
        P.tile0 = total;
        total += (int64_t)P.tiles_m * ((P.N + shape_cols(P.shape) - 1) / shape_cols(P.shape));
        P.flags = flags_for(P, esz);
    }
    if (total > sc.tcap) {
        if (sc.dt) cudaFree(sc.dt);
        sc.dt = nullptr;
        sc.tcap = 0;
        cudaError_t e = cudaMalloc(&sc.dt, sizeof(int32_t) * total);
        if (e != cudaSuccess) return fail(TC_ERROR_OUT_OF_MEMORY, cudaGetErrorString(e));
        sc.tcap = total;
    }
    std::vector<int32_t> tp = tile_table(ps, total);
    cudaError_t e = cudaMemcpyAsync(sc.dp, ps.data(), sizeof(BatchProblem) * ps.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sc.dt, tp.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    const double one = 1.0, zero = 0.0;
    const float onef = 1.0f, zerof = 0.0f;
    const void *alpha = b.dtype == TC_F64 ? (const void *)&one : (const void *)&onef;
    const void *beta = b.dtype == TC_F64 ? (const void *)&zero : (const void *)&zerof;
    std::vector<double> t;
    for (int r = 0; r <= reps; ++r) {
        cudaEventRecord(sc.e0, st);
        tc_status s = launch_simt(b.dtype, stages, sc.dp, sc.dt, 0, total, alpha, beta, st);
        cudaEventRecord(sc.e1, st);
        if (s != TC_SUCCESS) return s;
        e = cudaEventSynchronize(sc.e1);
        if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
        float ms = 0;
        cudaEventElapsedTime(&ms, sc.e0, sc.e1);
        if (r > 0) t.push_back(ms * 1e-3);
    }
    std::sort(t.begin(), t.end());
    *sec = t[t.size() / 2];
    return TC_SUCCESS;
}

std::string class_key(const BatchImpl &b, const std::tuple<int, int, int> &c) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "?";
    return "batch|" + b.spec + "|" + std::to_string((int)b.dtype) + "|m" + std::to_string(std::get<0>(c)) + "k" +
           std::to_string(std::get<1>(c)) + "n" + std::to_string(std::get<2>(c)) + "|" + name;
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
    b.stream_layout = dtype == TC_BF16X3;
    for (const auto &P : b.probs) b.stream_layout = b.stream_layout && stream_eligible(P);  // no pointers yet
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
    if (policy < 0 || policy > 2)
        return fail(TC_ERROR_INVALID_ARGUMENT, "policy is 0 (fixed), 1 (rule) or 2 (autotuned)");
    if (policy == 2 && !batch->b.has_tuning)
        return fail(TC_ERROR_INVALID_ARGUMENT, "policy 2 needs tc_batch_autotune first");
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
    if (b.dtype == TC_BF16X3 && b.bf_stream) {
        bool ok = true;
        for (const auto &P : b.probs) ok = ok && stream_eligible(P);
        if (!ok) {  // an operand is not 16-byte aligned: GETT tiles instead
            const int keep = b.policy;
            b.policy = 1;
            b.stream_layout = false;
            assign_tiles(b);
            b.policy = keep == 2 ? 1 : keep;
        }
    }
    if (b.total_tiles >= ((int64_t)1 << 31)) return fail(TC_ERROR_INVALID_EXTENT, "2^31 tiles or more in one batch");
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
        if (b.dtype != TC_BF16X3)
            for (auto &P : b.probs) P.flags = flags_for(P, b.dtype == TC_F64 ? 8 : 4);
        cudaError_t e = cudaMemcpy(b.dprobs, b.probs.data(), sizeof(BatchProblem) * b.count, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
        if (b.dtype == TC_BF16X3) {
            const size_t db = gett_desc_bytes();
            std::vector<unsigned char> hd(db * b.count);
            for (int slot = 0; slot < b.count; ++slot) gett_fill_batch_desc(b.probs[slot], b.bn, hd.data() + db * slot);
            e = cudaMemcpy(b.ddescs, hd.data(), hd.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
        }
        std::vector<int32_t> tp = tile_table(b.probs, b.total_tiles);
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
    cudaStream_t st = (cudaStream_t)stream;
    b.last_stream = stream;
    auto range = [&](int slot) {
        const int64_t t0 = b.probs[slot].tile0;
        return std::make_pair(t0, slot + 1 < b.count ? b.probs[slot + 1].tile0 : b.total_tiles);
    };
    if (b.dtype == TC_BF16X3) {
        const float a = *(const float *)alpha, be = *(const float *)beta;
        int one_stage = 1;
        for (const auto &P : b.probs)
            if (P.K > 32) one_stage = 0;
        auto run = [&](int64_t t0, int64_t t1) {
            if (b.bf_stream) return stream_launch_batch(b.dprobs, b.dtile_prob, t0, t1, a, be, b.nprod, b.dstatus, stream);
            return gett_launch_batch(b.ddescs, b.dtile_prob, t0, t1, b.bn, a, be, b.nprod, b.dstatus, one_stage, 0,
                                     stream);
        };
        if (one_launch_per_problem) {
            for (int slot = 0; slot < b.count; ++slot) {
                tc_status s = run(range(slot).first, range(slot).second);
                if (s != TC_SUCCESS) return s;
            }
            return TC_SUCCESS;
        }
        return run(0, b.total_tiles);
    }
    if (one_launch_per_problem) {
        for (int slot = 0; slot < b.count; ++slot) {
            tc_status s = launch_simt(b.dtype, b.stages, b.dprobs, b.dtile_prob, range(slot).first, range(slot).second,
                                      alpha, beta, st);
            if (s != TC_SUCCESS) return s;
        }
        return TC_SUCCESS;
    }
    return launch_simt(b.dtype, b.stages, b.dprobs, b.dtile_prob, 0, b.total_tiles, alpha, beta, st);
}

tc_status tc_batch_autotune(tc_batch batch, void *stream, int32_t reps, tc_batch_tuning *classes, int32_t capacity,
                            int32_t *n_classes) {
    if (!batch) return fail(TC_ERROR_INVALID_ARGUMENT, "batch is NULL");
    if (reps < 1) return fail(TC_ERROR_INVALID_ARGUMENT, "reps < 1");
    if (capacity < 0 || (capacity > 0 && !classes)) return fail(TC_ERROR_INVALID_ARGUMENT, "bad class buffer");
    BatchImpl &b = batch->b;
    tc_status s = tc_batch_prepare(batch);  // checks the operands, uploads the table
    if (s != TC_SUCCESS) return s;
    cudaStream_t st = (cudaStream_t)stream;
    b.last_stream = stream;
    std::vector<tc_batch_tuning> rows;
    if (b.dtype == TC_BF16X3) {
        // candidates for the whole batch: GETT tiles 128 x 128 and 128 x 256,
        // and the stream kernel where every problem suits it
        const float onef = 1.0f, zerof = 0.0f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        bool stream_ok = b.stream_layout;
        for (const auto &P : b.probs) stream_ok = stream_ok && stream_eligible(P);
        const int ncand = stream_ok ? 3 : 2;
        double tw[3] = {0, 0, 0};
        const int saved_policy = b.policy, saved_bn = b.tuned_bn, saved_stream = b.tuned_stream;
        for (int w = 0; w < ncand && s == TC_SUCCESS; ++w) {
            b.tuned_bn = w == 0 ? 128 : 256;
            b.tuned_stream = w == 2;
            b.policy = 2;
            assign_tiles(b);
            s = tc_batch_prepare(batch);
            std::vector<double> t;
            for (int r = 0; r <= reps && s == TC_SUCCESS; ++r) {
                cudaEventRecord(e0, st);
                s = tc_batch_execute(batch, &onef, &zerof, 0, stream);
                cudaEventRecord(e1, st);
                if (s != TC_SUCCESS) break;
                cudaError_t e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    s = fail(TC_ERROR_CUDA, cudaGetErrorString(e));
                    break;
                }
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) t.push_back(ms * 1e-3);
            }
            if (s == TC_SUCCESS) {
                std::sort(t.begin(), t.end());
                tw[w] = t[t.size() / 2];
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (s == TC_SUCCESS) s = tc_batch_device_status(batch);
        if (s != TC_SUCCESS) {
            b.policy = saved_policy;
            b.tuned_bn = saved_bn;
            b.tuned_stream = saved_stream;
            assign_tiles(b);
            return s;
        }
        int best = 0;
        for (int w = 1; w < ncand; ++w)
            if (tw[w] < tw[best]) best = w;
        b.tuned_bn = best == 0 ? 128 : 256;
        b.tuned_stream = best == 2;
        b.has_tuning = true;
        b.policy = 2;
        assign_tiles(b);
        tc_batch_tuning r{};
        r.m_log2 = r.k_log2 = r.n_class = -1;
        r.problems = b.count;
        r.candidates = ncand;
        r.kernel = best == 2 ? 2 : 1;
        r.tile_m = 128;
        r.tile_n = best == 2 ? 128 : b.tuned_bn;
        r.k_chunk = 32;
        r.seconds_best = tw[best];
        // the rule: the stream kernel where possible, else the padded-column width
        if (stream_ok) {
            r.seconds_rule = tw[2];
        } else {
            BatchImpl probe = b;
            probe.ddescs = nullptr, probe.dstatus = nullptr, probe.dprobs = nullptr, probe.dtile_prob = nullptr;
            probe.policy = 1;
            assign_tiles(probe);
            r.seconds_rule = probe.bn == 256 ? tw[1] : tw[0];
        }
        r.seconds_fixed = tw[1];
        rows.push_back(r);
    } else {
        // per shape class: every (tile shape, K chunk) candidate timed on
        // the class's problems alone
        std::map<std::tuple<int, int, int>, std::vector<int>> groups;
        for (int slot = 0; slot < b.count; ++slot) groups[class_of(b.probs[slot])].push_back(slot);
        TuneScratch sc;
        cudaError_t e = cudaMalloc(&sc.dp, sizeof(BatchProblem) * b.count);
        if (e != cudaSuccess) return fail(TC_ERROR_OUT_OF_MEMORY, cudaGetErrorString(e));
        cudaEventCreate(&sc.e0);
        cudaEventCreate(&sc.e1);
        std::map<std::tuple<int, int, int>, std::pair<int, int>> chosen;
        for (auto &g : groups) {
            const auto &cls = g.first;
            const int64_t kmax = (int64_t)1 << std::get<1>(cls);
            int64_t mmax = 0;
            for (int slot : g.second) mmax = std::max(mmax, b.probs[slot].M);
            tc_batch_tuning r{};
            r.m_log2 = std::get<0>(cls);
            r.k_log2 = std::get<1>(cls);
            r.n_class = std::get<2>(cls);
            r.problems = (int32_t)g.second.size();
            r.kernel = 0;
            std::map<std::string, int> cached;
            if (tuning_get(class_key(b, cls), cached) && cached.count("batch_tile_m") && cached.count("batch_k_chunk")) {
                const int tm = cached["batch_tile_m"], bk = cached["batch_k_chunk"];
                const int sh = ceil_log2(tm) - 3;
                if (sh >= 0 && sh < kShapes && shape_rows(sh) == tm && stage_fits(sh, bk) &&
                    (bk == 8 || bk == 16 || bk == 32)) {
                    chosen[cls] = {sh, bk};
                    r.tile_m = tm;
                    r.tile_n = shape_cols(sh);
                    r.k_chunk = bk;
                    r.seconds_best = r.seconds_rule = r.seconds_fixed = -1;
                    rows.push_back(r);
                    continue;
                }
            }
            const std::pair<int, int> rule = rule_choice(mmax, kmax), fixed = fixed_choice(kmax);
            double best = -1;
            std::pair<int, int> arg = rule;
            for (int sh = 0; sh < kShapes && s == TC_SUCCESS; ++sh) {
                for (int bk : {8, 16, 32}) {
                    if (!stage_fits(sh, bk) || !chunk_useful(bk, kmax)) continue;
                    std::vector<BatchProblem> ps;
                    ps.reserve(g.second.size());
                    int64_t dummy = 0;
                    for (int slot : g.second) {
                        ps.push_back(b.probs[slot]);
                        set_tiles_of(ps.back(), sh, bk, dummy);
                    }
                    double t = 0;
                    s = time_subset(b, ps, 2, reps, sc, st, &t);
                    if (s != TC_SUCCESS) break;
                    ++r.candidates;
                    if (best < 0 || t < best) {
                        best = t;
                        arg = {sh, bk};
                    }
                    if (std::make_pair(sh, bk) == rule) r.seconds_rule = t;
                    if (std::make_pair(sh, bk) == fixed) r.seconds_fixed = t;
                }
            }
            if (s != TC_SUCCESS) return s;
            chosen[cls] = arg;
            r.tile_m = shape_rows(arg.first);
            r.tile_n = shape_cols(arg.first);
            r.k_chunk = arg.second;
            r.seconds_best = best;
            rows.push_back(r);
            tuning_put(class_key(b, cls), {{"batch_tile_m", r.tile_m}, {"batch_k_chunk", r.k_chunk}});
        }
        // pipeline depth for the whole batch at the chosen tiles
        std::vector<BatchProblem> all(b.probs);
        int64_t dummy = 0;
        for (auto &P : all) set_tiles_of(P, chosen[class_of(P)].first, chosen[class_of(P)].second, dummy);
        double t2 = 0, t3 = 0;
        s = time_subset(b, all, 2, reps, sc, st, &t2);
        if (s == TC_SUCCESS) s = time_subset(b, all, 3, reps, sc, st, &t3);
        if (s != TC_SUCCESS) return s;
        b.tuned = chosen;
        b.tuned_stages = t3 < t2 ? 3 : 2;
        b.has_tuning = true;
        b.policy = 2;
        assign_tiles(b);
    }
    if (n_classes) *n_classes = (int32_t)rows.size();
    for (int32_t i = 0; i < capacity && i < (int32_t)rows.size(); ++i) classes[i] = rows[i];
    return TC_SUCCESS;
}

tc_status tc_batch_config(tc_batch batch, int32_t *policy, int32_t *stages, int32_t *tile_n, int32_t *kernel) {
    if (!batch) return fail(TC_ERROR_INVALID_ARGUMENT, "batch is NULL");
    const BatchImpl &b = batch->b;
    const bool bf = b.dtype == TC_BF16X3;
    if (policy) *policy = b.policy;
    if (stages) *stages = bf ? 0 : b.stages;
    if (tile_n) *tile_n = bf ? (b.bf_stream ? 128 : b.bn) : 0;
    if (kernel) *kernel = bf ? (b.bf_stream ? 2 : 1) : 0;
    return TC_SUCCESS;
}

tc_status tc_batch_problem_tiles(tc_batch batch, int32_t problem, int32_t *tile_m, int32_t *tile_n,
                                 int32_t *k_chunk) {
    if (!batch) return fail(TC_ERROR_INVALID_ARGUMENT, "batch is NULL");
    const BatchImpl &b = batch->b;
    if (problem < 0 || problem >= b.count) return fail(TC_ERROR_INVALID_ARGUMENT, "problem out of range");
    int slot = 0;
    while (b.order[slot] != problem) ++slot;
    const BatchProblem &P = b.probs[slot];
    const bool simt = b.dtype != TC_BF16X3;
    if (tile_m) *tile_m = simt ? shape_rows(P.shape) : 128;
    if (tile_n) *tile_n = simt ? shape_cols(P.shape) : (b.bf_stream ? 128 : b.bn);
    if (k_chunk) *k_chunk = P.bk;
    return TC_SUCCESS;
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
