// Nest executor: runs one Section 2 algorithm (a loop nest around one BLAS
// kernel) on the GPU, plus the SIMT form of the fused GETT for FP64/FP32.
//
// Reading of the sequential loop nests for a parallel device (the paper
// describes sequential CPU loops only):
//  * Loops keep their nest order.  Iterations of a free loop write disjoint
//    C slices and run concurrently.
//  * A contracted loop that encloses a free loop becomes a device-wide
//    phase: one launch per iteration, in order, C carried through memory.
//  * The remaining contracted loops (those with no free loop inside them)
//    run in order inside each task, C held in registers.
//  * Every C element therefore sees one fixed chain of fused multiply-adds
//    acc = fma(alpha*a, b, acc) over the contracted indices in nest order
//    (phase loops, then in-task loops, then the kernel's own contracted
//    index), starting from beta*C.  Algorithms with the same contracted
//    order give bitwise identical results.
//  * Copies (Section 2: a matrix slice without a unit-stride dimension)
//    materialise the slice into a contiguous workspace at the phase they
//    belong to, once per combination of the loops the slice depends on.
//
// Kernels: dot, axpy, gemv and ger run one thread per output element of a
// kernel call (kernel outputs fastest across threads, then the innermost
// free loop), reading operands straight from L1/L2 -- the BLAS-1/2 shape.
// gemm runs as a shared-memory tiled register-blocked kernel -- the BLAS-3
// shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "tc_internal.h"

namespace tc {

struct Dims {
    int n;
    int64_t ext[kMaxModes];
    int64_t sA[kMaxModes], sB[kMaxModes], sC[kMaxModes];
};

struct PhaseDesc {
    Dims out;   // kernel output modes, first fastest
    Dims task;  // free sliced loops, outermost first (innermost fastest)
    Dims red;   // contracted: in-task loops outermost first, kernel index last
    int64_t total;
    const void *A;
    const void *B;
    void *C;
    double alpha, beta;
    int init;       // 0: acc = C, 1: acc = beta*C, 2: acc = 0
    int alpha_one;  // alpha == 1: skip the scaling multiply
};

struct TileDesc {
    Dims m;     // M modes (first fastest): strides sA and sC
    Dims n;     // N modes: strides sB and sC
    Dims red;   // K modes, outermost first
    Dims task;  // tasks: free sliced loops, outermost first
    int64_t M, N, K;
    int64_t tiles_m, tiles_n;
    const void *A;
    const void *B;
    void *C;
    double alpha, beta;
    int init, alpha_one;
    int a_m_fast, b_n_fast;  // load mapping: M (N) contiguous in memory
    int64_t tile0;           // batched form: the problem's first tile in the list
};

struct GatherDesc {
    int n;
    int64_t ext[2 * kMaxModes];
    int64_t ss[2 * kMaxModes];  // source strides
    int64_t sd[2 * kMaxModes];  // destination strides
    int64_t total;
    const void *src;
    void *dst;
};

namespace {

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }

// ---------------------------------------------------------------- dot/axpy/gemv/ger
template <typename T>
__global__ void __launch_bounds__(256) elementwise_kernel(const PhaseDesc d) {
    const T *__restrict__ A = (const T *)d.A;
    const T *__restrict__ B = (const T *)d.B;
    T *__restrict__ C = (T *)d.C;
    const T alpha = (T)d.alpha, beta = (T)d.beta;
    const int nr = d.red.n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < d.total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e, oA = 0, oB = 0, oC = 0;
        for (int m = 0; m < d.out.n; ++m) {
            int64_t x = r % d.out.ext[m];
            r /= d.out.ext[m];
            oA += x * d.out.sA[m];
            oB += x * d.out.sB[m];
            oC += x * d.out.sC[m];
        }
        for (int m = d.task.n - 1; m >= 0; --m) {
            int64_t x = r % d.task.ext[m];
            r /= d.task.ext[m];
            oA += x * d.task.sA[m];
            oB += x * d.task.sB[m];
            oC += x * d.task.sC[m];
        }
        T acc;
        if (d.init == 2) {
            acc = T(0);
        } else {
            acc = C[oC];
            if (d.init == 1) acc = beta * acc;
        }
        if (nr == 0) {
            T a = A[oA];
            if (!d.alpha_one) a = alpha * a;
            acc = fma_t<T>(a, B[oB], acc);
        } else {
            int64_t idx[kMaxModes];
            for (int m = 0; m < nr; ++m) idx[m] = 0;
            const int64_t kext = d.red.ext[nr - 1];
            const int64_t ksA = d.red.sA[nr - 1], ksB = d.red.sB[nr - 1];
            for (;;) {
                int64_t pa = oA, pb = oB;
                for (int m = 0; m < nr - 1; ++m) {
                    pa += idx[m] * d.red.sA[m];
                    pb += idx[m] * d.red.sB[m];
                }
                for (int64_t k = 0; k < kext; ++k) {
                    T a = A[pa];
                    if (!d.alpha_one) a = alpha * a;
                    acc = fma_t<T>(a, B[pb], acc);
                    pa += ksA;
                    pb += ksB;
                }
                int m = nr - 2;
                while (m >= 0) {
                    if (++idx[m] < d.red.ext[m]) break;
                    idx[m] = 0;
                    --m;
                }
                if (m < 0) break;
            }
        }
        C[oC] = acc;
    }
}

// Cooperative reduction (a phase with few outputs whose innermost contracted
// index has unit stride in an input): a group of G lanes (a power of two,
// 4..32) per kernel output splits that index (red's last mode), so the
// group's loads are contiguous; each lane sums its share over every in-task
// contracted loop, then the group adds the lanes' partial sums with a fixed
// butterfly (the same order every run).
template <typename T, int G>
__global__ void __launch_bounds__(256) coop_reduce_kernel(const PhaseDesc d) {
    const T *__restrict__ A = (const T *)d.A;
    const T *__restrict__ B = (const T *)d.B;
    T *__restrict__ C = (T *)d.C;
    const int gl = threadIdx.x % G;  // lane within the group
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
    const int nr = d.red.n;
    const int64_t kext = d.red.ext[nr - 1], ksA = d.red.sA[nr - 1], ksB = d.red.sB[nr - 1];
    // every lane of a warp runs the same number of rounds (shuffles need the
    // whole warp): the round's output is e = warp's first + the group's
    const int64_t first = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    for (int64_t base = first - (threadIdx.x % 32) / G; base < d.total; base += groups) {
        const int64_t e = base + (threadIdx.x % 32) / G;
        const bool live = e < d.total;
        int64_t r = live ? e : 0, oA = 0, oB = 0, oC = 0;
        for (int m = 0; m < d.out.n; ++m) {
            const int64_t x = r % d.out.ext[m];
            r /= d.out.ext[m];
            oA += x * d.out.sA[m];
            oB += x * d.out.sB[m];
            oC += x * d.out.sC[m];
        }
        for (int m = d.task.n - 1; m >= 0; --m) {
            const int64_t x = r % d.task.ext[m];
            r /= d.task.ext[m];
            oA += x * d.task.sA[m];
            oB += x * d.task.sB[m];
            oC += x * d.task.sC[m];
        }
        T acc = T(0);
        int64_t idx[kMaxModes];
        for (int m = 0; m < nr - 1; ++m) idx[m] = 0;
        for (;;) {
            int64_t pa = oA, pb = oB;
            for (int m = 0; m < nr - 1; ++m) {
                pa += idx[m] * d.red.sA[m];
                pb += idx[m] * d.red.sB[m];
            }
            if (live)
                for (int64_t k = gl; k < kext; k += G) acc = fma_t<T>(A[pa + k * ksA], B[pb + k * ksB], acc);
            int m = nr - 2;
            while (m >= 0) {
                if (++idx[m] < d.red.ext[m]) break;
                idx[m] = 0;
                --m;
            }
            if (m < 0) break;
        }
#pragma unroll
        for (int off = G / 2; off > 0; off /= 2) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (live && gl == 0) {
            T v = d.alpha_one ? acc : (T)d.alpha * acc;
            if (d.init == 0) v += C[oC];
            else if (d.init == 1) v = fma_t<T>((T)d.beta, C[oC], v);
            C[oC] = v;
        }
    }
}

// ---------------------------------------------------------------- gemm / SIMT GETT
// One CTA computes a BM x BN tile of one task's C slice; K runs over the
// linearised contracted space in chunks of BK staged through shared memory.
template <typename T, int BM, int BN, int BK, int TM, int TN>
__device__ __forceinline__ void tile_body(const TileDesc &d, int64_t bid) {
    constexpr int TX = BN / TN, TY = BM / TM, NT = TX * TY;
    // A thread owns rows ty*V + r + g*TY*V (r < V, g < TM/V) and likewise
    // columns: with V = 4 for FP32 each group is one 16-byte shared-memory
    // read, so a K step issues TM/4 + TN/4 loads for TM*TN FMAs instead of
    // TM + TN; FP64 (V = 1) is bound by the DFMA rate either way.
    constexpr int V = (sizeof(T) == 4 && TM % 4 == 0 && TN % 4 == 0) ? 4 : 1;
    auto row_of = [](int ty_, int i) { return (i / V) * (TY * V) + ty_ * V + i % V; };
    auto col_of = [](int tx_, int j) { return (j / V) * (TX * V) + tx_ * V + j % V; };
    // two stage buffers; rows padded by 4 elements so that the K-contiguous
    // store mapping below spreads a warp over all 32 banks
    constexpr int PAD = 4;
    __shared__ __align__(16) T As[2][BK][BM + PAD];
    __shared__ __align__(16) T Bs[2][BK][BN + PAD];
    __shared__ int64_t offAm[BM], offCm[BM], offBn[BN], offCn[BN];
    __shared__ int64_t kA[2][BK], kB[2][BK];
    const T *__restrict__ A = (const T *)d.A;
    const T *__restrict__ B = (const T *)d.B;
    T *__restrict__ C = (T *)d.C;
    const T alpha = (T)d.alpha, beta = (T)d.beta;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;

    const int64_t tm = bid % d.tiles_m;
    bid /= d.tiles_m;
    const int64_t tn = bid % d.tiles_n;
    int64_t task = bid / d.tiles_n;
    int64_t tA = 0, tB = 0, tC = 0;
    for (int m = d.task.n - 1; m >= 0; --m) {
        int64_t x = task % d.task.ext[m];
        task /= d.task.ext[m];
        tA += x * d.task.sA[m];
        tB += x * d.task.sB[m];
        tC += x * d.task.sC[m];
    }
    for (int i = tid; i < BM; i += NT) {
        int64_t mm = tm * BM + i;
        int64_t oa = -1, oc = -1;
        if (mm < d.M) {
            oa = tA;
            oc = tC;
            for (int m = 0; m < d.m.n; ++m) {
                int64_t x = mm % d.m.ext[m];
                mm /= d.m.ext[m];
                oa += x * d.m.sA[m];
                oc += x * d.m.sC[m];
            }
        }
        offAm[i] = oa;
        offCm[i] = oc;
    }
    for (int j = tid; j < BN; j += NT) {
        int64_t nn = tn * BN + j;
        int64_t ob = -1, oc = -1;
        if (nn < d.N) {
            ob = tB;
            oc = 0;
            for (int m = 0; m < d.n.n; ++m) {
                int64_t x = nn % d.n.ext[m];
                nn /= d.n.ext[m];
                ob += x * d.n.sB[m];
                oc += x * d.n.sC[m];
            }
        }
        offBn[j] = ob;
        offCn[j] = oc;
    }
    __syncthreads();

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t om = offCm[row_of(ty, i)];
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t on = offCn[col_of(tx, j)];
            T v = T(0);
            if (d.init != 2 && om >= 0 && on >= 0) {
                v = C[om + on];
                if (d.init == 1) v = beta * v;
            }
            acc[i][j] = v;
        }
    }

    // K offsets of a stage into table buffer b (threads kk < BK); the K
    // position's digits in 32-bit arithmetic when K fits (a 64-bit division
    // is a long dependent sequence, and the other warps wait for these
    // tables at the stage's barrier)
    auto k_tables = [&](int64_t k0, int b) {
        for (int kk = tid; kk < BK; kk += NT) {
            int64_t k = k0 + kk;
            int64_t oa = -1, ob = -1;
            if (k < d.K) {
                oa = 0;
                ob = 0;
                if (d.K < (int64_t(1) << 31)) {
                    uint32_t k32 = (uint32_t)k;
                    for (int m = d.red.n - 1; m >= 0; --m) {
                        const uint32_t e = (uint32_t)d.red.ext[m];
                        const int64_t x = (int64_t)(k32 % e);
                        k32 /= e;
                        oa += x * d.red.sA[m];
                        ob += x * d.red.sB[m];
                    }
                } else {
                    for (int m = d.red.n - 1; m >= 0; --m) {
                        int64_t x = k % d.red.ext[m];
                        k /= d.red.ext[m];
                        oa += x * d.red.sA[m];
                        ob += x * d.red.sB[m];
                    }
                }
            }
            kA[b][kk] = oa;
            kB[b][kk] = ob;
        }
    };
    // Element e of a stage's R x BK operand tile: with M (N) contiguous in
    // memory, consecutive threads take consecutive rows; otherwise groups
    // of 8 threads take 8 consecutive K positions of one row (32-byte runs
    // in memory; with the padded rows a warp's stores hit 32 distinct banks).
    static_assert(BK % 8 == 0, "K stage is a multiple of 8");
    auto place = [](int e, bool rfast, int R, int &r, int &kk) {
        if (rfast) {
            r = e % R;
            kk = e / R;
        } else {
            r = (e / 8) % R;
            kk = (e / (8 * R)) * 8 + e % 8;
        }
    };
    // a stage's A and B elements of this thread, into registers
    constexpr int LA = BM * BK / NT, LB = BN * BK / NT;
    static_assert(LA * NT == BM * BK && LB * NT == BN * BK, "even split");
    T ra[LA], rb[LB];
    auto load_stage = [&](int b) {
#pragma unroll
        for (int l = 0; l < LA; ++l) {
            int i, kk;
            place(tid + l * NT, d.a_m_fast, BM, i, kk);
            const int64_t om = offAm[i], ok = kA[b][kk];
            T v = T(0);
            if (om >= 0 && ok >= 0) {
                v = A[om + ok];
                if (!d.alpha_one) v = alpha * v;
            }
            ra[l] = v;
        }
#pragma unroll
        for (int l = 0; l < LB; ++l) {
            int j, kk;
            place(tid + l * NT, d.b_n_fast, BN, j, kk);
            const int64_t on = offBn[j], ok = kB[b][kk];
            rb[l] = (on >= 0 && ok >= 0) ? B[on + ok] : T(0);
        }
    };
    auto store_stage = [&](int sb) {
#pragma unroll
        for (int l = 0; l < LA; ++l) {
            int i, kk;
            place(tid + l * NT, d.a_m_fast, BM, i, kk);
            As[sb][kk][i] = ra[l];
        }
#pragma unroll
        for (int l = 0; l < LB; ++l) {
            int j, kk;
            place(tid + l * NT, d.b_n_fast, BN, j, kk);
            Bs[sb][kk][j] = rb[l];
        }
    };
    // FP32 with alpha = 1: the stage's elements go straight to shared memory
    // with 4-byte asynchronous copies (zero-filled past the extents), so no
    // register holds them and no second pass stores them; the same values
    // land in the same places as through load_stage + store_stage
    const bool async_copy = sizeof(T) == 4 && d.alpha_one;
    auto async_stage = [&](int b) {
        auto cp4 = [](void *dst, const void *src, bool valid) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(dst)),
                         "l"(src), "r"(valid ? 4 : 0)
                         : "memory");
        };
#pragma unroll
        for (int l = 0; l < LA; ++l) {
            int i, kk;
            place(tid + l * NT, d.a_m_fast, BM, i, kk);
            const int64_t om = offAm[i], ok = kA[b][kk];
            const bool v = om >= 0 && ok >= 0;
            cp4(&As[b][kk][i], v ? A + om + ok : A, v);
        }
#pragma unroll
        for (int l = 0; l < LB; ++l) {
            int j, kk;
            place(tid + l * NT, d.b_n_fast, BN, j, kk);
            const int64_t on = offBn[j], ok = kB[b][kk];
            const bool v = on >= 0 && ok >= 0;
            cp4(&Bs[b][kk][j], v ? B + on + ok : B, v);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto async_wait = []() { asm volatile("cp.async.wait_all;" ::: "memory"); };
    // Stage s sits in buffer s & 1 (shared memory and K tables alike).
    // While stage s is multiplied, stage s + 1's global loads are in flight
    // and then stored to the other buffer, whose last reader (stage s - 1)
    // finished before the barrier that ended the previous iteration; one
    // barrier per stage.  Stage s + 2's K tables go to buffer s & 1 right
    // after stage s + 1's loads have read theirs (buffer s & 1 was last read
    // by stage s's loads, before that barrier), so that their integer work
    // overlaps the multiplications instead of delaying the barrier.
    k_tables(0, 0);
    __syncthreads();
    if (async_copy) {
        async_stage(0);
        async_wait();
    } else {
        load_stage(0);
        store_stage(0);
    }
    if (BK < d.K) k_tables(BK, 1);
    __syncthreads();
    int sb = 0;
    for (int64_t k0 = 0; k0 < d.K; k0 += BK, sb ^= 1) {
        const bool more = k0 + BK < d.K;
        if (more) {
            if (async_copy) async_stage(sb ^ 1);
            else load_stage(sb ^ 1);
        }
        if (k0 + 2 * BK < d.K) k_tables(k0 + 2 * BK, sb);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
            if constexpr (V == 4) {
#pragma unroll
                for (int g = 0; g < TM / 4; ++g) {
                    const float4 v = *reinterpret_cast<const float4 *>(&As[sb][kk][row_of(ty, 4 * g)]);
                    a[4 * g] = v.x;
                    a[4 * g + 1] = v.y;
                    a[4 * g + 2] = v.z;
                    a[4 * g + 3] = v.w;
                }
#pragma unroll
                for (int g = 0; g < TN / 4; ++g) {
                    const float4 v = *reinterpret_cast<const float4 *>(&Bs[sb][kk][col_of(tx, 4 * g)]);
                    b[4 * g] = v.x;
                    b[4 * g + 1] = v.y;
                    b[4 * g + 2] = v.z;
                    b[4 * g + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = As[sb][kk][row_of(ty, i)];
#pragma unroll
                for (int j = 0; j < TN; ++j) b[j] = Bs[sb][kk][col_of(tx, j)];
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma_t<T>(a[i], b[j], acc[i][j]);
        }
        if (more) {
            if (async_copy) async_wait();
            else store_stage(sb ^ 1);
        }
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t om = offCm[row_of(ty, i)];
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t on = offCn[col_of(tx, j)];
            if (om >= 0 && on >= 0) C[om + on] = acc[i][j];
        }
    }
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) tile_kernel(const TileDesc d) {
    tile_body<T, BM, BN, BK, TM, TN>(d, blockIdx.x);
}

// Batched form of the SIMT GETT (no paper counterpart): CTA t computes tile
// t of the flattened tile list of many problems, each with its own
// descriptor (modes, strides, operands); the descriptor of the tile's
// problem is copied to shared memory first.  A problem's tiles compute
// exactly as tile_kernel computes them, whatever else is in the batch.
template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
tile_batch_kernel(const TileDesc *__restrict__ descs, const int32_t *__restrict__ tile_prob) {
    __shared__ __align__(16) TileDesc sd;
    static_assert(sizeof(TileDesc) % 8 == 0, "descriptor in 8-byte words");
    constexpr int kWords = sizeof(TileDesc) / 8;
    const int q = tile_prob[blockIdx.x];
    for (int w = threadIdx.x; w < kWords; w += blockDim.x)
        ((int64_t *)&sd)[w] = ((const int64_t *)(descs + q))[w];
    __syncthreads();
    tile_body<T, BM, BN, BK, TM, TN>(sd, (int64_t)blockIdx.x - sd.tile0);
}

// ---------------------------------------------------------------- copy
template <typename T>
__global__ void __launch_bounds__(256) gather_kernel(const GatherDesc g) {
    const T *__restrict__ src = (const T *)g.src;
    T *__restrict__ dst = (T *)g.dst;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e, os = 0, od = 0;
        for (int m = 0; m < g.n; ++m) {
            int64_t x = r % g.ext[m];
            r /= g.ext[m];
            os += x * g.ss[m];
            od += x * g.sd[m];
        }
        dst[od] = src[os];
    }
}

// ---------------------------------------------------------------- host helpers
int g_sm_count = 0;

int sm_count() {
    if (g_sm_count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0) g_sm_count = 1;
    }
    return g_sm_count;
}

int device_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int64_t grid_for(int64_t total, int per_block) {
    int64_t blocks = (total + per_block - 1) / per_block;
    int64_t cap = (int64_t)sm_count() * 32;
    return std::max<int64_t>(1, std::min(blocks, cap));
}

void add_dim(Dims &d, int64_t ext, int64_t sA, int64_t sB, int64_t sC) {
    d.ext[d.n] = ext;
    d.sA[d.n] = sA;
    d.sB[d.n] = sB;
    d.sC[d.n] = sC;
    ++d.n;
}

// Per-operand addressing for one execution: original or workspace layout.
struct OpView {
    bool copied = false;
    const char *base = nullptr;        // workspace base when copied
    int64_t ws_stride[kMaxIdx] = {};   // workspace stride per index id
    bool ws_has[kMaxIdx] = {};
    // copy description
    std::vector<int> copy_ids;         // kernel modes, then non-phase dependencies
    int64_t elems = 0;
};

struct NestLayout {
    std::vector<int> phase_pos;   // positions of phase loops (contracted, <= q)
    std::vector<int> task_ids;    // free loop index ids, nest order
    std::vector<int> red_ids;     // contracted in-task loops, then kernel k
    std::vector<int> out_ids;     // kernel output modes
    OpView view[3];
    size_t ws_offset[3] = {0, 0, 0};
    size_t ws_bytes = 0;
};

NestLayout layout_for(const Plan &p, const Algorithm &alg) {
    NestLayout L;
    for (int pos = 0; pos < alg.nloops; ++pos) {
        int id = alg.loops[pos];
        if (p.cls[id] == CLS_CONTRACTED) {
            if (pos <= alg.q) L.phase_pos.push_back(pos);
            else L.red_ids.push_back(id);
        } else {
            L.task_ids.push_back(id);
        }
    }
    switch (alg.kernel) {
    case TC_KERNEL_DOT: L.red_ids.push_back(alg.kidx[0]); break;
    case TC_KERNEL_AXPY: L.out_ids.push_back(alg.kidx[0]); break;
    case TC_KERNEL_GEMV:
        L.out_ids.push_back(alg.kidx[0]);
        L.red_ids.push_back(alg.kidx[1]);
        break;
    case TC_KERNEL_GER:
        L.out_ids.push_back(alg.kidx[0]);
        L.out_ids.push_back(alg.kidx[1]);
        break;
    case TC_KERNEL_GEMM:
        L.out_ids.push_back(alg.kidx[0]);
        L.out_ids.push_back(alg.kidx[1]);
        L.red_ids.push_back(alg.kidx[2]);
        break;
    }
    size_t esz[3] = {elem_bytes_ab(p.dtype), elem_bytes_ab(p.dtype), elem_bytes_c(p.dtype)};
    size_t off = 0;
    for (int o = 0; o < 3; ++o) {
        if (alg.copy_level[o] == -2) continue;
        OpView &v = L.view[o];
        v.copied = true;
        const Layout &lay = p.op[o];
        // kernel modes in storage order, then the loops the slice depends on
        // that are not fixed by the phase, in nest order
        for (int m = 0; m < lay.n; ++m)
            for (int r = 0; r < alg.nk; ++r)
                if (lay.idx[m] == alg.kidx[r]) v.copy_ids.push_back(lay.idx[m]);
        for (int pos = 0; pos < alg.nloops; ++pos) {
            int id = alg.loops[pos];
            if (!lay.has(id)) continue;
            bool phase = p.cls[id] == CLS_CONTRACTED && pos <= alg.q;
            if (!phase) v.copy_ids.push_back(id);
        }
        int64_t s = 1;
        for (int id : v.copy_ids) {
            v.ws_stride[id] = s;
            v.ws_has[id] = true;
            s *= p.ext[id];
        }
        v.elems = s;
        L.ws_offset[o] = off;
        off += ((size_t)s * esz[o] + 255) / 256 * 256;
    }
    L.ws_bytes = off;
    return L;
}

template <typename T>
tc_status launch_gather(const GatherDesc &g, cudaStream_t st) {
    int64_t grid = grid_for(g.total, 256);
    gather_kernel<T><<<(unsigned)grid, 256, 0, st>>>(g);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TC_SUCCESS : fail(TC_ERROR_CUDA, cudaGetErrorString(e));
}

// The gather moves elements of the operand's own size (FP64, FP32, or the
// 16-bit inputs of the BF16 / FP16 forms).
tc_status launch_copy(const Plan &p, int o, const OpView &v, const char *src_base,
                      void *dst, bool scatter, cudaStream_t st, double frac = 1.0) {
    GatherDesc g;
    std::memset(&g, 0, sizeof(g));
    g.n = (int)v.copy_ids.size();
    for (int m = 0; m < g.n; ++m) {
        int id = v.copy_ids[m];
        g.ext[m] = p.ext[id];
        int64_t orig = p.op[o].stride_of(id);
        int64_t ws = v.ws_stride[id];
        g.ss[m] = scatter ? ws : orig;
        g.sd[m] = scatter ? orig : ws;
    }
    g.total = frac >= 1.0 ? v.elems : std::max<int64_t>(1, (int64_t)(v.elems * frac));
    g.src = scatter ? dst : src_base;
    g.dst = scatter ? (void *)src_base : dst;
    const size_t eb = o == OP_C ? elem_bytes_c(p.dtype) : elem_bytes_ab(p.dtype);
    if (eb == 8) return launch_gather<double>(g, st);
    if (eb == 2) return launch_gather<unsigned short>(g, st);
    return launch_gather<float>(g, st);
}

template <typename T>
tc_status run_nest(Plan &p, const Algorithm &alg, T alpha, const T *A, const T *B,
                   T beta, T *C, cudaStream_t st, const Probe *probe) {
    NestLayout L = layout_for(p, alg);
    char *ws = (char *)p.workspace;
    const char *base[3] = {(const char *)A, (const char *)B, (const char *)C};
    const size_t esz = elem_bytes_ab(p.dtype);  // A and B (16 bits for the BF16 / FP16 forms)
    // tensor-core dtypes run their gemm phases on the tensor-core GETT
    const bool tensor = p.dtype != TC_F64 && p.dtype != TC_F32;
    // stride of index id in operand o as the phase kernel sees it
    auto stride_in = [&](int o, int id) -> int64_t {
        if (L.view[o].copied) return L.view[o].ws_has[id] ? L.view[o].ws_stride[id] : 0;
        return p.op[o].stride_of(id);
    };
    auto fill = [&](Dims &d, const std::vector<int> &ids) {
        d.n = 0;
        for (int id : ids)
            add_dim(d, p.ext[id], stride_in(OP_A, id), stride_in(OP_B, id), stride_in(OP_C, id));
    };
    const int init0 = beta == T(0) ? 2 : (beta == T(1) ? 0 : 1);
    const bool alpha_one = alpha == T(1);
    const bool tiled = alg.kernel == TC_KERNEL_GEMM;

    PhaseDesc pd;
    TileDesc td;
    int coop_g = 0;  // lanes per output of coop_reduce_kernel (0: elementwise_kernel)
    std::memset(&pd, 0, sizeof(pd));
    std::memset(&td, 0, sizeof(td));
    int64_t ntasks = 1;
    for (int id : L.task_ids) ntasks *= p.ext[id];
    if (tiled) {
        std::vector<int> mi{L.out_ids[0]}, ni{L.out_ids[1]};
        fill(td.m, mi);
        fill(td.n, ni);
        fill(td.red, L.red_ids);
        fill(td.task, L.task_ids);
        td.M = p.ext[L.out_ids[0]];
        td.N = p.ext[L.out_ids[1]];
        td.K = 1;
        for (int id : L.red_ids) td.K *= p.ext[id];
        td.alpha = alpha;
        td.beta = beta;
        td.alpha_one = alpha_one;
        // map threads along whichever of M / K is contiguous in memory
        int64_t kinA = td.red.n ? td.red.sA[td.red.n - 1] : 0;
        int64_t kinB = td.red.n ? td.red.sB[td.red.n - 1] : 0;
        td.a_m_fast = td.m.sA[0] <= kinA || kinA == 0;
        td.b_n_fast = td.n.sB[0] <= kinB || kinB == 0;
    } else {
        fill(pd.out, L.out_ids);
        fill(pd.task, L.task_ids);
        fill(pd.red, L.red_ids);
        int64_t nout = 1;
        for (int id : L.out_ids) nout *= p.ext[id];
        pd.total = nout * ntasks;
        pd.alpha = alpha;
        pd.beta = beta;
        pd.alpha_one = alpha_one;
        // Access pattern per kernel (Table 1 rows 1-4): one thread per
        // kernel output with consecutive threads along the output mode that
        // is contiguous in C (elementwise_kernel; ger's two output modes are
        // ordered so) -- axpy's vector and gemv's matrix with its free index
        // contiguous are then read coalesced; dot and gemv sum their own
        // contracted index in that thread.  When a phase has fewer outputs
        // than the device holds threads in one wave and its innermost
        // contracted index has unit stride in an input, a group of lanes per
        // output splits that index instead (coop_reduce_kernel, loads
        // contiguous across the group): the reduction, not the output count,
        // then sets the parallelism.
        const int kr = pd.red.n - 1;
        if (alg.kernel == TC_KERNEL_GER && pd.out.n == 2 && pd.out.sC[1] < pd.out.sC[0]) {
            std::swap(pd.out.ext[0], pd.out.ext[1]);
            std::swap(pd.out.sA[0], pd.out.sA[1]);
            std::swap(pd.out.sB[0], pd.out.sB[1]);
            std::swap(pd.out.sC[0], pd.out.sC[1]);
        }
        const bool k_unit = kr >= 0 && (pd.red.sA[kr] == 1 || pd.red.sB[kr] == 1);
        if (k_unit && pd.red.ext[kr] > 1 && pd.total < (int64_t)device_sms() * 1024) coop_g = 1;
        if (coop_g) {
            const int64_t kext = pd.red.ext[kr];
            coop_g = kext <= 4 ? 4 : (kext <= 8 ? 8 : (kext <= 16 ? 16 : 32));
        }
    }

    // C copy (reading for a C slice without a unit-stride mode): gather once,
    // run every phase on the workspace, scatter back at the end
    void *Cptr = C;
    tc_status s;
    const bool first_probe = !probe || probe->first;
    const double frac0 = probe ? probe->fraction : 1.0;
    if (L.view[OP_C].copied) {
        Cptr = ws + L.ws_offset[OP_C];
        if (init0 != 2 && first_probe) {
            s = launch_copy(p, OP_C, L.view[OP_C], base[OP_C], Cptr, false, st, frac0);
            if (s != TC_SUCCESS) return s;
        }
    }

    const int nph = (int)L.phase_pos.size();
    // one phase: its copies, then its kernel over `frac` of the work
    auto run_phase = [&](const std::vector<int64_t> &ph, bool first, int changed_from,
                         double frac) -> tc_status {
        // operand bases for this phase: fixed contracted indices applied
        const char *opb[2];
        for (int o = 0; o < 2; ++o) {
            int64_t off = 0;
            for (int k = 0; k < nph; ++k) off += ph[k] * p.op[o].stride_of(alg.loops[L.phase_pos[k]]);
            opb[o] = base[o] + off * (int64_t)esz;
        }
        const void *Aeff = opb[0], *Beff = opb[1];
        for (int o = 0; o < 2; ++o) {
            if (!L.view[o].copied) continue;
            void *dst = ws + L.ws_offset[o];
            int level = alg.copy_level[o];
            bool redo = first || level > alg.q;
            if (!redo) {
                for (int k = changed_from; k < nph; ++k)
                    if (L.phase_pos[k] <= level) redo = true;
            }
            if (redo) {
                tc_status cs = launch_copy(p, o, L.view[o], opb[o], dst, false, st, frac);
                if (cs != TC_SUCCESS) return cs;
            }
            if (o == 0) Aeff = dst;
            else Beff = dst;
        }
        const int init = first ? init0 : 0;
        auto cut = [&](int64_t n) { return frac >= 1.0 ? n : std::max<int64_t>(1, (int64_t)(n * frac)); };
        if (tiled && tensor) {
            NestGemm g;
            std::memset(&g, 0, sizeof(g));
            g.m = {td.m.ext[0], td.m.sA[0], 0, td.m.sC[0]};
            g.n = {td.n.ext[0], 0, td.n.sB[0], td.n.sC[0]};
            g.nk = td.red.n;
            for (int m = 0; m < td.red.n; ++m) g.k[m] = {td.red.ext[m], td.red.sA[m], td.red.sB[m], 0};
            g.nt = td.task.n;  // innermost task loop first (fastest)
            for (int m = 0; m < td.task.n; ++m) {
                const int x = td.task.n - 1 - m;
                g.t[m] = {td.task.ext[x], td.task.sA[x], td.task.sB[x], td.task.sC[x]};
            }
            g.A = Aeff;
            g.B = Beff;
            g.C = Cptr;
            g.alpha = (float)alpha;
            // init 0 (C += alpha acc, the later phases) is beta = 1
            g.init = init == 2 ? 2 : 1;
            g.beta = init == 1 ? (float)beta : 1.0f;
            return gett_launch_nest(p, g, frac, st);
        } else if (tiled) {
            td.A = Aeff;
            td.B = Beff;
            td.C = Cptr;
            td.init = init;
            if constexpr (sizeof(T) == 8) {
                constexpr int BM = 64, BN = 64;
                td.tiles_m = (td.M + BM - 1) / BM;
                td.tiles_n = (td.N + BN - 1) / BN;
                int64_t grid = cut(td.tiles_m * td.tiles_n * ntasks);
                tile_kernel<T, 64, 64, 16, 4, 4><<<(unsigned)grid, 256, 0, st>>>(td);
            } else {
                constexpr int BM = 128, BN = 128;
                td.tiles_m = (td.M + BM - 1) / BM;
                td.tiles_n = (td.N + BN - 1) / BN;
                int64_t grid = cut(td.tiles_m * td.tiles_n * ntasks);
                tile_kernel<T, 128, 128, 16, 8, 8><<<(unsigned)grid, 256, 0, st>>>(td);
            }
        } else {
            PhaseDesc q = pd;
            q.A = Aeff;
            q.B = Beff;
            q.C = Cptr;
            q.init = init;
            q.total = cut(pd.total);
            if (coop_g) {
                const int64_t grid = grid_for(q.total * coop_g, 256);
                switch (coop_g) {
                    case 4: coop_reduce_kernel<T, 4><<<(unsigned)grid, 256, 0, st>>>(q); break;
                    case 8: coop_reduce_kernel<T, 8><<<(unsigned)grid, 256, 0, st>>>(q); break;
                    case 16: coop_reduce_kernel<T, 16><<<(unsigned)grid, 256, 0, st>>>(q); break;
                    default: coop_reduce_kernel<T, 32><<<(unsigned)grid, 256, 0, st>>>(q); break;
                }
            } else {
                int64_t grid = grid_for(q.total, 256);
                elementwise_kernel<T><<<(unsigned)grid, 256, 0, st>>>(q);
            }
        }
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? TC_SUCCESS : fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    };

    if (probe) {
        std::vector<int64_t> ph(nph, 0);
        for (int k = 0; k < nph && k < (int)probe->phase.size(); ++k)
            ph[k] = std::min<int64_t>(probe->phase[k], p.ext[alg.loops[L.phase_pos[k]]] - 1);
        return run_phase(ph, probe->first, probe->changed_from, probe->fraction);
    }

    std::vector<int64_t> ph(nph, 0);
    bool first = true;
    int changed_from = 0;  // outermost phase digit that changed
    for (;;) {
        s = run_phase(ph, first, changed_from, 1.0);
        if (s != TC_SUCCESS) return s;
        first = false;
        // advance the phase odometer (innermost phase loop fastest)
        int k = nph - 1;
        while (k >= 0) {
            if (++ph[k] < p.ext[alg.loops[L.phase_pos[k]]]) break;
            ph[k] = 0;
            --k;
        }
        if (k < 0) break;
        changed_from = k;
    }
    if (L.view[OP_C].copied) {
        s = launch_copy(p, OP_C, L.view[OP_C], base[OP_C], Cptr, true, st);
        if (s != TC_SUCCESS) return s;
    }
    return TC_SUCCESS;
}

// SIMT GETT: the whole contraction as one tiled kernel, M = free indices
// of A, N = free indices of B, K = contracted indices.
// The SIMT GETT's descriptor: M = free indices of A, N = free indices of B
// (each sorted by their C stride), K = contracted indices with the one
// contiguous in A (or else in B) innermost; tiles of 64 x 64 (FP64) or
// 128 x 128 (FP32).
template <typename T>
void describe_gett_simt(const Plan &p, T alpha, const T *A, const T *B, T beta, T *C, TileDesc &td) {
    std::memset(&td, 0, sizeof(td));
    auto by_c_stride = [&](std::vector<int> ids) {
        std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) {
            return p.op[OP_C].stride_of(x) < p.op[OP_C].stride_of(y);
        });
        return ids;
    };
    std::vector<int> mi = by_c_stride(p.freeA), ni = by_c_stride(p.freeB);
    // K: the contracted index contiguous in A (or else in B) innermost
    std::vector<int> ki(p.contracted);
    std::stable_sort(ki.begin(), ki.end(), [&](int x, int y) {
        int64_t mx = std::min(p.op[OP_A].stride_of(x), p.op[OP_B].stride_of(x));
        int64_t my = std::min(p.op[OP_A].stride_of(y), p.op[OP_B].stride_of(y));
        return mx > my;
    });
    auto fill = [&](Dims &d, const std::vector<int> &ids) {
        d.n = 0;
        for (int id : ids)
            add_dim(d, p.ext[id], p.op[OP_A].stride_of(id), p.op[OP_B].stride_of(id),
                    p.op[OP_C].stride_of(id));
    };
    fill(td.m, mi);
    fill(td.n, ni);
    fill(td.red, ki);
    fill(td.task, p.batch);  // batch indices: one task per value, all three operands offset
    td.M = td.N = td.K = 1;
    for (int id : mi) td.M *= p.ext[id];
    for (int id : ni) td.N *= p.ext[id];
    for (int id : ki) td.K *= p.ext[id];
    td.A = A;
    td.B = B;
    td.C = C;
    td.alpha = alpha;
    td.beta = beta;
    td.alpha_one = alpha == T(1);
    td.init = beta == T(0) ? 2 : (beta == T(1) ? 0 : 1);
    int64_t kinA = td.red.n ? td.red.sA[td.red.n - 1] : 0;
    int64_t kinB = td.red.n ? td.red.sB[td.red.n - 1] : 0;
    td.a_m_fast = td.m.n ? (td.m.sA[0] <= kinA || kinA == 0) : 0;
    td.b_n_fast = td.n.n ? (td.n.sB[0] <= kinB || kinB == 0) : 0;
    const int64_t bm = sizeof(T) == 8 ? 64 : 128;
    td.tiles_m = (td.M + bm - 1) / bm;
    td.tiles_n = (td.N + bm - 1) / bm;
}

int64_t task_count(const TileDesc &td) {
    int64_t t = 1;
    for (int m = 0; m < td.task.n; ++m) t *= td.task.ext[m];
    return t;
}

template <typename T>
tc_status run_gett_simt(Plan &p, T alpha, const T *A, const T *B, T beta, T *C,
                        cudaStream_t st, const Probe *probe) {
    TileDesc td;
    describe_gett_simt<T>(p, alpha, A, B, beta, C, td);
    auto cut = [&](int64_t n) {
        return !probe || probe->fraction >= 1.0 ? n : std::max<int64_t>(1, (int64_t)(n * probe->fraction));
    };
    const int64_t tiles = td.tiles_m * td.tiles_n * task_count(td);
    if (tiles > 0x7fffffff) return fail(TC_ERROR_INVALID_EXTENT, "too many tiles for one launch");
    if constexpr (sizeof(T) == 8)
        tile_kernel<T, 64, 64, 16, 4, 4><<<(unsigned)cut(tiles), 256, 0, st>>>(td);
    else
        tile_kernel<T, 128, 128, 16, 8, 8><<<(unsigned)cut(tiles), 256, 0, st>>>(td);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TC_SUCCESS
                            : fail(TC_ERROR_CUDA, std::string("GETT tile_kernel launch (") +
                                                      std::to_string(td.tiles_m * td.tiles_n) + " tiles): " +
                                                      cudaGetErrorString(e));
}

}  // namespace

size_t simt_desc_bytes() { return sizeof(TileDesc); }

int64_t simt_fill_desc(const Plan &p, const void *A, const void *B, void *C, int64_t tile0, void *out) {
    TileDesc td;
    if (p.dtype == TC_F64)
        describe_gett_simt<double>(p, 1.0, (const double *)A, (const double *)B, 0.0, (double *)C, td);
    else
        describe_gett_simt<float>(p, 1.0f, (const float *)A, (const float *)B, 0.0f, (float *)C, td);
    td.tile0 = tile0;
    std::memcpy(out, &td, sizeof(td));
    return td.tiles_m * td.tiles_n * task_count(td);
}

tc_status simt_launch_batch(tc_dtype dt, const void *ddescs, const int32_t *dtile_prob, int64_t ntiles,
                            void *stream) {
    if (ntiles <= 0) return TC_SUCCESS;
    if (ntiles > 0x7fffffff) return fail(TC_ERROR_INVALID_ARGUMENT, "batch has too many tiles");
    cudaStream_t st = (cudaStream_t)stream;
    if (dt == TC_F64)
        tile_batch_kernel<double, 64, 64, 16, 4, 4>
            <<<(unsigned)ntiles, 256, 0, st>>>((const TileDesc *)ddescs, dtile_prob);
    else
        tile_batch_kernel<float, 128, 128, 16, 8, 8>
            <<<(unsigned)ntiles, 256, 0, st>>>((const TileDesc *)ddescs, dtile_prob);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TC_SUCCESS : fail(TC_ERROR_CUDA, cudaGetErrorString(e));
}

int64_t nest_phase_items(const Plan &p, const Algorithm &alg, bool *tiled) {
    NestLayout L = layout_for(p, alg);
    int64_t ntasks = 1;
    for (int id : L.task_ids) ntasks *= p.ext[id];
    if (alg.kernel == TC_KERNEL_GEMM) {
        *tiled = true;
        const int64_t bm = p.dtype == TC_F64 ? 64 : 128;
        return ((p.ext[L.out_ids[0]] + bm - 1) / bm) * ((p.ext[L.out_ids[1]] + bm - 1) / bm) * ntasks;
    }
    *tiled = false;
    int64_t nout = 1;
    for (int id : L.out_ids) nout *= p.ext[id];
    return nout * ntasks;
}

int64_t gett_items(const Plan &p) {
    int64_t M = 1, N = 1, H = 1;
    for (int id : p.freeA) M *= p.ext[id];
    for (int id : p.freeB) N *= p.ext[id];
    for (int id : p.batch) H *= p.ext[id];
    if (p.dtype == TC_F64) return ((M + 63) / 64) * ((N + 63) / 64) * H;
    if (p.dtype == TC_F32) return ((M + 127) / 128) * ((N + 127) / 128) * H;
    const int64_t bn = p.gett_bn ? p.gett_bn : (N >= 256 ? 256 : 128);
    return ((M + 127) / 128) * ((N + bn - 1) / bn) * H;
}

size_t nest_workspace_bytes(const Plan &p, const Algorithm &alg) {
    return layout_for(p, alg).ws_bytes;
}

tc_status ensure_device_resources(Plan &p, size_t workspace_bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    if (p.device < 0) {
        p.device = dev;
    } else if (p.device != dev) {
        return fail(TC_ERROR_INVALID_ARGUMENT, "plan used on a different device than its first execute");
    }
    if (!p.dev_status) {
        e = cudaMalloc((void **)&p.dev_status, sizeof(int) * 4);
        if (e != cudaSuccess) return fail(TC_ERROR_OUT_OF_MEMORY, cudaGetErrorString(e));
        cudaMemset(p.dev_status, 0, sizeof(int) * 4);
    }
    if (workspace_bytes > p.workspace_bytes) {
        if (p.workspace) cudaFree(p.workspace);
        p.workspace = nullptr;
        p.workspace_bytes = 0;
        e = cudaMalloc(&p.workspace, workspace_bytes);
        if (e != cudaSuccess) {
            p.workspace = nullptr;
            return fail(TC_ERROR_OUT_OF_MEMORY, cudaGetErrorString(e));
        }
        p.workspace_bytes = workspace_bytes;
    }
    return TC_SUCCESS;
}

tc_status exec_nest(Plan &p, const Algorithm &alg, const void *alpha, const void *A,
                    const void *B, const void *beta, void *C, void *stream, const Probe *probe) {
    if (p.dtype != TC_F64 && p.dtype != TC_F32 && alg.kernel != TC_KERNEL_GEMM)
        return fail(TC_ERROR_UNSUPPORTED_DTYPE,
                    "at tensor-core dtypes only the gemm loop nests (on the tensor cores) and the GETT run; "
                    "dot / axpy / gemv / ger nests run in FP64 or FP32");
    if (p.dtype == TC_E4M3)
        return fail(TC_ERROR_UNSUPPORTED_DTYPE, "TC_E4M3 runs the fused GETT (algorithm 0) only");
    tc_status s = ensure_device_resources(p, nest_workspace_bytes(p, alg));
    if (s != TC_SUCCESS) return s;
    p.last_stream = stream;
    cudaStream_t st = (cudaStream_t)stream;
    if (p.dtype == TC_F64)
        return run_nest<double>(p, alg, *(const double *)alpha, (const double *)A,
                                (const double *)B, *(const double *)beta, (double *)C, st, probe);
    return run_nest<float>(p, alg, *(const float *)alpha, (const float *)A, (const float *)B,
                           *(const float *)beta, (float *)C, st, probe);
}

tc_status exec_gett_simt(Plan &p, const void *alpha, const void *A, const void *B,
                         const void *beta, void *C, void *stream, const Probe *probe) {
    tc_status s = ensure_device_resources(p, 0);
    if (s != TC_SUCCESS) return s;
    p.last_stream = stream;
    cudaStream_t st = (cudaStream_t)stream;
    if (p.dtype == TC_F64)
        return run_gett_simt<double>(p, *(const double *)alpha, (const double *)A,
                                     (const double *)B, *(const double *)beta, (double *)C, st, probe);
    return run_gett_simt<float>(p, *(const float *)alpha, (const float *)A, (const float *)B,
                                *(const float *)beta, (float *)C, st, probe);
}

}  // namespace tc

// ---------------------------------------------------------------- no-alloc entry point
// A variant of the loop-nest executor whose copy workspace lives in a fixed
// device array instead of memory the plan allocates.  The paper has no
// counterpart; it serves callers that must not allocate device memory.
namespace tc {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB per device
constexpr int kMaxDevices = 64;

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (host code cannot use the symbol itself as a device pointer).
tc_status static_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(TC_ERROR_INVALID_ARGUMENT, "device ordinal too large");
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) return fail(TC_ERROR_CUDA, e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address");
        g_static_ptr[dev] = ptr;
    }
    *out = g_static_ptr[dev];
    return TC_SUCCESS;
}

}  // namespace
}  // namespace tc

extern "C" tc_status tc_execute_no_alloc(tc_plan plan, const void *alpha, const void *A, const void *B,
                                         const void *beta, void *C, void *stream) {
    using namespace tc;
    if (!plan) return fail(TC_ERROR_INVALID_ARGUMENT, "plan is NULL");
    if (!alpha || !beta || !A || !B || !C) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    Plan &p = plan->p;
    if (p.dtype != TC_F64 && p.dtype != TC_F32)
        return fail(TC_ERROR_UNSUPPORTED_DTYPE, "tc_execute_no_alloc runs the FP64/FP32 loop-nest algorithms");
    const Algorithm &alg = p.algs[p.selected];
    if (alg.kernel == TC_KERNEL_GETT)
        return fail(TC_ERROR_INVALID_ALGORITHM, "tc_execute_no_alloc runs the loop-nest algorithms (ids >= 1)");
    const size_t need = nest_workspace_bytes(p, alg);
    if (need > kStaticScratchBytes)
        return fail(TC_ERROR_INVALID_ARGUMENT,
                    "algorithm needs " + std::to_string(need) + " bytes of copy scratch; the static scratch holds " +
                        std::to_string(kStaticScratchBytes) + " bytes (use tc_execute)");
    void *scratch = nullptr;
    tc_status s = static_scratch(&scratch);
    if (s != TC_SUCCESS) return s;
    // run the same executor with the workspace pointed at the static array
    void *saved = p.workspace;
    const size_t saved_bytes = p.workspace_bytes;
    p.workspace = scratch;
    p.workspace_bytes = kStaticScratchBytes;
    cudaStream_t st = (cudaStream_t)stream;
    if (p.dtype == TC_F64)
        s = run_nest<double>(p, alg, *(const double *)alpha, (const double *)A, (const double *)B,
                             *(const double *)beta, (double *)C, st, nullptr);
    else
        s = run_nest<float>(p, alg, *(const float *)alpha, (const float *)A, (const float *)B,
                            *(const float *)beta, (float *)C, st, nullptr);
    p.workspace = saved;
    p.workspace_bytes = saved_bytes;
    return s;
}
