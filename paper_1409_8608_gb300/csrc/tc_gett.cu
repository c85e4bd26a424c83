// Fused GETT (algorithm 0): the whole contraction in one kernel, with no
// paper counterpart.  M = free indices of A, N = free indices of B,
// K = contracted indices; C tile = M x N, K loops over every contracted
// index.  FP64 / FP32 run the SIMT tiled form (tc_exec.cu); the tensor-core
// dtypes run here on the 5th-generation tensor cores:
//
//   producer warps 0-7   load A/B tiles from global memory through the
//                        operands' own strides (no transpose pass, any
//                        permutation), convert or split them and store the
//                        canonical no-swizzle K-major core-matrix layout
//                        (8 rows x 16 bytes per core matrix) in shared memory;
//   MMA warp 8           one elected thread issues tcgen05.mma (kind::f16 for
//                        BF16/FP16 and the split-BF16 slices, kind::tf32) into
//                        an FP32 accumulator in tensor memory, and signals
//                        stage reuse / completion with tcgen05.commit;
//   epilogue warps 0-7   tcgen05.ld the accumulator, apply alpha and beta*C
//                        and store FP32 C.
//
// Split-BF16 ("BF16X3"): each FP32 input x is split into three BF16 slices
// x = h0 + h1 + h2 (h0 = rn(x), h1 = rn(x - h0), h2 = rn(x - h0 - h1)); the
// kept slice products are ordered by weight: 3 products keep (0,0) (0,1)
// (1,0); 6 add (0,2) (1,1) (2,0); 9 add (1,2) (2,1) (2,2).
//
// Every wait on an mbarrier is bounded (%globaltimer); on expiry the kernel
// records TC_ERROR_TIMEOUT in the plan's status word, stops issuing work,
// drains what it issued, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "tc_internal.h"

namespace tc {

tc_status exec_gett_simt(Plan &p, const void *alpha, const void *A, const void *B,
                         const void *beta, void *C, void *stream);

namespace {

enum GettKind { GK_BF16X3 = 0, GK_BF16 = 1, GK_F16 = 2, GK_TF32 = 3 };

constexpr int kBM = 128;                  // accumulator rows = TMEM lanes
constexpr int kBK = 32;                   // K elements per pipeline stage
constexpr int kProducerWarps = 8;
constexpr int kProducerThreads = kProducerWarps * 32;
constexpr int kMmaWarp = kProducerWarps;  // warp 8
constexpr int kThreads = kProducerThreads + 32;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

struct GettDesc {
    int nm, nn, nk;                       // number of M / N / K modes
    int64_t m_ext[kMaxModes], m_sA[kMaxModes], m_sC[kMaxModes];
    int64_t n_ext[kMaxModes], n_sB[kMaxModes], n_sC[kMaxModes];
    int64_t k_ext[kMaxModes], k_sA[kMaxModes], k_sB[kMaxModes];  // outermost first
    int64_t M, N, K;
    int64_t tiles_m, tiles_n;
    const void *A;
    const void *B;
    float *C;
    float alpha, beta;
    int init;         // 1: C = alpha*acc + beta*C, 2: C = alpha*acc
    int a_kfast, b_kfast;
    int nprod;        // split products (BF16X3)
    int *status;
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false when the limit expired.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > kWaitLimitNs) return false;
    }
    return true;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Producer-only barrier that also ORs a predicate across the producers.
__device__ __forceinline__ bool producers_sync_or(bool pred) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.cta.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(out)
        : "r"((uint32_t)pred), "n"(kProducerThreads)
        : "memory");
    return out != 0;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor, no swizzle, K-major: core matrices of
// 8 rows x 16 bytes; lbo = byte distance between core matrices adjacent in
// K, sbo = byte distance between adjacent 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, swizzle none
}

template <int KIND>
__device__ __forceinline__ void mma_issue(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    if constexpr (KIND == GK_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// ------------------------------------------------------------------ layout
template <int KIND>
struct KindTraits {
    static constexpr int kElemBytes = KIND == GK_TF32 ? 4 : 2;  // smem operand element
    static constexpr int kSlices = KIND == GK_BF16X3 ? 3 : 1;
    static constexpr int kChunk = 16 / kElemBytes;              // K elements per 16-byte row
    static constexpr int kKc = kBK / kChunk;                    // core matrices along K per stage
    static constexpr int kKsteps = kBK * kElemBytes / 32;       // MMA instructions along K per stage
    static constexpr uint32_t kFmt = KIND == GK_TF32 ? 2u : (KIND == GK_F16 ? 0u : 1u);
    using In = typename std::conditional<KIND == GK_BF16 ? true : false, __nv_bfloat16,
                                         typename std::conditional<KIND == GK_F16, __half, float>::type>::type;
};

template <int KIND, int BN, int STAGES>
struct SmemPlan {
    using T = KindTraits<KIND>;
    static constexpr int kATile = kBM * kBK * T::kElemBytes;   // one slice
    static constexpr int kBTile = BN * kBK * T::kElemBytes;
    static constexpr int kStage = T::kSlices * (kATile + kBTile);
    static constexpr int kOpBytes = STAGES * kStage;
    static constexpr int kKTab = STAGES * kBK * 8 * 2;
    static constexpr int kRowTab = (kBM + BN) * 8 * 2;
    static constexpr int kBars = (2 * STAGES + 1) * 8 + 16;
    static constexpr int kTotal = kOpBytes + kKTab + kRowTab + kBars;
};

__device__ __forceinline__ void decode(int64_t x, int n, const int64_t *ext, const int64_t *s1,
                                       const int64_t *s2, int64_t &o1, int64_t &o2) {
    // first mode fastest
    for (int m = 0; m < n; ++m) {
        int64_t v = x % ext[m];
        x /= ext[m];
        o1 += v * s1[m];
        o2 += v * s2[m];
    }
}

// Loads CH consecutive K elements of one operand row and writes the
// converted / split 16-byte rows into every slice.
template <int KIND>
__device__ __forceinline__ void produce_chunk(const typename KindTraits<KIND>::In *__restrict__ src,
                                              int64_t rowoff, const int64_t *koff, char *dst,
                                              int slice_stride) {
    using T = KindTraits<KIND>;
    constexpr int CH = T::kChunk;
    if constexpr (KIND == GK_BF16X3) {
        float x[CH];
#pragma unroll
        for (int e = 0; e < CH; ++e) {
            int64_t ko = koff[e];
            x[e] = (rowoff >= 0 && ko >= 0) ? __ldg(src + rowoff + ko) : 0.0f;
        }
        uint32_t w0[CH / 2], w1[CH / 2], w2[CH / 2];
#pragma unroll
        for (int e = 0; e < CH; e += 2) {
            __nv_bfloat16 h0a = __float2bfloat16_rn(x[e]);
            float r1a = x[e] - __bfloat162float(h0a);
            __nv_bfloat16 h1a = __float2bfloat16_rn(r1a);
            __nv_bfloat16 h2a = __float2bfloat16_rn(r1a - __bfloat162float(h1a));
            __nv_bfloat16 h0b = __float2bfloat16_rn(x[e + 1]);
            float r1b = x[e + 1] - __bfloat162float(h0b);
            __nv_bfloat16 h1b = __float2bfloat16_rn(r1b);
            __nv_bfloat16 h2b = __float2bfloat16_rn(r1b - __bfloat162float(h1b));
            w0[e / 2] = pack_bf16(h0a, h0b);
            w1[e / 2] = pack_bf16(h1a, h1b);
            w2[e / 2] = pack_bf16(h2a, h2b);
        }
        *(uint4 *)(dst) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        *(uint4 *)(dst + slice_stride) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *(uint4 *)(dst + 2 * slice_stride) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
    } else if constexpr (KIND == GK_TF32) {
        uint32_t w[CH];
#pragma unroll
        for (int e = 0; e < CH; ++e) {
            int64_t ko = koff[e];
            float v = (rowoff >= 0 && ko >= 0) ? __ldg(src + rowoff + ko) : 0.0f;
            w[e] = f32_to_tf32(v);
        }
        *(uint4 *)(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
        unsigned short h[CH];
#pragma unroll
        for (int e = 0; e < CH; ++e) {
            int64_t ko = koff[e];
            const unsigned short *s16 = (const unsigned short *)src;
            h[e] = (rowoff >= 0 && ko >= 0) ? __ldg(s16 + rowoff + ko) : (unsigned short)0;
        }
        uint32_t w[CH / 2];
#pragma unroll
        for (int e = 0; e < CH; e += 2) w[e / 2] = (uint32_t)h[e] | ((uint32_t)h[e + 1] << 16);
        *(uint4 *)(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

template <int KIND, int BN, int STAGES>
__global__ void __launch_bounds__(kThreads, 1) gett_tc_kernel(const GettDesc d) {
    using T = KindTraits<KIND>;
    using SP = SmemPlan<KIND, BN, STAGES>;
    using In = typename T::In;
    extern __shared__ __align__(1024) char smem[];
    char *ops = smem;
    int64_t *kA = (int64_t *)(smem + SP::kOpBytes);          // [STAGES][kBK]
    int64_t *kB = kA + STAGES * kBK;
    int64_t *rowA = kB + STAGES * kBK;                        // [kBM]
    int64_t *cM = rowA + kBM;
    int64_t *rowB = cM + kBM;                                 // [BN]
    int64_t *cN = rowB + BN;
    uint64_t *full = (uint64_t *)(cN + BN);
    uint64_t *empty = full + STAGES;
    uint64_t *accum = empty + STAGES;
    uint32_t *tmem_slot = (uint32_t *)(accum + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t tile_m = blockIdx.x % d.tiles_m;
    const int64_t tile_n = blockIdx.x / d.tiles_m;
    const int64_t m0 = tile_m * kBM, n0 = tile_n * BN;
    const int nkt = (int)((d.K + kBK - 1) / kBK);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], kProducerThreads);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kMmaWarp) tmem_alloc(tmem_slot, BN);
    // row tables
    for (int i = threadIdx.x; i < kBM; i += kThreads) {
        int64_t mm = m0 + i, oa = -1, oc = -1;
        if (mm < d.M) {
            oa = 0;
            oc = 0;
            decode(mm, d.nm, d.m_ext, d.m_sA, d.m_sC, oa, oc);
        }
        rowA[i] = oa;
        cM[i] = oc;
    }
    for (int j = threadIdx.x; j < BN; j += kThreads) {
        int64_t nn = n0 + j, ob = -1, oc = -1;
        if (nn < d.N) {
            ob = 0;
            oc = 0;
            decode(nn, d.nn, d.n_ext, d.n_sB, d.n_sC, ob, oc);
        }
        rowB[j] = ob;
        cN[j] = oc;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < kProducerWarps) {
        // ---------------------------------------------------------- producers
        const int pt = threadIdx.x;
        const In *__restrict__ Ap = (const In *)d.A;
        const In *__restrict__ Bp = (const In *)d.B;
        constexpr int KC = T::kKc, CH = T::kChunk;
        for (int t = 0; t < nkt; ++t) {
            const int s = t % STAGES;
            bool bad = false;
            if (t >= STAGES) bad = !mbar_wait(&empty[s], ((t / STAGES) - 1) & 1);
            if (pt < kBK) {
                int64_t k = (int64_t)t * kBK + pt, oa = -1, ob = -1;
                if (k < d.K) {
                    oa = 0;
                    ob = 0;
                    // K modes outermost first: innermost mode fastest
                    for (int m = d.nk - 1; m >= 0; --m) {
                        int64_t v = k % d.k_ext[m];
                        k /= d.k_ext[m];
                        oa += v * d.k_sA[m];
                        ob += v * d.k_sB[m];
                    }
                }
                kA[s * kBK + pt] = oa;
                kB[s * kBK + pt] = ob;
            }
            if (producers_sync_or(bad || *abort_flag)) {
                if (pt == 0) {
                    *abort_flag = 1;
                    atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
                }
                break;
            }
            char *stage = ops + s * SP::kStage;
            // A rows
            for (int c = pt; c < kBM * KC; c += kProducerThreads) {
                int row, kc;
                if (d.a_kfast) { row = c / KC; kc = c % KC; }
                else { row = c % kBM; kc = c / kBM; }
                char *dst = stage + (kc * (kBM / 8) + row / 8) * 128 + (row % 8) * 16;
                produce_chunk<KIND>(Ap, rowA[row], kA + s * kBK + kc * CH, dst, SP::kATile);
            }
            // B rows
            char *bst = stage + T::kSlices * SP::kATile;
            for (int c = pt; c < BN * KC; c += kProducerThreads) {
                int row, kc;
                if (d.b_kfast) { row = c / KC; kc = c % KC; }
                else { row = c % BN; kc = c / BN; }
                char *dst = bst + (kc * (BN / 8) + row / 8) * 128 + (row % 8) * 16;
                produce_chunk<KIND>(Bp, rowB[row], kB + s * kBK + kc * CH, dst, SP::kBTile);
            }
            fence_proxy_async_smem();
            mbar_arrive(&full[s]);
        }
    } else if (lane == 0) {
        // ---------------------------------------------------------- MMA issuer
        constexpr uint32_t idesc = (1u << 4) | (T::kFmt << 7) | (T::kFmt << 10) |
                                   ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
        constexpr uint32_t lboA = (kBM / 8) * 128, lboB = (BN / 8) * 128;
        const int pa[9] = {0, 0, 1, 0, 1, 2, 1, 2, 2};
        const int pb[9] = {0, 1, 0, 2, 1, 0, 2, 1, 2};
        const int nprod = KIND == GK_BF16X3 ? d.nprod : 1;
        const uint32_t base = smem_u32(ops);
        for (int t = 0; t < nkt; ++t) {
            const int s = t % STAGES;
            if (*abort_flag || !mbar_wait(&full[s], (t / STAGES) & 1)) {
                *abort_flag = 1;
                atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
                break;
            }
            tc_fence_after();
            const uint32_t sa = base + s * SP::kStage;
            const uint32_t sb = sa + T::kSlices * SP::kATile;
#pragma unroll
            for (int ks = 0; ks < T::kKsteps; ++ks) {
                for (int q = 0; q < nprod; ++q) {
                    uint64_t ad = smem_desc(sa + pa[q] * SP::kATile + ks * 2 * lboA, lboA, 128);
                    uint64_t bd = smem_desc(sb + pb[q] * SP::kBTile + ks * 2 * lboB, lboB, 128);
                    mma_issue<KIND>(tmem, ad, bd, idesc, (t | ks | q) != 0);
                }
            }
            mma_commit(&empty[s]);
        }
        mma_commit(accum);  // fires once every issued MMA has completed
    }

    // -------------------------------------------------------------- epilogue
    if (warp < kProducerWarps) {
        const bool ok = mbar_wait(accum, 0);
        if (!ok) {
            *abort_flag = 1;
            atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
        }
        tc_fence_after();
        if (ok && !*abort_flag) {
            const int quarter = warp % 4, half = warp / 4;
            const int row = quarter * 32 + lane;
            const int64_t om = cM[row];
            float *__restrict__ C = d.C;
            for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, r);
                if (om >= 0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int64_t on = cN[c0 + j];
                        if (on < 0) continue;
                        float v = d.alpha * __uint_as_float(r[j]);
                        if (d.init == 1) v = fmaf(d.beta, C[om + on], v);
                        C[om + on] = v;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem, BN);
    }
}

// ------------------------------------------------------------------ host side
template <int KIND, int BN, int STAGES>
tc_status launch_gett(const GettDesc &d, cudaStream_t st) {
    using SP = SmemPlan<KIND, BN, STAGES>;
    static_assert(SP::kTotal <= 227 * 1024, "shared memory budget");
    auto kern = gett_tc_kernel<KIND, BN, STAGES>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SP::kTotal);
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    int64_t grid = d.tiles_m * d.tiles_n;
    if (grid > 0x7FFFFFFF) return fail(TC_ERROR_INVALID_EXTENT, "too many GETT tiles");
    kern<<<(unsigned)grid, kThreads, SP::kTotal, st>>>(d);
    e = cudaGetLastError();
    return e == cudaSuccess ? TC_SUCCESS : fail(TC_ERROR_CUDA, cudaGetErrorString(e));
}

template <int KIND>
tc_status launch_kind(GettDesc &d, int bn, cudaStream_t st) {
    if (bn == 256) {
        d.tiles_n = (d.N + 255) / 256;
        if constexpr (KIND == GK_BF16X3) return launch_gett<KIND, 256, 2>(d, st);
        else return launch_gett<KIND, 256, 4>(d, st);
    }
    d.tiles_n = (d.N + 127) / 128;
    if constexpr (KIND == GK_BF16X3) return launch_gett<KIND, 128, 4>(d, st);
    else return launch_gett<KIND, 128, 6>(d, st);
}

}  // namespace

size_t gett_workspace_bytes(const Plan &) { return 0; }

void gett_release(Plan &) {}

tc_status exec_gett(Plan &p, const void *alpha, const void *A, const void *B, const void *beta,
                    void *C, void *stream) {
    if (p.dtype == TC_F64 || p.dtype == TC_F32) return exec_gett_simt(p, alpha, A, B, beta, C, stream);
    tc_status s = ensure_device_resources(p, 0);
    if (s != TC_SUCCESS) return s;
    p.last_stream = stream;
    GettDesc d;
    std::memset(&d, 0, sizeof(d));
    auto by_c_stride = [&](std::vector<int> ids) {
        std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) {
            return p.op[OP_C].stride_of(x) < p.op[OP_C].stride_of(y);
        });
        return ids;
    };
    std::vector<int> mi = by_c_stride(p.freeA), ni = by_c_stride(p.freeB);
    // K order: the innermost K mode is the contracted index with the smallest
    // stride in the larger input, so that operand streams along K
    int64_t sizeA = 1, sizeB = 1;
    for (int m = 0; m < p.op[OP_A].n; ++m) sizeA *= p.ext[p.op[OP_A].idx[m]];
    for (int m = 0; m < p.op[OP_B].n; ++m) sizeB *= p.ext[p.op[OP_B].idx[m]];
    const int big = sizeB >= sizeA ? OP_B : OP_A;
    std::vector<int> ki(p.contracted);
    std::stable_sort(ki.begin(), ki.end(), [&](int x, int y) {
        return p.op[big].stride_of(x) > p.op[big].stride_of(y);
    });
    d.nm = (int)mi.size();
    d.nn = (int)ni.size();
    d.nk = (int)ki.size();
    d.M = d.N = d.K = 1;
    for (int m = 0; m < d.nm; ++m) {
        int id = mi[m];
        d.m_ext[m] = p.ext[id];
        d.m_sA[m] = p.op[OP_A].stride_of(id);
        d.m_sC[m] = p.op[OP_C].stride_of(id);
        d.M *= p.ext[id];
    }
    for (int m = 0; m < d.nn; ++m) {
        int id = ni[m];
        d.n_ext[m] = p.ext[id];
        d.n_sB[m] = p.op[OP_B].stride_of(id);
        d.n_sC[m] = p.op[OP_C].stride_of(id);
        d.N *= p.ext[id];
    }
    for (int m = 0; m < d.nk; ++m) {
        int id = ki[m];
        d.k_ext[m] = p.ext[id];
        d.k_sA[m] = p.op[OP_A].stride_of(id);
        d.k_sB[m] = p.op[OP_B].stride_of(id);
        d.K *= p.ext[id];
    }
    const int64_t kinA = d.nk ? d.k_sA[d.nk - 1] : 1, kinB = d.nk ? d.k_sB[d.nk - 1] : 1;
    const int64_t rowA = d.nm ? d.m_sA[0] : INT64_MAX, rowB = d.nn ? d.n_sB[0] : INT64_MAX;
    d.a_kfast = kinA <= rowA;
    d.b_kfast = kinB <= rowB;
    d.A = A;
    d.B = B;
    d.C = (float *)C;
    d.alpha = *(const float *)alpha;
    d.beta = *(const float *)beta;
    d.init = d.beta == 0.0f ? 2 : 1;
    d.nprod = p.split_products;
    d.status = p.dev_status;
    d.tiles_m = (d.M + kBM - 1) / kBM;
    const int bn = d.N >= 256 ? 256 : 128;
    cudaStream_t st = (cudaStream_t)stream;
    switch (p.dtype) {
    case TC_BF16X3: return launch_kind<GK_BF16X3>(d, bn, st);
    case TC_BF16: return launch_kind<GK_BF16>(d, bn, st);
    case TC_F16: return launch_kind<GK_F16>(d, bn, st);
    case TC_TF32: return launch_kind<GK_TF32>(d, bn, st);
    default: return fail(TC_ERROR_UNSUPPORTED_DTYPE, "dtype has no tensor-core GETT");
    }
}

}  // namespace tc
