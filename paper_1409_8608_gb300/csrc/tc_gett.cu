// Fused GETT (algorithm 0): the whole contraction in one kernel, with no
// paper counterpart.  M = free indices of A, N = free indices of B,
// K = contracted indices; C tile = M x N, K loops over every contracted
// index.  FP64 / FP32 run the SIMT tiled form (tc_exec.cu); the tensor-core
// dtypes run here on the 5th-generation tensor cores:
//
// The kernel is persistent (one CTA per SM walks the tile list, M tiles
// fastest so that CTAs sharing a B tile run together) and warp-specialised:
//
//   TMA warp 13          streams each operand's box (tile rows x 16 or 32 K
//                        positions, one or two K stages, any permutation of
//                        the operand's modes, described by a CUtensorMap over
//                        its own strides: no transpose pass) into a staging
//                        ring with cp.async.bulk.tensor and mbarrier
//                        transaction counts;
//   converter warps 4-11 convert or split the staged inputs (or, for an
//                        operand TMA cannot describe, load it straight from
//                        global memory through its strides) and store the
//                        canonical no-swizzle K-major core-matrix layout
//                        (8 rows x 16 bytes per core matrix) in a ring of
//                        16-K operand stages; with both operands staged they
//                        work as two groups of four taking alternate stages;
//   MMA warp 12          one elected thread issues tcgen05.mma (kind::f16 for
//                        BF16/FP16 and the split-BF16 slices, kind::tf32) into
//                        one of two FP32 accumulators in tensor memory, and
//                        signals stage reuse / tile completion with
//                        tcgen05.commit;
//   epilogue warps 0-3   tcgen05.ld the finished accumulator, apply alpha and
//                        beta*C and store FP32 C while the MMA warp already
//                        fills the other accumulator.
//
// Split-BF16 ("BF16X3"): each FP32 input x is split into three BF16 slices
// x = h0 + h1 + h2 exactly (h0 = rn(x); h1 = x - h0 truncated to BF16;
// h2 = the rest, itself a BF16 value: see split3x2); the
// kept slice products are ordered by weight: 3 products keep (0,0) (0,1)
// (1,0); 6 add (0,2) (1,1) (2,0); 9 add (1,2) (2,1) (2,2).
//
// Every wait on an mbarrier is bounded (%globaltimer); on expiry the kernel
// records TC_ERROR_TIMEOUT in the plan's status word, stops issuing work,
// drains what it issued, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "tc_internal.h"
#include "tc_tcgen05.cuh"

namespace tc {

namespace {

using namespace dev;

enum GettKind { GK_BF16X3 = 0, GK_BF16 = 1, GK_F16 = 2, GK_TF32 = 3, GK_TF32X3 = 4, GK_E4M3 = 5 };

// MMA on TF32 words (kind::tf32, 4-byte operand elements)
__host__ __device__ constexpr bool tf32_kind(int k) { return k == GK_TF32 || k == GK_TF32X3; }
// FP32 inputs, converted (or split) by the converter warps
__host__ __device__ constexpr bool float_input(int k) {
    return k == GK_BF16X3 || k == GK_TF32 || k == GK_TF32X3 || k == GK_E4M3;
}

constexpr int kBM = 128;                  // accumulator rows = TMEM lanes
constexpr int kBK = 32;                   // K elements per stage, global-load path
constexpr int kBKT = 16;                  // K elements per stage, TMA path
constexpr int kBoxK = 32;                 // most K positions one TMA box covers (two stages)
constexpr int64_t kTwoStageBoxMinK = 128; // shorter K keeps one-stage boxes (finer refill of the ring)
constexpr int64_t kCompChunkK = 256;      // default K chunk of the compensated split-BF16 form
constexpr int kConvGroups = 2;            // converter groups taking turns (TMA-staged operands)
constexpr int64_t kPackMaxBytes = int64_t(64) << 20;  // largest pre-converted input
constexpr int64_t kPackBothMaxBytes = int64_t(2) << 30;  // both inputs pre-converted: their images
constexpr int64_t kPackBothMinMN = 1024;                   // auto: both inputs pre-converted from these M, N
constexpr int kPackRatio = 8;             // auto: the smaller input has <= 1/8 the elements
constexpr int kEpiWarps = 4;              // warps 0-3
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kProducerWarps = 8;         // warps 4-11
constexpr int kProducerThreads = kProducerWarps * 32;
constexpr int kMmaWarp = kEpiWarps + kProducerWarps;  // warp 12
constexpr int kTmaWarp = kMmaWarp + 1;                // warp 13
constexpr int kThreads = (kTmaWarp + 1) * 32;
constexpr int kTmaRank = 5;

struct GettDesc {
    int nm, nn, nk;                       // number of M / N / K modes
    int64_t m_ext[kMaxModes], m_sA[kMaxModes], m_sC[kMaxModes];
    int64_t n_ext[kMaxModes], n_sB[kMaxModes], n_sC[kMaxModes];
    int n_chain;                          // C offset of column n is n * n_sC[0]
    int64_t k_ext[kMaxModes], k_sA[kMaxModes], k_sB[kMaxModes];  // outermost first
    int64_t M, N, K;
    int64_t tiles_m, tiles_n;
    // batch (Hadamard) indices, in A, B and C: the tile list runs over
    // batch values outermost, then N tiles, then M tiles (batch_offsets)
    int nb;
    int64_t b_ext[kMaxModes], b_sA[kMaxModes], b_sB[kMaxModes], b_sC[kMaxModes];
    const void *A;
    const void *B;
    float *C;
    float alpha, beta;
    int init;         // 1: C = alpha*acc + beta*C, 2: C = alpha*acc
    int a_map, b_map; // producer mapping: 0 rows across lanes, 1 K chunks
                      // across lanes, 2 16-byte vectors along K
    int nprod;        // split products (BF16X3)
    int64_t num_tiles;
    int *status;
    // TMA staging (per operand 0 = A, 1 = B): enabled flag, the tensor-map
    // dimension of each row mode and of each K mode with its coordinate
    // multiplier, the staging offset of tile row r (r * srow) and of the
    // stage's K position k (sk[k]), and whether sk runs in aligned fours.
    int tma[2];
    int row_dim[2][kMaxModes];
    int k_dim[2][kMaxModes];
    int64_t k_mul[2][kMaxModes];
    int srow[2];
    int sk[2][kBoxK];
    int sk_vec4[2];
    uint32_t tma_bytes;  // staged bytes per box (both operands)
    int spb;             // K stages per TMA box: 1 (16 K positions) or 2 (32)
    double tile_frac;    // micro-benchmark: run this fraction of the tiles
    int chunk_stages;    // compensated form: K stages per TMEM chunk
    int split;           // split-BF16: (0,0) products in their own accumulator
    const float *qscale; // E4M3: the scales of A and B (powers of two, device memory)
    // batched form: per-problem descriptors (num_tiles, status, nprod,
    // alpha, beta and init are the batch's, in this descriptor), the
    // problem of each tile, and each problem's first tile
    const GettDesc *probs;
    const int32_t *tile_prob;
    int64_t tile0;
    int64_t tile_begin;  // first tile of this launch (batched form; else 0)
    int one_stage;       // batched form: every problem's K fits one stage
    // pre-converted input (0 none, 1 A, 2 B, 3 both): its stage images,
    // laid out [row tile][K stage][slice][core-matrix image] as the
    // converters would write them to shared memory (3: A's at pk_base, B's
    // at pkb_base)
    int pk;
    const char *pk_base;
    int64_t pk_tile_bytes;  // one row tile's images (every K stage)
    const char *pkb_base;
    int64_t pkb_tile_bytes;
};

// number of batch values of a descriptor (1 without batch indices)
inline int64_t batch_count(const GettDesc &d) {
    int64_t h = 1;
    for (int m = 0; m < d.nb; ++m) h *= d.b_ext[m];
    return h;
}

// Named barrier over one warp role that also ORs a predicate across it.
template <int ID, int COUNT>
__device__ __forceinline__ bool role_sync_or(bool pred) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.cta.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(out)
        : "r"((uint32_t)pred), "n"(ID), "n"(COUNT)
        : "memory");
    return out != 0;
}

// ---- CTA pairs (cta_group::2): two CTAs of a cluster of two share each MMA.
// The pair's MMA is M = 256: each CTA holds 128 rows of A and half of the
// B tile in its own shared memory (at the same offsets), and each CTA's
// tensor memory receives its 128 rows of the accumulator.  One thread of
// the even CTA issues the MMAs; its commits arrive on both CTAs' barriers.
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Every thread of both CTAs: release this CTA's prior writes, acquire the
// peer's.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The shared::cluster address of the same shared-memory offset in CTA `rank`.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Arrival on an mbarrier of another CTA of the cluster (release at cluster
// scope: this thread's prior shared-memory writes are visible to a thread
// that acquires the barrier's phase).
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait that acquires at cluster scope (barriers other CTAs of the
// pair arrive on); false when the limit expired.
__device__ __forceinline__ bool mbar_wait_cl(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait_cl(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait_cl(bar, parity)) {
        if (globaltimer() - t0 > kWaitLimitNs) return false;
    }
    return true;
}

// One warp of each CTA of the pair allocates collectively; the address is
// the same in both CTAs.
__device__ __forceinline__ void tmem_alloc2(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc2(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Commit of the pair's MMAs issued so far by this thread: arrives once on
// the barrier at this shared-memory offset in every CTA of `mask`.
__device__ __forceinline__ void mma_commit2(uint64_t *bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(mask)
        : "memory");
}

template <int KIND, bool PAIR = false>
__device__ __forceinline__ void mma_issue(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    if constexpr (PAIR && tf32_kind(KIND)) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else if constexpr (PAIR) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else if constexpr (tf32_kind(KIND)) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else if constexpr (KIND == GK_E4M3) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
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

// 64 consecutive columns of this warp's 32 lanes with one wait: the load
// latency is paid once per 64 columns instead of once per 32.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Two 32-column loads (the split accumulators) and their FP32 sum: both
// loads and the wait in one statement, so no use of the registers can be
// scheduled before the wait.
__device__ __forceinline__ void tmem_ld32_sum(uint32_t ta, uint32_t tb, uint32_t (&r)[32]) {
    uint32_t a[32], b[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%65];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
          "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]),
          "=r"(a[16]), "=r"(a[17]), "=r"(a[18]), "=r"(a[19]), "=r"(a[20]), "=r"(a[21]), "=r"(a[22]), "=r"(a[23]),
          "=r"(a[24]), "=r"(a[25]), "=r"(a[26]), "=r"(a[27]), "=r"(a[28]), "=r"(a[29]), "=r"(a[30]), "=r"(a[31]),
          "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]),
          "=r"(b[8]), "=r"(b[9]), "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15]),
          "=r"(b[16]), "=r"(b[17]), "=r"(b[18]), "=r"(b[19]), "=r"(b[20]), "=r"(b[21]), "=r"(b[22]), "=r"(b[23]),
          "=r"(b[24]), "=r"(b[25]), "=r"(b[26]), "=r"(b[27]), "=r"(b[28]), "=r"(b[29]), "=r"(b[30]), "=r"(b[31])
        : "r"(ta), "r"(tb)
        : "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__fadd_rn(__uint_as_float(a[j]), __uint_as_float(b[j])));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st32_zero(uint32_t taddr) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
        "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr), "r"(0u)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}


// ------------------------------------------------------------------ layout
template <int KIND, int BK>
struct KindTraits {
    static constexpr int kElemBytes = tf32_kind(KIND) ? 4 : (KIND == GK_E4M3 ? 1 : 2);  // smem operand element
    static constexpr int kSlices = KIND == GK_BF16X3 ? 3 : (KIND == GK_TF32X3 ? 2 : 1);
    static constexpr int kChunk = 16 / kElemBytes;              // K elements per 16-byte row
    static constexpr int kKc = BK / kChunk;                     // core matrices along K per stage
    static constexpr int kKsteps = BK * kElemBytes / 32;        // MMA instructions along K per stage
    // instruction-descriptor operand format: kind::tf32 TF32 = 2; kind::f16
    // F16 = 0, BF16 = 1; kind::f8f6f4 E4M3 = 0
    static constexpr uint32_t kFmt = tf32_kind(KIND) ? 2u : ((KIND == GK_F16 || KIND == GK_E4M3) ? 0u : 1u);
    using In = typename std::conditional<KIND == GK_BF16, __nv_bfloat16,
                                         typename std::conditional<KIND == GK_F16, __half, float>::type>::type;
    static constexpr int kInBytes = sizeof(In);
    static constexpr int kVec = 16 / kInBytes;                  // input elements per 16-byte load
};

// STAGES: depth of the operand ring (converted tiles the MMA reads);
// SSTG: depth of the TMA staging ring (0 = no TMA staging).  The staging
// ring is the deeper one: it covers the load latency.
// PAIR: a CTA of a pair holds half of the B tile (BN / 2 rows).
template <int KIND, int BN, int STAGES, int BK, int SSTG, bool BATCH = false, bool PAIR = false>
struct SmemPlan {
    static constexpr bool TMA = SSTG > 0;
    static constexpr int kSstg = SSTG > 0 ? SSTG : 1;         // slots of two-stage boxes
    static constexpr int kBNL = PAIR ? BN / 2 : BN;            // B rows held by this CTA
    using T = KindTraits<KIND, BK>;
    static constexpr int kATile = kBM * BK * T::kElemBytes;    // one slice
    static constexpr int kBTile = kBNL * BK * T::kElemBytes;
    static constexpr int kStage = T::kSlices * (kATile + kBTile);
    static constexpr int kOpBytes = STAGES * kStage;
    // staged input boxes cover up to kBoxK K positions (two stages)
    static constexpr int kStgA = TMA ? kBM * kBoxK * T::kInBytes : 0;
    static constexpr int kStgB = TMA ? kBNL * kBoxK * T::kInBytes : 0;
    static constexpr int kStgBytes = SSTG * (kStgA + kStgB);
    // K-offset and row-offset tables of the global-load path: per stage slot
    // (or, in the batched form, per converter group and double-buffered)
    static constexpr int kKSlots = BATCH ? (STAGES > 4 ? STAGES : 4) : STAGES;
    static constexpr int kRowBufs = BATCH ? 4 : 2;
    static constexpr int kKTab = kKSlots * BK * 8 * 2;
    static constexpr int kRowTab = kRowBufs * (kBM + BN) * 8;
    // batched form: per-tile records the converters leave for the epilogue
    static constexpr int kRecs = BATCH ? 8 : 0;
    static constexpr int kColTab = 2 * BN * 8;                  // epilogue, double-buffered
    // with one-stage boxes the staging ring holds twice as many slots
    static constexpr int kBars = (2 * STAGES + 4 * kSstg + 5) * 8 + 16;
    static constexpr int kTotal = kOpBytes + kStgBytes + kKTab + kRowTab + kColTab + kRecs * 64 + kRecs * 16 + kBars;
};

// x = q * y + r for non-negative x, y > 0: 32-bit division when both fit
// (a 64-bit division is a long dependent instruction sequence, and these
// sit on the per-tile critical path of every role)
__device__ __forceinline__ int64_t divmod(int64_t x, int64_t y, int64_t &r) {
    if (((x | y) >> 31) == 0) {
        const uint32_t q = (uint32_t)x / (uint32_t)y;
        r = x - (int64_t)q * y;
        return q;
    }
    const int64_t q = x / y;
    r = x - q * y;
    return q;
}

__device__ __forceinline__ void decode(int64_t x, int n, const int64_t *ext, const int64_t *s1,
                                       const int64_t *s2, int64_t &o1, int64_t &o2) {
    // first mode fastest
    for (int m = 0; m < n; ++m) {
        int64_t v;
        x = divmod(x, ext[m], v);
        o1 += v * s1[m];
        o2 += v * s2[m];
    }
}

// Converts N (4 or 8) FP32 values into the 16-bit slices or TF32 words
// and stores them at dst (one slice after another, slice_stride apart).
// qs: E4M3 only, the operand's inverse scale (a power of two).
template <int KIND, int N>
__device__ __forceinline__ void store_converted(const float (&x)[N], char *dst, int slice_stride, float qs = 1.0f) {
    if constexpr (KIND == GK_BF16X3) {
        uint32_t w0[N / 2], w1[N / 2], w2[N / 2];
#pragma unroll
        for (int e = 0; e < N; e += 2) split3x2(x[e], x[e + 1], w0[e / 2], w1[e / 2], w2[e / 2]);
        if constexpr (N == 8) {
            *(uint4 *)(dst) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
            *(uint4 *)(dst + slice_stride) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
            *(uint4 *)(dst + 2 * slice_stride) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
        } else {
            *(uint2 *)(dst) = make_uint2(w0[0], w0[1]);
            *(uint2 *)(dst + slice_stride) = make_uint2(w1[0], w1[1]);
            *(uint2 *)(dst + 2 * slice_stride) = make_uint2(w2[0], w2[1]);
        }
    } else if constexpr (KIND == GK_TF32X3) {  // N == 4: x = hi + lo (+ at most 2^-22 |x|)
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            h[e] = f32_to_tf32(x[e]);
            l[e] = f32_to_tf32(x[e] - __uint_as_float(h[e]));  // the difference is exact
        }
        *(uint4 *)(dst) = make_uint4(h[0], h[1], h[2], h[3]);
        *(uint4 *)(dst + slice_stride) = make_uint4(l[0], l[1], l[2], l[3]);
    } else if constexpr (KIND == GK_E4M3) {  // N == 4 or 16: x * qs rounded to E4M3, saturating
        (void)slice_stride;
        uint32_t w[N / 4];
#pragma unroll
        for (int e = 0; e < N; e += 4) {
            const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(x[e] * qs, x[e + 1] * qs), __NV_SATFINITE, __NV_E4M3);
            const uint32_t hi =
                __nv_cvt_float2_to_fp8x2(make_float2(x[e + 2] * qs, x[e + 3] * qs), __NV_SATFINITE, __NV_E4M3);
            w[e / 4] = lo | (hi << 16);
        }
        if constexpr (N == 16) *(uint4 *)(dst) = make_uint4(w[0], w[1], w[2], w[3]);
        else *(uint32_t *)(dst) = w[0];
    } else {  // TF32: N == 4
        *(uint4 *)(dst) = make_uint4(f32_to_tf32(x[0]), f32_to_tf32(x[1]), f32_to_tf32(x[2]),
                                     f32_to_tf32(x[3]));
    }
}

// Global-load path: one operand's share of a stage (ROWS rows x BK K
// elements), loads first (all in flight), then conversion and stores.
// MAP 2: 16-byte vector loads along K (contiguity and alignment checked on
// the host); MAP 1: K chunks across lanes; MAP 0: rows across lanes.  Maps 0
// and 1 load through the offset tables one element at a time (any strides).
template <int KIND, int BK, int ROWS, int MAP, int NT = kProducerThreads>
__device__ __forceinline__ void produce_operand(const typename KindTraits<KIND, BK>::In *__restrict__ src,
                                                const int64_t *rowoff, const int64_t *koff, char *tile,
                                                int slice_stride, int pt, float qs = 1.0f) {
    using T = KindTraits<KIND, BK>;
    constexpr int KC = T::kKc, CH = T::kChunk;
    constexpr bool kFloatIn = float_input(KIND);
    if constexpr (MAP == 2) {
        constexpr int UPR = BK / T::kVec;  // 16-byte loads per row per stage
        constexpr int NU = ROWS * UPR / NT;
        static_assert(NU * NT == ROWS * UPR, "even split");
        uint4 v[NU];
#pragma unroll
        for (int i = 0; i < NU; ++i) {
            const int u = pt + i * NT;
            const int row = u / UPR, k = (u % UPR) * T::kVec;
            const int64_t ro = rowoff[row], ko = koff[k];
            v[i] = (ro >= 0 && ko >= 0) ? __ldg((const uint4 *)(src + ro + ko)) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int i = 0; i < NU; ++i) {
            const int u = pt + i * NT;
            const int row = u / UPR, k = (u % UPR) * T::kVec;
            const int kc = k / CH, byte = (k % CH) * T::kElemBytes;
            char *dst = tile + (kc * (ROWS / 8) + row / 8) * 128 + (row % 8) * 16 + byte;
            if constexpr (kFloatIn) {
                float x[4] = {__uint_as_float(v[i].x), __uint_as_float(v[i].y), __uint_as_float(v[i].z),
                              __uint_as_float(v[i].w)};
                store_converted<KIND, 4>(x, dst, slice_stride, qs);
            } else {
                *(uint4 *)(dst) = v[i];
            }
        }
    } else {
        constexpr int NC = ROWS * KC / NT;
        static_assert(NC * NT == ROWS * KC, "even split");
        using L = typename std::conditional<kFloatIn, float, unsigned short>::type;
        const L *s = (const L *)src;
        L x[NC][CH];
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            const int c = pt + i * NT;
            const int row = MAP == 1 ? c / KC : c % ROWS;
            const int kc = MAP == 1 ? c % KC : c / ROWS;
            const int64_t ro = rowoff[row];
#pragma unroll
            for (int e = 0; e < CH; ++e) {
                const int64_t ko = koff[kc * CH + e];
                x[i][e] = (ro >= 0 && ko >= 0) ? __ldg(s + ro + ko) : L(0);
            }
        }
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            const int c = pt + i * NT;
            const int row = MAP == 1 ? c / KC : c % ROWS;
            const int kc = MAP == 1 ? c % KC : c / ROWS;
            char *dst = tile + (kc * (ROWS / 8) + row / 8) * 128 + (row % 8) * 16;
            if constexpr (kFloatIn) {
                store_converted<KIND, CH>(x[i], dst, slice_stride, qs);
            } else {
                uint32_t w[CH / 2];
#pragma unroll
                for (int e = 0; e < CH; e += 2) w[e / 2] = (uint32_t)x[i][e] | ((uint32_t)x[i][e + 1] << 16);
                *(uint4 *)(dst) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
}

template <int KIND, int BK, int ROWS, int NT = kProducerThreads>
__device__ __forceinline__ void produce_any(const typename KindTraits<KIND, BK>::In *__restrict__ src,
                                            const int64_t *rowoff, const int64_t *koff, char *tile,
                                            int slice_stride, int map, int pt, float qs = 1.0f) {
    if (map == 2) produce_operand<KIND, BK, ROWS, 2, NT>(src, rowoff, koff, tile, slice_stride, pt, qs);
    else if (map == 1) produce_operand<KIND, BK, ROWS, 1, NT>(src, rowoff, koff, tile, slice_stride, pt, qs);
    else produce_operand<KIND, BK, ROWS, 0, NT>(src, rowoff, koff, tile, slice_stride, pt, qs);
}

// TMA path: converts one operand's staged box (ROWS rows x BK K positions,
// laid out as the box's dimensions) into the core-matrix layout.  Row r of
// the tile sits at r * srow, K position k at sk[k] (elements); rows past the
// operand's extent were filled with zeros by the TMA unit.
template <int KIND, int BK, int ROWS, int NT = kProducerThreads>
__device__ __forceinline__ void convert_staged(const char *stg, int srow, const int *sk, int vec4,
                                               char *tile, int slice_stride, int pt) {
    using T = KindTraits<KIND, BK>;
    using In = typename T::In;
    constexpr int KC = T::kKc, CH = T::kChunk;
    constexpr int NC = ROWS * KC / NT;  // NT threads share the box
    static_assert(NC * NT == ROWS * KC, "even split");
    constexpr bool kFloatIn = float_input(KIND);
    const In *s = (const In *)stg;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        const int c = pt + i * NT;
        const int row = c % ROWS, kc = c / ROWS;  // rows across lanes: conflict-free stores
        char *dst = tile + (kc * (ROWS / 8) + row / 8) * 128 + (row % 8) * 16;
        const In *base = s + row * srow;
        if constexpr (kFloatIn) {
            float x[CH];
            if (vec4) {
#pragma unroll
                for (int e = 0; e < CH; e += 4) {
                    float4 v = *(const float4 *)(base + sk[kc * CH + e]);
                    x[e] = v.x;
                    x[e + 1] = v.y;
                    x[e + 2] = v.z;
                    x[e + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int e = 0; e < CH; ++e) x[e] = base[sk[kc * CH + e]];
            }
            store_converted<KIND, CH>(x, dst, slice_stride);
        } else {
            const unsigned short *b16 = (const unsigned short *)base;
            uint32_t w[CH / 2];
#pragma unroll
            for (int e = 0; e < CH; e += 2)
                w[e / 2] = (uint32_t)b16[sk[kc * CH + e]] | ((uint32_t)b16[sk[kc * CH + e + 1]] << 16);
            *(uint4 *)(dst) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Pre-converted input: one stage image (BYTES, contiguous) copied to the
// stage with 16-byte asynchronous copies shared by NT threads; the caller
// waits with cp_async_wait_all before publishing the stage.
template <int BYTES, int NT>
__device__ __forceinline__ void copy_packed(const char *src, char *dst, int pt) {
    static_assert(BYTES % (16 * NT) == 0, "even split");
#pragma unroll
    for (int i = 0; i < BYTES / (16 * NT); ++i) {
        const int u = (pt + i * NT) * 16;
        cp_async16(dst + u, src + u);
    }
}

// Batch indices: tile lt of a problem is tile lt % (tiles_m * tiles_n) of
// batch value lt / (tiles_m * tiles_n); returns the former and adds the
// batch value's offsets in A, B and C (first batch index fastest).
__device__ __forceinline__ int64_t batch_offsets(const GettDesc &P, int64_t lt, int64_t &oA, int64_t &oB,
                                                 int64_t &oC) {
    oA = oB = oC = 0;
    if (P.nb == 0) return lt;
    int64_t r;
    int64_t bt = divmod(lt, P.tiles_m * P.tiles_n, r);
    for (int m = 0; m < P.nb; ++m) {
        int64_t v;
        bt = divmod(bt, P.b_ext[m], v);
        oA += v * P.b_sA[m];
        oB += v * P.b_sB[m];
        oC += v * P.b_sC[m];
    }
    return r;
}

// The descriptor of a tile's problem: the launch's own, or in the batched
// form the one its tile-to-problem table names.
template <bool BATCH>
__device__ __forceinline__ const GettDesc &tile_desc(const GettDesc &d, int64_t tile) {
    if constexpr (BATCH) return d.probs[d.tile_prob[tile]];
    else return d;
}

// Epilogue stores of W accumulator columns c0.. of this thread's row (C
// offset om, -1 = no row): columns at on0 + j*lin when lin != 0 (the tile's
// columns form one stride), else through the tile's column table cn
// (-1 = past N).  C = alpha*acc (init 2) or alpha*acc + beta*C (init 1).
template <int W>
__device__ __forceinline__ void store_cols(const uint32_t (&r)[W], float *__restrict__ C, int64_t om, int c0,
                                           int64_t lin, int64_t on0, int64_t nval, const int64_t *cn,
                                           float alpha, float beta, int init) {
    if (om < 0) return;
    if (lin != 0) {
        float *p = C + om + on0 + (int64_t)c0 * lin;
        const int64_t jn = nval - c0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            if (j < jn) {
                float v = alpha * __uint_as_float(r[j]);
                if (init == 1) v = fmaf(beta, *p, v);
                *p = v;
            }
            p += lin;
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const int64_t on = cn[c0 + j];
        if (on < 0) continue;
        float v = alpha * __uint_as_float(r[j]);
        if (init == 1) v = fmaf(beta, C[om + on], v);
        C[om + on] = v;
    }
}

// COMP (split-BF16 with long K): the MMA accumulates chunks of
// chunk_stages K stages into two alternating TMEM accumulators; the
// epilogue folds each finished chunk into a float-float running sum
// (hi, lo) kept in TMEM (TwoSum), so the FP32 rounding of the accumulator
// grows with the chunk length instead of with K.
// BATCH: the tiles of many problems in one launch (global-load inputs).
// PAIR: clusters of two CTAs share each MMA (cta_group::2, M = 256): a tile
// is 256 x BN; each CTA stages and converts its 128 rows of A and half of
// the BN rows of B, and its tensor memory holds its 128 rows of C.
// d.split (split-BF16, not COMP): the weight-1 slice product (0,0)
// accumulates in one tensor-memory accumulator and the smaller products
// in another, added in the epilogue: only K/16 of the FP32 roundings happen
// at the magnitude of the whole sum.  The two take both halves of the
// tensor memory, so the accumulators are not double-buffered then.
template <int KIND, int BN, int STAGES, int BK, int SSTG, bool COMP, bool BATCH, bool PAIR = false>
__global__ void __launch_bounds__(kThreads, 1)
gett_tc_kernel(const GettDesc d, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB) {
    using T = KindTraits<KIND, BK>;
    using SP = SmemPlan<KIND, BN, STAGES, BK, SSTG, BATCH, PAIR>;
    // (pairs with the compensated form: both inputs pre-converted only)
    static_assert(!(PAIR && BATCH), "CTA pairs: not in the batched form");
    constexpr bool TMA = SP::TMA;
    constexpr int SS = SP::kSstg;
    constexpr int BNL = SP::kBNL;  // B rows this CTA stages and converts
    using In = typename T::In;
    extern __shared__ __align__(1024) char smem[];
    char *ops = smem;
    char *stg = smem + SP::kOpBytes;                          // [SSTG][A box | B box]
    int64_t *kA = (int64_t *)(stg + SP::kStgBytes);           // [STAGES][BK]
    int64_t *kB = kA + SP::kKSlots * BK;
    int64_t *rowA = kB + SP::kKSlots * BK;                    // [kRowBufs][kBM]
    int64_t *rowB = rowA + SP::kRowBufs * kBM;                // [kRowBufs][BN]
    int64_t *cN = rowB + SP::kRowBufs * BN;                   // [2][BN]
    int64_t *trec = cN + 2 * BN;                              // [kRecs][8] batched tile records
    uint64_t *rfull = (uint64_t *)(trec + SP::kRecs * 8);     // [kRecs] record written
    uint64_t *rempty = rfull + SP::kRecs;                     // [kRecs] record read
    uint64_t *full = rempty + SP::kRecs;                      // operand stage filled
    constexpr int kRecMod = SP::kRecs > 0 ? SP::kRecs : 1;    // record ring index (batched form only)
    uint64_t *empty = full + STAGES;                          // operand stage consumed
    uint64_t *sfull = empty + STAGES;                         // staged box landed
    uint64_t *sempty = sfull + 2 * SS;                        // staged box converted
    uint64_t *tfull = sempty + 2 * SS;                        // [2]
    uint64_t *tempty = tfull + 2;                             // [2]
    uint64_t *drain = tempty + 2;
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nkt = (int)((d.K + BK - 1) / BK);
    constexpr uint32_t kTmemCols = COMP ? 4 * BN : 2 * BN;
    static_assert(kTmemCols <= 512, "tensor memory columns");
    // pairs: this CTA's rank in its pair; a pair (or a lone CTA) is one
    // slot of the persistent tile walk
    const uint32_t crank = PAIR ? cluster_ctarank() : 0u;
    const int64_t slot0 = PAIR ? (int64_t)(blockIdx.x >> 1) : (int64_t)blockIdx.x;
    const int64_t nslots = PAIR ? (int64_t)(gridDim.x >> 1) : (int64_t)gridDim.x;
    // accumulators per tile: one (double-buffered) or the split pair
    const bool split = !COMP && d.split != 0;
    const int nbuf = split ? 1 : 2;
    // barriers the other CTA of a pair arrives on are waited on with
    // acquire at cluster scope; arrivals for the MMA issuer go to rank 0
    auto bwait = [&](uint64_t *bar, uint32_t parity) -> bool {
        if constexpr (PAIR) return mbar_wait_cl(bar, parity);
        else return mbar_wait(bar, parity);
    };
    auto btry = [&](uint64_t *bar, uint32_t parity) -> bool {
        if constexpr (PAIR) return mbar_try_wait_cl(bar, parity);
        else return mbar_try_wait(bar, parity);
    };
    auto arrive_issuer = [&](uint64_t *bar) {
        if constexpr (PAIR) mbar_arrive_remote(mapa_shared(smem_u32(bar), 0u));
        else mbar_arrive(bar);
    };
    // accumulation units per tile: one, or the K chunks of the compensated form
    const int cstg = COMP ? (d.chunk_stages > 0 ? d.chunk_stages : nkt) : nkt;
    const int nch = (nkt + cstg - 1) / cstg;
    const bool any_tma = TMA && (d.tma[0] || d.tma[1]);
    const bool any_ldg = !TMA || !d.tma[0] || !d.tma[1];
    // both operands staged by TMA (or one staged and the other
    // pre-converted): the converter warps split into two groups of four that
    // take alternate stages, so one group's waits and barrier overlap the
    // other's conversion
    const bool grouped = (TMA && !BATCH && any_tma && (d.tma[0] || d.pk == 1) && (d.tma[1] || d.pk == 2)) ||
                         (BATCH && d.one_stage);
    constexpr int kPkA = T::kSlices * SP::kATile, kPkB = T::kSlices * SP::kBTile;  // stage image bytes
    // staging ring geometry: SS slots of two-stage boxes, or 2 * SS slots of
    // one-stage boxes (the same bytes)
    // A pre-converted input has no staged box: its share of the staging
    // bytes holds further slots of the other input's boxes (up to the
    // 2 * SS slots the barriers are laid out for).
    const int spb_r = d.spb > 1 ? d.spb : 1;
    const int boxA = d.pk == 1 ? 0 : (spb_r == 1 ? SP::kStgA / 2 : SP::kStgA);
    const int boxB = d.pk == 2 ? 0 : (spb_r == 1 ? SP::kStgB / 2 : SP::kStgB);
    const int NSL = !TMA ? 2 * SS : min(2 * SS, SP::kStgBytes / (boxA + boxB));

    if (threadIdx.x == 0) {
        // one arrival per converter warp that converts a stage: all eight,
        // or the four of one group when the groups take turns
        const uint32_t conv_warps = grouped ? kProducerThreads / 32 / kConvGroups : kProducerThreads / 32;
        for (int s = 0; s < STAGES; ++s) {
            // pairs: both CTAs' converters arrive on rank 0's barrier; with
            // both inputs pre-converted the copying lane arms it alone
            mbar_init(&full[s], d.pk == 3 ? (PAIR && crank == 0 ? 2u : 1u) : conv_warps * (PAIR ? 2 : 1));
            mbar_init(&empty[s], 1);
        }
        // a staging slot is free again once every stage of its box is converted
        const int spb = d.spb > 1 ? d.spb : 1;
        for (int s = 0; s < NSL; ++s) {
            mbar_init(&sfull[s], 1);
            mbar_init(&sempty[s], conv_warps * spb);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            // one arrival per epilogue warp (of both CTAs of a pair)
            mbar_init(&tempty[b], kEpiThreads / 32 * (PAIR ? 2 : 1));
        }
        for (int r = 0; r < SP::kRecs; ++r) {
            mbar_init(&rfull[r], 1);
            mbar_init(&rempty[r], 1);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if constexpr (PAIR) {
        // both CTAs run and their barriers are initialised before any
        // arrival crosses the pair or the pair allocates tensor memory
        cluster_sync_all();
        if (warp == kMmaWarp) tmem_alloc2(tmem_slot, kTmemCols);
    } else {
        if (warp == kMmaWarp) tmem_alloc(tmem_slot, kTmemCols);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp >= kEpiWarps && warp < kMmaWarp) {
        // ---------------------------------------------------------- converters
        const int pt = threadIdx.x - kEpiThreads;
        // E4M3: each input divided by its scale (a power of two, exact)
        float qa = 1.0f, qb = 1.0f;
        if constexpr (KIND == GK_E4M3) {
            qa = 1.0f / d.qscale[0];
            qb = 1.0f / d.qscale[1];
        }
        // with a pre-converted input the kernel is launched as a programmatic
        // dependent of the pre-pass: its other roles start at once (the TMA
        // warp streams the other input), the converters wait here until the
        // pre-pass grid has completed and its stores are visible
        if (!BATCH && d.pk) asm volatile("griddepcontrol.wait;" ::: "memory");
        int64_t g = 0;
        int it = 0;
        bool stop = false;
        const int spb_c = d.spb > 1 ? d.spb : 1;  // stages per staged box
        if (BATCH && grouped) {
            // batched form, one K stage per tile: the groups take alternate
            // tiles, each with its own double-buffered offset tables, so one
            // group's global-load latency overlaps the other's conversion
            constexpr int kGT = kProducerThreads / kConvGroups;
            static_assert(kConvGroups == 2, "table buffers per group");
            const int gp = pt / kGT, ptg = pt % kGT;
            int gi = 0;  // this group's tile count
            // every batched problem is a strided GEMM (one M, N and K mode):
            // its fields are read with independent loads, and the problem
            // index of the group's next tile is fetched one tile ahead
            int64_t tile = d.tile_begin + blockIdx.x;
            for (int k = 0; k < gp; ++k) tile += gridDim.x;  // this group's first tile
            g = gp;
            int32_t q = tile < d.num_tiles ? d.tile_prob[tile] : 0;
            for (; tile < d.num_tiles && !stop; tile += (int64_t)kConvGroups * gridDim.x, g += kConvGroups) {
                const int64_t next = tile + (int64_t)kConvGroups * gridDim.x;
                const int32_t q_next = next < d.num_tiles ? d.tile_prob[next] : 0;
                const GettDesc &P = d.probs[q];
                const int64_t pM = P.M, pN = P.N, pK = P.K, ptm = P.tiles_m, pt0 = P.tile0;
                const int64_t sAm = P.m_sA[0], sCm = P.m_sC[0], sBn = P.n_sB[0], sCn = P.n_sC[0];
                const int64_t sAk = P.k_sA[0], sBk = P.k_sB[0];
                const In *__restrict__ Ap = (const In *)P.A;
                const In *__restrict__ Bp = (const In *)P.B;
                float *const Cp = P.C;
                const int amap = P.a_map, bmap = P.b_map;
                q = q_next;
                int64_t mt;
                const int64_t nt = divmod(tile - pt0, ptm, mt);
                const int64_t m0 = mt * kBM, n0 = nt * BN;
                const int s = (int)(g % STAGES);
                const uint32_t ph = (uint32_t)((g / STAGES) & 1);
                const int bix = gp * 2 + (gi & 1);
                ++gi;
                int64_t *rA = rowA + bix * kBM, *rB = rowB + bix * BN;
                int64_t *tA = kA + bix * BK, *tB = kB + bix * BK;
                bool bad = g >= STAGES && !mbar_wait(&empty[s], ph ^ 1u);
                for (int i = ptg; i < kBM; i += kGT) rA[i] = m0 + i < pM ? (m0 + i) * sAm : -1;
                for (int j = ptg; j < BN; j += kGT) rB[j] = n0 + j < pN ? (n0 + j) * sBn : -1;
                if (ptg < BK) {  // one stage: the K position is the thread's
                    tA[ptg] = ptg < pK ? ptg * sAk : -1;
                    tB[ptg] = ptg < pK ? ptg * sBk : -1;
                }
                const bool quit = gp == 0 ? role_sync_or<1, kGT>(bad || *abort_flag)
                                          : role_sync_or<3, kGT>(bad || *abort_flag);
                if (quit) {
                    if (ptg == 0) {
                        *abort_flag = 1;
                        atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
                    }
                    stop = true;
                    break;
                }
                if (ptg == 0 && !stop) {
                    // what the epilogue needs of this tile, so that it reads no
                    // problem descriptor from global memory: a ring of records
                    // with its own barriers (written here, read there)
                    const int r = (int)(g % kRecMod);
                    if (g >= kRecMod && !mbar_wait(&rempty[r], (uint32_t)(((g / kRecMod) - 1) & 1))) {
                        *abort_flag = 1;
                        atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
                    }
                    int64_t *rec = trec + r * 8;
                    rec[0] = (int64_t)Cp;
                    rec[1] = pM - m0;                   // valid rows of the tile
                    rec[2] = sCm;
                    rec[3] = sCn;
                    rec[4] = m0 * sCm + n0 * sCn;
                    rec[5] = min((int64_t)BN, pN - n0);  // valid columns
                    mbar_arrive(&rfull[r]);
                }
                char *stage = ops + s * SP::kStage;
                produce_any<KIND, BK, kBM, kGT>(Ap, rA, tA, stage, SP::kATile, amap, ptg);
                produce_any<KIND, BK, BN, kGT>(Bp, rB, tB, stage + T::kSlices * SP::kATile, SP::kBTile, bmap, ptg);
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[s]);
            }
        } else if (grouped) {
            constexpr int kGT = kProducerThreads / kConvGroups;  // threads per group
            // a group starts stage g once it has finished g - kConvGroups; the
            // parity waits on a slot's barriers stay unambiguous only while
            // both rings have at least kConvGroups slots
            static_assert(!TMA || (STAGES >= kConvGroups && SSTG >= kConvGroups), "ring depth vs groups");
            const int gp = pt / kGT, ptg = pt % kGT;
            for (int64_t tile = d.tile_begin + slot0; tile < d.num_tiles && !stop; tile += nslots) {
                const char *pkt = nullptr;  // this tile's pre-converted images
                if (d.pk) {
                    int64_t mt;
                    const int64_t nt = divmod(tile, d.tiles_m, mt);
                    // pairs: images of 128-row (A) or BN/2-row (B) tiles,
                    // two per pair tile
                    const int64_t it_ = d.pk == 1 ? mt : nt;
                    pkt = d.pk_base + (PAIR ? 2 * it_ + crank : it_) * d.pk_tile_bytes;
                }
                for (int kt = 0; kt < nkt; ++kt, ++g) {
                    if ((int)(g % kConvGroups) != gp) continue;  // another group's stage
                    const int s = (int)(g % STAGES);
                    const uint32_t ph = (uint32_t)((g / STAGES) & 1);
                    const int64_t gb = g / spb_c;  // the TMA box of this stage
                    const int half = (int)(g - gb * spb_c);
                    const int ss = (int)(gb % NSL);
                    const uint32_t sph = (uint32_t)((gb / NSL) & 1);
                    const bool e_ok = g < STAGES || btry(&empty[s], ph ^ 1u);
                    const bool f_ok = mbar_try_wait(&sfull[ss], sph);
                    bool bad = false;
                    if (!e_ok) bad = !bwait(&empty[s], ph ^ 1u);
                    if (!f_ok && !bad) bad = !mbar_wait(&sfull[ss], sph);
                    // named barriers 1, 3, 4, 5 (0: the whole CTA, 2: the epilogue)
                    bool quit;
                    if (gp == 0) quit = role_sync_or<1, kGT>(bad || *abort_flag);
                    else if (gp == 1) quit = role_sync_or<3, kGT>(bad || *abort_flag);
                    else if (gp == 2) quit = role_sync_or<4, kGT>(bad || *abort_flag);
                    else quit = role_sync_or<5, kGT>(bad || *abort_flag);
                    if (quit) {
                        if (ptg == 0) {
                            *abort_flag = 1;
                            atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
                        }
                        stop = true;
                        break;
                    }
                    char *stage = ops + s * SP::kStage;
                    const char *box = stg + ss * (boxA + boxB);
                    // a pre-converted input's copies go first: they complete
                    // while the other input is converted
                    if (d.pk == 1) copy_packed<kPkA, kGT>(pkt + kt * kPkA, stage, ptg);
                    else if (d.pk == 2) copy_packed<kPkB, kGT>(pkt + kt * kPkB, stage + kPkA, ptg);
                    if (d.pk != 1)
                        convert_staged<KIND, BK, kBM, kGT>(box, d.srow[0], d.sk[0] + half * BK, d.sk_vec4[0], stage,
                                                           SP::kATile, ptg);
                    if (d.pk != 2)
                        convert_staged<KIND, BK, BNL, kGT>(box + boxA, d.srow[1], d.sk[1] + half * BK, d.sk_vec4[1],
                                                           stage + kPkA, SP::kBTile, ptg);
                    if (d.pk) cp_async_wait_all();
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        arrive_issuer(&full[s]);
                        mbar_arrive(&sempty[ss]);
                    }
                }
            }
        }
        for (int64_t tile = d.tile_begin + blockIdx.x; tile < d.num_tiles && !stop && !grouped && !PAIR && d.pk != 3;
             tile += gridDim.x, ++it) {
            const GettDesc &P = tile_desc<BATCH>(d, tile);
            int64_t boA, boB, boC;
            const int64_t lt = batch_offsets(P, BATCH ? tile - P.tile0 : tile, boA, boB, boC);
            const int nkt_t = BATCH ? (int)((P.K + BK - 1) / BK) : nkt;
            const In *__restrict__ Ap = (const In *)P.A + boA;
            const In *__restrict__ Bp = (const In *)P.B + boB;
            int64_t mt;
            const int64_t nt = divmod(lt, P.tiles_m, mt);
            const int64_t m0 = mt * kBM, n0 = nt * BN;
            int64_t *rA = rowA + (it & 1) * kBM;
            int64_t *rB = rowB + (it & 1) * BN;
            for (int kt = 0; kt < nkt_t; ++kt, ++g) {
                const int s = (int)(g % STAGES);
                const uint32_t ph = (uint32_t)((g / STAGES) & 1);
                const int64_t gb = g / spb_c;  // the TMA box of this stage
                const int half = (int)(g - gb * spb_c);
                const int ss = (int)(gb % NSL);
                // both barriers polled back to back (their latencies overlap);
                // the bounded waits only when one is not complete yet
                const uint32_t sph = (uint32_t)((gb / NSL) & 1);
                const bool e_ok = g < STAGES || mbar_try_wait(&empty[s], ph ^ 1u);
                const bool f_ok = !any_tma || mbar_try_wait(&sfull[ss], sph);
                bool bad = false;
                if (!e_ok) bad = !mbar_wait(&empty[s], ph ^ 1u);
                if (!f_ok && !bad) bad = !mbar_wait(&sfull[ss], sph);
                if (any_ldg) {
                    if (kt == 0) {
                        for (int i = pt; i < kBM; i += kProducerThreads) {
                            int64_t mm = m0 + i, oa = -1, oc = 0;
                            if (mm < P.M) {
                                oa = 0;
                                decode(mm, P.nm, P.m_ext, P.m_sA, P.m_sC, oa, oc);
                            }
                            rA[i] = oa;
                        }
                        for (int j = pt; j < BN; j += kProducerThreads) {
                            int64_t nn = n0 + j, ob = -1, oc = 0;
                            if (nn < P.N) {
                                ob = 0;
                                decode(nn, P.nn, P.n_ext, P.n_sB, P.n_sC, ob, oc);
                            }
                            rB[j] = ob;
                        }
                    }
                    if (pt < BK) {
                        int64_t k = (int64_t)kt * BK + pt, oa = -1, ob = -1;
                        if (k < P.K) {
                            oa = 0;
                            ob = 0;
                            if (P.K < (int64_t(1) << 31)) {  // 32-bit digits when they fit
                                uint32_t k32 = (uint32_t)k;
                                for (int m = P.nk - 1; m >= 0; --m) {  // innermost K mode fastest
                                    const uint32_t e = (uint32_t)P.k_ext[m];
                                    const int64_t v = (int64_t)(k32 % e);
                                    k32 /= e;
                                    oa += v * P.k_sA[m];
                                    ob += v * P.k_sB[m];
                                }
                            } else {
                                for (int m = P.nk - 1; m >= 0; --m) {
                                    int64_t v = k % P.k_ext[m];
                                    k /= P.k_ext[m];
                                    oa += v * P.k_sA[m];
                                    ob += v * P.k_sB[m];
                                }
                            }
                        }
                        kA[s * BK + pt] = oa;
                        kB[s * BK + pt] = ob;
                    }
                }
                if (role_sync_or<1, kProducerThreads>(bad || *abort_flag)) {
                    if (pt == 0) {
                        *abort_flag = 1;
                        atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
                    }
                    stop = true;
                    break;
                }
                char *stage = ops + s * SP::kStage;
                char *bstage = stage + T::kSlices * SP::kATile;
                // a pre-converted input (never in the batched form) is copied
                // first: its copies complete while the other is produced
                const int pk = BATCH ? 0 : d.pk;
                if (pk) {
                    const char *pkt = d.pk_base + (pk == 1 ? mt : nt) * d.pk_tile_bytes;
                    if (pk == 1) copy_packed<kPkA, kProducerThreads>(pkt + kt * kPkA, stage, pt);
                    else copy_packed<kPkB, kProducerThreads>(pkt + kt * kPkB, bstage, pt);
                }
                if (pk != 1) {
                    if (TMA && d.tma[0])
                        convert_staged<KIND, BK, kBM>(stg + ss * (boxA + boxB), d.srow[0], d.sk[0] + half * BK,
                                                      d.sk_vec4[0], stage, SP::kATile, pt);
                    else
                        produce_any<KIND, BK, kBM>(Ap, rA, kA + s * BK, stage, SP::kATile, P.a_map, pt, qa);
                }
                if (pk != 2) {
                    if (TMA && d.tma[1])
                        convert_staged<KIND, BK, BN>(stg + ss * (boxA + boxB) + boxA, d.srow[1],
                                                     d.sk[1] + half * BK, d.sk_vec4[1], bstage, SP::kBTile, pt);
                    else
                        produce_any<KIND, BK, BN>(Bp, rB, kB + s * BK, bstage, SP::kBTile, P.b_map, pt, qb);
                }
                if (pk) cp_async_wait_all();
                // each lane publishes its stores to the async proxy; the warp's
                // lanes are ordered by __syncwarp and lane 0 arrives for all
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&full[s]);
                    if (any_tma) mbar_arrive(&sempty[ss]);
                }
            }
        }
    } else if (warp == kTmaWarp) {
        // ---------------------------------------------------------- TMA issue
        if (!BATCH && d.pk == 3) {
            // both inputs pre-converted: one lane copies each stage's two
            // images (contiguous runs of the workspace) straight into the
            // operand ring with 1-D bulk copies; the converters stay idle.
            // Pairs: each CTA copies its 128 rows of A and its half of the
            // tile's B rows into its own ring (images of 128-row and
            // BN/2-row tiles, two per pair tile)
            if (lane == 0) {
                asm volatile("griddepcontrol.wait;" ::: "memory");  // the pre-pass grids are complete
                constexpr uint32_t kImgA = (uint32_t)(T::kSlices * SP::kATile);
                constexpr uint32_t kImgB = (uint32_t)(T::kSlices * SP::kBTile);
                int64_t g = 0;
                bool stop = false;
                for (int64_t tile = d.tile_begin + slot0; tile < d.num_tiles && !stop; tile += nslots) {
                    int64_t mt;
                    const int64_t nt = divmod(tile, d.tiles_m, mt);
                    const char *ia = d.pk_base + (PAIR ? 2 * mt + crank : mt) * d.pk_tile_bytes;
                    const char *ib = d.pkb_base + (PAIR ? 2 * nt + crank : nt) * d.pkb_tile_bytes;
                    for (int kt = 0; kt < nkt; ++kt, ++g) {
                        const int s = (int)(g % STAGES);
                        if (*abort_flag ||
                            (g >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((g / STAGES) - 1) & 1)))) {
                            stop = true;
                            break;
                        }
                        char *stage = ops + s * SP::kStage;
                        mbar_arrive_expect_tx(&full[s], kImgA + kImgB);
                        bulk_load(stage, ia + kt * (int64_t)kImgA, kImgA, &full[s]);
                        bulk_load(stage + kImgA, ib + kt * (int64_t)kImgB, kImgB, &full[s]);
                    }
                }
                if (stop) {
                    *abort_flag = 1;
                    atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
                    // the copies still in flight land before the CTA may
                    // exit: each slot's last issue completes its phase
                    for (int64_t q = g > STAGES ? g - STAGES : 0; q < g; ++q)
                        mbar_wait(&full[q % STAGES], (uint32_t)((q / STAGES) & 1));
                }
            }
        } else if (TMA && any_tma && lane == 0) {
            int64_t g = 0;
            bool stop = false;
            // box coordinates of a tile's rows, and of one of its K stages
            auto tile_rc = [&](int64_t tile, int32_t (&rc)[2][kTmaRank]) {
                int64_t mt;
                const int64_t nt = divmod(tile, d.tiles_m, mt);
#pragma unroll
                for (int o = 0; o < 2; ++o)
#pragma unroll
                    for (int x = 0; x < kTmaRank; ++x) rc[o][x] = 0;
                // pairs: this CTA's 128 rows of the 256-row tile, and its
                // half of the tile's B rows
                int64_t r = (PAIR ? 2 * mt + crank : mt) * kBM, v;
                for (int m = 0; m < d.nm; ++m) {
                    r = divmod(r, d.m_ext[m], v);
#pragma unroll
                    for (int x = 0; x < kTmaRank; ++x)
                        if (d.row_dim[0][m] == x) rc[0][x] = (int32_t)v;
                }
                r = nt * BN + (PAIR ? crank * BNL : 0);
                for (int m = 0; m < d.nn; ++m) {
                    r = divmod(r, d.n_ext[m], v);
#pragma unroll
                    for (int x = 0; x < kTmaRank; ++x)
                        if (d.row_dim[1][m] == x) rc[1][x] = (int32_t)v;
                }
            };
            auto stage_c = [&](const int32_t (&rc)[2][kTmaRank], int kt, int32_t (&c)[2][kTmaRank]) {
#pragma unroll
                for (int o = 0; o < 2; ++o)
#pragma unroll
                    for (int x = 0; x < kTmaRank; ++x) c[o][x] = rc[o][x];
                // the host keeps K below 2^31 on this path
                uint32_t k = (uint32_t)kt * (uint32_t)BK;
                for (int m = d.nk - 1; m >= 0; --m) {
                    const uint32_t e = (uint32_t)d.k_ext[m];
                    const uint32_t v = k % e;
                    k /= e;
#pragma unroll
                    for (int o = 0; o < 2; ++o) {
                        const int dd = d.k_dim[o][m];
                        const int32_t add = (int32_t)(v * (uint32_t)d.k_mul[o][m]);
#pragma unroll
                        for (int x = 0; x < kTmaRank; ++x)
                            if (dd == x) c[o][x] += add;
                    }
                }
            };
            int32_t rc[2][kTmaRank];
            const int spb = d.spb > 1 ? d.spb : 1;  // g counts boxes here
            for (int64_t tile = d.tile_begin + slot0; tile < d.num_tiles && !stop; tile += nslots) {
                tile_rc(tile, rc);
                for (int kt = 0; kt < nkt; kt += spb, ++g) {
                    const int s = (int)(g % NSL);
                    if (g >= NSL && (*abort_flag || !mbar_wait(&sempty[s], (uint32_t)(((g / NSL) - 1) & 1)))) {
                        stop = true;
                        break;
                    }
                    int32_t c[2][kTmaRank];
                    stage_c(rc, kt, c);
                    char *box = stg + s * (boxA + boxB);
                    mbar_arrive_expect_tx(&sfull[s], d.tma_bytes);
                    if (d.tma[0]) tma_load_5d(box, &tmA, &sfull[s], c[0]);
                    if (d.tma[1]) tma_load_5d(box + boxA, &tmB, &sfull[s], c[1]);
                }
            }
            if (stop) {
                *abort_flag = 1;
                atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
            }
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // ---------------------------------------------------------- MMA issuer
        // (pairs: rank 0 issues for both CTAs; the other MMA warp only
        // takes part in the tensor-memory allocation)
        if (lane == 0 && crank == 0) {
            constexpr uint32_t kM = PAIR ? 2 * kBM : kBM;
            constexpr uint32_t idesc = (1u << 4) | (T::kFmt << 7) | (T::kFmt << 10) |
                                       ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
            constexpr uint32_t lboA = (kBM / 8) * 128, lboB = (BNL / 8) * 128;
            // slice pairs in product order (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
            // (1,2) (2,1) (2,2), one nibble per product
            constexpr uint64_t kPa = 0x221210100ull, kPb = 0x212012010ull;
            // slice products: split-BF16 3 / 6 / 9; 3xTF32 hi.hi, hi.lo, lo.hi
            const int nprod = KIND == GK_BF16X3 ? d.nprod : (KIND == GK_TF32X3 ? 3 : 1);
            const uint32_t base = smem_u32(ops);
            // descriptors of stage slot 0, slice 0, first K step: every other
            // operand tile differs only in its start address, whose field is
            // the descriptor's low bits (address >> 4, below 2^14 for any
            // shared-memory offset), so adding (offset >> 4) moves it.  With
            // the products unrolled the issuing thread spends a few
            // independent instructions per MMA (a dependent chain per MMA
            // left the N = 128 tensor pipe idle most of the time).
            const uint64_t ad0 = smem_desc(base, lboA, 128);
            const uint64_t bd0 = smem_desc(base + T::kSlices * SP::kATile, lboB, 128);
            auto issue_stage = [&](auto np, uint64_t as, uint64_t bs, uint32_t dt, bool first) {
                constexpr int NP = decltype(np)::value;
#pragma unroll
                for (int ks = 0; ks < T::kKsteps; ++ks) {
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        const uint32_t qa = (uint32_t)(kPa >> (4 * q)) & 15u, qb = (uint32_t)(kPb >> (4 * q)) & 15u;
                        const uint64_t ad = as + (uint64_t)((qa * SP::kATile + ks * 2 * lboA) >> 4);
                        const uint64_t bd = bs + (uint64_t)((qb * SP::kBTile + ks * 2 * lboB) >> 4);
                        // each accumulator starts from zero with its own
                        // first product of the unit
                        const bool fresh = first && ks == 0 && q == (split && q > 0 ? 1 : 0);
                        const uint32_t dq = split && q > 0 ? dt + (uint32_t)BN : dt;
                        mma_issue<KIND, PAIR>(dq, ad, bd, idesc, !fresh);
                    }
                }
            };
            int64_t g = 0;
            int64_t u = 0;  // accumulation units (tiles, or K chunks of tiles)
            bool stop = false;
            auto commit = [&](uint64_t *bar) {
                if constexpr (PAIR) mma_commit2(bar, (uint16_t)3);  // both CTAs' barriers
                else mma_commit(bar);
            };
            for (int64_t tile = d.tile_begin + slot0; tile < d.num_tiles && !stop; tile += nslots) {
                const int nkt_t = BATCH ? (int)((tile_desc<BATCH>(d, tile).K + BK - 1) / BK) : nkt;
                const int cstg_t = BATCH ? nkt_t : cstg, nch_t = BATCH ? 1 : nch;
                for (int c = 0; c < nch_t && !stop; ++c, ++u) {
                    const int buf = (int)(u % nbuf);
                    if (u >= nbuf && !bwait(&tempty[buf], (uint32_t)(((u / nbuf) - 1) & 1))) {
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    // split: the (0,0) products at column 0, the others at BN
                    const uint32_t dt = tmem + (uint32_t)(buf * BN);
                    const int kt_end = min(nkt_t, (c + 1) * cstg_t);
                    for (int kt = c * cstg_t; kt < kt_end; ++kt, ++g) {
                        const int s = (int)(g % STAGES);
                        if (*abort_flag || !bwait(&full[s], (uint32_t)((g / STAGES) & 1))) {
                            stop = true;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t so = (uint64_t)((s * SP::kStage) >> 4);
                        const bool first = kt == c * cstg_t;
                        if constexpr (KIND == GK_BF16X3) {
                            if (nprod == 6) issue_stage(std::integral_constant<int, 6>{}, ad0 + so, bd0 + so, dt, first);
                            else if (nprod == 3) issue_stage(std::integral_constant<int, 3>{}, ad0 + so, bd0 + so, dt, first);
                            else issue_stage(std::integral_constant<int, 9>{}, ad0 + so, bd0 + so, dt, first);
                        } else {
                            issue_stage(std::integral_constant<int, KIND == GK_TF32X3 ? 3 : 1>{}, ad0 + so, bd0 + so, dt,
                                        first);
                        }
                        commit(&empty[s]);
                    }
                    commit(&tfull[buf]);  // arrives when this unit's MMAs are done
                }
            }
            if (stop) {
                *abort_flag = 1;
                atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
            }
            // nothing issued may still run when the tensor memory is freed
            if constexpr (PAIR) mma_commit2(drain, (uint16_t)1);
            else mma_commit(drain);
            mbar_wait(drain, 0);
        } else if (PAIR && !BATCH && d.pk == 3 && lane == 0) {
            // both inputs pre-converted, second CTA of a pair: its copies
            // complete on its own stage barriers; this lane passes each
            // completed stage on to the issuer's barrier in the first CTA
            int64_t g = 0;
            bool stop = false;
            for (int64_t tile = d.tile_begin + slot0; tile < d.num_tiles && !stop; tile += nslots) {
                for (int kt = 0; kt < nkt; ++kt, ++g) {
                    const int s = (int)(g % STAGES);
                    if (*abort_flag || !mbar_wait(&full[s], (uint32_t)((g / STAGES) & 1))) {
                        stop = true;
                        break;
                    }
                    mbar_arrive_remote(mapa_shared(smem_u32(&full[s]), 0u));
                }
            }
            if (stop) {
                *abort_flag = 1;
                atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- epilogue
        const int et = threadIdx.x;  // 0..127 = accumulator row = TMEM lane
        // E4M3: the products carry both inputs' scales
        float alpha_e = d.alpha;
        if constexpr (KIND == GK_E4M3) alpha_e = d.alpha * d.qscale[0] * d.qscale[1];
        int it = 0;
        int64_t u = 0;
        for (int64_t tile = d.tile_begin + slot0; tile < d.num_tiles; tile += nslots, ++it) {
            const int nch_t = BATCH ? 1 : nch;
            float *__restrict__ C;
            int64_t *cn = cN + (it & 1) * BN;
            int64_t nval, lin = 0, on0 = 0, om = -1;
            bool rec_ok = true;
            if (BATCH && grouped) {
                // the tile's record, left by the converters
                const int r = it % kRecMod;
                rec_ok = mbar_wait(&rfull[r], (uint32_t)((it / kRecMod) & 1));
                const int64_t *rec = trec + r * 8;
                C = (float *)rec[0];
                nval = rec[5];
                lin = rec[3];
                om = et < rec[1] ? rec[4] + (int64_t)et * rec[2] : -1;
            } else {
                const GettDesc &P = tile_desc<BATCH>(d, tile);
                int64_t boA, boB, boC;
                const int64_t lt = batch_offsets(P, BATCH ? tile - P.tile0 : tile, boA, boB, boC);
                C = P.C + boC;
                int64_t mt;
                const int64_t nt = divmod(lt, P.tiles_m, mt);
                // pairs: this CTA's 128 rows of the 256-row tile; every CTA
                // holds all BN columns of its rows
                const int64_t m0 = (PAIR ? 2 * mt + crank : mt) * kBM, n0 = nt * BN;
                // one stride across the tile's columns: no column table
                nval = min((int64_t)BN, P.N - n0);
                if (P.nn == 0) {
                    lin = 0;  // a single column: the table
                } else if (P.n_chain) {
                    lin = P.n_sC[0];
                    on0 = n0 * lin;
                } else if ([&] { int64_t rr; divmod(n0, P.n_ext[0], rr); return rr + BN <= P.n_ext[0]; }()) {
                    int64_t ob = 0;
                    decode(n0, P.nn, P.n_ext, P.n_sB, P.n_sC, ob, on0);
                    lin = P.n_sC[0];
                }
                if (lin == 0) {
                    for (int j = et; j < BN; j += kEpiThreads) {
                        int64_t nn = n0 + j, ob = 0, oc = -1;
                        if (nn < P.N) {
                            oc = 0;
                            decode(nn, P.nn, P.n_ext, P.n_sB, P.n_sC, ob, oc);
                        }
                        cn[j] = oc;
                    }
                }
                {
                    int64_t mm = m0 + et, oa = 0;
                    if (mm < P.M) {
                        om = 0;
                        decode(mm, P.nm, P.m_ext, P.m_sA, P.m_sC, oa, om);
                    }
                }
            }
            if (!rec_ok) {
                *abort_flag = 1;
                atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
            }
            if (role_sync_or<2, kEpiThreads>(*abort_flag)) break;
            if (BATCH && grouped && et == 0) mbar_arrive(&rempty[it % kRecMod]);  // record read by all
            const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
            bool aborted = false;
            for (int c = 0; c < nch_t; ++c, ++u) {
                const int buf = (int)(u % nbuf);
                bool ok = bwait(&tfull[buf], (uint32_t)((u / nbuf) & 1));
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld needs the whole warp
                if (!ok) {
                    *abort_flag = 1;
                    atomicExch(d.status, (int)TC_ERROR_TIMEOUT);
                    aborted = true;
                    break;  // the next role barrier sees the abort
                }
                tc_fence_after();
                const uint32_t acc = tmem + lane_off + (uint32_t)(buf * BN);
                const uint32_t hi = tmem + lane_off + (uint32_t)(2 * BN), lo = hi + (uint32_t)BN;
                const bool last = c == nch_t - 1;
                if constexpr (!COMP) {
                    if (split) {
                        // (0,0) products + the smaller ones, one rounding
#pragma unroll 1
                        for (int c0 = 0; c0 < BN; c0 += 32) {
                            uint32_t r[32];
                            tmem_ld32_sum(acc + (uint32_t)c0, acc + (uint32_t)(BN + c0), r);
                            store_cols<32>(r, C, om, c0, lin, on0, nval, cn, alpha_e, d.beta, d.init);
                        }
                    } else {
#pragma unroll 1
                        for (int c0 = 0; c0 < BN; c0 += 64) {
                            uint32_t r[64];
                            tmem_ld64(acc + (uint32_t)c0, r);
                            store_cols<64>(r, C, om, c0, lin, on0, nval, cn, alpha_e, d.beta, d.init);
                        }
                    }
                } else {
#pragma unroll 1
                    for (int c0 = 0; c0 < BN; c0 += 32) {
                        uint32_t r[32];
                        tmem_ld32(acc + (uint32_t)c0, r);
                        if constexpr (COMP) {
                            // two 32-register arrays live at a time (r and t)
                            if (nch_t > 1) {
                                if (c == 0) {
                                    tmem_st32(hi + (uint32_t)c0, r);
                                    tmem_st32_zero(lo + (uint32_t)c0);
                                    continue;
                                }
                                uint32_t t[32];
                                if (last) {  // result = hi + (lo + chunk): one rounding per step
                                    tmem_ld32(lo + (uint32_t)c0, t);
#pragma unroll
                                    for (int j = 0; j < 32; ++j)
                                        r[j] = __float_as_uint(__fadd_rn(__uint_as_float(t[j]), __uint_as_float(r[j])));
                                    tmem_ld32(hi + (uint32_t)c0, t);
#pragma unroll
                                    for (int j = 0; j < 32; ++j)
                                        r[j] = __float_as_uint(__fadd_rn(__uint_as_float(t[j]), __uint_as_float(r[j])));
                                } else {  // (hi, err) = TwoSum(hi, chunk); lo += err
                                    tmem_ld32(hi + (uint32_t)c0, t);
#pragma unroll
                                    for (int j = 0; j < 32; ++j) {
                                        const float a = __uint_as_float(t[j]), b = __uint_as_float(r[j]);
                                        const float s2 = __fadd_rn(a, b);
                                        const float bb = __fsub_rn(s2, a);
                                        t[j] = __float_as_uint(s2);
                                        r[j] = __float_as_uint(
                                            __fadd_rn(__fsub_rn(a, __fsub_rn(s2, bb)), __fsub_rn(b, bb)));
                                    }
                                    tmem_st32(hi + (uint32_t)c0, t);
                                    tmem_ld32(lo + (uint32_t)c0, t);
#pragma unroll
                                    for (int j = 0; j < 32; ++j)
                                        t[j] = __float_as_uint(__fadd_rn(__uint_as_float(t[j]), __uint_as_float(r[j])));
                                    tmem_st32(lo + (uint32_t)c0, t);
                                    continue;
                                }
                            }
                        }
                        store_cols<32>(r, C, om, c0, lin, on0, nval, cn, alpha_e, d.beta, d.init);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) arrive_issuer(&tempty[buf]);
            }
            if (aborted) continue;
        }
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) {
        // neither CTA frees its tensor memory or leaves while the pair's
        // MMAs or the other CTA's arrivals may still reach it
        cluster_sync_all();
        if (warp == kMmaWarp) {
            tc_fence_after();
            tmem_dealloc2(tmem, kTmemCols);
        }
    } else if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// Pre-conversion of one FP32 input (op 0 = A, 1 = B): for every row tile
// (rows rows) and K stage (bk positions) the stage image the converter warps
// would write to shared memory -- the split-BF16 slices or TF32 words in the
// core-matrix layout, slice after slice -- with zeros for rows past the
// extent and K positions past K.  One thread per 16-byte core-matrix row.
template <int KIND>
__global__ void __launch_bounds__(128) pack_kernel(const GettDesc d, int op, int rows, int bk, int64_t rtiles,
                                                   char *out) {
    using T = KindTraits<KIND, kBKT>;  // chunk and element size do not depend on BK
    constexpr int CH = T::kChunk;
    const int kcn = bk / CH;
    const int64_t nkt = (d.K + bk - 1) / bk;
    const int64_t R = op == 0 ? d.M : d.N;
    // rtiles row tiles (the last ones may lie wholly past R: zeros)
    const int64_t total = rtiles * nkt * kcn * rows;
    // let the GETT that depends on this grid launch now (its converters
    // wait for this grid's completion before reading the images)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const float *__restrict__ src = (const float *)(op == 0 ? d.A : d.B);
    const int nr = op == 0 ? d.nm : d.nn;
    const int64_t *rext = op == 0 ? d.m_ext : d.n_ext;
    const int64_t *rs = op == 0 ? d.m_sA : d.n_sB;
    const int64_t *ks = op == 0 ? d.k_sA : d.k_sB;
    const int slice = rows * bk * T::kElemBytes;
    // when the innermost K mode holds whole chunks (its extent a multiple
    // of CH; then so is K), a chunk's K positions are one run of that mode:
    // one decode per chunk, and 16-byte loads where the run is contiguous
    // and aligned
    const bool whole = d.nk > 0 && d.k_ext[d.nk - 1] % CH == 0;
    const int64_t s_in = d.nk > 0 ? ks[d.nk - 1] : 0;
    // E4M3: the input divided by its scale (a power of two, written by the
    // scale kernel earlier in the stream)
    float qs = 1.0f;
    if constexpr (KIND == GK_E4M3) qs = 1.0f / d.qscale[op];
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x) {
        // rows fastest, then K chunks, K stages, row tiles (divmod: 32-bit
        // divisions whenever the values fit)
        int64_t row, kc, kt;
        int64_t q = divmod(c, rows, row);
        q = divmod(q, kcn, kc);
        const int64_t rt = divmod(q, nkt, kt);
        int64_t r = rt * rows + row, ro = -1;
        if (r < R) {
            ro = 0;
            for (int m = 0; m < nr; ++m) {  // first row mode fastest
                int64_t v;
                r = divmod(r, rext[m], v);
                ro += v * rs[m];
            }
        }
        float x[CH];
        if (whole) {
            int64_t k = kt * bk + kc * CH, ko = 0;
#pragma unroll
            for (int e = 0; e < CH; ++e) x[e] = 0.0f;
            if (ro >= 0 && k < d.K) {
                for (int m = d.nk - 1; m >= 0; --m) {
                    int64_t v;
                    k = divmod(k, d.k_ext[m], v);
                    ko += v * ks[m];
                }
                const float *p = src + ro + ko;
                if (s_in == 1 && ((uintptr_t)p & 15) == 0) {
#pragma unroll
                    for (int e = 0; e < CH; e += 4) {
                        const float4 v4 = *reinterpret_cast<const float4 *>(p + e);
                        x[e] = v4.x;
                        x[e + 1] = v4.y;
                        x[e + 2] = v4.z;
                        x[e + 3] = v4.w;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < CH; ++e) x[e] = p[e * s_in];
                }
            }
        }
#pragma unroll
        for (int e = 0; e < CH && !whole; ++e) {
            int64_t k = kt * bk + kc * CH + e;
            x[e] = 0.0f;
            if (ro >= 0 && k < d.K) {
                int64_t ko = 0;
                for (int m = d.nk - 1; m >= 0; --m) {  // innermost K mode fastest
                    int64_t v;
                    k = divmod(k, d.k_ext[m], v);
                    ko += v * ks[m];
                }
                x[e] = src[ro + ko];
            }
        }
        char *dst = out + (rt * nkt + kt) * (int64_t)(T::kSlices * slice) + (kc * (rows / 8) + row / 8) * 128 +
                    (row % 8) * 16;
        store_converted<KIND, CH>(x, dst, slice, qs);
    }
}

// Pre-conversion of one 16-bit input (BF16 / FP16; op 0 = A, 1 = B) for the
// both-inputs path: its stage images in the core-matrix layout, the values
// as they are, zeros for rows past the extent and K positions past K.  One
// thread per 16-byte core-matrix row (8 K positions of one row).
__global__ void __launch_bounds__(128) pack16_kernel(const GettDesc d, int op, int rows, int bk, int64_t rtiles,
                                                     char *out) {
    constexpr int CH = 8;
    const int kcn = bk / CH;
    const int64_t nkt = (d.K + bk - 1) / bk;
    const int64_t R = op == 0 ? d.M : d.N;
    const int64_t total = rtiles * nkt * kcn * rows;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const uint16_t *__restrict__ src = (const uint16_t *)(op == 0 ? d.A : d.B);
    const int nr = op == 0 ? d.nm : d.nn;
    const int64_t *rext = op == 0 ? d.m_ext : d.n_ext;
    const int64_t *rs = op == 0 ? d.m_sA : d.n_sB;
    const int64_t *ks = op == 0 ? d.k_sA : d.k_sB;
    const int64_t slice = (int64_t)rows * bk * 2;
    const bool whole = d.nk > 0 && d.k_ext[d.nk - 1] % CH == 0;  // a chunk is one run of the innermost K mode
    const int64_t s_in = d.nk > 0 ? ks[d.nk - 1] : 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t row, kc, kt;
        int64_t q = divmod(c, rows, row);
        q = divmod(q, kcn, kc);
        const int64_t rt = divmod(q, nkt, kt);
        int64_t r = rt * rows + row, ro = -1;
        if (r < R) {
            ro = 0;
            for (int m = 0; m < nr; ++m) {
                int64_t v;
                r = divmod(r, rext[m], v);
                ro += v * rs[m];
            }
        }
        uint16_t x[CH];
#pragma unroll
        for (int e = 0; e < CH; ++e) x[e] = 0;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        bool vec = false;
        if (ro >= 0 && whole) {
            int64_t k = kt * bk + kc * CH, ko = 0;
            if (k < d.K) {
                for (int m = d.nk - 1; m >= 0; --m) {
                    int64_t v;
                    k = divmod(k, d.k_ext[m], v);
                    ko += v * ks[m];
                }
                const uint16_t *p = src + ro + ko;
                if (s_in == 1 && ((uintptr_t)p & 15) == 0) {
                    w = *reinterpret_cast<const uint4 *>(p);
                    vec = true;
                } else {
#pragma unroll
                    for (int e = 0; e < CH; ++e) x[e] = p[e * s_in];
                }
            }
        } else if (ro >= 0) {
#pragma unroll
            for (int e = 0; e < CH; ++e) {
                int64_t k = kt * bk + kc * CH + e;
                if (k < d.K) {
                    int64_t ko = 0;
                    for (int m = d.nk - 1; m >= 0; --m) {  // innermost K mode fastest
                        int64_t v;
                        k = divmod(k, d.k_ext[m], v);
                        ko += v * ks[m];
                    }
                    x[e] = src[ro + ko];
                }
            }
        }
        if (!vec)
            w = make_uint4(x[0] | ((uint32_t)x[1] << 16), x[2] | ((uint32_t)x[3] << 16), x[4] | ((uint32_t)x[5] << 16),
                           x[6] | ((uint32_t)x[7] << 16));
        char *dst = out + (rt * nkt + kt) * slice + (kc * (rows / 8) + row / 8) * 128 + (row % 8) * 16;
        *(uint4 *)dst = w;
    }
}

// E4M3 scales: the largest magnitude of each input over its modes, then the
// power of two s with max / s <= 448 (E4M3's largest finite value), so that
// dividing by s is exact and no input saturates.
struct AbsmaxDesc {
    int n;            // modes (0: the operand is dense, read [0, total) linearly)
    int64_t ext[kMaxModes], stride[kMaxModes];
    int64_t total;
    const float *src;
    unsigned *out;    // the maximum as float bits (non-negative: ordered as integers)
};

__global__ void __launch_bounds__(256) absmax_kernel(const AbsmaxDesc a) {
    float m = 0.0f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t off = e;
        if (a.n) {
            int64_t r = e;
            off = 0;
            for (int k = 0; k < a.n; ++k) {
                const int64_t x = r % a.ext[k];
                r /= a.ext[k];
                off += x * a.stride[k];
            }
        }
        m = fmaxf(m, fabsf(a.src[off]));  // a NaN input is passed over
    }
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(a.out, __float_as_uint(m));
}

__global__ void e4m3_scale_kernel(const unsigned *mx, float *scale) {
    if (threadIdx.x < 2) {
        const float m = __uint_as_float(mx[threadIdx.x]);
        float sc = 1.0f;
        if (m > 0.0f && isfinite(m)) sc = ldexpf(1.0f, (int)ceilf(log2f(m / 448.0f)));
        scale[threadIdx.x] = sc;
    }
}

// ------------------------------------------------------------------ host side
int g_gett_sms = 0;

template <int KIND, int BN, int STAGES, int BK, int SSTG, bool COMP = false, bool BATCH = false, bool PAIR = false>
tc_status launch_gett(const GettDesc &d, const CUtensorMap &ta, const CUtensorMap &tb, cudaStream_t st) {
    using SP = SmemPlan<KIND, BN, STAGES, BK, SSTG, BATCH, PAIR>;
    static_assert(SP::kTotal <= 227 * 1024, "shared memory budget");
    // at least 116 KB so that one CTA (and one tensor-memory allocation of
    // up to 512 columns) occupies each SM
    constexpr int kSmem = SP::kTotal > 116 * 1024 ? SP::kTotal : 116 * 1024;
    auto kern = gett_tc_kernel<KIND, BN, STAGES, BK, SSTG, COMP, BATCH, PAIR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    if (g_gett_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_gett_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_gett_sms <= 0) g_gett_sms = 1;
    }
    // after a pre-pass (d.pk): programmatic stream serialization, so the
    // kernel's prologue and the TMA stream overlap the pre-pass
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (!BATCH && d.pk) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    int64_t grid = std::min<int64_t>(d.num_tiles - d.tile_begin, g_gett_sms);
    if constexpr (PAIR) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = 2;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
        // one pair per two SMs that can hold one at the same time (the
        // persistent walk assumes every pair is resident)
        static int max_pairs = 0;
        if (max_pairs == 0) {
            cudaLaunchConfig_t q = cfg;
            q.gridDim = dim3((unsigned)(2 * (g_gett_sms / 2)));
            q.attrs = &attr[na - 1];
            q.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, kern, &q) != cudaSuccess || n <= 0) {
                cudaGetLastError();
                n = g_gett_sms / 2;
            }
            max_pairs = std::min(n, g_gett_sms / 2);
        }
        grid = 2 * std::min<int64_t>(d.num_tiles - d.tile_begin, max_pairs);
    }
    cfg.gridDim = dim3((unsigned)grid);
    cfg.attrs = attr;
    cfg.numAttrs = na;
    e = cudaLaunchKernelEx(&cfg, kern, d, ta, tb);
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    e = cudaGetLastError();
    return e == cudaSuccess ? TC_SUCCESS : fail(TC_ERROR_CUDA, cudaGetErrorString(e));
}

template <int KIND>
tc_status launch_kind(GettDesc &d, int bn, bool tma, bool comp, bool pair, const CUtensorMap &ta,
                      const CUtensorMap &tb, cudaStream_t st) {
    d.tiles_n = (d.N + bn - 1) / bn;
    d.num_tiles = d.tiles_m * d.tiles_n * batch_count(d);
    if (d.tile_frac < 1.0) d.num_tiles = std::max<int64_t>(1, (int64_t)(d.num_tiles * d.tile_frac));
    // CTA pairs with both inputs pre-converted (pair tiles of 256 x BN;
    // per CTA 128 rows of A and BN/2 of B in each 32-position stage):
    // split-BF16 256 x 256 (four stages) or compensated 256 x 128, whose
    // two chunk accumulators and (hi, lo) take each CTA's 512 tensor-memory
    // columns
    if (pair && d.pk == 3) {
        if constexpr (KIND == GK_BF16X3) {
            if (comp) return launch_gett<KIND, 128, 5, kBK, 0, true, false, true>(d, ta, tb, st);
            if (bn == 256) return launch_gett<KIND, 256, 4, kBK, 0, false, false, true>(d, ta, tb, st);
        }
        return fail(TC_ERROR_UNSUPPORTED_DTYPE, "no CTA-pair launch for this pre-converted form");
    }
    // CTA pairs (tiles of 256 x 256): four operand stages of 128 + 128
    // rows and three staging slots of two-stage boxes
    if constexpr (KIND == GK_BF16X3 || KIND == GK_TF32) {
        if (pair) return launch_gett<KIND, 256, 4, kBKT, 3, false, false, true>(d, ta, tb, st);
    }
    // <KIND, BN, operand stages, BK, staging slots (boxes of up to two stages; 0 = no TMA)>
    if constexpr (KIND == GK_BF16X3) {
        if (comp) {  // 128 x 128 tiles: two chunk accumulators and (hi, lo) fill the tensor memory
            if (tma) return launch_gett<KIND, 128, 3, kBKT, 3, true>(d, ta, tb, st);
            return launch_gett<KIND, 128, 4, kBK, 0, true>(d, ta, tb, st);
        }
    }
    if constexpr (KIND == GK_E4M3) {  // global-load path only: 32-K stages of 1-byte elements
        if (bn == 256) return launch_gett<KIND, 256, 6, kBK, 0>(d, ta, tb, st);
        return launch_gett<KIND, 128, 8, kBK, 0>(d, ta, tb, st);
    } else if constexpr (KIND == GK_TF32X3) {  // two 4-byte slices per operand: 192 KB of rings
        if (comp) {
            if (tma) return launch_gett<KIND, 128, 3, kBKT, 3, true>(d, ta, tb, st);
            return launch_gett<KIND, 128, 3, kBK, 0, true>(d, ta, tb, st);
        }
        if (tma) {
            if (bn == 128) return launch_gett<KIND, 128, 3, kBKT, 3>(d, ta, tb, st);
            return launch_gett<KIND, 256, 2, kBKT, 2>(d, ta, tb, st);
        }
        if (bn == 256) return launch_gett<KIND, 256, 2, kBK, 0>(d, ta, tb, st);
        return launch_gett<KIND, 128, 3, kBK, 0>(d, ta, tb, st);
    } else {
    if (tma) {  // 16-K stages, staged input boxes
        if (bn == 128) {
            if constexpr (KIND == GK_BF16X3) return launch_gett<KIND, 128, 3, kBKT, 3>(d, ta, tb, st);
            else if constexpr (KIND == GK_TF32) return launch_gett<KIND, 128, 4, kBKT, 4>(d, ta, tb, st);
            else return launch_gett<KIND, 128, 6, kBKT, 8>(d, ta, tb, st);
        }
        // two operand stages, three staging slots: the staging ring covers
        // the box latency (3 slots beat 2 by 10-20 % on 512^3 i=j=16)
        if constexpr (KIND == GK_BF16X3) return launch_gett<KIND, 256, 2, kBKT, 3>(d, ta, tb, st);
        else if constexpr (KIND == GK_TF32) return launch_gett<KIND, 256, 2, kBKT, 3>(d, ta, tb, st);
        else return launch_gett<KIND, 256, 4, kBKT, 4>(d, ta, tb, st);
    }
    if (bn == 256) {
        if constexpr (KIND == GK_BF16X3) return launch_gett<KIND, 256, 2, kBK, 0>(d, ta, tb, st);
        else if constexpr (KIND == GK_TF32) return launch_gett<KIND, 256, 3, kBK, 0>(d, ta, tb, st);
        else return launch_gett<KIND, 256, 6, kBK, 0>(d, ta, tb, st);
    }
    if constexpr (KIND == GK_BF16X3) return launch_gett<KIND, 128, 4, kBK, 0>(d, ta, tb, st);
    else if constexpr (KIND == GK_TF32) return launch_gett<KIND, 128, 6, kBK, 0>(d, ta, tb, st);
    else return launch_gett<KIND, 128, 8, kBK, 0>(d, ta, tb, st);
    }  // not TF32X3
}

// Distinct 32-byte sectors one warp touches on its first load under a
// global-load mapping (0: rows across lanes, 1: K chunks across lanes).
int64_t sectors_for(int map, int rows, int chunk, int elem_bytes, int nrow_modes,
                    const int64_t *row_ext, const int64_t *row_s, int nk, const int64_t *k_ext,
                    const int64_t *k_s) {
    const int KC = kBK / chunk;
    std::vector<int64_t> secs;
    for (int lane = 0; lane < 32; ++lane) {
        int row, kc;
        if (map == 1) { row = lane / KC; kc = lane % KC; }
        else { row = lane % rows; kc = lane / rows; }
        int64_t r = row, off = 0;
        for (int m = 0; m < nrow_modes; ++m) {
            off += (r % row_ext[m]) * row_s[m];
            r /= row_ext[m];
        }
        int64_t k = (int64_t)kc * chunk;
        for (int m = nk - 1; m >= 0; --m) {
            off += (k % k_ext[m]) * k_s[m];
            k /= k_ext[m];
        }
        secs.push_back(off * elem_bytes / 32);
    }
    std::sort(secs.begin(), secs.end());
    return std::unique(secs.begin(), secs.end()) - secs.begin();
}

// 16-byte vector loads along K are legal when the innermost K mode is
// contiguous, its extent is a multiple of the vector, every other stride of
// the operand is a multiple of the vector and the base is 16-byte aligned.
bool vec_ok(const void *base, int vec, int nrow_modes, const int64_t *row_s, int nk, const int64_t *k_ext,
            const int64_t *k_s) {
    if (nk == 0 || ((uintptr_t)base & 15) != 0) return false;
    if (k_s[nk - 1] != 1 || k_ext[nk - 1] % vec != 0) return false;
    for (int m = 0; m < nrow_modes; ++m)
        if (row_s[m] % vec != 0) return false;
    for (int m = 0; m < nk - 1; ++m)
        if (k_s[m] % vec != 0) return false;
    return true;
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool encoder() {
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    return true;
}

// Describes one input as a rank-5 TMA tensor over its own modes and stride
// so that one box is one pipeline stage: ROWS tile rows along its first row
// mode, the stage's BK K positions along its K modes.  Returns false when
// TMA cannot describe it (the operand then takes the global-load path).
// nrow/row_ext/row_s: the operand's row modes (M for A, N for B), first
// mode fastest; K modes as in the descriptor (outermost first).
bool plan_tma_operand(const Plan &p, int opnd, const void *base, int in_bytes, int rows, int nrow,
                      const int64_t *row_ext, const int64_t *row_s, int nk, const int64_t *k_ext,
                      const int64_t *k_s, GettDesc &d, CUtensorMap &map, int kpb) {
    const int o = opnd == OP_A ? 0 : 1;
    if (((uintptr_t)base & 15) != 0 || nrow < 1) return false;
    if (row_ext[0] % rows != 0) return false;  // tiles must be boxes of the first row mode
    // the stage's K positions: whole innermost K modes, then part of the next
    int64_t cover = 1;
    std::vector<int64_t> kbox(nk, 1);
    int m = nk - 1;
    for (; m >= 0 && cover < kpb; --m) {
        if (cover * k_ext[m] <= kpb) {
            kbox[m] = k_ext[m];
            cover *= k_ext[m];
        } else {
            if (k_ext[m] % (kpb / cover) != 0 || kpb % cover != 0) return false;
            kbox[m] = kpb / cover;
            cover = kpb;
        }
    }
    int64_t K = 1;
    for (int x = 0; x < nk; ++x) K *= k_ext[x];
    if (cover != kpb && cover != K) return false;
    // tensor dimensions: the operand's own modes (split K modes share one),
    // the stride-1 mode first
    struct Dim { int64_t ext, stride; int64_t box; };
    std::vector<Dim> dims;
    auto dim_of_stride = [&](int64_t stride) -> int {
        for (size_t x = 0; x < dims.size(); ++x)
            if (dims[x].stride == stride) return (int)x;
        return -1;
    };
    const Layout &L = p.op[opnd];
    for (int x = 0; x < L.n; ++x) dims.push_back({p.ext[L.idx[x]], L.stride[x], 1});
    std::stable_sort(dims.begin(), dims.end(), [](const Dim &a, const Dim &b) { return a.stride < b.stride; });
    if (dims.empty() || dims[0].stride != 1 || (int)dims.size() > kTmaRank) return false;
    for (int x = 0; x < nrow; ++x) {
        int dd = dim_of_stride(row_s[x]);
        if (dd < 0) return false;
        d.row_dim[o][x] = dd;
        if (x == 0) dims[dd].box = rows;
    }
    for (int x = 0; x < nk; ++x) {
        // a split K mode has stride = base stride * inner extent: map it to
        // the tensor dimension of its base stride with a multiplier
        int dd = dim_of_stride(k_s[x]);
        int64_t mul = 1;
        if (dd < 0) {
            for (size_t y = 0; y < dims.size() && dd < 0; ++y)
                if (dims[y].stride > 0 && k_s[x] % dims[y].stride == 0 && k_s[x] / dims[y].stride < dims[y].ext &&
                    dims[y].ext % (k_s[x] / dims[y].stride) == 0) {
                    dd = (int)y;
                    mul = k_s[x] / dims[y].stride;
                }
            if (dd < 0) return false;
        }
        d.k_dim[o][x] = dd;
        d.k_mul[o][x] = mul;
        if (kbox[x] > 1) dims[dd].box = std::max<int64_t>(dims[dd].box, kbox[x] * mul);
    }
    // box limits and the 16-byte rules
    for (auto &dm : dims)
        if (dm.box > 256) return false;
    if ((dims[0].box * in_bytes) % 16 != 0) return false;
    for (size_t x = 1; x < dims.size(); ++x)
        if ((dims[x].stride * in_bytes) % 16 != 0) return false;
    // staging offsets: box laid out with dimension 0 fastest
    std::vector<int64_t> bstride(dims.size(), 1);
    for (size_t x = 1; x < dims.size(); ++x) bstride[x] = bstride[x - 1] * dims[x - 1].box;
    int64_t box_elems = bstride.back() * dims.back().box;
    if (box_elems != (int64_t)rows * kpb && box_elems != (int64_t)rows * K) return false;
    d.srow[o] = (int)bstride[d.row_dim[o][0]];
    bool v4 = true;
    for (int k = 0; k < kpb; ++k) {
        int64_t kk = k, off = 0;
        bool valid = k < K;
        for (int x = nk - 1; x >= 0; --x) {
            int64_t v = kk % kbox[x];
            kk /= kbox[x];
            off += v * d.k_mul[o][x] * bstride[d.k_dim[o][x]];
        }
        d.sk[o][k] = valid ? (int)off : 0;
        if (k % 4 == 0 && (off % 4 != 0)) v4 = false;
        if (k % 4 != 0 && off != d.sk[o][k - 1] + 1) v4 = false;
    }
    if (d.srow[o] % 4 != 0 || in_bytes != 4) v4 = false;
    d.sk_vec4[o] = v4 ? 1 : 0;
    if (K < kpb || K % kpb != 0) return false;  // every box covers kpb valid K positions
    // encode (rank 5: unused dimensions have extent 1)
    if (!encoder()) return false;
    cuuint64_t gdim[kTmaRank], gstride[kTmaRank - 1];
    cuuint32_t box[kTmaRank], estr[kTmaRank];
    int64_t span = 16;
    for (auto &dm : dims) span = std::max<int64_t>(span, dm.stride * dm.ext * in_bytes);
    span = (span + 15) / 16 * 16;
    for (int x = 0; x < kTmaRank; ++x) {
        const bool real = x < (int)dims.size();
        gdim[x] = real ? (cuuint64_t)dims[x].ext : 1;
        box[x] = real ? (cuuint32_t)dims[x].box : 1;
        estr[x] = 1;
        if (x > 0) gstride[x - 1] = real ? (cuuint64_t)(dims[x].stride * in_bytes) : (cuuint64_t)span;
    }
    CUtensorMapDataType dt = in_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                           : (p.dtype == TC_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    CUresult r = g_encode(&map, dt, kTmaRank, const_cast<void *>(base), gdim, gstride, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    for (int x = (int)dims.size(); x < kTmaRank; ++x) {
        // unused dimensions: nothing maps there
    }
    return true;
}

}  // namespace

// bytes of a pre-converted input element: TF32 word, three BF16 slices, or
// two TF32 words
int image_bytes(tc_dtype dt) {
    return dt == TC_TF32 ? 4 : (dt == TC_TF32X3 ? 8 : ((dt == TC_BF16 || dt == TC_F16) ? 2 : (dt == TC_E4M3 ? 1 : 6)));
}

// Pre-conversion choice for the tensor-core GETT (0 none, 1 A, 2 B: the
// input with fewer elements, 3 both) and a bound on the stage images' bytes.
int pack_choice(const Plan &p, int64_t &bound) {
    bound = 0;
    // 16-bit and E4M3 inputs: the both-inputs form only
    const bool in16 = p.dtype == TC_BF16 || p.dtype == TC_F16 || p.dtype == TC_E4M3;
    if ((p.dtype != TC_BF16X3 && p.dtype != TC_TF32 && p.dtype != TC_TF32X3 && !in16) || p.gett_pack == 0 ||
        !p.batch.empty())
        return 0;
    int64_t M = 1, N = 1, K = 1;
    for (int id : p.freeA) M *= p.ext[id];
    for (int id : p.freeB) N *= p.ext[id];
    for (int id : p.contracted) K *= p.ext[id];
    // both inputs: on request (3), and by default for the compensated form
    // (whose 128-column tiles would otherwise convert each input once per
    // tile of the other) and wherever both M and N reach kPackBothMinMN (each
    // input would be converted or re-laid out at least four times); A's
    // rows round up to a 128-row tile, B's to a 256-row one, K to a
    // 32-position stage, plus the alignment of B's images
    int64_t comp_k = 0;
    if (p.dtype == TC_BF16X3 || p.dtype == TC_TF32X3) comp_k = p.comp_chunk < 0 ? kCompChunkK : p.comp_chunk;
    const bool comp = comp_k > 0 && K > comp_k;
    if (p.gett_pack == 3 || (p.gett_pack == 1 && (comp || (M >= kPackBothMinMN && N >= kPackBothMinMN)))) {
        const int64_t b2 = (M + N + 512) * (K + kBK - 1) * image_bytes(p.dtype) + 256;
        if (b2 <= kPackBothMaxBytes) {
            bound = b2;
            return 3;
        }
        if (p.gett_pack == 3) return 0;
    }
    if (in16) return 0;
    const bool a_small = M <= N;  // the same choice as the K order's "larger input"
    const int64_t R = a_small ? M : N;
    // auto: only where the two inputs are contiguous along different
    // contracted indices (a K order then has to trade one input's TMA rows
    // against the other's); elsewhere the small input streams well as it is
    auto unit_index = [&](int o) {
        for (int m = 0; m < p.op[o].n; ++m)
            if (p.op[o].stride_of(p.op[o].idx[m]) == 1) return p.op[o].idx[m];
        return -1;
    };
    const int us = unit_index(a_small ? OP_A : OP_B), ub = unit_index(a_small ? OP_B : OP_A);
    const bool permuted = us >= 0 && p.cls[us] == CLS_CONTRACTED && us != ub;
    // rows rounded up to a 256-row tile, K to a 32-position stage
    const int64_t b = (R + 255) * (K + kBK - 1) * image_bytes(p.dtype);
    if (b > kPackMaxBytes) return 0;
    if (p.gett_pack == 1 && (!permuted || (a_small ? M : N) * kPackRatio > (a_small ? N : M))) return 0;
    bound = b;
    return a_small ? 1 : 2;
}

size_t gett_workspace_bytes(const Plan &p) {
    int64_t bound = 0;
    pack_choice(p, bound);
    return (size_t)bound;
}

void gett_release(Plan &) {}

// The GETT's modes: M = free indices of A and N = free indices of B, each
// sorted by their C stride; the K order as below.  pk: the pre-converted
// input (0 none, 1 A, 2 B).
tc_status describe_modes(const Plan &p, int pk, GettDesc &d) {
    auto by_c_stride = [&](std::vector<int> ids) {
        std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) {
            return p.op[OP_C].stride_of(x) < p.op[OP_C].stride_of(y);
        });
        return ids;
    };
    std::vector<int> mi = by_c_stride(p.freeA), ni = by_c_stride(p.freeB);
    const int in_bytes = (p.dtype == TC_BF16 || p.dtype == TC_F16) ? 2 : 4;
    const int vec = 16 / in_bytes;
    // K order.  The innermost K mode is the contracted index with the
    // smallest stride in the larger input, so that operand streams along K.
    // When the other input is contiguous along a different contracted index
    // (A = iaj against B = jbic), the innermost index is split into
    // (outer, vec) and the other input's contiguous index goes between them:
    // a K stage then covers several values of it (whole 32-byte sectors, or
    // a TMA box at least 16 bytes wide) while the larger input keeps 16-byte
    // vectors.
    int64_t sizeA = 1, sizeB = 1;
    for (int m = 0; m < p.op[OP_A].n; ++m) sizeA *= p.ext[p.op[OP_A].idx[m]];
    for (int m = 0; m < p.op[OP_B].n; ++m) sizeB *= p.ext[p.op[OP_B].idx[m]];
    const int big = sizeB >= sizeA ? OP_B : OP_A, small = big == OP_B ? OP_A : OP_B;
    // a pre-converted smaller input (pk) is read as stage images, so the K
    // order follows the larger input alone
    std::vector<int> ki(p.contracted);
    std::stable_sort(ki.begin(), ki.end(), [&](int x, int y) {
        return p.op[big].stride_of(x) > p.op[big].stride_of(y);
    });
    struct KMode { int64_t ext, sA, sB; };
    std::vector<KMode> kmodes;
    for (int id : ki) kmodes.push_back({p.ext[id], p.op[OP_A].stride_of(id), p.op[OP_B].stride_of(id)});
    if (ki.size() >= 2 && !pk) {
        const int inner = ki.back();
        int other = -1;
        for (int id : ki)
            if (id != inner && p.op[small].stride_of(id) == 1) other = id;
        const int64_t ein = p.ext[inner];
        // Where K allows two-stage (32-position) TMA boxes, the larger input
        // keeps 32-byte runs (8 FP32 values) and the other input 16-byte runs
        // of its own index: that costs the fewest box rows per K position.
        // (The K order does not depend on the input path, so every path sums
        // in the same order.)
        int64_t ktot = 1;
        for (int id : ki) ktot *= p.ext[id];
        const int vsplit = (other >= 0 && in_bytes == 4 && ktot % kBoxK == 0 &&
                            ktot >= kTwoStageBoxMinK && ein % (2 * vec) == 0 && ein > 2 * vec &&
                            p.ext[other] % vec == 0)
                               ? 2 * vec
                               : vec;
        if (other >= 0 && p.op[big].stride_of(inner) == 1 && ein % vsplit == 0 && ein > vsplit &&
            p.op[small].stride_of(inner) != 1) {
            std::vector<KMode> km;
            for (int id : ki)
                if (id != inner && id != other)
                    km.push_back({p.ext[id], p.op[OP_A].stride_of(id), p.op[OP_B].stride_of(id)});
            const int64_t sAi = p.op[OP_A].stride_of(inner), sBi = p.op[OP_B].stride_of(inner);
            km.push_back({ein / vsplit, sAi * vsplit, sBi * vsplit});
            km.push_back({p.ext[other], p.op[OP_A].stride_of(other), p.op[OP_B].stride_of(other)});
            km.push_back({(int64_t)vsplit, sAi, sBi});
            kmodes = km;
        }
    }
    d.nm = (int)mi.size();
    d.nn = (int)ni.size();
    d.nk = (int)kmodes.size();
    if (d.nk > kMaxModes) return fail(TC_ERROR_INVALID_SPEC, "too many contracted modes for GETT");
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
    d.n_chain = 1;
    for (int m = 0; m + 1 < d.nn; ++m)
        if (d.n_sC[m + 1] != d.n_sC[m] * d.n_ext[m]) d.n_chain = 0;
    for (int m = 0; m < d.nk; ++m) {
        d.k_ext[m] = kmodes[m].ext;
        d.k_sA[m] = kmodes[m].sA;
        d.k_sB[m] = kmodes[m].sB;
        d.K *= kmodes[m].ext;
    }
    d.nb = (int)p.batch.size();
    for (int m = 0; m < d.nb; ++m) {
        const int id = p.batch[m];
        d.b_ext[m] = p.ext[id];
        d.b_sA[m] = p.op[OP_A].stride_of(id);
        d.b_sB[m] = p.op[OP_B].stride_of(id);
        d.b_sC[m] = p.op[OP_C].stride_of(id);
    }
    return TC_SUCCESS;
}


tc_status exec_gett(Plan &p, const void *alpha, const void *A, const void *B, const void *beta,
                    void *C, void *stream, const Probe *probe) {
    if (p.dtype == TC_F64 || p.dtype == TC_F32) return exec_gett_simt(p, alpha, A, B, beta, C, stream, probe);
    tc_status s = ensure_device_resources(p, 0);
    if (s != TC_SUCCESS) return s;
    p.last_stream = stream;
    GettDesc d;
    std::memset(&d, 0, sizeof(d));
    // a pre-converted smaller input is read as stage images, so the K order
    // follows the larger input alone
    int64_t pk_bound = 0;
    const int pk = pack_choice(p, pk_bound);
    s = describe_modes(p, pk, d);
    if (s != TC_SUCCESS) return s;
    const int in_bytes = (p.dtype == TC_BF16 || p.dtype == TC_F16) ? 2 : 4;
    const int vec = 16 / in_bytes;
    const int chunk = (p.dtype == TC_TF32 || p.dtype == TC_TF32X3) ? 4 : (p.dtype == TC_E4M3 ? 16 : 8);
    int bn = p.gett_bn == 128 || p.gett_bn == 256 ? p.gett_bn : (d.N >= 256 ? 256 : 128);
    // compensated accumulation (split-BF16 only): K chunks of comp_k elements
    int64_t comp_k = 0;
    if (p.dtype == TC_BF16X3 || p.dtype == TC_TF32X3) comp_k = p.comp_chunk < 0 ? kCompChunkK : p.comp_chunk;
    const bool comp = comp_k > 0 && d.K > comp_k;
    if (comp) bn = 128;
    // TMA staging for each operand TMA can describe (tiles of 128 x bn, or
    // in a CTA pair 128 rows of A and bn / 2 rows of B per CTA)
    CUtensorMap tmA, tmB;
    std::memset(&tmA, 0, sizeof(tmA));
    std::memset(&tmB, 0, sizeof(tmB));
    bool tma = false;
    d.spb = 1;
    auto plan_tma = [&](GettDesc &dd, CUtensorMap &ma, CUtensorMap &mb, int brows) -> bool {
        dd.tma[0] = pk != 1 && plan_tma_operand(p, OP_A, A, in_bytes, kBM, dd.nm, dd.m_ext, dd.m_sA, dd.nk, dd.k_ext,
                                                dd.k_sA, dd, ma, kBKT);
        dd.tma[1] = pk != 2 && plan_tma_operand(p, OP_B, B, in_bytes, brows, dd.nn, dd.n_ext, dd.n_sB, dd.nk,
                                                dd.k_ext, dd.k_sB, dd, mb, kBKT);
        bool any = dd.tma[0] || dd.tma[1];
        // boxes of two stages where the K modes allow them for at least as
        // many operands: each TMA box costs a fixed few hundred cycles on top
        // of its bytes, so fewer, larger boxes move more data per SM
        if (dd.K % kBoxK == 0 && dd.K >= kTwoStageBoxMinK) {
            GettDesc d2 = dd;
            CUtensorMap a2, b2;
            std::memset(&a2, 0, sizeof(a2));
            std::memset(&b2, 0, sizeof(b2));
            const bool ta = pk != 1 && plan_tma_operand(p, OP_A, A, in_bytes, kBM, dd.nm, dd.m_ext, dd.m_sA, dd.nk,
                                                        dd.k_ext, dd.k_sA, d2, a2, kBoxK);
            const bool tb = pk != 2 && plan_tma_operand(p, OP_B, B, in_bytes, brows, dd.nn, dd.n_ext, dd.n_sB, dd.nk,
                                                        dd.k_ext, dd.k_sB, d2, b2, kBoxK);
            if ((ta || tb) && (int)ta + (int)tb >= (int)(bool)dd.tma[0] + (int)(bool)dd.tma[1]) {
                dd = d2;
                dd.tma[0] = ta;
                dd.tma[1] = tb;
                ma = a2;
                mb = b2;
                dd.spb = kBoxK / kBKT;
                any = true;
            }
        }
        const int kpb = dd.spb * kBKT;
        dd.tma_bytes = (uint32_t)((dd.tma[0] ? kBM * kpb * in_bytes : 0) + (dd.tma[1] ? brows * kpb * in_bytes : 0));
        return any;
    };
    // CTA pairs: FP32-input tensor kinds on 256-wide tiles without
    // compensation, more than one 128-row tile, and every operand either
    // TMA-staged or pre-converted (the converters' grouped path)
    bool pair = false;
    // batch indices: the global-load path (the TMA warp and the
    // pre-converted images walk M and N tiles only)
    // (E4M3: the global-load path only)
    // (both inputs pre-converted: no input is staged)
    if (p.gett_tma && pk != 3 && p.dtype != TC_E4M3 && d.nb == 0 && d.K < (int64_t(1) << 31)) {  // 32-bit K positions in the TMA warp
        if (p.gett_pair && (p.dtype == TC_BF16X3 || p.dtype == TC_TF32) && !comp && bn == 256 && d.M > kBM) {
            GettDesc dp = d;
            CUtensorMap pa, pb;
            std::memset(&pa, 0, sizeof(pa));
            std::memset(&pb, 0, sizeof(pb));
            if (plan_tma(dp, pa, pb, bn / 2) && (dp.tma[0] || pk == 1) && (dp.tma[1] || pk == 2)) {
                d = dp;
                tmA = pa;
                tmB = pb;
                tma = true;
                pair = true;
            }
        }
        if (!pair) tma = plan_tma(d, tmA, tmB, bn);
    }
    // CTA pairs with both inputs pre-converted: no staging, so every
    // layout qualifies (more than one 128-row tile; split-BF16 on 256-wide
    // tiles or compensated)
    if (pk == 3 && p.gett_pair && d.M > kBM && d.nb == 0 && p.dtype == TC_BF16X3 && (comp || bn == 256))
        pair = true;
    if (comp) d.chunk_stages = (int)(comp_k / (tma ? kBKT : kBK));
    // global-load mappings (used by operands without TMA staging)
    auto pick = [&](const void *base, int rows, int nrow, const int64_t *rext, const int64_t *rs,
                    const int64_t *ks) {
        if (vec_ok(base, vec, nrow, rs, d.nk, d.k_ext, ks)) return 2;
        int64_t s0 = sectors_for(0, rows, chunk, in_bytes, nrow, rext, rs, d.nk, d.k_ext, ks);
        int64_t s1 = sectors_for(1, rows, chunk, in_bytes, nrow, rext, rs, d.nk, d.k_ext, ks);
        return s1 < s0 ? 1 : 0;
    };
    d.a_map = pick(A, kBM, d.nm, d.m_ext, d.m_sA, d.k_sA);
    d.b_map = pick(B, bn, d.nn, d.n_ext, d.n_sB, d.k_sB);
    d.A = A;
    d.B = B;
    d.C = (float *)C;
    d.alpha = *(const float *)alpha;
    d.beta = *(const float *)beta;
    d.init = d.beta == 0.0f ? 2 : 1;
    d.nprod = p.split_products;
    d.status = p.dev_status;
    d.tiles_m = pair ? (d.M + 2 * kBM - 1) / (2 * kBM) : (d.M + kBM - 1) / kBM;
    d.tile_frac = probe ? probe->fraction : 1.0;
    // split accumulators: split-BF16 without the compensated form; by
    // default only past 64 contracted positions (6K/16 > 24 accumulations
    // into one FP32 accumulator), where the roundings of the single
    // accumulator reach the 1e-6 level
    constexpr int64_t kSplitMinK = 65;
    const bool want_split = p.gett_split > 0 || (p.gett_split < 0 && d.K >= kSplitMinK);
    d.split = ((p.dtype == TC_BF16X3 || p.dtype == TC_TF32X3) && !comp && want_split) ? 1 : 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (p.dtype == TC_E4M3) {
        // the inputs' scales, written before the pre-passes and the GETT read
        // them (stream order)
        if (!p.qbuf) {
            cudaError_t e = cudaMalloc(&p.qbuf, 16);
            if (e != cudaSuccess) {
                p.qbuf = nullptr;
                return fail(TC_ERROR_OUT_OF_MEMORY, cudaGetErrorString(e));
            }
        }
        unsigned *mx = (unsigned *)p.qbuf;
        float *scale = (float *)((char *)p.qbuf + 8);
        cudaMemsetAsync(mx, 0, 8, st);
        for (int o = 0; o < 2; ++o) {
            const Layout &L = p.op[o == 0 ? OP_A : OP_B];
            AbsmaxDesc a;
            std::memset(&a, 0, sizeof(a));
            int64_t total = 1, span = 1;
            for (int m = 0; m < L.n; ++m) {
                a.ext[m] = p.ext[L.idx[m]];
                a.stride[m] = L.stride[m];
                total *= a.ext[m];
                span += (a.ext[m] - 1) * a.stride[m];
            }
            a.n = span == total ? 0 : L.n;
            a.total = total;
            a.src = (const float *)(o == 0 ? A : B);
            a.out = mx + o;
            const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8));
            absmax_kernel<<<(unsigned)grid, 256, 0, st>>>(a);
        }
        e4m3_scale_kernel<<<1, 32, 0, st>>>(mx, scale);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
        d.qscale = scale;
    }
    if (pk == 3) {
        // both inputs' stage images (128-row tiles of A, bn-row tiles of B,
        // 32-position K stages), A's first, then B's on a 256-byte boundary;
        // the GETT copies each stage's two images with 1-D bulk copies.
        // Pairs: B in bn/2-row tiles, both inputs in an even number of row
        // tiles (two per pair tile; rows past the extent are zeros)
        const int64_t nktp = (d.K + kBK - 1) / kBK;
        const int brows = pair ? bn / 2 : bn;
        const int64_t stA = (int64_t)kBM * kBK * image_bytes(p.dtype), stB = (int64_t)brows * kBK * image_bytes(p.dtype);
        const int64_t rtA = pair ? 2 * ((d.M + 2 * kBM - 1) / (2 * kBM)) : (d.M + kBM - 1) / kBM;
        const int64_t rtB = pair ? 2 * ((d.N + bn - 1) / bn) : (d.N + bn - 1) / bn;
        const int64_t offB = (rtA * nktp * stA + 255) / 256 * 256;
        // offB + rtB * nktp * stB <= pk_bound (rows round up by less than
        // 128 and bn <= 256, K by less than 32)
        s = ensure_device_resources(p, (size_t)pk_bound);
        if (s != TC_SUCCESS) return s;
        d.pk = 3;
        d.pk_base = (const char *)p.workspace;
        d.pk_tile_bytes = nktp * stA;
        d.pkb_base = (const char *)p.workspace + offB;
        d.pkb_tile_bytes = nktp * stB;
        for (int o = 0; o < 2; ++o) {
            const int rows = o == 0 ? kBM : brows;
            const int64_t rt = o == 0 ? rtA : rtB;
            const int64_t bytes = rt * nktp * (o == 0 ? stA : stB);
            const int64_t chunks =
                bytes / 16 / (p.dtype == TC_TF32X3 ? 2 : (p.dtype == TC_BF16X3 ? 3 : 1));  // 16-byte rows of slice 0
            const unsigned grid = (unsigned)std::min<int64_t>((chunks + 127) / 128, 152 * 16);
            char *out = (char *)p.workspace + (o == 0 ? 0 : offB);
            if (p.dtype == TC_BF16 || p.dtype == TC_F16) pack16_kernel<<<grid, 128, 0, st>>>(d, o, rows, kBK, rt, out);
            else if (p.dtype == TC_E4M3) pack_kernel<GK_E4M3><<<grid, 128, 0, st>>>(d, o, rows, kBK, rt, out);
            else if (p.dtype == TC_TF32) pack_kernel<GK_TF32><<<grid, 128, 0, st>>>(d, o, rows, kBK, rt, out);
            else if (p.dtype == TC_TF32X3) pack_kernel<GK_TF32X3><<<grid, 128, 0, st>>>(d, o, rows, kBK, rt, out);
            else pack_kernel<GK_BF16X3><<<grid, 128, 0, st>>>(d, o, rows, kBK, rt, out);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    } else if (pk) {
        // the smaller input's stage images, for the stage depth the launch
        // uses; pairs read them as two images per pair tile (an even count)
        const int bkp = tma ? kBKT : kBK;
        const int rows = pk == 1 ? kBM : (pair ? bn / 2 : bn);
        const int64_t R = pk == 1 ? d.M : d.N;
        const int64_t nktp = (d.K + bkp - 1) / bkp;
        const int64_t stage_bytes = (int64_t)rows * bkp * image_bytes(p.dtype);
        const int64_t rtiles = pair ? 2 * ((R + 2 * rows - 1) / (2 * rows)) : (R + rows - 1) / rows;
        const int64_t bytes = rtiles * nktp * stage_bytes;
        // bytes <= pk_bound: rows round up by less than 256, K by less than 32
        s = ensure_device_resources(p, (size_t)pk_bound);
        if (s != TC_SUCCESS) return s;
        d.pk = pk;
        d.pk_base = (const char *)p.workspace;
        d.pk_tile_bytes = nktp * stage_bytes;
        const int64_t chunks = bytes / 16 / (p.dtype == TC_TF32 ? 1 : (p.dtype == TC_TF32X3 ? 2 : 3));  // one per 16-byte row of slice 0
        const unsigned grid = (unsigned)std::min<int64_t>((chunks + 127) / 128, 152 * 16);
        if (p.dtype == TC_TF32)
            pack_kernel<GK_TF32><<<grid, 128, 0, st>>>(d, pk - 1, rows, bkp, rtiles, (char *)p.workspace);
        else if (p.dtype == TC_TF32X3)
            pack_kernel<GK_TF32X3><<<grid, 128, 0, st>>>(d, pk - 1, rows, bkp, rtiles, (char *)p.workspace);
        else
            pack_kernel<GK_BF16X3><<<grid, 128, 0, st>>>(d, pk - 1, rows, bkp, rtiles, (char *)p.workspace);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    }
    if (p.dtype == TC_E4M3) return launch_kind<GK_E4M3>(d, bn, false, false, false, tmA, tmB, st);
    switch (p.dtype) {
    case TC_BF16X3: return launch_kind<GK_BF16X3>(d, bn, tma, comp, pair, tmA, tmB, st);
    case TC_BF16: return launch_kind<GK_BF16>(d, bn, tma, comp, false, tmA, tmB, st);
    case TC_F16: return launch_kind<GK_F16>(d, bn, tma, comp, false, tmA, tmB, st);
    case TC_TF32: return launch_kind<GK_TF32>(d, bn, tma, comp, pair, tmA, tmB, st);
    case TC_TF32X3: return launch_kind<GK_TF32X3>(d, bn, tma, comp, false, tmA, tmB, st);
    default: return fail(TC_ERROR_UNSUPPORTED_DTYPE, "dtype has no tensor-core GETT");
    }
}

// ------------------------------------------------------------ gemm nests
// One phase of a gemm loop nest at a tensor dtype: the GETT kernel on its
// global-load path, M and N one mode each, the nest's concurrent loops as
// batch modes, its in-task contracted loops and kernel index as K (nest
// order).  Split-BF16 keeps the GETT's accuracy settings (split
// accumulators past K = 64, compensation past the chunk).
tc_status gett_launch_nest(Plan &p, const NestGemm &g, double frac, void *stream) {
    GettDesc d;
    std::memset(&d, 0, sizeof(d));
    d.nm = d.nn = 1;
    d.m_ext[0] = g.m.ext;
    d.m_sA[0] = g.m.sA;
    d.m_sC[0] = g.m.sC;
    d.n_ext[0] = g.n.ext;
    d.n_sB[0] = g.n.sB;
    d.n_sC[0] = g.n.sC;
    d.n_chain = 1;
    d.M = g.m.ext;
    d.N = g.n.ext;
    d.nk = g.nk;
    d.K = 1;
    for (int m = 0; m < g.nk; ++m) {
        d.k_ext[m] = g.k[m].ext;
        d.k_sA[m] = g.k[m].sA;
        d.k_sB[m] = g.k[m].sB;
        d.K *= g.k[m].ext;
    }
    d.nb = g.nt;
    for (int m = 0; m < g.nt; ++m) {
        d.b_ext[m] = g.t[m].ext;
        d.b_sA[m] = g.t[m].sA;
        d.b_sB[m] = g.t[m].sB;
        d.b_sC[m] = g.t[m].sC;
    }
    const int in_bytes = (p.dtype == TC_BF16 || p.dtype == TC_F16) ? 2 : 4;
    const int vec = 16 / in_bytes, chunk = (p.dtype == TC_TF32 || p.dtype == TC_TF32X3) ? 4 : 8;
    int bn = d.N >= 256 ? 256 : 128;
    int64_t comp_k = 0;
    if (p.dtype == TC_BF16X3 || p.dtype == TC_TF32X3) comp_k = p.comp_chunk < 0 ? kCompChunkK : p.comp_chunk;
    const bool comp = comp_k > 0 && d.K > comp_k;
    if (comp) {
        bn = 128;
        d.chunk_stages = (int)(comp_k / kBK);
    }
    auto pick = [&](const void *base, int rows, int nrow, const int64_t *rext, const int64_t *rs,
                    const int64_t *ks) {
        if (vec_ok(base, vec, nrow, rs, d.nk, d.k_ext, ks)) return 2;
        int64_t s0 = sectors_for(0, rows, chunk, in_bytes, nrow, rext, rs, d.nk, d.k_ext, ks);
        int64_t s1 = sectors_for(1, rows, chunk, in_bytes, nrow, rext, rs, d.nk, d.k_ext, ks);
        return s1 < s0 ? 1 : 0;
    };
    d.a_map = pick(g.A, kBM, d.nm, d.m_ext, d.m_sA, d.k_sA);
    d.b_map = pick(g.B, bn, d.nn, d.n_ext, d.n_sB, d.k_sB);
    d.A = g.A;
    d.B = g.B;
    d.C = (float *)g.C;
    d.alpha = g.alpha;
    d.beta = g.beta;
    d.init = g.init;
    d.nprod = p.split_products;
    d.status = p.dev_status;
    d.tiles_m = (d.M + kBM - 1) / kBM;
    d.tile_frac = frac;
    const bool want_split = p.gett_split > 0 || (p.gett_split < 0 && d.K >= 65);
    d.split = ((p.dtype == TC_BF16X3 || p.dtype == TC_TF32X3) && !comp && want_split) ? 1 : 0;
    CUtensorMap none;
    std::memset(&none, 0, sizeof(none));
    cudaStream_t st = (cudaStream_t)stream;
    switch (p.dtype) {
    case TC_BF16X3: return launch_kind<GK_BF16X3>(d, bn, false, comp, false, none, none, st);
    case TC_BF16: return launch_kind<GK_BF16>(d, bn, false, false, false, none, none, st);
    case TC_F16: return launch_kind<GK_F16>(d, bn, false, false, false, none, none, st);
    case TC_TF32: return launch_kind<GK_TF32>(d, bn, false, false, false, none, none, st);
    case TC_TF32X3: return launch_kind<GK_TF32X3>(d, bn, false, comp, false, none, none, st);
    default: return fail(TC_ERROR_UNSUPPORTED_DTYPE, "dtype has no tensor-core gemm");
    }
}

// ------------------------------------------------------------ batched form
size_t gett_desc_bytes() { return sizeof(GettDesc); }

void gett_fill_batch_desc(const BatchProblem &P, int bn, void *out) {
    GettDesc d;
    std::memset(&d, 0, sizeof(d));
    d.nm = d.nn = d.nk = 1;
    d.M = P.M;
    d.N = P.N;
    d.K = P.K;
    d.m_ext[0] = P.M;
    d.m_sA[0] = P.sAm;
    d.m_sC[0] = P.sCm;
    d.n_ext[0] = P.N;
    d.n_sB[0] = P.sBn;
    d.n_sC[0] = P.sCn;
    d.n_chain = 1;
    d.k_ext[0] = P.K;
    d.k_sA[0] = P.sAk;
    d.k_sB[0] = P.sBk;
    d.A = P.A;
    d.B = P.B;
    d.C = (float *)P.C;
    d.tiles_m = P.tiles_m;
    d.tiles_n = (P.N + bn - 1) / bn;
    d.tile0 = P.tile0;
    auto pick = [&](const void *base, int rows, const int64_t *rext, const int64_t *rs, const int64_t *ks) {
        if (vec_ok(base, 4, 1, rs, 1, d.k_ext, ks)) return 2;
        int64_t s0 = sectors_for(0, rows, 8, 4, 1, rext, rs, 1, d.k_ext, ks);
        int64_t s1 = sectors_for(1, rows, 8, 4, 1, rext, rs, 1, d.k_ext, ks);
        return s1 < s0 ? 1 : 0;
    };
    d.a_map = pick(P.A, kBM, d.m_ext, d.m_sA, d.k_sA);
    d.b_map = pick(P.B, bn, d.n_ext, d.n_sB, d.k_sB);
    std::memcpy(out, &d, sizeof(d));
}

int64_t gett_fill_plan_desc(const Plan &p, int bn, const void *A, const void *B, void *C, int64_t tile0, void *out) {
    GettDesc d;
    std::memset(&d, 0, sizeof(d));
    if (describe_modes(p, 0, d) != TC_SUCCESS) return -1;
    const int in_bytes = (p.dtype == TC_BF16 || p.dtype == TC_F16) ? 2 : 4;
    const int vec = 16 / in_bytes, chunk = (p.dtype == TC_TF32 || p.dtype == TC_TF32X3) ? 4 : 8;
    auto pick = [&](const void *base, int rows, int nrow, const int64_t *rext, const int64_t *rs,
                    const int64_t *ks) {
        if (vec_ok(base, vec, nrow, rs, d.nk, d.k_ext, ks)) return 2;
        int64_t s0 = sectors_for(0, rows, chunk, in_bytes, nrow, rext, rs, d.nk, d.k_ext, ks);
        int64_t s1 = sectors_for(1, rows, chunk, in_bytes, nrow, rext, rs, d.nk, d.k_ext, ks);
        return s1 < s0 ? 1 : 0;
    };
    d.a_map = pick(A, kBM, d.nm, d.m_ext, d.m_sA, d.k_sA);
    d.b_map = pick(B, bn, d.nn, d.n_ext, d.n_sB, d.k_sB);
    d.A = A;
    d.B = B;
    d.C = (float *)C;
    d.tiles_m = (d.M + kBM - 1) / kBM;
    d.tiles_n = (d.N + bn - 1) / bn;
    d.tile0 = tile0;
    std::memcpy(out, &d, sizeof(d));
    return d.tiles_m * d.tiles_n * batch_count(d);
}

tc_status gett_launch_batch(const void *ddescs, const int32_t *dtile_prob, int64_t t_begin, int64_t t_end, int bn,
                            float alpha, float beta, int nprod, int *dstatus, int one_stage, int split,
                            void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    GettDesc d;
    std::memset(&d, 0, sizeof(d));
    d.probs = (const GettDesc *)ddescs;
    d.tile_prob = dtile_prob;
    d.tile_begin = t_begin;
    d.num_tiles = t_end;
    d.alpha = alpha;
    d.beta = beta;
    d.init = beta == 0.0f ? 2 : 1;
    d.nprod = nprod;
    d.status = dstatus;
    d.tile_frac = 1.0;
    d.one_stage = one_stage;
    d.split = split;
    CUtensorMap none;
    std::memset(&none, 0, sizeof(none));
    if (bn == 128) return launch_gett<GK_BF16X3, 128, 4, kBK, 0, false, true>(d, none, none, st);
    return launch_gett<GK_BF16X3, 256, 2, kBK, 0, false, true>(d, none, none, st);
}

// Bounded-wait self-test: thread 0 waits on an mbarrier with the wait every
// kernel here uses; with `signal` a thread of another warp arrives first.
__device__ int g_selftest_status;

__global__ void bounded_wait_selftest_kernel(unsigned long long limit_ns, int signal) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 32 && signal) mbar_arrive(&bar);
    if (threadIdx.x == 0) g_selftest_status = mbar_wait(&bar, 0, limit_ns) ? (int)TC_SUCCESS : (int)TC_ERROR_TIMEOUT;
}

}  // namespace tc

extern "C" tc_status tc_selftest_bounded_wait(int64_t limit_ns, int32_t signal, void *stream) {
    using namespace tc;
    if (limit_ns <= 0 || limit_ns > 10000000000LL)
        return fail(TC_ERROR_INVALID_ARGUMENT, "limit_ns must be in (0, 1e10]");
    cudaStream_t st = (cudaStream_t)stream;
    const int init = -1;
    cudaError_t e = cudaMemcpyToSymbolAsync(g_selftest_status, &init, sizeof(int), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        bounded_wait_selftest_kernel<<<1, 64, 0, st>>>((unsigned long long)limit_ns, signal != 0);
        e = cudaGetLastError();
    }
    int out = -1;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(&out, g_selftest_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    if (out == (int)TC_ERROR_TIMEOUT) return fail(TC_ERROR_TIMEOUT, "bounded wait ran out (self-test)");
    return out == (int)TC_SUCCESS ? TC_SUCCESS : fail(TC_ERROR_CUDA, "self-test kernel did not report");
}
