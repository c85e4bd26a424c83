// Split-BF16 stream kernel of the batched form (no paper counterpart): many
// small contractions C[m + n*M] = sum_k A[m + k*M] B[k + n*K] (A, B and C
// dense with m, k and m fastest: "abc=ai,ibc"), K <= 32 and a multiple of
// 4, M <= 128.  Such a batch is bound by HBM: B is read once, C written once.
//
// The tile is 128 columns n of one problem with all of its M rows, computed
// as one MMA per slice product with the columns on the 128 tensor-memory
// lanes: D[n, m] = sum_k B[k, n] A[m, k] (MMA M = 128, N = M rounded up to
// 16, K = 16 or 32), so that no row of the MMA is padding except past N.
// The persistent kernel (one CTA per SM) is warp-specialised:
//
//   producer warp 0      fetches the problem records of 32 tiles at a time
//                        (one per lane, so their latency is paid once per 32
//                        tiles) into a ring of tile records the other roles
//                        read from shared memory; then one 1-D bulk copy of the tile's B run (128 x K
//                        contiguous FP32) and one of the problem's A (M x K)
//                        into a byte ring that packs tiles by their actual
//                        size (about nine in flight: the copies take a few
//                        microseconds to land), counted in bytes on an
//                        mbarrier per tile;
//   converter warps 2-5  split each FP32 value into three BF16 slices
//                        x = h0 + h1 + h2 and store both operands in the
//                        no-swizzle K-major core-matrix layout (zeros past K);
//   MMA warp 1           one thread issues the six slice products
//                        (0,0) (0,1) (1,0) (0,2) (1,1) (2,0) per 16-K step
//                        into one of four tensor-memory accumulators;
//   epilogue warps 6-13  two groups of four taking alternate tiles (the
//                        epilogue is the slowest role: one group left the MMA
//                        waiting on accumulators): tcgen05.ld 32 columns at a
//                        time, transpose them through a per-warp buffer and
//                        store each tile row's contiguous run of C (m
//                        fastest) with whole-warp coalesced stores, alpha and
//                        beta applied.
//
// Every mbarrier wait is bounded; on expiry the kernel records
// TC_ERROR_TIMEOUT in the status word, stops, waits for its own copies and
// MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "tc_internal.h"
#include "tc_tcgen05.cuh"

namespace tc {

namespace {

using namespace dev;

constexpr int kRows = 128;                      // tile columns n = MMA rows = TMEM lanes
constexpr int kMaxM = 128;                      // problem rows m (MMA N <= 128)
constexpr int kMaxK = 32;
constexpr int kRawSlots = 12;                   // tiles in the raw ring at most
constexpr int kRawBytes = 94 * 1024;            // raw FP32 ring: each tile's B run and A, packed
constexpr int kRecs = 32;                       // tile records in shared memory (the producer's lead)
constexpr int kConvSlots = 2;                   // converted operand ring
constexpr int kAccs = 4;                        // TMEM accumulators of kMaxM columns
constexpr int kMaxRawTile = kRows * kMaxK * 4 + kMaxM * kMaxK * 4;  // B run + A, at most
constexpr int kOpA = 3 * kRows * kMaxK * 2;     // three slices of the 128 x Kpad B tile
constexpr int kOpB = 3 * kMaxM * kMaxK * 2;     // three slices of the Mpad x Kpad A
constexpr int kConvSlot = kOpA + kOpB;
constexpr int kStgFloats = 32 * 33;             // per epilogue warp: 32 x 32 transpose, pitch 33
constexpr int kWProducer = 0, kWMma = 1, kWConv = 2, kConvWarps = 4, kWEpi = 6;
constexpr int kEpiGroups = 2;                   // epilogue groups of four warps, taking alternate tiles
constexpr int kEpiWarps = 4 * kEpiGroups;
constexpr int kStreamThreads = (kWEpi + kEpiWarps) * 32;
constexpr int kStreamSmem = kRawBytes + kConvSlots * kConvSlot + kEpiWarps * kStgFloats * 4 + 128;
static_assert(kMaxRawTile <= kRawBytes, "a tile fits the raw ring");
static_assert(kStreamSmem <= 232448, "shared memory budget");

struct StreamArgs {
    const BatchProblem *probs;
    const int32_t *tile_prob;
    int64_t t_begin, t_end;
    float alpha, beta;
    int init;  // 2: C = alpha*acc; 1: C = alpha*acc + beta*C
    int nprod;
    int *status;
};

struct STile {
    const float *A;
    const float *B;
    float *C;
    int M, K, nvalid;
    int64_t n0;
};

__device__ __forceinline__ STile stream_tile(const StreamArgs &a, int64_t t) {
    const BatchProblem *__restrict__ P = a.probs + a.tile_prob[t];
    STile s;
    s.n0 = (t - P->tile0) * kRows;
    s.M = (int)P->M;
    s.K = (int)P->K;
    s.nvalid = (int)min((int64_t)kRows, P->N - s.n0);
    s.A = (const float *)P->A;
    s.B = (const float *)P->B;
    s.C = (float *)P->C;
    return s;
}

// core-matrix byte offset of (row, 8-element K chunk kc) in a K-major
// operand of `rows` rows (K chunks outermost: lbo = rows * 16, sbo = 128)
__device__ __forceinline__ int cm_off(int row, int kc, int rows) { return (kc * (rows / 8) + row / 8) * 128 + (row % 8) * 16; }

__device__ __forceinline__ void split8_store(const float (&x)[8], char *dst, int slice) {
    uint32_t w0[4], w1[4], w2[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) split3x2(x[e], x[e + 1], w0[e / 2], w1[e / 2], w2[e / 2]);
    *(uint4 *)dst = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    *(uint4 *)(dst + slice) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *(uint4 *)(dst + 2 * slice) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
}

__global__ void __launch_bounds__(kStreamThreads, 1) stream_kernel(const StreamArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    char *raw = (char *)smem;
    char *conv = raw + kRawBytes;
    float *stg_all = (float *)(conv + kConvSlots * kConvSlot);
    __shared__ __align__(8) uint64_t raw_full[kRawSlots], raw_empty[kRawSlots];
    __shared__ int raw_off[kRawSlots];  // byte offset of each raw tile in the ring
    __shared__ STile recs[kRecs];       // tile i's record at i % kRecs
    __shared__ __align__(8) uint64_t rec_full[kRecs], rec_empty[kRecs];
    __shared__ __align__(8) uint64_t conv_full[kConvSlots], conv_empty[kConvSlots];
    __shared__ __align__(8) uint64_t acc_full[kAccs], acc_empty[kAccs], drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kRawSlots; ++i) mbar_init(&raw_full[i], 1), mbar_init(&raw_empty[i], kConvWarps);
        for (int i = 0; i < kConvSlots; ++i) mbar_init(&conv_full[i], kConvWarps), mbar_init(&conv_empty[i], 1);
        for (int i = 0; i < kAccs; ++i) mbar_init(&acc_full[i], 1), mbar_init(&acc_empty[i], 4);
        for (int i = 0; i < kRecs; ++i) mbar_init(&rec_full[i], 1), mbar_init(&rec_empty[i], 4);
        mbar_init(&drain, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kWMma) tmem_alloc(&tmem_slot, kAccs * kMaxM);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    auto give_up = [&]() {
        abort_flag = 1;
        atomicExch(a.status, (int)TC_ERROR_TIMEOUT);
    };
    const int64_t first = a.t_begin + blockIdx.x, step = gridDim.x;

    if (warp == kWProducer) {
        // ------------------------------------------------------------ producer
        // byte ring: tiles take [pos, pos + size) in order, none wrapping the
        // end; released in order by the converters (lane 0 keeps the books)
        int64_t head = 0, tail = 0, oldest = 0, i = 0;
        int64_t ends[kRawSlots];  // ring end of each tile in flight
        bool stop = false;
        for (int64_t base = 0; !stop; base += 32) {
            const int64_t tl = first + (base + lane) * step;  // lane l: tile base + l
            const STile mine = tl < a.t_end ? stream_tile(a, tl) : STile{};
            const int64_t left = (a.t_end - first + step - 1) / step - base;  // tiles of this CTA left
            if (left <= 0) break;
            const int nb = left < 32 ? (int)left : 32;
            for (int jj = 0; jj < nb; ++jj, ++i) {
                STile s;
                s.A = (const float *)__shfl_sync(0xffffffffu, (unsigned long long)mine.A, jj);
                s.B = (const float *)__shfl_sync(0xffffffffu, (unsigned long long)mine.B, jj);
                s.C = (float *)__shfl_sync(0xffffffffu, (unsigned long long)mine.C, jj);
                s.n0 = __shfl_sync(0xffffffffu, mine.n0, jj);
                s.M = __shfl_sync(0xffffffffu, mine.M, jj);
                s.K = __shfl_sync(0xffffffffu, mine.K, jj);
                s.nvalid = __shfl_sync(0xffffffffu, mine.nvalid, jj);
                if (lane == 0) {
                    const uint32_t bytesB = (uint32_t)(s.nvalid * s.K * 4), bytesA = (uint32_t)(s.M * s.K * 4);
                    const int64_t offA = (bytesB + 127) & ~127, size = offA + ((bytesA + 127) & ~127);
                    int64_t pos = head % kRawBytes;
                    if (pos + size > kRawBytes) {  // skip the ring's end
                        head += kRawBytes - pos;
                        pos = 0;
                    }
                    while (!stop && (head + size - tail > kRawBytes || i - oldest >= kRawSlots)) {
                        const int o = (int)(oldest % kRawSlots);
                        if (abort_flag || !mbar_wait(&raw_empty[o], (uint32_t)((oldest / kRawSlots) & 1))) stop = true;
                        else tail = ends[o], ++oldest;
                    }
                    // the record slot: its previous tile's epilogue has read it
                    const int q = (int)(i % kRecs);
                    if (!stop && i >= kRecs && !mbar_wait(&rec_empty[q], (uint32_t)(((i / kRecs) - 1) & 1)))
                        stop = true;
                    if (stop || abort_flag) {
                        stop = true;
                        give_up();
                    } else {
                        recs[q] = s;
                        mbar_arrive(&rec_full[q]);  // releases recs[q] to the epilogue
                        const int r = (int)(i % kRawSlots);
                        raw_off[r] = (int)pos;
                        ends[r] = head + size;
                        head += size;
                        mbar_arrive_expect_tx(&raw_full[r], bytesB + bytesA);  // releases raw_off[r], recs[q]
                        bulk_load(raw + pos, s.B + s.n0 * s.K, bytesB, &raw_full[r]);
                        bulk_load(raw + pos + offA, s.A, bytesA, &raw_full[r]);
                    }
                }
                stop = __shfl_sync(0xffffffffu, stop, 0);
                if (stop) break;
            }
        }
        // nothing may still be copying into shared memory at exit
        if (lane == 0)
            for (int64_t jj = oldest; jj < i; ++jj) mbar_wait(&raw_full[jj % kRawSlots], (uint32_t)((jj / kRawSlots) & 1));
    } else if (warp >= kWConv && warp < kWConv + kConvWarps) {
        // ----------------------------------------------------------- converters
        const int ct = threadIdx.x - kWConv * 32;  // 0..127: tile row n, and row m of A
        int64_t i = 0;
        for (int64_t t = first; t < a.t_end; t += step, ++i) {
            const int r = (int)(i % kRawSlots), c = (int)(i % kConvSlots);
            bool ok = !abort_flag && mbar_wait(&raw_full[r], (uint32_t)((i / kRawSlots) & 1));
            if (ok && i >= kConvSlots) ok = mbar_wait(&conv_empty[c], (uint32_t)(((i / kConvSlots) - 1) & 1));
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) give_up();
                break;
            }
            const STile s = recs[i % kRecs];  // written before raw_full[r] was armed
            const int K = s.K, M = s.M, Kp = K <= 16 ? 16 : 32, Mp = (M + 15) & ~15;
            const float *rawB = (const float *)(raw + raw_off[r]);
            const float *rawA = (const float *)(raw + raw_off[r] + ((s.nvalid * K * 4 + 127) & ~127));
            char *opA = conv + c * kConvSlot, *opB = opA + kOpA;
            // B tile -> the MMA's A operand: row n = ct (rows past nvalid keep
            // whatever they held: they only reach accumulator rows never stored)
            if (ct < s.nvalid) {
                const int sliceA = kRows * Kp * 2;
#pragma unroll
                for (int kc = 0; kc < kMaxK / 8; ++kc) {
                    if (kc >= Kp / 8) break;
                    float x[8];
                    const int k0 = kc * 8;
                    if (k0 + 8 <= K) {
                        const float4 u = *(const float4 *)(rawB + ct * K + k0), v = *(const float4 *)(rawB + ct * K + k0 + 4);
                        x[0] = u.x, x[1] = u.y, x[2] = u.z, x[3] = u.w, x[4] = v.x, x[5] = v.y, x[6] = v.z, x[7] = v.w;
                    } else if (k0 + 4 <= K) {
                        const float4 u = *(const float4 *)(rawB + ct * K + k0);
                        x[0] = u.x, x[1] = u.y, x[2] = u.z, x[3] = u.w, x[4] = x[5] = x[6] = x[7] = 0.0f;
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) x[e] = 0.0f;
                    }
                    split8_store(x, opA + cm_off(ct, kc, kRows), sliceA);
                }
            }
            // A -> the MMA's B operand: row m = ct, zeros past M and past K
            if (ct < Mp) {
                const int sliceB = Mp * Kp * 2;
#pragma unroll
                for (int kc = 0; kc < kMaxK / 8; ++kc) {
                    if (kc >= Kp / 8) break;
                    float x[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int k = kc * 8 + e;
                        x[e] = (ct < M && k < K) ? rawA[ct + k * M] : 0.0f;
                    }
                    split8_store(x, opB + cm_off(ct, kc, Mp), sliceB);
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&raw_empty[r]);
                mbar_arrive(&conv_full[c]);
            }
        }
    } else if (warp == kWMma) {
        // ------------------------------------------------------------------ MMA
        if (lane == 0) {
            // slice pairs in product order (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
            constexpr uint32_t kPa = 0x210100u, kPb = 0x012010u;
            bool issued = false;
            int64_t i = 0;
            for (int64_t t = first; t < a.t_end; t += step, ++i) {
                const int c = (int)(i % kConvSlots), b = (int)(i % kAccs);
                bool ok = !abort_flag && mbar_wait(&conv_full[c], (uint32_t)((i / kConvSlots) & 1));
                if (ok && i >= kAccs) ok = mbar_wait(&acc_empty[b], (uint32_t)(((i / kAccs) - 1) & 1));
                if (!ok) {
                    give_up();
                    break;
                }
                tc_fence_after();
                const STile s = recs[i % kRecs];  // visible through the converters' arrival
                const int Kp = s.K <= 16 ? 16 : 32, Mp = (s.M + 15) & ~15;
                const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Mp >> 3) << 17) |
                                       ((uint32_t)(kRows >> 4) << 24);
                const uint32_t sa = smem_u32(conv + c * kConvSlot), sb = sa + kOpA;
                const uint32_t sliceA = kRows * Kp * 2, sliceB = Mp * Kp * 2;
                const uint32_t lboA = kRows * 16, lboB = Mp * 16;
                const uint32_t dt = tmem + (uint32_t)(b * kMaxM);
                // descriptors of slice 0, first K step; the others differ in
                // the address field only (address >> 4, below 2^14), moved by
                // adding (offset >> 4); the products unrolled, so the issuing
                // thread spends a few independent instructions per MMA
                const uint64_t ad0 = smem_desc(sa, lboA, 128), bd0 = smem_desc(sb, lboB, 128);
                auto issue = [&](auto np) {
                    constexpr int NP = decltype(np)::value;
                    for (int ks = 0; ks < Kp / 16; ++ks) {
#pragma unroll
                        for (int q = 0; q < NP; ++q) {
                            const uint32_t qa = (kPa >> (4 * q)) & 15u, qb = (kPb >> (4 * q)) & 15u;
                            const uint64_t ad = ad0 + (uint64_t)((qa * sliceA + ks * 2 * lboA) >> 4);
                            const uint64_t bd = bd0 + (uint64_t)((qb * sliceB + ks * 2 * lboB) >> 4);
                            mma_f16(dt, ad, bd, idesc, (ks == 0 && q == 0) ? 0u : 1u);
                        }
                    }
                };
                if (a.nprod == 6) issue(std::integral_constant<int, 6>{});
                else issue(std::integral_constant<int, 3>{});
                mma_commit(&conv_empty[c]);
                mma_commit(&acc_full[b]);
                issued = true;
            }
            if (issued) {  // every MMA issued is complete before the memory is freed
                mma_commit(&drain);
                mbar_wait(&drain, 0);
            }
        }
        __syncwarp();
    } else if (warp >= kWEpi) {
        // ------------------------------------------------------------- epilogue
        const int qd = warp % 4;  // this warp's TMEM lane quadrant = tile rows 32 qd ...
        const int grp = (warp - kWEpi) / 4;  // tiles grp, grp + kEpiGroups, ...
        float *stg = stg_all + (warp - kWEpi) * kStgFloats;
        int64_t i = grp;
        const int64_t t1 = first + grp * step, gstep = kEpiGroups * step;
        for (int64_t t = t1; t < a.t_end; t += gstep, i += kEpiGroups) {
            const int b = (int)(i % kAccs), q = (int)(i % kRecs);
            bool ok = !abort_flag && mbar_wait(&rec_full[q], (uint32_t)((i / kRecs) & 1));
            STile s{};
            if (ok) s = recs[q];
            ok = ok && mbar_wait(&acc_full[b], (uint32_t)((i / kAccs) & 1));
            // the tile's MMAs are done, so the converters and the MMA warp
            // have read the record too: its slot may take tile i + kRecs
            __syncwarp();
            if (lane == 0 && ok) mbar_arrive(&rec_empty[q]);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) give_up();
                break;
            }
            tc_fence_after();
            const int M = s.M, nbase = qd * 32;
            for (int c0 = 0; c0 < M; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * kMaxM + c0), v);
                if (c0 + 32 >= M) {  // the accumulator is free for the next tile
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acc_empty[b]);
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = __uint_as_float(v[j]);
                __syncwarp();
                // lane = column c0 + lane of every row: all 32 reads, then all
                // 32 stores (row rr: C[(n0 + nbase + rr) * M + c0 + lane])
                float x[32];
#pragma unroll
                for (int rr = 0; rr < 32; ++rr) x[rr] = a.alpha * stg[rr * 33 + lane];
                __syncwarp();  // the buffer is free for the next chunk
                const int mv = min(32, M - c0), rows = min(32, s.nvalid - nbase);
                if (lane < mv) {
                    float *Crow = s.C + (s.n0 + nbase) * M + c0 + lane;
                    if (a.init == 1) {
#pragma unroll
                        for (int rr = 0; rr < 32; ++rr)
                            if (rr < rows) x[rr] = fmaf(a.beta, Crow[(int64_t)rr * M], x[rr]);
                    }
#pragma unroll
                    for (int rr = 0; rr < 32; ++rr)
                        if (rr < rows) Crow[(int64_t)rr * M] = x[rr];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kWMma) {
        tc_fence_after();
        tmem_dealloc(tmem, kAccs * kMaxM);
    }
}

int g_stream_sms = 0;

}  // namespace

bool stream_eligible(const BatchProblem &P) {
    return P.sAm == 1 && P.sAk == P.M && P.sBk == 1 && P.sBn == P.K && P.sCm == 1 && P.sCn == P.M && P.K % 4 == 0 &&
           P.K <= kMaxK && P.M <= kMaxM && P.N >= 1 && ((uintptr_t)P.A & 15) == 0 && ((uintptr_t)P.B & 15) == 0 &&
           ((uintptr_t)P.C & 3) == 0;
}

int64_t stream_tiles(const BatchProblem &P) { return (P.N + kRows - 1) / kRows; }

tc_status stream_launch_batch(const BatchProblem *dprobs, const int32_t *dtile_prob, int64_t t_begin, int64_t t_end,
                              float alpha, float beta, int nprod, int *dstatus, void *stream) {
    if (t_end <= t_begin) return TC_SUCCESS;
    if (g_stream_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_stream_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_stream_sms <= 0) g_stream_sms = 1;
        cudaFuncSetAttribute(stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStreamSmem);
    }
    if (nprod != 3 && nprod != 6) return fail(TC_ERROR_INVALID_ARGUMENT, "stream kernel: 3 or 6 slice products");
    StreamArgs a;
    a.probs = dprobs;
    a.tile_prob = dtile_prob;
    a.t_begin = t_begin;
    a.t_end = t_end;
    a.alpha = alpha;
    a.beta = beta;
    a.init = beta == 0.0f ? 2 : 1;
    a.nprod = nprod;
    a.status = dstatus;
    const int64_t grid = std::min<int64_t>(t_end - t_begin, g_stream_sms);
    stream_kernel<<<(unsigned)grid, kStreamThreads, kStreamSmem, (cudaStream_t)stream>>>(a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TC_SUCCESS : fail(TC_ERROR_CUDA, cudaGetErrorString(e));
}

}  // namespace tc
