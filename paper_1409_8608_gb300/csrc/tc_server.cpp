// Serving loop with continuous batching (no paper counterpart; the
// project's serving addition).
//
// A worker thread owns the device side.  Requests (spec, extents, dtype,
// host inputs, optional host output) queue in arrival order; each keeps the
// plan its submission built (spec, index classes, layouts: no algorithm
// enumeration).  The worker
//   * admits the head of the queue when a slot is free and its operands
//     (A, B, C) fit in what is left of the device-memory budget -- a
//     first-fit arena carved out of one allocation made at creation -- and
//     otherwise counts an admission stall and waits (no reordering);
//   * files every admitted request under its batch class: FP64 or FP32 (the
//     SIMT GETT), split-BF16 with K <= 64, split-BF16 with 64 < K <= 256
//     (split accumulators), or solo (split-BF16 with longer K, compensated,
//     and the other tensor dtypes: one launch each);
//   * whenever one of its streams is free, turns the class whose oldest
//     request waited longest into ONE batched launch of all its admitted
//     requests (up to a problem and tile cap): their inputs copied in, one
//     descriptor per request and the flattened tile table uploaded from the
//     stream's pinned staging, one persistent kernel over every tile, the
//     results copied out, one completion event;
//   * polls the streams' events, frees the finished batch's memory and
//     slots, and admits more -- requests that arrive while batches run form
//     the next batches, and batches on different streams overlap.
// A request's arithmetic depends only on the request: its class, its K
// order and its tile shapes follow from its own spec, extents and dtype,
// never from the batch around it, so its result is the same alone and in
// any mix.  Latency is measured from submission to the moment the worker
// sees the completion of the request's batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tc_internal.h"

namespace tc {
namespace {

using Clock = std::chrono::steady_clock;

constexpr int kClasses = 4;              // batched classes (see above)
constexpr int kSolo = -1;
constexpr int kMaxBatchProblems = 256;
constexpr int64_t kMaxBatchTiles = int64_t(1) << 20;
constexpr int64_t kSplitMinK = 65;       // split accumulators past K = 64
constexpr int64_t kBatchMaxK = 256;      // longer split-BF16 K runs compensated, solo

struct Request {
    int64_t id = 0;
    std::unique_ptr<Plan> plan;  // spec, classes, layouts (GETT only)
    tc_dtype dtype = TC_F32;
    const void *hA = nullptr;
    const void *hB = nullptr;
    void *hC = nullptr;
    size_t bytesA = 0, bytesB = 0, bytesC = 0;
    double flops = 0;
    int cls = kSolo;
    int64_t K = 1;
    Clock::time_point t_submit;
    // device side
    size_t offset = 0, bytes = 0;
};

struct Result {
    bool done = false;
    tc_status status = TC_SUCCESS;
    double latency = 0;
    std::string message;  // error text of a failed request
};

// One stream's batch in flight and the stream's own staging buffers.
struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<std::unique_ptr<Request>> reqs;
    char *hdesc = nullptr, *ddesc = nullptr;        // descriptors (pinned host, device)
    int32_t *htile = nullptr, *dtile = nullptr;     // tile -> problem
    int *hstatus = nullptr, *dstatus = nullptr;     // bounded-wait status word
};

// First-fit allocator over one device allocation, blocks coalesced on free.
class Arena {
  public:
    void init(size_t size) {
        free_.clear();
        free_[0] = size;
        size_ = size;
    }
    bool alloc(size_t n, size_t *off) {
        n = (n + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, start = it->first + n;
            free_.erase(it);
            if (rest) free_[start] = rest;
            used_ += n;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = (n + 255) / 256 * 256;
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

size_t operand_bytes(const Plan &p, int o) {
    int64_t n = 1;
    for (int m = 0; m < p.op[o].n; ++m) n *= p.ext[p.op[o].idx[m]];
    return (size_t)n * (o == OP_C ? elem_bytes_c(p.dtype) : elem_bytes_ab(p.dtype));
}

}  // namespace

struct ServerImpl {
    int64_t budget = 0;
    int slots = 0;
    std::vector<Slot> streams;
    void *arena_base = nullptr;
    Arena arena;
    int device = 0;
    size_t desc_bytes = 0;  // one problem descriptor (the larger of the two kinds)
    void *ctrl_dev = nullptr, *ctrl_host = nullptr;  // every slot's staging, one allocation each

    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::unique_ptr<Request>> queue;
    std::unordered_map<int64_t, Result> results;
    std::condition_variable done_cv;
    int64_t next_id = 1;
    bool stop = false;
    std::thread worker;

    // worker-only state
    std::deque<std::unique_ptr<Request>> pending[kClasses + 1];  // [kClasses]: solo
    int admitted = 0;  // admitted and not finished (pending or on the device)
    const char *last_action = "start";  // the worker's last CUDA call, for diagnostics
    bool warned = false;

    // statistics (under mu)
    std::vector<double> latencies;
    double flops_served = 0;
    int64_t stalls = 0, completed = 0, failed = 0, peak_inflight = 0, batches = 0, max_batch = 0;
    Clock::time_point t_first, t_last;
    bool any = false;

    void finish(std::unique_ptr<Request> &r, tc_status st, const std::string &msg = "") {
        const double lat = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
        arena.release(r->offset, r->bytes);
        --admitted;
        std::lock_guard<std::mutex> g(mu);
        Result &res = results[r->id];
        res.done = true;
        res.status = st;
        res.latency = lat;
        if (st != TC_SUCCESS) res.message = msg.empty() ? std::string(tc_last_error()) : msg;
        if (st == TC_SUCCESS) {
            latencies.push_back(lat);
            flops_served += r->flops;
            ++completed;
        } else {
            ++failed;
        }
        t_last = Clock::now();
        done_cv.notify_all();
    }

    void operands(const Request &r, char **dA, char **dB, char **dC) {
        char *base = (char *)arena_base + r.offset;
        *dA = base;
        *dB = *dA + (r.bytesA + 255) / 256 * 256;
        *dC = *dB + (r.bytesB + 255) / 256 * 256;
    }

    // Inputs of one request in, on the slot's stream.
    tc_status copy_in(const Request &r, cudaStream_t st) {
        char *dA, *dB, *dC;
        operands(r, &dA, &dB, &dC);
        last_action = "cudaMemcpyAsync (inputs)";
        cudaError_t e = cudaMemcpyAsync(dA, r.hA, r.bytesA, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dB, r.hB, r.bytesB, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess)
            return fail(TC_ERROR_CUDA, std::string("copy of the inputs (arena offset ") + std::to_string(r.offset) +
                                           "): " + cudaGetErrorString(e));
        return TC_SUCCESS;
    }

    // The class whose oldest pending request arrived first.
    int next_class() {
        int best = -2;
        int64_t best_id = 0;
        for (int c = 0; c <= kClasses; ++c) {
            if (pending[c].empty()) continue;
            const int64_t id = pending[c].front()->id;
            if (best == -2 || id < best_id) {
                best = c;
                best_id = id;
            }
        }
        return best;
    }

    // Forms and launches one batch of class c on slot k (solo: one request).
    void launch(int c, int k) {
        cudaError_t stale = cudaGetLastError();  // not this batch's
        if (stale != cudaSuccess && !warned) {
            warned = true;
            std::fprintf(stderr, "tc_server: cleared a CUDA error left by '%s': %s\n", last_action,
                         cudaGetErrorString(stale));
        }
        Slot &S = streams[k];
        cudaStream_t st = S.stream;
        S.reqs.clear();
        tc_status s = TC_SUCCESS;
        std::string msg;
        if (c == kClasses) {  // solo: the plan's own GETT (compensated or other tensor dtypes)
            std::unique_ptr<Request> r = std::move(pending[c].front());
            pending[c].pop_front();
            s = copy_in(*r, st);
            char *dA, *dB, *dC;
            operands(*r, &dA, &dB, &dC);
            if (s == TC_SUCCESS) {
                Plan &p = *r->plan;
                p.device = device;
                p.dev_status = S.dstatus;  // the slot's status word: nothing to allocate
                p.gett_pack = 0;           // no workspace
                const double one = 1.0, zero = 0.0;
                const float onef = 1.0f, zerof = 0.0f;
                const bool f64 = r->dtype == TC_F64;
                last_action = "exec_gett (solo)";
                s = exec_gett(p, f64 ? (const void *)&one : (const void *)&onef, dA, dB,
                              f64 ? (const void *)&zero : (const void *)&zerof, dC, st);
                p.dev_status = nullptr;
                if (s != TC_SUCCESS) msg = std::string("execute: ") + tc_last_error();
            }
            S.reqs.push_back(std::move(r));
        } else {
            // one descriptor per request, the flattened tile list, one launch
            const bool simt = c < 2;
            int bn = 128;
            if (!simt) {
                const Plan &p0 = *pending[c].front()->plan;
                int64_t N = 1;
                for (int id : p0.freeB) N *= p0.ext[id];
                bn = N >= 256 ? 256 : 128;
            }
            // descriptors at the stride of the kernel's own descriptor type
            const size_t stride = simt ? simt_desc_bytes() : gett_desc_bytes();
            int64_t ntiles = 0;
            while (!pending[c].empty() && (int)S.reqs.size() < kMaxBatchProblems) {
                Request &r = *pending[c].front();
                char *dA, *dB, *dC;
                operands(r, &dA, &dB, &dC);
                char *hd = S.hdesc + S.reqs.size() * stride;
                const int64_t t = simt ? simt_fill_desc(*r.plan, dA, dB, dC, ntiles, hd)
                                       : gett_fill_plan_desc(*r.plan, bn, dA, dB, dC, ntiles, hd);
                if (t >= 0 && ntiles + t > kMaxBatchTiles && !S.reqs.empty()) break;  // the next batch's
                if (t < 0 || ntiles + t > kMaxBatchTiles) {
                    // a request no batch can hold: it fails alone, the batch goes on
                    std::unique_ptr<Request> bad = std::move(pending[c].front());
                    pending[c].pop_front();
                    finish(bad, fail(TC_ERROR_INVALID_ARGUMENT, t < 0 ? "request has too many contracted modes"
                                                                      : "request has more tiles than a batch holds"));
                    continue;
                }
                for (int64_t x = 0; x < t; ++x) S.htile[ntiles + x] = (int32_t)S.reqs.size();
                ntiles += t;
                s = copy_in(r, st);
                S.reqs.push_back(std::move(pending[c].front()));
                pending[c].pop_front();
                if (s != TC_SUCCESS) break;
            }
            if (s == TC_SUCCESS && !S.reqs.empty()) {
                last_action = "cudaMemcpyAsync (batch tables)";
                cudaError_t e = cudaMemcpyAsync(S.ddesc, S.hdesc, S.reqs.size() * stride,
                                                cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(S.dtile, S.htile, (size_t)ntiles * sizeof(int32_t), cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) s = fail(TC_ERROR_CUDA, cudaGetErrorString(e));
            }
            if (s == TC_SUCCESS && !S.reqs.empty()) {
                last_action = "batched launch";
                if (simt)
                    s = simt_launch_batch(c == 0 ? TC_F64 : TC_F32, S.ddesc, S.dtile, ntiles, st);
                else
                    s = gett_launch_batch(S.ddesc, S.dtile, 0, ntiles, bn, 1.0f, 0.0f, 6, S.dstatus, 0,
                                          c == 3 ? 1 : 0, st);
                if (s != TC_SUCCESS) msg = std::string("batched launch: ") + tc_last_error();
            }
        }
        // results out, the status word, the completion event
        for (auto &r : S.reqs) {
            if (s != TC_SUCCESS || !r->hC) continue;
            char *dA, *dB, *dC;
            operands(*r, &dA, &dB, &dC);
            last_action = "cudaMemcpyAsync (result)";
            cudaError_t e = cudaMemcpyAsync(r->hC, dC, r->bytesC, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) s = fail(TC_ERROR_CUDA, cudaGetErrorString(e));
        }
        if (s == TC_SUCCESS) {
            last_action = "status word / event";
            cudaError_t e = cudaMemcpyAsync(S.hstatus, S.dstatus, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaEventRecord(S.done, st);
            if (e != cudaSuccess) s = fail(TC_ERROR_CUDA, cudaGetErrorString(e));
        }
        if (s != TC_SUCCESS) {
            cudaStreamSynchronize(st);
            for (auto &r : S.reqs) finish(r, s, msg);
            S.reqs.clear();
            return;
        }
        S.busy = true;
        std::lock_guard<std::mutex> g(mu);
        ++batches;
        max_batch = std::max<int64_t>(max_batch, (int64_t)S.reqs.size());
    }

    void run() {
        cudaSetDevice(device);
        for (;;) {
            bool progressed = false;
            // completions: a batch is done when its event is
            for (Slot &S : streams) {
                if (!S.busy) continue;
                last_action = "cudaEventQuery";
                cudaError_t q = cudaEventQuery(S.done);
                if (q == cudaErrorNotReady) continue;
                tc_status st = TC_SUCCESS;
                std::string msg;
                if (q != cudaSuccess) {
                    st = TC_ERROR_CUDA;
                    msg = std::string("completion: ") + cudaGetErrorString(q);
                } else if (*S.hstatus != 0) {
                    st = TC_ERROR_TIMEOUT;
                    msg = "a bounded device wait gave up";
                    *S.hstatus = 0;
                    cudaMemsetAsync(S.dstatus, 0, sizeof(int), S.stream);
                }
                for (auto &r : S.reqs) finish(r, st, msg);
                S.reqs.clear();
                S.busy = false;
                progressed = true;
            }
            // admissions, in arrival order
            for (;;) {
                std::unique_ptr<Request> r;
                {
                    std::unique_lock<std::mutex> g(mu);
                    if (queue.empty() || admitted >= slots) break;
                    Request &h = *queue.front();
                    const size_t need = (h.bytesA + 255) / 256 * 256 + (h.bytesB + 255) / 256 * 256 +
                                        (h.bytesC + 255) / 256 * 256;
                    size_t off = 0;
                    if (!arena.alloc(need, &off)) {
                        ++stalls;  // waits for memory to come back
                        break;
                    }
                    r = std::move(queue.front());
                    queue.pop_front();
                    r->offset = off;
                    r->bytes = need;
                    ++admitted;
                    peak_inflight = std::max<int64_t>(peak_inflight, (int64_t)admitted);
                }
                const int c = r->cls == kSolo ? kClasses : r->cls;
                pending[c].push_back(std::move(r));
                progressed = true;
            }
            // launches: every free stream takes the next class's batch
            for (size_t k = 0; k < streams.size(); ++k) {
                if (streams[k].busy) continue;
                const int c = next_class();
                if (c < 0) break;
                launch(c, (int)k);
                progressed = true;
            }
            {
                std::unique_lock<std::mutex> g(mu);
                bool busy = false;
                for (Slot &S : streams) busy |= S.busy;
                bool waiting = next_class() >= 0;
                if (stop && queue.empty() && !busy && !waiting) return;
                if (!progressed) {
                    if (!busy && !waiting && queue.empty()) cv.wait_for(g, std::chrono::milliseconds(5));
                    else {
                        g.unlock();
                        std::this_thread::sleep_for(std::chrono::microseconds(20));
                    }
                }
            }
        }
    }
};

}  // namespace tc

using namespace tc;

struct tc_server_s {
    ServerImpl s;
};

extern "C" {

tc_status tc_server_create(tc_server *out, int64_t budget_bytes, int32_t slots, int32_t streams) {
    if (!out) return fail(TC_ERROR_INVALID_ARGUMENT, "out is NULL");
    *out = nullptr;
    if (budget_bytes < (1 << 20) || slots < 1 || streams < 1 || streams > 64)
        return fail(TC_ERROR_INVALID_ARGUMENT, "budget >= 1 MiB, slots >= 1, 1 <= streams <= 64");
    auto *h = new (std::nothrow) tc_server_s();
    if (!h) return fail(TC_ERROR_OUT_OF_MEMORY, "host allocation failed");
    ServerImpl &S = h->s;
    cudaGetDevice(&S.device);
    S.budget = budget_bytes;
    S.slots = slots;
    S.desc_bytes = std::max(simt_desc_bytes(), gett_desc_bytes());
    // per stream: descriptors, tile table, status word (256-byte aligned parts)
    const size_t dbytes = ((size_t)kMaxBatchProblems * S.desc_bytes + 255) / 256 * 256;
    const size_t tbytes = (size_t)kMaxBatchTiles * sizeof(int32_t);
    const size_t per = dbytes + tbytes + 256;
    cudaError_t e = cudaMalloc(&S.arena_base, (size_t)budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&S.ctrl_dev, per * streams);
    if (e == cudaSuccess) e = cudaHostAlloc(&S.ctrl_host, per * streams, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMemset(S.ctrl_dev, 0, per * streams);
    if (e != cudaSuccess) {
        if (S.arena_base) cudaFree(S.arena_base);
        if (S.ctrl_dev) cudaFree(S.ctrl_dev);
        if (S.ctrl_host) cudaFreeHost(S.ctrl_host);
        delete h;
        return fail(TC_ERROR_OUT_OF_MEMORY, cudaGetErrorString(e));
    }
    std::memset(S.ctrl_host, 0, per * streams);
    S.arena.init((size_t)budget_bytes);
    S.streams.resize(streams);
    for (int i = 0; i < streams; ++i) {
        Slot &k = S.streams[i];
        cudaStreamCreateWithFlags(&k.stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&k.done, cudaEventDisableTiming);
        char *hd = (char *)S.ctrl_host + per * i, *dd = (char *)S.ctrl_dev + per * i;
        k.hdesc = hd;
        k.ddesc = dd;
        k.htile = (int32_t *)(hd + dbytes);
        k.dtile = (int32_t *)(dd + dbytes);
        k.hstatus = (int *)(hd + dbytes + tbytes);
        k.dstatus = (int *)(dd + dbytes + tbytes);
    }
    S.worker = std::thread([&S] { S.run(); });
    *out = h;
    return TC_SUCCESS;
}

tc_status tc_server_submit(tc_server server, const char *spec, const int64_t *extents, tc_dtype dtype,
                           const void *A, const void *B, void *C, int64_t *request_id) {
    if (!server || !spec || !extents || !A || !B || !request_id)
        return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    if (dtype == TC_E4M3) return fail(TC_ERROR_UNSUPPORTED_DTYPE, "the serving loop does not run TC_E4M3");
    ServerImpl &S = server->s;
    // validate and size the request: spec, classes and layouts only (the
    // request runs the GETT; its plan has no other algorithm)
    auto r = std::make_unique<Request>();
    r->plan = std::make_unique<Plan>();
    tc_status s = build_plan(*r->plan, spec, extents, nullptr, dtype, false);
    if (s != TC_SUCCESS) return s;
    const Plan &p = *r->plan;
    r->dtype = dtype;
    r->hA = A;
    r->hB = B;
    r->hC = C;
    r->bytesA = operand_bytes(p, OP_A);
    r->bytesB = operand_bytes(p, OP_B);
    r->bytesC = operand_bytes(p, OP_C);
    double f = 2.0;
    for (int x = 0; x < p.nidx; ++x) f *= (double)p.ext[x];
    r->flops = f;
    for (int id : p.contracted) r->K *= p.ext[id];
    // batch class: the SIMT GETT (FP64, FP32), split-BF16 by K, else solo
    if (dtype == TC_F64) r->cls = 0;
    else if (dtype == TC_F32) r->cls = 1;
    else if (dtype == TC_BF16X3 && r->K <= kBatchMaxK) r->cls = r->K >= kSplitMinK ? 3 : 2;
    else r->cls = kSolo;
    const size_t need = (r->bytesA + 255) / 256 * 256 + (r->bytesB + 255) / 256 * 256 + (r->bytesC + 255) / 256 * 256;
    if ((int64_t)need > S.budget) return fail(TC_ERROR_ADMISSION, "request larger than the whole budget");
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> g(S.mu);
        if (S.stop) return fail(TC_ERROR_INVALID_ARGUMENT, "server is shutting down");
        r->id = S.next_id++;
        *request_id = r->id;
        S.results[r->id] = Result();
        if (!S.any) {
            S.t_first = r->t_submit;
            S.any = true;
        }
        S.queue.push_back(std::move(r));
    }
    S.cv.notify_one();
    return TC_SUCCESS;
}

tc_status tc_server_poll(tc_server server, int64_t request_id, int32_t *done, double *latency) {
    if (!server || !done) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    ServerImpl &S = server->s;
    std::lock_guard<std::mutex> g(S.mu);
    auto it = S.results.find(request_id);
    if (it == S.results.end()) return fail(TC_ERROR_INVALID_ARGUMENT, "unknown request id");
    *done = it->second.done ? 1 : 0;
    if (latency) *latency = it->second.latency;
    if (it->second.done && it->second.status != TC_SUCCESS) return fail(it->second.status, it->second.message);
    return TC_SUCCESS;
}

tc_status tc_server_wait(tc_server server, int64_t request_id, double timeout_s) {
    if (!server) return fail(TC_ERROR_INVALID_ARGUMENT, "server is NULL");
    ServerImpl &S = server->s;
    std::unique_lock<std::mutex> g(S.mu);
    auto it = S.results.find(request_id);
    if (it == S.results.end()) return fail(TC_ERROR_INVALID_ARGUMENT, "unknown request id");
    const bool ok = S.done_cv.wait_for(g, std::chrono::duration<double>(timeout_s),
                                       [&] { return S.results[request_id].done; });
    if (!ok) return fail(TC_ERROR_TIMEOUT, "request not finished within the timeout");
    const Result &res = S.results[request_id];
    if (res.status != TC_SUCCESS) return fail(res.status, res.message);
    return TC_SUCCESS;
}

tc_status tc_server_stats(tc_server server, tc_server_report *out) {
    if (!server || !out) return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    ServerImpl &S = server->s;
    std::lock_guard<std::mutex> g(S.mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = S.completed;
    out->failed = S.failed;
    out->admission_stalls = S.stalls;
    out->peak_inflight = S.peak_inflight;
    out->queued = (int64_t)S.queue.size();
    out->flops_served = S.flops_served;
    out->batches = S.batches;
    out->max_batch = S.max_batch;
    if (S.any && S.completed > 0)
        out->span_seconds = std::chrono::duration<double>(S.t_last - S.t_first).count();
    if (!S.latencies.empty()) {
        std::vector<double> l = S.latencies;
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) { return l[std::min(l.size() - 1, (size_t)(q * (l.size() - 1) + 0.5))]; };
        out->p50_seconds = pct(0.50);
        out->p99_seconds = pct(0.99);
        out->max_seconds = l.back();
    }
    return TC_SUCCESS;
}

tc_status tc_server_destroy(tc_server server) {
    if (!server) return TC_SUCCESS;
    ServerImpl &S = server->s;
    {
        std::lock_guard<std::mutex> g(S.mu);
        S.stop = true;
    }
    S.cv.notify_all();
    if (S.worker.joinable()) S.worker.join();  // drains the queue first
    for (Slot &k : S.streams) {
        cudaStreamDestroy(k.stream);
        cudaEventDestroy(k.done);
    }
    if (S.arena_base) cudaFree(S.arena_base);
    if (S.ctrl_dev) cudaFree(S.ctrl_dev);
    if (S.ctrl_host) cudaFreeHost(S.ctrl_host);
    delete server;
    return TC_SUCCESS;
}

}  // extern "C"
