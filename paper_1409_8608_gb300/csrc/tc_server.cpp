// Serving loop with continuous batching (no paper counterpart; the
// project's serving addition).
//
// A worker thread owns the device side.  Requests (spec, extents, dtype,
// host inputs, optional host output) queue in arrival order.  The worker
//   * admits the head of the queue when a slot is free and its operands
//     (A, B, C) fit in what is left of the device-memory budget -- a
//     first-fit arena carved out of one allocation made at creation -- and
//     otherwise counts an admission stall and waits (no reordering);
//   * runs each admitted request on one of its streams: inputs copied in,
//     the contraction with the plan cached for the request's key (spec,
//     extents, dtype: a request's arithmetic never depends on its
//     neighbours), the result copied out when the caller asked for it;
//   * polls the in-flight requests' events, frees their memory and slots as
//     they finish, and admits more -- requests that arrive while others run
//     join at once, and their kernels overlap on the device.
// Latency is measured from submission to the moment the worker sees the
// request's completion event.
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

struct Request {
    int64_t id = 0;
    std::string spec;
    std::vector<int64_t> extents;
    tc_dtype dtype = TC_F32;
    const void *hA = nullptr;
    const void *hB = nullptr;
    void *hC = nullptr;
    size_t bytesA = 0, bytesB = 0, bytesC = 0;
    double flops = 0;
    Clock::time_point t_submit;
    // device side
    size_t offset = 0, bytes = 0;
    int stream = 0;
    cudaEvent_t done_event = nullptr;
    tc_plan plan = nullptr;
};

struct Result {
    bool done = false;
    tc_status status = TC_SUCCESS;
    double latency = 0;
    std::string message;  // error text of a failed request
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
    std::vector<cudaStream_t> streams;
    void *arena_base = nullptr;
    Arena arena;
    int device = 0;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::unique_ptr<Request>> queue;
    std::unordered_map<int64_t, Result> results;
    std::condition_variable done_cv;
    int64_t next_id = 1;
    bool stop = false;
    std::thread worker;

    // worker-only state
    std::vector<std::unique_ptr<Request>> inflight;
    const char *last_action = "start";  // the worker's last CUDA call, for diagnostics
    bool warned = false;
    std::map<std::string, tc_plan> plans;
    int rr = 0;

    // statistics (under mu)
    std::vector<double> latencies;
    double flops_served = 0;
    int64_t stalls = 0, completed = 0, failed = 0, peak_inflight = 0;
    Clock::time_point t_first, t_last;
    bool any = false;

    std::string key(const Request &r) {
        std::string k = r.spec + "|" + std::to_string((int)r.dtype);
        for (int64_t e : r.extents) k += "," + std::to_string(e);
        return k;
    }

    void finish(std::unique_ptr<Request> &r, tc_status st, const std::string &msg = "") {
        const double lat = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
        arena.release(r->offset, r->bytes);
        last_action = "cudaEventDestroy";
        if (r->done_event) cudaEventDestroy(r->done_event);
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

    tc_status launch(Request &r) {
        // an error left by an earlier call on this thread must not be
        // attributed to this request's launches
        cudaError_t stale = cudaGetLastError();
        if (stale != cudaSuccess && !warned) {
            warned = true;
            std::fprintf(stderr, "tc_server: cleared a CUDA error left by '%s' before request %lld: %s\n",
                         last_action, (long long)r.id, cudaGetErrorString(stale));
        }
        cudaStream_t st = streams[r.stream];
        last_action = "cudaMemcpyAsync (inputs)";
        char *base = (char *)arena_base + r.offset;
        char *dA = base;
        char *dB = dA + (r.bytesA + 255) / 256 * 256;
        char *dC = dB + (r.bytesB + 255) / 256 * 256;
        cudaError_t e = cudaMemcpyAsync(dA, r.hA, r.bytesA, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess)
            return fail(TC_ERROR_CUDA, std::string("copy of A (") + std::to_string(r.bytesA) + " bytes at arena offset " +
                                           std::to_string(r.offset) + "): " + cudaGetErrorString(e));
        e = cudaMemcpyAsync(dB, r.hB, r.bytesB, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess)
            return fail(TC_ERROR_CUDA, std::string("copy of B (") + std::to_string(r.bytesB) + " bytes at arena offset " +
                                           std::to_string(r.offset) + "): " + cudaGetErrorString(e));
        const double one = 1.0, zero = 0.0;
        const float onef = 1.0f, zerof = 0.0f;
        const bool f64 = r.dtype == TC_F64;
        last_action = "tc_execute";
        tc_status s = tc_execute(r.plan, f64 ? (const void *)&one : (const void *)&onef, dA, dB,
                                 f64 ? (const void *)&zero : (const void *)&zerof, dC, st);
        if (s != TC_SUCCESS) return fail(s, std::string("execute: ") + tc_last_error());
        if (r.hC) {
            last_action = "cudaMemcpyAsync (result)";
            e = cudaMemcpyAsync(r.hC, dC, r.bytesC, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return fail(TC_ERROR_CUDA, cudaGetErrorString(e));
        }
        last_action = "cudaEventCreate/Record";
        e = cudaEventCreateWithFlags(&r.done_event, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(r.done_event, st);
        return e == cudaSuccess ? TC_SUCCESS : fail(TC_ERROR_CUDA, cudaGetErrorString(e));
    }

    void run() {
        cudaSetDevice(device);
        for (;;) {
            // completions
            for (size_t i = 0; i < inflight.size();) {
                last_action = "cudaEventQuery";
                cudaError_t q = cudaEventQuery(inflight[i]->done_event);
                if (q == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                finish(inflight[i], q == cudaSuccess ? TC_SUCCESS : TC_ERROR_CUDA,
                       q == cudaSuccess ? "" : std::string("completion: ") + cudaGetErrorString(q));
                inflight.erase(inflight.begin() + i);
            }
            // admissions, in arrival order
            std::unique_ptr<Request> r;
            {
                std::unique_lock<std::mutex> g(mu);
                if (stop && queue.empty() && inflight.empty()) return;
                if (queue.empty() || (int)inflight.size() >= slots) {
                    if (inflight.empty()) cv.wait_for(g, std::chrono::milliseconds(5));
                    else g.unlock(), std::this_thread::sleep_for(std::chrono::microseconds(20));
                    continue;
                }
                Request &h = *queue.front();
                const size_t need = (h.bytesA + 255) / 256 * 256 + (h.bytesB + 255) / 256 * 256 +
                                    (h.bytesC + 255) / 256 * 256;
                size_t off = 0;
                if (!arena.alloc(need, &off)) {
                    ++stalls;  // waits for memory to come back
                    g.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(20));
                    continue;
                }
                r = std::move(queue.front());
                queue.pop_front();
                r->offset = off;
                r->bytes = need;
            }
            // plans are cached per stream: one plan never runs on two
            // streams at once (tc_execute refuses that)
            r->stream = rr++ % (int)streams.size();
            const std::string pkey = key(*r) + "#" + std::to_string(r->stream);
            auto it = plans.find(pkey);
            if (it == plans.end()) {
                tc_plan p = nullptr;
                tc_status s = tc_plan_create(&p, r->spec.c_str(), r->extents.data(), nullptr, r->dtype);
                // requests on one stream reuse its plan back to back: no plan
                // workspace (the GETT's pre-converted input) to keep apart
                if (s == TC_SUCCESS) s = tc_plan_set_gett_pack(p, 0);
                if (s != TC_SUCCESS) {
                    if (p) tc_plan_destroy(p);
                    finish(r, s);
                    continue;
                }
                it = plans.emplace(pkey, p).first;
            }
            r->plan = it->second;  // algorithm 0, the fused GETT
            tc_status s = launch(*r);
            if (s != TC_SUCCESS) {
                cudaStreamSynchronize(streams[r->stream]);
                finish(r, s);
                continue;
            }
            inflight.push_back(std::move(r));
            std::lock_guard<std::mutex> g(mu);
            peak_inflight = std::max<int64_t>(peak_inflight, (int64_t)inflight.size());
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
    cudaError_t e = cudaMalloc(&S.arena_base, (size_t)budget_bytes);
    if (e != cudaSuccess) {
        delete h;
        return fail(TC_ERROR_OUT_OF_MEMORY, cudaGetErrorString(e));
    }
    S.arena.init((size_t)budget_bytes);
    for (int i = 0; i < streams; ++i) {
        cudaStream_t st;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        S.streams.push_back(st);
    }
    S.worker = std::thread([&S] { S.run(); });
    *out = h;
    return TC_SUCCESS;
}

tc_status tc_server_submit(tc_server server, const char *spec, const int64_t *extents, tc_dtype dtype,
                           const void *A, const void *B, void *C, int64_t *request_id) {
    if (!server || !spec || !extents || !A || !B || !request_id)
        return fail(TC_ERROR_INVALID_ARGUMENT, "NULL argument");
    ServerImpl &S = server->s;
    // validate and size the request with a throw-away plan (host work only)
    tc_plan p = nullptr;
    tc_status s = tc_plan_create(&p, spec, extents, nullptr, dtype);
    if (s != TC_SUCCESS) return s;
    auto r = std::make_unique<Request>();
    r->spec = spec;
    r->extents.assign(extents, extents + p->p.nidx);
    r->dtype = dtype;
    r->hA = A;
    r->hB = B;
    r->hC = C;
    r->bytesA = operand_bytes(p->p, OP_A);
    r->bytesB = operand_bytes(p->p, OP_B);
    r->bytesC = operand_bytes(p->p, OP_C);
    double f = 0;
    tc_plan_flops(p, &f);
    r->flops = f;
    tc_plan_destroy(p);
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
    for (auto &kv : S.plans) tc_plan_destroy(kv.second);
    for (cudaStream_t st : S.streams) cudaStreamDestroy(st);
    if (S.arena_base) cudaFree(S.arena_base);
    delete server;
    return TC_SUCCESS;
}

}  // extern "C"
