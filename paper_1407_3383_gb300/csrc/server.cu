// Serving loop: continuous batching of integer and polynomial products.
//
// The paper's products (Sections 5.2, 5.3) run one at a time on one core.
// Here a native scheduler thread keeps the transform tables of the three
// 62-bit primes resident and admits requests in arrival order into a fixed
// number of slots (CUDA streams) as long as the device-memory arena has room
// for the request's operands, output and workspace.  A request that arrives
// while others run is admitted as soon as a slot and memory free up, so the
// work of several requests overlaps on the device.  Each request's latency
// is measured on the host from submission to the completion of its last
// copy back.
//
// Memory admission: one device arena allocated at creation, first-fit free
// list with coalescing.  No allocation happens per request.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gbntt.h"
#include "kernels.h"
#include "plan.h"

using namespace gbntt;
using Clock = std::chrono::steady_clock;

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// First-fit free list over [0, size) with coalescing on release.
class Arena {
  public:
    void reset(size_t size) {
        free_.clear();
        free_[0] = size;
    }
    bool alloc(size_t n, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
  private:
    std::map<size_t, size_t> free_;
};

enum ReqState { kPending = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Request {
    uint64_t id = 0;
    unsigned kind = 0;          // NTT_REQ_INTMUL or NTT_REQ_POLYMUL
    unsigned prime = 0;         // polymul: index of P1..P3
    unsigned flags = 0;
    const void* a = nullptr;
    const void* b = nullptr;
    void* c = nullptr;
    size_t na = 0, nb = 0;
    size_t need = 0, off = 0;
    int slot = -1;
    int state = kPending;
    int status = NTT_OK;
    Clock::time_point t_submit, t_done;
    cudaEvent_t done = nullptr;
};

}  // namespace

struct ntt_server {
    ntt_server_config cfg{};
    int device = 0;
    intmul_plan* ip = nullptr;
    void* arena_base = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<bool> busy;
    std::vector<cudaEvent_t> events;       // one per slot, reused
    std::deque<Request*> pending;
    std::vector<Request*> running;
    std::map<uint64_t, Request*> table;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    uint64_t completed = 0;
    size_t peak_inflight = 0;
};

namespace {

size_t word_bytes_of(const Request* r) { return r->kind == NTT_REQ_INTMUL ? 4 : 8; }

// Device bytes of a request: operands, output, scratch.
size_t need_bytes(const ntt_server* S, const Request* r) {
    const size_t wb = word_bytes_of(r);
    size_t n = 0;
    const bool dev = (r->flags & NTT_REQ_DEVICE) != 0;
    if (!dev) {
        n += align256(r->na * wb) + align256(r->nb * wb);
        n += align256((r->kind == NTT_REQ_INTMUL ? r->na + r->nb : r->na + r->nb - 1) * wb);
    }
    if (r->kind == NTT_REQ_INTMUL) {
        n += align256(intmul_workspace_size(S->ip, r->na, r->nb));
    } else {
        int k = 1;
        while ((1ull << k) < r->na + r->nb - 1) ++k;
        const ntt_plan* np = S->ip->plans[r->prime][k];
        n += np ? align256(polymul_ws_bytes(np, 1, NTT_SCHED_FUSED)) : 0;
    }
    return std::max<size_t>(n, 256);
}

// Enqueue the whole request on its slot's stream.
int launch_request(ntt_server* S, Request* r) {
    cudaStream_t st = S->streams[r->slot];
    unsigned char* base = static_cast<unsigned char*>(S->arena_base) + r->off;
    const size_t wb = word_bytes_of(r);
    const size_t nc = (r->kind == NTT_REQ_INTMUL) ? r->na + r->nb : r->na + r->nb - 1;
    const void* da = r->a;
    const void* db = r->b;
    void* dc = r->c;
    size_t off = 0;
    if (!(r->flags & NTT_REQ_DEVICE)) {
        void* a_dev = base + off;
        off += align256(r->na * wb);
        void* b_dev = base + off;
        off += align256(r->nb * wb);
        dc = base + off;
        off += align256(nc * wb);
        if (cudaMemcpyAsync(a_dev, r->a, r->na * wb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(b_dev, r->b, r->nb * wb, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return NTT_ERR_CUDA;
        da = a_dev;
        db = b_dev;
    }
    void* ws = base + off;
    const size_t ws_bytes = r->need - off;
    int rc;
    if (r->kind == NTT_REQ_INTMUL) {
        rc = intmul_crt(S->ip, static_cast<const uint32_t*>(da), r->na, static_cast<const uint32_t*>(db), r->nb,
                        static_cast<uint32_t*>(dc), ws, ws_bytes, st);
    } else {
        int k = 1;
        while ((1ull << k) < r->na + r->nb - 1) ++k;
        rc = polymul_mod_p_batch(S->ip->plans[r->prime][k], da, r->na, db, r->nb, 1, dc, NTT_SCHED_FUSED,
                                 ws, ws_bytes, st);
    }
    if (rc != NTT_OK) return rc;
    if (!(r->flags & NTT_REQ_DEVICE) &&
        cudaMemcpyAsync(r->c, dc, nc * wb, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return NTT_ERR_CUDA;
    if (cudaEventRecord(r->done, st) != cudaSuccess) return NTT_ERR_CUDA;
    return NTT_OK;
}

void worker_loop(ntt_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    while (!S->stop) {
        bool progressed = false;
        // completions
        for (size_t i = 0; i < S->running.size();) {
            Request* r = S->running[i];
            const cudaError_t q = cudaEventQuery(r->done);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            r->t_done = Clock::now();
            r->state = (q == cudaSuccess) ? kDone : kFailed;
            if (q != cudaSuccess) r->status = NTT_ERR_CUDA;
            S->arena.release(r->off, r->need);
            S->busy[r->slot] = false;
            S->running.erase(S->running.begin() + static_cast<long>(i));
            ++S->completed;
            progressed = true;
        }
        // admissions, in arrival order
        while (!S->pending.empty()) {
            Request* r = S->pending.front();
            int slot = -1;
            for (size_t s = 0; s < S->busy.size(); ++s)
                if (!S->busy[s]) { slot = static_cast<int>(s); break; }
            if (slot < 0) break;
            size_t off = 0;
            if (!S->arena.alloc(r->need, &off)) break;     // wait for memory to free up
            S->pending.pop_front();
            r->off = off;
            r->slot = slot;
            r->done = S->events[slot];
            S->busy[slot] = true;
            const int rc = launch_request(S, r);
            if (rc != NTT_OK) {
                cudaStreamSynchronize(S->streams[slot]);   // nothing left reading the region
                r->status = rc;
                r->state = kFailed;
                r->t_done = Clock::now();
                S->arena.release(r->off, r->need);
                S->busy[slot] = false;
                ++S->completed;
            } else {
                r->state = kRunning;
                S->running.push_back(r);
                S->peak_inflight = std::max(S->peak_inflight, S->running.size());
            }
            progressed = true;
        }
        if (progressed) S->cv.notify_all();
        if (S->running.empty() && S->pending.empty()) {
            S->cv.wait(lock, [&] { return S->stop || !S->pending.empty(); });
        } else {
            S->cv.wait_for(lock, std::chrono::microseconds(20));
        }
    }
}

}  // namespace

extern "C" int ntt_server_create(const ntt_server_config* cfg, ntt_server** out) {
    if (!cfg || !out || cfg->slots == 0 || cfg->slots > 64 || cfg->mem_bytes < 4096 || cfg->max_limbs == 0)
        return NTT_ERR_ARG;
    *out = nullptr;
    ntt_server* S = new (std::nothrow) ntt_server();
    if (!S) return NTT_ERR_OOM;
    S->cfg = *cfg;
    cudaGetDevice(&S->device);
    // transform lengths for both request kinds: a polynomial product of
    // max_limbs-word operands needs one doubling more than an integer product
    // of max_limbs-limb operands (two limbs per coefficient)
    int rc = intmul_plan_create(2 * cfg->max_limbs, &S->ip);
    if (rc != NTT_OK) {
        delete S;
        return rc;
    }
    if (cudaMalloc(&S->arena_base, cfg->mem_bytes) != cudaSuccess) {
        cudaGetLastError();
        intmul_plan_destroy(S->ip);
        delete S;
        return NTT_ERR_OOM;
    }
    S->arena.reset(cfg->mem_bytes / 256 * 256);
    S->streams.resize(cfg->slots);
    S->events.resize(cfg->slots);
    S->busy.assign(cfg->slots, false);
    for (unsigned i = 0; i < cfg->slots; ++i) {
        cudaStreamCreateWithFlags(&S->streams[i], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&S->events[i], cudaEventDisableTiming);
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return NTT_OK;
}

extern "C" int ntt_server_submit(ntt_server* S, unsigned kind, unsigned prime, const void* a, size_t na,
                                 const void* b, size_t nb, void* c, unsigned flags, uint64_t* id_out) {
    if (!S || !a || !b || !c || !id_out || na == 0 || nb == 0) return NTT_ERR_ARG;
    if (kind != NTT_REQ_INTMUL && kind != NTT_REQ_POLYMUL) return NTT_ERR_ARG;
    if (kind == NTT_REQ_POLYMUL && prime > 2) return NTT_ERR_ARG;
    Request* r = new (std::nothrow) Request();
    if (!r) return NTT_ERR_OOM;
    r->kind = kind;
    r->prime = prime;
    r->flags = flags;
    r->a = a;
    r->b = b;
    r->c = c;
    r->na = na;
    r->nb = nb;
    // size check against the resident plans
    const size_t chunks = (kind == NTT_REQ_INTMUL) ? (na + 1) / 2 + (nb + 1) / 2 - 1 : na + nb - 1;
    int k = 1;
    while ((1ull << k) < chunks) ++k;
    if (k > static_cast<int>(S->ip->max_log2n)) {
        delete r;
        gbntt_set_error("ntt_server_submit: request larger than the server's max_limbs");
        return NTT_ERR_SIZE;
    }
    r->need = need_bytes(S, r);
    if (r->need > S->cfg.mem_bytes) {
        delete r;
        gbntt_set_error("ntt_server_submit: request needs more device memory than the arena holds");
        return NTT_ERR_OOM;
    }
    {
        std::lock_guard<std::mutex> lock(S->mu);
        r->id = S->next_id++;
        r->t_submit = Clock::now();
        S->table[r->id] = r;
        S->pending.push_back(r);
    }
    S->cv.notify_all();
    *id_out = r->id;
    return NTT_OK;
}

static int finish_query(Request* r, int* state, double* latency_ms) {
    if (state) *state = r->state;
    if (latency_ms && (r->state == kDone || r->state == kFailed))
        *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    return r->state == kFailed ? r->status : NTT_OK;
}

extern "C" int ntt_server_poll(ntt_server* S, uint64_t id, int* state, double* latency_ms) {
    if (!S) return NTT_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->table.find(id);
    if (it == S->table.end()) return NTT_ERR_ARG;
    return finish_query(it->second, state, latency_ms);
}

extern "C" int ntt_server_wait(ntt_server* S, uint64_t id, int timeout_ms, double* latency_ms) {
    if (!S) return NTT_ERR_ARG;
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->table.find(id);
    if (it == S->table.end()) return NTT_ERR_ARG;
    Request* r = it->second;
    const bool ok = S->cv.wait_for(lock, std::chrono::milliseconds(timeout_ms),
                                   [&] { return r->state == kDone || r->state == kFailed; });
    if (!ok) return NTT_ERR_TIMEOUT;
    return finish_query(r, nullptr, latency_ms);
}

extern "C" int ntt_server_release(ntt_server* S, uint64_t id) {
    if (!S) return NTT_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->table.find(id);
    if (it == S->table.end()) return NTT_ERR_ARG;
    if (it->second->state != kDone && it->second->state != kFailed) return NTT_ERR_ARG;
    delete it->second;
    S->table.erase(it);
    return NTT_OK;
}

extern "C" int ntt_server_stats(ntt_server* S, uint64_t* completed, uint64_t* pending, uint64_t* running,
                                uint64_t* peak_inflight) {
    if (!S) return NTT_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    if (completed) *completed = S->completed;
    if (pending) *pending = S->pending.size();
    if (running) *running = S->running.size();
    if (peak_inflight) *peak_inflight = S->peak_inflight;
    return NTT_OK;
}

extern "C" int ntt_server_destroy(ntt_server* S) {
    if (!S) return NTT_ERR_ARG;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (size_t i = 0; i < S->streams.size(); ++i) {
        cudaStreamSynchronize(S->streams[i]);
        cudaStreamDestroy(S->streams[i]);
        cudaEventDestroy(S->events[i]);
    }
    for (auto& kv : S->table) delete kv.second;   // every request, pending or not
    if (S->arena_base) cudaFree(S->arena_base);
    if (S->ip) intmul_plan_destroy(S->ip);
    delete S;
    return NTT_OK;
}
