// Polynomial products of host-resident operands, with the copies overlapped.
//
// polymul_mod_p_batch_host() runs the products of polymul_mod_p_batch (fused
// schedule, Section 5.2) for operands and results that live in host memory.
// The batch is cut into chunks of at most `chunk` products (smaller at both
// ends of a long batch, see chunk_sizes).  Chunk i is copied to
// the device on a copy stream, multiplied on the caller's stream and copied
// back on a second copy stream, so that the upload of chunk i+1, the product
// of chunk i and the download of chunk i-1 run at the same time.  Three sets
// of device staging buffers (operands and result of one chunk each) rotate
// between the chunks; one workspace serves the products, which run in order
// on the caller's stream.  Events order the stages:
//   upload(i)   after the product of chunk i-3 (it read the same operand set),
//   product(i)  after upload(i) and after download(i-3) (same result set),
//   download(i) after product(i),
// and the caller's stream waits for the last download.
//
// The copy streams and events are created once per device, on the first
// call there, and kept until the process exits.  One host mutex per device
// serialises the enqueueing, so concurrent callers cannot interleave their
// event records.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gbntt.h"
#include "kernels.h"
#include "plan.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kSets = 3;

struct CopyStreams {
    bool ready = false;
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t start = nullptr;
    cudaEvent_t uploaded[kSets] = {}, multiplied[kSets] = {}, downloaded[kSets] = {};
};

std::mutex g_mu[kMaxDevices];
CopyStreams g_cs[kMaxDevices];

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

struct StageLayout {
    size_t a, b, c, ws, set, total;   // bytes of each piece; set = a + b + c
};

StageLayout stage_layout(const ntt_plan* P, size_t na, size_t nb, size_t chunk) {
    StageLayout L{};
    const size_t wb = P->word_bytes;
    L.a = round256(chunk * na * wb);
    L.b = round256(chunk * nb * wb);
    L.c = round256(chunk * (na + nb - 1) * wb);
    L.ws = round256(gbntt::polymul_ws_bytes(P, chunk, NTT_SCHED_FUSED));
    L.set = L.a + L.b + L.c;
    L.total = kSets * L.set + L.ws;
    return L;
}

// Creates the copy streams and events of the current device (caller holds
// the device's mutex).
int ensure_streams(CopyStreams& cs) {
    if (cs.ready) return NTT_OK;
    bool ok = cudaStreamCreateWithFlags(&cs.up, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&cs.down, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&cs.start, cudaEventDisableTiming) == cudaSuccess;
    for (int s = 0; ok && s < kSets; ++s)
        ok = cudaEventCreateWithFlags(&cs.uploaded[s], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&cs.multiplied[s], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&cs.downloaded[s], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        gbntt_set_error(std::string("polymul_mod_p_batch_host: stream/event creation: ") +
                        cudaGetErrorString(cudaGetLastError()));
        return NTT_ERR_CUDA;
    }
    cs.ready = true;
    return NTT_OK;
}

// Chunk sizes for `batch` products with at most `chunk` per chunk.  The
// first upload and the last product and download overlap nothing, so for
// three or more full chunks the pipeline ramps: chunk/4, chunk/2, then full
// chunks, then chunk/2 and chunk/4 (the remainder goes before the ramp-down).
std::vector<size_t> chunk_sizes(size_t batch, size_t chunk) {
    std::vector<size_t> v;
    if (batch >= 3 * chunk && chunk >= 4) {
        const size_t q = chunk / 4, h = chunk / 2;
        v.push_back(q);
        v.push_back(h);
        size_t rem = batch - 2 * (q + h);
        while (rem > chunk) {
            v.push_back(chunk);
            rem -= chunk;
        }
        v.push_back(rem);
        v.push_back(h);
        v.push_back(q);
    } else {
        for (size_t first = 0; first < batch; first += chunk) v.push_back(std::min(chunk, batch - first));
    }
    return v;
}

}  // namespace

extern "C" size_t polymul_host_stage_size(const ntt_plan* plan, size_t na, size_t nb, size_t chunk) {
    if (!plan || na == 0 || nb == 0 || chunk == 0) return 0;
    if (na + nb - 1 > (size_t(1) << plan->log2n)) return 0;
    return stage_layout(plan, na, nb, chunk).total;
}

extern "C" int polymul_mod_p_batch_host(const ntt_plan* plan, const void* h_a, size_t na,
                                        const void* h_b, size_t nb, size_t batch, void* h_c,
                                        size_t chunk, void* d_stage, size_t stage_bytes,
                                        void* stream) {
    const ntt_plan* P = plan;
    if (!P) return NTT_ERR_ARG;
    if (batch == 0) return NTT_OK;
    if (!h_a || !h_b || !h_c || na == 0 || nb == 0 || chunk == 0) {
        gbntt_set_error("polymul_mod_p_batch_host: null operand, empty polynomial or zero chunk");
        return NTT_ERR_ARG;
    }
    if (na + nb - 1 > (size_t(1) << P->log2n)) {
        gbntt_set_error("polymul_mod_p_batch_host: na + nb - 1 exceeds the plan's n");
        return NTT_ERR_SIZE;
    }
    if (chunk > batch) chunk = batch;
    const StageLayout L = stage_layout(P, na, nb, chunk);
    if (!d_stage || stage_bytes < L.total || (reinterpret_cast<uintptr_t>(d_stage) & 255)) {
        gbntt_set_error("polymul_mod_p_batch_host: staging buffer of " + std::to_string(L.total) +
                        " bytes (256-byte aligned) required for chunks of " + std::to_string(chunk));
        return NTT_ERR_WORKSPACE;
    }
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return NTT_ERR_CUDA;
    }
    if (device < 0 || device >= kMaxDevices || device != P->device) {
        gbntt_set_error("polymul_mod_p_batch_host: the plan's device must be current");
        return NTT_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu[device]);
    CopyStreams& cs = g_cs[device];
    int rc = ensure_streams(cs);
    if (rc != NTT_OK) return rc;

    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t wb = P->word_bytes, nc = na + nb - 1;
    unsigned char* base = static_cast<unsigned char*>(d_stage);
    void* ws = L.ws ? base + kSets * L.set : nullptr;
    auto fail = [](cudaError_t e) {
        gbntt_set_error(std::string("polymul_mod_p_batch_host: ") + cudaGetErrorString(e));
        return NTT_ERR_CUDA;
    };
    cudaError_t e;
    // both copy streams start after the work already on the caller's stream
    if ((e = cudaEventRecord(cs.start, st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(cs.up, cs.start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(cs.down, cs.start, 0)) != cudaSuccess)
        return fail(e);

    const std::vector<size_t> sizes = chunk_sizes(batch, chunk);
    const size_t nchunks = sizes.size();
    size_t first = 0;
    for (size_t i = 0; i < nchunks; first += sizes[i], ++i) {
        const int s = static_cast<int>(i % kSets);
        const size_t cnt = sizes[i];
        unsigned char* da = base + s * L.set;
        unsigned char* db = da + L.a;
        unsigned char* dc = db + L.b;
        if (i >= kSets && (e = cudaStreamWaitEvent(cs.up, cs.multiplied[s], 0)) != cudaSuccess)
            return fail(e);
        if ((e = cudaMemcpyAsync(da, static_cast<const unsigned char*>(h_a) + first * na * wb,
                                 cnt * na * wb, cudaMemcpyHostToDevice, cs.up)) != cudaSuccess ||
            (e = cudaMemcpyAsync(db, static_cast<const unsigned char*>(h_b) + first * nb * wb,
                                 cnt * nb * wb, cudaMemcpyHostToDevice, cs.up)) != cudaSuccess ||
            (e = cudaEventRecord(cs.uploaded[s], cs.up)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, cs.uploaded[s], 0)) != cudaSuccess)
            return fail(e);
        if (i >= kSets && (e = cudaStreamWaitEvent(st, cs.downloaded[s], 0)) != cudaSuccess)
            return fail(e);
        rc = polymul_mod_p_batch(P, da, na, db, nb, cnt, dc, NTT_SCHED_FUSED, ws, L.ws, stream);
        if (rc != NTT_OK) return rc;
        if ((e = cudaEventRecord(cs.multiplied[s], st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(cs.down, cs.multiplied[s], 0)) != cudaSuccess ||
            (e = cudaMemcpyAsync(static_cast<unsigned char*>(h_c) + first * nc * wb, dc, cnt * nc * wb,
                                 cudaMemcpyDeviceToHost, cs.down)) != cudaSuccess ||
            (e = cudaEventRecord(cs.downloaded[s], cs.down)) != cudaSuccess)
            return fail(e);
    }
    // downloads run in order on their stream: the last one ends the call
    const int last = static_cast<int>((nchunks - 1) % kSets);
    if ((e = cudaStreamWaitEvent(st, cs.downloaded[last], 0)) != cudaSuccess) return fail(e);
    return NTT_OK;
}
