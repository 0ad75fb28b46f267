// Uneven batches of polynomial products with mixed moduli (the batched form
// of Section 5.2's product; Remark 6 of Section 2.2 notes that one vector
// operation may serve several moduli at once).
//
// A batch plan sorts the products once, on the host:
//  - products whose transform length 2^k fits one thread block
//    (k <= tile_max_log) become items of up to 16 equal-size, equal-modulus
//    products, ordered by decreasing size; one persistent kernel drains them
//    from a ticket counter; each item's transforms are truncated to the
//    blocks its longest output needs (Section 5.1's TFT);
//  - longer products are grouped into buckets of equal (modulus, k), each
//    run as the three global passes of the fused schedule.
// The work of a run can be captured once into a CUDA graph whose branches
// (the persistent kernel and the buckets, spread over internal streams)
// overlap on the device; later runs with the same buffers replay it.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/gbntt.h"
#include "kernels.h"
#include "plan.h"

using namespace gbntt;

namespace {

constexpr int kBatchStreams = 4;

struct Bucket {
    unsigned prime;
    int log2n;
    unsigned first, count;
    ntt_plan* plan;
    size_t ws_off;
    long long subs;      // 2^16-point row slots kept (products of 2^17 .. 2^24 points)
    bool tft;            // n < 2^16: every product's output needs few enough column blocks to truncate
};

}  // namespace

struct polymul_batch_plan {
    int device = 0;
    unsigned wb = 0;
    unsigned flags = 0;
    std::vector<uint64_t> primes;
    std::vector<ntt_plan*> small_plans;          // per prime (may be null)
    std::map<std::pair<unsigned, int>, ntt_plan*> big_plans;
    std::vector<Bucket> buckets;
    size_t count = 0;
    void* d_block = nullptr;                     // descriptors, items, modulus constants
    BatchDesc* d_desc = nullptr;
    void* d_items = nullptr;
    void* d_plans = nullptr;
    void* d_tfts = nullptr;                      // inverse-TFT constants per modulus
    unsigned nitems = 0;
    size_t small_smem = 0;
    int small_grid = 0;
    size_t ticket_off = 0;
    size_t ws_bytes = 0;
    // graph replay
    cudaStream_t streams[kBatchStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t joins[kBatchStreams] = {};
    cudaGraphExec_t exec = nullptr;
    const void* ga = nullptr;
    const void* gb = nullptr;
    void* gc = nullptr;
    void* gws = nullptr;
};

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int log2_ceil(unsigned long long x) {
    int k = 0;
    while ((1ull << k) < x) ++k;
    return std::max(k, 1);
}

template <class Ar, class TwOf>
int build_device_block(polymul_batch_plan* B, const std::vector<BatchDesc>& descs,
                       const std::vector<SmallItem<Ar>>& items, TwOf) {
    std::vector<DevPlan<Ar>> dps(B->primes.size());
    std::vector<TftConsts<Ar>> tfts(B->primes.size());
    for (size_t i = 0; i < B->primes.size(); ++i) {
        if (!B->small_plans[i]) continue;
        if constexpr (sizeof(typename Ar::word) == 4) {
            dps[i] = B->small_plans[i]->dp32;
            tfts[i] = B->small_plans[i]->tft32;
        } else {
            dps[i] = B->small_plans[i]->dp64;
            tfts[i] = B->small_plans[i]->tft64;
        }
    }
    const size_t off_desc = 0;
    const size_t off_items = align256(off_desc + descs.size() * sizeof(BatchDesc));
    const size_t off_plans = align256(off_items + items.size() * sizeof(SmallItem<Ar>));
    const size_t off_tfts = align256(off_plans + dps.size() * sizeof(DevPlan<Ar>));
    const size_t total = align256(off_tfts + tfts.size() * sizeof(TftConsts<Ar>));
    if (cudaMalloc(&B->d_block, std::max<size_t>(total, 256)) != cudaSuccess) {
        cudaGetLastError();
        return NTT_ERR_OOM;
    }
    unsigned char* base = static_cast<unsigned char*>(B->d_block);
    std::vector<unsigned char> host(total, 0);
    std::copy(reinterpret_cast<const unsigned char*>(descs.data()),
              reinterpret_cast<const unsigned char*>(descs.data() + descs.size()), host.begin() + off_desc);
    std::copy(reinterpret_cast<const unsigned char*>(items.data()),
              reinterpret_cast<const unsigned char*>(items.data() + items.size()), host.begin() + off_items);
    std::copy(reinterpret_cast<const unsigned char*>(dps.data()),
              reinterpret_cast<const unsigned char*>(dps.data() + dps.size()), host.begin() + off_plans);
    std::copy(reinterpret_cast<const unsigned char*>(tfts.data()),
              reinterpret_cast<const unsigned char*>(tfts.data() + tfts.size()), host.begin() + off_tfts);
    if (total && cudaMemcpy(base, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
        gbntt_set_error("batch plan upload failed");
        return NTT_ERR_CUDA;
    }
    B->d_desc = reinterpret_cast<BatchDesc*>(base + off_desc);
    B->d_items = base + off_items;
    B->d_plans = base + off_plans;
    B->d_tfts = base + off_tfts;
    B->nitems = static_cast<unsigned>(items.size());
    size_t smem = 0;
    for (const auto& it : items)
        smem = std::max(smem, tile_smem_bytes(sizeof(typename Ar::word), static_cast<int>(it.logL),
                                              small_lppc(static_cast<int>(it.logL)) + 1));
    B->small_smem = smem;
    return NTT_OK;
}

// Group products into items (one-block sizes) and buckets (two-pass sizes);
// returns the descriptors in execution order.
template <class Ar, class TwOf>
int plan_products(polymul_batch_plan* B, const polymul_desc* h, size_t count, TwOf tw_of) {
    const int tile_max = (B->wb == 4) ? kTileMaxLog32 : kTileMaxLog64;
    struct Ent {
        size_t idx;
        int k;
        bool tft;   // two-pass sizes below 2^16: truncated transforms pay for this product
    };
    std::vector<Ent> small, big;
    for (size_t t = 0; t < count; ++t) {
        const polymul_desc& d = h[t];
        if (d.na == 0 || d.nb == 0 || d.prime >= B->primes.size()) {
            gbntt_set_error("batch descriptor " + std::to_string(t) + ": empty operand or bad modulus index");
            return NTT_ERR_ARG;
        }
        const int k = log2_ceil(static_cast<unsigned long long>(d.na) + d.nb - 1);
        const uint64_t p = B->primes[d.prime];
        if (k > static_cast<int>(__builtin_ctzll(p - 1)) || k > 24) {
            gbntt_set_error("batch descriptor " + std::to_string(t) + ": product too long for its modulus");
            return NTT_ERR_SIZE;
        }
        const long long nc = static_cast<long long>(d.na) + d.nb - 1;
        const bool tft = k < 16 && tft_kb(nc, k) <= kColTftMaxBlocks;
        (k <= tile_max ? small : big).push_back({t, k, tft});
    }
    // items: decreasing size, then modulus, then decreasing output length
    // (so that the products of one item need about as many blocks of the
    // truncated transform)
    auto out_len = [&](const Ent& e) { return static_cast<long long>(h[e.idx].na) + h[e.idx].nb - 1; };
    std::stable_sort(small.begin(), small.end(), [&](const Ent& x, const Ent& y) {
        if (x.k != y.k) return x.k > y.k;
        if (h[x.idx].prime != h[y.idx].prime) return h[x.idx].prime < h[y.idx].prime;
        return out_len(x) > out_len(y);
    });
    std::vector<BatchDesc> descs;
    std::vector<SmallItem<Ar>> items;
    std::vector<int> max_small_k(B->primes.size(), 0);
    for (size_t s = 0; s < small.size();) {
        const int k = small[s].k;
        const unsigned pr = h[small[s].idx].prime;
        const unsigned cap = 1u << small_lppc(k);
        SmallItem<Ar> it{};
        it.first = static_cast<unsigned>(descs.size());
        it.prime = pr;
        it.logL = static_cast<unsigned>(k);
        const uint64_t p = B->primes[pr];
        const uint64_t ninv = host::pow_mod((1ull << k) % p, p - 2, p);
        const uint64_t r = (B->wb == 4) ? ((1ull << 32) % p)
                                        : static_cast<uint64_t>((static_cast<unsigned __int128>(1) << 64) % p);
        it.scale = tw_of(host::mul_mod(ninv, r, p), p);
        it.kb = k >= kTileTftMinLog ? static_cast<unsigned>(tft_kb(out_len(small[s]), k)) : 16u;
        if (it.kb > static_cast<unsigned>(kTileTftMaxBlocks)) it.kb = 16;   // the full transforms
        while (s < small.size() && small[s].k == k && h[small[s].idx].prime == pr && it.count < cap) {
            const polymul_desc& d = h[small[s].idx];
            descs.push_back(BatchDesc{d.a_off, d.b_off, d.c_off, d.na, d.nb});
            ++it.count;
            ++s;
        }
        items.push_back(it);
        max_small_k[pr] = std::max(max_small_k[pr], k);
    }
    for (size_t i = 0; i < B->primes.size(); ++i) {
        if (!max_small_k[i]) continue;
        int rc = ntt_plan_create(B->primes[i], static_cast<unsigned>(max_small_k[i]), 0, &B->small_plans[i]);
        if (rc != NTT_OK) return rc;
    }
    // buckets: equal (modulus, k), and below 2^16 points equal truncation class
    std::stable_sort(big.begin(), big.end(), [&](const Ent& x, const Ent& y) {
        if (x.k != y.k) return x.k > y.k;
        if (h[x.idx].prime != h[y.idx].prime) return h[x.idx].prime < h[y.idx].prime;
        return x.tft < y.tft;
    });
    size_t ws = 256;   // the ticket counter
    B->ticket_off = 0;
    for (size_t s = 0; s < big.size();) {
        Bucket bk{};
        bk.prime = h[big[s].idx].prime;
        bk.log2n = big[s].k;
        bk.first = static_cast<unsigned>(descs.size());
        bk.tft = big[s].tft;
        // products of 2^17 .. 2^24 points keep lam = ceil(L / 2^16) of their
        // n2 = 2^(k-16) rows (whole blocks of n2/16 rows past 16 rows): the
        // truncated transform of Section 5.1 with Algorithm 1's rows; their
        // kept rows take consecutive slots of the bucket's workspace
        const long long n2 = bk.log2n > 16 ? (1LL << (bk.log2n - 16)) : 0;
        while (s < big.size() && big[s].k == bk.log2n && h[big[s].idx].prime == bk.prime &&
               big[s].tft == bk.tft) {
            const polymul_desc& d = h[big[s].idx];
            BatchDesc bd{d.a_off, d.b_off, d.c_off, d.na, d.nb, static_cast<unsigned long long>(bk.subs)};
            if (n2) {
                const long long L = static_cast<long long>(d.na) + d.nb - 1;
                long long lam = std::min<long long>(n2, (L + 65535) >> 16);
                if (n2 > 16) lam = (lam + n2 / 16 - 1) / (n2 / 16) * (n2 / 16);
                bk.subs += lam;
            }
            descs.push_back(bd);
            ++bk.count;
            ++s;
        }
        auto key = std::make_pair(bk.prime, bk.log2n);
        if (!B->big_plans.count(key)) {
            ntt_plan* np = nullptr;
            int rc = ntt_plan_create(B->primes[bk.prime], static_cast<unsigned>(bk.log2n), 0, &np);
            if (rc != NTT_OK) return rc;
            B->big_plans[key] = np;
        }
        bk.plan = B->big_plans[key];
        bk.ws_off = ws;
        // sized for the untruncated schedule, which a tuned launch shape may
        // select at run time (the kept rows need no more than that)
        ws = align256(ws + 2 * (size_t(1) << bk.log2n) * B->wb * bk.count);
        B->buckets.push_back(bk);
    }
    B->ws_bytes = ws;
    int rc = build_device_block<Ar>(B, descs, items, tw_of);
    if (rc != NTT_OK) return rc;
    if (B->nitems) {
        int dev = 0, sms = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        occ = batch_small_occupancy<Ar>(B->small_smem);
        B->small_grid = std::max(1, std::min<int>(sms * occ, static_cast<int>(B->nitems)));
    }
    return NTT_OK;
}

template <class Ar>
int enqueue(polymul_batch_plan* B, const void* a, const void* b, void* c, void* ws, cudaStream_t st0,
            bool spread) {
    using word = typename Ar::word;
    unsigned char* wsb = static_cast<unsigned char*>(ws);
    unsigned* ticket = reinterpret_cast<unsigned*>(wsb + B->ticket_off);
    const word* A = static_cast<const word*>(a);
    const word* Bp = static_cast<const word*>(b);
    word* C = static_cast<word*>(c);
    if (spread) {
        cudaEventRecord(B->fork, st0);
        for (int i = 1; i < kBatchStreams; ++i) cudaStreamWaitEvent(B->streams[i], B->fork, 0);
    }
    int rc = NTT_OK;
    if (B->nitems) {
        cudaMemsetAsync(ticket, 0, sizeof(unsigned), st0);
        rc = launch_batch_small<Ar>(static_cast<const DevPlan<Ar>*>(B->d_plans),
                                    static_cast<const TftConsts<Ar>*>(B->d_tfts), B->d_desc, B->d_items,
                                    B->nitems, ticket, A, Bp, C, B->small_smem, B->small_grid, st0);
        if (rc != NTT_OK) return rc;
    }
    for (size_t i = 0; i < B->buckets.size(); ++i) {
        const Bucket& bk = B->buckets[i];
        cudaStream_t s = spread ? B->streams[1 + i % (kBatchStreams - 1)] : st0;
        const ntt_plan* np = bk.plan;
        word* wsp = reinterpret_cast<word*>(wsb + bk.ws_off);
        if constexpr (sizeof(word) == 4)
            rc = launch_batch_bucket<Ar>(np, np->dp32, A, Bp, C, B->d_desc + bk.first, bk.count, wsp,
                                         np->pm_scale32, s, bk.subs, bk.tft);
        else
            rc = launch_batch_bucket<Ar>(np, np->dp64, A, Bp, C, B->d_desc + bk.first, bk.count, wsp,
                                         np->pm_scale64, s, bk.subs, bk.tft);
        if (rc != NTT_OK) return rc;
    }
    if (spread) {
        for (int i = 1; i < kBatchStreams; ++i) {
            cudaEventRecord(B->joins[i], B->streams[i]);
            cudaStreamWaitEvent(st0, B->joins[i], 0);
        }
    }
    return NTT_OK;
}

int enqueue_any(polymul_batch_plan* B, const void* a, const void* b, void* c, void* ws, cudaStream_t st,
                bool spread) {
    return B->wb == 4 ? enqueue<Mont32>(B, a, b, c, ws, st, spread)
                      : enqueue<Shoup64L>(B, a, b, c, ws, st, spread);
}

void destroy_graph(polymul_batch_plan* B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    B->ga = B->gb = nullptr;
    B->gc = B->gws = nullptr;
}

}  // namespace

extern "C" int polymul_batch_plan_create(const uint64_t* primes, unsigned nprimes, const polymul_desc* h_desc,
                                         size_t count, unsigned flags, polymul_batch_plan** out) {
    if (!out || !primes || nprimes == 0 || nprimes > 64 || (!h_desc && count)) return NTT_ERR_ARG;
    *out = nullptr;
    unsigned wb = 0;
    for (unsigned i = 0; i < nprimes; ++i) {
        const unsigned w = (primes[i] >> 32) ? 8 : 4;
        if (wb && w != wb) {
            gbntt_set_error("batch moduli must share one word size (all < 2^32 or all >= 2^32)");
            return NTT_ERR_MODULUS;
        }
        wb = w;
        uint64_t g, w0;
        int rc = ntt_root_of_unity(primes[i], 4, &g, &w0);
        if (rc != NTT_OK || (primes[i] >> 62)) return rc != NTT_OK ? rc : NTT_ERR_MODULUS;
    }
    polymul_batch_plan* B = new (std::nothrow) polymul_batch_plan();
    if (!B) return NTT_ERR_OOM;
    cudaGetDevice(&B->device);
    B->wb = wb;
    B->flags = flags;
    B->count = count;
    B->primes.assign(primes, primes + nprimes);
    B->small_plans.assign(nprimes, nullptr);
    int rc;
    if (wb == 4)
        rc = plan_products<Mont32>(B, h_desc, count, [](uint64_t v, uint64_t p) {
            return host::tw32_of(v, static_cast<uint32_t>(p), host::inv_pow2_32(static_cast<uint32_t>(p)));
        });
    else
        rc = plan_products<Shoup64L>(B, h_desc, count, [](uint64_t v, uint64_t p) { return host::tw64_of(v, p); });
    if (rc == NTT_OK) {
        for (int i = 0; i < kBatchStreams; ++i)
            if (cudaStreamCreateWithFlags(&B->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&B->joins[i], cudaEventDisableTiming) != cudaSuccess)
                rc = NTT_ERR_CUDA;
        if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess) rc = NTT_ERR_CUDA;
    }
    if (rc != NTT_OK) {
        polymul_batch_plan_destroy(B);
        return rc;
    }
    *out = B;
    return NTT_OK;
}

extern "C" int polymul_batch_plan_destroy(polymul_batch_plan* B) {
    if (!B) return NTT_ERR_ARG;
    cudaDeviceSynchronize();
    destroy_graph(B);
    for (auto* p : B->small_plans)
        if (p) ntt_plan_destroy(p);
    for (auto& kv : B->big_plans) ntt_plan_destroy(kv.second);
    if (B->d_block) cudaFree(B->d_block);
    for (int i = 0; i < kBatchStreams; ++i) {
        if (B->streams[i]) cudaStreamDestroy(B->streams[i]);
        if (B->joins[i]) cudaEventDestroy(B->joins[i]);
    }
    if (B->fork) cudaEventDestroy(B->fork);
    delete B;
    return NTT_OK;
}

extern "C" size_t polymul_batch_workspace_size(const polymul_batch_plan* B) { return B ? B->ws_bytes : 0; }

extern "C" int polymul_batch_run(polymul_batch_plan* B, const void* d_a, const void* d_b, void* d_c,
                                 void* d_ws, size_t ws_bytes, unsigned mode, void* stream) {
    if (!B || !d_a || !d_b || !d_c || mode > NTT_BATCH_GRAPH) return NTT_ERR_ARG;
    if (!d_ws || ws_bytes < B->ws_bytes || (reinterpret_cast<uintptr_t>(d_ws) & 255)) {
        gbntt_set_error("polymul_batch_run: workspace of " + std::to_string(B->ws_bytes) +
                        " bytes (256-byte aligned) required");
        return NTT_ERR_WORKSPACE;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (mode == NTT_BATCH_DIRECT) return enqueue_any(B, d_a, d_b, d_c, d_ws, st, false);
    if (mode == NTT_BATCH_STREAMS) return enqueue_any(B, d_a, d_b, d_c, d_ws, st, true);
    // graph: capture once per buffer set, replay afterwards
    if (!B->exec || B->ga != d_a || B->gb != d_b || B->gc != d_c || B->gws != d_ws) {
        destroy_graph(B);
        cudaStream_t cap = B->streams[0];
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess)
            return NTT_ERR_CUDA;
        int rc = enqueue_any(B, d_a, d_b, d_c, d_ws, cap, true);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cap, &g);
        if (rc != NTT_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            gbntt_set_error("polymul_batch_run: graph capture failed");
            return rc != NTT_OK ? rc : NTT_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&B->exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            B->exec = nullptr;
            gbntt_set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
            return NTT_ERR_CUDA;
        }
        B->ga = d_a;
        B->gb = d_b;
        B->gc = d_c;
        B->gws = d_ws;
    }
    if (cudaGraphLaunch(B->exec, st) != cudaSuccess) {
        gbntt_set_error(std::string("cudaGraphLaunch: ") + cudaGetErrorString(cudaGetLastError()));
        return NTT_ERR_CUDA;
    }
    return NTT_OK;
}
