// Integer product by Kronecker segmentation and the three-prime transform
// (Section 5.3).
//
// a and b (little-endian 32-bit limbs) are cut into chunks of h bits, giving
// polynomials A, B with A(2^h) = a, B(2^h) = b.  h is the paper's choice:
// the largest h (here at most 96) for which every coefficient of C = A B,
// a sum of at most m = min(da, db) products of h-bit chunks, stays below
// 2^H with H = 2 h + bitlength(m) <= 183 < log2(P1 P2 P3) for the three
// primes P_i = k_i 2^40 + 1 of the 62-bit window -- so the number d of
// chunks is minimal (80 to 90 bits at the sizes served).  C is recovered
// exactly from C mod P1, P2, P3 (three polynomial products over Z/P_iZ,
// Section 5.2) by Garner's mixed-radix Chinese remaindering:
//     x1 = r1,  x2 = (r2 - x1) P1^-1 mod P2,
//     x3 = ((r3 - x1) P1^-1 - x2) P2^-1 mod P3,
//     c  = x1 + P1 (x2 + P2 x3)          (exact, < P1 P2 P3).
// Finally C(2^h) is evaluated: coefficient k (three words) lands at bit h k,
// each 64-bit word of the result sums the slices of the (at most four)
// coefficients overlapping it, and carries are propagated by a parallel scan
// of (generate, propagate, kill) states over the words.  The integer matrix
// product keeps h = 64.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include "../../include/gbntt.h"
#include "kernels.h"
#include "plan.h"

using u128 = unsigned __int128;

namespace gbntt {

namespace {

constexpr int kCarryThreads = 256;
constexpr int kCarryPerThread = 4;
constexpr int kCarryBlock = kCarryThreads * kCarryPerThread;   // words per block
constexpr uint8_t kKill = 0, kProp = 1, kGen = 2;

__device__ __forceinline__ uint8_t carry_combine(uint8_t before, uint8_t after) {
    return after == kProp ? before : after;
}

struct CrtArgs {
    uint64_t P1, P2, P3;
    Tw64 inv12, inv13, inv23;
    Tw64 r64[3];   // 2^64 rem P_i (chunks wider than 64 bits)
};

// Chunk k of h bits (64 <= h <= 96) of a limb array of n limbs: bits
// [k h, k h + h), from at most four limbs, as (low 64 bits, high part).
__device__ __forceinline__ void chunk_bits(const uint32_t* x, long long n, long long k, int h, uint64_t& lo,
                                           uint64_t& hi) {
    const long long b0 = k * h;
    const long long i0 = b0 >> 5;
    const int r = static_cast<int>(b0 & 31);
    u128 v = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (i0 + q < n) v |= static_cast<u128>(x[i0 + q]) << (32 * q);
    v >>= r;
    v &= (static_cast<u128>(1) << h) - 1;
    lo = static_cast<uint64_t>(v);
    hi = static_cast<uint64_t>(v >> 64);
}

// chunk k of a limb array (two limbs, the high one may be past the end)
__device__ __forceinline__ uint64_t chunk_of(const uint32_t* x, long long n, long long k) {
    const long long i = 2 * k;
    const uint64_t lo = (i < n) ? x[i] : 0u;
    const uint64_t hi = (i + 1 < n) ? x[i + 1] : 0u;
    return lo | (hi << 32);
}

// x < 2^64 < 8 P (P > 2^61) reduced by conditional subtraction of 4P, 2P, P.
__device__ __forceinline__ uint64_t reduce_chunk(uint64_t x, uint64_t P) {
    x = (x >= 4 * P) ? x - 4 * P : x;
    x = (x >= 2 * P) ? x - 2 * P : x;
    return (x >= P) ? x - P : x;
}

// Operand chunks of h bits reduced modulo each prime: red[i][0 .. da) = a,
// red[i][da .. da+db) = b.  A chunk lo + 2^64 hi is hi (2^64 rem P) + lo.
__global__ void k_split(const uint32_t* __restrict__ a, long long na, const uint32_t* __restrict__ b,
                        long long nb, long long da, long long db, int h, uint64_t* __restrict__ red,
                        long long red_stride, CrtArgs C) {
    const long long total = da + db;
    const uint64_t P[3] = {C.P1, C.P2, C.P3};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        uint64_t lo, hi;
        if (k < da)
            chunk_bits(a, na, k, h, lo, hi);
        else
            chunk_bits(b, nb, k - da, h, lo, hi);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const Shoup64 A{P[i], 0};
            red[i * red_stride + k] = A.add(A.mulw(hi, C.r64[i]), reduce_chunk(lo, P[i]));
        }
    }
}

// Integer matrices: entry e of A (na limbs) and of B (nb limbs) -> d chunks
// each, reduced modulo each prime.  red layout per prime: [A entries | B
// entries], d words per entry.
__global__ void k_split_mat(const uint32_t* __restrict__ a, long long na, const uint32_t* __restrict__ b,
                            long long nb, long long nn, long long d, uint64_t* __restrict__ red,
                            long long red_stride, CrtArgs C) {
    const long long total = 2 * nn * d;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long e = idx / d, k = idx - e * d;
        const uint64_t ch = (e < nn) ? chunk_of(a + e * na, na, k) : chunk_of(b + (e - nn) * nb, nb, k);
        red[idx] = reduce_chunk(ch, C.P1);
        red[red_stride + idx] = reduce_chunk(ch, C.P2);
        red[2 * red_stride + idx] = reduce_chunk(ch, C.P3);
    }
}

// Garner reconstruction of every product coefficient into three 64-bit words.
__global__ void k_crt(const uint64_t* __restrict__ r, long long r_stride, long long nc,
                      uint64_t* __restrict__ W, CrtArgs C) {
    const Shoup64 A2{C.P2, 0}, A3{C.P3, 0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nc;
         k += (long long)gridDim.x * blockDim.x) {
        const uint64_t r1 = r[k], r2 = r[r_stride + k], r3 = r[2 * r_stride + k];
        const uint64_t x1 = r1;                                   // < P1 < P2 < P3
        const uint64_t x2 = A2.mulw(A2.sub(r2, x1), C.inv12);
        const uint64_t x3 = A3.mulw(A3.sub(A3.mulw(A3.sub(r3, x1), C.inv13), x2), C.inv23);
        // c = x1 + P1 (x2 + P2 x3)
        const u128 t = static_cast<u128>(C.P2) * x3 + x2;        // < 2^125
        const uint64_t t0 = static_cast<uint64_t>(t), t1 = static_cast<uint64_t>(t >> 64);
        const u128 m0 = static_cast<u128>(C.P1) * t0 + x1;
        const u128 m1 = static_cast<u128>(C.P1) * t1 + static_cast<uint64_t>(m0 >> 64);
        W[3 * k] = static_cast<uint64_t>(m0);
        W[3 * k + 1] = static_cast<uint64_t>(m1);
        W[3 * k + 2] = static_cast<uint64_t>(m1 >> 64);
    }
}

// Bits [off, off + 64) of the 192-bit value c = (w0, w1, w2) (off may be
// negative: the slice then starts below c's first bit).
__device__ __forceinline__ uint64_t slice64(const uint64_t* w, long long off) {
    if (off <= -64 || off >= 192) return 0;
    if (off < 0) return w[0] << (-off);
    const int q = static_cast<int>(off >> 6), r = static_cast<int>(off & 63);
    const uint64_t a = w[q];
    const uint64_t b = (q + 1 < 3) ? w[q + 1] : 0;
    return r ? (a >> r) | (b << (64 - r)) : a;
}

// Word j of sum_k c_k 2^(h k) before carries: the 64-bit slices of the
// coefficients overlapping bits [64 j, 64 j + 64), as (low word, high part
// <= 3).  With h = 64 these are w0(c_j) + w1(c_{j-1}) + w2(c_{j-2}).
template <bool H64>
__device__ __forceinline__ void column_sum(const uint64_t* W, long long nc, long long j, int h, uint64_t& lo,
                                           uint64_t& hi) {
    u128 s = 0;
    if (H64) {                                      // word-aligned coefficients: three fixed terms
        if (j >= 0 && j < nc) s += W[3 * j];
        if (j - 1 >= 0 && j - 1 < nc) s += W[3 * (j - 1) + 1];
        if (j - 2 >= 0 && j - 2 < nc) s += W[3 * (j - 2) + 2];
    } else if (j >= 0) {
        const long long top = 64 * j + 63;
        long long k = (64 * j - 191 + h - 1) / h;   // first k with h k + 192 > 64 j
        if (64 * j - 191 <= 0) k = 0;
        const long long k1 = std::min(nc - 1, top / h);
        for (; k <= k1; ++k) s += slice64(W + 3 * k, 64 * j - h * k);
    }
    lo = static_cast<uint64_t>(s);
    hi = static_cast<uint64_t>(s >> 64);
}

// u_j = lo_j + hi_{j-1}: its low word v_j and its carry state.
template <bool H64>
__device__ __forceinline__ uint8_t word_state(const uint64_t* W, long long nc, long long j, int h, uint64_t& v) {
    uint64_t lo, hi, plo, phi;
    column_sum<H64>(W, nc, j, h, lo, hi);
    column_sum<H64>(W, nc, j - 1, h, plo, phi);
    const u128 u = static_cast<u128>(lo) + phi;
    v = static_cast<uint64_t>(u);
    if (u >> 64) return kGen;
    return (v == ~0ull) ? kProp : kKill;
}

__device__ __forceinline__ void store_word(uint32_t* c, long long nlimbs, long long j, uint64_t v) {
    if (2 * j < nlimbs) c[2 * j] = static_cast<uint32_t>(v);
    if (2 * j + 1 < nlimbs) c[2 * j + 1] = static_cast<uint32_t>(v >> 32);
}

// Pass 1: per word its carry-free value (stored into c) and its carry state
// relative to the start of its block (stored into st); per block the state
// of the whole block (agg).
template <bool H64>
__global__ void __launch_bounds__(kCarryThreads)
k_carry_local(const uint64_t* __restrict__ W, long long nc, long long nwords, int h, uint32_t* __restrict__ c,
              long long nlimbs, uint8_t* __restrict__ st, uint8_t* __restrict__ agg, long long nblocks) {
    __shared__ uint8_t warp_tot[kCarryThreads / 32];
    // entry blockIdx.y of a batch of integers laid out back to back
    W += blockIdx.y * 3 * nc;
    c += blockIdx.y * nlimbs;
    st += blockIdx.y * nwords;
    agg += blockIdx.y * nblocks;
    const long long j0 = static_cast<long long>(blockIdx.x) * kCarryBlock + threadIdx.x * kCarryPerThread;
    uint8_t s[kCarryPerThread];
    uint8_t tot = kProp;
    for (int e = 0; e < kCarryPerThread; ++e) {
        const long long j = j0 + e;
        uint64_t v = 0;
        s[e] = kKill;
        if (j < nwords) {
            s[e] = word_state<H64>(W, nc, j, h, v);
            store_word(c, nlimbs, j, v);
        }
        tot = carry_combine(tot, s[e]);
    }
    // exclusive scan of thread totals across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t incl = tot;
    for (int off = 1; off < 32; off <<= 1) {
        const uint8_t o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl = carry_combine(o, incl);
    }
    uint8_t excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = kProp;
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint8_t wpre = kProp;
    for (int w = 0; w < warp; ++w) wpre = carry_combine(wpre, warp_tot[w]);
    uint8_t pre = carry_combine(wpre, excl);
    for (int e = 0; e < kCarryPerThread; ++e) {
        const long long j = j0 + e;
        if (j < nwords) st[j] = pre;          // state of the words before j in this block
        pre = carry_combine(pre, s[e]);
    }
    if (threadIdx.x == kCarryThreads - 1) {
        uint8_t all = kProp;
        for (int w = 0; w < kCarryThreads / 32; ++w) all = carry_combine(all, warp_tot[w]);
        agg[blockIdx.x] = all;
    }
}

// Pass 2 (one block per entry): carry into each block, from the block states in order.
__global__ void k_carry_blocks(uint8_t* __restrict__ agg, long long nblocks) {
    __shared__ uint8_t part[1024];
    agg += blockIdx.x * nblocks;
    const int t = threadIdx.x;
    const long long per = (nblocks + blockDim.x - 1) / blockDim.x;
    const long long b0 = t * per, b1 = std::min(nblocks, b0 + per);
    uint8_t tot = kProp;
    for (long long b = b0; b < b1; ++b) tot = carry_combine(tot, agg[b]);
    part[t] = tot;
    __syncthreads();
    uint8_t pre = kProp;
    for (int u = 0; u < t; ++u) pre = carry_combine(pre, part[u]);
    for (long long b = b0; b < b1; ++b) {
        const uint8_t s = agg[b];
        agg[b] = (pre == kGen) ? 1 : 0;      // the carry into block b (no carry into word 0)
        pre = carry_combine(pre, s);
    }
}

// Pass 3: add the incoming carry of every word.
__global__ void __launch_bounds__(kCarryThreads)
k_carry_apply(long long nwords, uint32_t* __restrict__ c, long long nlimbs,
              const uint8_t* __restrict__ st, const uint8_t* __restrict__ blk_carry, long long nblocks) {
    c += blockIdx.y * nlimbs;
    st += blockIdx.y * nwords;
    blk_carry += blockIdx.y * nblocks;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nwords;
         j += (long long)gridDim.x * blockDim.x) {
        const uint8_t s = st[j];
        const uint32_t cin = (s == kGen) ? 1u : (s == kProp ? blk_carry[j / kCarryBlock] : 0u);
        if (!cin) continue;
        uint64_t v = (2 * j < nlimbs) ? c[2 * j] : 0u;
        if (2 * j + 1 < nlimbs) v |= static_cast<uint64_t>(c[2 * j + 1]) << 32;
        store_word(c, nlimbs, j, v + 1);
    }
}

int grid_of(long long n, int threads) {
    return static_cast<int>(std::max(1LL, std::min((n + threads - 1) / threads, 152LL * 16)));
}

struct Layout {
    int log2n, h;
    long long da, db, nc, nwords, nblocks;
    size_t off_red, off_res, off_W, off_st, off_agg, off_poly, poly_bytes, total;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int bit_length(long long m) {
    int b = 0;
    while (m > 0) ++b, m >>= 1;
    return b;
}

// Section 5.3's chunk size: the largest h (64 <= h <= 96) with
// 2 h + bitlength(min(da, db)) <= 183, da, db the chunk counts of a and b.
int chunk_bits_for(size_t na, size_t nb) {
    for (int h = 96; h > 64; --h) {
        const long long da = static_cast<long long>((32 * na + h - 1) / h);
        const long long db = static_cast<long long>((32 * nb + h - 1) / h);
        if (2 * h + bit_length(std::min(da, db)) <= 183) return h;
    }
    return 64;
}

Layout layout_of(const intmul_plan* P, size_t na, size_t nb) {
    Layout L{};
    L.h = chunk_bits_for(na, nb);
    L.da = static_cast<long long>((32 * na + L.h - 1) / L.h);
    L.db = static_cast<long long>((32 * nb + L.h - 1) / L.h);
    L.nc = L.da + L.db - 1;
    L.nwords = static_cast<long long>((na + nb + 1) / 2);
    L.nblocks = (L.nwords + kCarryBlock - 1) / kCarryBlock;
    int k = 1;
    while ((1LL << k) < L.nc) ++k;
    L.log2n = k;
    size_t off = 0;
    L.off_red = off;
    off = align256(off + 3 * static_cast<size_t>(L.da + L.db) * 8);
    L.off_res = off;
    off = align256(off + 3 * static_cast<size_t>(L.nc) * 8);
    L.off_W = off;
    off = align256(off + 3 * static_cast<size_t>(L.nc) * 8);
    L.off_st = off;
    off = align256(off + static_cast<size_t>(L.nwords));
    L.off_agg = off;
    off = align256(off + static_cast<size_t>(L.nblocks));
    L.off_poly = off;
    size_t poly = 0;
    if (k <= static_cast<int>(P->max_log2n) && P->plans[0][k])
        poly = align256(polymul_ws_bytes(P->plans[0][k], 1, NTT_SCHED_FUSED));
    L.poly_bytes = poly;
    L.total = align256(off + 3 * poly);                 // one product workspace per prime
    return L;
}

// Helper streams of an intmul plan: the three primes' products run
// concurrently, the second and third on two streams forked from the
// caller's stream (one pair per caller stream) and joined back by events.
struct Helpers {
    std::mutex mu;
    std::map<cudaStream_t, std::array<cudaStream_t, 2>> by_stream;
};

int helper_streams(const intmul_plan* P, cudaStream_t st, std::array<cudaStream_t, 2>& out) {
    Helpers* H = static_cast<Helpers*>(P->helpers);
    std::lock_guard<std::mutex> lock(H->mu);
    auto it = H->by_stream.find(st);
    if (it == H->by_stream.end()) {
        std::array<cudaStream_t, 2> s{};
        for (auto& x : s)
            if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) return NTT_ERR_CUDA;
        it = H->by_stream.emplace(st, s).first;
    }
    out = it->second;
    return NTT_OK;
}

}  // namespace
}  // namespace gbntt

using namespace gbntt;

extern "C" int intmul_plan_create(size_t max_limbs, intmul_plan** out) {
    if (!out || max_limbs == 0) return NTT_ERR_ARG;
    *out = nullptr;
    // product of two max_limbs operands: 2 ceil(max_limbs/2) - 1 coefficients
    const long long d = static_cast<long long>((max_limbs + 1) / 2);
    int kmax = 1;
    while ((1LL << kmax) < 2 * d - 1) ++kmax;
    if (kmax > 24) {
        gbntt_set_error("intmul_plan_create: operands above 2^24 64-bit chunks are not supported");
        return NTT_ERR_SIZE;
    }
    intmul_plan* P = new (std::nothrow) intmul_plan();
    if (!P) return NTT_ERR_OOM;
    cudaGetDevice(&P->device);
    P->max_log2n = static_cast<unsigned>(kmax);
    P->helpers = new (std::nothrow) Helpers();
    if (!P->helpers) {
        delete P;
        return NTT_ERR_OOM;
    }
    for (int i = 0; i < 3; ++i) {
        int rc = ntt_find_prime(62, 40, static_cast<unsigned>(i), &P->P[i]);
        if (rc != NTT_OK) {
            delete P;
            return rc;
        }
    }
    for (int i = 0; i < 3; ++i)
        for (int k = 1; k <= kmax; ++k) {
            int rc = ntt_plan_create(P->P[i], static_cast<unsigned>(k), 0, &P->plans[i][k]);
            if (rc != NTT_OK) {
                for (int a = 0; a < 3; ++a)
                    for (int b = 1; b <= kmax; ++b)
                        if (P->plans[a][b]) ntt_plan_destroy(P->plans[a][b]);
                delete static_cast<Helpers*>(P->helpers);
                delete P;
                return rc;
            }
        }
    auto inv = [](uint64_t a, uint64_t p) { return host::pow_mod(a % p, p - 2, p); };
    P->inv12 = host::tw64_of(inv(P->P[0], P->P[1]), P->P[1]);
    P->inv13 = host::tw64_of(inv(P->P[0], P->P[2]), P->P[2]);
    P->inv23 = host::tw64_of(inv(P->P[1], P->P[2]), P->P[2]);
    for (int i = 0; i < 3; ++i)
        P->r64[i] = host::tw64_of(static_cast<uint64_t>((static_cast<u128>(1) << 64) % P->P[i]), P->P[i]);
    *out = P;
    return NTT_OK;
}

extern "C" int intmul_plan_destroy(intmul_plan* plan) {
    if (!plan) return NTT_ERR_ARG;
    if (Helpers* H = static_cast<Helpers*>(plan->helpers)) {
        for (auto& kv : H->by_stream)
            for (cudaStream_t x : kv.second) {
                cudaStreamSynchronize(x);
                cudaStreamDestroy(x);
            }
        delete H;
    }
    for (int i = 0; i < 3; ++i)
        for (int k = 1; k <= 24; ++k)
            if (plan->plans[i][k]) ntt_plan_destroy(plan->plans[i][k]);
    delete plan;
    return NTT_OK;
}

extern "C" size_t intmul_workspace_size(const intmul_plan* plan, size_t na, size_t nb) {
    if (!plan || na == 0 || nb == 0) return 0;
    return layout_of(plan, na, nb).total;
}

extern "C" int intmul_crt(const intmul_plan* plan, const uint32_t* d_a, size_t na, const uint32_t* d_b,
                          size_t nb, uint32_t* d_c, void* d_ws, size_t ws_bytes, void* stream) {
    if (!plan || !d_a || !d_b || !d_c || na == 0 || nb == 0) return NTT_ERR_ARG;
    const Layout L = layout_of(plan, na, nb);
    if (L.log2n > static_cast<int>(plan->max_log2n)) {
        gbntt_set_error("intmul_crt: operands larger than the plan was created for");
        return NTT_ERR_SIZE;
    }
    if (!d_ws || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(d_ws) & 255)) {
        gbntt_set_error("intmul_crt: workspace of " + std::to_string(L.total) +
                        " bytes (256-byte aligned) required");
        return NTT_ERR_WORKSPACE;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(d_ws);
    uint64_t* red = reinterpret_cast<uint64_t*>(ws + L.off_red);
    uint64_t* res = reinterpret_cast<uint64_t*>(ws + L.off_res);
    uint64_t* W = reinterpret_cast<uint64_t*>(ws + L.off_W);
    uint8_t* sst = ws + L.off_st;
    uint8_t* agg = ws + L.off_agg;
    uint64_t* poly = reinterpret_cast<uint64_t*>(ws + L.off_poly);
    CrtArgs C{plan->P[0], plan->P[1], plan->P[2], plan->inv12, plan->inv13, plan->inv23,
              {plan->r64[0], plan->r64[1], plan->r64[2]}};
    const long long red_stride = L.da + L.db;

    prof_begin_call(st);
    k_split<<<grid_of(red_stride, 256), 256, 0, st>>>(d_a, static_cast<long long>(na), d_b,
                                                       static_cast<long long>(nb), L.da, L.db, L.h, red,
                                                       red_stride, C);
    prof_mark(st, "k_split");
    // the three residue products concurrently: prime 1 on the caller's
    // stream, primes 2 and 3 on its helper streams
    std::array<cudaStream_t, 2> hs{};
    int rc = helper_streams(plan, st, hs);
    if (rc != NTT_OK) return rc;
    cudaEvent_t ev[3];
    for (auto& e : ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return NTT_ERR_CUDA;
    cudaEventRecord(ev[0], st);
    const cudaStream_t sp[3] = {st, hs[0], hs[1]};
    for (int i = 0; i < 3; ++i) {
        if (i) cudaStreamWaitEvent(sp[i], ev[0], 0);
        const ntt_plan* np = plan->plans[i][L.log2n];
        rc = launch_polymul_fused<Shoup64L>(np, np->dp64, red + i * red_stride, L.da, red + i * red_stride + L.da,
                                            L.db, 1, res + i * L.nc,
                                            reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(poly) +
                                                                        i * L.poly_bytes),
                                            np->pm_scale64, sp[i]);
        if (rc != NTT_OK) break;
        if (i) {
            cudaEventRecord(ev[i], sp[i]);
            cudaStreamWaitEvent(st, ev[i], 0);
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (rc != NTT_OK) return rc;
    k_crt<<<grid_of(L.nc, 256), 256, 0, st>>>(res, L.nc, L.nc, W, C);
    prof_mark(st, "k_crt");
    (L.h == 64 ? k_carry_local<true> : k_carry_local<false>)<<<static_cast<unsigned>(L.nblocks), kCarryThreads, 0, st>>>(
        W, L.nc, L.nwords, L.h, d_c, static_cast<long long>(na + nb), sst, agg, L.nblocks);
    prof_mark(st, "k_carry_local");
    k_carry_blocks<<<1, 1024, 0, st>>>(agg, L.nblocks);
    prof_mark(st, "k_carry_blocks");
    k_carry_apply<<<grid_of(L.nwords, kCarryThreads), kCarryThreads, 0, st>>>(
        L.nwords, d_c, static_cast<long long>(na + nb), sst, agg, L.nblocks);
    prof_mark(st, "k_carry_apply");
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        gbntt_set_error(std::string("intmul_crt: ") + cudaGetErrorString(e));
        return NTT_ERR_CUDA;
    }
    return NTT_OK;
}

// ---------------------------------------------------------------- integer matrices

namespace {

struct MatLayout {
    int log2n;
    long long nn, d, nc, nwords, nblocks;
    size_t off_red, off_res, off_W, off_st, off_agg, off_poly, total;
};

MatLayout mat_layout_of(const intmul_plan* P, unsigned n, size_t na, size_t nb) {
    MatLayout L{};
    L.nn = static_cast<long long>(n) * n;
    L.d = static_cast<long long>(std::max((na + 1) / 2, (nb + 1) / 2));
    L.nc = 2 * L.d - 1;
    // a sum of n < 2^32 products of 2d-chunk operands: 2d words plus one
    // word for the sum's top, which also receives the third CRT word of the
    // highest coefficient
    L.nwords = 2 * L.d + 1;
    L.nblocks = (L.nwords + kCarryBlock - 1) / kCarryBlock;
    int k = 1;
    while ((1LL << k) < L.nc) ++k;
    L.log2n = k;
    size_t off = 0;
    L.off_red = off;
    off = align256(off + 3 * static_cast<size_t>(2 * L.nn * L.d) * 8);
    L.off_res = off;
    off = align256(off + 3 * static_cast<size_t>(L.nn * L.nc) * 8);
    L.off_W = off;
    off = align256(off + 3 * static_cast<size_t>(L.nn * L.nc) * 8);
    L.off_st = off;
    off = align256(off + static_cast<size_t>(L.nn * L.nwords));
    L.off_agg = off;
    off = align256(off + static_cast<size_t>(L.nn * L.nblocks));
    L.off_poly = off;
    L.total = align256(off + 3 * static_cast<size_t>(L.nn) * (size_t(1) << k) * 8);
    (void)P;
    return L;
}

}  // namespace

extern "C" size_t intmat_workspace_size(const intmul_plan* plan, unsigned n, size_t na, size_t nb) {
    if (!plan || n == 0 || na == 0 || nb == 0) return 0;
    return mat_layout_of(plan, n, na, nb).total;
}

extern "C" int intmat_mul(const intmul_plan* plan, const uint32_t* d_A, size_t na, const uint32_t* d_B,
                          size_t nb, unsigned n, uint32_t* d_C, void* d_ws, size_t ws_bytes, void* stream) {
    if (!plan || !d_A || !d_B || !d_C || n == 0 || n > 255 || na == 0 || nb == 0) return NTT_ERR_ARG;
    const MatLayout L = mat_layout_of(plan, n, na, nb);
    if (L.log2n > static_cast<int>(plan->max_log2n)) {
        gbntt_set_error("intmat_mul: entries larger than the plan was created for");
        return NTT_ERR_SIZE;
    }
    // every coefficient of C is a sum of n d products below 2^128
    if (static_cast<double>(n) * static_cast<double>(L.d) >= 3.6e16) return NTT_ERR_SIZE;
    if (!d_ws || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(d_ws) & 255)) {
        gbntt_set_error("intmat_mul: workspace of " + std::to_string(L.total) +
                        " bytes (256-byte aligned) required");
        return NTT_ERR_WORKSPACE;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(d_ws);
    uint64_t* red = reinterpret_cast<uint64_t*>(ws + L.off_red);
    uint64_t* res = reinterpret_cast<uint64_t*>(ws + L.off_res);
    uint64_t* W = reinterpret_cast<uint64_t*>(ws + L.off_W);
    uint8_t* sst = ws + L.off_st;
    uint8_t* agg = ws + L.off_agg;
    uint64_t* poly = reinterpret_cast<uint64_t*>(ws + L.off_poly);
    CrtArgs C{plan->P[0], plan->P[1], plan->P[2], plan->inv12, plan->inv13, plan->inv23,
              {plan->r64[0], plan->r64[1], plan->r64[2]}};
    const long long red_stride = 2 * L.nn * L.d;
    const long long nlimbs = static_cast<long long>(na + nb + 1);
    prof_begin_call(st);
    k_split_mat<<<grid_of(red_stride, 256), 256, 0, st>>>(d_A, static_cast<long long>(na), d_B,
                                                          static_cast<long long>(nb), L.nn, L.d, red,
                                                          red_stride, C);
    prof_mark(st, "k_split_mat");
    for (int i = 0; i < 3; ++i) {
        const ntt_plan* np = plan->plans[i][L.log2n];
        const uint64_t* Ai = red + i * red_stride;
        int rc = launch_polymat<Shoup64L>(np, np->dp64, Ai, Ai + L.nn * L.d, static_cast<int>(n), L.d,
                                          res + i * L.nn * L.nc, poly, np->inv_scale64, np->r64, st);
        if (rc != NTT_OK) return rc;
    }
    k_crt<<<grid_of(L.nn * L.nc, 256), 256, 0, st>>>(res, L.nn * L.nc, L.nn * L.nc, W, C);
    prof_mark(st, "k_crt");
    const unsigned ny = static_cast<unsigned>(L.nn);
    k_carry_local<true><<<dim3(static_cast<unsigned>(L.nblocks), ny), kCarryThreads, 0, st>>>(
        W, L.nc, L.nwords, 64, d_C, nlimbs, sst, agg, L.nblocks);
    prof_mark(st, "k_carry_local");
    k_carry_blocks<<<ny, 1024, 0, st>>>(agg, L.nblocks);
    prof_mark(st, "k_carry_blocks");
    k_carry_apply<<<dim3(static_cast<unsigned>(std::min<long long>(L.nblocks * 4, 4096)), ny), kCarryThreads, 0, st>>>(
        L.nwords, d_C, nlimbs, sst, agg, L.nblocks);
    prof_mark(st, "k_carry_apply");
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        gbntt_set_error(std::string("intmat_mul: ") + cudaGetErrorString(e));
        return NTT_ERR_CUDA;
    }
    return NTT_OK;
}
