// Products of n = 4096 points on one thread-block cluster (single-product
// latency).
//
// One block working alone on a 4096-point product spends most of its time in
// the dependency chains of its passes: three transforms of 12 stages on one
// SM.  Here the eight CTAs of a cluster (eight SMs) share each product,
// exchanging data through distributed shared memory.  The transform is
// Algorithm 1 (Section 5.1) with n = 64 x 64 rows x columns,
// element (r, c) = a[64 r + c]:
//   column phase  the 64-point transform of every column along r, then the
//                 twiddle w_4096^(c [pos]_6) (the plan's 64 x 64 tile table);
//   row phase     the 64-point transform of every row along c.
// Each 64-point transform is itself Algorithm 1 split 8 x 8 in registers:
// a thread owns column j1 of the split, runs an 8-point DIF down it, applies
// w_64^(j1 [t]_3), and the rows of the split are the second pass.  Position
// p of a transformed line then holds frequency [p]_6, as in the engine.
//
// CTA q of the cluster owns columns 8q .. 8q+7 in the column phase and rows
// (positions) 8q .. 8q+7 in the row phase; a row's 64 words live in all
// eight CTAs after the column phase and are pulled from their shared memory
// once a cluster barrier has made them visible.  The row phase also does the
// pointwise product and the first inverse passes; the inverse column phase
// pulls the product's columns back the same way, and the last pass scales by
// n^-1 (times the Montgomery factor) and stores.  Three cluster barriers in
// all; the last one only keeps a CTA's shared memory alive until every other
// CTA has read it.
#pragma once
#include <cooperative_groups.h>

#include "engine.cuh"

namespace gbntt {

constexpr int kClLog = 12;        // n = 2^12 = 64 x 64
constexpr int kClCtas = 8;        // CTAs per cluster, one cluster per product
constexpr int kClThreads = 128;   // 2 operands x 8 lines x 8 split columns
constexpr int kClMaxBatch = 16;   // larger batches take the one-block kernel (throughput)
constexpr int kClS = 9;           // words per position in the column buffers (8 columns + pad)
constexpr int kClR = 65;          // words per row in the row buffers (64 + pad)

__host__ __device__ constexpr size_t cluster_smem_words() {
    return size_t(2) * 64 * kClS + size_t(2) * 8 * kClR + size_t(8) * kClR + size_t(64) * kClS;
}

// Arrival without a release fence: used only to say "this CTA reads no other
// CTA's shared memory any more".  Every remote load a thread made before it
// has returned (its value was consumed by the stores that precede the
// arrival), and the CTA's later writes are read by no other CTA, so there is
// nothing to order.
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// One product per cluster: a (na words) and b (nb words) of product
// blockIdx.x / 8, c (na + nb - 1 words) out.  ZHALF: na, nb <= 2048, so rows
// r >= 32 are zero.  `ar` is the arithmetic policy, `scale` = n^-1 times the
// Montgomery factor of the pointwise product, in multiplicand form.
template <class Ar, bool ZHALF>
__global__ void __cluster_dims__(kClCtas, 1, 1) __launch_bounds__(kClThreads)
k_cluster_polymul(DevPlan<Ar> P, const typename WideForm<Ar>::type ar, const typename Ar::word* __restrict__ a,
                  long long na, const typename Ar::word* __restrict__ b, long long nb,
                  typename Ar::word* __restrict__ c, typename Ar::tw scale) {
    namespace cg = cooperative_groups;
    using Ax = typename WideForm<Ar>::type;
    using word = typename Ar::word;
    using tw = typename Ar::tw;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smraw[];
    word* S = reinterpret_cast<word*>(smraw);   // [op][pos * kClS + cl]: column phase, read by the cluster
    word* R = S + 2 * 64 * kClS;                 // [op][rl * kClR + k]: row phase, local
    word* U = R + 2 * 8 * kClR;                  // [rl * kClR + col]: inverse rows, read by the cluster
    word* S2 = U + 8 * kClR;                     // [pos * kClS + cl]: inverse column phase, local
    const int q = static_cast<int>(cluster.block_rank());
    const long long prod = blockIdx.x / kClCtas;
    const int op = threadIdx.x >> 6, lo = threadIdx.x & 7, hi = (threadIdx.x >> 3) & 7;
    const tw* l64f = P.line64x8[0];
    const tw* l64i = P.line64x8[1];
    const tw* tf = P.tile_fwd[kClLog];
    const tw* ti = P.tile_inv[kClLog];
    // Every twiddle a thread will use, loaded up front with 32-bit words so
    // that the table latencies overlap the operand loads instead of following
    // one another phase by phase (a thread's (lo, hi) is its (column, split
    // column) or (column, block) in every pass).  64-bit words load them
    // where they are used (register budget).
    constexpr bool kPre = sizeof(word) == 4;
    tw wf[8], wi[8], gf[8], gi[8];
    if constexpr (kPre) {
        const int col = 8 * q + lo;
#pragma unroll
        for (int t = 1; t < 8; ++t) wf[t] = l64f[hi * 8 + t];
#pragma unroll
        for (int u = 0; u < 8; ++u) gf[u] = tf[(8 * hi + u) * 64 + col];
        if (op == 0) {
#pragma unroll
            for (int t = 1; t < 8; ++t) wi[t] = l64i[hi * 8 + t];
#pragma unroll
            for (int u = 0; u < 8; ++u) gi[u] = ti[(8 * hi + u) * 64 + col];
        }
    }
    auto line_f = [&](int j1, int t) { if constexpr (kPre) return wf[t]; else return l64f[j1 * 8 + t]; };
    auto line_i = [&](int j1, int t) { if constexpr (kPre) return wi[t]; else return l64i[j1 * 8 + t]; };
    auto glob_f = [&](int pos, int col, int u) { if constexpr (kPre) return gf[u]; else return tf[pos * 64 + col]; };
    auto glob_i = [&](int pos, int col, int u) { if constexpr (kPre) return gi[u]; else return ti[pos * 64 + col]; };

    // column phase, first pass: thread (op, column 8q + lo, split column hi)
    {
        const int cl = lo, j1 = hi;
        const long long col = 8 * q + cl;
        const word* in = op ? b + prod * nb : a + prod * na;
        const long long len = op ? nb : na;
        word x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const long long idx = 64LL * (8 * t + j1) + col;
            x[t] = word(0);
            if ((!ZHALF || t < 4) && idx < len) x[t] = in[idx];
        }
        dif_regs<Ax, 8, ZHALF>(ar, x, P.rc);
#pragma unroll
        for (int t = 1; t < 8; ++t) x[t] = ar.mulw(x[t], line_f(j1, t));
        word* s = S + op * 64 * kClS;
#pragma unroll
        for (int t = 0; t < 8; ++t) s[(8 * t + j1) * kClS + cl] = x[t];
    }
    __syncthreads();
    // column phase, second pass and the 64 x 64 twiddle: thread (op, lo, block hi)
    {
        const int cl = lo, tp = hi;
        const int col = 8 * q + cl;
        word* s = S + op * 64 * kClS;
        word x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = s[(8 * tp + u) * kClS + cl];
        dif_regs<Ax, 8>(ar, x, P.rc);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int pos = 8 * tp + u;
            s[pos * kClS + cl] = ar.mulw(x[u], glob_f(pos, col, u));
        }
    }
    cluster.sync();
    // row phase, first pass: thread (op, row 8q + lo, split column hi); word
    // 8 t + j1 of the row sits in CTA t
    {
        const int rl = lo, j1 = hi;
        const int pos = 8 * q + rl;
        word x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const word* rs = cluster.map_shared_rank(S, t);
            x[t] = rs[op * 64 * kClS + pos * kClS + j1];
        }
        dif_regs<Ax, 8>(ar, x, P.rc);
#pragma unroll
        for (int t = 1; t < 8; ++t) x[t] = ar.mulw(x[t], line_f(j1, t));
        word* rr = R + (op * 8 + rl) * kClR;
#pragma unroll
        for (int t = 0; t < 8; ++t) rr[8 * t + j1] = x[t];
    }
    __syncthreads();
    // row phase, second pass of both operands, pointwise product, its inverse:
    // thread (row lo, block hi)
    if (op == 0) {
        word* ra = R + lo * kClR + 8 * hi;
        word* rb = R + (8 + lo) * kClR + 8 * hi;
        word xa[8], xb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            xa[u] = ra[u];
            xb[u] = rb[u];
        }
        dif_regs<Ax, 8>(ar, xa, P.rc);
        dif_regs<Ax, 8>(ar, xb, P.rc);
#pragma unroll
        for (int u = 0; u < 8; ++u) xa[u] = ar.mulmont(xa[u], xb[u]);
        dit_regs<Ax, 8>(ar, xa, P.rci);
#pragma unroll
        for (int u = 0; u < 8; ++u) ra[u] = xa[u];
    }
    __syncthreads();
    // inverse of the row phase's first pass: thread (row lo, split column hi)
    if (op == 0) {
        const int rl = lo, j1 = hi;
        const word* ra = R + rl * kClR;
        word x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) x[t] = ra[8 * t + j1];
#pragma unroll
        for (int t = 1; t < 8; ++t) x[t] = ar.mulw(x[t], line_i(j1, t));
        dit_regs<Ax, 8>(ar, x, P.rci);
#pragma unroll
        for (int t = 0; t < 8; ++t) U[rl * kClR + 8 * t + j1] = x[t];
    }
    cluster.sync();
    // inverse column phase, its second pass first: thread (column 8q + lo,
    // block hi); positions 8 hi .. 8 hi + 7 sit in CTA hi
    if (op == 0) {
        const int cl = lo, tp = hi;
        const int col = 8 * q + cl;
        const word* ru = cluster.map_shared_rank(U, tp);
        word x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int pos = 8 * tp + u;
            x[u] = ar.mulw(ru[u * kClR + col], glob_i(pos, col, u));
        }
        dit_regs<Ax, 8>(ar, x, P.rci);
#pragma unroll
        for (int u = 0; u < 8; ++u) S2[(8 * tp + u) * kClS + cl] = x[u];
    }
    cluster_arrive_relaxed();          // this CTA reads no other CTA's memory from here on
    __syncthreads();
    // inverse of the column phase's first pass, scaled store: thread
    // (column 8q + lo, split column hi)
    if (op == 0) {
        const int cl = lo, j1 = hi;
        const long long col = 8 * q + cl;
        const long long nc = na + nb - 1;
        word x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) x[t] = S2[(8 * t + j1) * kClS + cl];
#pragma unroll
        for (int t = 1; t < 8; ++t) x[t] = ar.mulw(x[t], line_i(j1, t));
        dit_regs<Ax, 8>(ar, x, P.rci);
        word* out = c + prod * nc;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const long long idx = 64LL * (8 * t + j1) + col;
            if (idx < nc) out[idx] = ar.canon(ar.mulw(x[t], scale));
        }
    }
    cluster_wait_acquire();            // keep this CTA's shared memory until the cluster has read it
}

}  // namespace gbntt
