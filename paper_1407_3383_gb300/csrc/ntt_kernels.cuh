// Transform and polynomial-product kernels (sm_103a) and their launchers.
//
// Fused schedule (the library's default):
//   n <= 2^tile_max_log : one thread block per product (several for short
//       vectors); load with zero padding, two forward transforms, pointwise
//       product, inverse transform and scaled store, all in shared memory.
//   larger n : Algorithm 1 once more at the global level, n = n2 x n1
//       (n2 = 2^floor(k/2) rows of n1 words):
//       pass 1  columns: load (zero padded) n2 x w slabs, transform each
//               column, apply the step-2 twiddle w_n^(j1 [j2]), write;
//       pass 2  rows: transform rows of both operands, multiply them
//               pointwise, inverse-transform the product rows, write;
//       pass 3  columns: inverse twiddle, inverse column transforms, scale
//               by n^-1 (and the Montgomery factor), crop, store.
//   Operand traffic: read a, b once; write c once; the transformed operands
//   make one round trip through the caller's workspace.
//
// Plain schedule (the baseline the fused one is measured against): one
// launch per radix-2 stage over global memory.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <string>

#include "../../include/gbntt.h"
#include "cluster.cuh"
#include "direct.cuh"
#include "subvec.cuh"
#include "kernels.h"
#include "plan.h"

namespace gbntt {

constexpr int kThreads = 256;
// shared memory above which a one-block product leaves room for one block per SM
constexpr size_t kTileWideSmem = 114 * 1024;

// Multiprocessor count of a device, queried once per device (every caller
// writes the same value, so concurrent first calls are harmless).
inline int sm_count(int device) {
    static int cache[64] = {};
    if (device < 0 || device >= 64) return 1;
    if (!cache[device]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 1;
        }
        cache[device] = n;
    }
    return cache[device];
}

__host__ __device__ inline VecLayout tile_layout(int logL, int lognvec) {
    VecLayout L{};
    L.logL = logL;
    L.lognvec = lognvec;
    if (logL <= kMaxLineLog) {
        L.CS = 1;
        L.RS = 0;
        L.VS = (1 << logL) + 1;
        L.vfast = true;
    } else {
        const int L1 = 1 << tile_l1(logL), L2 = 1 << tile_l2(logL);
        L.CS = 1;
        L.RS = L1 + 1;
        L.VS = L2 * L.RS;
        L.vfast = false;
    }
    return L;
}

__host__ __device__ inline long long layout_words(const VecLayout& L) {
    return (1LL << L.lognvec) * static_cast<long long>(L.VS);
}

// w columns (vectors) of length 2^logL, element i of column v at v + i*(w+1)
// (with one extra word per tile row when the column is itself a tile).
__host__ __device__ inline VecLayout slab_layout(int logL, int logw) {
    VecLayout L{};
    const int w = 1 << logw;
    L.logL = logL;
    L.lognvec = logw;
    L.VS = 1;
    L.CS = w + 1;
    L.vfast = true;
    if (logL > kMaxLineLog) L.RS = (1 << tile_l1(logL)) * (w + 1) + 1;
    return L;
}

__host__ __device__ inline long long slab_words(const VecLayout& L) {
    if (L.logL <= kMaxLineLog) return (1LL << L.logL) * static_cast<long long>(L.CS);
    return (1LL << tile_l2(L.logL)) * static_cast<long long>(L.RS);
}

// ------------------------------------------------------------------ fused kernels

// One block per product group, the whole product in shared memory.  NT
// threads: tiles that leave room for one block per SM run 512 threads, so
// that an SM holds 16 warps instead of 8; grids smaller than the GPU (a few
// products, where each block has an SM to itself) run 1024 threads with
// 32-bit words and 512 with 64-bit words.  TFT: the transforms are
// truncated to the kb of 16 blocks of 2^logL/16 positions that the
// na + nb - 1 output words need (Section 5.1; logL >= 5).
template <class Ar, int NT = kThreads, bool TFT = false>
__global__ void __launch_bounds__(NT)
k_tile_polymul(DevPlan<Ar> P, const typename Ar::word* __restrict__ a, long long na,
               const typename Ar::word* __restrict__ b, long long nb,
               typename Ar::word* __restrict__ c, long long batch, int logL, int lppc,
               typename Ar::tw scale, int kb, TftConsts<Ar> K) {
    using word = typename Ar::word;
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    const int ppc = 1 << lppc;
    const long long prod0 = static_cast<long long>(blockIdx.x) << lppc;
    const long long L = 1LL << logL;
    const VecLayout LA = tile_layout(logL, lppc + 1);
    for (long long idx = threadIdx.x; idx < (L << lppc); idx += blockDim.x) {
        const int v = static_cast<int>(idx >> logL);
        const long long i = idx & (L - 1);
        const long long prod = prod0 + v;
        word xa = 0, xb = 0;
        if (prod < batch) {
            if (i < na) xa = a[prod * na + i];
            if (i < nb) xb = b[prod * nb + i];
        }
        sm[vec_addr(LA, v, static_cast<int>(i))] = xa;
        sm[vec_addr(LA, v + ppc, static_cast<int>(i))] = xb;
    }
    __syncthreads();
    if (TFT)
        vec_fwd_t<Ar>(P, sm, LA, kb, K);
    else
        vec_fwd<Ar>(P, sm, LA, nullptr);
    const long long Lk = TFT ? (static_cast<long long>(kb) << (logL - 4)) : L;   // positions kept
    for (long long idx = threadIdx.x; idx < (L << lppc); idx += blockDim.x) {
        const int v = static_cast<int>(idx >> logL);
        const long long i = idx & (L - 1);
        if (TFT && i >= Lk) continue;
        const long long pa = vec_addr(LA, v, static_cast<int>(i)), pb = vec_addr(LA, v + ppc, static_cast<int>(i));
        sm[pa] = P.ar.mulmont(sm[pa], sm[pb]);
    }
    __syncthreads();
    const VecLayout LC = tile_layout(logL, lppc);
    if (TFT)
        vec_inv_t<Ar>(P, sm, LC, kb, K);
    else
        vec_inv<Ar>(P, sm, LC, nullptr);
    const long long nc = na + nb - 1;
    for (long long idx = threadIdx.x; idx < (nc << lppc); idx += blockDim.x) {
        const int v = static_cast<int>(idx / nc);
        const long long i = idx - v * nc;
        const long long prod = prod0 + v;
        if (prod < batch) c[prod * nc + i] = P.ar.canon(P.ar.mulw(sm[vec_addr(LC, v, static_cast<int>(i))], scale));
    }
}

template <class Ar, bool FWD>
__global__ void __launch_bounds__(kThreads)
k_tile_ntt(DevPlan<Ar> P, typename Ar::word* __restrict__ data, long long batch, int logL,
           int lppc, typename Ar::tw scale) {
    using word = typename Ar::word;
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    const long long prod0 = static_cast<long long>(blockIdx.x) << lppc;
    const long long L = 1LL << logL;
    const VecLayout LA = tile_layout(logL, lppc);
    for (long long idx = threadIdx.x; idx < (L << lppc); idx += blockDim.x) {
        const int v = static_cast<int>(idx >> logL);
        const long long i = idx & (L - 1);
        const long long prod = prod0 + v;
        sm[vec_addr(LA, v, static_cast<int>(i))] = (prod < batch) ? data[prod * L + i] : word(0);
    }
    __syncthreads();
    if (FWD)
        vec_fwd<Ar>(P, sm, LA, nullptr);
    else
        vec_inv<Ar>(P, sm, LA, nullptr);
    for (long long idx = threadIdx.x; idx < (L << lppc); idx += blockDim.x) {
        const int v = static_cast<int>(idx >> logL);
        const long long i = idx & (L - 1);
        const long long prod = prod0 + v;
        if (prod < batch) {
            word x = sm[vec_addr(LA, v, static_cast<int>(i))];
            data[prod * L + i] = P.ar.canon(FWD ? x : P.ar.mulw(x, scale));
        }
    }
}

// Pass 1: forward column transforms of a slab of w columns, then the
// global twiddle.  blockIdx.z selects operand 0 or 1 (src0/src1).  Uniform
// batches read product t at src + t*len; uneven batches (desc != null) at
// the descriptor's offsets and lengths.  ZHALF: every operand has at most
// n/2 words, so the upper half of every column is zero padding.
// KN nonzero: n = 2^KN and the block shape are fixed at compile time (the
// runtime arguments must agree), so the index arithmetic of every pass
// folds away.  TFT (k2 = 4 .. 8): only the rows of the kb column blocks
// that the product's output needs are formed and stored (kb given for
// uniform batches, from the descriptor's lengths for uneven ones).
template <class Ar, bool ZHALF, int KN = 0, int LOGW = 0, bool TFT = false>
__global__ void __launch_bounds__(kThreads)
k_col_fwd(DevPlan<Ar> P, const typename Ar::word* src0, long long len0,
          const typename Ar::word* src1, long long len1, typename Ar::word* dst,
          long long dst_stride, long long dst_off1, int logN, int k2, int logw, long long prod_base,
          const BatchDesc* __restrict__ desc, int kb) {
    using word = typename Ar::word;
    if (KN) {
        logN = KN;
        k2 = KN / 2;
        logw = LOGW;
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    const int k1 = logN - k2;
    const long long n1 = 1LL << k1;
    const int w = 1 << logw;
    const long long c0 = static_cast<long long>(blockIdx.x) << logw;
    const long long prod = prod_base + blockIdx.y;
    const word* src;
    long long len;
    if (desc) {
        const BatchDesc d = desc[prod];
        src = blockIdx.z ? src1 + d.boff : src0 + d.aoff;
        len = blockIdx.z ? d.nb : d.na;
        if (TFT) kb = tft_kb(static_cast<long long>(d.na) + d.nb - 1, logN);
    } else {
        len = blockIdx.z ? len1 : len0;
        src = (blockIdx.z ? src1 : src0) + prod * len;
    }
    word* out = dst + prod * dst_stride + (blockIdx.z ? dst_off1 : 0);
    const VecLayout L = slab_layout(k2, logw);
    const long long total = (1LL << k2) << logw;
    for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const long long row = idx >> logw;
        const int col = static_cast<int>(idx & (w - 1));
        const long long e = row * n1 + c0 + col;
        sm[vec_addr(L, col, static_cast<int>(row))] = (e < len) ? src[e] : word(0);
    }
    __syncthreads();
    Hook<Ar> h{P.glob_fwd, static_cast<int>(n1), 0, 1, static_cast<int>(c0)};
    if (TFT) {
        PhaseGeom g{k2, logw, 0, L.VS, 0, L.CS, true};
        phase_fwd_t<Ar, ZHALF>(P, sm, g, &h, kb, TftConsts<Ar>{});   // the forward TFT needs no constants
        const long long kept = (static_cast<long long>(kb) << (k2 - 4)) << logw;
        for (long long idx = threadIdx.x; idx < kept; idx += blockDim.x) {
            const long long row = idx >> logw;
            const int col = static_cast<int>(idx & (w - 1));
            out[row * n1 + c0 + col] = sm[vec_addr(L, col, static_cast<int>(row))];
        }
        return;
    }
    vec_fwd<Ar, ZHALF>(P, sm, L, &h);        // ZHALF: the upper half of every column is padding
    for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const long long row = idx >> logw;
        const int col = static_cast<int>(idx & (w - 1));
        out[row * n1 + c0 + col] = sm[vec_addr(L, col, static_cast<int>(row))];
    }
}

// Pass 3: inverse twiddle and inverse column transforms, scaled, cropped
// store of the first out_len words of each product.  TFT (k2 = 4 .. 8):
// only the rows of the kb kept column blocks are read; each column's outer
// 16-point pass is solved by the inverse TFT with the zero rows above.
template <class Ar, int KN = 0, int LOGW = 0, bool TFT = false>
__global__ void __launch_bounds__(kThreads)
k_col_inv(DevPlan<Ar> P, const typename Ar::word* src, long long src_stride,
          typename Ar::word* dst, long long out_len, int logN, int k2, int logw,
          const typename Ar::tw* __restrict__ itab, long long prod_base,
          const BatchDesc* __restrict__ desc, int kb, TftConsts<Ar> K) {
    using word = typename Ar::word;
    if (KN) {
        logN = KN;
        k2 = KN / 2;
        logw = LOGW;
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    const int k1 = logN - k2;
    const long long n1 = 1LL << k1;
    const int w = 1 << logw;
    const long long c0 = static_cast<long long>(blockIdx.x) << logw;
    const long long prod = prod_base + blockIdx.y;
    const word* in = src + prod * src_stride;
    word* outp;
    if (desc) {
        const BatchDesc d = desc[prod];
        outp = dst + d.coff;
        out_len = static_cast<long long>(d.na) + d.nb - 1;
    } else {
        outp = dst + prod * out_len;
    }
    if (TFT) kb = tft_kb(out_len, logN);
    const VecLayout L = slab_layout(k2, logw);
    const long long total = (1LL << k2) << logw;
    const long long loaded = TFT ? (static_cast<long long>(kb) << (k2 - 4)) << logw : total;
    for (long long idx = threadIdx.x; idx < loaded; idx += blockDim.x) {
        const long long row = idx >> logw;
        const int col = static_cast<int>(idx & (w - 1));
        sm[vec_addr(L, col, static_cast<int>(row))] = in[row * n1 + c0 + col];
    }
    __syncthreads();
    // itab = inverse step-2 twiddles with the final scaling folded in
    Hook<Ar> h{itab, static_cast<int>(n1), 0, 1, static_cast<int>(c0)};
    if (TFT) {
        PhaseGeom g{k2, logw, 0, L.VS, 0, L.CS, true};
        phase_inv_t<Ar>(P, sm, g, &h, kb, K);
    } else {
        vec_inv<Ar>(P, sm, L, &h);
    }
    for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const long long row = idx >> logw;
        const int col = static_cast<int>(idx & (w - 1));
        const long long e = row * n1 + c0 + col;
        if (e < out_len) outp[e] = P.ar.canon(sm[vec_addr(L, col, static_cast<int>(row))]);
    }
}

// Pass 2 of the product: rows of both transformed operands -> forward row
// transforms, pointwise product, inverse row transforms of the product.
// ws per product: [0, n) operand a, [n, 2n) operand b; result over a.
// TFT: blocks whose rows all lie past the kb kept column blocks of their
// product (kb given, or from the descriptor's lengths) return at once.
template <class Ar, int KN = 0, int LRPC = 0, bool TFT = false>
__global__ void __launch_bounds__(kThreads)
k_row_polymul(DevPlan<Ar> P, typename Ar::word* ws, long long ws_stride, int logN, int k2,
              int lrpc, long long prod_base, const BatchDesc* __restrict__ desc, int kb) {
    using word = typename Ar::word;
    if (KN) {
        logN = KN;
        k2 = KN / 2;
        lrpc = LRPC;
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    const int k1 = logN - k2;
    const long long n1 = 1LL << k1, N = 1LL << logN;
    const int rpc = 1 << lrpc;
    const long long r0 = static_cast<long long>(blockIdx.x) << lrpc;
    if (TFT) {
        if (desc) {
            const BatchDesc d = desc[prod_base + blockIdx.y];
            kb = tft_kb(static_cast<long long>(d.na) + d.nb - 1, logN);
        }
        if (r0 >= (static_cast<long long>(kb) << (k2 - 4))) return;
    }
    word* base = ws + (prod_base + blockIdx.y) * ws_stride;
    const VecLayout L = tile_layout(k1, lrpc + 1);
    const long long total = (2LL << lrpc) << k1;
    for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int v = static_cast<int>(idx >> k1);
        const long long i = idx & (n1 - 1);
        const int arr = v >> lrpc;
        const long long row = r0 + (v & (rpc - 1));
        sm[vec_addr(L, v, static_cast<int>(i))] = base[arr * N + row * n1 + i];
    }
    __syncthreads();
    vec_fwd<Ar>(P, sm, L, nullptr);
    for (long long idx = threadIdx.x; idx < (static_cast<long long>(rpc) << k1); idx += blockDim.x) {
        const int v = static_cast<int>(idx >> k1);
        const long long i = idx & (n1 - 1);
        const long long pa = vec_addr(L, v, static_cast<int>(i)), pb = vec_addr(L, v + rpc, static_cast<int>(i));
        sm[pa] = P.ar.mulmont(sm[pa], sm[pb]);
    }
    __syncthreads();
    const VecLayout LC = tile_layout(k1, lrpc);
    vec_inv<Ar>(P, sm, LC, nullptr);
    for (long long idx = threadIdx.x; idx < (static_cast<long long>(rpc) << k1); idx += blockDim.x) {
        const int v = static_cast<int>(idx >> k1);
        const long long i = idx & (n1 - 1);
        base[(r0 + v) * n1 + i] = sm[vec_addr(LC, v, static_cast<int>(i))];
    }
}

// Row transforms in place (standalone large transforms).
template <class Ar, bool FWD>
__global__ void __launch_bounds__(kThreads)
k_row_ntt(DevPlan<Ar> P, typename Ar::word* data, int logN, int k2, int lrpc, long long prod_base) {
    using word = typename Ar::word;
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    const int k1 = logN - k2;
    const long long n1 = 1LL << k1;
    const long long r0 = static_cast<long long>(blockIdx.x) << lrpc;
    word* base = data + ((prod_base + blockIdx.y) << logN);
    const VecLayout L = tile_layout(k1, lrpc);
    const long long total = (1LL << lrpc) << k1;
    for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int v = static_cast<int>(idx >> k1);
        const long long i = idx & (n1 - 1);
        sm[vec_addr(L, v, static_cast<int>(i))] = base[(r0 + v) * n1 + i];
    }
    __syncthreads();
    if (FWD)
        vec_fwd<Ar>(P, sm, L, nullptr);
    else
        vec_inv<Ar>(P, sm, L, nullptr);
    for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int v = static_cast<int>(idx >> k1);
        const long long i = idx & (n1 - 1);
        base[(r0 + v) * n1 + i] = P.ar.canon(sm[vec_addr(L, v, static_cast<int>(i))]);
    }
}

// ------------------------------------------------------------------ uneven batches

// Persistent kernel for the one-block products of an uneven, mixed-modulus
// batch: every block takes items from a global ticket until none are left;
// each item is the whole fused product (load with zero padding, two forward
// transforms, pointwise product, inverse transform, scaled store) for up to
// 16 products in shared memory.  The modulus constants of the current item
// are copied into shared memory when the modulus changes.
template <class Ar>
__global__ void __launch_bounds__(kThreads)
k_batch_small(const DevPlan<Ar>* __restrict__ plans, const TftConsts<Ar>* __restrict__ tfts,
              const BatchDesc* __restrict__ desc,
              const SmallItem<Ar>* __restrict__ items, unsigned nitems, unsigned* ticket,
              const typename Ar::word* __restrict__ a, const typename Ar::word* __restrict__ b,
              typename Ar::word* __restrict__ c) {
    using word = typename Ar::word;
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    __shared__ DevPlan<Ar> P;
    __shared__ TftConsts<Ar> K;
    __shared__ BatchDesc sd[kSmallMaxPerItem];
    __shared__ unsigned s_item;
    __shared__ int s_prime;
    if (threadIdx.x == 0) s_prime = -1;
    for (;;) {
        __syncthreads();                       // previous item fully stored
        if (threadIdx.x == 0) s_item = atomicAdd(ticket, 1u);
        __syncthreads();
        const unsigned it = s_item;
        if (it >= nitems) break;
        const SmallItem<Ar> I = items[it];
        if (static_cast<int>(I.prime) != s_prime) {
            const unsigned* src = reinterpret_cast<const unsigned*>(plans + I.prime);
            unsigned* dst = reinterpret_cast<unsigned*>(&P);
            for (int i = threadIdx.x; i < static_cast<int>(sizeof(DevPlan<Ar>) / 4); i += blockDim.x)
                dst[i] = src[i];
            const unsigned* ksrc = reinterpret_cast<const unsigned*>(tfts + I.prime);
            unsigned* kdst = reinterpret_cast<unsigned*>(&K);
            for (int i = threadIdx.x; i < static_cast<int>(sizeof(TftConsts<Ar>) / 4); i += blockDim.x)
                kdst[i] = ksrc[i];
        }
        if (threadIdx.x < I.count) sd[threadIdx.x] = desc[I.first + threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) s_prime = static_cast<int>(I.prime);
        const int logL = static_cast<int>(I.logL);
        const int lppc = small_lppc(logL);
        const int ppc = 1 << lppc;
        const int L = 1 << logL;
        const VecLayout LA = tile_layout(logL, lppc + 1);
        for (int idx = threadIdx.x; idx < (L << lppc); idx += blockDim.x) {
            const int v = idx >> logL;
            const int i = idx & (L - 1);
            word xa = 0, xb = 0;
            if (v < static_cast<int>(I.count)) {
                if (i < static_cast<int>(sd[v].na)) xa = a[sd[v].aoff + i];
                if (i < static_cast<int>(sd[v].nb)) xb = b[sd[v].boff + i];
            }
            sm[vec_addr(LA, v, i)] = xa;
            sm[vec_addr(LA, v + ppc, i)] = xb;
        }
        __syncthreads();
        const int kb = static_cast<int>(I.kb);
        const bool tft = kb < 16;                     // the plan sets 16 where truncation does not pay
        if (tft)
            vec_fwd_t<Ar>(P, sm, LA, kb, K);
        else
            vec_fwd<Ar>(P, sm, LA, nullptr);
        const int Lk = tft ? (kb << (logL - 4)) : L;     // positions kept
        for (int idx = threadIdx.x; idx < (L << lppc); idx += blockDim.x) {
            const int v = idx >> logL;
            const int i = idx & (L - 1);
            if (i >= Lk) continue;
            const int pa = vec_addr(LA, v, i), pb = vec_addr(LA, v + ppc, i);
            sm[pa] = P.ar.mulmont(sm[pa], sm[pb]);
        }
        __syncthreads();
        const VecLayout LC = tile_layout(logL, lppc);
        if (tft)
            vec_inv_t<Ar>(P, sm, LC, kb, K);
        else
            vec_inv<Ar>(P, sm, LC, nullptr);
        for (int idx = threadIdx.x; idx < (L << lppc); idx += blockDim.x) {
            const int v = idx >> logL;
            const int i = idx & (L - 1);
            if (v < static_cast<int>(I.count) && i < static_cast<int>(sd[v].na + sd[v].nb - 1))
                c[sd[v].coff + i] = P.ar.canon(P.ar.mulw(sm[vec_addr(LC, v, i)], I.scale));
        }
    }
}

// ------------------------------------------------------------------ polynomial matrices

// Zero-padded copy of the 2 n^2 entries (A then B, d coefficients each) into
// rows of 2^logN words.
template <class Ar>
__global__ void k_polymat_pad(const typename Ar::word* __restrict__ A, const typename Ar::word* __restrict__ B,
                              typename Ar::word* __restrict__ ws, long long nn, long long d, int logN) {
    const long long N = 1LL << logN;
    const long long total = (2 * nn) << logN;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long e = idx >> logN, k = idx & (N - 1);
        typename Ar::word x = 0;
        if (k < d) x = (e < nn) ? A[e * d + k] : B[(e - nn) * d + k];
        ws[idx] = x;
    }
}

// At every frequency k: C^(k) = A^(k) B^(k), an n x n matrix product over
// F_p.  Sums of Montgomery products carry a factor 2^-w, removed at the end
// by the fixed product with r = 2^w rem p.
// Step 2 of the polynomial matrix product: at every frequency k, the n x n
// product C(k) = A(k) B(k).  One warp takes 32 consecutive frequencies (lanes
// read consecutive words of every entry) and one 4 x 4 tile of C; the warps
// of a block share the frequencies, so A's rows are reused from L1.
// LAZY (32-bit words, K >= 3): the 64-bit products are summed in 64 bits and
// folded into a residue every K terms (K (p-1)^2 < 2^64), so a term costs
// one wide multiply-add; the fold is hi 2^32 + lo rem p by two fixed-
// multiplicand products (r = 2^32 rem p, one = 1).  Otherwise every term is
// a Montgomery product summed mod p and the sum is multiplied by r.
template <class Ar, bool LAZY>
__global__ void __launch_bounds__(256)
k_polymat_freq(Ar ar, const typename Ar::word* __restrict__ At, const typename Ar::word* __restrict__ Bt,
               typename Ar::word* __restrict__ Ct, int n, int logN, typename Ar::tw r, typename Ar::tw one,
               int K) {
    using word = typename Ar::word;
    constexpr int T = 4;
    const long long N = 1LL << logN;
    const int nt1 = (n + T - 1) / T;
    const long long ntiles = static_cast<long long>(nt1) * nt1;
    const long long warp = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const long long tile = warp % ntiles, kg = warp / ntiles;
    const long long k = (kg << 5) + (threadIdx.x & 31);
    if (k >= N) return;
    const int i0 = static_cast<int>(tile / nt1) * T, j0 = static_cast<int>(tile % nt1) * T;
    const word* a_base[T];
    const word* b_base[T];
#pragma unroll
    for (int u = 0; u < T; ++u) {
        a_base[u] = At + ((static_cast<long long>(min(i0 + u, n - 1)) * n) << logN) + k;   // row i0+u, l = 0
        b_base[u] = Bt + (static_cast<long long>(min(j0 + u, n - 1)) << logN) + k;         // l = 0, column j0+u
    }
    const long long a_step = N, b_step = static_cast<long long>(n) << logN;
    word res[T][T];
#pragma unroll
    for (int u = 0; u < T; ++u)
#pragma unroll
        for (int v = 0; v < T; ++v) res[u][v] = word(0);
    if constexpr (LAZY) {
        uint64_t acc[T][T];
        for (int l0 = 0; l0 < n; l0 += K) {
#pragma unroll
            for (int u = 0; u < T; ++u)
#pragma unroll
                for (int v = 0; v < T; ++v) acc[u][v] = 0;
            const int l1 = min(n, l0 + K);
            for (int l = l0; l < l1; ++l) {
                word a[T], b[T];
#pragma unroll
                for (int u = 0; u < T; ++u) {
                    a[u] = a_base[u][l * a_step];
                    b[u] = b_base[u][l * b_step];
                }
#pragma unroll
                for (int u = 0; u < T; ++u)
#pragma unroll
                    for (int v = 0; v < T; ++v) acc[u][v] += static_cast<uint64_t>(a[u]) * b[v];
            }
#pragma unroll
            for (int u = 0; u < T; ++u)
#pragma unroll
                for (int v = 0; v < T; ++v) {
                    const word f = ar.add(ar.mulw(static_cast<word>(acc[u][v] >> 32), r),
                                          ar.mulw(static_cast<word>(acc[u][v]), one));
                    res[u][v] = ar.add(res[u][v], f);
                }
        }
    } else {
        for (int l = 0; l < n; ++l) {
            word a[T], b[T];
#pragma unroll
            for (int u = 0; u < T; ++u) {
                a[u] = a_base[u][l * a_step];
                b[u] = b_base[u][l * b_step];
            }
#pragma unroll
            for (int u = 0; u < T; ++u)
#pragma unroll
                for (int v = 0; v < T; ++v) res[u][v] = ar.add(res[u][v], ar.mulmont(a[u], b[v]));
        }
#pragma unroll
        for (int u = 0; u < T; ++u)
#pragma unroll
            for (int v = 0; v < T; ++v) res[u][v] = ar.mulw(res[u][v], r);
    }
#pragma unroll
    for (int u = 0; u < T; ++u)
#pragma unroll
        for (int v = 0; v < T; ++v)
            if (i0 + u < n && j0 + v < n) Ct[((static_cast<long long>(i0 + u) * n + j0 + v) << logN) + k] = res[u][v];
}

// Shared-memory form of the per-frequency products for 32-bit words and
// n in {8, 16, 32}: a block stages A(k) and B(k) for F consecutive
// frequencies (entries read as F-word runs: whole 32-byte sectors), each
// thread forms a 4 x 4 tile of one C(k) from shared memory (four scalar
// words of A, one 16-byte vector of B per term) with 64-bit sums of the
// products, and C goes back through shared memory as F-word runs.  A 64-bit
// sum s = H 2^32 + L (any s < 2^64) is brought to s 2^-32 rem p by one
// Montgomery reduction of t = H (2^32 rem p) + L < p 2^32; the final product
// by r = 2^32 rem p removes the 2^-32.  Sums are folded every K terms.
template <int NN>
struct PmShared {
    static constexpr int NT = NN / 4, TPF = NT * NT;            // tiles (threads) per frequency
    static constexpr int F = (256 / TPF) > 8 ? (256 / TPF) : 8;  // frequencies per block
    static constexpr int THREADS = F * TPF;
    static constexpr int AS = NN + 1;                            // A row stride
    static constexpr int AF = ((NN * AS + 31) / 32) * 32 + 4;    // A per frequency (4 banks apart)
    static constexpr int BF = NN * NN + 4;                       // B (and C) per frequency
    static constexpr size_t words = size_t(F) * (AF + BF);
};

template <int NN>
__global__ void __launch_bounds__(PmShared<NN>::THREADS)
k_polymat_freq_s(Mont32 ar, const uint32_t* __restrict__ At, const uint32_t* __restrict__ Bt,
                 uint32_t* __restrict__ Ct, int logN, Tw32 r, uint32_t r1, int K) {
    using S = PmShared<NN>;
    extern __shared__ __align__(16) unsigned char smraw[];
    uint32_t* sA = reinterpret_cast<uint32_t*>(smraw);
    uint32_t* sB = sA + S::F * S::AF;
    const long long N = 1LL << logN;
    const long long k0 = static_cast<long long>(blockIdx.x) * S::F;
    const int tid = threadIdx.x;
#pragma unroll 4
    for (int it = 0; it < NN * NN * S::F / S::THREADS; ++it) {
        const int idx = it * S::THREADS + tid;
        const int f = idx % S::F, e = idx / S::F;               // entry e = row * NN + column
        const bool in = k0 + f < N;
        const long long g = (static_cast<long long>(e) << logN) + k0 + f;
        sA[f * S::AF + (e / NN) * S::AS + (e % NN)] = in ? At[g] : 0u;
        sB[f * S::BF + e] = in ? Bt[g] : 0u;
    }
    __syncthreads();
    const int f = tid / S::TPF, tile = tid % S::TPF;
    const int i0 = (tile / S::NT) * 4, j0 = (tile % S::NT) * 4;
    const uint32_t* a_f = sA + f * S::AF + i0 * S::AS;
    const uint32_t* b_f = sB + f * S::BF + j0;
    uint32_t res[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) res[u][v] = 0;
    for (int l0 = 0; l0 < NN; l0 += K) {
        uint64_t acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0;
        const int l1 = min(NN, l0 + K);
        for (int l = l0; l < l1; ++l) {
            uint32_t a[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = a_f[u * S::AS + l];
            const uint4 bv = *reinterpret_cast<const uint4*>(b_f + l * NN);
            const uint32_t b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += static_cast<uint64_t>(a[u]) * b[v];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const uint64_t t = static_cast<uint64_t>(static_cast<uint32_t>(acc[u][v] >> 32)) * r1 +
                                   static_cast<uint32_t>(acc[u][v]);
                const uint32_t q = static_cast<uint32_t>(t) * ar.pinv;
                const uint32_t red = ar.sub_sel(static_cast<uint32_t>(t >> 32), __umulhi(q, ar.p));
                res[u][v] = ar.add(res[u][v], red);
            }
    }
    __syncthreads();                                             // B is read; C reuses its space
    uint32_t* c_f = sB + f * S::BF + i0 * NN + j0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        uint4 cv;
        cv.x = ar.mulw(res[u][0], r);
        cv.y = ar.mulw(res[u][1], r);
        cv.z = ar.mulw(res[u][2], r);
        cv.w = ar.mulw(res[u][3], r);
        *reinterpret_cast<uint4*>(c_f + u * NN) = cv;
    }
    __syncthreads();
#pragma unroll 4
    for (int it = 0; it < NN * NN * S::F / S::THREADS; ++it) {
        const int idx = it * S::THREADS + tid;
        const int ff = idx % S::F, e = idx / S::F;
        if (k0 + ff < N) Ct[(static_cast<long long>(e) << logN) + k0 + ff] = sB[ff * S::BF + e];
    }
}

// The same for 64-bit words (Shoup64L, p < 2^62): 128-bit sums of the
// products, folded every K = floor((2^64 - 1) / (p - 1)) terms (so a sum is
// below p 2^64) by one Montgomery reduction to s 2^-64 rem p; the final
// product by r = 2^64 rem p removes the 2^-64.  4 frequencies per block at
// n = 32 to fit shared memory.
template <int NN>
struct PmShared64 {
    static constexpr int NT = NN / 4, TPF = NT * NT;
    static constexpr int F = (256 / TPF) > 4 ? (256 / TPF) : 4;
    static constexpr int THREADS = F * TPF;
    static constexpr int AS = NN + 1;
    static constexpr int AF = NN * AS + 1 + ((NN * AS + 1) & 1);   // even: keeps B 16-byte aligned
    static constexpr int BF = NN * NN + 2;
    static constexpr size_t words = size_t(F) * (AF + BF);
};

template <int NN>
__global__ void __launch_bounds__(PmShared64<NN>::THREADS)
k_polymat_freq_s64(Shoup64L ar, const uint64_t* __restrict__ At, const uint64_t* __restrict__ Bt,
                   uint64_t* __restrict__ Ct, int logN, Tw64 r, int K) {
    using S = PmShared64<NN>;
    using u128 = unsigned __int128;
    extern __shared__ __align__(16) unsigned char smraw[];
    uint64_t* sA = reinterpret_cast<uint64_t*>(smraw);
    uint64_t* sB = sA + S::F * S::AF;
    const long long N = 1LL << logN;
    const long long k0 = static_cast<long long>(blockIdx.x) * S::F;
    const int tid = threadIdx.x;
#pragma unroll 4
    for (int it = 0; it < NN * NN * S::F / S::THREADS; ++it) {
        const int idx = it * S::THREADS + tid;
        const int f = idx % S::F, e = idx / S::F;
        const bool in = k0 + f < N;
        const long long g = (static_cast<long long>(e) << logN) + k0 + f;
        sA[f * S::AF + (e / NN) * S::AS + (e % NN)] = in ? At[g] : 0ull;
        sB[f * S::BF + e] = in ? Bt[g] : 0ull;
    }
    __syncthreads();
    const int f = tid / S::TPF, tile = tid % S::TPF;
    const int i0 = (tile / S::NT) * 4, j0 = (tile % S::NT) * 4;
    const uint64_t* a_f = sA + f * S::AF + i0 * S::AS;
    const uint64_t* b_f = sB + f * S::BF + j0;
    uint64_t res[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) res[u][v] = 0;
    for (int l0 = 0; l0 < NN; l0 += K) {
        u128 acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0;
        const int l1 = min(NN, l0 + K);
        for (int l = l0; l < l1; ++l) {
            uint64_t a[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = a_f[u * S::AS + l];
            const ulonglong2 b01 = *reinterpret_cast<const ulonglong2*>(b_f + l * NN);
            const ulonglong2 b23 = *reinterpret_cast<const ulonglong2*>(b_f + l * NN + 2);
            const uint64_t b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += static_cast<u128>(a[u]) * b[v];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const uint64_t lo = static_cast<uint64_t>(acc[u][v]), hi = static_cast<uint64_t>(acc[u][v] >> 64);
                const uint64_t q = lo * ar.pinv;
                const uint64_t t = __umul64hi(q, ar.p);
                const uint64_t red = (hi >= t) ? hi - t : hi - t + ar.p;
                res[u][v] = ar.add(res[u][v], red);
            }
    }
    __syncthreads();
    uint64_t* c_f = sB + f * S::BF + i0 * NN + j0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) c_f[u * NN + v] = ar.canon(ar.mulw(res[u][v], r));
    __syncthreads();
#pragma unroll 4
    for (int it = 0; it < NN * NN * S::F / S::THREADS; ++it) {
        const int idx = it * S::THREADS + tid;
        const int ff = idx % S::F, e = idx / S::F;
        if (k0 + ff < N) Ct[(static_cast<long long>(e) << logN) + k0 + ff] = sB[ff * S::BF + e];
    }
}

template <class Ar>
__global__ void k_polymat_crop(Ar ar, const typename Ar::word* __restrict__ ws, typename Ar::word* __restrict__ C,
                               long long nn, long long dc, int logN) {
    const long long total = nn * dc;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long e = idx / dc, k = idx - e * dc;
        C[idx] = ar.canon(ws[(e << logN) + k]);
    }
}

// ------------------------------------------------------------------ plain kernels

template <class Ar>
__global__ void k_plain_load(const typename Ar::word* a, long long na, const typename Ar::word* b,
                             long long nb, typename Ar::word* ws, int logN, long long batch) {
    const long long N = 1LL << logN;
    const long long total = (2 * batch) << logN;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long arr = idx >> logN, i = idx & (N - 1);
        typename Ar::word x = 0;
        if (arr < batch) {
            if (i < na) x = a[arr * na + i];
        } else if (i < nb) {
            x = b[(arr - batch) * nb + i];
        }
        ws[idx] = x;
    }
}

// One radix-2 DIF stage of half-span 2^logh on narr arrays of 2^logN words.
template <class Ar>
__global__ void k_plain_dif(DevPlan<Ar> P, typename Ar::word* ws, long long narr, int logN, int logh) {
    const long long half = 1LL << (logN - 1);
    const long long total = narr * half;
    const long long h = 1LL << logh;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long arr = idx >> (logN - 1), i = idx & (half - 1);
        const long long j = i & (h - 1), blk = i >> logh;
        typename Ar::word* x = ws + (arr << logN) + (blk << (logh + 1)) + j;
        const auto u = x[0], v = x[h];
        x[0] = P.ar.add(u, v);
        x[h] = P.ar.mulw(P.ar.sub(u, v), P.plain_fwd[j << (logN - 1 - logh)]);
    }
}

template <class Ar>
__global__ void k_plain_dit(DevPlan<Ar> P, typename Ar::word* ws, long long narr, int logN, int logh) {
    const long long half = 1LL << (logN - 1);
    const long long total = narr * half;
    const long long h = 1LL << logh;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long arr = idx >> (logN - 1), i = idx & (half - 1);
        const long long j = i & (h - 1), blk = i >> logh;
        typename Ar::word* x = ws + (arr << logN) + (blk << (logh + 1)) + j;
        const auto u = x[0];
        const auto t = P.ar.mulw(x[h], P.plain_inv[j << (logN - 1 - logh)]);
        x[0] = P.ar.add(u, t);
        x[h] = P.ar.sub(u, t);
    }
}

template <class Ar>
__global__ void k_plain_pointwise(DevPlan<Ar> P, typename Ar::word* ws, long long count,
                                  long long boff) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < count;
         idx += (long long)gridDim.x * blockDim.x)
        ws[idx] = P.ar.mulmont(ws[idx], ws[idx + boff]);
}

template <class Ar>
__global__ void k_plain_store(DevPlan<Ar> P, const typename Ar::word* ws, typename Ar::word* c,
                              long long nc, int logN, long long batch, typename Ar::tw scale) {
    const long long total = batch * nc;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long arr = idx / nc, i = idx - arr * nc;
        c[idx] = P.ar.canon(P.ar.mulw(ws[(arr << logN) + i], scale));
    }
}

// ------------------------------------------------------------------ launchers

template <class K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(bytes));
}

static int grid_for(long long total) {
    long long blocks = (total + kThreads - 1) / kThreads;
    return static_cast<int>(std::max(1LL, std::min(blocks, 152LL * 32)));
}

static int row_lrpc(int k1, int operands) {
    // short rows: enough rows that the lanes of a warp span >= 32 lines
    if (k1 <= kMaxLineLog) return operands == 2 ? 4 : 5;
    return operands == 2 ? 0 : 1;
}

static int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        gbntt_set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return NTT_ERR_CUDA;
    }
    return NTT_OK;
}

static constexpr long long kMaxGridY = 65535;

// The three direct 256 x 256 kernels (n = 2^16 above the one-block limit):
// uniform batches (desc == null: product t at a + t*na, b + t*nb,
// c + t*(na+nb-1)) or uneven ones (desc: offsets and lengths per product,
// a, b, c the flat buffers).  ws holds 2n words per product.
template <class Ar>
const TftConsts<Ar>& tft_consts(const ntt_plan* plan) {
    if constexpr (std::is_same<Ar, Mont32>::value) return plan->tft32;
    else if constexpr (std::is_same<Ar, Shoup64L>::value) return plan->tft64;
    else return plan->tftf;
}

// The three direct 256 x 256 kernels (n = 2^16 above the one-block limit):
// uniform batches (desc == null: product t at a + t*na, b + t*nb,
// c + t*(na+nb-1)) or uneven ones (desc: offsets and lengths per product,
// a, b, c the flat buffers).  ws holds 2n words per product.  Products
// shorter than n take the truncated transforms (TFT) over the 16 B rows
// their na + nb - 1 output words need; full-length uniform batches run the
// plain kernels.
template <class Ar>
int launch_polymul_direct(const ntt_plan* plan, const DevPlan<Ar>& dp, const typename Ar::word* a,
                          long long na, const typename Ar::word* b, long long nb, long long batch,
                          typename Ar::word* c, typename Ar::word* ws, const BatchDesc* desc,
                          cudaStream_t st, bool want_tma = false) {
    using word = typename Ar::word;
    constexpr long long N = 1LL << (2 * kDLog);
    const size_t smem_c = direct_col_smem_words() * sizeof(word);
    const size_t smem_r = direct_row_smem_words() * sizeof(word);
    const bool zhalf = !desc && 2 * std::max(na, nb) <= N;
    // the truncated kernels pay off from 13 of the 16 row blocks down
    // (measured: 14 blocks cost 1.01 of the full step, 12 blocks 0.90)
    const int beta = desc ? 16 : tft_blocks(na + nb - 1);
    const bool tft = desc != nullptr || beta <= kDTftMaxBlocks;
    auto kcf = tft ? (zhalf ? k_col_fwd_d<Ar, true, true> : k_col_fwd_d<Ar, false, true>)
                   : (zhalf ? k_col_fwd_d<Ar, true> : k_col_fwd_d<Ar, false>);
    auto kci = tft ? k_col_inv_d<Ar, true> : k_col_inv_d<Ar>;
    auto krp = tft ? k_row_polymul_d<Ar, kDRowsPerBlock, true> : k_row_polymul_d<Ar, kDRowsPerBlock>;
    if (allow_smem(kcf, smem_c) != cudaSuccess || allow_smem(kci, smem_c) != cudaSuccess ||
        allow_smem(krp, smem_r) != cudaSuccess)
        return check_launch("smem attr");
    const auto* itab = static_cast<const typename Ar::tw*>(plan->glob_inv_pm);
    const unsigned row_blocks = static_cast<unsigned>(16 * (tft ? beta : 16) / kDRowsPerBlock);
    // TMA tiles (shape-table choice) for zero-half operands of whole rows
    // (16-byte aligned bases)
    CUtensorMap map_a{}, map_b{};
    bool tma = want_tma && zhalf && na % kDLine == 0 && nb % kDLine == 0 && batch < (1LL << 31);
    if (tma) {
        const CUtensorMapDataType dt = sizeof(word) == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                       : std::is_same<word, double>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                                            : CU_TENSOR_MAP_DATA_TYPE_UINT64;
        const uint32_t box[3] = {kDCols, kDLine / 2, 1};
        const uint64_t da[3] = {kDLine, static_cast<uint64_t>(na / kDLine), static_cast<uint64_t>(batch)};
        const uint64_t db[3] = {kDLine, static_cast<uint64_t>(nb / kDLine), static_cast<uint64_t>(batch)};
        const uint64_t sa[2] = {kDLine * sizeof(word), static_cast<uint64_t>(na) * sizeof(word)};
        const uint64_t sb[2] = {kDLine * sizeof(word), static_cast<uint64_t>(nb) * sizeof(word)};
        tma = encode_tensor_map_3d(&map_a, dt, const_cast<word*>(a), da, sa, box) &&
              encode_tensor_map_3d(&map_b, dt, const_cast<word*>(b), db, sb, box);
    }
    int* err = tma ? device_error_flag() : nullptr;
    tma = tma && err;
    auto kct = tft ? k_col_fwd_tma<Ar, true> : k_col_fwd_tma<Ar, false>;
    const size_t smem_t = smem_c + 16;
    if (tma && allow_smem(kct, smem_t) != cudaSuccess) return check_launch("smem attr");
    for (long long p0 = 0; p0 < batch; p0 += kMaxGridY) {
        const unsigned nbat = static_cast<unsigned>(std::min(batch - p0, kMaxGridY));
        if (tma)
            kct<<<dim3(kDLine / kDCols, nbat, 2), kDThreads, smem_t, st>>>(dp, map_a, map_b, ws, 2 * N, N, p0,
                                                                           tft ? beta : 16, err);
        else
            kcf<<<dim3(kDLine / kDCols, nbat, 2), kDThreads, smem_c, st>>>(dp, dp.ar, a, na, na, b, nb, nb, ws, 2 * N, N,
                                                                           p0, desc, tft ? beta : 16);
        prof_mark(st, tma ? (tft ? "k_col_fwd_tma_tft" : "k_col_fwd_tma") : (tft ? "k_col_fwd_d_tft" : "k_col_fwd_d"));
        krp<<<dim3(row_blocks, nbat, 1), kDRowsPerBlock * 16, smem_r, st>>>(dp, wide_form(dp.ar), ws, 2 * N, p0, desc);
        prof_mark(st, tft ? "k_row_polymul_d_tft" : "k_row_polymul_d");
        kci<<<dim3(kDLine / kDCols, nbat, 1), kDThreads, smem_c, st>>>(dp, wide_form(dp.ar), ws, 2 * N, c, na + nb - 1,
                                                                       na + nb - 1, itab, plan->glob_inv_pm_w, p0, desc,
                                                                       tft ? beta : 16, tft_consts<Ar>(plan));
        prof_mark(st, tft ? "k_col_inv_d_tft" : "k_col_inv_d");
    }
    return check_launch("direct polymul passes");
}

template <class Ar>
const DevPlan<Ar>& devplan_of(const ntt_plan* plan) {
    if constexpr (std::is_same<Ar, Mont32>::value) return plan->dp32;
    else if constexpr (std::is_same<Ar, Shoup64L>::value) return plan->dp64;
    else return plan->dpf;
}

template <class Ar, bool TFT>
auto pre_kernel(int M) {
    return M == 2 ? k_pre_fwd<Ar, 2, TFT> : M == 4 ? k_pre_fwd<Ar, 4, TFT> : M == 8 ? k_pre_fwd<Ar, 8, TFT>
                                                                           : k_pre_fwd<Ar, 16, TFT>;
}

template <class Ar, bool TFT>
auto post_kernel(int M) {
    return M == 2 ? k_post_inv<Ar, 2, TFT> : M == 4 ? k_post_inv<Ar, 4, TFT> : M == 8 ? k_post_inv<Ar, 8, TFT>
                                                                             : k_post_inv<Ar, 16, TFT>;
}

template <class Ar, bool ZHALF, bool TFT>
auto colx_fwd_kernel(int C) {
    return C == 5 ? k_colx_fwd<Ar, 5, ZHALF, TFT> : C == 6 ? k_colx_fwd<Ar, 6, ZHALF, TFT>
         : C == 7 ? k_colx_fwd<Ar, 7, ZHALF, TFT> : k_colx_fwd<Ar, 8, ZHALF, TFT>;
}

template <class Ar, bool TFT>
auto colx_inv_kernel(int C) {
    return C == 5 ? k_colx_inv<Ar, 5, TFT> : C == 6 ? k_colx_inv<Ar, 6, TFT>
         : C == 7 ? k_colx_inv<Ar, 7, TFT> : k_colx_inv<Ar, 8, TFT>;
}

// The 2^16-point stage of a product of n = 2^17 .. 2^20 points: `count`
// uniform sub-products at ws + s 2^17 (operand a) and + 2^16 (operand b),
// transformed, multiplied and inverse-transformed in place by the child plan.
template <class Ar>
int launch_sub_products(const ntt_plan* core, typename Ar::word* ws, long long count, cudaStream_t st) {
    using word = typename Ar::word;
    const DevPlan<Ar>& dpc = devplan_of<Ar>(core);
    constexpr long long S = 2 * kSubN;
    const size_t smem_c = direct_col_smem_words() * sizeof(word);
    const size_t smem_r = direct_row_smem_words() * sizeof(word);
    auto kcf = k_col_fwd_d<Ar, false>;
    auto krp = k_row_polymul_d<Ar, kDRowsPerBlock>;
    auto kci = k_col_inv_d<Ar>;
    if (allow_smem(kcf, smem_c) != cudaSuccess || allow_smem(kci, smem_c) != cudaSuccess ||
        allow_smem(krp, smem_r) != cudaSuccess)
        return check_launch("smem attr");
    const auto* itab = static_cast<const typename Ar::tw*>(core->glob_inv_pm);
    for (long long p0 = 0; p0 < count; p0 += kMaxGridY) {
        const unsigned nb = static_cast<unsigned>(std::min(count - p0, kMaxGridY));
        kcf<<<dim3(kDLine / kDCols, nb, 2), kDThreads, smem_c, st>>>(dpc, dpc.ar, ws, kSubN, S, ws + kSubN, kSubN, S, ws,
                                                                     S, kSubN, p0, nullptr, 16);
        prof_mark(st, "k_col_fwd_d");
        krp<<<dim3(kDLine / kDRowsPerBlock, nb, 1), kDRowsPerBlock * 16, smem_r, st>>>(dpc, wide_form(dpc.ar), ws, S,
                                                                                       p0, nullptr);
        prof_mark(st, "k_row_polymul_d");
        kci<<<dim3(kDLine / kDCols, nb, 1), kDThreads, smem_c, st>>>(dpc, wide_form(dpc.ar), ws, S, ws, kSubN, S,
                                                                     itab, core->glob_inv_pm_w, p0, nullptr, 16,
                                                                     TftConsts<Ar>{});
        prof_mark(st, "k_col_inv_d");
    }
    return check_launch("sub-product passes");
}

// Products of n = 2^17 .. 2^24 points (Algorithm 1 with n1 = 2^16): the pass
// across the rows, the 2^16-point stage on the rows, the inverse pass.
// Every product keeps only the rows its na + nb - 1 words need (TFT:
// lam = ceil((na + nb - 1) / 2^16), rounded up to whole R2-row blocks for
// n2 > 16).  Uneven batches (desc) take each product's lam from its
// descriptor and its rows from slot desc.sub on; `subs` is the bucket's
// total of kept rows, the number of 2^16-point sub-products.
template <class Ar>
int launch_polymul_sub(const ntt_plan* plan, const DevPlan<Ar>& dp, const typename Ar::word* a, long long na,
                       const typename Ar::word* b, long long nb, long long batch, typename Ar::word* c,
                       typename Ar::word* ws, const BatchDesc* desc, cudaStream_t st, long long subs = 0) {
    using word = typename Ar::word;
    const int m = static_cast<int>(plan->log2n) - kSubLog;
    const int M = 1 << m;
    const long long L = na + nb - 1;
    int lam = desc ? M : static_cast<int>(std::min<long long>(M, (L + kSubN - 1) / kSubN));
    int B = 16;
    if (M > 16) {                                       // column kernels: whole blocks of R2 rows
        const int R2 = M / 16;
        B = (lam + R2 - 1) / R2;
        lam = B * R2;
    }
    const bool tft = desc ? true : lam < M;
    const long long rows_stride = static_cast<long long>(lam) * 2 * kSubN;
    const auto* pre = static_cast<const typename Ar::tw*>(plan->pre_fwd);
    const auto* pre_inv = static_cast<const typename Ar::tw*>(plan->pre_inv);
    const size_t smem_x = size_t(M) * kDCols * sizeof(word);
    const bool zhalf = !desc && 2 * std::max(na, nb) <= (1LL << plan->log2n);
    prof_begin_call(st);
    for (long long p0 = 0; p0 < batch; p0 += kMaxGridY) {
        const unsigned nbat = static_cast<unsigned>(std::min(batch - p0, kMaxGridY));
        if (M <= 16) {
            auto kpre = tft ? pre_kernel<Ar, true>(M) : pre_kernel<Ar, false>(M);
            kpre<<<dim3(kSubN / kSubThreads, nbat, 2), kSubThreads, 0, st>>>(dp.ar, dp, a, na, na, b, nb, nb, ws,
                                                                             rows_stride, 2 * kSubN, kSubN, pre,
                                                                             p0, desc, lam);
        } else {
            auto kx = tft ? (zhalf ? colx_fwd_kernel<Ar, true, true>(m) : colx_fwd_kernel<Ar, false, true>(m))
                          : (zhalf ? colx_fwd_kernel<Ar, true, false>(m) : colx_fwd_kernel<Ar, false, false>(m));
            if (allow_smem(kx, smem_x) != cudaSuccess) return check_launch("smem attr");
            kx<<<dim3(kSubN / kDCols, nbat, 2), kDThreads, smem_x, st>>>(dp, a, na, na, b, nb, nb, ws, rows_stride,
                                                                         2 * kSubN, kSubN, pre, p0, desc, B);
        }
        prof_mark(st, "k_pre_fwd");
    }
    int rc = launch_sub_products<Ar>(plan->core, ws, desc ? subs : batch * lam, st);
    if (rc != NTT_OK) return rc;
    for (long long p0 = 0; p0 < batch; p0 += kMaxGridY) {
        const unsigned nbat = static_cast<unsigned>(std::min(batch - p0, kMaxGridY));
        if (M <= 16) {
            auto kpost = tft ? post_kernel<Ar, true>(M) : post_kernel<Ar, false>(M);
            kpost<<<dim3(kSubN / kSubThreads, nbat, 1), kSubThreads, 0, st>>>(
                dp.ar, dp, tft_consts<Ar>(plan), ws, rows_stride, 2 * kSubN, c, L, L, pre_inv, p0, desc, lam);
        } else {
            auto kx = tft ? colx_inv_kernel<Ar, true>(m) : colx_inv_kernel<Ar, false>(m);
            if (allow_smem(kx, smem_x) != cudaSuccess) return check_launch("smem attr");
            kx<<<dim3(kSubN / kDCols, nbat, 1), kDThreads, smem_x, st>>>(dp, tft_consts<Ar>(plan), ws, rows_stride,
                                                                         2 * kSubN, c, L, L, pre_inv, p0, desc, B);
        }
        prof_mark(st, "k_post_inv");
    }
    return check_launch("sub-vector passes");
}

// Standalone 2^16-point transforms of `batch` vectors in place with the
// direct kernels (data 16-byte aligned): forward = column pass with the
// global twiddle, then row pass; inverse = row pass, then column pass with
// the inverse global twiddle (n^-1 folded in).
template <class Ar>
int launch_ntt_direct(const DevPlan<Ar>& dp, typename Ar::word* data, long long batch, bool fwd,
                      cudaStream_t st) {
    using word = typename Ar::word;
    constexpr long long N = 1LL << (2 * kDLog);
    const size_t smem_c = direct_col_smem_words() * sizeof(word);
    const size_t smem_r = direct_ntt_row_smem_words() * sizeof(word);
    auto krow = fwd ? k_row_ntt_d<Ar, true, kDNttRowsPerBlock> : k_row_ntt_d<Ar, false, kDNttRowsPerBlock>;
    if (allow_smem(k_col_fwd_d<Ar, false>, smem_c) != cudaSuccess ||
        allow_smem(k_col_inv_d<Ar>, smem_c) != cudaSuccess || allow_smem(krow, smem_r) != cudaSuccess)
        return check_launch("smem attr");
    prof_begin_call(st);
    for (long long p0 = 0; p0 < batch; p0 += kMaxGridY) {
        const unsigned nbat = static_cast<unsigned>(std::min(batch - p0, kMaxGridY));
        const dim3 gc(kDLine / kDCols, nbat, 1), gr(kDLine / kDNttRowsPerBlock, nbat, 1);
        if (fwd) {
            k_col_fwd_d<Ar, false><<<gc, kDThreads, smem_c, st>>>(dp, dp.ar, data, N, N, data, N, N, data, N, 0, p0,
                                                                  nullptr, 16);
            prof_mark(st, "k_col_fwd_d");
            krow<<<gr, kDNttRowsPerBlock * 16, smem_r, st>>>(dp, data, p0);
            prof_mark(st, "k_row_ntt_fwd_d");
        } else {
            krow<<<gr, kDNttRowsPerBlock * 16, smem_r, st>>>(dp, data, p0);
            prof_mark(st, "k_row_ntt_inv_d");
            k_col_inv_d<Ar><<<gc, kDThreads, smem_c, st>>>(dp, wide_form(dp.ar), data, N, data, N, N, dp.glob_inv, dp.wglob[1], p0, nullptr, 16,
                                                           TftConsts<Ar>{});
            prof_mark(st, "k_col_inv_d");
        }
    }
    return check_launch("direct ntt passes");
}

// Standalone transforms of n = 2^17 .. 2^24 points in place (data 16-byte
// aligned): forward = pass across the rows, then 2^16-point transforms of the
// rows by the child plan; inverse = the reverse.
template <class Ar>
int launch_ntt_sub(const ntt_plan* plan, const DevPlan<Ar>& dp, typename Ar::word* data, long long batch,
                   bool fwd, cudaStream_t st) {
    using word = typename Ar::word;
    const int m = static_cast<int>(plan->log2n) - kSubLog;
    const int M = 1 << m;
    const long long n = static_cast<long long>(M) * kSubN;
    const DevPlan<Ar>& dpc = devplan_of<Ar>(plan->core);
    const auto* pre = static_cast<const typename Ar::tw*>(plan->pre_fwd);
    const auto* pre_inv = static_cast<const typename Ar::tw*>(plan->pre_inv);
    const size_t smem_x = size_t(M) * kDCols * sizeof(word);
    int rc = NTT_OK;
    if (!fwd) {
        rc = launch_ntt_direct<Ar>(dpc, data, batch * M, false, st);
        if (rc != NTT_OK) return rc;
    }
    prof_begin_call(st);
    for (long long p0 = 0; p0 < batch; p0 += kMaxGridY) {
        const unsigned nbat = static_cast<unsigned>(std::min(batch - p0, kMaxGridY));
        if (fwd && M <= 16) {
            pre_kernel<Ar, false>(M)<<<dim3(kSubN / kSubThreads, nbat, 1), kSubThreads, 0, st>>>(
                dp.ar, dp, data, n, n, data, n, n, data, n, kSubN, 0, pre, p0, nullptr, M);
        } else if (fwd) {
            auto kx = colx_fwd_kernel<Ar, false, false>(m);
            if (allow_smem(kx, smem_x) != cudaSuccess) return check_launch("smem attr");
            kx<<<dim3(kSubN / kDCols, nbat, 1), kDThreads, smem_x, st>>>(dp, data, n, n, data, n, n, data, n, kSubN,
                                                                         0, pre, p0, nullptr, 16);
        } else if (M <= 16) {
            post_kernel<Ar, false>(M)<<<dim3(kSubN / kSubThreads, nbat, 1), kSubThreads, 0, st>>>(
                dp.ar, dp, TftConsts<Ar>{}, data, n, kSubN, data, n, n, pre_inv, p0, nullptr, M);
        } else {
            auto kx = colx_inv_kernel<Ar, false>(m);
            if (allow_smem(kx, smem_x) != cudaSuccess) return check_launch("smem attr");
            kx<<<dim3(kSubN / kDCols, nbat, 1), kDThreads, smem_x, st>>>(dp, TftConsts<Ar>{}, data, n, kSubN, data,
                                                                         n, n, pre_inv, p0, nullptr, 16);
        }
        prof_mark(st, fwd ? "k_pre_fwd" : "k_post_inv");
    }
    rc = check_launch("sub-vector pass");
    if (rc != NTT_OK || !fwd) return rc;
    return launch_ntt_direct<Ar>(dpc, data, batch * M, true, st);
}

// A few 4096-point products, each on one thread-block cluster of 8 CTAs
// (latency: the three transforms of a product spread over 8 SMs).
template <class Ar>
int launch_polymul_cluster(const DevPlan<Ar>& dp, const typename Ar::word* a, long long na,
                           const typename Ar::word* b, long long nb, long long batch, typename Ar::word* c,
                           typename Ar::tw scale, cudaStream_t st) {
    const bool zh = na <= 2048 && nb <= 2048;
    auto k = zh ? k_cluster_polymul<Ar, true> : k_cluster_polymul<Ar, false>;
    const size_t smem = cluster_smem_words() * sizeof(typename Ar::word);
    if (allow_smem(k, smem) != cudaSuccess) return check_launch("smem attr");
    k<<<static_cast<unsigned>(kClCtas * batch), kClThreads, smem, st>>>(dp, wide_form(dp.ar), a, na, b, nb, c,
                                                                        scale);
    prof_mark(st, "k_cluster_polymul");
    return check_launch("k_cluster_polymul");
}

template <class Ar>
int launch_polymul_fused(const ntt_plan* plan, const DevPlan<Ar>& dp, const typename Ar::word* a,
                         long long na, const typename Ar::word* b, long long nb, long long batch,
                         typename Ar::word* c, typename Ar::word* ws, typename Ar::tw scale,
                         cudaStream_t st) {
    using word = typename Ar::word;
    const int k = static_cast<int>(plan->log2n);
    const LaunchCfg cfg = launch_cfg(sizeof(word), k, plan->tile_max_log);
    prof_begin_call(st);
    if constexpr (!std::is_same<Ar, Fma50>::value) {
        if (k == kClLog && batch <= kClMaxBatch && dp.line64x8[0] && dp.tile_fwd[kClLog])
            return launch_polymul_cluster<Ar>(dp, a, na, b, nb, batch, c, scale, st);
    }
    if (k <= plan->tile_max_log) {
        const int lppc = cfg.lppc;
        const size_t smem = layout_words(tile_layout(k, lppc + 1)) * sizeof(word);
        const long long blocks = (batch + (1LL << lppc) - 1) >> lppc;
        const bool few = blocks < sm_count(plan->device);
        const bool wide = few || smem > kTileWideSmem;
        // truncated transforms when the output leaves enough of the 16
        // blocks of n/16 positions empty
        const int kb = k >= kTileTftMinLog ? tft_kb(na + nb - 1, k) : 16;
        const bool tft = kb <= kTileTftMaxBlocks;   // else the full transforms
        auto kt = tft ? (wide ? k_tile_polymul<Ar, 2 * kThreads, true> : k_tile_polymul<Ar, kThreads, true>)
                      : (wide ? k_tile_polymul<Ar, 2 * kThreads> : k_tile_polymul<Ar, kThreads>);
        int nt = wide ? 2 * kThreads : kThreads;
        if constexpr (sizeof(word) == 4) {
            if (few) {
                kt = tft ? k_tile_polymul<Ar, 4 * kThreads, true> : k_tile_polymul<Ar, 4 * kThreads>;
                nt = 4 * kThreads;
            }
        }
        if (allow_smem(kt, smem) != cudaSuccess) return check_launch("smem attr");
        for (long long b0 = 0; b0 < blocks; b0 += 0x7fffffffLL) {
            const long long nb0 = std::min(blocks - b0, 0x7fffffffLL);
            const long long p0 = b0 << lppc;
            kt<<<static_cast<unsigned>(nb0), nt, smem, st>>>(
                dp, a + p0 * na, na, b + p0 * nb, nb, c + p0 * (na + nb - 1), batch - p0, k, lppc,
                scale, kb, tft_consts<Ar>(plan));
            prof_mark(st, tft ? "k_tile_polymul_tft" : "k_tile_polymul");
        }
        return check_launch("k_tile_polymul");
    }
    if (cfg.logw == 0 && k == 2 * kDLog)
        return launch_polymul_direct<Ar>(plan, dp, a, na, b, nb, batch, c, ws, nullptr, st, (cfg.lppc & 1) != 0);
    if (cfg.logw == 0 && plan->core) return launch_polymul_sub<Ar>(plan, dp, a, na, b, nb, batch, c, ws, nullptr, st);
    const int k2 = plan->k2, k1 = plan->k1;
    const long long N = 1LL << k;
    const int logw = cfg.logw;
    const size_t smem_c = slab_words(slab_layout(k2, logw)) * sizeof(word);
    const int lrpc = cfg.lrpc;
    const size_t smem_r = layout_words(tile_layout(k1, lrpc + 1)) * sizeof(word);
    const bool zhalf = 2 * std::max(na, nb) <= N;
    // truncated transforms (columns of 16 .. 256 words) when the output
    // leaves enough of the 16 column blocks empty
    const int kb = (k2 >= 4 && k2 <= kMaxLineLog) ? tft_kb(na + nb - 1, k) : 16;
    const bool tft = kb <= kColTftMaxBlocks;
    auto kcf = tft ? (zhalf ? k_col_fwd<Ar, true, 0, 0, true> : k_col_fwd<Ar, false, 0, 0, true>)
                   : (zhalf ? k_col_fwd<Ar, true> : k_col_fwd<Ar, false>);
    auto kci = tft ? k_col_inv<Ar, 0, 0, true> : k_col_inv<Ar>;
    auto krp = tft ? k_row_polymul<Ar, 0, 0, true> : k_row_polymul<Ar>;
    // compile-time geometry for the shape of the 2^16-point 32-bit products
    if (sizeof(word) == 4 && k == 16 && logw == 5 && lrpc == 4 && !tft) {
        kcf = zhalf ? k_col_fwd<Ar, true, 16, 5> : k_col_fwd<Ar, false, 16, 5>;
        kci = k_col_inv<Ar, 16, 5>;
        krp = k_row_polymul<Ar, 16, 4>;
    }
    const auto* itab = static_cast<const typename Ar::tw*>(plan->glob_inv_pm);
    if (allow_smem(kcf, smem_c) != cudaSuccess || allow_smem(kci, smem_c) != cudaSuccess ||
        allow_smem(krp, smem_r) != cudaSuccess)
        return check_launch("smem attr");
    // rows of the row pass: the kept column blocks' rows, in whole blocks
    // of 2^lrpc rows
    const long long rows = tft ? (static_cast<long long>(kb) << (k2 - 4)) : (1LL << k2);
    const unsigned row_blocks = static_cast<unsigned>((rows + (1LL << lrpc) - 1) >> lrpc);
    for (long long p0 = 0; p0 < batch; p0 += kMaxGridY) {
        const unsigned nbat = static_cast<unsigned>(std::min(batch - p0, kMaxGridY));
        dim3 gc(static_cast<unsigned>((1LL << k1) >> logw), nbat, 2);
        kcf<<<gc, kThreads, smem_c, st>>>(dp, a, na, b, nb, ws, 2 * N, N, k, k2, logw, p0, nullptr, kb);
        prof_mark(st, tft ? "k_col_fwd_tft" : "k_col_fwd");
        dim3 gr(row_blocks, nbat, 1);
        krp<<<gr, kThreads, smem_r, st>>>(dp, ws, 2 * N, k, k2, lrpc, p0, nullptr, kb);
        prof_mark(st, tft ? "k_row_polymul_tft" : "k_row_polymul");
        dim3 gi(static_cast<unsigned>((1LL << k1) >> logw), nbat, 1);
        kci<<<gi, kThreads, smem_c, st>>>(dp, ws, 2 * N, c, na + nb - 1, k, k2, logw, itab, p0, nullptr, kb,
                                          tft_consts<Ar>(plan));
        prof_mark(st, tft ? "k_col_inv_tft" : "k_col_inv");
    }
    return check_launch("fused polymul passes");
}

template <class Ar>
int launch_polymul_plain(const ntt_plan* plan, const DevPlan<Ar>& dp, const typename Ar::word* a,
                         long long na, const typename Ar::word* b, long long nb, long long batch,
                         typename Ar::word* c, typename Ar::word* ws, typename Ar::tw scale,
                         cudaStream_t st) {
    const int k = static_cast<int>(plan->log2n);
    const long long N = 1LL << k;
    prof_begin_call(st);
    k_plain_load<Ar><<<grid_for(2 * batch * N), kThreads, 0, st>>>(a, na, b, nb, ws, k, batch);
    prof_mark(st, "k_plain_load");
    for (int lh = k - 1; lh >= 0; --lh) {
        k_plain_dif<Ar><<<grid_for(batch * N), kThreads, 0, st>>>(dp, ws, 2 * batch, k, lh);
        prof_mark(st, "k_plain_dif");
    }
    k_plain_pointwise<Ar><<<grid_for(batch * N), kThreads, 0, st>>>(dp, ws, batch * N, batch * N);
    prof_mark(st, "k_plain_pointwise");
    for (int lh = 0; lh < k; ++lh) {
        k_plain_dit<Ar><<<grid_for(batch * N / 2), kThreads, 0, st>>>(dp, ws, batch, k, lh);
        prof_mark(st, "k_plain_dit");
    }
    k_plain_store<Ar><<<grid_for(batch * (na + nb - 1)), kThreads, 0, st>>>(dp, ws, c, na + nb - 1,
                                                                           k, batch, scale);
    prof_mark(st, "k_plain_store");
    return check_launch("plain polymul stages");
}

template <class Ar>
int launch_batch_small(const DevPlan<Ar>* d_plans, const TftConsts<Ar>* d_tfts, const BatchDesc* d_desc,
                       const void* d_items, unsigned nitems, unsigned* d_ticket, const typename Ar::word* a,
                       const typename Ar::word* b, typename Ar::word* c, size_t smem, int grid,
                       cudaStream_t st) {
    if (nitems == 0) return NTT_OK;
    if (allow_smem(k_batch_small<Ar>, smem) != cudaSuccess) return check_launch("smem attr");
    k_batch_small<Ar><<<grid, kThreads, smem, st>>>(
        d_plans, d_tfts, d_desc, static_cast<const SmallItem<Ar>*>(d_items), nitems, d_ticket, a, b, c);
    prof_mark(st, "k_batch_small");
    return check_launch("k_batch_small");
}

// Blocks of the persistent kernel resident per SM at `smem` bytes.
template <class Ar>
int batch_small_occupancy(size_t smem) {
    if (allow_smem(k_batch_small<Ar>, smem) != cudaSuccess) return 1;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_small<Ar>, kThreads, smem) != cudaSuccess)
        return 1;
    return occ > 0 ? occ : 1;
}

template <class Ar>
int launch_batch_bucket(const ntt_plan* plan, const DevPlan<Ar>& dp, const typename Ar::word* a,
                        const typename Ar::word* b, typename Ar::word* c, const BatchDesc* d_desc,
                        long long count, typename Ar::word* ws, typename Ar::tw scale,
                        cudaStream_t st, long long subs, bool tft_bucket) {
    using word = typename Ar::word;
    const int k = static_cast<int>(plan->log2n);
    const LaunchCfg cfg = launch_cfg(sizeof(word), k, plan->tile_max_log);
    if (cfg.logw == 0 && k == 2 * kDLog) return launch_polymul_direct<Ar>(plan, dp, a, 0, b, 0, count, c, ws, d_desc, st);
    if (cfg.logw == 0 && plan->core)
        return launch_polymul_sub<Ar>(plan, dp, a, 0, b, 0, count, c, ws, d_desc, st, subs);
    const int k2 = plan->k2, k1 = plan->k1;
    const long long N = 1LL << k;
    const int logw = cfg.logw, lrpc = cfg.lrpc;
    const size_t smem_c = slab_words(slab_layout(k2, logw)) * sizeof(word);
    const size_t smem_r = layout_words(tile_layout(k1, lrpc + 1)) * sizeof(word);
    const auto* itab = static_cast<const typename Ar::tw*>(plan->glob_inv_pm);
    // a truncating bucket: every product runs the column blocks its own
    // output needs
    const bool tft = tft_bucket && k2 >= 4 && k2 <= kMaxLineLog;
    auto kcf = tft ? k_col_fwd<Ar, false, 0, 0, true> : k_col_fwd<Ar, false>;
    auto kci = tft ? k_col_inv<Ar, 0, 0, true> : k_col_inv<Ar>;
    auto krp = tft ? k_row_polymul<Ar, 0, 0, true> : k_row_polymul<Ar>;
    if (allow_smem(kcf, smem_c) != cudaSuccess || allow_smem(kci, smem_c) != cudaSuccess ||
        allow_smem(krp, smem_r) != cudaSuccess)
        return check_launch("smem attr");
    for (long long p0 = 0; p0 < count; p0 += kMaxGridY) {
        const unsigned nbat = static_cast<unsigned>(std::min(count - p0, kMaxGridY));
        dim3 gc(static_cast<unsigned>((1LL << k1) >> logw), nbat, 2);
        kcf<<<gc, kThreads, smem_c, st>>>(dp, a, 0, b, 0, ws, 2 * N, N, k, k2, logw, p0, d_desc, 16);
        prof_mark(st, tft ? "k_col_fwd_tft" : "k_col_fwd");
        dim3 gr(static_cast<unsigned>((1LL << k2) >> lrpc), nbat, 1);
        krp<<<gr, kThreads, smem_r, st>>>(dp, ws, 2 * N, k, k2, lrpc, p0, d_desc, 16);
        prof_mark(st, tft ? "k_row_polymul_tft" : "k_row_polymul");
        dim3 gi(static_cast<unsigned>((1LL << k1) >> logw), nbat, 1);
        kci<<<gi, kThreads, smem_c, st>>>(dp, ws, 2 * N, c, 0, k, k2, logw, itab, p0, d_desc, 16,
                                          tft_consts<Ar>(plan));
        prof_mark(st, tft ? "k_col_inv_tft" : "k_col_inv");
    }
    return check_launch("batch bucket passes");
}

// forward declaration (defined below)
template <class Ar>
int launch_ntt(const ntt_plan* plan, const DevPlan<Ar>& dp, typename Ar::word* data, long long batch,
               bool fwd, typename Ar::tw scale, cudaStream_t st);

template <int NN>
int launch_polymat_freq_s64(const Shoup64L& ar, const uint64_t* At, const uint64_t* Bt, uint64_t* Ct, int logN,
                            Tw64 r, cudaStream_t st) {
    using S = PmShared64<NN>;
    const size_t smem = S::words * sizeof(uint64_t);
    if (allow_smem(k_polymat_freq_s64<NN>, smem) != cudaSuccess) return check_launch("smem attr");
    const long long N = 1LL << logN;
    const int K = static_cast<int>(std::min<uint64_t>(~uint64_t(0) / (ar.p - 1), 1u << 30));
    k_polymat_freq_s64<NN><<<static_cast<unsigned>((N + S::F - 1) / S::F), S::THREADS, smem, st>>>(
        ar, At, Bt, Ct, logN, r, K);
    return NTT_OK;
}

template <int NN>
int launch_polymat_freq_s(const Mont32& ar, const uint32_t* At, const uint32_t* Bt, uint32_t* Ct, int logN,
                          Tw32 r, int K, cudaStream_t st) {
    using S = PmShared<NN>;
    const size_t smem = S::words * sizeof(uint32_t);
    if (allow_smem(k_polymat_freq_s<NN>, smem) != cudaSuccess) return check_launch("smem attr");
    const long long N = 1LL << logN;
    const uint32_t r1 = static_cast<uint32_t>((uint64_t(1) << 32) % ar.p);
    k_polymat_freq_s<NN><<<static_cast<unsigned>((N + S::F - 1) / S::F), S::THREADS, smem, st>>>(
        ar, At, Bt, Ct, logN, r, r1, K);
    return NTT_OK;
}

// Polynomial matrix product (Section 5.2): transforms of every entry, n x n
// products at every frequency, inverse transforms of the entries of C.
// ws: 3 n^2 rows of n words.
template <class Ar>
int launch_polymat(const ntt_plan* plan, const DevPlan<Ar>& dp, const typename Ar::word* A,
                   const typename Ar::word* B, int n, long long d, typename Ar::word* C,
                   typename Ar::word* ws, typename Ar::tw inv_scale, typename Ar::tw r, cudaStream_t st) {
    const int k = static_cast<int>(plan->log2n);
    const long long N = 1LL << k, nn = static_cast<long long>(n) * n;
    typename Ar::word* At = ws;
    typename Ar::word* Bt = ws + nn * N;
    typename Ar::word* Ct = ws + 2 * nn * N;
    // n = 2^16 with the direct kernels: the column passes read the entries
    // with their zero padding and write C cropped, so no pad or crop pass
    const bool direct = k == 2 * kDLog && launch_cfg(sizeof(typename Ar::word), k, plan->tile_max_log).logw == 0;
    prof_begin_call(st);
    int rc;
    if (direct) {
        constexpr long long NL = 1LL << (2 * kDLog);
        const size_t smem_c = direct_col_smem_words() * sizeof(typename Ar::word);
        const size_t smem_r = direct_ntt_row_smem_words() * sizeof(typename Ar::word);
        const bool zh = 2 * d <= NL;
        auto kcf = zh ? k_col_fwd_d<Ar, true> : k_col_fwd_d<Ar, false>;
        if (allow_smem(kcf, smem_c) != cudaSuccess || allow_smem(k_col_inv_d<Ar>, smem_c) != cudaSuccess ||
            allow_smem(k_row_ntt_d<Ar, true, kDNttRowsPerBlock>, smem_r) != cudaSuccess ||
            allow_smem(k_row_ntt_d<Ar, false, kDNttRowsPerBlock>, smem_r) != cudaSuccess)
            return check_launch("smem attr");
        for (long long p0 = 0; p0 < nn; p0 += kMaxGridY) {
            const unsigned nb = static_cast<unsigned>(std::min(nn - p0, kMaxGridY));
            kcf<<<dim3(kDLine / kDCols, nb, 2), kDThreads, smem_c, st>>>(dp, dp.ar, A, d, d, B, d, d, ws, NL, nn * NL, p0,
                                                                        nullptr, 16);
            prof_mark(st, "k_col_fwd_d");
        }
        for (long long p0 = 0; p0 < 2 * nn; p0 += kMaxGridY) {
            const unsigned nb = static_cast<unsigned>(std::min(2 * nn - p0, kMaxGridY));
            k_row_ntt_d<Ar, true, kDNttRowsPerBlock>
                <<<dim3(kDLine / kDNttRowsPerBlock, nb, 1), kDNttRowsPerBlock * 16, smem_r, st>>>(dp, ws, p0);
            prof_mark(st, "k_row_ntt_fwd_d");
        }
    } else {
        k_polymat_pad<Ar><<<grid_for(2 * nn * N), kThreads, 0, st>>>(A, B, ws, nn, d, k);
        prof_mark(st, "k_polymat_pad");
        rc = launch_ntt<Ar>(plan, dp, At, 2 * nn, true, inv_scale, st);
        if (rc != NTT_OK) return rc;
    }
    {
        const long long nt1 = (n + 3) / 4, warps = nt1 * nt1 * ((N + 31) >> 5);
        const unsigned blocks = static_cast<unsigned>((warps + 7) / 8);
        typename Ar::tw one = r;
        int K = 1;
        if constexpr (std::is_same<Ar, Mont32>::value) {
            const uint64_t p = dp.ar.p, pm1 = p - 1;
            one.w = static_cast<uint32_t>((uint64_t(1) << 32) % p);     // 1 in Montgomery form
            one.c = one.w * dp.ar.pinv;
            K = pm1 == 0 ? 1 << 30 : static_cast<int>(std::min<uint64_t>(~uint64_t(0) / (pm1 * pm1), 1u << 30));
        }
        bool done = false;
        if constexpr (std::is_same<Ar, Mont32>::value) {
            if (n == 8 || n == 16 || n == 32) {
                const int rc = n == 8    ? launch_polymat_freq_s<8>(dp.ar, At, Bt, Ct, k, r, K, st)
                               : n == 16 ? launch_polymat_freq_s<16>(dp.ar, At, Bt, Ct, k, r, K, st)
                                         : launch_polymat_freq_s<32>(dp.ar, At, Bt, Ct, k, r, K, st);
                if (rc != NTT_OK) return rc;
                done = true;
            }
        } else if constexpr (std::is_same<Ar, Shoup64L>::value) {
            if (n == 8 || n == 16 || n == 32) {
                const int rc = n == 8    ? launch_polymat_freq_s64<8>(dp.ar, At, Bt, Ct, k, r, st)
                               : n == 16 ? launch_polymat_freq_s64<16>(dp.ar, At, Bt, Ct, k, r, st)
                                         : launch_polymat_freq_s64<32>(dp.ar, At, Bt, Ct, k, r, st);
                if (rc != NTT_OK) return rc;
                done = true;
            }
        }
        if (done) {
        } else if (K >= 3)
            k_polymat_freq<Ar, true><<<blocks, 256, 0, st>>>(dp.ar, At, Bt, Ct, n, k, r, one, K);
        else
            k_polymat_freq<Ar, false><<<blocks, 256, 0, st>>>(dp.ar, At, Bt, Ct, n, k, r, one, K);
        prof_mark(st, "k_polymat_freq");
    }
    if (direct) {
        constexpr long long NL = 1LL << (2 * kDLog);
        const size_t smem_c = direct_col_smem_words() * sizeof(typename Ar::word);
        const size_t smem_r = direct_ntt_row_smem_words() * sizeof(typename Ar::word);
        for (long long p0 = 0; p0 < nn; p0 += kMaxGridY) {
            const unsigned nb = static_cast<unsigned>(std::min(nn - p0, kMaxGridY));
            k_row_ntt_d<Ar, false, kDNttRowsPerBlock>
                <<<dim3(kDLine / kDNttRowsPerBlock, nb, 1), kDNttRowsPerBlock * 16, smem_r, st>>>(dp, Ct, p0);
            prof_mark(st, "k_row_ntt_inv_d");
            k_col_inv_d<Ar><<<dim3(kDLine / kDCols, nb, 1), kDThreads, smem_c, st>>>(dp, wide_form(dp.ar), Ct, NL, C, 2 * d - 1,
                                                                                    2 * d - 1, dp.glob_inv, dp.wglob[1], p0,
                                                                                    nullptr, 16, TftConsts<Ar>{});
            prof_mark(st, "k_col_inv_d");
        }
        return check_launch("polymat kernels");
    }
    rc = launch_ntt<Ar>(plan, dp, Ct, nn, false, inv_scale, st);
    if (rc != NTT_OK) return rc;
    k_polymat_crop<Ar><<<grid_for(nn * (2 * d - 1)), kThreads, 0, st>>>(dp.ar, Ct, C, nn, 2 * d - 1, k);
    prof_mark(st, "k_polymat_crop");
    return check_launch("polymat kernels");
}

template <class Ar>
int launch_ntt(const ntt_plan* plan, const DevPlan<Ar>& dp, typename Ar::word* data, long long batch,
               bool fwd, typename Ar::tw scale, cudaStream_t st) {
    using word = typename Ar::word;
    const int k = static_cast<int>(plan->log2n);
    if (k <= plan->tile_max_log) {
        const int lppc = (k <= kMaxLineLog) ? 5 : 0;
        const size_t smem = layout_words(tile_layout(k, lppc)) * sizeof(word);
        auto kern = fwd ? k_tile_ntt<Ar, true> : k_tile_ntt<Ar, false>;
        if (allow_smem(kern, smem) != cudaSuccess) return check_launch("smem attr");
        const long long blocks = (batch + (1LL << lppc) - 1) >> lppc;
        prof_begin_call(st);
        kern<<<static_cast<unsigned>(blocks), kThreads, smem, st>>>(dp, data, batch, k, lppc, scale);
        prof_mark(st, fwd ? "k_tile_ntt_fwd" : "k_tile_ntt_inv");
        return check_launch("k_tile_ntt");
    }
    const int k2 = plan->k2, k1 = plan->k1;
    const long long N = 1LL << k;
    int logw = launch_cfg(sizeof(word), k, plan->tile_max_log).logw;
    if (logw == 0) {
        if ((reinterpret_cast<uintptr_t>(data) & 15) == 0) {
            if (k == 2 * kDLog) return launch_ntt_direct<Ar>(dp, data, batch, fwd, st);
            if (plan->core) return launch_ntt_sub<Ar>(plan, dp, data, batch, fwd, st);
        }
        logw = generic_global_cfg(sizeof(word), k).logw;
    }
    const size_t smem_c = slab_words(slab_layout(k2, logw)) * sizeof(word);
    const int lrpc = row_lrpc(k1, 1);
    const size_t smem_r = layout_words(tile_layout(k1, lrpc)) * sizeof(word);
    auto krow = fwd ? k_row_ntt<Ar, true> : k_row_ntt<Ar, false>;
    if (allow_smem(k_col_fwd<Ar, false>, smem_c) != cudaSuccess ||
        allow_smem(k_col_inv<Ar>, smem_c) != cudaSuccess || allow_smem(krow, smem_r) != cudaSuccess)
        return check_launch("smem attr");
    prof_begin_call(st);
    for (long long p0 = 0; p0 < batch; p0 += kMaxGridY) {
        const unsigned nbat = static_cast<unsigned>(std::min(batch - p0, kMaxGridY));
        dim3 gc(static_cast<unsigned>((1LL << k1) >> logw), nbat, 1);
        dim3 gr(static_cast<unsigned>((1LL << k2) >> lrpc), nbat, 1);
        if (fwd) {
            k_col_fwd<Ar, false><<<gc, kThreads, smem_c, st>>>(dp, data, N, data, N, data, N, 0, k, k2,
                                                               logw, p0, nullptr, 16);
            prof_mark(st, "k_col_fwd");
            krow<<<gr, kThreads, smem_r, st>>>(dp, data, k, k2, lrpc, p0);
            prof_mark(st, "k_row_ntt_fwd");
        } else {
            krow<<<gr, kThreads, smem_r, st>>>(dp, data, k, k2, lrpc, p0);
            prof_mark(st, "k_row_ntt_inv");
            k_col_inv<Ar><<<gc, kThreads, smem_c, st>>>(dp, data, N, data, N, k, k2, logw, dp.glob_inv,
                                                        p0, nullptr, 16, TftConsts<Ar>{});
            prof_mark(st, "k_col_inv");
        }
    }
    return check_launch("ntt passes");
}

}  // namespace gbntt
