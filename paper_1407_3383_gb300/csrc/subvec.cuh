// Transforms of n = 2^17 .. 2^24 points as Algorithm 1 with n1 = 2^16 and
// n2 = n / 2^16 (Section 5.1): step 1 is an n2-point transform across the
// sub-vectors, step 2 the twiddle w_n^(j1 [j2]), step 3 the 2^16-point
// transforms of the n2 rows (the direct kernels of the plan's 2^16-point
// child plan).  For n2 <= 16 one thread owns column j1 of the n2 x 2^16
// array and keeps its n2 words in registers; for n2 = 32 .. 256 the columns
// go through a column kernel shaped like the direct 2^16-point one.
//
// Products take the TFT at this level too: a product of L output words
// needs only lam = ceil(L / 2^16) of the n2 rows (step 1 truncated to lam
// outputs, step 3 on lam rows, and the inverse TFT across the rows at the
// end).  Rows go to the workspace interleaved -- row j2 of operand a at
// (prod lam + j2) 2^17, of b 2^16 further -- so that the 2^16-point stage
// sees a uniform batch of sub-products.
#pragma once
#include "direct.cuh"
#include "tft.cuh"

namespace gbntt {

constexpr int kSubLog = 16;
constexpr long long kSubN = 1LL << kSubLog;
constexpr int kSubThreads = 256;

// Steps 1 and 2: read rows j2 < M of every product's operand (zero beyond
// its length), M-point DIF across them (truncated to lam outputs with TFT),
// twiddle, and write row j2 < lam to dst + prod*dprod + j2*dsub (+ doff1 for
// operand b, blockIdx.z = 1).  In place when dst is the source.  With
// descriptors and TFT, lam is the product's own ceil(L / 2^16) and its rows
// start at slot d.sub: dst + (d.sub + j2)*dsub.
template <class Ar, int M, bool TFT>
__global__ void __launch_bounds__(kSubThreads)
k_pre_fwd(Ar ar, DevPlan<Ar> P, const typename Ar::word* __restrict__ src0, long long len0, long long sstride0,
          const typename Ar::word* __restrict__ src1, long long len1, long long sstride1,
          typename Ar::word* dst, long long dprod, long long dsub, long long doff1,
          const typename Ar::tw* __restrict__ pre, long long prod_base, const BatchDesc* __restrict__ desc,
          int lam) {
    using word = typename Ar::word;
    const long long j1 = static_cast<long long>(blockIdx.x) * kSubThreads + threadIdx.x;
    const long long prod = prod_base + blockIdx.y;
    const word* src;
    long long len, first = prod * dprod;
    if (desc) {
        const BatchDesc d = desc[prod];
        src = blockIdx.z ? src1 + d.boff : src0 + d.aoff;
        len = blockIdx.z ? d.nb : d.na;
        if (TFT) {
            lam = static_cast<int>(std::min<long long>(M, (static_cast<long long>(d.na) + d.nb - 1 + kSubN - 1) / kSubN));
            first = static_cast<long long>(d.sub) * dsub;
        }
    } else {
        src = blockIdx.z ? src1 + prod * sstride1 : src0 + prod * sstride0;
        len = blockIdx.z ? len1 : len0;
    }
    word x[16];
#pragma unroll
    for (int j2 = 0; j2 < 16; ++j2) {
        x[j2] = word(0);
        if (j2 < M && j2 * kSubN + j1 < len) x[j2] = src[j2 * kSubN + j1];
    }
    if (TFT)
        tdif<Ar, M, 0>(ar, x, P.rc, lam);
    else
        dif_sub<Ar, M, 0>(ar, x, P.rc);
    word* out = dst + first + (blockIdx.z ? doff1 : 0) + j1;
#pragma unroll
    for (int j2 = 0; j2 < M; ++j2)
        if (!TFT || j2 < lam) out[j2 * dsub] = ar.mulw(x[j2], pre[j2 * kSubN + j1]);
}

// The inverse: rows j2 < lam of src + prod*sprod + j2*ssub, inverse twiddle
// (with n2^-1 folded into pre_inv), inverse M-point transform across the
// rows (the inverse TFT with zero inputs above lam, with TFT), canonical
// store of the first out_len words at dst + prod*dprod (or the descriptor's
// offset and length; with descriptors and TFT the product's own lam and row
// slots from d.sub, as in k_pre_fwd).
template <class Ar, int M, bool TFT>
__global__ void __launch_bounds__(kSubThreads)
k_post_inv(Ar ar, DevPlan<Ar> P, TftConsts<Ar> K, const typename Ar::word* src, long long sprod, long long ssub,
           typename Ar::word* dst, long long out_len, long long dprod, const typename Ar::tw* __restrict__ pre_inv,
           long long prod_base, const BatchDesc* __restrict__ desc, int lam) {
    using word = typename Ar::word;
    const long long j1 = static_cast<long long>(blockIdx.x) * kSubThreads + threadIdx.x;
    const long long prod = prod_base + blockIdx.y;
    long long first = prod * sprod;
    if (desc && TFT) {
        const BatchDesc d = desc[prod];
        lam = static_cast<int>(std::min<long long>(M, (static_cast<long long>(d.na) + d.nb - 1 + kSubN - 1) / kSubN));
        first = static_cast<long long>(d.sub) * ssub;
    }
    const word* in = src + first + j1;
    word x[16];
#pragma unroll
    for (int j2 = 0; j2 < 16; ++j2) {
        x[j2] = word(0);
        if (j2 < M && (!TFT || j2 < lam)) x[j2] = ar.mulw(in[j2 * ssub], pre_inv[j2 * kSubN + j1]);
    }
    if (TFT && lam >= M) {
        // every row kept (uneven batches): the plain inverse, same residues
        dit_sub<Ar, M, 0>(ar, x, P.rci);
    } else if (TFT) {
        // the inverse TFT returns 16 times its inputs, which pre_inv scaled
        // by 1/M: multiply by M/16
        itft_z<Ar, M, 0>(ar, x, P.rc, P.rci, K, lam);
        if (M < 16) {
#pragma unroll
            for (int j2 = 0; j2 < M; ++j2) x[j2] = ar.mulw(x[j2], K.inv2k[4 - Log2<M>::v]);
        }
    } else {
        dit_sub<Ar, M, 0>(ar, x, P.rci);
    }
    word* out;
    long long len;
    if (desc) {
        const BatchDesc d = desc[prod];
        out = dst + d.coff;
        len = static_cast<long long>(d.na) + d.nb - 1;
    } else {
        out = dst + prod * dprod;
        len = out_len;
    }
#pragma unroll
    for (int j2 = 0; j2 < M; ++j2)
        if (j2 * kSubN + j1 < len) out[j2 * kSubN + j1] = ar.canon(x[j2]);
}

// Steps 1 and 2 for n2 = 2^C = 32 .. 256 rows: each column of the
// n2 x 2^16 array (rows at stride 2^16) is transformed like a column of the
// direct 2^16-point kernels, split 16 x R2 (R2 = n2 / 16): an outer radix-16
// pass on rows R2 t + j1 with the twiddle w_(n2)^(j1 [t]_4) of the plan's
// line table, an inner radix-R2 pass on blocks of R2 positions, then the
// step-2 twiddle w_n^(c [pos]_C); position pos goes to dst + prod*dprod +
// pos*dsub (+ doff1 for operand b).  32 columns per block.  ZHALF: rows at or
// beyond n2/2 are zero.  TFT: only the first B of the 16 blocks are formed;
// with descriptors, B is the product's own and its rows start at slot d.sub.
template <class Ar, int C, bool ZHALF, bool TFT>
__global__ void __launch_bounds__(kDThreads)
k_colx_fwd(DevPlan<Ar> P, const typename Ar::word* __restrict__ src0, long long len0, long long sstride0,
           const typename Ar::word* __restrict__ src1, long long len1, long long sstride1, typename Ar::word* dst,
           long long dprod, long long dsub, long long doff1, const typename Ar::tw* __restrict__ pre,
           long long prod_base, const BatchDesc* __restrict__ desc, int beta) {
    using word = typename Ar::word;
    constexpr int LC = 1 << C, R2 = LC / 16;
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    const int v = threadIdx.x & (kDCols - 1), g = threadIdx.x / kDCols;
    const long long c = static_cast<long long>(blockIdx.x) * kDCols + v;
    const long long prod = prod_base + blockIdx.y;
    const word* src;
    long long len, first = prod * dprod;
    int B = 16;
    if (desc) {
        const BatchDesc d = desc[prod];
        src = blockIdx.z ? src1 + d.boff : src0 + d.aoff;
        len = blockIdx.z ? d.nb : d.na;
        if (TFT) {
            const long long lam = (static_cast<long long>(d.na) + d.nb - 1 + kSubN - 1) / kSubN;
            B = static_cast<int>((lam + R2 - 1) / R2);
            first = static_cast<long long>(d.sub) * dsub;
        }
    } else {
        src = blockIdx.z ? src1 + prod * sstride1 : src0 + prod * sstride0;
        len = blockIdx.z ? len1 : len0;
        if (TFT) B = beta;
    }
    const typename Ar::tw* ltab = P.line_fwd[C];
#pragma unroll
    for (int i = 0; i < (R2 + kDGroups - 1) / kDGroups; ++i) {
        const int j1 = g + kDGroups * i;
        if (j1 >= R2) break;
        word x[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const long long e = static_cast<long long>(R2 * t + j1) * kSubN + c;
            x[t] = word(0);
            if ((!ZHALF || t < 8) && e < len) x[t] = src[e];
        }
        if (TFT)
            tdif16<Ar, ZHALF>(P.ar, x, P.rc, B);
        else
            dif_regs<Ar, 16, ZHALF>(P.ar, x, P.rc);
#pragma unroll
        for (int t = 1; t < 16; ++t)
            if (!TFT || t < B) x[t] = P.ar.mulw(x[t], ltab[j1 * 16 + t]);
#pragma unroll
        for (int t = 0; t < 16; ++t)
            if (!TFT || t < B) sm[(R2 * t + j1) * kDCols + v] = x[t];
    }
    __syncthreads();
    word* out = dst + first + (blockIdx.z ? doff1 : 0) + c;
#pragma unroll
    for (int i = 0; i < kDItems; ++i) {
        const int blk = g + kDGroups * i;
        if (TFT && blk >= B) continue;
        word x[16];
#pragma unroll
        for (int t = 0; t < R2; ++t) x[t] = sm[(R2 * blk + t) * kDCols + v];
        dif_sub<Ar, R2, 0>(P.ar, x, P.rc);
#pragma unroll
        for (int t = 0; t < R2; ++t) {
            const long long pos = R2 * blk + t;
            out[pos * dsub] = P.ar.mulw(x[t], pre[pos * kSubN + c]);
        }
    }
}

// The inverse of k_colx_fwd: positions of the B formed blocks read from
// src + prod*sprod + pos*ssub, inverse step-2 twiddle (n2^-1 folded into
// pre_inv), inverse radix-R2 pass, inverse outer pass (the inverse TFT with
// TFT), canonical store of the first out_len words of the product at
// dst + prod*dprod (or the descriptor's offset and length), row stride 2^16.
template <class Ar, int C, bool TFT>
__global__ void __launch_bounds__(kDThreads)
k_colx_inv(DevPlan<Ar> P, TftConsts<Ar> K, const typename Ar::word* src, long long sprod, long long ssub,
           typename Ar::word* dst, long long out_len, long long dprod, const typename Ar::tw* __restrict__ pre_inv,
           long long prod_base, const BatchDesc* __restrict__ desc, int beta) {
    using word = typename Ar::word;
    constexpr int LC = 1 << C, R2 = LC / 16;
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    const int v = threadIdx.x & (kDCols - 1), g = threadIdx.x / kDCols;
    const long long c = static_cast<long long>(blockIdx.x) * kDCols + v;
    const long long prod = prod_base + blockIdx.y;
    word* out;
    long long len, first = prod * sprod;
    int B = 16;
    if (desc) {
        const BatchDesc d = desc[prod];
        out = dst + d.coff;
        len = static_cast<long long>(d.na) + d.nb - 1;
        if (TFT) {
            B = static_cast<int>(((len + kSubN - 1) / kSubN + R2 - 1) / R2);
            first = static_cast<long long>(d.sub) * ssub;
        }
    } else {
        out = dst + prod * dprod;
        len = out_len;
        if (TFT) B = beta;
    }
    const word* in = src + first + c;
#pragma unroll
    for (int i = 0; i < kDItems; ++i) {
        const int blk = g + kDGroups * i;
        if (TFT && blk >= B) continue;
        word x[16];
#pragma unroll
        for (int t = 0; t < R2; ++t) {
            const long long pos = R2 * blk + t;
            x[t] = P.ar.mulw(in[pos * ssub], pre_inv[pos * kSubN + c]);
        }
        dit_sub<Ar, R2, 0>(P.ar, x, P.rci);
#pragma unroll
        for (int t = 0; t < R2; ++t) sm[(R2 * blk + t) * kDCols + v] = x[t];
    }
    __syncthreads();
    const typename Ar::tw* ltab = P.line_inv[C];
#pragma unroll
    for (int i = 0; i < (R2 + kDGroups - 1) / kDGroups; ++i) {
        const int j1 = g + kDGroups * i;
        if (j1 >= R2) break;
        word x[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = (!TFT || t < B) ? sm[(R2 * t + j1) * kDCols + v] : word(0);
#pragma unroll
        for (int t = 1; t < 16; ++t)
            if (!TFT || t < B) x[t] = P.ar.mulw(x[t], ltab[j1 * 16 + t]);
        if (TFT)
            itft16_z16(P.ar, x, P.rc, P.rci, K, B);
        else
            dit_regs<Ar, 16>(P.ar, x, P.rci);
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const long long e = static_cast<long long>(R2 * t + j1) * kSubN + c;
            if (e < len) out[e] = P.ar.canon(x[t]);
        }
    }
}

}  // namespace gbntt
