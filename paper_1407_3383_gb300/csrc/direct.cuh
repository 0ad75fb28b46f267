// Direct kernels for products of n = 2^16 = 256 x 256 points.
//
// The same decomposition as the generic global schedule (Algorithm 1 at the
// global level, n = n2 x n1 with n1 = n2 = 256, and every 256-word line once
// more split 16 x 16), but the two radix-16 passes of a line are arranged so
// that global memory is read by the first pass straight into registers and
// written by the last pass straight from registers.  Every word crosses
// shared memory once per kernel (one store, one load), and the row kernel
// keeps both operands' inner 16-point transforms, their pointwise product
// and the first inverse pass of the product in one thread's registers.
//
// Positions and twiddles agree word for word with the generic engine:
//   outer pass (sub-transform size 256): a thread owns column j1 of the
//       16 x 16 split of a line and holds rows t = 0..15, i.e. line
//       positions 16 t + j1; DIF-16, then w_256^(j1 [t]_4) on register t;
//   inner pass (size 16): a thread owns block `blk`, positions 16 blk + t;
//       DIF-16 (bit-mirrored result in place), then in the column kernel
//       the global twiddle w_n^(c [pos]_8) of Algorithm 1's step 2.
// The inverse kernels run the same passes in reverse with w^-1 (DIT), the
// twiddle of each pass applied before its butterflies.
#pragma once
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "engine.cuh"
#include "tft.cuh"
#include "tma.cuh"

namespace gbntt {

constexpr int kDLog = 8;                         // line length 2^8 in both directions
constexpr int kDLine = 1 << kDLog;
constexpr int kDCols = 32;                       // columns per column block (one per lane)
constexpr int kDThreads = 256;
constexpr int kDGroups = kDThreads / kDCols;     // warps of a column block
constexpr int kDItems = 16 / kDGroups;           // 16-point columns or blocks per thread
static_assert(kDItems * kDGroups == 16, "column blocks cover 16 x 16 lines");
// Column blocks per SM the compiler must fit with 32-bit words: 4 leaves up
// to 64 registers a thread, which measured 4% faster per product step than
// the 32-48 the compiler picks unbounded (more loads in flight per thread).
// 64-bit words would spill under that bound.  For them 3 blocks (up to 85
// registers, with the step-2 twiddles loaded and applied in two halves) run
// the column pass 5% faster than 2 blocks (128 registers), which in turn
// were 37% faster than the 168 registers the compiler picks unbounded.
constexpr int kDColMinBlocks = 4;
constexpr int kDColMinBlocks64 = 3;   // 64-bit words: up to 85 registers (step-2 twiddles in two halves)
constexpr int kDColInvMinBlocks64 = 3;   // the inverse column pass fits 3 blocks (up to 85) without spilling

__host__ __device__ constexpr size_t direct_col_smem_words() { return size_t(kDCols) * kDLine; }

// A twiddle from a table of (multiplicand, companion) pairs.  CTW with the
// 32-bit Montgomery policies reads the multiplicand w~ alone: Mont32 forms
// its companion w~ p^-1 rem 2^32 with one multiply, Mont32W needs none.
// Half the table traffic, and half the registers when the compiler keeps a
// thread's twiddles live.
template <class Ar, bool CTW>
__device__ __forceinline__ typename Ar::tw load_tw(const Ar& ar, const typename Ar::tw* p) {
    if constexpr (CTW && std::is_base_of<Mont32, Ar>::value) {
        const uint32_t w = p->w;
        return Tw32{w, Ar::kWide ? 0u : w * ar.pinv};
    } else {
        return *p;
    }
}

// Twiddle i of a plan table.  The 32-bit Montgomery policies read the
// multiplicand alone from the table's 4-byte copy `w` (whole sectors per
// warp; the pairs would bring in every companion too), other policies the
// (multiplicand, companion) pair.
template <class Ax>
__device__ __forceinline__ typename Ax::tw tw_at(const Ax& ar, const typename Ax::tw* pairs, const uint32_t* w,
                                                 long long i) {
    if constexpr (std::is_base_of<Mont32, Ax>::value) {
        const uint32_t x = w[i];
        return Tw32{x, Ax::kWide ? 0u : x * ar.pinv};
    } else {
        return pairs[i];
    }
}

// 16-row blocks of the column transforms that a product of `len` output
// words needs (the TFT length rounded up to whole blocks: 1..16).
__host__ __device__ inline int tft_blocks(long long len) {
    const long long b = (len + 16 * kDLine - 1) / (16 * kDLine);
    return static_cast<int>(b < 1 ? 1 : (b > 16 ? 16 : b));
}

// Number of leading rows (of 256 words) of column c that lie inside an
// operand of `len` words: row r holds word r*256 + c.
__device__ __forceinline__ int dcol_rows(long long len, long long c) {
    const long long lim = len - c;
    if (lim <= 0) return 0;
    return static_cast<int>(std::min<long long>(kDLine, (lim + kDLine - 1) >> kDLog));
}

// Pass 1: forward column transforms of 32 columns of one operand (blockIdx.z
// selects a or b), zero padding beyond the operand's length, the global
// twiddle, and the store into the workspace.  ZHALF: rows >= 128 are all
// padding (both operands have at most n/2 words).  TFT: only the first
// 16 B rows of the transform are formed (B = beta, or from the descriptor's
// product length): the truncated Fourier transform of Section 5.1 with
// Algorithm 1's rows, its outer 16-point pass truncated to B outputs.
template <class Ar, bool ZHALF, bool TFT = false>
__global__ void __launch_bounds__(kDThreads, sizeof(typename Ar::word) == 4 ? kDColMinBlocks : kDColMinBlocks64)
k_col_fwd_d(DevPlan<Ar> P, const Ar ar, const typename Ar::word* __restrict__ src0, long long len0, long long sstride0,
            const typename Ar::word* __restrict__ src1, long long len1, long long sstride1,
            typename Ar::word* __restrict__ dst, long long dst_stride, long long dst_off1, long long prod_base,
            const BatchDesc* __restrict__ desc, int beta) {
    using word = typename Ar::word;
    using tw = typename Ar::tw;
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    const int v = threadIdx.x & (kDCols - 1), g = threadIdx.x / kDCols;
    const long long c0 = static_cast<long long>(blockIdx.x) * kDCols;
    const long long prod = prod_base + blockIdx.y;
    const word* src;
    long long len;
    int B = 16;
    if (desc) {
        const BatchDesc d = desc[prod];
        src = blockIdx.z ? src1 + d.boff : src0 + d.aoff;
        len = blockIdx.z ? d.nb : d.na;
        if (TFT) B = tft_blocks(static_cast<long long>(d.na) + d.nb - 1);
    } else {
        len = blockIdx.z ? len1 : len0;
        src = blockIdx.z ? src1 + prod * sstride1 : src0 + prod * sstride0;
        if (TFT) B = beta;
    }
    const int rows = dcol_rows(len, c0 + v);
    const word* in = src + c0 + v;
    const tw* ltab = P.line_fwd[kDLog];
    const uint32_t* ltab_w = P.wline[0];
#pragma unroll
    for (int i = 0; i < kDItems; ++i) {
        const int j1 = g + kDGroups * i;
        word x[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int row = 16 * t + j1;
            x[t] = word(0);
            if ((!ZHALF || t < 8) && row < rows) x[t] = in[static_cast<long long>(row) * kDLine];
        }
        if (TFT)
            tdif16<Ar, ZHALF>(ar, x, P.rc, B);
        else
            dif_regs<Ar, 16, ZHALF>(ar, x, P.rc);
#pragma unroll
        for (int t = 1; t < 16; ++t)
            if (!TFT || t < B) x[t] = ar.mulw(x[t], tw_at(ar, ltab, ltab_w, j1 * 16 + t));
#pragma unroll
        for (int t = 0; t < 16; ++t)
            if (!TFT || t < B) sm[(16 * t + j1) * kDCols + v] = x[t];
    }
    __syncthreads();
    word* out = dst + prod * dst_stride + (blockIdx.z ? dst_off1 : 0) + c0 + v;
    const tw* gt = P.glob_fwd + c0 + v;
    const uint32_t* gt_w = P.wglob[0] ? P.wglob[0] + c0 + v : nullptr;
#pragma unroll
    for (int i = 0; i < kDItems; ++i) {
        const int blk = g + kDGroups * i;
        if (TFT && blk >= B) continue;
        // the step-2 twiddles are loaded before any store to dst: the
        // compiler cannot prove that the plan tables and dst do not
        // overlap, and a load after a store would wait for it (16 L2 round
        // trips one after another instead of one)
        tw w[16];
        if constexpr (sizeof(word) == 4) {            // 32-bit words: before the pass, to overlap it
#pragma unroll
            for (int t = 0; t < 16; ++t) w[t] = tw_at(ar, gt, gt_w, (16 * blk + t) * kDLine);
        }
        word x[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = sm[(16 * blk + t) * kDCols + v];
        dif_regs<Ar, 16>(ar, x, P.rc);
        if constexpr (sizeof(word) != 4) {            // wider words: after it, in two halves (register pressure)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int t = 8 * h; t < 8 * h + 8; ++t) w[t] = tw_at(ar, gt, gt_w, (16 * blk + t) * kDLine);
#pragma unroll
                for (int t = 8 * h; t < 8 * h + 8; ++t) out[(16 * blk + t) * kDLine] = ar.mulw(x[t], w[t]);
            }
        } else {
#pragma unroll
            for (int t = 0; t < 16; ++t) out[(16 * blk + t) * kDLine] = ar.mulw(x[t], w[t]);
        }
    }
}

// k_col_fwd_d for uniform batches of zero-half operands made of whole
// 256-word rows, with the input tile brought in by one TMA copy: operand z of
// product prod is the 3-D tensor (256 columns, na/256 rows, batch) of
// map_a / map_b, and the box (32 columns, 128 rows) at (c0, 0, prod) -- rows
// past the operand are the copy's zero fill -- lands in shared memory in the
// layout the outer pass reads (row r, column v at r*32 + v).  Each thread
// then reads its 8 rows 16 t + j1 and writes its 16 outputs to the same
// positions, which no other thread touches.
template <class Ar, bool TFT>
__global__ void __launch_bounds__(kDThreads)
k_col_fwd_tma(DevPlan<Ar> P, const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
              typename Ar::word* __restrict__ dst, long long dst_stride, long long dst_off1, long long prod_base,
              int beta, int* err) {
    using word = typename Ar::word;
    using tw = typename Ar::tw;
    extern __shared__ __align__(128) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + direct_col_smem_words() * sizeof(word));
    const int v = threadIdx.x & (kDCols - 1), g = threadIdx.x / kDCols;
    const long long c0 = static_cast<long long>(blockIdx.x) * kDCols;
    const long long prod = prod_base + blockIdx.y;
    const CUtensorMap* map = blockIdx.z ? &map_b : &map_a;
    if (!tma_block_load_3d(sm, map, static_cast<int>(c0), 0, static_cast<int>(prod),
                           static_cast<unsigned>(kDCols * (kDLine / 2) * sizeof(word)), bar, err))
        return;
    const int B = TFT ? beta : 16;
    const tw* ltab = P.line_fwd[kDLog];
    const uint32_t* ltab_w = P.wline[0];
#pragma unroll
    for (int i = 0; i < kDItems; ++i) {
        const int j1 = g + kDGroups * i;
        word x[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = (t < 8) ? sm[(16 * t + j1) * kDCols + v] : word(0);
        if (TFT)
            tdif16<Ar, true>(P.ar, x, P.rc, B);
        else
            dif_regs<Ar, 16, true>(P.ar, x, P.rc);
#pragma unroll
        for (int t = 1; t < 16; ++t)
            if (!TFT || t < B) x[t] = P.ar.mulw(x[t], tw_at(P.ar, ltab, ltab_w, j1 * 16 + t));
#pragma unroll
        for (int t = 0; t < 16; ++t)
            if (!TFT || t < B) sm[(16 * t + j1) * kDCols + v] = x[t];
    }
    __syncthreads();
    word* out = dst + prod * dst_stride + (blockIdx.z ? dst_off1 : 0) + c0 + v;
    const tw* gt = P.glob_fwd + c0 + v;
    const uint32_t* gt_w = P.wglob[0] ? P.wglob[0] + c0 + v : nullptr;
#pragma unroll
    for (int i = 0; i < kDItems; ++i) {
        const int blk = g + kDGroups * i;
        if (TFT && blk >= B) continue;
        tw w[16];                                     // loaded before the stores (see k_col_fwd_d)
#pragma unroll
        for (int t = 0; t < 16; ++t) w[t] = tw_at(P.ar, gt, gt_w, (16 * blk + t) * kDLine);
        word x[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = sm[(16 * blk + t) * kDCols + v];
        dif_regs<Ar, 16>(P.ar, x, P.rc);
#pragma unroll
        for (int t = 0; t < 16; ++t) out[(16 * blk + t) * kDLine] = P.ar.mulw(x[t], w[t]);
    }
}

// 16 consecutive words of shared memory (16-byte aligned) as 16-byte vectors.
template <class W> struct Vec16;
template <> struct Vec16<uint32_t> { using type = uint4; };
template <> struct Vec16<uint64_t> { using type = ulonglong2; };
template <> struct Vec16<double> { using type = double2; };

template <class word>
__device__ __forceinline__ void sm_load16(const word* p, word (&x)[16]) {
    using V = typename Vec16<word>::type;
    constexpr int per = 16 / sizeof(word);
#pragma unroll
    for (int q = 0; q < 16 / per; ++q) {
        const V v = reinterpret_cast<const V*>(p)[q];
        word tmp[per];
        memcpy(tmp, &v, 16);
#pragma unroll
        for (int e = 0; e < per; ++e) x[q * per + e] = tmp[e];
    }
}

template <class word>
__device__ __forceinline__ void sm_store16(word* p, const word (&x)[16]) {
    using V = typename Vec16<word>::type;
    constexpr int per = 16 / sizeof(word);
#pragma unroll
    for (int q = 0; q < 16 / per; ++q) {
        word tmp[per];
#pragma unroll
        for (int e = 0; e < per; ++e) tmp[e] = x[q * per + e];
        V v;
        memcpy(&v, tmp, 16);
        reinterpret_cast<V*>(p)[q] = v;
    }
}

// Row-kernel shared layout: four pad words after every 16 positions
// (stride 20 per block of 16, 336 per line).  A thread's 16 consecutive
// positions of the inner pass are then 16-byte aligned and move as four
// 16-byte vectors without bank conflicts (the 8 lanes of a quarter warp hit
// 8 disjoint groups of 4 banks), and the scalar accesses of the outer passes
// are conflict-free because the two lines a warp touches differ by 16 banks.
struct RowLayout {
    static constexpr int kBlk = 20;
    static constexpr int kLine = 16 * kBlk + 16;
    __device__ __forceinline__ static int at(int line, int pos) { return line * kLine + (pos >> 4) * kBlk + (pos & 15); }
};

constexpr int kDRowsPerBlock = 4;      // rows of each operand per row block (64 threads)
constexpr int kDRowMinBlocks32 = 16;   // 32-bit words: 16 blocks per SM (up to 64 registers)
constexpr int kDRowMinBlocks64 = 10;  // 64-bit words: up to 96 registers (half the line twiddles live at once)   // 64-bit words: up to 128 registers
constexpr int kDNttRowsPerBlock = 8;   // standalone row transforms (128 threads)
constexpr int kDTftMaxBlocks = 13;     // uniform batches needing more row blocks run the full kernels

__host__ __device__ constexpr size_t direct_row_smem_words() { return size_t(2 * kDRowsPerBlock) * RowLayout::kLine; }
__host__ __device__ constexpr size_t direct_ntt_row_smem_words() { return size_t(kDNttRowsPerBlock) * RowLayout::kLine; }

// The row and inverse-column kernels take their arithmetic policy as a
// kernel parameter of its own (WideForm: Mont32W for 32-bit words) rather
// than reading it from the plan structure: measured on the 2^16-point
// benchmark product, the compiler then issues about 18% fewer instructions
// in the row kernel (0.1065 -> 0.0922 ms for 256 products).
//
// Pass 2: RPB rows of both transformed operands -> forward row transforms,
// pointwise product (Montgomery), inverse row transforms of the product,
// written over operand a in the workspace.  One thread per (row, j1); small
// blocks keep the barrier-separated phases of neighbouring blocks apart.
// TFT with descriptors: rows at or beyond the product's 16 B are not formed.
template <class Ar, int RPB, bool TFT = false>
__global__ void __launch_bounds__(RPB * 16, sizeof(typename Ar::word) == 4 ? kDRowMinBlocks32 : kDRowMinBlocks64)
k_row_polymul_d(DevPlan<Ar> P, const typename WideForm<Ar>::type ar, typename Ar::word* __restrict__ ws,
                long long ws_stride, long long prod_base,
                const BatchDesc* __restrict__ desc) {
    using word = typename Ar::word;
    using tw = typename Ar::tw;
    using RL = RowLayout;
    using Ax = typename WideForm<Ar>::type;
    constexpr long long N = 1LL << (2 * kDLog);
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    const int r0 = blockIdx.x * RPB;
    if (TFT && desc) {
        const BatchDesc d = desc[prod_base + blockIdx.y];
        if (r0 >= 16 * tft_blocks(static_cast<long long>(d.na) + d.nb - 1)) return;
    }
    word* base = ws + (prod_base + blockIdx.y) * ws_stride;
    const int j1 = threadIdx.x & 15, r = threadIdx.x >> 4;
    // outer forward pass of row r of operand i (line RPB i + r)
    const tw* lf = P.line256_t[0];
    const uint32_t* lf_w = P.wline_t[0];
    if constexpr (sizeof(word) == 8) {
        // 64-bit words: the two operands' passes unrolled together (more
        // independent work per thread; measured 0.326 -> 0.309 ms for 256
        // products, while 32-bit words ran 21% slower that way)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const word* in = base + i * N + static_cast<long long>(r0 + r) * kDLine + j1;
            word x[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) x[t] = in[16 * t];
            dif_regs<Ax, 16>(ar, x, P.rc);
#pragma unroll
            for (int t = 1; t < 16; ++t) {
                if (t == 8) asm volatile("" ::: "memory");   // at most half the twiddles live
                x[t] = ar.mulw(x[t], tw_at(ar, lf, lf_w, t * 16 + j1));
            }
#pragma unroll
            for (int t = 0; t < 16; ++t) sm[RL::at(RPB * i + r, 16 * t + j1)] = x[t];
        }
    } else {
#pragma unroll 1
        for (int i = 0; i < 2; ++i) {
            const word* in = base + i * N + static_cast<long long>(r0 + r) * kDLine + j1;
            word x[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) x[t] = in[16 * t];
            dif_regs<Ax, 16>(ar, x, P.rc);
#pragma unroll
            for (int t = 1; t < 16; ++t) x[t] = ar.mulw(x[t], tw_at(ar, lf, lf_w, t * 16 + j1));
#pragma unroll
            for (int t = 0; t < 16; ++t) sm[RL::at(RPB * i + r, 16 * t + j1)] = x[t];
        }
    }
    __syncthreads();
    // inner passes of both operands, pointwise product, inner inverse pass
    {
        const int blk = j1;
        word xa[16], xb[16];
        word* pa = sm + RL::at(r, 16 * blk);
        word* pb = sm + RL::at(RPB + r, 16 * blk);
        sm_load16(pa, xa);
        sm_load16(pb, xb);
        dif_regs<Ax, 16>(ar, xa, P.rc);
        dif_regs<Ax, 16>(ar, xb, P.rc);
#pragma unroll
        for (int t = 0; t < 16; ++t) xa[t] = ar.mulmont(xa[t], xb[t]);
        dit_regs<Ax, 16>(ar, xa, P.rci);
        sm_store16(pa, xa);
    }
    __syncthreads();
    // outer inverse pass of row r of the product
    {
        const tw* li = P.line256_t[1];
        const uint32_t* li_w = P.wline_t[1];
        word x[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = sm[RL::at(r, 16 * t + j1)];
#pragma unroll
        for (int t = 1; t < 16; ++t) {
            if (sizeof(word) == 8 && t == 8) asm volatile("" ::: "memory");   // 64-bit words: half the twiddles live
            x[t] = ar.mulw(x[t], tw_at(ar, li, li_w, t * 16 + j1));
        }
        dit_regs<Ax, 16>(ar, x, P.rci);
        word* o = base + static_cast<long long>(r0 + r) * kDLine + j1;
#pragma unroll
        for (int t = 0; t < 16; ++t) o[16 * t] = x[t];
    }
}

// Standalone row transforms of 256 words (the second pass of a forward
// 2^16-point transform, the first pass of an inverse one), in place, RPB rows
// per block.  The inner pass faces global memory with 16-byte vectors (a
// thread's 16 positions are consecutive), the outer pass with lanes over j1;
// the two meet once in shared memory.  data must be 16-byte aligned.
template <class Ar, bool FWD, int RPB>
__global__ void __launch_bounds__(RPB * 16)
k_row_ntt_d(DevPlan<Ar> P, typename Ar::word* __restrict__ data, long long prod_base) {
    using word = typename Ar::word;
    using tw = typename Ar::tw;
    using RL = RowLayout;
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    const int j1 = threadIdx.x & 15, r = threadIdx.x >> 4;
    word* line = data + ((prod_base + blockIdx.y) << (2 * kDLog)) + static_cast<long long>(blockIdx.x * RPB + r) * kDLine;
    word x[16];
    if (FWD) {
        const tw* lf = P.line256_t[0];
        const uint32_t* lf_w = P.wline_t[0];
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = line[16 * t + j1];
        dif_regs<Ar, 16>(P.ar, x, P.rc);
#pragma unroll
        for (int t = 1; t < 16; ++t) x[t] = P.ar.mulw(x[t], tw_at(P.ar, lf, lf_w, t * 16 + j1));
#pragma unroll
        for (int t = 0; t < 16; ++t) sm[RL::at(r, 16 * t + j1)] = x[t];
        __syncthreads();
        sm_load16(sm + RL::at(r, 16 * j1), x);
        dif_regs<Ar, 16>(P.ar, x, P.rc);
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = P.ar.canon(x[t]);
        sm_store16(line + 16 * j1, x);
    } else {
        const tw* li = P.line256_t[1];
        const uint32_t* li_w = P.wline_t[1];
        sm_load16(line + 16 * j1, x);
        dit_regs<Ar, 16>(P.ar, x, P.rci);
        sm_store16(sm + RL::at(r, 16 * j1), x);
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = sm[RL::at(r, 16 * t + j1)];
#pragma unroll
        for (int t = 1; t < 16; ++t) x[t] = P.ar.mulw(x[t], tw_at(P.ar, li, li_w, t * 16 + j1));
        dit_regs<Ar, 16>(P.ar, x, P.rci);
#pragma unroll
        for (int t = 0; t < 16; ++t) line[16 * t + j1] = x[t];
    }
}

// Pass 3: inverse global twiddle (with n^-1 and the Montgomery factor folded
// into itab), inverse column transforms, canonical cropped store of the first
// out_len words of each product.
// TFT: the inverse of the truncated forward pass -- inner passes on the B
// formed blocks, then per thread the inverse TFT of its 16-point outer pass
// (B known outputs, known zero inputs above them), scaled like the other
// unnormalised passes.
template <class Ar, bool TFT = false>
__global__ void __launch_bounds__(kDThreads, sizeof(typename Ar::word) == 4 ? kDColMinBlocks : kDColInvMinBlocks64)
k_col_inv_d(DevPlan<Ar> P, const typename WideForm<Ar>::type ar, const typename Ar::word* __restrict__ src,
            long long src_stride,
            typename Ar::word* __restrict__ dst, long long out_len, long long dst_stride,
            const typename Ar::tw* __restrict__ itab, const uint32_t* __restrict__ itab_w, long long prod_base,
            const BatchDesc* __restrict__ desc,
            int beta, TftConsts<Ar> K) {
    using word = typename Ar::word;
    using tw = typename Ar::tw;
    using Ax = typename WideForm<Ar>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    word* sm = reinterpret_cast<word*>(smraw);
    const int v = threadIdx.x & (kDCols - 1), g = threadIdx.x / kDCols;
    const long long c0 = static_cast<long long>(blockIdx.x) * kDCols;
    const long long prod = prod_base + blockIdx.y;
    const word* in = src + prod * src_stride + c0 + v;
    const tw* gt = itab + c0 + v;
    const uint32_t* gt_w = itab_w ? itab_w + c0 + v : nullptr;
    int B = 16;
    if (TFT) B = desc ? tft_blocks(static_cast<long long>(desc[prod].na) + desc[prod].nb - 1) : beta;
#pragma unroll
    for (int i = 0; i < kDItems; ++i) {
        const int blk = g + kDGroups * i;
        if (TFT && blk >= B) continue;
        word x[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const long long pos = 16 * blk + t;
            x[t] = ar.mulw(in[pos * kDLine], tw_at(ar, gt, gt_w, pos * kDLine));
        }
        dit_regs<Ax, 16>(ar, x, P.rci);
#pragma unroll
        for (int t = 0; t < 16; ++t) sm[(16 * blk + t) * kDCols + v] = x[t];
    }
    __syncthreads();
    word* outp;
    if (desc) {
        const BatchDesc d = desc[prod];
        outp = dst + d.coff;
        out_len = static_cast<long long>(d.na) + d.nb - 1;
    } else {
        outp = dst + prod * dst_stride;
    }
    const int rows = dcol_rows(out_len, c0 + v);
    word* o = outp + c0 + v;
    const tw* ltab = P.line_inv[kDLog];
    const uint32_t* ltab_w = P.wline[1];
#pragma unroll
    for (int i = 0; i < kDItems; ++i) {
        const int j1 = g + kDGroups * i;
        word x[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) x[t] = (!TFT || t < B) ? sm[(16 * t + j1) * kDCols + v] : word(0);
#pragma unroll
        for (int t = 1; t < 16; ++t)
            if (!TFT || t < B) x[t] = ar.mulw(x[t], tw_at(ar, ltab, ltab_w, j1 * 16 + t));
        if (TFT)
            itft16_z16(P.ar, x, P.rc, P.rci, K, B);
        else
            dit_regs<Ax, 16>(ar, x, P.rci);
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int row = 16 * t + j1;
            if (row < rows) o[static_cast<long long>(row) * kDLine] = ar.canon(x[t]);
        }
    }
}

}  // namespace gbntt
