// Shared-memory transform engine.
//
// Transform definition (Section 5.1): FFT_w(a)_i = sum_j w^(ij) a_j for a
// primitive n-th root w, n = 2^k; the forward transform here returns the
// TFT with l = n, i.e. position i holds A(w^[i]_k) (bit-mirrored order).
//
// Every transform is Algorithm 1 applied recursively.  For a length-M
// sub-transform split as R rows x M/R columns (R = 16 except possibly the
// last level):
//   step 1: R-point transforms down each column, done in registers by one
//           thread (radix-2 decimation-in-frequency butterflies, whose
//           output comes out bit-mirrored: register t holds row [t]);
//   step 2: the twiddle w_M^(j1 [t]) on row t of column j1 (Function 8 /
//           Remark 8 product by a precomputed multiplicand);
//   step 3: the M/R-point transforms of the rows, i.e. the next pass;
//   step 4: nothing to do -- the in-place result is already the bit-mirrored
//           order of the whole transform (the reordering in Algorithm 1's
//           proof).
// The inverse undoes the passes in reverse order with w^-1 (the text after
// Proposition 15), leaving a factor n that the callers fold into a final
// scaling.
//
// Vectors longer than 256 words are themselves split once more by
// Algorithm 1 into an L2 x L1 tile (L2 = 2^floor(k/2)) with a tile-level
// twiddle between the column phase and the row phase.
//
// Data layout in shared memory: a "line" is one run of butterflies (a
// column or a row of a tile, or a whole short vector).  Warp lanes are
// spread across lines, never along one, and every line/vector stride used
// by the kernels is 1 or odd, so each lane of a warp touches a different
// bank on every load and store of every pass.
#pragma once
#include <cstdint>

#include "modarith.cuh"

namespace gbntt {

constexpr int kMaxLineLog = 8;      // lines are at most 256 words
// Largest transform (log2) that one thread block holds whole, both operands
// resident in shared memory: 32-bit and 64-bit words.
constexpr int kTileMaxLog32 = 13;
constexpr int kTileMaxLog64 = 13;

// Per-modulus constants and table pointers, passed by value to every kernel
// (so they sit in the constant bank).
template <class Ar>
struct DevPlan {
    using tw = typename Ar::tw;
    Ar ar;
    tw rc[8];                        // w_16^e,  e < 8
    tw rci[8];                       // w_16^-e, e < 8
    const tw* line_fwd[kMaxLineLog + 1];   // [logM] (5..8): [j1*16 + t] = w_M^(j1 [t]_4)
    const tw* line_inv[kMaxLineLog + 1];
    // the 256-point line tables transposed, [t*16 + j1] = w_256^(+-j1 [t]_4):
    // lanes over j1 read consecutive entries (the direct row kernels)
    const tw* line256_t[2];
    const tw* tile_fwd[17];          // [logT] (9..16): [r*L1 + c] = w_T^(c [r]_l2)
    const tw* tile_inv[17];
    const tw* glob_fwd;              // [j2*n1 + j1] = w_N^(j1 [j2]_k2)
    const tw* glob_inv;              // w_N^-(j1 [j2]_k2) * N^-1
    const tw* plain_fwd;             // [e] = w_N^e, e < N/2
    const tw* plain_inv;
    // 32-bit plans only (null otherwise): the multiplicands w~ alone of the
    // tables the direct 2^16-point kernels read, 4 bytes per entry, so a warp
    // reads whole sectors of them instead of every other word of the pairs.
    // [0] forward, [1] inverse.
    const uint32_t* wline[2];        // line_fwd / line_inv at logM = 8
    const uint32_t* wline_t[2];      // line256_t
    const uint32_t* wglob[2];        // glob_fwd, glob_inv
    // 64-point sub-transforms split 8 x 8 (the cluster kernel of 4096-point
    // products): [j1*8 + t] = w_64^(+-j1 [t]_3)
    const tw* line64x8[2];
};

// One product of an uneven batch: word offsets of its operands and output in
// the batch's flat buffers, and the operand lengths.  `sub`: for products of
// 2^17 .. 2^24 points, the index of the product's first 2^16-point row slot
// in its bucket's workspace (the rows the truncated transform keeps).
struct BatchDesc {
    unsigned long long aoff, boff, coff;
    unsigned na, nb;
    unsigned long long sub;
};

// A work item of the persistent kernel: `count` products (descriptors
// desc[first .. first+count)) of one-block size 2^logL with modulus `prime`
// (index into the plan array), final scaling `scale`; kb < 16: the
// transforms are truncated to kb of the 16 blocks of 2^logL/16 positions
// (the most that any of the item's products needs).
template <class Ar>
struct SmallItem {
    unsigned first, count, prime, logL, kb;
    typename Ar::tw scale;
};

constexpr int kSmallMaxPerItem = 16;

// log2 of the products per block of the one-block sizes: 16 one-line vectors
// up to 256 words; tiles of 2^9, 2^10, 2^11 words hold 8, 4, 2 products, so
// that a block's column phase runs at least 512 lines (measured on 2^23
// output words per call: 2^9 points 0.26 -> 0.14 ms with 32-bit words,
// 0.71 -> 0.30 ms with 64-bit words; 2^10: 0.21 -> 0.16, 0.49 -> 0.34 ms)
__host__ __device__ inline int small_lppc(int logL) {
    return logL <= kMaxLineLog ? 4 : (logL < 12 ? 12 - logL : 0);
}

// Twiddle applied to every element of a vector at the outer end of a phase:
// element at position `pos` of line `x` of vector `v` is multiplied by
// tab[pos*A + x*B + v*C + off].
template <class Ar>
struct Hook {
    const typename Ar::tw* tab;
    int A, B, C, off;
};

template <int R>
struct RadixLog;
template <> struct RadixLog<2> { static constexpr int v = 1; };
template <> struct RadixLog<4> { static constexpr int v = 2; };
template <> struct RadixLog<8> { static constexpr int v = 3; };
template <> struct RadixLog<16> { static constexpr int v = 4; };

// R-point DIF in registers: natural order in, bit-mirrored order out.
// Stage with half-span h multiplies the difference by w_{2h}^j = w_16^(8j/h).
// ZHALF: the upper half of the inputs is known to be zero (zero padding),
// so the first stage is (u, 0) -> (u, u w) without the sum and difference.
template <class Ar, int R, bool ZHALF = false>
__device__ __forceinline__ void dif_regs(const Ar& ar, typename Ar::word (&x)[R],
                                         const typename Ar::tw* rc) {
    if (ZHALF) {
#pragma unroll
        for (int j = 0; j < R / 2; ++j)
            x[j + R / 2] = (j == 0) ? x[j] : ar.mulw(x[j], rc[(8 / (R / 2)) * j]);
    }
#pragma unroll
    for (int h = ZHALF ? R / 4 : R / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int s = 0; s < R; s += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                auto u = x[s + j];
                auto v = x[s + j + h];
                x[s + j] = ar.add(u, v);
                x[s + j + h] = (j == 0) ? ar.sub(u, v) : ar.mulw(ar.sub_lazy(u, v), rc[(8 / h) * j]);
            }
        }
    }
}

// Inverse of dif_regs up to the factor R: bit-mirrored in, natural out.
template <class Ar, int R>
__device__ __forceinline__ void dit_regs(const Ar& ar, typename Ar::word (&x)[R],
                                         const typename Ar::tw* rci) {
#pragma unroll
    for (int h = 1; h <= R / 2; h <<= 1) {
#pragma unroll
        for (int s = 0; s < R; s += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                auto u = x[s + j];
                auto v = (j == 0) ? x[s + j + h] : ar.mulw(x[s + j + h], rci[(8 / h) * j]);
                x[s + j] = ar.add(u, v);
                x[s + j + h] = ar.sub(u, v);
            }
        }
    }
}

// Geometry of one phase: nvec vectors x X lines each, line length 2^logL.
// Line (v, x) starts at v*VS + x*XS; consecutive elements are ES apart.
// Lanes take consecutive v when vfast, else consecutive x.
struct PhaseGeom {
    int logL;
    int lognvec;
    int logX;
    int VS, XS, ES;       // shared-memory word strides
    bool vfast;
};

// One pass of radix R over every line: sub-transforms of size 2^logM.
// FWD: DIF then twiddle; inverse: twiddle then DIT.  When M == R this is the
// innermost level; the hook (if any) applies there.
// nblk (nonzero): only the first nblk sub-transforms of every line run (the
// kept blocks of a truncated transform).
template <class Ar, int R, bool FWD, bool ZHALF = false>
__device__ __forceinline__ void run_pass(const DevPlan<Ar>& P, typename Ar::word* s,
                                         const PhaseGeom& g, int logM,
                                         const Hook<Ar>* hook, int nblk = 0) {
    using word = typename Ar::word;
    using tw = typename Ar::tw;
    constexpr int lr = RadixLog<R>::v;
    const int logMR = logM - lr;                 // log of j1 range
    const int lognl = g.lognvec + g.logX;         // log of number of lines
    const int items = nblk ? ((nblk << logMR) << lognl) : 1 << (lognl + g.logL - lr);
    const tw* ltab = (logMR > 0) ? (FWD ? P.line_fwd[logM] : P.line_inv[logM]) : nullptr;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int line = it & ((1 << lognl) - 1);
        const int k = it >> lognl;
        int v, xl;
        if (g.vfast) {
            v = line & ((1 << g.lognvec) - 1);
            xl = line >> g.lognvec;
        } else {
            xl = line & ((1 << g.logX) - 1);
            v = line >> g.logX;
        }
        const int j1 = k & ((1 << logMR) - 1);
        const int blk = k >> logMR;
        word* b = s + (v * g.VS + xl * g.XS + ((blk << logM) + j1) * g.ES);
        const int st = (1 << logMR) * g.ES;
        word x[R];
#pragma unroll
        for (int t = 0; t < (ZHALF ? R / 2 : R); ++t) x[t] = b[t * st];
        if (!FWD) {
            if (ltab) {
#pragma unroll
                for (int t = 1; t < R; ++t) x[t] = P.ar.mulw(x[t], ltab[j1 * 16 + t]);
            } else if (hook) {
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    const int pos = (blk << logM) + t;
                    x[t] = P.ar.mulw(x[t], hook->tab[pos * hook->A + xl * hook->B + v * hook->C + hook->off]);
                }
            }
            dit_regs<Ar, R>(P.ar, x, P.rci);
        } else {
            dif_regs<Ar, R, ZHALF>(P.ar, x, P.rc);
            if (ltab) {
#pragma unroll
                for (int t = 1; t < R; ++t) x[t] = P.ar.mulw(x[t], ltab[j1 * 16 + t]);
            } else if (hook) {
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    const int pos = (blk << logM) + t;
                    x[t] = P.ar.mulw(x[t], hook->tab[pos * hook->A + xl * hook->B + v * hook->C + hook->off]);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < R; ++t) b[t * st] = x[t];
    }
}

template <class Ar, bool FWD>
__device__ __forceinline__ void run_pass_r(const DevPlan<Ar>& P, typename Ar::word* s,
                                           const PhaseGeom& g, int logM, int lr,
                                           const Hook<Ar>* hook, int nblk = 0) {
    switch (lr) {
        case 4: run_pass<Ar, 16, FWD>(P, s, g, logM, hook, nblk); break;
        case 3: run_pass<Ar, 8, FWD>(P, s, g, logM, hook, nblk); break;
        case 2: run_pass<Ar, 4, FWD>(P, s, g, logM, hook, nblk); break;
        default: run_pass<Ar, 2, FWD>(P, s, g, logM, hook, nblk); break;
    }
}

// All passes of one phase.  Forward: logM = logL, logL-4, ..., the last with
// radix 2^logM (1..4); the hook applies at that last pass.  Inverse: the
// same passes in reverse order (hook first).  Ends with __syncthreads().
template <class Ar, bool ZHALF = false>
__device__ __forceinline__ void phase_fwd(const DevPlan<Ar>& P, typename Ar::word* s, const PhaseGeom& g,
                          const Hook<Ar>* hook) {
    int logM = g.logL;   // >= 1: plans have n >= 2
    if (ZHALF && logM > 4) {
        run_pass<Ar, 16, true, true>(P, s, g, logM, nullptr);
        __syncthreads();
        logM -= 4;
    }
    while (logM > 4) {
        run_pass<Ar, 16, true>(P, s, g, logM, nullptr);
        __syncthreads();
        logM -= 4;
    }
    run_pass_r<Ar, true>(P, s, g, logM, logM, hook);
    __syncthreads();
}

template <class Ar>
__device__ __forceinline__ void phase_inv(const DevPlan<Ar>& P, typename Ar::word* s, const PhaseGeom& g,
                          const Hook<Ar>* hook) {
    int last = g.logL - 4 * ((g.logL - 1) / 4);   // 1..4
    run_pass_r<Ar, false>(P, s, g, last, last, hook);
    __syncthreads();
    for (int logM = last + 4; logM <= g.logL; logM += 4) {
        run_pass<Ar, 16, false>(P, s, g, logM, nullptr);
        __syncthreads();
    }
}

// Layout of a set of vectors of length 2^logL in shared memory.
//   logL <= 8 : one line per vector, element i at v*VS + i*CS;
//   logL  > 8 : an L2 x L1 tile per vector, element r*L1 + c at v*VS + r*RS + c*CS.
struct VecLayout {
    int logL;
    int lognvec;
    int VS, RS, CS;
    bool vfast;   // lanes over vectors first (VS == 1 layouts)
};

__host__ __device__ inline int tile_l2(int logL) { return logL / 2; }
__host__ __device__ inline int tile_l1(int logL) { return logL - logL / 2; }

// Word offset of element i of vector v.
__device__ __forceinline__ int vec_addr(const VecLayout& L, int v, int i) {
    if (L.logL <= kMaxLineLog) return v * L.VS + i * L.CS;
    const int l1 = tile_l1(L.logL);
    return v * L.VS + (i >> l1) * L.RS + (i & ((1 << l1) - 1)) * L.CS;
}

// Forward transform of every vector.  vhook (optional) is applied to
// element `pos` of vector v as tab[pos*A + v*C + off] (its B is ignored).
// ZHALF: the second half of every vector is zero on input.
template <class Ar, bool ZHALF = false>
__device__ __forceinline__ void vec_fwd(const DevPlan<Ar>& P, typename Ar::word* s, const VecLayout& L,
                        const Hook<Ar>* vhook) {
    if (L.logL <= kMaxLineLog) {
        PhaseGeom g{L.logL, L.lognvec, 0, L.VS, 0, L.CS, true};
        phase_fwd<Ar, ZHALF>(P, s, g, vhook);
        return;
    }
    const int l2 = tile_l2(L.logL), l1 = tile_l1(L.logL);
    // column phase: lines (v, c) of length L2, tile twiddle at its end
    Hook<Ar> th{P.tile_fwd[L.logL], 1 << l1, 1, 0, 0};
    PhaseGeom gc{l2, L.lognvec, l1, L.VS, L.CS, L.RS, L.vfast};
    phase_fwd<Ar, ZHALF>(P, s, gc, &th);   // tile rows >= L2/2 hold the zero half
    // row phase: lines (v, r) of length L1; vector position = r*L1 + c
    PhaseGeom gr{l1, L.lognvec, l2, L.VS, L.RS, L.CS, L.vfast};
    if (vhook) {
        Hook<Ar> rh{vhook->tab, vhook->A, vhook->A << l1, vhook->C, vhook->off};
        phase_fwd<Ar>(P, s, gr, &rh);
    } else {
        phase_fwd<Ar>(P, s, gr, nullptr);
    }
}

template <class Ar>
__device__ __forceinline__ void vec_inv(const DevPlan<Ar>& P, typename Ar::word* s, const VecLayout& L,
                        const Hook<Ar>* vhook) {
    if (L.logL <= kMaxLineLog) {
        PhaseGeom g{L.logL, L.lognvec, 0, L.VS, 0, L.CS, true};
        phase_inv<Ar>(P, s, g, vhook);
        return;
    }
    const int l2 = tile_l2(L.logL), l1 = tile_l1(L.logL);
    PhaseGeom gr{l1, L.lognvec, l2, L.VS, L.RS, L.CS, L.vfast};
    if (vhook) {
        Hook<Ar> rh{vhook->tab, vhook->A, vhook->A << l1, vhook->C, vhook->off};
        phase_inv<Ar>(P, s, gr, &rh);
    } else {
        phase_inv<Ar>(P, s, gr, nullptr);
    }
    Hook<Ar> th{P.tile_inv[L.logL], 1 << l1, 1, 0, 0};
    PhaseGeom gc{l2, L.lognvec, l1, L.VS, L.CS, L.RS, L.vfast};
    phase_inv<Ar>(P, s, gc, &th);
}

}  // namespace gbntt
