// Truncated Fourier transforms of 16 registers (Section 5.1).
//
// The 16-point decimation-in-frequency network of dif_regs (stage half-span
// h multiplies the difference by w_2h^j = w_16^(8j/h)) leaves register t
// holding the value at w^[t]; the TFT of length l keeps only registers
// t < l.  Written recursively: an M-point sub-network on registers
// S .. S+M-1 is one stage of M/2 butterflies, then an M/2-point network on
// each half, so outputs t < M/2 depend on the sums alone.
//
//  * tdif16: forward TFT.  Registers t >= l come out undefined.
//  * itft16: inverse TFT (van der Hoeven's in-place form): on entry the
//    registers t < l hold transform values and the registers t >= l hold
//    known inputs; on return every register holds its input.  Exact (no
//    scale factor).  For M-point sub-problems with l >= M/2 the first half
//    of the outputs is complete, so its inverse gives the sums u_j; where the
//    upper input x_(j+M/2) is known, x_j = u_j - x_(j+M/2) and the difference
//    v_j = (x_j - x_(j+M/2)) w^j becomes a known input of the second half,
//    which is solved recursively; the remaining pairs follow from
//    x_j, x_(j+M/2) = (u_j +- v_j w^-j) / 2.  With l < M/2 the known inputs
//    give the sums u_j for j >= l, the first half is solved recursively, and
//    x_j = u_j - x_(j+M/2).
//  * itft16_z16: the same for known inputs that are all zero, returning 16
//    times the inputs -- the unnormalised scale of dit_regs, so that a
//    truncated inverse pass slots into a transform whose other passes are
//    unnormalised.
#pragma once
#include "engine.cuh"

namespace gbntt {

// Constants of the inverse TFT (w = w_16), in the policy's multiplicand form.
template <class Ar>
struct TftConsts {
    using tw = typename Ar::tw;
    tw inv2k[5];      // 2^-k, k = 0..4
    tw pow2k[5];      // 2^k
    tw rci_half[8];   // w^-e / 2
    tw rc_div8[8];    // w^e / 8
    tw rci_mul8[8];   // 8 w^-e
};

// Full M-point DIF on registers S .. S+M-1 (the sub-network of dif_regs).
template <class Ar, int M, int S>
__device__ __forceinline__ void dif_sub(const Ar& ar, typename Ar::word (&x)[16], const typename Ar::tw* rc) {
    if constexpr (M > 1) {
        constexpr int h = M / 2;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const auto u = x[S + j], v = x[S + j + h];
            x[S + j] = ar.add(u, v);
            x[S + j + h] = (j == 0) ? ar.sub(u, v) : ar.mulw(ar.sub_lazy(u, v), rc[(8 / h) * j]);
        }
        dif_sub<Ar, h, S>(ar, x, rc);
        dif_sub<Ar, h, S + h>(ar, x, rc);
    }
}

// Unnormalised inverse of dif_sub (M times the inputs).
template <class Ar, int M, int S>
__device__ __forceinline__ void dit_sub(const Ar& ar, typename Ar::word (&x)[16], const typename Ar::tw* rci) {
    if constexpr (M > 1) {
        constexpr int h = M / 2;
        dit_sub<Ar, h, S>(ar, x, rci);
        dit_sub<Ar, h, S + h>(ar, x, rci);
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const auto u = x[S + j];
            const auto v = (j == 0) ? x[S + j + h] : ar.mulw(x[S + j + h], rci[(8 / h) * j]);
            x[S + j] = ar.add(u, v);
            x[S + j + h] = ar.sub(u, v);
        }
    }
}

template <int M>
struct Log2 { static constexpr int v = M <= 1 ? 0 : 1 + Log2<M / 2>::v; };
template <>
struct Log2<1> { static constexpr int v = 0; };

// Forward TFT: outputs t < l of the M-point DIF on registers S .. S+M-1.
// ZH: the inputs S+M/2 .. S+M-1 are zero (first stage only).
template <class Ar, int M, int S, bool ZH = false>
__device__ __forceinline__ void tdif(const Ar& ar, typename Ar::word (&x)[16], const typename Ar::tw* rc, int l) {
    if constexpr (M > 1) {
        constexpr int h = M / 2;
        if (l <= 0) return;
        if (l <= h) {
            if (!ZH) {
#pragma unroll
                for (int j = 0; j < h; ++j) x[S + j] = ar.add(x[S + j], x[S + j + h]);
            }
            tdif<Ar, h, S>(ar, x, rc, l);
        } else {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const auto u = x[S + j], v = x[S + j + h];
                if (ZH) {
                    x[S + j + h] = (j == 0) ? u : ar.mulw(u, rc[(8 / h) * j]);
                } else {
                    x[S + j] = ar.add(u, v);
                    x[S + j + h] = (j == 0) ? ar.sub(u, v) : ar.mulw(ar.sub_lazy(u, v), rc[(8 / h) * j]);
                }
            }
            dif_sub<Ar, h, S>(ar, x, rc);
            tdif<Ar, h, S + h>(ar, x, rc, l - h);
        }
    }
}

// Inverse TFT, exact: registers t < l hold outputs, t >= l known inputs.
template <class Ar, int M, int S>
__device__ __forceinline__ void itft(const Ar& ar, typename Ar::word (&x)[16], const typename Ar::tw* rc,
                                     const typename Ar::tw* rci, const TftConsts<Ar>& K, int l) {
    using word = typename Ar::word;
    if constexpr (M > 1) {
        constexpr int h = M / 2;
        if (l <= 0) return;
        if (l >= M) {                                   // every output known
            dit_sub<Ar, M, S>(ar, x, rci);
#pragma unroll
            for (int j = 0; j < M; ++j) x[S + j] = ar.mulw(x[S + j], K.inv2k[Log2<M>::v]);
            return;
        }
        if (l >= h) {
            dit_sub<Ar, h, S>(ar, x, rci);              // h u_j
#pragma unroll
            for (int j = 0; j < h; ++j) x[S + j] = ar.mulw(x[S + j], K.inv2k[Log2<M>::v]);   // u_j / 2
            word keep[h];
#pragma unroll
            for (int j = 0; j < h; ++j) {
                keep[j] = x[S + h + j];
                if (j >= l - h) {                       // x_(j+h) is a known input
                    const word uj = ar.add(x[S + j], x[S + j]);
                    const word xj = ar.sub(uj, keep[j]);
                    x[S + j] = xj;
                    x[S + h + j] = (j == 0) ? ar.sub(xj, keep[j]) : ar.mulw(ar.sub_lazy(xj, keep[j]), rc[(8 / h) * j]);
                }
            }
            itft<Ar, h, S + h>(ar, x, rc, rci, K, l - h);   // v_j for every j
#pragma unroll
            for (int j = 0; j < h; ++j) {
                if (j < l - h) {
                    const word t = ar.mulw(x[S + h + j], K.rci_half[(8 / h) * j]);   // v_j w^-j / 2
                    const word a = x[S + j];
                    x[S + j] = ar.add(a, t);
                    x[S + h + j] = ar.sub(a, t);
                } else {
                    x[S + h + j] = keep[j];
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < h; ++j)
                if (j >= l) x[S + j] = ar.add(x[S + j], x[S + h + j]);   // u_j from known inputs
            itft<Ar, h, S>(ar, x, rc, rci, K, l);
#pragma unroll
            for (int j = 0; j < h; ++j) x[S + j] = ar.sub(x[S + j], x[S + h + j]);
        }
    }
}

// Inverse TFT with all known inputs zero (registers t >= l hold 0 on entry
// and on return); returns 16 times the inputs in registers t < l.
template <class Ar, int M, int S>
__device__ __forceinline__ void itft_z(const Ar& ar, typename Ar::word (&x)[16], const typename Ar::tw* rc,
                                       const typename Ar::tw* rci, const TftConsts<Ar>& K, int l) {
    using word = typename Ar::word;
    constexpr int q = 4 - Log2<M>::v;                   // 16 / M = 2^q
    if constexpr (M == 1) {
        if (l >= 1) x[S] = ar.mulw(x[S], K.pow2k[4]);
    } else {
        constexpr int h = M / 2;
        if (l <= 0) return;
        if (l >= M) {
            dit_sub<Ar, M, S>(ar, x, rci);              // M x_j
            if (q > 0) {
#pragma unroll
                for (int j = 0; j < M; ++j) x[S + j] = ar.mulw(x[S + j], K.pow2k[q]);
            }
            return;
        }
        if (l >= h) {
            dit_sub<Ar, h, S>(ar, x, rci);              // h u_j -> U_j = 8 u_j
            if (q > 0) {
#pragma unroll
                for (int j = 0; j < h; ++j) x[S + j] = ar.mulw(x[S + j], K.pow2k[q]);
            }
#pragma unroll
            for (int j = 0; j < h; ++j) {
                if (j >= l - h) {                       // x_(j+h) = 0: 16 x_j = 2 U_j, v_j = x_j w^j
                    const word U = x[S + j];
                    x[S + j] = ar.add(U, U);
                    x[S + h + j] = ar.mulw(U, K.rc_div8[(8 / h) * j]);
                }
            }
            itft<Ar, h, S + h>(ar, x, rc, rci, K, l - h);
#pragma unroll
            for (int j = 0; j < h; ++j) {
                if (j < l - h) {
                    const word t = ar.mulw(x[S + h + j], K.rci_mul8[(8 / h) * j]);   // 8 v_j w^-j
                    const word U = x[S + j];
                    x[S + j] = ar.add(U, t);
                    x[S + h + j] = ar.sub(U, t);
                } else {
                    x[S + h + j] = word(0);
                }
            }
        } else {
            itft_z<Ar, h, S>(ar, x, rc, rci, K, l);     // u_j = x_j here
        }
    }
}

template <class Ar, bool ZH = false>
__device__ __forceinline__ void tdif16(const Ar& ar, typename Ar::word (&x)[16], const typename Ar::tw* rc, int l) {
    tdif<Ar, 16, 0, ZH>(ar, x, rc, l);
}

template <class Ar>
__device__ __forceinline__ void itft16_z16(const Ar& ar, typename Ar::word (&x)[16], const typename Ar::tw* rc,
                                           const typename Ar::tw* rci, const TftConsts<Ar>& K, int l) {
    itft_z<Ar, 16, 0>(ar, x, rc, rci, K, l);
}

// ------------------------------------------------------------------ truncated engine phases
//
// The truncated transform of Section 5.1 inside the shared-memory engine
// (one-block products and the column passes of the two-pass sizes).  A
// product of l output words through an n-point transform needs the values
// at w^[i] for i < l only, i.e. the first kb = ceil(16 l / n) of the 16
// blocks of n/16 positions (Algorithm 1's lambda rounded up to whole blocks
// of the outermost 16-way split).  In the engine's layouts those are:
//  * one-line vectors (n <= 256): positions [0, kb n/16) of the line;
//  * L2 x L1 tiles: rows [0, kb L2/16) (the column phase's outer radix-16
//    pass puts block t of its output into rows t L2/16 .. (t+1) L2/16 - 1).
// The outer radix-16 pass of the column phase (the whole line for one-line
// vectors) keeps registers t < kb (tdif16); inner passes and the row phase
// run on the kept blocks and rows only.  The inverse runs the kept blocks'
// inner passes, then solves the outer pass with itft16_z16: the operands and
// the product vanish at every position >= kb n/16, so the 16 - kb unknown
// registers of each outer butterfly network are known zero inputs.
// itft16_z16 returns 16 times the inputs, the scale of dit_regs, so the
// final scaling by n^-1 is unchanged.

// Products whose output needs few enough of the 16 blocks run truncated
// transforms: one-block tiles (n = 2^9 .. 2^13) at most kTileTftMaxBlocks,
// the two-pass sizes below 2^16 at most kColTftMaxBlocks.  Measured on 2^23
// output words per call, time against the full transforms at kb = 9 / 12:
// tiles 0.80 .. 1.0 / 0.95 .. 1.05, two-pass 0.77 .. 0.82 / 0.88 .. 0.96;
// one-line vectors (n <= 256) gain nothing and stay untruncated.
constexpr int kTileTftMinLog = 9;
constexpr int kTileTftMaxBlocks = 11;
constexpr int kColTftMaxBlocks = 12;

// Blocks of n/16 positions that l output words occupy (1..16); n = 2^logn,
// logn >= 4.
__host__ __device__ inline int tft_kb(long long l, int logn) {
    const long long blk = 1LL << (logn - 4);
    const long long b = (l + blk - 1) / blk;
    return static_cast<int>(b < 1 ? 1 : (b > 16 ? 16 : b));
}

// Outer radix-16 pass of a truncated phase over lines of 2^g.logL words
// (4 <= g.logL <= 8): forward, the first kb outputs of each 16-point DIF
// then the line twiddle (or the hook when the line is one 16-point
// transform); inverse, the twiddle on the kb known outputs and the
// inverse TFT with zero inputs above them.  Registers t >= kb are neither
// formed nor stored.
template <class Ar, bool FWD, bool ZHALF = false>
__device__ __forceinline__ void run_pass_tout(const DevPlan<Ar>& P, typename Ar::word* s, const PhaseGeom& g,
                                              const Hook<Ar>* hook, int kb, const TftConsts<Ar>& K) {
    using word = typename Ar::word;
    using tw = typename Ar::tw;
    const int logM = g.logL;
    const int logMR = logM - 4;
    const int lognl = g.lognvec + g.logX;
    const int items = 1 << (lognl + logMR);
    const tw* ltab = (logMR > 0) ? (FWD ? P.line_fwd[logM] : P.line_inv[logM]) : nullptr;
    const Hook<Ar>* hk = (logMR > 0) ? nullptr : hook;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int line = it & ((1 << lognl) - 1);
        const int j1 = it >> lognl;
        int v, xl;
        if (g.vfast) {
            v = line & ((1 << g.lognvec) - 1);
            xl = line >> g.lognvec;
        } else {
            xl = line & ((1 << g.logX) - 1);
            v = line >> g.logX;
        }
        word* b = s + (v * g.VS + xl * g.XS + j1 * g.ES);
        const int st = (1 << logMR) * g.ES;
        word x[16];
        if (FWD) {
#pragma unroll
            for (int t = 0; t < 16; ++t) x[t] = (!ZHALF || t < 8) ? b[t * st] : word(0);
            tdif16<Ar, ZHALF>(P.ar, x, P.rc, kb);
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                if (t < kb) {
                    if (ltab) {
                        if (t) x[t] = P.ar.mulw(x[t], ltab[j1 * 16 + t]);
                    } else if (hk) {
                        x[t] = P.ar.mulw(x[t], hk->tab[t * hk->A + xl * hk->B + v * hk->C + hk->off]);
                    }
                    b[t * st] = x[t];
                }
            }
        } else {
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                x[t] = word(0);
                if (t < kb) {
                    x[t] = b[t * st];
                    if (ltab) {
                        if (t) x[t] = P.ar.mulw(x[t], ltab[j1 * 16 + t]);
                    } else if (hk) {
                        x[t] = P.ar.mulw(x[t], hk->tab[t * hk->A + xl * hk->B + v * hk->C + hk->off]);
                    }
                }
            }
            itft16_z16<Ar>(P.ar, x, P.rc, P.rci, K, kb);
#pragma unroll
            for (int t = 0; t < 16; ++t)
                if (t < kb) b[t * st] = x[t];
        }
    }
}

// Forward column phase (or whole-line phase) truncated to kb blocks:
// lines of 2^g.logL words, 4 <= g.logL <= 8; the hook applies at the
// innermost pass as in phase_fwd.  Ends with __syncthreads().
template <class Ar, bool ZHALF = false>
__device__ __forceinline__ void phase_fwd_t(const DevPlan<Ar>& P, typename Ar::word* s, const PhaseGeom& g,
                                            const Hook<Ar>* hook, int kb, const TftConsts<Ar>& K) {
    run_pass_tout<Ar, true, ZHALF>(P, s, g, hook, kb, K);
    __syncthreads();
    if (g.logL > 4) {
        run_pass_r<Ar, true>(P, s, g, g.logL - 4, g.logL - 4, hook, kb);
        __syncthreads();
    }
}

template <class Ar>
__device__ __forceinline__ void phase_inv_t(const DevPlan<Ar>& P, typename Ar::word* s, const PhaseGeom& g,
                                            const Hook<Ar>* hook, int kb, const TftConsts<Ar>& K) {
    if (g.logL > 4) {
        run_pass_r<Ar, false>(P, s, g, g.logL - 4, g.logL - 4, hook, kb);
        __syncthreads();
    }
    run_pass_tout<Ar, false>(P, s, g, hook, kb, K);
    __syncthreads();
}

// One pass of radix R over the first nx lines (x index, the rows of a tile
// layout with lanes over rows: g.vfast false) of every vector; the work per
// line is run_pass's without a hook.  Items are numbered with the row
// fastest, then the vector, then the sub-transform: item it is row
// it mod nx of the quotient's (vector, sub-transform), the quotient taken
// as (it * magic) >> 32 with magic = ceil(2^32 / nx) (exact for
// it < 2^32 / nx).
template <class Ar, int R, bool FWD>
__device__ __forceinline__ void run_pass_nx(const DevPlan<Ar>& P, typename Ar::word* s, const PhaseGeom& g,
                                            int logM, int nx, unsigned long long magic) {
    using word = typename Ar::word;
    using tw = typename Ar::tw;
    constexpr int lr = RadixLog<R>::v;
    const int logMR = logM - lr;
    const int items = (nx << g.lognvec) << (g.logL - lr);
    const tw* ltab = (logMR > 0) ? (FWD ? P.line_fwd[logM] : P.line_inv[logM]) : nullptr;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int q = static_cast<int>((static_cast<unsigned long long>(it) * magic) >> 32);
        const int xl = it - q * nx;
        const int v = q & ((1 << g.lognvec) - 1);
        const int k = q >> g.lognvec;
        const int j1 = k & ((1 << logMR) - 1);
        const int blk = k >> logMR;
        word* b = s + (v * g.VS + xl * g.XS + ((blk << logM) + j1) * g.ES);
        const int st = (1 << logMR) * g.ES;
        word x[R];
#pragma unroll
        for (int t = 0; t < R; ++t) x[t] = b[t * st];
        if (!FWD) {
            if (ltab) {
#pragma unroll
                for (int t = 1; t < R; ++t) x[t] = P.ar.mulw(x[t], ltab[j1 * 16 + t]);
            }
            dit_regs<Ar, R>(P.ar, x, P.rci);
        } else {
            dif_regs<Ar, R>(P.ar, x, P.rc);
            if (ltab) {
#pragma unroll
                for (int t = 1; t < R; ++t) x[t] = P.ar.mulw(x[t], ltab[j1 * 16 + t]);
            }
        }
#pragma unroll
        for (int t = 0; t < R; ++t) b[t * st] = x[t];
    }
}

template <class Ar, bool FWD>
__device__ __forceinline__ void run_pass_nx_r(const DevPlan<Ar>& P, typename Ar::word* s, const PhaseGeom& g,
                                              int logM, int lr, int nx, unsigned long long magic) {
    switch (lr) {
        case 4: run_pass_nx<Ar, 16, FWD>(P, s, g, logM, nx, magic); break;
        case 3: run_pass_nx<Ar, 8, FWD>(P, s, g, logM, nx, magic); break;
        case 2: run_pass_nx<Ar, 4, FWD>(P, s, g, logM, nx, magic); break;
        default: run_pass_nx<Ar, 2, FWD>(P, s, g, logM, nx, magic); break;
    }
}

// Forward transform of every vector truncated to kb blocks (layouts of
// tile_layout with 2^L.logL >= 16; tiles have lanes over rows).  Entries
// outside the kept blocks are left as they were.
template <class Ar>
__device__ __forceinline__ void vec_fwd_t(const DevPlan<Ar>& P, typename Ar::word* s, const VecLayout& L, int kb,
                                          const TftConsts<Ar>& K) {
    if (L.logL <= kMaxLineLog) {
        PhaseGeom g{L.logL, L.lognvec, 0, L.VS, 0, L.CS, true};
        phase_fwd_t<Ar>(P, s, g, nullptr, kb, K);
        return;
    }
    const int l2 = tile_l2(L.logL), l1 = tile_l1(L.logL);
    Hook<Ar> th{P.tile_fwd[L.logL], 1 << l1, 1, 0, 0};
    PhaseGeom gc{l2, L.lognvec, l1, L.VS, L.CS, L.RS, L.vfast};
    phase_fwd_t<Ar>(P, s, gc, &th, kb, K);
    const int nx = kb << (l2 - 4);
    const unsigned long long magic = ((1ull << 32) + nx - 1) / nx;
    PhaseGeom gr{l1, L.lognvec, l2, L.VS, L.RS, L.CS, false};
    int logM = l1;
    while (logM > 4) {
        run_pass_nx<Ar, 16, true>(P, s, gr, logM, nx, magic);
        __syncthreads();
        logM -= 4;
    }
    run_pass_nx_r<Ar, true>(P, s, gr, logM, logM, nx, magic);
    __syncthreads();
}

template <class Ar>
__device__ __forceinline__ void vec_inv_t(const DevPlan<Ar>& P, typename Ar::word* s, const VecLayout& L, int kb,
                                          const TftConsts<Ar>& K) {
    if (L.logL <= kMaxLineLog) {
        PhaseGeom g{L.logL, L.lognvec, 0, L.VS, 0, L.CS, true};
        phase_inv_t<Ar>(P, s, g, nullptr, kb, K);
        return;
    }
    const int l2 = tile_l2(L.logL), l1 = tile_l1(L.logL);
    const int nx = kb << (l2 - 4);
    const unsigned long long magic = ((1ull << 32) + nx - 1) / nx;
    PhaseGeom gr{l1, L.lognvec, l2, L.VS, L.RS, L.CS, false};
    const int last = l1 - 4 * ((l1 - 1) / 4);
    run_pass_nx_r<Ar, false>(P, s, gr, last, last, nx, magic);
    __syncthreads();
    for (int logM = last + 4; logM <= l1; logM += 4) {
        run_pass_nx<Ar, 16, false>(P, s, gr, logM, nx, magic);
        __syncthreads();
    }
    Hook<Ar> th{P.tile_inv[L.logL], 1 << l1, 1, 0, 0};
    PhaseGeom gc{l2, L.lognvec, l1, L.VS, L.CS, L.RS, L.vfast};
    phase_inv_t<Ar>(P, s, gc, &th, kb, K);
}

}  // namespace gbntt
