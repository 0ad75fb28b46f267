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

}  // namespace gbntt
