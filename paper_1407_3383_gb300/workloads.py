"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds only random-number generation: it draws words, sizes and
arrival times.  It contains none of the modular arithmetic of the method, and
both the CUDA path's tests/bench and the CPU oracle's tests take their inputs
from here.

Generator: splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), written from its published definition and
vectorised over numpy uint64 (wrapping arithmetic).

* uniform residues in [0, p): draw 64 bits, reject draws >= floor(2^64/p) p,
  return the draw rem p (no modulo bias);
* log-uniform sizes: round(exp(U(ln lo, ln hi))) with U built from the top
  53 bits of a draw;
* exponential inter-arrival gaps for a Poisson stream.

Configurations (seed = 0x5EED0000 + index):
  0  one product mod 998244353, two length-2048 operands (N = 4096)
  1  256 products mod 3*2^30+1 of two length-2^15 operands (N = 2^16)
  2  one length-2^24 transform and 1024 products of length 2^12 mod a
     62-bit prime k*2^40+1
  3  10,000 products, lengths log-uniform in [2^6, 2^18], prime chosen
     uniformly among three 62-bit primes
  4  Poisson stream of integer products, operand sizes log-uniform in
     [2^14, 2^28] bits rounded to whole 32-bit limbs
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_GEN_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libworkloads.so")
_gen = None


def _gen_lib():
    """workloads_gen.c (the same stream in C, for speed), or None when it is
    not built; the numpy code below gives identical draws."""
    global _gen
    if _gen is None:
        _gen = False
        if os.path.exists(_GEN_LIB):
            lib = ctypes.CDLL(_GEN_LIB)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.wl_u64.argtypes = [u64p, ctypes.c_void_p, ctypes.c_size_t]
            lib.wl_uniform_mod.argtypes = [u64p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t]
            _gen = lib
    return _gen or None

SEED_BASE = 0x5EED0000
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Moduli named by the workloads (verified prime by the oracle's tests).
P_A = 998244353            # 119 * 2^23 + 1
P_B = 3221225473           # 3 * 2^30 + 1
P_TABLE11 = 469762049      # 7 * 2^26 + 1
P_TABLE12 = 1108307720798209  # 63 * 2^44 + 1
# The first three primes k * 2^40 + 1 in (2^61, 2^62) for ascending k.
P1 = 2305919975027638273
P2 = 2305926572097404929
P3 = 2305940865748566017


class SplitMix64:
    """splitmix64 stream; every method advances the same state."""

    def __init__(self, seed: int, native: bool = True):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.native = native

    def _c(self):
        return _gen_lib() if self.native else None

    def u64(self, n: int) -> np.ndarray:
        n = int(n)
        lib = self._c()
        if lib is not None:
            out = np.empty(n, dtype=np.uint64)
            st = ctypes.c_uint64(int(self.state))
            lib.wl_u64(ctypes.byref(st), out.ctypes.data, n)
            self.state = np.uint64(st.value)
            return out
        with np.errstate(over="ignore"):
            idx = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + idx * _GAMMA
            self.state = self.state + np.uint64(n) * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform_mod(self, p: int, n: int) -> np.ndarray:
        """n residues uniform in [0, p), by rejection of the top partial block."""
        n = int(n)
        p = int(p)
        lib = self._c()
        if lib is not None and p > 1 and p % 2:
            out = np.empty(n, dtype=np.uint64)
            st = ctypes.c_uint64(int(self.state))
            lib.wl_uniform_mod(ctypes.byref(st), p, out.ctypes.data, n)
            self.state = np.uint64(st.value)
            return out
        limit = np.uint64(((1 << 64) // p) * p - 1)   # accept draws <= limit
        out = np.empty(n, dtype=np.uint64)
        filled = 0
        while filled < n:
            want = n - filled
            draw = self.u64(want + want // 16 + 16)
            ok = draw[draw <= limit]
            take = min(want, ok.size)
            # Rejected/unused draws are consumed; the stream stays deterministic.
            out[filled:filled + take] = ok[:take] % np.uint64(p)
            filled += take
        return out

    def unit(self, n: int) -> np.ndarray:
        """Doubles uniform in [0, 1) from the top 53 bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def log_uniform_int(self, lo: int, hi: int, n: int) -> np.ndarray:
        u = self.unit(n)
        v = np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
        return np.clip(np.rint(v), lo, hi).astype(np.int64)

    def choice(self, k: int, n: int) -> np.ndarray:
        return (self.unit(n) * k).astype(np.int64)

    def exponential(self, rate: float, n: int) -> np.ndarray:
        u = self.unit(n)
        return -np.log1p(-u) / rate

    def limbs(self, n: int) -> np.ndarray:
        """n uniform 32-bit limbs."""
        return (self.u64(n) >> np.uint64(32)).astype(np.uint32)


def rng(config_index: int, sub: int = 0) -> SplitMix64:
    return SplitMix64(SEED_BASE + config_index + (sub << 32))


def pair_batch(p: int, count: int, na: int, nb: int, seed: int):
    """count operand pairs uniform in [0, p): a (count, na), b (count, nb)."""
    g = SplitMix64(seed)
    a = g.uniform_mod(p, count * na).reshape(count, na)
    b = g.uniform_mod(p, count * nb).reshape(count, nb)
    return a, b


def config0():
    """One product mod 998244353 of two length-2048 operands."""
    a, b = pair_batch(P_A, 1, 2048, 2048, SEED_BASE + 0)
    return P_A, a[0], b[0]


def config1(count: int = 256, length: int = 1 << 15):
    """count products mod 3*2^30+1 of two length-2^15 operands (uint32)."""
    a, b = pair_batch(P_B, count, length, length, SEED_BASE + 1)
    return P_B, a.astype(np.uint32), b.astype(np.uint32)


def config2_transform(log2n: int = 24):
    g = SplitMix64(SEED_BASE + 2)
    return P1, g.uniform_mod(P1, 1 << log2n)


def config2_products(count: int = 1024, length: int = 1 << 12):
    a, b = pair_batch(P1, count, length, length, SEED_BASE + 2 + (1 << 32))
    return P1, a, b


def config3_shapes(count: int = 10000, lo: int = 1 << 6, hi: int = 1 << 18):
    """Lengths (same for both operands) and prime index per product."""
    g = SplitMix64(SEED_BASE + 3)
    lengths = g.log_uniform_int(lo, hi, count)
    prime_idx = g.choice(3, count)
    return lengths, prime_idx


def config3_operands(lengths, prime_idx, seed_sub: int = 1):
    """Concatenated operands for the uneven batch; product t uses P[prime_idx[t]]."""
    primes = np.array([P1, P2, P3], dtype=np.uint64)
    g = SplitMix64(SEED_BASE + 3 + (seed_sub << 32))
    a_list, b_list = [], []
    for L, pi in zip(lengths, prime_idx):
        p = int(primes[pi])
        a_list.append(g.uniform_mod(p, int(L)))
        b_list.append(g.uniform_mod(p, int(L)))
    return [int(primes[i]) for i in prime_idx], a_list, b_list


def config4_requests(count: int, rate: float, lo_bits: int = 1 << 14,
                     hi_bits: int = 1 << 28):
    """Poisson stream: (arrival times in s, operand sizes in 32-bit limbs)."""
    g = SplitMix64(SEED_BASE + 4)
    gaps = g.exponential(rate, count)
    bits = g.log_uniform_int(lo_bits, hi_bits, count)
    limbs = np.maximum(1, np.rint(bits / 32.0)).astype(np.int64)
    return np.cumsum(gaps), limbs


def int_operands(nlimbs: int, seed: int):
    g = SplitMix64(seed)
    return g.limbs(nlimbs), g.limbs(nlimbs)
