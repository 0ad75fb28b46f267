"""CPU oracle for the modular NTT / polynomial / integer product path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library: the arithmetic lives in ``oracle.c`` (plain C,
``unsigned __int128``), compiled here with gcc into ``_build/liboracle.so``
and called through ctypes.  Every routine follows a definition from van der
Hoeven, Lecerf and Quintin, "Modular SIMD arithmetic in Mathemagix" (2014):

* ``mulmod`` / ``mulmod_vec``  -- (x y) rem p, the output of Functions 6, 8,
  13 and 16 (Sections 2.2, 2.3, 3.3);
* ``dft`` / ``idft``  -- FFT_w by its definition, in bit-mirrored order
  (Section 5.1, the TFT with l = n), and its inverse;
* ``polymul`` / ``poly_coeff`` -- the schoolbook product over Z/pZ
  (Section 5.2);
* ``intmul`` -- the schoolbook product of integers in 32-bit limbs
  (Section 5.3's integer product);
* ``is_prime``, ``least_generator``, ``root_of_unity``, ``find_prime`` --
  the moduli p = k 2^l + 1 and their roots of unity (Sections 1, 5.1).

``cpu_ntt.c`` (same library) adds ``ntt_polymul_batch``: the textbook
radix-2 transform product, the O(n log n) CPU reference that the benchmark
times beside the schoolbook oracle.  It is not a parity oracle; the tests pin
it to the schoolbook product.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "cpu_ntt.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u64 = ctypes.c_uint64
_sz = ctypes.c_size_t
_p64 = ctypes.POINTER(ctypes.c_uint64)
_p32 = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile oracle.c and cpu_ntt.c into _build/liboracle.so with gcc (OpenMP on)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(s) for s in _SRCS))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp] + _SRCS)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "orc_mulmod": (_u64, [_u64, _u64, _u64]),
            "orc_addmod": (_u64, [_u64, _u64, _u64]),
            "orc_submod": (_u64, [_u64, _u64, _u64]),
            "orc_powmod": (_u64, [_u64, _u64, _u64]),
            "orc_invmod_prime": (_u64, [_u64, _u64]),
            "orc_is_prime": (ctypes.c_int, [_u64]),
            "orc_prime_factors": (ctypes.c_int, [_u64, _p64, ctypes.c_int]),
            "orc_least_generator": (_u64, [_u64]),
            "orc_root_of_unity": (_u64, [_u64, ctypes.c_uint]),
            "orc_find_prime": (ctypes.c_int, [ctypes.c_uint, ctypes.c_uint, ctypes.c_uint, _p64]),
            "orc_bit_mirror": (_u64, [_u64, ctypes.c_uint]),
            "orc_eval": (_u64, [_u64, _p64, _sz, _u64]),
            "orc_dft": (None, [_u64, _u64, _p64, ctypes.c_uint, _p64]),
            "orc_idft": (None, [_u64, _u64, _p64, ctypes.c_uint, _p64]),
            "orc_poly_coeff": (_u64, [_u64, _p64, _sz, _p64, _sz, _sz]),
            "orc_polymul": (None, [_u64, _p64, _sz, _p64, _sz, _p64]),
            "orc_polymul_batch": (None, [_u64, _p64, _sz, _p64, _sz, _sz, _p64]),
            "orc_polymul_ragged": (None, [_p64, _p64, _p64, _p64, _p64, _p64, _p64,
                                          _p64, _p64, _sz]),
            "orc_intmul": (None, [_p32, _sz, _p32, _sz, _p32]),
            "orc_polymat_mul": (None, [_u64, _p64, _p64, _sz, _sz, _p64]),
            "orc_mulmod_vec": (None, [_u64, _p64, _p64, _sz, _p64]),
            "orc_num_threads": (ctypes.c_int, []),
            "orc_ntt_polymul_batch": (ctypes.c_int, [_u64, _p64, _sz, _p64, _sz, _sz, _p64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _u64arr(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint64))


def _ptr64(a: np.ndarray):
    return a.ctypes.data_as(_p64)


def _ptr32(a: np.ndarray):
    return a.ctypes.data_as(_p32)


# ---- scalar arithmetic ------------------------------------------------------

def mulmod(x: int, y: int, p: int) -> int:
    return int(_load().orc_mulmod(x, y, p))


def addmod(x: int, y: int, p: int) -> int:
    return int(_load().orc_addmod(x, y, p))


def submod(x: int, y: int, p: int) -> int:
    return int(_load().orc_submod(x, y, p))


def powmod(b: int, e: int, p: int) -> int:
    return int(_load().orc_powmod(b, e, p))


def invmod_prime(a: int, p: int) -> int:
    return int(_load().orc_invmod_prime(a, p))


def mulmod_vec(p: int, x, y) -> np.ndarray:
    x = _u64arr(x)
    y = _u64arr(y)
    assert x.shape == y.shape
    z = np.empty_like(x)
    _load().orc_mulmod_vec(p, _ptr64(x), _ptr64(y), x.size, _ptr64(z))
    return z


# ---- primes and roots -------------------------------------------------------

def is_prime(n: int) -> bool:
    return bool(_load().orc_is_prime(n))


def prime_factors(n: int) -> list[int]:
    buf = np.zeros(64, dtype=np.uint64)
    k = _load().orc_prime_factors(n, _ptr64(buf), 64)
    return [int(v) for v in buf[:k]]


def least_generator(p: int) -> int:
    return int(_load().orc_least_generator(p))


def root_of_unity(p: int, log2n: int) -> int:
    """g^((p-1)/2^log2n) with g the least generator; 0 if 2^log2n does not divide p-1."""
    return int(_load().orc_root_of_unity(p, log2n))


def find_prime(bits: int, min_l: int, index: int) -> int:
    out = np.zeros(1, dtype=np.uint64)
    rc = _load().orc_find_prime(bits, min_l, index, _ptr64(out))
    if rc != 0:
        raise ValueError("no such prime")
    return int(out[0])


def bit_mirror(i: int, k: int) -> int:
    return int(_load().orc_bit_mirror(i, k))


# ---- transforms and products ------------------------------------------------

def eval_poly(p: int, a, x: int) -> int:
    a = _u64arr(a)
    return int(_load().orc_eval(p, _ptr64(a), a.size, x))


def dft(p: int, w: int, a) -> np.ndarray:
    """out[i] = A(w^[i]_k) for len(a) = 2^k (bit-mirrored order)."""
    a = _u64arr(a)
    k = int(a.size).bit_length() - 1
    assert a.size == 1 << k
    out = np.empty_like(a)
    _load().orc_dft(p, w, _ptr64(a), k, _ptr64(out))
    return out


def idft(p: int, w: int, ahat) -> np.ndarray:
    ahat = _u64arr(ahat)
    k = int(ahat.size).bit_length() - 1
    assert ahat.size == 1 << k
    out = np.empty_like(ahat)
    _load().orc_idft(p, w, _ptr64(ahat), k, _ptr64(out))
    return out


def poly_coeff(p: int, a, b, k: int) -> int:
    a = _u64arr(a)
    b = _u64arr(b)
    return int(_load().orc_poly_coeff(p, _ptr64(a), a.size, _ptr64(b), b.size, k))


def polymul(p: int, a, b) -> np.ndarray:
    a = _u64arr(a)
    b = _u64arr(b)
    if a.size == 0 or b.size == 0:
        return np.zeros(0, dtype=np.uint64)
    c = np.empty(a.size + b.size - 1, dtype=np.uint64)
    _load().orc_polymul(p, _ptr64(a), a.size, _ptr64(b), b.size, _ptr64(c))
    return c


def polymul_batch(p: int, a, b) -> np.ndarray:
    """a: (count, na), b: (count, nb) -> (count, na+nb-1), OpenMP over products."""
    a = _u64arr(a)
    b = _u64arr(b)
    count, na = a.shape
    count2, nb = b.shape
    assert count == count2
    c = np.empty((count, na + nb - 1), dtype=np.uint64)
    _load().orc_polymul_batch(p, _ptr64(a), na, _ptr64(b), nb, count, _ptr64(c))
    return c


def ntt_polymul_batch(p: int, a, b) -> np.ndarray:
    """a: (count, na), b: (count, nb) -> (count, na+nb-1) through the textbook
    radix-2 transform product (cpu_ntt.c), OpenMP over products.  The CPU
    timing reference; parity is checked against polymul_batch."""
    a = _u64arr(a)
    b = _u64arr(b)
    count, na = a.shape
    count2, nb = b.shape
    assert count == count2
    c = np.empty((count, na + nb - 1), dtype=np.uint64)
    rc = _load().orc_ntt_polymul_batch(p, _ptr64(a), na, _ptr64(b), nb, count, _ptr64(c))
    if rc != 0:
        raise MemoryError("orc_ntt_polymul_batch: scratch allocation failed")
    return c


def polymul_ragged(ps, a_list, b_list) -> list[np.ndarray]:
    """Products of uneven lengths, each with its own modulus (OpenMP over products)."""
    count = len(ps)
    na = np.array([len(x) for x in a_list], dtype=np.uint64)
    nb = np.array([len(x) for x in b_list], dtype=np.uint64)
    nc = na + nb - 1
    aoff = np.concatenate([[0], np.cumsum(na)[:-1]]).astype(np.uint64)
    boff = np.concatenate([[0], np.cumsum(nb)[:-1]]).astype(np.uint64)
    coff = np.concatenate([[0], np.cumsum(nc)[:-1]]).astype(np.uint64)
    a = _u64arr(np.concatenate(a_list))
    b = _u64arr(np.concatenate(b_list))
    c = np.empty(int(nc.sum()), dtype=np.uint64)
    psa = _u64arr(ps)
    _load().orc_polymul_ragged(_ptr64(psa), _ptr64(a), _ptr64(aoff), _ptr64(na),
                               _ptr64(b), _ptr64(boff), _ptr64(nb), _ptr64(c),
                               _ptr64(coff), count)
    return [c[int(coff[t]):int(coff[t] + nc[t])] for t in range(count)]


def polymat_mul(p: int, A, B) -> np.ndarray:
    """A, B: (n, n, d) -> C: (n, n, 2d-1), C_ij = sum_l A_il B_lj over Z/pZ."""
    A = _u64arr(A)
    B = _u64arr(B)
    n, n2, d = A.shape
    assert n == n2 and B.shape == A.shape
    C = np.empty((n, n, 2 * d - 1), dtype=np.uint64)
    _load().orc_polymat_mul(p, _ptr64(A), _ptr64(B), n, d, _ptr64(C))
    return C


def intmul(a, b) -> np.ndarray:
    """Schoolbook product of little-endian uint32 limb arrays -> na+nb limbs."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.uint32))
    c = np.empty(a.size + b.size, dtype=np.uint32)
    _load().orc_intmul(_ptr32(a), a.size, _ptr32(b), b.size, _ptr32(c))
    return c


def num_threads() -> int:
    return int(_load().orc_num_threads())
