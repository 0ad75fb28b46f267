"""Pins for the CPU oracle: checks against facts fixed by the paper and by
the mathematics (closed forms, invariants, brute force on tiny inputs), each
chosen so that a dropped term, a wrong sign/index or a transposed operand in
oracle/oracle.c fails at least one of them.  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1407_3383_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

NTT_PRIMES = [W.P_A, W.P_B, W.P_TABLE11, W.P_TABLE12, W.P1, W.P2, W.P3,
              985661441, 943718401]


def _paper_primes():
    rows = []
    with open(os.path.join(GOLDEN, "paper_primes.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p, k, l, *_ = line.split()
            rows.append((int(p), int(k), int(l)))
    return rows


# ---------------------------------------------------------------- modular products

@pytest.mark.parametrize("p", [2, 3, 5, 7, 17, 97, 193, 257, 1000])
def test_mulmod_exhaustive_vs_repeated_addition(p):
    """x*y rem p equals y-fold repeated modular addition of x (a different
    algorithm), for every x, y < p."""
    xs = np.repeat(np.arange(p, dtype=np.uint64), p)
    ys = np.tile(np.arange(p, dtype=np.uint64), p)
    got = O.mulmod_vec(p, xs, ys).reshape(p, p)
    for x in range(p):
        acc = 0
        row = got[x]
        for y in range(p):
            assert int(row[y]) == acc
            acc += x
            if acc >= p:
                acc -= p


@pytest.mark.parametrize("p", NTT_PRIMES)
def test_mulmod_fermat_and_closed_forms(p):
    g = W.SplitMix64(p)
    xs = g.uniform_mod(p, 64)
    for x in xs:
        x = int(x)
        if x:
            assert O.powmod(x, p - 1, p) == 1          # Fermat
            assert O.mulmod(x, O.invmod_prime(x, p), p) == 1
    assert O.mulmod(p - 1, p - 1, p) == 1              # (-1)^2 = 1
    assert O.addmod(p - 1, 1, p) == 0
    assert O.submod(0, 1, p) == p - 1
    # p = k 2^l + 1  =>  k * 2^l = -1 (mod p)
    l = (p - 1 & -(p - 1)).bit_length() - 1
    k = (p - 1) >> l
    assert O.mulmod(k, O.powmod(2, l, p), p) == p - 1


def test_mulmod_extreme_operands_match_bigint():
    """Operands near 2^64 (where a 64-bit truncation would show) against
    Python's arbitrary-precision integers."""
    p = (1 << 64) - 59   # largest prime below 2^64
    assert O.is_prime(p)
    for x, y in [(p - 1, p - 1), (p - 2, 2), ((1 << 63) + 5, (1 << 63) + 7), (1 << 63, 3)]:
        assert O.mulmod(x, y, p) == (x * y) % p


def test_wilson_small_primes():
    for p in [5, 7, 13, 17, 97, 193, 257, 7681, 12289]:
        acc = 1
        for i in range(1, p):
            acc = O.mulmod(acc, i, p)
        assert acc == p - 1


# ---------------------------------------------------------------- primes

def test_paper_primes_golden():
    for p, k, l in _paper_primes():
        assert O.is_prime(p)
        assert p == k * (1 << l) + 1 and k % 2 == 1
        assert O.root_of_unity(p, l) != 0
        assert O.root_of_unity(p, l + 1) == 0


def _sieve(n):
    s = bytearray([1]) * n
    s[0] = s[1] = 0
    for i in range(2, int(n ** 0.5) + 1):
        if s[i]:
            s[i * i::i] = bytearray(len(s[i * i::i]))
    return s


def test_is_prime_vs_sieve():
    s = _sieve(30000)
    for n in range(30000):
        assert O.is_prime(n) == bool(s[n]), n


def test_is_prime_rejects_strong_pseudoprimes():
    # Composite numbers (factorisations checked here) that pass Miller-Rabin
    # for the first few prime bases; the last passes every base up to 31.
    cases = {2047: [23, 89], 1373653: [829, 1657], 25326001: [2251, 11251],
             3215031751: [151, 751, 28351],
             2152302898747: [6763, 10627, 29947],
             3474749660383: [1303, 16927, 157543],
             341550071728321: [10670053, 32010157],
             3825123056546413051: [149491, 747451, 34233211],
             (1 << 59) - 1: [179951, 3203431780337]}
    for n, fac in cases.items():
        assert math.prod(fac) == n
        assert not O.is_prime(n)
    for n in [561, 1105, 1729, 2465, 2821, 6601, 8911, 41041]:   # Carmichael
        assert not O.is_prime(n)
    for e in [31, 61]:                                            # Mersenne primes
        assert O.is_prime((1 << e) - 1)


def test_prime_factors_vs_trial_division():
    for n in range(2, 5000):
        want = []
        m = n
        d = 2
        while d * d <= m:
            if m % d == 0:
                want.append(d)
                while m % d == 0:
                    m //= d
            d += 1
        if m > 1:
            want.append(m)
        assert sorted(O.prime_factors(n)) == want
    assert sorted(O.prime_factors(W.P_A - 1)) == [2, 7, 17]       # 2^23 * 7 * 17


def _order(g, p):
    x, k = g % p, 1
    while x != 1:
        x = x * g % p
        k += 1
    return k


def test_least_generator_brute_force():
    s = _sieve(2000)
    for p in range(3, 2000):
        if not s[p]:
            continue
        g = O.least_generator(p)
        assert _order(g, p) == p - 1
        for h in range(2, g):
            assert _order(h, p) < p - 1


def test_least_generator_workload_primes():
    # The workload statement for 998244353 names 3 as its primitive root.
    assert O.least_generator(W.P_A) == 3
    for p in [W.P_B, W.P1, W.P2, W.P3, W.P_TABLE11]:
        g = O.least_generator(p)
        for q in O.prime_factors(p - 1):
            assert O.powmod(g, (p - 1) // q, p) != 1


@pytest.mark.parametrize("p", NTT_PRIMES)
def test_root_of_unity_has_exact_order(p):
    v2 = (p - 1 & -(p - 1)).bit_length() - 1
    for log2n in sorted({1, 2, 5, 12, min(v2, 16), v2}):
        w = O.root_of_unity(p, log2n)
        n = 1 << log2n
        assert O.powmod(w, n, p) == 1
        assert O.powmod(w, n // 2, p) == p - 1     # so the order is exactly n
        if log2n < v2:
            w2 = O.root_of_unity(p, log2n + 1)
            assert O.mulmod(w2, w2, p) == w
    assert O.root_of_unity(p, v2 + 1) == 0


def test_find_prime_62bit():
    got = [O.find_prime(62, 40, i) for i in range(3)]
    assert got == [W.P1, W.P2, W.P3]
    step = 1 << 40
    for p in got:
        assert (1 << 61) < p < (1 << 62) and (p - 1) % step == 0 and O.is_prime(p)
    # nothing prime was skipped between 2^61 and P3
    k0 = (1 << 61) // step + 1
    hits = [k for k in range(k0, (W.P3 - 1) // step + 1) if O.is_prime(k * step + 1)]
    assert [k * step + 1 for k in hits] == got


def test_bit_mirror():
    assert [O.bit_mirror(i, 3) for i in range(8)] == [0, 4, 2, 6, 1, 5, 3, 7]
    for k in [1, 5, 11]:
        for i in range(0, 1 << k, max(1, (1 << k) // 64)):
            assert O.bit_mirror(i, k) == int(format(i, f"0{k}b")[::-1], 2)


# ---------------------------------------------------------------- transforms

def test_dft_hand_example_f17():
    # p = 17, least generator 3, w = 3^4 = 13 (order 4).  A = 1 + 2X + 3X^2 + 4X^3.
    # Bit-mirrored order evaluates at w^0, w^2, w^1, w^3 = 1, 16, 13, 4:
    # A(1) = 10, A(16) = A(-1) = -2 = 15, A(13) = 9322 = 6, A(4) = 313 = 7 (mod 17).
    assert O.root_of_unity(17, 2) == 13
    assert O.dft(17, 13, [1, 2, 3, 4]).tolist() == [10, 15, 6, 7]


@pytest.mark.parametrize("p,k", [(W.P_A, 6), (W.P_B, 5), (W.P1, 7), (17, 4)])
def test_dft_special_inputs(p, k):
    n = 1 << k
    w = O.root_of_unity(p, k)
    delta = np.zeros(n, dtype=np.uint64)
    delta[0] = 1
    assert (O.dft(p, w, delta) == 1).all()
    c = 12345 % p
    const = np.full(n, c, dtype=np.uint64)
    out = O.dft(p, w, const)
    assert int(out[0]) == n * c % p and (out[1:] == 0).all()
    e1 = np.zeros(n, dtype=np.uint64)
    e1[1] = 1
    out = O.dft(p, w, e1)
    for i in range(n):
        rev = int(format(i, f"0{k}b")[::-1], 2)
        assert int(out[i]) == pow(w, rev, p)


@pytest.mark.parametrize("p,k", [(W.P_A, 6), (W.P1, 5)])
def test_dft_geometric_closed_form(p, k):
    """a_j = r^j has A(x) = (1 - (r x)^n) / (1 - r x) = (1 - r^n) / (1 - r x)."""
    n = 1 << k
    w = O.root_of_unity(p, k)
    r = 987654321 % p
    a = [pow(r, j, p) for j in range(n)]
    out = O.dft(p, w, a)
    for i in range(n):
        x = pow(w, int(format(i, f"0{k}b")[::-1], 2), p)
        den = (1 - r * x) % p
        assert den != 0
        assert int(out[i]) == (1 - pow(r, n, p)) * pow(den, -1, p) % p


def _textbook_fft(a, w, p):
    """Recursive radix-2 Cooley-Tukey in natural order (a different algorithm)."""
    n = len(a)
    if n == 1:
        return list(a)
    ev = _textbook_fft(a[0::2], w * w % p, p)
    od = _textbook_fft(a[1::2], w * w % p, p)
    out = [0] * n
    t = 1
    for i in range(n // 2):
        out[i] = (ev[i] + t * od[i]) % p
        out[i + n // 2] = (ev[i] - t * od[i]) % p
        t = t * w % p
    return out


@pytest.mark.parametrize("p,k", [(W.P_A, 8), (W.P_B, 7), (W.P2, 9), (W.P_TABLE12, 6)])
def test_dft_matches_textbook_fft_and_inverts(p, k):
    n = 1 << k
    w = O.root_of_unity(p, k)
    a = W.SplitMix64(k * 7 + 1).uniform_mod(p, n)
    got = O.dft(p, w, a)
    nat = _textbook_fft([int(v) for v in a], w, p)
    want = [nat[int(format(i, f"0{k}b")[::-1], 2)] for i in range(n)]
    assert got.tolist() == want
    assert (O.idft(p, w, got) == a).all()
    # linearity
    b = W.SplitMix64(k * 7 + 2).uniform_mod(p, n)
    s = (a.astype(object) + b.astype(object)) % p
    assert (O.dft(p, w, s).astype(object) == (got.astype(object) + O.dft(p, w, b).astype(object)) % p).all()


def test_convolution_theorem():
    p, k = W.P_A, 6
    n = 1 << k
    w = O.root_of_unity(p, k)
    g = W.SplitMix64(99)
    a = g.uniform_mod(p, n // 2)
    b = g.uniform_mod(p, n // 2)
    c = O.polymul(p, a, b)                      # length n - 1 < n: no wrap
    pad = lambda v: np.concatenate([v, np.zeros(n - v.size, dtype=np.uint64)])
    lhs = O.dft(p, w, pad(c))
    rhs = O.mulmod_vec(p, O.dft(p, w, pad(a)), O.dft(p, w, pad(b)))
    assert (lhs == rhs).all()


# ---------------------------------------------------------------- polynomial products

@pytest.mark.parametrize("p", [W.P_A, W.P_B, W.P1, 17])
def test_polymul_binomials(p):
    m, n = 300, 217
    a = [math.comb(m, i) % p for i in range(m + 1)]
    b = [math.comb(n, i) % p for i in range(n + 1)]
    c = O.polymul(p, a, b)
    assert c.tolist() == [math.comb(m + n, i) % p for i in range(m + n + 1)]


def test_polymul_geometric_times_one_minus_x():
    p = W.P3
    n = 1000
    c = O.polymul(p, np.ones(n, dtype=np.uint64), [1, p - 1])
    want = np.zeros(n + 1, dtype=np.uint64)
    want[0] = 1
    want[n] = p - 1
    assert (c == want).all()


@pytest.mark.parametrize("p", [W.P1, W.P_B])
def test_polymul_all_minus_one(p):
    """a_i = b_j = p - 1: c_k = (#terms) * (p-1)^2 = #terms (mod p).  Long
    sums of maximal 62-bit products exercise the accumulator's reductions."""
    na, nb = 700, 333
    c = O.polymul(p, np.full(na, p - 1, dtype=np.uint64), np.full(nb, p - 1, dtype=np.uint64))
    for k in range(na + nb - 1):
        terms = min(k, na - 1) - max(0, k - nb + 1) + 1
        assert int(c[k]) == terms % p


def test_polymul_kronecker_bigint():
    """Exact integer convolution via Kronecker substitution in Python big
    integers, then reduced mod p (an independent exact method)."""
    p = W.P2
    g = W.SplitMix64(5)
    a = g.uniform_mod(p, 97)
    b = g.uniform_mod(p, 64)
    B = 2 * 62 + 8
    A = sum(int(v) << (B * i) for i, v in enumerate(a))
    Bv = sum(int(v) << (B * i) for i, v in enumerate(b))
    C = A * Bv
    mask = (1 << B) - 1
    want = [((C >> (B * k)) & mask) % p for k in range(a.size + b.size - 1)]
    assert O.polymul(p, a, b).tolist() == want
    for k in [0, 5, 96, 159]:
        assert O.poly_coeff(p, a, b, k) == want[k]


def test_polymul_edges_and_batches():
    p = W.P_A
    assert O.polymul(p, [5], [7]).tolist() == [35]
    assert O.polymul(p, [], [1, 2]).size == 0
    g = W.SplitMix64(11)
    a = g.uniform_mod(p, 4 * 50).reshape(4, 50)
    b = g.uniform_mod(p, 4 * 30).reshape(4, 30)
    cb = O.polymul_batch(p, a, b)
    for t in range(4):
        assert (cb[t] == O.polymul(p, a[t], b[t])).all()
    ps = [W.P1, W.P2, W.P3]
    al = [g.uniform_mod(q, n) for q, n in zip(ps, [3, 40, 17])]
    bl = [g.uniform_mod(q, n) for q, n in zip(ps, [9, 1, 17])]
    cr = O.polymul_ragged(ps, al, bl)
    for q, x, y, z in zip(ps, al, bl, cr):
        assert (z == O.polymul(q, x, y)).all()


# ---------------------------------------------------------------- integer products

def _to_int(limbs):
    return sum(int(v) << (32 * i) for i, v in enumerate(limbs))


@pytest.mark.parametrize("na,nb", [(1, 1), (3, 7), (64, 64), (257, 100)])
def test_intmul_vs_python_int(na, nb):
    g = W.SplitMix64(na * 1000 + nb)
    a = g.limbs(na)
    b = g.limbs(nb)
    c = O.intmul(a, b)
    assert c.size == na + nb
    assert _to_int(c) == _to_int(a) * _to_int(b)


def test_intmul_all_ones_closed_form():
    n = 200
    a = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
    c = O.intmul(a, a)
    # (2^(32n) - 1)^2 = 2^(64n) - 2^(32n+1) + 1
    want = (1 << (64 * n)) - (1 << (32 * n + 1)) + 1
    assert _to_int(c) == want
    assert int(c[0]) == 1 and int(c[n]) == 0xFFFFFFFE


# ---------------------------------------------------------------- inputs

def test_splitmix64_reference_output():
    # First outputs of splitmix64 seeded with 0 (reference implementation).
    g = W.SplitMix64(0)
    assert [int(v) for v in g.u64(2)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_uniform_mod_deterministic_and_in_range():
    for p in [W.P_B, W.P1, 3]:
        x = W.SplitMix64(7).uniform_mod(p, 10000)
        y = W.SplitMix64(7).uniform_mod(p, 10000)
        assert (x == y).all() and int(x.max()) < p
    # with p = 3 every residue appears with frequency close to 1/3
    x = W.SplitMix64(8).uniform_mod(3, 30000)
    assert np.all(np.abs(np.bincount(x.astype(np.int64)) - 10000) < 400)


# ---------------------------------------------------------------- polynomial matrices

def test_polymat_mul_reduces_to_polymul_and_identity():
    p = W.P_TABLE11
    g = W.SplitMix64(31)
    A = g.uniform_mod(p, 1 * 1 * 40).reshape(1, 1, 40)
    B = g.uniform_mod(p, 1 * 1 * 40).reshape(1, 1, 40)
    assert (O.polymat_mul(p, A, B)[0, 0] == O.polymul(p, A[0, 0], B[0, 0])).all()
    n, d = 4, 9
    I = np.zeros((n, n, d), dtype=np.uint64)
    for i in range(n):
        I[i, i, 0] = 1
    B = g.uniform_mod(p, n * n * d).reshape(n, n, d)
    C = O.polymat_mul(p, I, B)
    assert (C[:, :, :d] == B).all() and (C[:, :, d:] == 0).all()


def test_polymat_mul_entry_sums():
    """Each entry is the sum over l of separate products (Python big-int sums)."""
    p = W.P_B
    g = W.SplitMix64(32)
    n, d = 3, 17
    A = g.uniform_mod(p, n * n * d).reshape(n, n, d)
    B = g.uniform_mod(p, n * n * d).reshape(n, n, d)
    C = O.polymat_mul(p, A, B)
    for i in range(n):
        for j in range(n):
            acc = np.zeros(2 * d - 1, dtype=object)
            for l in range(n):
                acc = acc + O.polymul(p, A[i, l], B[l, j]).astype(object)
            assert (C[i, j].astype(object) == acc % p).all()


@pytest.mark.parametrize("p", [W.P_A, W.P_B, W.P1, 17])
def test_cpu_ntt_reference_equals_schoolbook(p):
    """The O(n log n) CPU reference (cpu_ntt.c, timed by the benchmark) gives
    the schoolbook products word for word: ragged and degree-0 operands,
    sizes from one word to 2^12 points, and all-(p-1) operands."""
    g = W.SplitMix64(0xC0DE + p % 1009)
    shapes = [(1, 1), (1, 7), (3, 5), (16, 17), (100, 29), (1024, 1024), (2048, 2047)]
    if p == 17:                                  # 17 - 1 = 2^4: transforms of at most 16 points
        shapes = [(1, 1), (2, 3), (8, 9), (5, 12)]
    for na, nb in shapes:
        a = g.uniform_mod(p, 3 * na).reshape(3, na)
        b = g.uniform_mod(p, 3 * nb).reshape(3, nb)
        assert (O.ntt_polymul_batch(p, a, b) == O.polymul_batch(p, a, b)).all(), (p, na, nb)
    n = 8 if p == 17 else 512
    a = np.full((1, n), p - 1, dtype=np.uint64)
    assert (O.ntt_polymul_batch(p, a, a) == O.polymul_batch(p, a, a)).all()
