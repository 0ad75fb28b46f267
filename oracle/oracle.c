/*
 * oracle.c -- CPU oracle for the modular NTT / polynomial / integer product
 * path.  TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and
 * the CPU-baseline leg of bench.py may load this library.  The product path
 * (the CUDA library) shares no code, header, table or helper with it.
 *
 * Every function below computes its result straight from the definition of
 * the quantity (schoolbook sums, evaluation by Horner's rule, square-and-
 * multiply powers), in exact integer arithmetic with unsigned __int128 for
 * the double-width products.  Nothing here uses an NTT, a precomputed
 * quotient, Montgomery form or any blocking/reordering: it is meant to be
 * checked against van der Hoeven, Lecerf and Quintin, "Modular SIMD
 * arithmetic in Mathemagix" (2014) by eye.
 *
 * Residues are represented by their representative in {0, ..., p-1}
 * (Section 2, the convention stated before Section 2.1).
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* (x * y) rem p for x, y < p < 2^64: the plain definition of the modular
 * product that Functions 6, 8, 13 and 16 all compute (Sections 2.2-3.3). */
uint64_t orc_mulmod(uint64_t x, uint64_t y, uint64_t p) {
    return (uint64_t)(((u128)x * (u128)y) % p);
}

/* (x + y) rem p (Section 2.1, Function 1's output), exact in 65 bits. */
uint64_t orc_addmod(uint64_t x, uint64_t y, uint64_t p) {
    return (uint64_t)(((u128)x + (u128)y) % p);
}

/* (x - y) rem p for x, y < p. */
uint64_t orc_submod(uint64_t x, uint64_t y, uint64_t p) {
    return (uint64_t)(((u128)x + (u128)p - (u128)y) % p);
}

/* b^e rem p by square-and-multiply. */
uint64_t orc_powmod(uint64_t b, uint64_t e, uint64_t p) {
    uint64_t r = 1 % p;
    b %= p;
    while (e) {
        if (e & 1) r = orc_mulmod(r, b, p);
        b = orc_mulmod(b, b, p);
        e >>= 1;
    }
    return r;
}

/* Inverse of a modulo a prime p by Fermat's little theorem: a^(p-2). */
uint64_t orc_invmod_prime(uint64_t a, uint64_t p) {
    return orc_powmod(a, p - 2, p);
}

/* Deterministic Miller-Rabin for n < 2^64 with the first twelve prime bases
 * (correct for all n < 3.3e24).  Used to check that p = k 2^l + 1 is prime
 * (Section 1: FFTs over F_p with p = k 2^l + 1). */
int orc_is_prime(uint64_t n) {
    static const uint64_t small[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == small[i]) return 1;
        if (n % small[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = orc_powmod(small[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; r++) {
            x = orc_mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* Distinct prime factors of n (n >= 2) by trial division, stopping early
 * when the remaining cofactor is prime.  Returns their count. */
int orc_prime_factors(uint64_t n, uint64_t* f, int max_f) {
    int k = 0;
    if (n < 2) return 0;
    for (uint64_t d = 2; n > 1; d = (d == 2) ? 3 : d + 2) {
        if (orc_is_prime(n)) {
            if (k < max_f) f[k++] = n;
            break;
        }
        if (d * d > n) {
            if (k < max_f) f[k++] = n;
            break;
        }
        if (n % d == 0) {
            if (k < max_f) f[k++] = d;
            while (n % d == 0) n /= d;
        }
    }
    return k;
}

/* The least generator of the multiplicative group F_p^* (p prime): the
 * smallest g with g^((p-1)/q) != 1 for every prime q dividing p - 1. */
uint64_t orc_least_generator(uint64_t p) {
    uint64_t f[64];
    if (p == 2) return 1;
    int k = orc_prime_factors(p - 1, f, 64);
    for (uint64_t g = 2; g < p; g++) {
        int ok = 1;
        for (int i = 0; i < k; i++)
            if (orc_powmod(g, (p - 1) / f[i], p) == 1) { ok = 0; break; }
        if (ok) return g;
    }
    return 0;
}

/* A primitive n-th root of unity, n = 2^log2n dividing p - 1: the power
 * g^((p-1)/n) of the least generator g (Section 5.1 asks only for some
 * primitive n-th root; this fixes the choice).  Returns 0 if 2^log2n does
 * not divide p - 1. */
uint64_t orc_root_of_unity(uint64_t p, unsigned log2n) {
    if (log2n >= 64) return 0;
    uint64_t n = (uint64_t)1 << log2n;
    if ((p - 1) % n != 0) return 0;
    return orc_powmod(orc_least_generator(p), (p - 1) / n, p);
}

/* The index-th prime (0-based) of the form p = k 2^min_l + 1 with
 * 2^(bits-1) < p < 2^bits, for ascending k.  Returns 0 on success. */
int orc_find_prime(unsigned bits, unsigned min_l, unsigned index, uint64_t* out) {
    if (bits < 3 || bits > 63 || min_l >= bits - 1) return -1;
    uint64_t lo = (uint64_t)1 << (bits - 1);
    uint64_t step = (uint64_t)1 << min_l;
    uint64_t k = lo / step + 1;
    unsigned found = 0;
    for (;; k++) {
        u128 p = (u128)k * step + 1;
        if (p >> bits) return -1;
        if (orc_is_prime((uint64_t)p)) {
            if (found == index) { *out = (uint64_t)p; return 0; }
            found++;
        }
    }
}

/* Bitwise mirror [i]_k of i in length k (Section 5.1). */
uint64_t orc_bit_mirror(uint64_t i, unsigned k) {
    uint64_t r = 0;
    for (unsigned j = 0; j < k; j++) r |= ((i >> j) & 1) << (k - 1 - j);
    return r;
}

/* A(x) rem p for A = a_0 + a_1 X + ... + a_{n-1} X^{n-1}, by Horner's rule. */
uint64_t orc_eval(uint64_t p, const uint64_t* a, size_t n, uint64_t x) {
    uint64_t acc = 0;
    for (size_t j = n; j-- > 0;) acc = orc_addmod(orc_mulmod(acc, x, p), a[j] % p, p);
    return acc;
}

/* FFT_w of (a_0, ..., a_{n-1}), n = 2^k, listed in bit-mirrored order as
 * in the TFT definition with l = n (Section 5.1):
 *     out[i] = A(w^[i]_k) = sum_j w^([i]_k j) a_j.
 * Quadratic: one Horner evaluation per output. */
void orc_dft(uint64_t p, uint64_t w, const uint64_t* a, unsigned k, uint64_t* out) {
    size_t n = (size_t)1 << k;
    for (size_t i = 0; i < n; i++)
        out[i] = orc_eval(p, a, n, orc_powmod(w, orc_bit_mirror(i, k), p));
}

/* Inverse of orc_dft: given ahat in bit-mirrored order (position i holds
 * A(w^[i]_k)), return a_j = n^{-1} sum_m A(w^m) w^{-jm}. */
void orc_idft(uint64_t p, uint64_t w, const uint64_t* ahat, unsigned k, uint64_t* out) {
    size_t n = (size_t)1 << k;
    uint64_t winv = orc_invmod_prime(w, p);
    uint64_t ninv = orc_invmod_prime(n % p, p);
    for (size_t j = 0; j < n; j++) {
        uint64_t wj = orc_powmod(winv, j, p);
        uint64_t wjm = 1; /* w^{-jm}, m = 0, 1, ... */
        uint64_t acc = 0;
        for (size_t m = 0; m < n; m++) {
            uint64_t v = ahat[orc_bit_mirror(m, k)];
            acc = orc_addmod(acc, orc_mulmod(v, wjm, p), p);
            wjm = orc_mulmod(wjm, wj, p);
        }
        out[j] = orc_mulmod(acc, ninv, p);
    }
}

/* One coefficient c_k = sum_{i+j=k} a_i b_j rem p of the product of two
 * polynomials of degrees < na and < nb (Section 5.2's polynomial product). */
uint64_t orc_poly_coeff(uint64_t p, const uint64_t* a, size_t na,
                        const uint64_t* b, size_t nb, size_t k) {
    size_t i0 = (k + 1 > nb) ? k + 1 - nb : 0;
    size_t i1 = (k < na - 1) ? k : na - 1;
    u128 acc = 0;
    unsigned pending = 0;
    /* each term is < p^2; with p < 2^62 eight of them stay below 2^127, so
     * reducing the running sum every 8 terms keeps it from wrapping */
    const unsigned batch = (p >> 62) ? 1u : 8u;
    if (na == 0 || nb == 0 || k > na + nb - 2) return 0;
    for (size_t i = i0; i <= i1; i++) {
        acc += (u128)(a[i] % p) * (u128)(b[k - i] % p);
        if (++pending == batch) { acc %= p; pending = 0; }
    }
    return (uint64_t)(acc % p);
}

/* Schoolbook product c = a b over Z/pZ, c of length na + nb - 1. */
void orc_polymul(uint64_t p, const uint64_t* a, size_t na,
                 const uint64_t* b, size_t nb, uint64_t* c) {
    if (na == 0 || nb == 0) return;
    for (size_t k = 0; k < na + nb - 1; k++) c[k] = orc_poly_coeff(p, a, na, b, nb, k);
}

/* count independent products of equal shapes, laid out back to back:
 * a[t*na ..], b[t*nb ..], c[t*(na+nb-1) ..].  Products are spread over
 * OpenMP threads when the library is built with OpenMP. */
void orc_polymul_batch(uint64_t p, const uint64_t* a, size_t na,
                       const uint64_t* b, size_t nb, size_t count, uint64_t* c) {
    if (na == 0 || nb == 0) return;
    const size_t nc = na + nb - 1;
    long long idx;
    /* one work item per output coefficient of every product */
#pragma omp parallel for schedule(dynamic, 256)
    for (idx = 0; idx < (long long)(count * nc); idx++) {
        const size_t t = (size_t)idx / nc, k = (size_t)idx % nc;
        c[idx] = orc_poly_coeff(p, a + t * na, na, b + t * nb, nb, k);
    }
}

/* Products of uneven shapes and moduli: product t has modulus ps[t],
 * operands a[aoff[t] .. aoff[t]+na[t]), b[boff[t] ..) and output
 * c[coff[t] .. coff[t]+na[t]+nb[t]-1). */
void orc_polymul_ragged(const uint64_t* ps, const uint64_t* a, const uint64_t* aoff,
                        const uint64_t* na, const uint64_t* b, const uint64_t* boff,
                        const uint64_t* nb, uint64_t* c, const uint64_t* coff, size_t count) {
    long long t;
#pragma omp parallel for schedule(dynamic, 1)
    for (t = 0; t < (long long)count; t++)
        orc_polymul(ps[t], a + aoff[t], na[t], b + boff[t], nb[t], c + coff[t]);
}

/* Product of two n x n matrices of polynomials over Z/pZ (Section 5.2's
 * polynomial matrix product), straight from the definition:
 * C_ij = sum_l A_il B_lj, each A_il B_lj a schoolbook polynomial product.
 * A, B: entry (i, j) at ((i n + j) d ...), d coefficients each; C: entry
 * (i, j) at ((i n + j)(2d - 1) ...).  OpenMP over the entries of C. */
void orc_polymat_mul(uint64_t p, const uint64_t* A, const uint64_t* B, size_t n, size_t d, uint64_t* C) {
    const size_t dc = 2 * d - 1;
    long long e;
#pragma omp parallel for schedule(dynamic, 1)
    for (e = 0; e < (long long)(n * n); e++) {
        const size_t i = (size_t)e / n, j = (size_t)e % n;
        uint64_t* c = C + (size_t)e * dc;
        for (size_t k = 0; k < dc; k++) c[k] = 0;
        for (size_t l = 0; l < n; l++) {
            const uint64_t* a = A + (i * n + l) * d;
            const uint64_t* b = B + (l * n + j) * d;
            for (size_t k = 0; k < dc; k++) c[k] = orc_addmod(c[k], orc_poly_coeff(p, a, d, b, d, k), p);
        }
    }
}

/* Schoolbook product of two non-negative integers given as little-endian
 * 32-bit limbs (Section 5.3 multiplies integers a, b of at most N bits).
 * c has na + nb limbs. */
void orc_intmul(const uint32_t* a, size_t na, const uint32_t* b, size_t nb, uint32_t* c) {
    memset(c, 0, (na + nb) * sizeof(uint32_t));
    for (size_t i = 0; i < na; i++) {
        uint64_t carry = 0;
        for (size_t j = 0; j < nb; j++) {
            uint64_t t = (uint64_t)a[i] * b[j] + c[i + j] + carry;
            c[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        c[i + nb] = (uint32_t)carry;
    }
}

/* Element-wise modular products z_i = (x_i y_i) rem p. */
void orc_mulmod_vec(uint64_t p, const uint64_t* x, const uint64_t* y, size_t n, uint64_t* z) {
    for (size_t i = 0; i < n; i++) z[i] = orc_mulmod(x[i], y[i], p);
}

/* Number of OpenMP threads a parallel region of this library uses. */
int orc_num_threads(void) {
    int n = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
#endif
    return n;
}
