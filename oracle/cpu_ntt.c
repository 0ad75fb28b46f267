/*
 * cpu_ntt.c -- the textbook radix-2 number-theoretic transform product on
 * the CPU, the O(n log n) CPU reference that the benchmark times beside the
 * schoolbook oracle.  TEST INFRASTRUCTURE ONLY, like oracle.c (built into
 * the same library): only tests/, __graft_entry__.smoke() and the CPU leg of
 * bench.py may load it, and the CUDA library shares nothing with it.
 *
 * It is not the parity oracle: the GPU results are compared with oracle.c's
 * schoolbook products, and the tests pin this routine to those as well.
 *
 * What it computes (Section 5.2's product through Section 5.1's transform):
 * with n = 2^k >= na + nb - 1 and w a primitive n-th root of unity,
 *     c = n^-1 FFT_{w^-1}( FFT_w(a) * FFT_w(b) )
 * truncated to its first na + nb - 1 coefficients, which is the product
 * a b over Z/pZ by the convolution theorem.  Each transform is the
 * iterative Cooley-Tukey form: operands permuted into bit-mirrored order,
 * then log2 n passes of butterflies (u, v) -> (u + v w^j, u - v w^j) over
 * blocks of length 2, 4, ..., n, with the block's root w^(n/len) stepped
 * by one product per butterfly.  Every product is (u128) x y rem p; sums
 * and differences are reduced by one comparison.  No lazy reduction, no
 * precomputed quotients, no vector instructions.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

typedef unsigned __int128 u128;

uint64_t orc_powmod(uint64_t b, uint64_t e, uint64_t p);
uint64_t orc_invmod_prime(uint64_t a, uint64_t p);
uint64_t orc_root_of_unity(uint64_t p, unsigned log2n);
uint64_t orc_bit_mirror(uint64_t i, unsigned k);

static uint64_t mul(uint64_t x, uint64_t y, uint64_t p) { return (uint64_t)(((u128)x * y) % p); }
static uint64_t add(uint64_t x, uint64_t y, uint64_t p) { uint64_t s = x + y; return s >= p ? s - p : s; }
static uint64_t sub(uint64_t x, uint64_t y, uint64_t p) { return x >= y ? x - y : x + p - y; }

/* In-place transform of x (n = 2^k words) with the primitive n-th root w:
 * natural order in, natural order out (x_i <- sum_j w^(ij) x_j). */
static void ntt_inplace(uint64_t* x, unsigned k, uint64_t w, uint64_t p) {
    const size_t n = (size_t)1 << k;
    for (size_t i = 0; i < n; i++) {
        const size_t j = (size_t)orc_bit_mirror(i, k);
        if (i < j) { uint64_t t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const uint64_t wl = orc_powmod(w, n / len, p);
        for (size_t s = 0; s < n; s += len) {
            uint64_t t = 1;
            for (size_t j = 0; j < len / 2; j++) {
                const uint64_t u = x[s + j], v = mul(x[s + j + len / 2], t, p);
                x[s + j] = add(u, v, p);
                x[s + j + len / 2] = sub(u, v, p);
                t = mul(t, wl, p);
            }
        }
    }
}

/* c = a b over Z/pZ (c: na + nb - 1 words) through transforms of the
 * smallest power-of-two length n >= na + nb - 1; p - 1 must be divisible
 * by n.  Returns 0, or -1 if the scratch cannot be allocated. */
int orc_ntt_polymul(uint64_t p, const uint64_t* a, size_t na, const uint64_t* b, size_t nb, uint64_t* c) {
    if (na == 0 || nb == 0) return 0;
    const size_t nc = na + nb - 1;
    unsigned k = 0;
    while (((size_t)1 << k) < nc) k++;
    const size_t n = (size_t)1 << k;
    uint64_t* x = calloc(n, sizeof(uint64_t));
    uint64_t* y = calloc(n, sizeof(uint64_t));
    if (!x || !y) { free(x); free(y); return -1; }
    for (size_t i = 0; i < na; i++) x[i] = a[i] % p;
    for (size_t i = 0; i < nb; i++) y[i] = b[i] % p;
    const uint64_t w = k ? orc_root_of_unity(p, k) : 1;
    ntt_inplace(x, k, w, p);
    ntt_inplace(y, k, w, p);
    for (size_t i = 0; i < n; i++) x[i] = mul(x[i], y[i], p);
    ntt_inplace(x, k, orc_invmod_prime(w, p), p);
    const uint64_t ninv = orc_invmod_prime(n % p, p);
    for (size_t i = 0; i < nc; i++) c[i] = mul(x[i], ninv, p);
    free(x);
    free(y);
    return 0;
}

/* count products of equal shapes laid out back to back (as
 * orc_polymul_batch), spread over OpenMP threads one product each. */
int orc_ntt_polymul_batch(uint64_t p, const uint64_t* a, size_t na, const uint64_t* b, size_t nb,
                          size_t count, uint64_t* c) {
    if (na == 0 || nb == 0) return 0;
    const size_t nc = na + nb - 1;
    int rc = 0;
    long long t;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : rc)
    for (t = 0; t < (long long)count; t++)
        rc |= orc_ntt_polymul(p, a + (size_t)t * na, na, b + (size_t)t * nb, nb, c + (size_t)t * nc);
    return rc;
}
