/* splitmix64 draws for the seeded input generators (workloads.py), in C for
 * speed.  The stream is the one workloads.SplitMix64 draws with numpy: the
 * k-th draw after state s is mix(s + k * gamma), k = 1, 2, ..., and the
 * state advances by gamma per draw (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).  This file holds input
 * generation only: random words, and uniform residues by rejection of the
 * top partial block of 2^64, in the same blocks as the numpy version so that
 * both consume the stream identically. */
#include <stddef.h>
#include <stdint.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* n successive draws into out; *state advances by n * gamma. */
void wl_u64(uint64_t* state, uint64_t* out, size_t n) {
    uint64_t s = *state;
    for (size_t k = 0; k < n; ++k) out[k] = mix(s + (uint64_t)(k + 1) * GAMMA);
    *state = s + (uint64_t)n * GAMMA;
}

/* n residues uniform in [0, p): blocks of want + want/16 + 16 draws (want =
 * residues still missing), accepting draws <= floor(2^64 / p) p - 1 in
 * order; every draw of a block is consumed, accepted or not. */
void wl_uniform_mod(uint64_t* state, uint64_t p, uint64_t* out, size_t n) {
    const uint64_t q = UINT64_MAX / p;   /* floor(2^64 / p) for odd p > 1 */
    const uint64_t limit = q * p - 1;
    uint64_t s = *state;
    size_t filled = 0;
    while (filled < n) {
        const size_t want = n - filled;
        const size_t block = want + want / 16 + 16;
        for (size_t k = 0; k < block; ++k) {
            const uint64_t d = mix(s + (uint64_t)(k + 1) * GAMMA);
            if (d <= limit && filled < n) out[filled++] = d % p;
        }
        s += (uint64_t)block * GAMMA;
    }
    *state = s;
}
