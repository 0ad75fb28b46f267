// Internal plan object behind the opaque `ntt_plan` handle.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>

#include "engine.cuh"
#include "tft.cuh"

struct ntt_plan {
    uint64_t p = 0;
    unsigned log2n = 0;
    unsigned flags = 0;
    unsigned word_bytes = 0;    // 4 (p < 2^32) or 8 (p < 2^62, or doubles with NTT_FLAG_FP64)
    unsigned v2 = 0;            // 2-adic valuation of p - 1
    uint64_t g = 0;             // least generator of F_p^*
    uint64_t omega = 0;         // g^((p-1)/n)
    uint64_t omega_inv = 0;
    uint64_t n_inv = 0;
    int device = 0;
    int tile_max_log = 0;       // largest n done by one CTA (both operands resident)
    int k2 = 0, k1 = 0;         // n = 2^k2 rows x 2^k1 columns when log2n > tile_max_log
    void* d_tables = nullptr;   // one device allocation holding every table
    // inverse step-2 twiddles times n^-1 R (products after Montgomery
    // pointwise steps); passed to the kernels as an argument of its own
    const void* glob_inv_pm = nullptr;
    const uint32_t* glob_inv_pm_w = nullptr;   // its multiplicands alone (32-bit plans)
    size_t table_bytes = 0;
    void* d_wtables = nullptr;  // 32-bit plans: the multiplicand-only tables (DevPlan::wline ...)
    gbntt::DevPlan<gbntt::Mont32> dp32{};
    gbntt::DevPlan<gbntt::Shoup64L> dp64{};
    gbntt::DevPlan<gbntt::Fma50> dpf{};         // NTT_FLAG_FP64 plans
    // scaling constants, already in the policy's multiplicand form
    gbntt::Tw32 inv_scale32{}, pm_scale32{};   // n^-1 ; n^-1 * 2^32 (after Montgomery products)
    gbntt::Tw64 inv_scale64{}, pm_scale64{};   // n^-1 ; n^-1 * 2^64
    gbntt::Tw32 r32{};                          // 2^32 rem p (undoes a Montgomery product)
    gbntt::Tw64 r64{};                          // 2^64 rem p
    gbntt::TwF inv_scalef{};                    // n^-1 (FP64 plans; no Montgomery factor)
    // n = 2^17 .. 2^24: Algorithm 1 with n1 = 2^16 and n2 = n / 2^16 -- a
    // pass across the n2 sub-vectors (in registers for n2 <= 16, a column
    // kernel above), then 2^16-point transforms by the child plan `core`
    // (same modulus); pre_fwd[j2 2^16 + j1] = w_n^(j1 [j2]), pre_inv the
    // inverse twiddles times n2^-1
    ntt_plan* core = nullptr;
    const void* pre_fwd = nullptr;
    const void* pre_inv = nullptr;
    void* d_pre = nullptr;
    // constants of the 16-point inverse TFT, per word policy
    gbntt::TftConsts<gbntt::Mont32> tft32{};
    gbntt::TftConsts<gbntt::Shoup64L> tft64{};
    gbntt::TftConsts<gbntt::Fma50> tftf{};
};

// Three-prime integer product plan (intmul.cu): the primes, a transform plan
// per prime and length, and the Garner constants.
struct intmul_plan {
    int device = 0;
    unsigned max_log2n = 0;
    uint64_t P[3] = {0, 0, 0};
    ntt_plan* plans[3][25] = {};
    gbntt::Tw64 inv12{}, inv13{}, inv23{};   // P1^-1 mod P2, P1^-1 mod P3, P2^-1 mod P3
    gbntt::Tw64 r64[3]{};                    // 2^64 mod P_i
    void* helpers = nullptr;                 // per caller stream: two streams for primes 2 and 3
};

namespace gbntt {
namespace host {

uint64_t mul_mod(uint64_t a, uint64_t b, uint64_t p);
uint64_t pow_mod(uint64_t a, uint64_t e, uint64_t p);
bool is_prime_u64(uint64_t n);
uint64_t least_generator(uint64_t p);
unsigned two_adic(uint64_t x);
uint32_t inv_pow2_32(uint32_t p);   // p^-1 rem 2^32 (p odd)
uint64_t inv_pow2_64(uint64_t p);   // p^-1 rem 2^64 (p odd)
Tw32 tw32_of(uint64_t value, uint32_t p, uint32_t pinv);
Tw64 tw64_of(uint64_t value, uint64_t p);

}  // namespace host
}  // namespace gbntt

// Thread-local last error message for ntt_last_error().
void gbntt_set_error(const std::string& msg);
