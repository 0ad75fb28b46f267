// Host planner: moduli, roots of unity and the twiddle tables of a plan.
//
// Section 5.1 precomputes and caches every root of unity and power the
// transform needs; here they are built once per plan on the host, converted
// to the multiplicand form of the word policy (Montgomery form plus Remark 8
// companion for 32-bit words, Function 8's Shoup quotient for 64-bit words)
// and copied to the device in one allocation.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/gbntt.h"
#include "plan.h"

using u128 = unsigned __int128;

namespace gbntt {
namespace host {

uint64_t mul_mod(uint64_t a, uint64_t b, uint64_t p) {
    return static_cast<uint64_t>((static_cast<u128>(a) * b) % p);
}

uint64_t pow_mod(uint64_t a, uint64_t e, uint64_t p) {
    uint64_t acc = 1 % p, base = a % p;
    for (; e; e >>= 1, base = mul_mod(base, base, p))
        if (e & 1) acc = mul_mod(acc, base, p);
    return acc;
}

unsigned two_adic(uint64_t x) { return x ? static_cast<unsigned>(__builtin_ctzll(x)) : 64u; }

// Strong-probable-prime test to one base a (n odd, n > a).
static bool sprp(uint64_t n, uint64_t a) {
    const unsigned s = two_adic(n - 1);
    const uint64_t d = (n - 1) >> s;
    uint64_t x = pow_mod(a, d, n);
    if (x == 1 || x == n - 1) return true;
    for (unsigned i = 1; i < s; ++i) {
        x = mul_mod(x, x, n);
        if (x == n - 1) return true;
        if (x == 1) return false;
    }
    return false;
}

// Deterministic for 64-bit n: the primes up to 37 as bases suffice below 3.3e24.
bool is_prime_u64(uint64_t n) {
    static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t b : bases) {
        if (n % b == 0) return n == b;
    }
    for (uint64_t b : bases)
        if (!sprp(n, b)) return false;
    return true;
}

// Distinct prime divisors of m (m >= 2).
static std::vector<uint64_t> distinct_primes(uint64_t m) {
    std::vector<uint64_t> out;
    const unsigned tz = two_adic(m);
    if (tz) {
        out.push_back(2);
        m >>= tz;
    }
    for (uint64_t q = 3; m > 1; q += 2) {
        if (is_prime_u64(m)) { out.push_back(m); break; }
        if (q > m / q) { out.push_back(m); break; }
        if (m % q == 0) {
            out.push_back(q);
            do m /= q; while (m % q == 0);
        }
    }
    return out;
}

uint64_t least_generator(uint64_t p) {
    if (p == 2) return 1;
    const std::vector<uint64_t> qs = distinct_primes(p - 1);
    for (uint64_t g = 2; g < p; ++g) {
        bool gen = true;
        for (uint64_t q : qs)
            if (pow_mod(g, (p - 1) / q, p) == 1) { gen = false; break; }
        if (gen) return g;
    }
    return 0;
}

// Newton iteration x <- x (2 - p x) doubles the number of correct low bits.
uint32_t inv_pow2_32(uint32_t p) {
    uint32_t x = p;                      // correct to 3 bits for odd p
    for (int i = 0; i < 4; ++i) x *= 2u - p * x;
    return x;
}
uint64_t inv_pow2_64(uint64_t p) {
    uint64_t x = p;
    for (int i = 0; i < 5; ++i) x *= 2u - p * x;
    return x;
}

Tw32 tw32_of(uint64_t value, uint32_t p, uint32_t pinv) {
    const uint32_t w = static_cast<uint32_t>((static_cast<uint64_t>(value % p) << 32) % p);
    return Tw32{w, w * pinv};
}

Tw64 tw64_of(uint64_t value, uint64_t p) {
    const uint64_t v = value % p;
    const uint64_t c = static_cast<uint64_t>((static_cast<u128>(v) << 64) / p);
    return Tw64{v, c};
}

}  // namespace host
}  // namespace gbntt

using namespace gbntt;
using namespace gbntt::host;

static thread_local std::string g_last_error;
void gbntt_set_error(const std::string& msg) { g_last_error = msg; }
extern "C" const char* ntt_last_error(void) { return g_last_error.c_str(); }

static unsigned bit_mirror(uint64_t i, int k) {
    uint64_t r = 0;
    for (int j = 0; j < k; ++j) r = (r << 1) | ((i >> j) & 1);
    return static_cast<unsigned>(r);
}

extern "C" int ntt_find_prime(unsigned bits, unsigned min_l, unsigned index, uint64_t* p_out) {
    if (!p_out || bits < 3 || bits > 63 || min_l + 1 >= bits) {
        gbntt_set_error("ntt_find_prime: need 3 <= bits <= 63 and min_l < bits - 1");
        return NTT_ERR_ARG;
    }
    const uint64_t step = 1ull << min_l;
    const uint64_t lo = 1ull << (bits - 1);
    unsigned seen = 0;
    for (uint64_t k = lo / step + 1;; ++k) {
        const u128 cand = static_cast<u128>(k) * step + 1;
        if (cand >> bits) break;
        if (is_prime_u64(static_cast<uint64_t>(cand))) {
            if (seen == index) {
                *p_out = static_cast<uint64_t>(cand);
                return NTT_OK;
            }
            ++seen;
        }
    }
    gbntt_set_error("ntt_find_prime: window exhausted");
    return NTT_ERR_SIZE;
}

static int check_modulus(uint64_t p, unsigned log2n) {
    if (p < 3 || (p & 1) == 0 || (p >> 62) != 0) {
        gbntt_set_error("modulus must be odd, >= 3 and < 2^62");
        return NTT_ERR_MODULUS;
    }
    if (!is_prime_u64(p)) {
        gbntt_set_error("modulus is not prime");
        return NTT_ERR_NOT_PRIME;
    }
    if (two_adic(p - 1) < 4) {
        gbntt_set_error("16 must divide p - 1");
        return NTT_ERR_MODULUS;
    }
    if (log2n > two_adic(p - 1)) {
        gbntt_set_error("2^log2n does not divide p - 1");
        return NTT_ERR_NO_ROOT;
    }
    return NTT_OK;
}

extern "C" int ntt_root_of_unity(uint64_t p, unsigned log2n, uint64_t* g_out, uint64_t* omega_out) {
    if (!g_out || !omega_out) return NTT_ERR_ARG;
    if (p < 3 || (p & 1) == 0) return NTT_ERR_MODULUS;
    if (!is_prime_u64(p)) return NTT_ERR_NOT_PRIME;
    if (log2n > two_adic(p - 1)) return NTT_ERR_NO_ROOT;
    const uint64_t g = least_generator(p);
    *g_out = g;
    *omega_out = pow_mod(g, (p - 1) >> log2n, p);
    return NTT_OK;
}

extern "C" int ntt_fixed_companion(uint64_t p, unsigned kind, unsigned word_bytes,
                                   const uint64_t* h_y, uint64_t* h_out, size_t n) {
    if ((!h_y || !h_out) && n) return NTT_ERR_ARG;
    if (word_bytes != 4 && word_bytes != 8) return NTT_ERR_ARG;
    if (p < 3 || (p & 1) == 0 || (word_bytes == 4 && (p >> 32))) return NTT_ERR_MODULUS;
    if (kind == NTT_MM_SHOUP) {
        const int bits = 8 * static_cast<int>(word_bytes);
        for (size_t i = 0; i < n; ++i) {
            const uint64_t y = h_y[i] % p;
            h_out[i] = static_cast<uint64_t>((static_cast<u128>(y) << bits) / p);
        }
        return NTT_OK;
    }
    if (kind == NTT_MM_MONT_FIXED) {
        if (word_bytes != 4) return NTT_ERR_ARG;
        const uint32_t pinv = inv_pow2_32(static_cast<uint32_t>(p));
        for (size_t i = 0; i < n; ++i) h_out[i] = tw32_of(h_y[i], static_cast<uint32_t>(p), pinv).c;
        return NTT_OK;
    }
    return NTT_ERR_ARG;
}

// ---------------------------------------------------------------- tables

namespace {

// Host image of the device table block; offsets are in table entries.
template <class TwT>
struct TableBuilder {
    std::vector<TwT> data;
    size_t add(size_t n) {
        // keep every sub-table 256-byte aligned
        const size_t align = 256 / sizeof(TwT);
        size_t off = (data.size() + align - 1) / align * align;
        data.resize(off + n);
        return off;
    }
};

template <class Conv>
void fill_line_table(std::vector<uint64_t>& vals, uint64_t p, uint64_t wM, int logM, bool fwd) {
    (void)fwd;
    const size_t M = size_t(1) << logM;
    vals.assign(M, 1);
    for (size_t j1 = 0; j1 < M / 16; ++j1) {
        const uint64_t base = pow_mod(wM, j1, p);
        for (int t = 0; t < 16; ++t) vals[j1 * 16 + t] = pow_mod(base, bit_mirror(t, 4), p);
    }
}

// vals[r*L1 + c] = w^(c [r]_l2), rows r < 2^l2, columns c < 2^l1.
void fill_outer_table(std::vector<uint64_t>& vals, uint64_t p, uint64_t w, int l2, int l1) {
    const size_t L2 = size_t(1) << l2, L1 = size_t(1) << l1;
    vals.resize(L2 * L1);
    for (size_t r = 0; r < L2; ++r) {
        const uint64_t base = pow_mod(w, bit_mirror(r, l2), p);
        uint64_t acc = 1;
        for (size_t c = 0; c < L1; ++c) {
            vals[r * L1 + c] = acc;
            acc = mul_mod(acc, base, p);
        }
    }
}

}  // namespace

template <class TwT, class Conv>
static void build_tables(ntt_plan* P, TableBuilder<TwT>& tb, Conv conv,
                         size_t (&line_off)[2][kMaxLineLog + 1], size_t (&tile_off)[2][17],
                         size_t (&glob_off)[3], size_t (&plain_off)[2], size_t (&linet_off)[2],
                         size_t (&l64x8_off)[2], uint64_t pm_factor) {
    const uint64_t p = P->p;
    const uint64_t g = P->g;
    auto root = [&](int logm, bool fwd) {
        uint64_t w = pow_mod(g, (p - 1) >> logm, p);
        return fwd ? w : pow_mod(w, p - 2, p);
    };
    std::vector<uint64_t> vals;
    for (int d = 0; d < 2; ++d) {
        const bool fwd = (d == 0);
        for (int lm = 0; lm <= kMaxLineLog; ++lm) line_off[d][lm] = SIZE_MAX;
        for (int lt = 0; lt <= 16; ++lt) tile_off[d][lt] = SIZE_MAX;
        plain_off[d] = SIZE_MAX;
        linet_off[d] = SIZE_MAX;
        l64x8_off[d] = SIZE_MAX;
        // 64-point sub-transforms split 8 x 8: [j1*8 + t] = w_64^(j1 [t]_3)
        if (P->v2 >= 6) {
            const uint64_t w64 = root(6, fwd);
            const size_t off = tb.add(64);
            for (int j1 = 0; j1 < 8; ++j1)
                for (int t = 0; t < 8; ++t)
                    tb.data[off + j1 * 8 + t] = conv(pow_mod(w64, uint64_t(j1) * bit_mirror(t, 3), p));
            l64x8_off[d] = off;
        }
        if (fwd) glob_off[0] = glob_off[1] = glob_off[2] = SIZE_MAX;
        // radix-16 pass tables for sub-transform sizes 2^5 .. 2^8
        for (int lm = 5; lm <= kMaxLineLog && lm <= static_cast<int>(P->v2); ++lm) {
            fill_line_table<Conv>(vals, p, root(lm, fwd), lm, fwd);
            const size_t off = tb.add(vals.size());
            for (size_t i = 0; i < vals.size(); ++i) tb.data[off + i] = conv(vals[i]);
            line_off[d][lm] = off;
            if (lm == kMaxLineLog) {           // transposed copy: [t*16 + j1] = vals[j1*16 + t]
                const size_t offt = tb.add(vals.size());
                for (size_t j1 = 0; j1 < 16; ++j1)
                    for (size_t t = 0; t < 16; ++t) tb.data[offt + t * 16 + j1] = conv(vals[j1 * 16 + t]);
                linet_off[d] = offt;
            }
        }
        // tile twiddles for every vector length above one line that the plan's kernels use
        std::vector<int> tiles;
        const int k = static_cast<int>(P->log2n);
        if (k <= P->tile_max_log) {
            // every tile size up to n, so one plan serves every shorter
            // one-block product with this modulus (uneven batches)
            for (int lt = kMaxLineLog + 1; lt <= k; ++lt) tiles.push_back(lt);
        } else {
            if (P->k2 > kMaxLineLog) tiles.push_back(P->k2);
            if (P->k1 > kMaxLineLog && P->k1 != P->k2) tiles.push_back(P->k1);
        }
        for (int lt : tiles) {
            fill_outer_table(vals, p, root(lt, fwd), tile_l2(lt), tile_l1(lt));
            const size_t off = tb.add(vals.size());
            for (size_t i = 0; i < vals.size(); ++i) tb.data[off + i] = conv(vals[i]);
            tile_off[d][lt] = off;
        }
        // the twiddle between the two global passes (Algorithm 1, step 2);
        // the inverse tables carry the final scaling: n^-1 for the inverse
        // transform, n^-1 R for a product whose pointwise step divided by R
        if (k > P->tile_max_log) {
            fill_outer_table(vals, p, root(k, fwd), P->k2, P->k1);
            if (fwd) {
                const size_t off = tb.add(vals.size());
                for (size_t i = 0; i < vals.size(); ++i) tb.data[off + i] = conv(vals[i]);
                glob_off[0] = off;
            } else {
                const uint64_t factors[2] = {P->n_inv, mul_mod(P->n_inv, pm_factor, p)};
                for (int f = 0; f < 2; ++f) {
                    const size_t off = tb.add(vals.size());
                    for (size_t i = 0; i < vals.size(); ++i)
                        tb.data[off + i] = conv(mul_mod(vals[i], factors[f], p));
                    glob_off[1 + f] = off;
                }
            }
        }
        // w_N^e, e < N/2, for the per-stage schedule
        if (P->flags & NTT_FLAG_PLAIN) {
            const size_t half = size_t(1) << (k - 1);
            const uint64_t w = root(k, fwd);
            const size_t off = tb.add(half);
            uint64_t acc = 1;
            for (size_t e = 0; e < half; ++e) {
                tb.data[off + e] = conv(acc);
                acc = mul_mod(acc, w, p);
            }
            plain_off[d] = off;
        }
    }
}

// Constants of the 16-point inverse TFT (w = w_16 of the transform tables).
template <class Ar, class Conv>
static void build_tft(const ntt_plan* P, TftConsts<Ar>& K, Conv conv) {
    const uint64_t p = P->p;
    const uint64_t w16 = pow_mod(P->g, (p - 1) >> 4, p);
    const uint64_t w16i = pow_mod(w16, p - 2, p);
    const uint64_t inv2 = (p + 1) / 2;
    const uint64_t inv8 = mul_mod(inv2, mul_mod(inv2, inv2, p), p);
    uint64_t a = 1, b = 1;
    for (int k = 0; k <= 4; ++k) {
        K.inv2k[k] = conv(a);
        K.pow2k[k] = conv(b);
        a = mul_mod(a, inv2, p);
        b = mul_mod(b, 2, p);
    }
    for (int e = 0; e < 8; ++e) {
        const uint64_t we = pow_mod(w16, e, p), wie = pow_mod(w16i, e, p);
        K.rci_half[e] = conv(mul_mod(wie, inv2, p));
        K.rc_div8[e] = conv(mul_mod(we, inv8, p));
        K.rci_mul8[e] = conv(mul_mod(wie, 8 % p, p));
    }
}

template <class Ar, class TwT, class Conv>
static int finish_plan(ntt_plan* P, DevPlan<Ar>& dp, Conv conv, uint64_t pm_factor) {
    TableBuilder<TwT> tb;
    size_t line_off[2][kMaxLineLog + 1], tile_off[2][17], glob_off[3], plain_off[2], linet_off[2], l64x8_off[2];
    build_tables<TwT>(P, tb, conv, line_off, tile_off, glob_off, plain_off, linet_off, l64x8_off, pm_factor);
    const uint64_t w16 = pow_mod(P->g, (P->p - 1) >> 4, P->p);
    const uint64_t w16i = pow_mod(w16, P->p - 2, P->p);
    for (int e = 0; e < 8; ++e) {
        dp.rc[e] = conv(pow_mod(w16, e, P->p));
        dp.rci[e] = conv(pow_mod(w16i, e, P->p));
    }
    P->table_bytes = tb.data.size() * sizeof(TwT);
    if (cudaMalloc(&P->d_tables, P->table_bytes ? P->table_bytes : 256) != cudaSuccess) {
        cudaGetLastError();
        gbntt_set_error("cudaMalloc of plan tables failed");
        return NTT_ERR_OOM;
    }
    if (P->table_bytes &&
        cudaMemcpy(P->d_tables, tb.data.data(), P->table_bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        gbntt_set_error(std::string("table upload: ") + cudaGetErrorString(cudaGetLastError()));
        return NTT_ERR_CUDA;
    }
    const TwT* base = static_cast<const TwT*>(P->d_tables);
    auto at = [&](size_t off) -> const TwT* { return off == SIZE_MAX ? nullptr : base + off; };
    for (int lm = 0; lm <= kMaxLineLog; ++lm) {
        dp.line_fwd[lm] = at(line_off[0][lm]);
        dp.line_inv[lm] = at(line_off[1][lm]);
    }
    for (int lt = 0; lt <= 16; ++lt) {
        dp.tile_fwd[lt] = at(tile_off[0][lt]);
        dp.tile_inv[lt] = at(tile_off[1][lt]);
    }
    dp.line256_t[0] = at(linet_off[0]);
    dp.line256_t[1] = at(linet_off[1]);
    dp.glob_fwd = at(glob_off[0]);
    dp.glob_inv = at(glob_off[1]);
    P->glob_inv_pm = at(glob_off[2]);
    dp.plain_fwd = at(plain_off[0]);
    dp.plain_inv = at(plain_off[1]);
    dp.line64x8[0] = at(l64x8_off[0]);
    dp.line64x8[1] = at(l64x8_off[1]);
    if constexpr (std::is_same<TwT, Tw32>::value) {
        // multiplicand-only copies of the direct kernels' tables
        // (the step-2 tables only at n = 2^16: larger sizes run the direct
        // kernels of their 2^16-point child plan)
        const bool g16 = P->log2n == 16;
        const size_t srcs[7] = {line_off[0][kMaxLineLog], line_off[1][kMaxLineLog], linet_off[0], linet_off[1],
                                g16 ? glob_off[0] : SIZE_MAX, g16 ? glob_off[1] : SIZE_MAX,
                                g16 ? glob_off[2] : SIZE_MAX};
        const size_t lens[7] = {256, 256, 256, 256, size_t(1) << P->log2n, size_t(1) << P->log2n,
                                size_t(1) << P->log2n};
        std::vector<uint32_t> w;
        size_t woff[7];
        for (int i = 0; i < 7; ++i) {
            woff[i] = SIZE_MAX;
            if (srcs[i] == SIZE_MAX) continue;
            woff[i] = w.size();
            for (size_t e = 0; e < lens[i]; ++e) w.push_back(tb.data[srcs[i] + e].w);
            while (w.size() % 64) w.push_back(0);    // 256-byte aligned pieces
        }
        if (!w.empty()) {
            if (cudaMalloc(&P->d_wtables, w.size() * 4) != cudaSuccess) {
                cudaGetLastError();
                gbntt_set_error("cudaMalloc of plan tables failed");
                return NTT_ERR_OOM;
            }
            if (cudaMemcpy(P->d_wtables, w.data(), w.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
                gbntt_set_error(std::string("table upload: ") + cudaGetErrorString(cudaGetLastError()));
                return NTT_ERR_CUDA;
            }
            const uint32_t* wb = static_cast<const uint32_t*>(P->d_wtables);
            auto wat = [&](int i) -> const uint32_t* { return woff[i] == SIZE_MAX ? nullptr : wb + woff[i]; };
            dp.wline[0] = wat(0);
            dp.wline[1] = wat(1);
            dp.wline_t[0] = wat(2);
            dp.wline_t[1] = wat(3);
            dp.wglob[0] = wat(4);
            dp.wglob[1] = wat(5);
            P->glob_inv_pm_w = wat(6);
        }
    }
    return NTT_OK;
}

// Tables of the pass across the n2 = n / 2^16 sub-vectors (n = 2^17 .. 2^24).
template <class TwT, class Conv>
static int build_pre_tables(ntt_plan* P, Conv conv) {
    const uint64_t p = P->p;
    const int m = static_cast<int>(P->log2n) - 16;
    const uint64_t w = pow_mod(P->g, (p - 1) >> P->log2n, p);
    const uint64_t wi = pow_mod(w, p - 2, p);
    const uint64_t n2_inv = pow_mod((uint64_t(1) << m) % p, p - 2, p);
    std::vector<uint64_t> vals;
    std::vector<TwT> host(size_t(2) << P->log2n);
    const size_t n = size_t(1) << P->log2n;
    fill_outer_table(vals, p, w, m, 16);
    for (size_t i = 0; i < n; ++i) host[i] = conv(vals[i]);
    fill_outer_table(vals, p, wi, m, 16);
    for (size_t i = 0; i < n; ++i) host[n + i] = conv(mul_mod(vals[i], n2_inv, p));
    if (cudaMalloc(&P->d_pre, host.size() * sizeof(TwT)) != cudaSuccess) {
        cudaGetLastError();
        gbntt_set_error("cudaMalloc of the sub-vector tables failed");
        return NTT_ERR_OOM;
    }
    if (cudaMemcpy(P->d_pre, host.data(), host.size() * sizeof(TwT), cudaMemcpyHostToDevice) != cudaSuccess) {
        gbntt_set_error(std::string("table upload: ") + cudaGetErrorString(cudaGetLastError()));
        return NTT_ERR_CUDA;
    }
    P->pre_fwd = P->d_pre;
    P->pre_inv = static_cast<const TwT*>(P->d_pre) + n;
    return NTT_OK;
}

extern "C" int ntt_plan_create(uint64_t p, unsigned log2n, unsigned flags, ntt_plan** out) {
    if (!out) return NTT_ERR_ARG;
    *out = nullptr;
    if (log2n < 1 || log2n > 24 || (flags & ~(NTT_FLAG_PLAIN | NTT_FLAG_CHECK | NTT_FLAG_FP64))) {
        gbntt_set_error("need 1 <= log2n <= 24 and known flags");
        return log2n > 24 ? NTT_ERR_SIZE : NTT_ERR_ARG;
    }
    int rc = check_modulus(p, log2n);
    if (rc != NTT_OK) return rc;
    if ((flags & NTT_FLAG_FP64) && (p >> 50)) {
        gbntt_set_error("NTT_FLAG_FP64 needs p < 2^50 (Function 16, m <= 50)");
        return NTT_ERR_MODULUS;
    }
    if ((flags & NTT_FLAG_FP64) && (flags & NTT_FLAG_PLAIN)) {
        gbntt_set_error("the one-launch-per-stage schedule has no FP64 form");
        return NTT_ERR_UNSUPPORTED;
    }
    ntt_plan* P = new (std::nothrow) ntt_plan();
    if (!P) return NTT_ERR_OOM;
    P->p = p;
    P->log2n = log2n;
    P->flags = flags;
    P->word_bytes = ((p >> 32) || (flags & NTT_FLAG_FP64)) ? 8 : 4;
    P->v2 = two_adic(p - 1);
    P->g = least_generator(p);
    P->omega = pow_mod(P->g, (p - 1) >> log2n, p);
    P->omega_inv = pow_mod(P->omega, p - 2, p);
    P->n_inv = pow_mod((1ull << log2n) % p, p - 2, p);
    P->tile_max_log = (P->word_bytes == 4) ? kTileMaxLog32 : kTileMaxLog64;
    P->k2 = static_cast<int>(log2n) / 2;
    P->k1 = static_cast<int>(log2n) - P->k2;
    if (cudaGetDevice(&P->device) != cudaSuccess) {
        cudaGetLastError();
        gbntt_set_error("no CUDA device");
        delete P;
        return NTT_ERR_CUDA;
    }
    if (flags & NTT_FLAG_FP64) {
        P->dpf.ar = Fma50{static_cast<double>(p), 1.0 / static_cast<double>(p)};
        auto conv = [](uint64_t v) { return TwF{static_cast<double>(v)}; };
        rc = finish_plan<Fma50, TwF>(P, P->dpf, conv, 1);
        P->inv_scalef = conv(P->n_inv);
        build_tft(P, P->tftf, conv);
    } else if (P->word_bytes == 4) {
        const uint32_t p32 = static_cast<uint32_t>(p);
        const uint32_t pinv = inv_pow2_32(p32);
        P->dp32.ar = Mont32{p32, pinv};
        auto conv = [p32, pinv](uint64_t v) { return tw32_of(v, p32, pinv); };
        rc = finish_plan<Mont32, Tw32>(P, P->dp32, conv, (1ull << 32) % p);
        P->inv_scale32 = conv(P->n_inv);
        P->pm_scale32 = conv(mul_mod(P->n_inv, (1ull << 32) % p, p));
        P->r32 = conv((1ull << 32) % p);
        build_tft(P, P->tft32, conv);
    } else {
        const uint64_t pinv = inv_pow2_64(p);
        P->dp64.ar = Shoup64L{p, pinv};
        auto conv = [p](uint64_t v) { return tw64_of(v, p); };
        const uint64_t r64 = static_cast<uint64_t>((static_cast<u128>(1) << 64) % p);
        rc = finish_plan<Shoup64L, Tw64>(P, P->dp64, conv, r64);
        P->inv_scale64 = conv(P->n_inv);
        P->pm_scale64 = conv(mul_mod(P->n_inv, r64, p));
        P->r64 = conv(r64);
        build_tft(P, P->tft64, conv);
    }
    if (rc == NTT_OK && log2n >= 17 && log2n <= 24) {
        rc = ntt_plan_create(p, 16, flags & ~NTT_FLAG_PLAIN, &P->core);
        if (rc == NTT_OK) {
            if (flags & NTT_FLAG_FP64)
                rc = build_pre_tables<TwF>(P, [](uint64_t v) { return TwF{static_cast<double>(v)}; });
            else if (P->word_bytes == 4)
                rc = build_pre_tables<Tw32>(P, [&](uint64_t v) { return tw32_of(v, static_cast<uint32_t>(p), P->dp32.ar.pinv); });
            else
                rc = build_pre_tables<Tw64>(P, [&](uint64_t v) { return tw64_of(v, p); });
        }
    }
    if (rc != NTT_OK) {
        if (P->core) ntt_plan_destroy(P->core);
        if (P->d_pre) cudaFree(P->d_pre);
        if (P->d_tables) cudaFree(P->d_tables);
        if (P->d_wtables) cudaFree(P->d_wtables);
        delete P;
        return rc;
    }
    *out = P;
    return NTT_OK;
}

extern "C" int ntt_plan_destroy(ntt_plan* plan) {
    if (!plan) return NTT_ERR_ARG;
    if (plan->core) ntt_plan_destroy(plan->core);
    if (plan->d_pre) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(plan->device);
        cudaDeviceSynchronize();
        cudaFree(plan->d_pre);
        cudaSetDevice(cur);
    }
    if (plan->d_tables || plan->d_wtables) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(plan->device);
        cudaDeviceSynchronize();
        if (plan->d_tables) cudaFree(plan->d_tables);
        if (plan->d_wtables) cudaFree(plan->d_wtables);
        cudaSetDevice(cur);
    }
    delete plan;
    return NTT_OK;
}

extern "C" int ntt_plan_get_info(const ntt_plan* plan, ntt_plan_info* out) {
    if (!plan || !out) return NTT_ERR_ARG;
    out->p = plan->p;
    out->g = plan->g;
    out->omega = plan->omega;
    out->omega_inv = plan->omega_inv;
    out->n_inv = plan->n_inv;
    out->log2n = plan->log2n;
    out->word_bytes = plan->word_bytes;
    out->v2 = plan->v2;
    out->tile_max_log = static_cast<uint32_t>(plan->tile_max_log);
    return NTT_OK;
}

extern "C" const char* ntt_status_str(int status) {
    switch (status) {
        case NTT_OK: return "NTT_OK";
        case NTT_ERR_ARG: return "NTT_ERR_ARG";
        case NTT_ERR_MODULUS: return "NTT_ERR_MODULUS";
        case NTT_ERR_NOT_PRIME: return "NTT_ERR_NOT_PRIME";
        case NTT_ERR_NO_ROOT: return "NTT_ERR_NO_ROOT";
        case NTT_ERR_SIZE: return "NTT_ERR_SIZE";
        case NTT_ERR_RANGE: return "NTT_ERR_RANGE";
        case NTT_ERR_OOM: return "NTT_ERR_OOM";
        case NTT_ERR_TIMEOUT: return "NTT_ERR_TIMEOUT";
        case NTT_ERR_CUDA: return "NTT_ERR_CUDA";
        case NTT_ERR_WORKSPACE: return "NTT_ERR_WORKSPACE";
        case NTT_ERR_UNSUPPORTED: return "NTT_ERR_UNSUPPORTED";
        default: return "NTT_ERR_UNKNOWN";
    }
}

extern "C" const char* ntt_version(void) { return "gbntt 0.1 (sm_103a)"; }
