// Element-wise modular products with each reduction the paper surveys,
// run on the GPU so that every variant (and the exact products the
// transform kernels use) can be checked word for word.
//
//  Barrett      Function 6 with the Table 3 parameters (alpha, s, t, h) for
//               the bit size m of p against the word size n
//  Shoup        Function 8 (fixed multiplicand y, psi = floor(2^n y / p))
//  Montgomery   Function 13 (with the m = n overflow test of its line 4)
//  FMA          Function 16 over IEEE double (m <= 50, Proposition 13)
//  Mont-fixed   the 32-bit kernels' twiddle product (Remark 8 form)
//  Mont-product the kernels' pointwise product (x y 2^-n rem p)
//  add / sub    the kernels' modular sum and difference (Section 2.1)
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/gbntt.h"
#include "kernels.h"
#include "plan.h"

namespace gbntt {

using u128 = unsigned __int128;

struct BarrettParams {
    unsigned s, t, h;
    uint64_t q;     // floor(2^(s+t) / p)
};

// Table 3: the column is picked by the bit size m of p relative to the word size n.
static BarrettParams barrett_params(uint64_t p, unsigned n) {
    const unsigned r = 64 - __builtin_clzll(p - 1);   // 2^(r-1) < p <= 2^r
    const unsigned m = 64 - __builtin_clzll(p);       // p < 2^m
    BarrettParams b{};
    if (m + 2 <= n) {
        b.s = r >= 2 ? r - 2 : 0;
        b.t = n + 1;
        b.h = 1;
    } else if (m + 1 == n) {
        b.s = r - 1;
        b.t = n;
        b.h = 2;
    } else {
        b.s = r - 1;
        b.t = n;
        b.h = 3;
    }
    b.q = static_cast<uint64_t>((static_cast<u128>(1) << (b.s + b.t)) / p);
    return b;
}

__device__ __forceinline__ uint32_t barrett32(uint64_t a, uint32_t p, BarrettParams B) {
    const uint64_t b = a >> B.s;
    const uint64_t c = (b * B.q) >> B.t;      // b q < alpha 2^t <= 2^64 (Proposition 1)
    uint64_t d = a - c * p;
    for (unsigned i = 0; i < B.h; ++i) d = (d >= p) ? d - p : d;
    return static_cast<uint32_t>(d);
}

__device__ __forceinline__ uint64_t barrett64(u128 a, uint64_t p, BarrettParams B) {
    const u128 b = a >> B.s;
    const u128 c = (b * B.q) >> B.t;          // b q < 2^128 (Proposition 1)
    u128 d = a - c * p;
    for (unsigned i = 0; i < B.h; ++i) d = (d >= p) ? d - p : d;
    return static_cast<uint64_t>(d);
}

// Function 13, n = m = 32: a < 2^32 p; chi p = -1 rem 2^32.
__device__ __forceinline__ uint32_t redc32(uint64_t a, uint32_t p, uint32_t chi) {
    const uint32_t b = static_cast<uint32_t>(a) * chi;
    const uint64_t c = a + static_cast<uint64_t>(b) * p;
    const uint32_t d = static_cast<uint32_t>(c >> 32);
    if (c < a) return d - p;                  // the sum wrapped: true d is d + 2^32
    return (d >= p) ? d - p : d;
}

// Function 13, n = m = 64.
__device__ __forceinline__ uint64_t redc64(u128 a, uint64_t p, uint64_t chi) {
    const uint64_t b = static_cast<uint64_t>(a) * chi;
    const u128 c = a + static_cast<u128>(b) * p;
    const uint64_t d = static_cast<uint64_t>(c >> 64);
    if (c < a) return d - p;
    return (d >= p) ? d - p : d;
}

// Function 16 (any rounding mode; round-to-nearest here): h + l = x y
// exactly, c = floor(h u) is within one of the true quotient, and the two
// final tests bring e into [0, p).
__device__ __forceinline__ uint64_t fma_mulmod(double x, double y, double p, double u) {
    const double hi = x * y;
    const double lo = fma(x, y, -hi);
    const double quo = floor(hi * u);
    double e = fma(-quo, p, hi) + lo;
    e = (e >= p) ? e - p : e;
    e = (e < 0.0) ? e + p : e;
    return static_cast<uint64_t>(e);
}

struct MMArgs {
    uint64_t p;
    unsigned kind;
    unsigned wb;
    BarrettParams bar;
    uint64_t chi;     // -p^-1 rem 2^n
    uint64_t pinv;    // p^-1 rem 2^n
    uint64_t r2;      // 2^(2n) rem p
    double dp, u;     // p and fl(1/p) for Function 16
};

__global__ void k_modmul_vec(MMArgs A, const uint64_t* __restrict__ x, const uint64_t* __restrict__ y,
                             const uint64_t* __restrict__ yc, uint64_t* __restrict__ z, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint64_t xi = x[i], yi = y[i];
        uint64_t r = 0;
        if (A.wb == 4) {
            const uint32_t p = static_cast<uint32_t>(A.p);
            const uint32_t x32 = static_cast<uint32_t>(xi), y32 = static_cast<uint32_t>(yi);
            switch (A.kind) {
                case NTT_MM_BARRETT:
                    r = barrett32(static_cast<uint64_t>(x32) * y32, p, A.bar);
                    break;
                case NTT_MM_SHOUP: {
                    const uint32_t c = __umulhi(x32, static_cast<uint32_t>(yc[i]));
                    uint64_t d = static_cast<uint64_t>(x32) * y32 - static_cast<uint64_t>(c) * p;
                    r = (d >= p) ? d - p : d;
                    break;
                }
                case NTT_MM_MONTGOMERY: {
                    const uint32_t chi = static_cast<uint32_t>(A.chi);
                    const uint32_t r2 = static_cast<uint32_t>(A.r2);
                    const uint32_t xm = redc32(static_cast<uint64_t>(x32) * r2, p, chi);
                    const uint32_t ym = redc32(static_cast<uint64_t>(y32) * r2, p, chi);
                    const uint32_t zm = redc32(static_cast<uint64_t>(xm) * ym, p, chi);
                    r = redc32(zm, p, chi);
                    break;
                }
                case NTT_MM_MONT_FIXED: {
                    const Mont32 ar{p, static_cast<uint32_t>(A.pinv)};
                    const uint32_t wm = static_cast<uint32_t>((static_cast<uint64_t>(y32) << 32) % p);
                    r = ar.mulw(x32, Tw32{wm, static_cast<uint32_t>(yc[i])});
                    break;
                }
                case NTT_MM_MONT_PRODUCT: {
                    const Mont32 ar{p, static_cast<uint32_t>(A.pinv)};
                    r = ar.mulmont(ar.mulmont(x32, y32), static_cast<uint32_t>(A.r2));
                    break;
                }
                case NTT_MM_MONT_FIXED_W: {
                    const Mont32W ar(Mont32{p, static_cast<uint32_t>(A.pinv)});
                    const uint32_t wm = static_cast<uint32_t>((static_cast<uint64_t>(y32) << 32) % p);
                    r = ar.mulw(x32, Tw32{wm, 0u});
                    break;
                }
                case NTT_MM_MONT_PRODUCT_W: {
                    const Mont32W ar(Mont32{p, static_cast<uint32_t>(A.pinv)});
                    r = ar.mulmont(ar.mulmont(x32, y32), static_cast<uint32_t>(A.r2));
                    break;
                }
                case NTT_MM_ADD: {
                    const Mont32 ar{p, static_cast<uint32_t>(A.pinv)};
                    r = ar.add(x32, y32);
                    break;
                }
                case NTT_MM_SUB: {
                    const Mont32 ar{p, static_cast<uint32_t>(A.pinv)};
                    r = ar.sub(x32, y32);
                    break;
                }
                default:
                    r = fma_mulmod(static_cast<double>(xi), static_cast<double>(yi), A.dp, A.u);
            }
        } else {
            const uint64_t p = A.p;
            switch (A.kind) {
                case NTT_MM_BARRETT:
                    r = barrett64(static_cast<u128>(xi) * yi, p, A.bar);
                    break;
                case NTT_MM_SHOUP: {   // the 64-bit kernels' lazy twiddle product, then canon
                    const Shoup64L ar{p, A.pinv};
                    r = ar.canon(ar.mulw(xi, Tw64{yi, yc[i]}));
                    break;
                }
                case NTT_MM_MONTGOMERY: {
                    const uint64_t xm = redc64(static_cast<u128>(xi) * A.r2, p, A.chi);
                    const uint64_t ym = redc64(static_cast<u128>(yi) * A.r2, p, A.chi);
                    const uint64_t zm = redc64(static_cast<u128>(xm) * ym, p, A.chi);
                    r = redc64(zm, p, A.chi);
                    break;
                }
                case NTT_MM_MONT_PRODUCT: {
                    const Shoup64L ar{p, A.pinv};
                    r = ar.mulmont(ar.mulmont(xi, yi), A.r2);
                    break;
                }
                case NTT_MM_ADD: {
                    const Shoup64L ar{p, A.pinv};
                    r = ar.canon(ar.add(xi, yi));
                    break;
                }
                case NTT_MM_SUB: {
                    const Shoup64L ar{p, A.pinv};
                    r = ar.canon(ar.sub(xi, yi));
                    break;
                }
                default:
                    r = fma_mulmod(static_cast<double>(xi), static_cast<double>(yi), A.dp, A.u);
            }
        }
        z[i] = r;
    }
}

// Throughput of one reduction: every thread runs 4 independent chains of
// `iters` dependent modular products on register values (x <- x y rem p),
// so the result measures the variant's arithmetic, not memory.
template <int KIND, int WB>
__global__ void k_modmul_rate(MMArgs A, uint64_t* out, int iters, uint64_t y, uint64_t yc) {
    uint64_t v[4];
    for (int c = 0; c < 4; ++c) v[c] = (threadIdx.x * 7919u + c * 104729u + blockIdx.x) % A.p;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint64_t x = v[c];
            if (WB == 4) {
                const uint32_t p = static_cast<uint32_t>(A.p);
                const uint32_t x32 = static_cast<uint32_t>(x), y32 = static_cast<uint32_t>(y);
                if (KIND == NTT_MM_BARRETT) x = barrett32(static_cast<uint64_t>(x32) * y32, p, A.bar);
                if (KIND == NTT_MM_SHOUP) {
                    const uint32_t q = __umulhi(x32, static_cast<uint32_t>(yc));
                    const uint64_t d = static_cast<uint64_t>(x32) * y32 - static_cast<uint64_t>(q) * p;
                    x = (d >= p) ? d - p : d;
                }
                if (KIND == NTT_MM_MONTGOMERY) {
                    x = redc32(static_cast<uint64_t>(x32) * y32, p, static_cast<uint32_t>(A.chi));
                }
                if (KIND == NTT_MM_MONT_FIXED) {
                    const Mont32 ar{p, static_cast<uint32_t>(A.pinv)};
                    x = ar.mulw(x32, Tw32{y32, static_cast<uint32_t>(yc)});
                }
            } else {
                if (KIND == NTT_MM_BARRETT) x = barrett64(static_cast<u128>(x) * y, A.p, A.bar);
                if (KIND == NTT_MM_SHOUP) x = Shoup64L{A.p, A.pinv}.canon(Shoup64L{A.p, A.pinv}.mulw(x, Tw64{y, yc}));
                if (KIND == NTT_MM_MONTGOMERY) x = redc64(static_cast<u128>(x) * y, A.p, A.chi);
            }
            if (KIND == NTT_MM_FMA)
                x = fma_mulmod(static_cast<double>(x), static_cast<double>(y), A.dp, A.u);
            v[c] = x;
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = v[0] ^ v[1] ^ v[2] ^ v[3];
}

int modmul_rate(uint64_t p, unsigned kind, unsigned word_bytes, int iters, double* per_s) {
    if (kind > NTT_MM_MONT_FIXED || (word_bytes != 4 && word_bytes != 8) || iters <= 0 || !per_s)
        return NTT_ERR_ARG;
    if (p < 3 || !(p & 1) || (word_bytes == 4 && (p >> 32)) || (word_bytes == 8 && (p >> 62)) ||
        (kind == NTT_MM_FMA && (p >> 50)) || (kind == NTT_MM_MONT_FIXED && word_bytes != 4))
        return NTT_ERR_MODULUS;
    MMArgs A{};
    A.p = p;
    A.kind = kind;
    A.wb = word_bytes;
    const unsigned nbits = word_bytes * 8;
    A.bar = barrett_params(p, nbits);
    if (nbits == 32) {
        A.pinv = host::inv_pow2_32(static_cast<uint32_t>(p));
        A.chi = static_cast<uint32_t>(0u - static_cast<uint32_t>(A.pinv));
    } else {
        A.pinv = host::inv_pow2_64(p);
        A.chi = 0 - A.pinv;
    }
    A.dp = static_cast<double>(p);
    A.u = 1.0 / A.dp;
    const uint64_t y = p / 3 + 1;
    uint64_t yc = 0;
    if (kind == NTT_MM_SHOUP) yc = static_cast<uint64_t>((static_cast<u128>(y) << nbits) / p);
    if (kind == NTT_MM_MONT_FIXED) yc = host::tw32_of(y, static_cast<uint32_t>(p), static_cast<uint32_t>(A.pinv)).c;
    uint64_t ymf = y;
    if (kind == NTT_MM_MONT_FIXED) ymf = host::tw32_of(y, static_cast<uint32_t>(p), static_cast<uint32_t>(A.pinv)).w;
    const int blocks = 152 * 8, threads = 256;
    uint64_t* out = nullptr;
    if (cudaMalloc(&out, sizeof(uint64_t) * blocks * threads) != cudaSuccess) return NTT_ERR_OOM;
    auto launch = [&](int it) {
#define GBNTT_RATE(K, W) \
    if (kind == K && word_bytes == W) k_modmul_rate<K, W><<<blocks, threads>>>(A, out, it, ymf, yc);
        GBNTT_RATE(NTT_MM_BARRETT, 4) GBNTT_RATE(NTT_MM_SHOUP, 4) GBNTT_RATE(NTT_MM_MONTGOMERY, 4)
        GBNTT_RATE(NTT_MM_FMA, 4) GBNTT_RATE(NTT_MM_MONT_FIXED, 4) GBNTT_RATE(NTT_MM_BARRETT, 8)
        GBNTT_RATE(NTT_MM_SHOUP, 8) GBNTT_RATE(NTT_MM_MONTGOMERY, 8) GBNTT_RATE(NTT_MM_FMA, 8)
#undef GBNTT_RATE
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch(16);
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    int rc = NTT_OK;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = NTT_ERR_CUDA;
    } else {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *per_s = 4.0 * iters * blocks * threads / (ms * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaGetLastError();
    return rc;
}

int launch_modmul_vec(uint64_t p, unsigned kind, unsigned word_bytes, const uint64_t* x,
                      const uint64_t* y, const uint64_t* yc, uint64_t* z, size_t n, cudaStream_t st) {
    if (kind > NTT_MM_MONT_PRODUCT_W || (word_bytes != 4 && word_bytes != 8)) return NTT_ERR_ARG;
    if ((kind == NTT_MM_MONT_FIXED_W || kind == NTT_MM_MONT_PRODUCT_W) && word_bytes != 4) return NTT_ERR_ARG;
    if (p < 3 || (p & 1) == 0 || (p >> 63)) return NTT_ERR_MODULUS;
    if (word_bytes == 4 && (p >> 32)) return NTT_ERR_MODULUS;
    if (word_bytes == 8 && (p >> 62) && kind != NTT_MM_MONTGOMERY && kind != NTT_MM_BARRETT)
        return NTT_ERR_MODULUS;
    if (kind == NTT_MM_FMA && (p >> 50)) return NTT_ERR_MODULUS;
    if (kind == NTT_MM_MONT_FIXED && word_bytes != 4) return NTT_ERR_ARG;
    if ((kind == NTT_MM_SHOUP || kind == NTT_MM_MONT_FIXED) && !yc && n) return NTT_ERR_ARG;
    if (n && (!x || !y || !z)) return NTT_ERR_ARG;
    MMArgs A{};
    A.p = p;
    A.kind = kind;
    A.wb = word_bytes;
    const unsigned nbits = word_bytes * 8;
    A.bar = barrett_params(p, nbits);
    if (nbits == 32) {
        A.pinv = host::inv_pow2_32(static_cast<uint32_t>(p));
        A.chi = static_cast<uint32_t>(0u - static_cast<uint32_t>(A.pinv));
        A.r2 = static_cast<uint64_t>((static_cast<u128>(1) << 64) % p);
    } else {
        A.pinv = host::inv_pow2_64(p);
        A.chi = 0 - A.pinv;
        const uint64_t r1 = static_cast<uint64_t>((static_cast<u128>(1) << 64) % p);
        A.r2 = host::mul_mod(r1, r1, p);
    }
    A.dp = static_cast<double>(p);
    A.u = 1.0 / A.dp;
    if (n == 0) return NTT_OK;
    long long blocks = (static_cast<long long>(n) + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_modmul_vec<<<static_cast<unsigned>(blocks), 256, 0, st>>>(A, x, y, yc, z, static_cast<long long>(n));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        gbntt_set_error(std::string("k_modmul_vec: ") + cudaGetErrorString(e));
        return NTT_ERR_CUDA;
    }
    return NTT_OK;
}

}  // namespace gbntt
