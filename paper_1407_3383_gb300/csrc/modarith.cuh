// Device modular arithmetic for the NTT kernels (sm_103a).
//
// Residues live in {0, ..., p-1} at every kernel boundary (Section 2: modular
// integers are stored as their representative in that range).  Two word
// policies drive every transform kernel:
//
//  * Mont32 -- odd p < 2^32 in 32-bit words, including the full-word case
//    m = n = 32 (p = 3*2^30+1).  Products by a fixed multiplicand (the
//    twiddles) use Montgomery's reduction with the precomputed multiplicand
//    of Remark 8 (Section 2.3.1): with w~ = w 2^32 rem p and
//    phi = w~ p^-1 rem 2^32, the product x w rem p is
//    hi(x w~) - hi((x phi rem 2^32) p), corrected once by +p.  The low halves
//    of x w~ and of the quotient times p agree by construction, so this is
//    the exact (x w~ - q p) / 2^32 of Function 13 written with the
//    subtracted quotient instead of the added one; it needs no overflow test
//    even when m = n and accepts any 32-bit x.  The general product (the
//    pointwise step) is Function 13 on the full product x y, giving
//    x y 2^-32 rem p; the 2^32 is folded into the final scaling.
//    Every correction is one subtraction with borrow: x - y rem p is
//    d = x - y (mod 2^32) plus p when x < y.  Addition takes x + y - p as a
//    64-bit value instead of Function 4's x - (p - y) (valid for m = n); the
//    Montgomery tails hi(x w~) - hi(q p) are the same subtraction.  Sums and differences get
//    the borrow as the high word of a 64-bit difference and add p with one
//    multiply-add (FMA pipe); the tails use a compare and a select, the form
//    that stays exact when both high products are equal.
//
//  * Shoup64 -- p < 2^62 in 64-bit words.  Fixed-multiplicand products use
//    Function 8 with n = 64 and psi = floor(2^64 w / p) (Proposition 4: the
//    quotient estimate is at most one short, so one conditional subtraction
//    finishes); since m <= n - 1 the difference fits in one word (the remark
//    after Proposition 4).  General products use Montgomery's reduction with
//    m = n = 64 as in the 32-bit case.  Additions use Function 1's
//    compare-and-subtract (no overflow since m <= n - 1).
#pragma once
#include <cstdint>

namespace gbntt {

struct Tw32 { uint32_t w, c; };   // twiddle in Montgomery form + companion
struct Tw64 { uint64_t w, c; };   // twiddle + Shoup quotient

struct Mont32 {
    using word = uint32_t;
    using tw = Tw32;
    static constexpr int kBits = 32;
    static constexpr bool kWide = false;   // the twiddle product reads the companion
    uint32_t p;      // odd modulus < 2^32
    uint32_t pinv;   // p^-1 rem 2^32

    // x - y rem p for x < p, y <= p: the high word of the 64-bit difference
    // is the borrow mask m, and d + p = m (2^32 - p) + d is one multiply-add.
    __device__ __forceinline__ uint32_t sub(uint32_t x, uint32_t y) const {
        const uint64_t d = static_cast<uint64_t>(x) - y;
        const uint32_t m = static_cast<uint32_t>(d >> 32);
        return m * (0u - p) + static_cast<uint32_t>(d);
    }
    // x + y rem p for x, y < p: z = x + y - p taken as a 64-bit two's
    // complement value (x + y < 2^33) is negative exactly when x + y < p, so
    // its high word is the mask and the correction is the same multiply-add.
    // Two integer additions instead of the three of Function 4's x - (p - y).
    __device__ __forceinline__ uint32_t add(uint32_t x, uint32_t y) const {
        const uint64_t z = static_cast<uint64_t>(x) + y - p;
        const uint32_t m = static_cast<uint32_t>(z >> 32);
        return m * (0u - p) + static_cast<uint32_t>(z);
    }
    // a difference that only feeds a twiddle product (any 32-bit input)
    __device__ __forceinline__ uint32_t sub_lazy(uint32_t x, uint32_t y) const { return sub(x, y); }
    // values are always fully reduced with this policy
    __device__ __forceinline__ uint32_t canon(uint32_t x) const { return x; }
    // The same difference written with a compare and a select; used for the
    // Montgomery tails, whose operands come straight from high products.
    __device__ __forceinline__ uint32_t sub_sel(uint32_t x, uint32_t y) const {
        const uint32_t d = x - y;
        return d + ((x < y) ? p : 0u);
    }
    // x * w rem p for any 32-bit x; t = (w 2^32 rem p, (w 2^32 rem p) p^-1 rem 2^32).
    __device__ __forceinline__ uint32_t mulw(uint32_t x, Tw32 t) const {
        const uint32_t q = x * t.c;
        const uint32_t h = __umulhi(x, t.w);   // < p
        const uint32_t l = __umulhi(q, p);     // < p
        return sub_sel(h, l);
    }
    // x * y * 2^-32 rem p for x, y < p.
    __device__ __forceinline__ uint32_t mulmont(uint32_t x, uint32_t y) const {
        const uint32_t lo = x * y;
        const uint32_t hi = __umulhi(x, y);
        const uint32_t q = lo * pinv;
        const uint32_t l = __umulhi(q, p);
        return sub_sel(hi, l);
    }
};

// Mont32W -- Mont32's residues and tables with two different instruction
// forms, chosen by measurement for the kernels whose work is dominated by
// twiddle and pointwise products (the row pass and the inverse column pass
// of the 2^16-point products):
//  * the product x w~ (or x y) is formed as one 32 x 32 -> 64-bit multiply;
//    its low word times p^-1 is the Montgomery quotient q, so the twiddle
//    product needs no companion: q = lo(x w~) p^-1 equals x phi rem 2^32
//    because phi = w~ p^-1, and the result is bit-identical to Mont32's;
//  * the tail h - l (+p when negative) takes the borrow mask from the high
//    word of the 64-bit difference and adds p with one multiply-add, as the
//    sums do, moving one instruction from the ALU pipe to the multiply-add
//    pipe.  For h, l < p the value is h - l when h >= l and h - l + p
//    otherwise, in [0, p) either way (a zero product gives h = l = 0).
struct Mont32W : Mont32 {
    static constexpr bool kWide = true;   // the twiddle product ignores the companion
    __host__ __device__ __forceinline__ explicit Mont32W(const Mont32& m) : Mont32(m) {}
    __device__ __forceinline__ uint32_t tail(uint32_t h, uint32_t l) const {
        const uint64_t d = static_cast<uint64_t>(h) - l;
        const uint32_t m = static_cast<uint32_t>(d >> 32);
        return m * (0u - p) + static_cast<uint32_t>(d);
    }
    // x * w rem p for any 32-bit x; reads t.w (= w 2^32 rem p) only.
    __device__ __forceinline__ uint32_t mulw(uint32_t x, Tw32 t) const {
        const uint64_t xw = static_cast<uint64_t>(x) * t.w;
        const uint32_t q = static_cast<uint32_t>(xw) * pinv;
        return tail(static_cast<uint32_t>(xw >> 32), __umulhi(q, p));
    }
    // x * y * 2^-32 rem p for x, y < p.
    __device__ __forceinline__ uint32_t mulmont(uint32_t x, uint32_t y) const {
        const uint64_t xy = static_cast<uint64_t>(x) * y;
        const uint32_t q = static_cast<uint32_t>(xy) * pinv;
        return tail(static_cast<uint32_t>(xy >> 32), __umulhi(q, p));
    }
};

// The form a kernel of the row and inverse-column passes computes with:
// Mont32W for 32-bit words, the policy itself otherwise.
template <class Ar> struct WideForm { using type = Ar; };
template <> struct WideForm<Mont32> { using type = Mont32W; };

template <class Ar>
__host__ __device__ __forceinline__ typename WideForm<Ar>::type wide_form(const Ar& ar) {
    return typename WideForm<Ar>::type(ar);
}

struct Shoup64 {
    using word = uint64_t;
    using tw = Tw64;
    static constexpr int kBits = 64;
    uint64_t p;      // modulus < 2^62
    uint64_t pinv;   // p^-1 rem 2^64

    __device__ __forceinline__ uint64_t add(uint64_t x, uint64_t y) const {
        uint64_t s = x + y;
        return (s >= p) ? s - p : s;
    }
    __device__ __forceinline__ uint64_t sub(uint64_t x, uint64_t y) const {
        uint64_t d = x - y;
        return (x >= y) ? d : d + p;
    }
    // x * w rem p for any 64-bit x; t = (w, floor(2^64 w / p)).
    __device__ __forceinline__ uint64_t mulw(uint64_t x, Tw64 t) const {
        uint64_t c = __umul64hi(x, t.c);
        uint64_t r = x * t.w - c * p;      // in [0, 2p) < 2^63
        return (r >= p) ? r - p : r;
    }
    // x * y * 2^-64 rem p for x, y < p.
    __device__ __forceinline__ uint64_t mulmont(uint64_t x, uint64_t y) const {
        uint64_t lo = x * y;
        uint64_t hi = __umul64hi(x, y);
        uint64_t q = lo * pinv;
        uint64_t l = __umul64hi(q, p);
        uint64_t r = hi - l;
        return (hi >= l) ? r : r + p;
    }
};

// Shoup64L -- the transform kernels' 64-bit policy: lazy residues in
// [0, 2p) (4p < 2^64 for p < 2^62).  The twiddle product is Function 8
// without its final test: x w - c p lies in [0, 2p) for every 64-bit x
// (Proposition 4: the quotient estimate is at most one short).  Sums and
// differences are taken modulo 2p with one test, except differences that
// feed a twiddle product, which skip it (x + 2p - y < 4p).  The general
// (pointwise) product is Montgomery's with m = 64 (x y < 4 p^2 < 2^64 p)
// and is fully reduced.  canon() brings a lazy value into [0, p) before it
// leaves a kernel.
struct Shoup64L {
    using word = uint64_t;
    using tw = Tw64;
    static constexpr int kBits = 64;
    uint64_t p;      // modulus < 2^62
    uint64_t pinv;   // p^-1 rem 2^64

    // s < 4p -> [0, 2p).  t = s - 2p read as a signed 64-bit value is
    // negative exactly when s < 2p (2p - s <= 2p < 2^63), so the choice
    // needs the sign of t's high word only, not a 64-bit comparison.
    __device__ __forceinline__ uint64_t red2(uint64_t s) const {
        const uint64_t t = s - 2 * p;
        return (static_cast<int64_t>(t) < 0) ? s : t;
    }
    __device__ __forceinline__ uint64_t add(uint64_t x, uint64_t y) const { return red2(x + y); }
    __device__ __forceinline__ uint64_t sub(uint64_t x, uint64_t y) const { return red2(x + 2 * p - y); }
    __device__ __forceinline__ uint64_t sub_lazy(uint64_t x, uint64_t y) const { return x + 2 * p - y; }
    __device__ __forceinline__ uint64_t mulw(uint64_t x, Tw64 t) const {
        const uint64_t c = __umul64hi(x, t.c);
        return x * t.w - c * p;
    }
    __device__ __forceinline__ uint64_t mulmont(uint64_t x, uint64_t y) const {
        const uint64_t lo = x * y;
        const uint64_t hi = __umul64hi(x, y);
        const uint64_t q = lo * pinv;
        const uint64_t l = __umul64hi(q, p);
        const uint64_t r = hi - l;                       // hi, l < p < 2^62: negative iff hi < l
        return (static_cast<int64_t>(r) < 0) ? r + p : r;
    }
    // [0, 2p) -> [0, p), with the same sign test
    __device__ __forceinline__ uint64_t canon(uint64_t x) const {
        const uint64_t t = x - p;
        return (static_cast<int64_t>(t) < 0) ? x : t;
    }
};

// Fma50 -- residues as IEEE doubles, p < 2^50 (m <= l - 2 with l = 53 for
// double).  Every product, twiddle or pointwise, is Function 16: the exact
// product split by one FMA into h + l, the quotient c = floor(h u) with
// u = 1/p rounded to nearest, d = h - c p by a second FMA, and e = d + l
// corrected once by +-p (Proposition 13: correct for any rounding mode when
// the product is below 2^(l-2) p).  Sums and differences stay in [0, p) with
// one correction each (exact: sums are below 2^51).  There is no Montgomery
// factor, so the pointwise product needs no extra scaling.
struct TwF { double w; };

struct Fma50 {
    using word = double;
    using tw = TwF;
    static constexpr int kBits = 53;
    double p;   // modulus < 2^50 (exact as a double)
    double u;   // 1/p rounded to nearest

    __device__ __forceinline__ double mul(double a, double b) const {
        const double h = a * b;
        const double l = fma(a, b, -h);
        const double c = floor(h * u);
        const double d = fma(-c, p, h);
        const double e = d + l;
        if (e >= p) return e - p;
        return (e < 0.0) ? e + p : e;
    }
    __device__ __forceinline__ double add(double x, double y) const {
        const double s = x + y;
        return (s >= p) ? s - p : s;
    }
    __device__ __forceinline__ double sub(double x, double y) const {
        const double d = x - y;
        return (d < 0.0) ? d + p : d;
    }
    // Function 16 wants a non-negative product, so differences stay reduced
    __device__ __forceinline__ double sub_lazy(double x, double y) const { return sub(x, y); }
    __device__ __forceinline__ double canon(double x) const { return x; }
    __device__ __forceinline__ double mulw(double x, TwF t) const { return mul(x, t.w); }
    __device__ __forceinline__ double mulmont(double x, double y) const { return mul(x, y); }
};

}  // namespace gbntt
