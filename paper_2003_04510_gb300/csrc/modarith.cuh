// modarith.cuh -- 64-bit modular arithmetic for sm_103a kernels.
//
// Residues are uint64.  Moduli are NTT-friendly primes below 2^62 (the
// configurations use 50- to 55-bit primes), so 4q still fits in a word and the
// lazy ranges below are safe.
//
//  * shoup_lazy / shoup: Shoup's modular multiplication by a constant
//    (the paper's Algo 2) with w' = floor(w * 2^64 / q).  The lazy form returns
//    a value in [0, 2q); the paper's correction "if r > p" is read as r >= q,
//    which the full form applies.
//  * mul_wide / mac: 64x64 -> 128-bit products accumulated without reduction
//    (the lazy reduction idea the paper applies to CRT accumulation, Sec. 5.3).
//  * barrett128: one reduction of a 128-bit accumulator V < 2^(b+61), where
//    b = bitlen(q).  mu = floor(2^(62+b) / q); the quotient estimate
//    floor((V >> (b-2)) * mu / 2^64) is the true quotient or one less, so the
//    remainder needs a single conditional subtraction.
#pragma once
#include <cstdint>

typedef uint64_t u64;

struct U128 {
    u64 lo, hi;
};

__device__ __forceinline__ u64 shoup_lazy(u64 x, u64 w, u64 wp, u64 q)
{
    u64 qh = __umul64hi(x, wp);
    return x * w - qh * q;  // in [0, 2q), exact mod 2^64
}

__device__ __forceinline__ u64 csub(u64 x, u64 q) { return x >= q ? x - q : x; }

// 32x32 -> 64-bit multiply-add and 32x32 -> high-32 multiply, written as PTX
// so each is one integer multiply-add instruction.
__device__ __forceinline__ u64 mad_wide(uint32_t a, uint32_t b, u64 c)
{
    u64 d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint32_t mul_hi32(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// The paper's modified Shoup multiplication (Sec. 5.2): the quotient
// floor(x * w' / 2^64) is estimated from three 32-bit partial products only
// (x1 w'1, hi(x1 w'0), hi(x0 w'1)); the dropped terms are each below one
// unit, so the estimate is the exact quotient minus 0, 1 or 2 and the
// remainder x*w - qh*q lies in [0, 4q).  Valid for any x < 2^64, w < q < 2^62.
__device__ __forceinline__ u64 shoup_approx(u64 x, u64 w, u64 wp, u64 q)
{
    const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
    const uint32_t p0 = (uint32_t)wp, p1 = (uint32_t)(wp >> 32);
    const u64 qh = mad_wide(x1, p1, (u64)mul_hi32(x1, p0) + mul_hi32(x0, p1));
    return x * w - qh * q;
}

// The same remainder with the subtraction folded into the multiply-adds:
// x*w - qh*q = x*w + qh*nq (mod 2^64), nq = 2^64 - q.  The low word comes
// from two chained 32x32 -> 64-bit multiply-adds, the high word from four
// 32-bit multiply-adds on top of its carry-in; exact mod 2^64, which is
// enough since the remainder is below 4q.
__device__ __forceinline__ u64 shoup_approx_nq(u64 x, u64 w, u64 wp, u64 nq)
{
    const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
    const uint32_t p0 = (uint32_t)wp, p1 = (uint32_t)(wp >> 32);
    const u64 qh = mad_wide(x1, p1, (u64)mul_hi32(x1, p0) + mul_hi32(x0, p1));
    const uint32_t h0 = (uint32_t)qh, h1 = (uint32_t)(qh >> 32);
    const uint32_t w0 = (uint32_t)w, w1 = (uint32_t)(w >> 32);
    const uint32_t n0 = (uint32_t)nq, n1 = (uint32_t)(nq >> 32);
    const u64 lo = mad_wide(h0, n0, mad_wide(x0, w0, 0ull));
    uint32_t hi = (uint32_t)(lo >> 32);
    hi += x0 * w1;
    hi += x1 * w0;
    hi += h0 * n1;
    hi += h1 * n0;
    return (lo & 0xFFFFFFFFull) | ((u64)hi << 32);
}

__device__ __forceinline__ u64 shoup(u64 x, u64 w, u64 wp, u64 q) { return csub(shoup_lazy(x, w, wp, q), q); }

// x w mod q, canonical: the modified Shoup product (remainder in [0, 4q))
// and two conditional subtractions.  Fewer wide multiplies than shoup()
// (which forms the exact Shoup quotient); nq = 2^64 - q, q < 2^62.
__device__ __forceinline__ u64 shoup_canon(u64 x, u64 w, u64 wp, u64 q, u64 nq)
{
    return csub(csub(shoup_approx_nq(x, w, wp, nq), 2 * q), q);
}

// x mod q for x below 2^64 and below a small multiple of q (at most 2^32 q),
// q > 2^32, r64 = floor(2^64 / q) (then below 2^32): the quotient estimate
// floor((x >> 32) r64 / 2^32) is floor(x / q) minus 0, 1 or 2 (the dropped
// low word of x is below q, and (x >> 32)(2^64 / q - r64) / 2^32 < 1), so
// the remainder lies in [0, 3q) and two conditional subtractions finish.
// One 32 x 32 high multiply and a 32 x 64 product instead of a Shoup product.
__device__ __forceinline__ u64 reduce_small(u64 x, u64 q, u64 r64)
{
    const uint32_t qh = mul_hi32((uint32_t)(x >> 32), (uint32_t)r64);
    const u64 r = x - (u64)qh * q;
    return csub(csub(r, 2 * q), q);
}

// The NTT's butterflies (ntt.cu; the throughput probe runs the same ones).
// Forward (Cooley-Tukey, Algo 4) with no correction step: the modified
// Shoup product t lies in [0, 4q), so each stage adds at most 4q to the
// range.  From inputs below 4q (the base conversions leave their outputs
// lazily reduced), values stay below (4 + 4 log N) q < 2^64 for q < 2^57.8
// and are reduced once, on the final store.  w = (value, Shoup companion),
// nq = 2^64 - q.
__device__ __forceinline__ void ct_bfly(u64 &x, u64 &y, ulonglong2 w, u64 nq, u64 q4)
{
    const u64 t = shoup_approx_nq(y, w.x, w.y, nq);
    y = x + q4 - t;
    x = x + t;
}

// Inverse (Gentleman-Sande) butterfly on values in [0, 4q): the sum is
// brought back below 4q with one conditional subtraction, the difference
// goes through the modified Shoup product, which lands in [0, 4q).
__device__ __forceinline__ void gs_bfly(u64 &x, u64 &y, ulonglong2 w, u64 nq, u64 q4)
{
    u64 s = x + y;
    s = s >= q4 ? s - q4 : s;
    const u64 d = x + q4 - y;
    y = shoup_approx_nq(d, w.x, w.y, nq);
    x = s;
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) { return csub(a + b, q); }

__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

__device__ __forceinline__ U128 mul_wide(u64 a, u64 b)
{
    U128 r;
    r.lo = a * b;
    r.hi = __umul64hi(a, b);
    return r;
}

__device__ __forceinline__ void mac(U128 &acc, u64 a, u64 b)
{
    u64 lo = a * b;
    u64 hi = __umul64hi(a, b);
    acc.lo += lo;
    acc.hi += hi + (acc.lo < lo ? 1ull : 0ull);
}

// V mod q for V = acc < 2^(b+61); s = b - 2 (1 <= s <= 60), mu = floor(2^(64+s) / q).
__device__ __forceinline__ u64 barrett128(U128 v, u64 q, u64 mu, unsigned s)
{
    // bits [s, s + 64) of v from two 32-bit funnel shifts (the word triple
    // starts one word higher when s >= 32; the shift amount is s mod 32)
    const uint32_t l0 = (uint32_t)v.lo, l1 = (uint32_t)(v.lo >> 32), h0 = (uint32_t)v.hi, h1 = (uint32_t)(v.hi >> 32);
    const bool up = s >= 32;
    const uint32_t w0 = up ? l1 : l0, w1 = up ? h0 : l1, w2 = up ? h1 : h0;
    const u64 u = ((u64)__funnelshift_r(w1, w2, s) << 32) | __funnelshift_r(w0, w1, s);
    u64 qh = __umul64hi(u, mu);
    u64 r = v.lo - qh * q;  // in [0, 2q)
    return csub(r, q);
}

__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, u64 q, u64 mu, unsigned s)
{
    return barrett128(mul_wide(a, b), q, mu, s);
}

// Lazy dot products of a residue vector with constant vectors (base
// conversion).  Operands are split at bit 28: x = x1*2^28 + x0, and the
// constant is stored pre-split as b0 | (b1 << 32).  Each term is four
// 32x32 -> 64-bit multiply-adds into three 64-bit accumulators with no carry
// handling: for x, b < 2^57 and at most 16 terms every accumulator stays below
// 2^63.  The 128-bit value is assembled once per output.
struct Acc3 {
    u64 a0, a1, a2;  // weights 1, 2^28, 2^56
};

__device__ __forceinline__ void split28(u64 x, uint32_t &x0, uint32_t &x1)
{
    x0 = (uint32_t)(x & 0xFFFFFFFull);
    x1 = (uint32_t)(x >> 28);
}

__device__ __forceinline__ void mac28(Acc3 &s, uint32_t x0, uint32_t x1, u64 bpacked)
{
    const uint32_t b0 = (uint32_t)bpacked, b1 = (uint32_t)(bpacked >> 32);
    s.a0 = mad_wide(x0, b0, s.a0);
    s.a1 = mad_wide(x0, b1, s.a1);
    s.a1 = mad_wide(x1, b0, s.a1);
    s.a2 = mad_wide(x1, b1, s.a2);
}

// Karatsuba form of mac28: three multiply-adds per term, x0*b0 (into a0),
// x1*b1 (into a2) and (x0+x1)*(b0+b1) (into a1, which then holds the sum of
// all three products' middle parts plus a0 and a2; acc3k_value takes them
// out).  xs = x0 + x1 is formed once per input.  For x, b < 2^57 and at most
// 16 terms: a0 < 2^60, a2 < 2^62 and a1 < 16 * 9 * 2^56 < 2^64, and the
// recovered middle sum x0*b1 + x1*b0 stays below 2^62, so acc3k_value returns
// exactly what acc3_value returns for the four-product form.
__device__ __forceinline__ void mac28k(Acc3 &s, uint32_t x0, uint32_t x1, uint32_t xs, u64 bpacked)
{
    const uint32_t b0 = (uint32_t)bpacked, b1 = (uint32_t)(bpacked >> 32);
    s.a0 = mad_wide(x0, b0, s.a0);
    s.a2 = mad_wide(x1, b1, s.a2);
    s.a1 = mad_wide(xs, b0 + b1, s.a1);
}

__device__ __forceinline__ U128 acc3_value(const Acc3 &s)
{
    U128 v;
    const u64 t1 = s.a1 << 28, t2 = s.a2 << 56;
    v.lo = s.a0 + t1;
    u64 c = v.lo < t1 ? 1ull : 0ull;
    v.lo += t2;
    c += v.lo < t2 ? 1ull : 0ull;
    v.hi = (s.a1 >> 36) + (s.a2 >> 8) + c;
    return v;
}

__device__ __forceinline__ U128 acc3k_value(const Acc3 &k)
{
    Acc3 t;
    t.a0 = k.a0;
    t.a1 = k.a1 - k.a0 - k.a2;
    t.a2 = k.a2;
    return acc3_value(t);
}

// V mod q, lazily in [0, 3q), straight from the Karatsuba accumulators
// (V = a0 + m 2^28 + a2 2^56, m = a1 - a0 - a2 >= 0, V < 2^(b+61)), without
// assembling the 128-bit value.  With s = b - 2 (28 <= s <= 56) and
// mu = floor(2^(64+s) / q) as for barrett128: the shifted value
// u' = a2 2^(56-s) + floor(m / 2^(s-28)) + floor(a0 / 2^s) is floor(V / 2^s)
// or one less (two dropped fractions, each below one), so
// floor(u' mu / 2^64) is floor(V / q) minus 0, 1 or 2 (Barrett's own estimate
// is the true quotient or one less), and V minus that multiple of q, formed
// modulo 2^64 from V's low word, lies in [0, 3q).  Every term fits a word:
// a2 2^(56-s) <= V / 2^s < 2^63.
__device__ __forceinline__ u64 acc3k_reduce_lazy(const Acc3 &k, u64 q, u64 mu, unsigned s)
{
    const u64 m = k.a1 - k.a0 - k.a2;
    const u64 u = (k.a2 << (56 - s)) + (m >> (s - 28)) + (k.a0 >> s);
    const u64 vlo = k.a0 + (m << 28) + (k.a2 << 56);
    return vlo - __umul64hi(u, mu) * q;
}
