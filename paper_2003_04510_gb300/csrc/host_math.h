// host_math.h -- host-side 64-bit modular helpers of the library (parameter
// generation, table building, key generation).  Not used by the kernels.
#pragma once
#include <cstdint>
#include <vector>

namespace he {
namespace hm {

typedef uint64_t u64;
typedef unsigned __int128 u128;

inline u64 mul(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }
inline u64 add(u64 a, u64 b, u64 m) { u64 s = a + b; return s >= m ? s - m : s; }
inline u64 sub(u64 a, u64 b, u64 m) { return a >= b ? a - b : a + m - b; }
inline u64 pw(u64 b, u64 e, u64 m)
{
    u64 r = 1 % m;
    b %= m;
    for (; e; e >>= 1) {
        if (e & 1) r = mul(r, b, m);
        b = mul(b, b, m);
    }
    return r;
}
inline u64 inv(u64 a, u64 m) { return pw(a % m, m - 2, m); }  // m prime
// Shoup companion floor(w * 2^64 / m), w < m
inline u64 shoup(u64 w, u64 m) { return (u64)(((u128)w << 64) / m); }
inline int bitlen(u64 x) { int b = 0; while (x) { b++; x >>= 1; } return b; }
inline u64 bitrev(u64 x, int bits)
{
    u64 r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1ull) << (bits - 1 - i);
    return r;
}

// Deterministic Miller-Rabin for 64-bit n with the seven-base set of
// J. Sinclair (2, 325, 9375, 28178, 450775, 9780504, 1795265022).
inline bool is_prime(u64 n)
{
    if (n < 2) return false;
    static const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 s : small) {
        if (n == s) return true;
        if (n % s == 0) return false;
    }
    u64 d = n - 1;
    int r = 0;
    while (!(d & 1)) { d >>= 1; r++; }
    static const u64 bases[] = {2, 325, 9375, 28178, 450775, 9780504, 1795265022};
    for (u64 a : bases) {
        u64 x = pw(a, d, n);
        if (x == 0 || x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int i = 1; i < r && witness; i++) {
            x = mul(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

// Distinct prime factors by trial division (n up to ~2^64 with small cofactors
// after removing powers of two, enough for q - 1 = 2N * m with m < 2^45).
inline std::vector<u64> prime_factors(u64 n)
{
    std::vector<u64> f;
    for (u64 p = 2; p * p <= n; p += (p == 2 ? 1 : 2)) {
        if (n % p != 0) continue;
        f.push_back(p);
        while (n % p == 0) n /= p;
        if (n > 1 && is_prime(n)) break;  // the cofactor is prime: done
    }
    if (n > 1) f.push_back(n);
    return f;
}

}  // namespace hm
}  // namespace he
