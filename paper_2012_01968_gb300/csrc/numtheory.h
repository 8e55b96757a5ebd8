// Host number theory for plan creation: primality, factoring q - 1, the
// smallest generator of Z_q^*, and psi = g^{(q-1)/2N}.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace ntt {
namespace nt {

typedef unsigned __int128 u128;
typedef uint64_t u64;

inline u64 mulmod(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }

inline u64 powmod(u64 b, u64 e, u64 m)
{
    u64 r = 1 % m;
    b %= m;
    for (; e; e >>= 1) {
        if (e & 1) r = mulmod(r, b, m);
        b = mulmod(b, b, m);
    }
    return r;
}

// Deterministic Miller-Rabin; bases 2..37 decide every 64-bit n.
inline bool is_prime(u64 n)
{
    static const u64 B[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 p : B)
        if (n % p == 0) return n == p;
    u64 d = n - 1;
    int s = __builtin_ctzll(d);
    d >>= s;
    for (u64 a : B) {
        u64 x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < s && comp; ++i) {
            x = mulmod(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

inline u64 gcd(u64 a, u64 b)
{
    while (b) {
        u64 t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Pollard's rho with Brent's cycle detection; n composite and odd.
inline u64 rho(u64 n)
{
    for (u64 c = 1;; ++c) {
        u64 y = 2, x = 2, g = 1, q = 1, ys = 2;
        u64 r = 1;
        const u64 m = 128;
        auto f = [&](u64 v) { return (mulmod(v, v, n) + c) % n; };
        do {
            x = y;
            for (u64 i = 0; i < r; ++i) y = f(y);
            u64 k = 0;
            do {
                ys = y;
                for (u64 i = 0; i < std::min(m, r - k); ++i) {
                    y = f(y);
                    q = mulmod(q, x > y ? x - y : y - x, n);
                }
                g = gcd(q, n);
                k += m;
            } while (k < r && g == 1);
            r <<= 1;
        } while (g == 1);
        if (g == n) {
            do {
                ys = f(ys);
                g = gcd(x > ys ? x - ys : ys - x, n);
            } while (g == 1);
        }
        if (g != n) return g;
    }
}

inline void factor_into(u64 n, std::vector<u64>& out)
{
    if (n == 1) return;
    for (u64 p : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull}) {
        if (n % p == 0) {
            out.push_back(p);
            while (n % p == 0) n /= p;
        }
    }
    if (n == 1) return;
    if (is_prime(n)) {
        out.push_back(n);
        return;
    }
    u64 d = rho(n);
    factor_into(d, out);
    factor_into(n / d, out);
}

// distinct prime factors, ascending
inline std::vector<u64> prime_factors(u64 n)
{
    std::vector<u64> f;
    factor_into(n, f);
    std::sort(f.begin(), f.end());
    f.erase(std::unique(f.begin(), f.end()), f.end());
    return f;
}

inline u64 smallest_generator(u64 q)
{
    const std::vector<u64> f = prime_factors(q - 1);
    for (u64 g = 2; g < q; ++g) {
        bool ok = true;
        for (u64 p : f)
            if (powmod(g, (q - 1) / p, q) == 1) {
                ok = false;
                break;
            }
        if (ok) return g;
    }
    return 0;
}

inline int bitlen(u64 x) { return x ? 64 - __builtin_clzll(x) : 0; }

inline u64 brv(u64 i, int bits)
{
    u64 r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// Shoup companion floor(w 2^64 / q), w < q
inline u64 shoup_companion(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

}  // namespace nt
}  // namespace ntt
