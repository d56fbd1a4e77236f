// Host-side prime-field arithmetic for planning (arXiv 2001.04109, Section 3.1).
//
// Primality (deterministic Miller-Rabin), Legendre symbols, Tonelli-Shanks
// square roots, a square root of −1 (Prop. 3.2), the sum-of-two-squares
// decomposition a² + b² ≡ −1 (Algorithm 3, "SoS"), the p ≡ 3 (mod 8) case
// a = 1, b = √−2 (proof of Thm 4.1), and the signed byte-digit split
// with the chunk lengths that keep FP32 tensor-core sums exact.
#pragma once
#include <stdint.h>

namespace fsk {
namespace host {

inline uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m) {
    return (uint64_t)((unsigned __int128)a * b % m);
}
inline uint64_t powmod64(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod64(r, a, m);
        a = mulmod64(a, a, m);
        e >>= 1;
    }
    return r;
}

// Deterministic for every n < 2^64 with these witnesses.
inline bool is_prime(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t q : small) {
        if (n % q == 0) return n == q;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++s;
    }
    for (uint64_t a : small) {
        uint64_t x = powmod64(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = mulmod64(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

// Euler's criterion: 1 for a non-zero square, p−1 for a non-square, 0 for 0.
inline uint64_t euler(uint64_t a, uint64_t p) { return powmod64(a % p, (p - 1) / 2, p); }
inline bool is_square(uint64_t a, uint64_t p) { return a % p == 0 || euler(a, p) == 1; }

inline uint64_t least_non_square(uint64_t p) {
    uint64_t s = 2;
    while (is_square(s, p)) ++s;
    return s;
}

// Tonelli-Shanks square root of a square a mod an odd prime p.
inline uint64_t sqrt_mod(uint64_t a, uint64_t p) {
    a %= p;
    if (a == 0) return 0;
    if (p % 4 == 3) return powmod64(a, (p + 1) / 4, p);
    uint64_t q = p - 1;
    int s = 0;
    while ((q & 1) == 0) {
        q >>= 1;
        ++s;
    }
    uint64_t z = least_non_square(p);
    uint64_t M = s, c = powmod64(z, q, p), t = powmod64(a, q, p), r = powmod64(a, (q + 1) / 2, p);
    while (t != 1) {
        uint64_t i = 0, t2 = t;
        while (t2 != 1) {
            t2 = mulmod64(t2, t2, p);
            ++i;
        }
        uint64_t b = c;
        for (uint64_t e = 0; e + i + 1 < M; ++e) b = mulmod64(b, b, p);
        M = i;
        c = mulmod64(b, b, p);
        t = mulmod64(t, c, p);
        r = mulmod64(r, b, p);
    }
    return r;
}

struct YChoice {
    int form;       // 0: i·I ; 1: I ⊗ [[a,b],[−b,a]]
    uint64_t a, b;  // i (form 0) or (a, b)
    int cost;       // y of Thm 4.1
};

// The paper's choice of skew-orthogonal Y for F_p (proof of Thm 4.1).
inline YChoice choose_y(uint64_t p) {
    YChoice y{};
    if (p % 4 == 1) {
        // x^((p−1)/4) for a non-square x squares to −1 (Prop. 3.2)
        uint64_t i = powmod64(least_non_square(p), (p - 1) / 4, p);
        y.form = 0;
        y.a = i < p - i ? i : p - i;
        y.b = 0;
        y.cost = 1;
    } else if (p % 8 == 3) {
        y.form = 1;
        y.a = 1;
        y.b = sqrt_mod(p - 2, p);  // −2 is a square when p ≡ 3 (mod 8)
        y.cost = 2;
    } else {
        // Algorithm 3 with k = −1: s the least non-square, c² = s − 1,
        // a² = −s⁻¹, so a² + (a·c)² = a²·s = −1.
        uint64_t s = least_non_square(p);
        uint64_t c = sqrt_mod(s - 1, p);
        uint64_t sinv = powmod64(s, p - 2, p);
        uint64_t r = mulmod64(p - 1, sinv, p);
        uint64_t a = sqrt_mod(r, p);
        y.form = 1;
        y.a = a;
        y.b = mulmod64(a, c, p);
        y.cost = 3;
    }
    return y;
}

// A sum of two squares a² + b² ≡ k (mod p) for any k (Algorithm 3, SoS):
// a square k is a² + 0²; otherwise, with s the least non-square, c² = s − 1
// (a square, being smaller than s) and a² = k·s⁻¹ (a quotient of two
// non-squares, so a square), a² + (a·c)² = a²·s = k.
inline void sos(uint64_t k, uint64_t p, uint64_t &a, uint64_t &b) {
    k %= p;
    if (is_square(k, p)) {
        a = sqrt_mod(k, p);
        b = 0;
        return;
    }
    const uint64_t s = least_non_square(p);
    const uint64_t c = sqrt_mod(s - 1, p);
    a = sqrt_mod(mulmod64(k, powmod64(s, p - 2, p), p), p);
    b = mulmod64(a, c, p);
}

// Algorithm 4 (nrsyf): for two non-squares α, β a matrix Y = [[a, b], [c, d]]
// with Y·Yᵀ = Diag(α, β): α = a² + b² (SoS), d = a·√(β/α), c = −b·d/a.
// a ≠ 0 because α is not a square.
inline void nrsyf(uint64_t alpha, uint64_t beta, uint64_t p, uint64_t &a, uint64_t &b, uint64_t &c,
                  uint64_t &d) {
    sos(alpha, p, a, b);
    const uint64_t ainv = powmod64(a, p - 2, p);
    d = mulmod64(a, sqrt_mod(mulmod64(beta, powmod64(alpha, p - 2, p), p), p), p);
    c = (p - mulmod64(mulmod64(b, d, p), ainv, p)) % p;
}

// Balanced base-256 digits of s ∈ [−(p−1)/2, (p−1)/2]: the low D−1 digits lie
// in [−128, 127]; the top one takes the rest.
inline void split_digits(int64_t s, int D, int *d) {
    for (int t = 0; t < D - 1; ++t) {
        int lo = (int)(int8_t)(uint8_t)(s & 0xFF);
        d[t] = lo;
        s = (s - lo) / 256;
    }
    d[D - 1] = (int)s;
}

}  // namespace host
}  // namespace fsk
