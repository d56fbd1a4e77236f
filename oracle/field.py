"""Prime-field helpers and skew-orthogonal matrices -- TEST INFRASTRUCTURE.

Plain Python integers throughout.  Follows Section 3.1 of arXiv 2001.04109:

* Definition (skew-orthogonal): Yᵀ = −Y⁻¹, i.e. Y·Yᵀ = −I.
* Prop. 3.2: for p ≡ 1 (mod 4) the field holds a square root i of −1, and
  Y = i·I is skew-orthogonal.
* Prop. 3.3: in every prime field there are a, b with a² + b² = −1, and
  Y = [[a, b], [−b, a]] ⊗ I is skew-orthogonal.
* Algorithm 3 (SoS): a, b with a² + b² ≡ k (mod p) from the least quadratic
  non-residue and two modular square roots.
* Proof of Thm 4.1: when p ≡ 3 (mod 8), −2 is a square and a = 1,
  b = √−2 gives the cheaper 2×2 form.
"""
from __future__ import annotations


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (first 13 prime bases)."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41)
    for q in small:
        if n % q == 0:
            return n == q
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def legendre(a: int, p: int) -> int:
    """Legendre symbol (a/p) for an odd prime p by Euler's criterion: 1, −1 or 0."""
    a %= p
    if a == 0:
        return 0
    t = pow(a, (p - 1) // 2, p)
    return 1 if t == 1 else -1


def sqrt_mod(a: int, p: int) -> int:
    """A square root of the quadratic residue a mod the odd prime p (Tonelli-Shanks)."""
    a %= p
    if a == 0:
        return 0
    if legendre(a, p) != 1:
        raise ValueError(f"{a} is not a square mod {p}")
    if p % 4 == 3:
        return pow(a, (p + 1) // 4, p)
    q, s = p - 1, 0
    while q % 2 == 0:
        q //= 2
        s += 1
    z = 2
    while legendre(z, p) != -1:
        z += 1
    m, c, t, r = s, pow(z, q, p), pow(a, q, p), pow(a, (q + 1) // 2, p)
    while t != 1:
        i, t2 = 0, t
        while t2 != 1:
            t2 = t2 * t2 % p
            i += 1
        b = pow(c, 1 << (m - i - 1), p)
        m, c, t, r = i, b * b % p, t * b * b % p, r * b % p
    return r


def least_non_residue(p: int) -> int:
    s = 2
    while legendre(s, p) == 1:
        s += 1
    return s


def sqrt_minus_one(p: int) -> int:
    """i with i² ≡ −1 (mod p), p ≡ 1 (mod 4) (Prop. 3.2).

    Following the proof of Prop. 3.2: x^((p−1)/4) squares to x^((p−1)/2),
    which is −1 exactly when x is a non-residue.  The smaller of the two
    roots {i, p−i} is returned so the choice is deterministic.
    """
    if p % 4 != 1:
        raise ValueError("−1 is a square only when p ≡ 1 (mod 4)")
    x = least_non_residue(p)
    i = pow(x, (p - 1) // 4, p)
    return min(i, p - i)


def sos(p: int, k: int) -> tuple[int, int]:
    """Algorithm 3 (SoS): (a, b) with a² + b² ≡ k (mod p), p an odd prime.

    If k is a square, (√k, 0).  Otherwise s, the least non-residue, is one
    more than a square c² (s − 1 is a residue since s is the least
    non-residue), k·s⁻¹ is a residue a², and k = a²·s = a² + (a·c)².
    """
    k %= p
    if legendre(k, p) == 1 or k == 0:
        return sqrt_mod(k, p), 0
    s = least_non_residue(p)
    c = sqrt_mod(s - 1, p)
    r = k * pow(s, -1, p) % p
    a = sqrt_mod(r, p)
    return a, a * c % p


def y_params(p: int) -> dict:
    """The skew-orthogonal Y the paper prescribes for F_p (proof of Thm 4.1).

    Returns ``{"form": "scalar", "i": i, "y": 1}`` for p ≡ 1 (mod 4);
    ``{"form": "2x2", "a": 1, "b": √−2, "y": 2}`` for p ≡ 3 (mod 8);
    otherwise ``{"form": "2x2", "a": a, "b": b, "y": 3}`` from SoS(p, −1).
    """
    if p % 4 == 1:
        return {"form": "scalar", "i": sqrt_minus_one(p), "y": 1}
    if p % 8 == 3:
        return {"form": "2x2", "a": 1, "b": sqrt_mod(p - 2, p), "y": 2}
    a, b = sos(p, p - 1)
    return {"form": "2x2", "a": a, "b": b, "y": 3}


def y_matrix(p: int, w: int, layout: str = "interleaved", params: dict | None = None):
    """The w×w skew-orthogonal Y as a list of lists of ints mod p.

    ``layout`` for the 2×2 form: ``"block"`` is [[aI, bI], [−bI, aI]] of
    Prop. 3.3; ``"interleaved"`` is I ⊗ [[a, b], [−b, a]] (the same matrix
    up to a symmetric permutation of rows and columns, hence also
    skew-orthogonal).  The 2×2 form needs w even.
    """
    prm = params or y_params(p)
    Y = [[0] * w for _ in range(w)]
    if prm["form"] == "scalar":
        for t in range(w):
            Y[t][t] = prm["i"] % p
        return Y
    if w % 2:
        raise ValueError("the 2×2 skew-orthogonal form needs an even dimension")
    a, b = prm["a"] % p, prm["b"] % p
    h = w // 2
    for t in range(h):
        if layout == "block":
            r0, r1 = t, t + h
        else:
            r0, r1 = 2 * t, 2 * t + 1
        Y[r0][r0] = a
        Y[r0][r1] = b
        Y[r1][r0] = (-b) % p
        Y[r1][r1] = a
    return Y
