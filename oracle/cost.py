"""Arithmetic operation counts of Section 4.1 and Appendix A.2 -- TEST INFRASTRUCTURE.

Counts are exact integers (``fractions.Fraction`` where a half appears) for
n×n inputs, n a power of two, as in Table 5:

* SYRK(n): classical n×n product by its transpose, n(n+1)/2 entries of n
  multiplications and n−1 additions each.
* MM(n): classical general product, n² entries of 2n − 1 operations.
* SW_l(n): Strassen-Winograd (Algorithm 1, 7 products and 15 additions)
  with l recursive levels over classical products.
* G_y-i(n): Algorithm 2 with i recursive levels, whose 2 general products
  use SW with i − 1 levels; Eq. (complexity) of Thm 4.1 with the addition
  count (7.5 + 2y)(n/2)² of Remark 4.1 and the Y cost y ∈ {0, 1, 2, 3}.
* Syrk-i(n): the classical 2×2 divide and conquer with i levels (4
  recursive products, 2 general products by SW with i − 1 levels, two half
  additions and one full addition of n/2 blocks).
"""
from __future__ import annotations

from fractions import Fraction


def syrk_classical(n: int) -> int:
    return n * (n + 1) // 2 * (2 * n - 1)


def mm_classical(n: int) -> int:
    return n * n * (2 * n - 1)


def sw(n: int, levels: int) -> int:
    if levels <= 0:
        return mm_classical(n)
    h = n // 2
    return 7 * sw(h, levels - 1) + 15 * h * h


def g(n: int, i: int, y: int) -> Fraction:
    """Algorithm 2 with i levels (Eq. complexity), Y costing y·(n/2)² per level."""
    if i <= 0:
        return Fraction(syrk_classical(n))
    h = n // 2
    return 3 * g(h, i - 1, y) + 2 * sw(h, i - 1) + (Fraction(15, 2) + 2 * y) * h * h


def syrk_dc(n: int, i: int) -> Fraction:
    """Classical divide and conquer with i levels (Syrk-i)."""
    if i <= 0:
        return Fraction(syrk_classical(n))
    h = n // 2
    return 4 * syrk_dc(h, i - 1) + 2 * sw(h, i - 1) + 2 * Fraction(h * (h + 1), 2) + h * h


def field_macs_fast(n: int, k: int, levels: int) -> int:
    """Field multiply-adds of Algorithm 2 with `levels` levels over classical leaves.

    Leaf syrk products count n(n+1)/2·k, general products n²·k (n, k the
    block sizes at that depth, assumed divisible by 2^levels).
    """
    if levels <= 0:
        return n * (n + 1) // 2 * k
    h, w = n // 2, k // 2
    return 3 * field_macs_fast(h, w, levels - 1) + 2 * h * h * w


def g_classical(n: int, i: int, y: int) -> Fraction:
    """Algorithm 2 with i levels whose general products are classical (ω = 3)."""
    if i <= 0:
        return Fraction(syrk_classical(n))
    h = n // 2
    return 3 * g_classical(h, i - 1, y) + 2 * mm_classical(h) + (Fraction(15, 2) + 2 * y) * h * h
