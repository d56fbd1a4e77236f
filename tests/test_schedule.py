"""The tensor-core leaf's exact-accumulation schedule (CPU only, no GPU needed).

These pin, independently of the kernels, the property that makes the bf16
digit leaf exact: every FP32 accumulator (a "unit") sums at most 2^24 in
magnitude, holds a single weight class 256^(i+j), and every (digit pair,
k-block) is accumulated exactly once.  The digit bounds themselves are
checked by brute force over all symmetric residues of small primes and at
the extremes of the large ones.
"""
import numpy as np
import pytest

import __graft_entry__
from paper_2001_04109_gb300 import ffsyrk


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def balanced_digits(s, D, b):
    """Signed digits of s in base b, each low digit in [−b/2, b/2)."""
    out = []
    for _ in range(D - 1):
        lo = ((s + b // 2) % b) - b // 2
        out.append(lo)
        s = (s - lo) // b
    out.append(s)
    return out


# 509 / 521: the last one-digit and the first two-digit prime; 131321 / 131357:
# the last two-digit (balanced base) and the first three-digit prime
DIGIT_EDGES = [509, 521, 131321, 131357]


@pytest.mark.parametrize("p", [3, 251, 257, 65521, 65537, 131071, 131041, 8388593, 16777213] + DIGIT_EDGES)
def test_digit_bounds_cover_every_residue(p):
    bounds = ffsyrk.digit_bounds(p)
    b = ffsyrk.digit_base(p)
    D = len(bounds)
    h = (p - 1) // 2
    samples = range(-h, h + 1) if p < 300000 else list(range(-h, -h + 70000)) + list(range(h - 70000, h + 1))
    seen = [0] * D
    for s in samples:
        d = balanced_digits(s, D, b)
        assert sum(dt * b ** t for t, dt in enumerate(d)) == s
        for t in range(D):
            assert abs(d[t]) <= bounds[t] <= 256
            seen[t] = max(seen[t], abs(d[t]))
    assert seen == bounds  # tight


@pytest.mark.parametrize("p,base,bounds", [(65521, 256, [128, 128]), (131071, 362, [181, 181]),
                                           (8388593, 256, [128, 128, 64]), (251, 256, [125]),
                                           (509, 256, [254]), (521, 256, [128, 1]),
                                           (131321, 362, [181, 181]), (131357, 256, [128, 128, 1])])
def test_digit_base_and_bounds(p, base, bounds):
    # below 2^16 byte digits are already balanced; p = 131071 with bytes would
    # need a top digit of 256 (chunks of 4 k-blocks for the top pair), the
    # balanced base 362 bounds both digits by 181 (8 k-blocks for every pair)
    assert ffsyrk.digit_base(p) == base
    assert ffsyrk.digit_bounds(p) == bounds
    if base != 256:
        assert all(nkb <= 8 for *_, nkb, _ in ffsyrk.leaf_schedule(p, 64))
        assert min(nkb for *_, nkb, first in ffsyrk.leaf_schedule(p, 64) if first) >= 4


@pytest.mark.parametrize("p", [251, 65521, 131071, 8388593] + DIGIT_EDGES)
@pytest.mark.parametrize("kblocks", [1, 3, 4, 5, 16, 17, 33, 64, 513])
def test_schedule_units_exact_and_complete(p, kblocks):
    bounds = ffsyrk.digit_bounds(p)
    D = len(bounds)
    segs = ffsyrk.leaf_schedule(p, kblocks)
    assert segs and segs[0][4]
    covered = {}
    unit_sum, unit_class = 0, None
    for i, j, kb0, nkb, first in segs:
        assert nkb >= 1 and 0 <= kb0 and kb0 + nkb <= kblocks
        if first:
            unit_sum, unit_class = 0, i + j
        assert i + j == unit_class                  # one weight per accumulator
        unit_sum += 64 * nkb * bounds[i] * bounds[j]
        assert unit_sum <= 1 << 24                  # every FP32 partial sum exact
        for kb in range(kb0, kb0 + nkb):
            covered[(i, j, kb)] = covered.get((i, j, kb), 0) + 1
    assert set(covered) == {(i, j, kb) for i in range(D) for j in range(D) for kb in range(kblocks)}
    assert all(c == 1 for c in covered.values())


def test_same_weight_pairs_share_a_unit_for_short_k():
    # p = 65521: pairs (0,1) and (1,0) both weigh 256; with 4 k-blocks they fit one unit
    segs = ffsyrk.leaf_schedule(65521, 4)
    units = sum(1 for s in segs if s[4])
    assert units == 3
    segs = ffsyrk.leaf_schedule(8388593, 4)
    assert sum(1 for s in segs if s[4]) == 5   # one unit per weight class, D = 3


@pytest.mark.parametrize("p,s", [(509, 254), (521, 128), (131321, 65341), (131357, 32640),
                                 (65521, 32640), (131071, 65341), (8388593, 4161408)])
def test_bound_residues_reach_every_digit_bound(p, s):
    # the GPU tests' extreme inputs: every digit of s sits at its bound
    bounds = ffsyrk.digit_bounds(p)
    d = balanced_digits(s, len(bounds), ffsyrk.digit_base(p))
    assert [abs(x) for x in d] == bounds


@pytest.mark.parametrize("p", [251, 509, 521, 65521, 131071, 131357, 8388593, 16777213])
def test_digit_products_rebuild_the_product(p):
    # Σ_{i,j} b^{i+j}·D_i·D_jᵀ = S·Sᵀ over the integers (S the signed
    # residues), hence ≡ X·Xᵀ mod p with the weights b^{i+j} taken mod p
    b = ffsyrk.digit_base(p)
    D = len(ffsyrk.digit_bounds(p))
    rng = np.random.default_rng(p)
    X = rng.integers(0, p, size=(6, 9)).astype(object)
    h = (p - 1) // 2
    S = np.where(X > h, X - p, X)
    digits = np.array([[balanced_digits(int(s), D, b) for s in row] for row in S], dtype=object)
    Dt = [digits[:, :, t] for t in range(D)]
    exact = sum(b ** (i + j) * Dt[i].dot(Dt[j].T) for i in range(D) for j in range(D))
    assert np.array_equal(exact, S.dot(S.T))
    weighted = sum(pow(b, i + j, p) * Dt[i].dot(Dt[j].T) for i in range(D) for j in range(D))
    assert np.array_equal(weighted % p, X.dot(X.T) % p)


# ---- the INT8 leaf: bytes of the two's complement, int32 units within 2^30 ----

def twos_bytes(s, D):
    """Digits of s as the D bytes of its two's complement: unsigned low bytes, signed top byte."""
    out = [(s >> (8 * t)) & 255 for t in range(D - 1)]
    out.append(s >> (8 * (D - 1)))  # floor division: the signed top digit
    return out


@pytest.mark.parametrize("p,D,bounds", [(251, 1, [125]), (257, 2, [255, 1]), (65521, 2, [255, 128]),
                                        (65537, 3, [255, 255, 1]), (131071, 3, [255, 255, 1]),
                                        (8388593, 3, [255, 255, 64]), (16777213, 3, [255, 255, 128])])
def test_i8_digit_count_and_bounds(p, D, bounds):
    # D is the least count whose top byte holds every symmetric residue's sign
    assert ffsyrk.i8_digit_bounds(p) == bounds and len(bounds) == D
    h = (p - 1) // 2
    assert -(1 << (8 * D - 1)) <= -h and h <= (1 << (8 * D - 1)) - 1
    if D > 1:
        assert h > (1 << (8 * (D - 1) - 1)) - 1  # one digit fewer would not do


@pytest.mark.parametrize("p", [3, 251, 257, 65521, 65537, 131071, 8388593, 16777213])
def test_i8_digits_cover_every_residue(p):
    bounds = ffsyrk.i8_digit_bounds(p)
    D = len(bounds)
    h = (p - 1) // 2
    samples = range(-h, h + 1) if p < 300000 else list(range(-h, -h + 70000)) + list(range(h - 70000, h + 1))
    seen = [0] * D
    for s in samples:
        d = twos_bytes(s, D)
        assert sum(dt * 256 ** t for t, dt in enumerate(d)) == s
        for t in range(D - 1):
            assert 0 <= d[t] <= 255 == bounds[t]
        assert -128 <= d[-1] <= 127 and abs(d[-1]) <= bounds[-1]   # fits a signed byte
        seen = [max(a, abs(x)) for a, x in zip(seen, d)]
    assert seen == bounds  # tight


@pytest.mark.parametrize("p", [251, 257, 65521, 131071, 8388593])
@pytest.mark.parametrize("kblocks", [1, 2, 3, 100, 128, 129, 300, 1000])
def test_i8_schedule_units_exact_and_complete(p, kblocks):
    bounds = ffsyrk.i8_digit_bounds(p)
    D = len(bounds)
    segs = ffsyrk.i8_schedule(p, kblocks)
    assert segs and segs[0][4]
    covered = {}
    unit_sum, unit_class = 0, None
    for i, j, kb0, nkb, first in segs:
        assert nkb >= 1 and 0 <= kb0 and kb0 + nkb <= kblocks
        if first:
            unit_sum, unit_class = 0, i + j
        assert i + j == unit_class
        unit_sum += 128 * nkb * bounds[i] * bounds[j]
        assert unit_sum <= 1 << 30                  # int32, with room for the reduction's offset
        for kb in range(kb0, kb0 + nkb):
            covered[(i, j, kb)] = covered.get((i, j, kb), 0) + 1
    assert set(covered) == {(i, j, kb) for i in range(D) for j in range(D) for kb in range(kblocks)}
    assert all(c == 1 for c in covered.values())


def test_i8_one_unit_per_class_up_to_16384():
    # p = 65521: K = 16384 (128 k-blocks) takes exactly one unit per weight class
    segs = ffsyrk.i8_schedule(65521, 128)
    assert sum(1 for s in segs if s[4]) == 3


@pytest.mark.parametrize("p", [251, 257, 65521, 131071, 8388593, 16777213])
def test_i8_digit_products_rebuild_the_product(p):
    # Σ_{i,j} 256^{i+j}·D_i·D_jᵀ = S·Sᵀ over the integers with the byte digits
    D = len(ffsyrk.i8_digit_bounds(p))
    rng = np.random.default_rng(p + 1)
    X = rng.integers(0, p, size=(6, 9)).astype(object)
    h = (p - 1) // 2
    S = np.where(X > h, X - p, X)
    digits = np.array([[twos_bytes(int(s), D) for s in row] for row in S], dtype=object)
    Dt = [digits[:, :, t] for t in range(D)]
    exact = sum(256 ** (i + j) * Dt[i].dot(Dt[j].T) for i in range(D) for j in range(D))
    assert np.array_equal(exact, S.dot(S.T))
    weighted = sum(pow(256, i + j, p) * Dt[i].dot(Dt[j].T) for i in range(D) for j in range(D))
    assert np.array_equal(weighted % p, X.dot(X.T) % p)


# ---- Karatsuba digit products: D(D+1)/2 plane products with weights ----

KS_PRIMES = [521, 65521, 8388593, 16777213, 3, 131071, 509]


@pytest.mark.parametrize("p", KS_PRIMES)
def test_karatsuba_planes_and_bounds(p):
    bounds, weights = ffsyrk.digit_planes(p)
    dig = ffsyrk.digit_bounds(p)
    D = len(dig)
    eligible = D >= 2 and ffsyrk.digit_base(p) == 256 and all(
        dig[i] + dig[j] <= 256 for i in range(D) for j in range(i + 1, D))
    if not eligible:
        assert bounds == [] and weights == []
        return
    assert len(bounds) == D * (D + 1) // 2
    assert bounds[:D] == dig
    sums = [(i, j) for i in range(D) for j in range(i + 1, D)]
    assert bounds[D:] == [dig[i] + dig[j] for i, j in sums]
    assert max(bounds) <= 256          # every plane entry an exact bf16 integer


@pytest.mark.parametrize("p", [521, 65521, 8388593, 16777213])
def test_karatsuba_weights_rebuild_the_product(p):
    # Σ_t w_t·plane_t(X)·plane_t(Z)ᵀ ≡ X·Zᵀ (mod p) for the library's weights,
    # with the planes formed here from the balanced digits (X and Z unequal,
    # as for the general products P3, P4)
    bounds, w = ffsyrk.digit_planes(p)
    b = ffsyrk.digit_base(p)
    D = len(ffsyrk.digit_bounds(p))
    rng = np.random.default_rng(p + 7)
    h = (p - 1) // 2
    X = rng.integers(0, p, size=(5, 11)).astype(object)
    Z = rng.integers(0, p, size=(7, 11)).astype(object)

    def planes(M):
        S = np.where(M > h, M - p, M)
        dg = np.array([[balanced_digits(int(s), D, b) for s in row] for row in S], dtype=object)
        out = [dg[:, :, t] for t in range(D)]
        out += [dg[:, :, i] + dg[:, :, j] for i in range(D) for j in range(i + 1, D)]
        assert all(abs(int(v)) <= bd for P, bd in zip(out, bounds) for v in P.ravel())
        return out

    PX, PZ = planes(X), planes(Z)
    total = sum(int(wt) * PX[t].dot(PZ[t].T) for t, wt in enumerate(w))
    assert np.array_equal(total % p, X.dot(Z.T) % p)
    # the schoolbook weights are what the rearrangement starts from
    assert len(w) == D * (D + 1) // 2


@pytest.mark.parametrize("p", [521, 65521, 8388593, 16777213])
@pytest.mark.parametrize("kblocks", [1, 3, 4, 5, 16, 17, 33, 64, 513])
def test_karatsuba_schedule_units_exact_and_complete(p, kblocks):
    bounds, _ = ffsyrk.digit_planes(p)
    P = len(bounds)
    segs = ffsyrk.leaf_schedule_ks(p, kblocks)
    assert segs and segs[0][4]
    covered = {}
    unit_sum, unit_plane = 0, None
    for i, j, kb0, nkb, first in segs:
        assert i == j and 0 <= i < P
        assert nkb >= 1 and 0 <= kb0 and kb0 + nkb <= kblocks
        if first:
            unit_sum, unit_plane = 0, i
        assert i == unit_plane                      # one product (one weight) per accumulator
        unit_sum += 64 * nkb * bounds[i] * bounds[i]
        assert unit_sum <= 1 << 24                  # every FP32 partial sum exact
        for kb in range(kb0, kb0 + nkb):
            covered[(i, kb)] = covered.get((i, kb), 0) + 1
    assert set(covered) == {(t, kb) for t in range(P) for kb in range(kblocks)}
    assert all(c == 1 for c in covered.values())


def test_karatsuba_units_per_span():
    # p = 65521: per 16 k-blocks P00 and P11 one unit each, the sum plane (≤ 256) four of 4
    segs = ffsyrk.leaf_schedule_ks(65521, 16)
    assert [(s[0], s[3]) for s in segs] == [(0, 16), (1, 16), (2, 4), (2, 4), (2, 4), (2, 4)]
