"""Pins of the oracle's field helpers, Algorithm 2 and cost model (CPU only).

* Y: Y·Yᵀ ≡ −I (Definition, Section 3.1), i² ≡ −1 (Prop. 3.2),
  a² + b² ≡ −1 (Prop. 3.3, Algorithm 3), −2 a square when p ≡ 3 mod 8
  (proof of Thm 4.1).
* Algorithm 2: the identities of the proof of Prop. 3.1 (Appendix A.1) on
  random blocks, and the end-to-end result against the schoolbook oracle.
  Planted mistakes (no mirror, a wrong sign, a Y that is not
  skew-orthogonal) must break the result.
* Costs: every entry of Table 5 (tests/golden/table5_opcounts.txt) and
  the 0.8·n³ leading term of Table 1.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import alg2, cost, field, winograd
from paper_2001_04109_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CONFIG_PRIMES = [65521, 131071, 8388593, 131041]


def sieve(n):
    s = np.ones(n + 1, dtype=bool)
    s[:2] = False
    for q in range(2, int(n ** 0.5) + 1):
        if s[q]:
            s[q * q::q] = False
    return s


def test_is_prime_against_sieve():
    s = sieve(100000)
    for x in range(100001):
        assert field.is_prime(x) == bool(s[x]), x
    for p in CONFIG_PRIMES:
        assert field.is_prime(p)
    assert not field.is_prime(65521 * 65537)


def test_legendre_and_sqrt_against_brute_force():
    for p in [q for q in range(3, 400) if field.is_prime(q)]:
        squares = {x * x % p for x in range(1, p)}
        for a in range(1, p):
            assert (field.legendre(a, p) == 1) == (a in squares)
            if a in squares:
                r = field.sqrt_mod(a, p)
                assert r * r % p == a


def test_sqrt_minus_one_exists_iff_p_1_mod_4():
    for p in [q for q in range(3, 20000) if field.is_prime(q)]:
        assert (field.legendre(p - 1, p) == 1) == (p % 4 == 1)
        if p % 4 == 1:
            i = field.sqrt_minus_one(p)
            assert i * i % p == p - 1
        else:
            with pytest.raises(ValueError):
                field.sqrt_minus_one(p)


def test_config_prime_classes_and_roots():
    assert 65521 % 4 == 1 and 8388593 % 4 == 1 and 131041 % 4 == 1
    assert 131071 % 8 == 7
    for p in [65521, 8388593, 131041]:
        i = field.y_params(p)["i"]
        assert i * i % p == p - 1
    # values checked independently of the oracle's own routine
    assert 24297 ** 2 % 65521 == 65520
    prm = field.y_params(131071)
    assert prm["form"] == "2x2" and prm["y"] == 3
    assert (prm["a"] ** 2 + prm["b"] ** 2) % 131071 == 131070


def test_sos_algorithm3_all_targets():
    for p in [q for q in range(3, 300) if field.is_prime(q)]:
        for k in range(p):
            a, b = field.sos(p, k)
            assert (a * a + b * b) % p == k
    for p in [q for q in range(3, 30000) if field.is_prime(q)] + CONFIG_PRIMES:
        a, b = field.sos(p, -1)
        assert (a * a + b * b) % p == p - 1


def test_minus_two_square_when_p_3_mod_8():
    for p in [q for q in range(3, 30000) if field.is_prime(q)]:
        if p % 8 == 3:
            assert field.legendre(p - 2, p) == 1
            prm = field.y_params(p)
            assert prm["a"] == 1 and (1 + prm["b"] ** 2) % p == p - 1 and prm["y"] == 2


def _yyt(Y, p):
    Y = np.array(Y, dtype=object)
    return Y.dot(Y.T) % p


@pytest.mark.parametrize("p", [5, 7, 11, 13, 19, 23, 65521, 131071, 8388593])
@pytest.mark.parametrize("layout", ["interleaved", "block"])
def test_y_skew_orthogonal(p, layout):
    for w in [2, 4, 6, 8]:
        Y = field.y_matrix(p, w, layout=layout)
        assert np.array_equal(_yyt(Y, p), (p - 1) * np.eye(w, dtype=object) % p)


def _rand(n, k, p, seed):
    return inputs.uniform_residues(n, k, p, seed).numpy().astype(object)


@pytest.mark.parametrize("p", [65521, 131071, 19, 11])
def test_appendix_identities(p):
    """The equations of the proof of Prop. 3.1 on random blocks."""
    A = _rand(12, 16, p, seed=p)
    w = 8
    Y = alg2.skew_y(p, w)

    def full(X):  # a recursive product returned in full, for the identities
        return X.dot(X.T) % p

    st = alg2.step(A, p, Y, full)
    A11, A12, A21, A22 = A[:6, :8], A[:6, 8:], A[6:, :8], A[6:, 8:]
    C = A.dot(A.T) % p
    T = lambda X: X.T
    eq = lambda X, Yv: np.array_equal(X % p, Yv % p)
    S1, S2, P4 = st["S1"], st["S2"], st["P4"]
    R1 = A11.dot(Y).dot(T(S2))
    R2 = A21.dot(Y).dot(T(A22))
    assert eq(st["P1"] + st["P2"], C[:6, :6])                       # U3 = C11
    assert eq(st["P1"] + st["P5"], S2.dot(T(S2)) + R1 + T(R1))       # U1
    assert eq(S2.dot(T(S2)), A22.dot(T(A22)) - A21.dot(T(A21)) - R2 - T(R2))
    assert eq(R1 + P4, R2 + A21.dot(T(A21)))
    assert eq(st["U1"] + P4 + T(P4), C[6:, 6:])                      # U5 = C22
    assert eq(st["U4"], C[6:, :6])                                   # U4 = C21
    assert eq(st["U3"], alg2.low(C[:6, :6]))                        # Low(U3)
    for name in ["P1", "P2", "P5", "U1"]:
        assert eq(st[name], T(st[name])), name


@pytest.mark.parametrize("p", [65521, 131071, 8388593, 13, 7, 3])
@pytest.mark.parametrize("shape", [(8, 8), (16, 8), (8, 16), (12, 20), (7, 9), (15, 17), (5, 3), (9, 1), (1, 6)])
def test_alg2_matches_oracle(p, shape):
    n, k = shape
    A = inputs.uniform_residues(n, k, p, seed=n * 31 + k).numpy().view(np.uint32)
    want = oracle.syrk(A, p, "lower")
    for levels in [1, 2, 3]:
        got = alg2.syrk(A.astype(object), p, levels)
        assert np.array_equal(got.astype(np.uint32), want), (p, shape, levels)
    got = alg2.syrk(A.astype(object), p, 2, layout="block")
    assert np.array_equal(got.astype(np.uint32), want)


@pytest.mark.parametrize("levels", [1, 2])
def test_classical_dc_matches_oracle(levels):
    p = 65521
    A = inputs.uniform_residues(10, 14, p, seed=3).numpy().view(np.uint32)
    got = alg2.classical_dc(A.astype(object), p, levels)
    assert np.array_equal(got.astype(np.uint32), oracle.syrk(A, p, "lower"))


def test_planted_mistakes_are_caught():
    p = 65521
    A = inputs.uniform_residues(16, 16, p, seed=9).numpy().view(np.uint32)
    want = oracle.syrk(A, p, "lower")
    # the mirror Up(U1) = Low(U1)ᵀ is mandatory
    bad = alg2.syrk(A.astype(object), p, 1, mirror=False)
    assert not np.array_equal(bad.astype(np.uint32), want)
    # a Y that is not skew-orthogonal (Y = I) breaks the identities
    bad = alg2.syrk(A.astype(object), p, 1, params={"form": "scalar", "i": 1, "y": 1})
    assert not np.array_equal(bad.astype(np.uint32), want)
    # a sign error in S2 = A22 − A21·Y
    Ao = A.astype(object)
    h, w = 8, 8
    Y = alg2.skew_y(p, w)

    def rec(X):
        return alg2.classical_syrk(X, p)

    st = alg2.step(Ao, p, Y, rec)
    S2_wrong = (Ao[h:, w:] + Ao[h:, :w].dot(Y)) % p
    assert not np.array_equal(S2_wrong, st["S2"])
    P4_wrong = st["S1"].dot(S2_wrong.T) % p
    U2 = (st["U1"] + P4_wrong) % p
    assert not np.array_equal((U2 + st["P3"]) % p, (Ao.dot(Ao.T) % p)[h:, :h])


@pytest.mark.parametrize("p", [65521, 8388593, 7, 3])
@pytest.mark.parametrize("shape", [(2, 2, 2), (4, 6, 8), (8, 4, 2), (10, 12, 6)])
def test_winograd_step_is_the_product(p, shape):
    # Algorithm 1 on even-sized blocks reaches A·B exactly, block by block
    m, k, n = shape
    rng = np.random.default_rng(m * 100 + k * 10 + n)
    A = rng.integers(0, p, size=(m, k)).astype(object)
    B = rng.integers(0, p, size=(k, n)).astype(object)
    st = winograd.step(A, B, p, lambda X, Z: X.dot(Z) % p)
    h, w, v = m // 2, k // 2, n // 2
    AB = A.dot(B) % p
    assert np.array_equal(st["C"], AB)
    # the block identities behind the post-additions
    assert np.array_equal(st["c3"], (A[:h, :w].dot(B[:w, :v]) + A[:h, w:].dot(B[w:, :v])) % p)
    assert np.array_equal(st["c5"], AB[h:, v:])
    # 8 pre-additions and 7 post-additions: 15 in all, 7 products
    assert len([x for x in st if x[0] in "st"]) == 8 and len([x for x in st if x[0] == "c"]) == 7
    assert len([x for x in st if x[0] == "p"]) == 7


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_winograd_recursive_product(levels):
    p = 131071
    rng = np.random.default_rng(levels)
    for m, k, n in [(16, 16, 16), (12, 20, 8), (7, 9, 5), (1, 4, 3)]:
        A = rng.integers(0, p, size=(m, k)).astype(object)
        B = rng.integers(0, p, size=(k, n)).astype(object)
        assert np.array_equal(winograd.product(A, B, p, levels), A.dot(B) % p)


def test_winograd_planted_sign_error_is_caught():
    p = 65521
    rng = np.random.default_rng(4)
    A = rng.integers(0, p, size=(8, 8)).astype(object)
    B = rng.integers(0, p, size=(8, 8)).astype(object)
    st = winograd.step(A, B, p, lambda X, Z: X.dot(Z) % p)
    # t4 = b21 + t3 (wrong sign) changes p3, hence c4 = C21
    t4_bad = (B[4:, :4] + st["t3"]) % p
    c4_bad = (st["c2"] + A[4:, 4:].dot(t4_bad)) % p
    assert not np.array_equal(c4_bad, (A.dot(B) % p)[4:, :4])


@pytest.mark.parametrize("p", [65521, 131071, 13])
@pytest.mark.parametrize("shape", [(16, 16), (24, 40), (13, 11), (32, 8)])
def test_alg2_with_winograd_general_products(p, shape):
    # the G-i variants: levels of Algorithm 2, Algorithm 1 one level less
    n, k = shape
    A = inputs.uniform_residues(n, k, p, seed=n + 7 * k).numpy().view(np.uint32)
    want = oracle.syrk(A, p, "lower")
    for levels in [2, 3]:
        for sw in [1, 2]:
            got = alg2.syrk(A.astype(object), p, levels, winograd=sw)
            assert np.array_equal(got.astype(np.uint32), want), (p, shape, levels, sw)


def _table5():
    rows = []
    with open(os.path.join(GOLDEN, "table5_opcounts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows.append((int(parts[0]), parts[1], parts[2:]))
    return rows


def test_table5_every_entry():
    ns = [4, 8, 16, 32, 64, 128]
    checked = 0
    for grp, name, vals in _table5():
        for n, v in zip(ns, vals):
            if v == "-":
                continue
            if name == "SYRK":
                got = cost.syrk_classical(n)
            elif name == "Syrk":
                got = cost.syrk_dc(n, grp)
            else:
                got = cost.g(n, grp, int(name[1]))
            assert got == int(v), (grp, name, n, got, v)
            checked += 1
    assert checked == 99  # every printed cell of Table 5


def test_table1_leading_terms():
    n = 1 << 22
    for y in [1, 2, 3]:
        r = float(cost.g_classical(n, 22, y)) / n ** 3
        assert abs(r - 0.8) < 1e-5
    assert abs(cost.syrk_classical(n) / n ** 3 - 1.0) < 1e-6
    # field multiply-adds, one level: 3/8·(1/2) + 2/8 = 7/16 of n³
    n = 1 << 12
    assert abs(cost.field_macs_fast(n, n, 1) / n ** 3 - 7 / 16) < 1e-3
    assert abs(cost.field_macs_fast(n, n, 8) / n ** 3 - 0.4) < 2e-3
