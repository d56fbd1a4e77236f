"""GPU parity of the Hermitian product over F_{p²} (Section 3.2; marked gpu).

C = A·Aᴴ with A ∈ F_{p²}^{n×k}, F_{p²} = F_p[i]/(i² − r), against the
oracle's definition: i² = −1 (p ≡ 3 mod 4, where Re C is a plain symmetric
product), another non-square r with −r a square (p ≡ 3 mod 4), and p ≡ 1
mod 4 (−r a non-square: the diagonal scaling pairs non-squares); odd
shapes, both triangles with the other one untouched, recursion depths and
both leaves for the real part, k = 0, the cached entry point, and a square r
rejected.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2001_04109_gb300 import ffsyrk, inputs
from parity_util import SENTINEL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def nonsquares(p):
    return [x for x in range(2, 200) if pow(x, (p - 1) // 2, p) == p - 1]


def check(A, p, r, uplo, Cre, Cim, n):
    want_re, want_im = oracle.herk(A.numpy(), p, r, uplo)
    mask = np.tril(np.ones((n, n), bool)) if uplo == "lower" else np.triu(np.ones((n, n), bool))
    sent = np.uint32(SENTINEL & 0xFFFFFFFF)
    for got, want, name in [(Cre, want_re, "Re"), (Cim, want_im, "Im")]:
        g = got.cpu().numpy().view(np.uint32)
        assert np.array_equal(g[:, :n][mask], want[mask]), f"{name} C differs from the oracle"
        assert np.all(g[:, :n][~mask] == sent) and np.all(g[:, n:] == sent), f"{name}: wrote outside"


def run(p, r, n, k, uplo="lower", seed=1, **kw):
    A = inputs.arbitrary_u32(n, 2 * k, seed=seed)
    Cre = torch.full((n, n + 2), SENTINEL, dtype=torch.int32, device="cuda")
    Cim = torch.full((n, n + 2), SENTINEL, dtype=torch.int32, device="cuda")
    plan = ffsyrk.HerkPlan(p, r, n, k, **kw)
    plan(A.cuda(), Cre[:, :n], Cim[:, :n], uplo=uplo)
    plan.sync_status()
    plan.close()
    check(A, p, r, uplo, Cre, Cim, n)


@pytest.mark.parametrize("p,r", [(131071, 131070), (131071, 3), (65521, None), (8388593, None),
                                 (251, None), (7, 6)])
@pytest.mark.parametrize("uplo", ["lower", "upper"])
def test_herk_fields_triangles(p, r, uplo):
    if r is None:
        r = nonsquares(p)[0]
    run(p, r, 301, 157, uplo=uplo, seed=p % 17)


@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("leaf", ["tc", "i64"])
def test_herk_depths_leaves(levels, leaf):
    p = 65521
    run(p, nonsquares(p)[1], 520, 300, levels=levels, leaf=leaf, seed=levels)
    run(131071, 131070, 333, 129, levels=levels, leaf=leaf, seed=levels + 5)


def test_herk_k_zero_cached_and_bad_r():
    p = 131071
    run(p, p - 1, 40, 0)
    A = inputs.uniform_residues(200, 2 * 90, p, seed=3)
    Cre, Cim = ffsyrk.herk(A.cuda(), p, p - 1)
    torch.cuda.synchronize()
    want_re, want_im = oracle.herk(A.numpy(), p, p - 1, "lower")
    assert np.array_equal(Cre.cpu().numpy().view(np.uint32), want_re)
    assert np.array_equal(Cim.cpu().numpy().view(np.uint32), want_im)
    with pytest.raises(ffsyrk.FfsyrkError) as e:
        ffsyrk.HerkPlan(65521, 4, 10, 10)   # 4 is a square
    assert e.value.code == ffsyrk.ERR_INVALID_ARG
