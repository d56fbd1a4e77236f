"""GPU parity with Algorithm 1 (Winograd) on the general products (marked gpu).

The paper's fsyrk computes Algorithm 2's general products P3 = X22·S4ᵀ and
P4 = S1·S2ᵀ with Strassen–Winograd, one level fewer than the syrk recursion
above them (Section 4.2, the G-i variants).  Forced on (winograd = 1, 2, or
the G-i maximum) at depths 2 and 3, the result stays bit-exact against the
oracle: odd shapes, every digit scheme, both leaves and tile widths, both
triangles with the other one untouched, the α/β update, plan reuse across
shapes, and the levels the plan reports.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2001_04109_gb300 import ffsyrk, inputs
from parity_util import SENTINEL, residues

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def run(A_host, p, uplo="lower", **plan_kw):
    n, k = A_host.shape
    C = torch.full((n, n + 3), SENTINEL, dtype=torch.int32, device="cuda")
    plan = ffsyrk.Plan(p, n, k, **plan_kw)
    plan(A_host.cuda(), C[:, :n], uplo=uplo)
    plan.sync_status()
    info = plan.info()
    plan.close()
    out = C.cpu().numpy().view(np.uint32)
    want = oracle.syrk(A_host.numpy(), p, uplo)
    mask = np.tril(np.ones((n, n), bool)) if uplo == "lower" else np.triu(np.ones((n, n), bool))
    assert np.array_equal(out[:, :n][mask], want[mask]), "result differs from the oracle"
    sent = np.uint32(SENTINEL & 0xFFFFFFFF)
    assert np.all(out[:, :n][~mask] == sent) and np.all(out[:, n:] == sent), "wrote outside"
    return info


@pytest.mark.parametrize("p", [65521, 131071, 8388593, 251, 13])
@pytest.mark.parametrize("levels,sw", [(2, 1), (3, 1), (3, 2)])
def test_winograd_levels_primes(p, levels, sw):
    n, k = 531, 397
    A = residues(n, k, p, seed=levels * 10 + sw)
    info = run(A, p, levels=levels, winograd=sw)
    assert info["winograd"][: levels] == [min(sw, levels - 1 - d) for d in range(levels)]


@pytest.mark.parametrize("leaf,tile_ctas", [("tc", 1), ("tc", 2), ("i64", None)])
@pytest.mark.parametrize("uplo", ["lower", "upper"])
def test_winograd_leaves_triangles(leaf, tile_ctas, uplo):
    p = 65521
    A = inputs.arbitrary_u32(777, 300, seed=4)  # entries above p
    run(A, p, uplo=uplo, leaf=leaf, tile_ctas=tile_ctas, levels=3, winograd=2)


def test_winograd_update_and_plan_reuse():
    p = 131071
    plan = ffsyrk.Plan(p, 700, 900, levels=2, winograd=1)
    for n, k in [(700, 900), (333, 257), (64, 900), (700, 1)]:
        A = residues(n, k, p, seed=n + k)
        C0 = inputs.uniform_residues(n, n, p, seed=5).numpy().view(np.uint32)
        C = torch.from_numpy(C0.view(np.int32).copy()).cuda()
        plan(A.cuda(), C, alpha=12345, beta=p - 2)
        plan.sync_status()
        want = oracle.syrk_update(A.numpy(), p, 12345, C0, p - 2, "lower")
        assert np.array_equal(C.cpu().numpy().view(np.uint32), want), (n, k)
    plan.close()


def test_winograd_off_and_auto_small():
    # the cost model keeps Algorithm 1 off at small sizes; 0 turns it off
    p = 65521
    A = residues(600, 600, p, seed=8)
    assert run(A, p, levels=3)["winograd"][:3] == [0, 0, 0]
    assert run(A, p, levels=3, winograd=0)["winograd"][:3] == [0, 0, 0]
