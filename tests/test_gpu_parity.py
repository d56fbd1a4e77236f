"""GPU parity: the CUDA path against the CPU oracle, bit-exactly (marked gpu).

Sizes span several tiles of each leaf (64×64 for the int64 leaf, 128×256 for
the tensor-core leaf, 128×128 for the INT8 leaf) with ragged tails; every recursion depth used in
practice; the three Y forms (scalar, a = 1 / b = √−2, Algorithm 3); inputs
above p; odd strides; both triangles; the degenerate n = 0, n = 1, k = 0.
"""
import numpy as np
import pytest
import torch

from paper_2001_04109_gb300 import ffsyrk, inputs
from parity_util import SENTINEL, check_against_oracle, gpu_syrk, residues

pytestmark = pytest.mark.gpu

PRIMES = [65521, 131071, 8388593, 16777213, 131041, 3, 11, 251]
LEAVES = ["i64", "tc", "i8"]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("leaf", LEAVES)
@pytest.mark.parametrize("levels", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (7, 9), (64, 64), (65, 63), (130, 257),
                                   (300, 301), (513, 250)])
def test_parity_shapes_levels(leaf, levels, shape):
    n, k = shape
    p = 65521
    A = residues(n, k, p, seed=n * 1000 + k)
    C, info = gpu_syrk(A, p, leaf=leaf, levels=levels)
    assert info["levels"] == levels
    check_against_oracle(A, p, C)


@pytest.mark.parametrize("leaf", LEAVES)
@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_parity_primes(leaf, p, levels):
    n, k = 389, 517
    A = residues(n, k, p, seed=p % 1000 + levels)
    C, info = gpu_syrk(A, p, leaf=leaf, levels=levels)
    check_against_oracle(A, p, C)


@pytest.mark.parametrize("leaf", LEAVES)
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_upper_strides_and_large_inputs(leaf, levels):
    p = 131071
    n, k = 333, 270
    A = inputs.arbitrary_u32(n, k, seed=5)  # entries far above p
    C, _ = gpu_syrk(A, p, leaf=leaf, levels=levels, uplo="upper", lda_pad=3, ldc_pad=5)
    check_against_oracle(A, p, C, uplo="upper")
    C, _ = gpu_syrk(A, p, leaf=leaf, levels=levels, uplo="lower", lda_pad=1, ldc_pad=1)
    check_against_oracle(A, p, C, uplo="lower")


@pytest.mark.parametrize("leaf", LEAVES)
def test_degenerate_sizes(leaf):
    p = 65521
    # k = 0: the selected triangle becomes zero, the rest is untouched
    dev = torch.device("cuda")
    for uplo in ["lower", "upper"]:
        C = torch.full((5, 5), SENTINEL, dtype=torch.int32, device=dev)
        A = torch.zeros((5, 0), dtype=torch.int32, device=dev)
        plan = ffsyrk.Plan(p, 5, 1, leaf=leaf, levels=1)
        plan(A, C, uplo=uplo)
        plan.sync_status()
        c = C.cpu().numpy()
        tri = np.tril(np.ones((5, 5), bool)) if uplo == "lower" else np.triu(np.ones((5, 5), bool))
        assert np.all(c[tri] == 0) and np.all(c[~tri] == SENTINEL)
        plan.close()
    # n = 0 is a no-op
    plan = ffsyrk.Plan(p, 4, 4, leaf=leaf)
    plan(torch.zeros((0, 4), dtype=torch.int32, device=dev), torch.zeros((0, 0), dtype=torch.int32, device=dev))
    plan.sync_status()
    plan.close()


@pytest.mark.parametrize("leaf", LEAVES)
def test_plan_reuse_across_shapes(leaf):
    p = 8388593
    plan = ffsyrk.Plan(p, 400, 300, leaf=leaf, levels=2)
    for n, k in [(400, 300), (17, 5), (399, 299), (256, 128), (400, 300)]:
        A = residues(n, k, p, seed=n + k)
        C = torch.full((n, n), SENTINEL, dtype=torch.int32, device="cuda")
        plan(A.cuda(), C)
        plan.sync_status()
        check_against_oracle(A, p, C.cpu().numpy().view(np.uint32))
    with pytest.raises(ffsyrk.FfsyrkError):
        plan(residues(401, 3, p, 1).cuda())
    plan.close()


def test_cached_entry_point_default_options():
    p = 65521
    A = residues(700, 600, p, seed=3)
    C = torch.full((700, 700), SENTINEL, dtype=torch.int32, device="cuda")
    ffsyrk.syrk(A.cuda(), p, C=C)
    torch.cuda.synchronize()
    check_against_oracle(A, p, C.cpu().numpy().view(np.uint32))


def test_y_choice_is_skew_orthogonal():
    for p in PRIMES:
        plan = ffsyrk.Plan(p, 8, 8, leaf="i64", levels=1)
        info = plan.info()
        plan.close()
        a, b = info["y_a"], info["y_b"]
        if p % 4 == 1:
            assert info["y_form"] == 0 and a * a % p == p - 1
        else:
            assert info["y_form"] == 1 and (a * a + b * b) % p == p - 1
            assert info["y_cost"] == (2 if p % 8 == 3 else 3)


def test_workspace_query_matches_plans():
    for p, n, k, kw in [(65521, 4096, 4096, {}), (131071, 3000, 5000, {"levels": 2}),
                        (8388593, 2048, 2048, {"levels": 3, "winograd": 2})]:
        plan = ffsyrk.Plan(p, n, k, **kw)
        assert plan.info()["workspace_bytes"] == ffsyrk.workspace_query(p, n, k, **kw)[0]
        plan.close()
