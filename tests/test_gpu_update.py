"""GPU parity of the update C ← α·A·Aᵀ + β·C mod p (marked gpu).

Section 4.2, Table 4 of the paper gives the schedule for the general update;
the library applies α and β where C is written (the leaf epilogue for the
classical path, the root post-addition otherwise).  Against the oracle's
definition: every depth, both tensor-core tile widths and the int64 leaf,
both triangles with the other one untouched, odd strides, α = 0, k = 0,
shared tiles, repeated calls with new (α, β) on one plan, the cached entry.
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


def start_matrix(n, p, uplo, seed, pad=0):
    """C0: residues < p on the triangle, SENTINEL elsewhere (and in guard columns)."""
    C0 = np.full((n, n + pad), np.uint32(SENTINEL & 0xFFFFFFFF), dtype=np.uint32)
    R = inputs.uniform_residues(n, n, p, seed=seed).numpy().view(np.uint32)
    mask = np.tril(np.ones((n, n), dtype=bool)) if uplo == "lower" else np.triu(np.ones((n, n), dtype=bool))
    C0[:, :n][mask] = R[mask]
    return C0


def run_update(A_host, p, alpha, beta, uplo="lower", leaf=None, levels=None, tile_ctas=None,
               lda_pad=0, ldc_pad=0, seed=1, plan=None):
    n, k = A_host.shape
    Abig = torch.full((n, k + lda_pad), 7, dtype=torch.int32, device="cuda")
    Abig[:, :k] = A_host.cuda()
    C0 = start_matrix(n, p, uplo, seed, ldc_pad)
    Cbig = torch.from_numpy(C0.view(np.int32)).cuda()
    own = plan is None
    if own:
        plan = ffsyrk.Plan(p, max(n, 1), max(k, 1), leaf=leaf, levels=levels, tile_ctas=tile_ctas)
    plan(Abig[:, :k], Cbig[:, :n], uplo=uplo, alpha=alpha, beta=beta)
    plan.sync_status()
    if own:
        plan.close()
    out = Cbig.cpu().numpy().view(np.uint32)
    want = oracle.syrk_update(A_host.numpy(), p, alpha, C0[:, :n], beta, uplo)
    assert np.array_equal(out[:, :n], want), "update differs from the oracle"
    if ldc_pad:
        assert np.all(out[:, n:] == np.uint32(SENTINEL & 0xFFFFFFFF)), "wrote past the last column"


@pytest.mark.parametrize("leaf,tile_ctas", [("tc", 1), ("tc", 2), ("i64", None)])
@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("uplo", ["lower", "upper"])
def test_update_depths_leaves_triangles(leaf, tile_ctas, levels, uplo):
    p = 65521
    n, k = 517, 389
    A = residues(n, k, p, seed=levels + 10)
    run_update(A, p, alpha=12345, beta=54321, uplo=uplo, leaf=leaf, levels=levels,
               tile_ctas=tile_ctas, seed=levels)


@pytest.mark.parametrize("p", [131071, 8388593, 251])
def test_update_primes_strides_large_inputs(p):
    n, k = 333, 270
    A = inputs.arbitrary_u32(n, k, seed=5)  # entries above p
    run_update(A, p, alpha=(1 << 32) - 3, beta=p + 2, uplo="lower", levels=1, lda_pad=3, ldc_pad=5)
    run_update(A, p, alpha=7, beta=p - 1, uplo="upper", levels=0, lda_pad=1, ldc_pad=3)


def test_update_alpha_zero_and_k_zero():
    p = 65521
    A = residues(200, 100, p, seed=3)
    run_update(A, p, alpha=0, beta=9, levels=0)
    run_update(A, p, alpha=0, beta=9, levels=1)
    run_update(residues(200, 0, p, seed=4), p, alpha=5, beta=9)   # k = 0: C ← β·C


def test_update_on_shared_tiles_and_repeated_calls():
    # few, long tiles (K shared among CTAs), then new (α, β) on the same plan
    p = 65521
    n, k = 1000, 5000
    A = residues(n, k, p, seed=6)
    plan = ffsyrk.Plan(p, n, k, leaf="tc", levels=0, tile_ctas=1)
    for alpha, beta in [(3, 4), (1, 0), (65520, 1), (2, 0)]:
        run_update(A, p, alpha, beta, plan=plan, seed=alpha)
    plan.close()


def test_cached_update_entry_point():
    p = 131071
    n, k = 300, 301
    A = residues(n, k, p, seed=2)
    C0 = start_matrix(n, p, "lower", 11)
    C = torch.from_numpy(C0.view(np.int32)).cuda()
    ffsyrk.syrk(A.cuda(), p, C=C, alpha=77, beta=88)
    torch.cuda.synchronize()
    want = oracle.syrk_update(A.numpy(), p, 77, C0, 88, "lower")
    assert np.array_equal(C.cpu().numpy().view(np.uint32), want)


def test_update_full_size_sampled_rows():
    # A 4096×4096 in the benchmark's launch configuration (SM-pair tiles)
    p, n, k = 65521, 4096, 4096
    A = inputs.uniform_residues(n, k, p, seed=2, device="cuda")
    C0 = inputs.uniform_residues(n, n, p, seed=3, device="cuda")
    C = C0.clone()
    plan = ffsyrk.Plan(p, n, k)
    plan(A, C, alpha=31337, beta=4242)
    plan.sync_status()
    plan.close()
    rows = np.array([0, 1, 255, 256, 2047, 4094, 4095], dtype=np.int64)
    prod = oracle.syrk_rows(A.cpu().numpy(), p, rows).astype(np.uint64)
    old = C0.cpu().numpy().view(np.uint32)[rows].astype(np.uint64)
    want = (31337 * prod + 4242 * old) % p
    got = C.cpu().numpy().view(np.uint32)[rows]
    for t, r in enumerate(rows):
        assert np.array_equal(got[t, : r + 1], want[t, : r + 1].astype(np.uint32)), f"row {r}"
        assert np.array_equal(got[t, r + 1:], old[t, r + 1:].astype(np.uint32)), f"row {r} upper"
