"""GPU parity of C ← α·A·D·Aᵀ + β·C mod p, D diagonal (Algorithm 5) or
block diagonal (Algorithm 6; marked gpu).

The library factors Diag(d) = Δ·Δᵀ on the host (Algorithm 4 for pairs of
non-squares), forms Ā = [A 0]·Δ on the device and runs the symmetric product
of Ā.  Against the oracle's schoolbook A·D·Aᵀ combined with the update's
definition: squares only, non-squares in odd and even counts (the odd count
adds a column), zeros in d, every depth and leaf, both triangles, α/β
including the LDLᵀ-style update C − A·D·Aᵀ, k = 1, strides, the cached
entry point, and a plan whose k bound is too small.  For Algorithm 6:
every kind of 2×2 block (antidiagonal, one zero corner, full), mixed with
1×1 blocks, against the oracle's A·B·Aᵀ; overlapping blocks are rejected.
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


def is_square(x, p):
    return x % p == 0 or pow(x, (p - 1) // 2, p) == 1


def diag_values(k, p, kind, seed):
    rng = np.random.default_rng(seed)
    d = [int(x) for x in rng.integers(0, 1 << 32, size=k, dtype=np.uint64)]
    if kind == "squares":
        d = [(x * x) % p for x in d]
    elif kind in ("odd_nonsq", "even_nonsq"):
        nonsq = [x for x in range(2, p) if not is_square(x, p)][:50]
        d = [(x * x) % p for x in d]
        want = 3 if kind == "odd_nonsq" else 4
        for t in range(min(want, k)):
            d[(t * 7) % k] = nonsq[t % len(nonsq)] * (t + 1) ** 2 % p
    elif kind == "zeros":
        for t in range(0, k, 3):
            d[t] = 0
    return d


def start_matrix(n, p, uplo, seed, pad=0):
    C0 = np.full((n, n + pad), np.uint32(SENTINEL & 0xFFFFFFFF), dtype=np.uint32)
    R = inputs.uniform_residues(n, n, p, seed=seed).numpy().view(np.uint32)
    mask = np.tril(np.ones((n, n), dtype=bool)) if uplo == "lower" else np.triu(np.ones((n, n), dtype=bool))
    C0[:, :n][mask] = R[mask]
    return C0, mask


def expected(A_host, d, p, alpha, C0, beta, mask):
    P = oracle.syrkd(A_host.numpy(), np.array(d, dtype=np.uint64), p, "full").astype(np.uint64)
    want = C0.copy()
    upd = (np.uint64(alpha % p) * P + np.uint64(beta % p) * C0.astype(np.uint64)) % np.uint64(p)
    want[mask] = upd[mask].astype(np.uint32)
    return want


def run_syrkd(A_host, d, p, alpha=1, beta=0, uplo="lower", leaf=None, levels=None,
              tile_ctas=None, lda_pad=0, ldc_pad=0, seed=1, plan=None):
    n, k = A_host.shape
    Abig = torch.full((n, k + lda_pad), 5, dtype=torch.int32, device="cuda")
    Abig[:, :k] = A_host.cuda()
    C0, mask = start_matrix(n, p, uplo, seed, ldc_pad)
    Cbig = torch.from_numpy(C0.view(np.int32)).cuda()
    own = plan is None
    if own:
        plan = ffsyrk.Plan(p, n, k + 1, leaf=leaf, levels=levels, tile_ctas=tile_ctas)
    plan.syrkd(Abig[:, :k], d, Cbig[:, :n], uplo=uplo, alpha=alpha, beta=beta)
    plan.sync_status()
    if own:
        plan.close()
    out = Cbig.cpu().numpy().view(np.uint32)
    want = expected(A_host, d, p, alpha, C0[:, :n], beta, mask)
    assert np.array_equal(out[:, :n], want), "A·D·Aᵀ differs from the oracle"
    if ldc_pad:
        assert np.all(out[:, n:] == np.uint32(SENTINEL & 0xFFFFFFFF)), "wrote past the last column"


@pytest.mark.parametrize("kind", ["squares", "odd_nonsq", "even_nonsq", "zeros", "random"])
@pytest.mark.parametrize("levels", [0, 1])
def test_syrkd_kinds_of_d(kind, levels):
    p = 65521
    n, k = 300, 257
    A = residues(n, k, p, seed=21)
    run_syrkd(A, diag_values(k, p, kind, seed=levels), p, levels=levels)


@pytest.mark.parametrize("p", [131071, 8388593, 11])
@pytest.mark.parametrize("uplo", ["lower", "upper"])
def test_syrkd_primes_triangles_strides(p, uplo):
    n, k = 261, 190
    A = inputs.arbitrary_u32(n, k, seed=8)  # entries above p
    d = diag_values(k, p, "random", seed=p % 101)
    run_syrkd(A, d, p, alpha=3, beta=p + 5, uplo=uplo, levels=1, lda_pad=3, ldc_pad=1)


@pytest.mark.parametrize("leaf,tile_ctas", [("tc", 1), ("tc", 2), ("i64", None)])
def test_syrkd_leaves(leaf, tile_ctas):
    p = 65521
    n, k = 400, 333
    A = residues(n, k, p, seed=4)
    run_syrkd(A, diag_values(k, p, "odd_nonsq", seed=9), p, leaf=leaf, tile_ctas=tile_ctas,
              levels=2)


def test_syrkd_ldlt_update_and_k_one():
    # C ← C − A·D·Aᵀ (α = p − 1, β = 1), the Schur-complement step of an LDLᵀ
    p = 131071
    A = residues(350, 129, p, seed=6)
    run_syrkd(A, diag_values(129, p, "random", seed=3), p, alpha=p - 1, beta=1, levels=1)
    for dval in [0, 1, 3, p - 1]:  # 3 and p − 1 are non-squares mod 131071
        run_syrkd(residues(70, 1, p, seed=dval), [dval], p, levels=0)


def test_syrkd_plan_reuse_and_cached_entry():
    p = 65521
    n, k = 280, 150
    A = residues(n, k, p, seed=12)
    plan = ffsyrk.Plan(p, n, k + 1, levels=1)
    for t, kind in enumerate(["even_nonsq", "odd_nonsq", "squares"]):
        run_syrkd(A, diag_values(k, p, kind, seed=t), p, alpha=t + 2, beta=t, plan=plan, seed=t)
    plan.close()
    d = diag_values(k, p, "odd_nonsq", seed=77)
    C = ffsyrk.syrkd(A.cuda(), d, p)
    torch.cuda.synchronize()
    want = oracle.syrkd(A.numpy(), np.array(d, dtype=np.uint64), p, "lower")
    assert np.array_equal(C.cpu().numpy().view(np.uint32), want)


def test_syrkd_plan_k_bound_too_small():
    p = 65521
    n, k = 64, 40
    A = residues(n, k, p, seed=1).cuda()
    plan = ffsyrk.Plan(p, n, k)
    d = diag_values(k, p, "odd_nonsq", seed=1)   # needs k + 1 columns
    with pytest.raises(ffsyrk.FfsyrkError) as e:
        plan.syrkd(A, d)
    assert e.value.code == ffsyrk.ERR_TOO_LARGE
    plan.syrkd(A, diag_values(k, p, "even_nonsq", seed=1))   # k columns: fits
    plan.sync_status()
    plan.close()


def block_diag(k, p, seed):
    rng = np.random.default_rng(seed)
    d = [int(x) for x in rng.integers(0, p, size=k)]
    e = [0] * max(k - 1, 0)
    j = 0
    while j + 1 < k:
        kind = int(rng.integers(0, 5))
        if kind == 0:
            j += 1
            continue
        e[j] = int(rng.integers(1, p))
        if kind == 1:
            d[j] = d[j + 1] = 0
        elif kind == 2:
            d[j] = 0
        elif kind == 3:
            d[j + 1] = 0
        j += 2
    return d, e


def run_syrkbd(A_host, d, e, p, alpha=1, beta=0, uplo="lower", levels=None, plan=None, seed=1,
               lda_pad=0):
    n, k = A_host.shape
    Abig = torch.full((n, k + lda_pad), 3, dtype=torch.int32, device="cuda")
    Abig[:, :k] = A_host.cuda()
    C0, mask = start_matrix(n, p, uplo, seed)
    C = torch.from_numpy(C0.view(np.int32)).cuda()
    own = plan is None
    if own:
        plan = ffsyrk.Plan(p, n, k + 1, levels=levels)
    plan.syrkbd(Abig[:, :k], d, e, C, uplo=uplo, alpha=alpha, beta=beta)
    plan.sync_status()
    if own:
        plan.close()
    P = oracle.syrkbd(A_host.numpy(), np.array(d, dtype=np.uint64), np.array(e, dtype=np.uint64),
                      p, "full").astype(np.uint64)
    want = C0.copy()
    upd = (np.uint64(alpha % p) * P + np.uint64(beta % p) * C0.astype(np.uint64)) % np.uint64(p)
    want[mask] = upd[mask].astype(np.uint32)
    assert np.array_equal(C.cpu().numpy().view(np.uint32), want), "A·B·Aᵀ differs from the oracle"


@pytest.mark.parametrize("p", [65521, 131071, 8388593, 7])
@pytest.mark.parametrize("levels", [0, 1])
def test_syrkbd_block_kinds(p, levels):
    n, k = 290, 211
    A = inputs.arbitrary_u32(n, k, seed=p % 97)
    d, e = block_diag(k, p, seed=p + levels)
    run_syrkbd(A, d, e, p, levels=levels, lda_pad=levels)


def test_syrkbd_update_upper_and_all_antidiagonal():
    p = 131071
    n, k = 333, 200
    A = residues(n, k, p, seed=31)
    d, e = block_diag(k, p, seed=5)
    run_syrkbd(A, d, e, p, alpha=p - 1, beta=1, uplo="upper", levels=1)
    # B = ⊕ [[0, β], [β, 0]]: every column takes part in an antidiagonal block
    rng = np.random.default_rng(9)
    e = [int(rng.integers(1, p)) if j % 2 == 0 else 0 for j in range(k - 1)]
    run_syrkbd(A, [0] * k, e, p, alpha=5, beta=7, levels=0)


def test_syrkbd_cached_and_rejects_overlap():
    p = 65521
    n, k = 150, 97
    A = residues(n, k, p, seed=2)
    d, e = block_diag(k, p, seed=3)
    C = ffsyrk.syrkbd(A.cuda(), d, e, p)
    torch.cuda.synchronize()
    want = oracle.syrkbd(A.numpy(), np.array(d, dtype=np.uint64), np.array(e, dtype=np.uint64), p,
                         "lower")
    assert np.array_equal(C.cpu().numpy().view(np.uint32), want)
    bad = list(e)
    bad[10] = bad[11] = 1
    plan = ffsyrk.Plan(p, n, k + 1)
    with pytest.raises(ffsyrk.FfsyrkError) as err:
        plan.syrkbd(A.cuda(), d, bad)
    assert err.value.code == ffsyrk.ERR_INVALID_ARG
    plan.close()


@pytest.mark.parametrize("p", [7, 11, 13, 97, 40961, 65521, 65537, 131071, 8388593])
def test_device_planner_matches_host_planner(p):
    # the device planner picks the same roots, pairs and term order as the
    # host's: the whole table W agrees entry for entry
    for seed in range(4):
        for k in [1, 2, 5, 64, 257, 1000]:
            d, e = block_diag(k, p, seed=seed * 7919 + k)
            if seed == 3:
                e = None
            assert ffsyrk.syrkbd_factor_device(p, d, e) == ffsyrk.syrkbd_factor(p, d, e), (p, seed, k)
