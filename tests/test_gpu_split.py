"""GPU parity of the tensor-core leaf when few, long tiles are shared by CTAs.

A launch with at most half as many tiles as CTAs, each tile at least 256
k-blocks of digit-pair MMAs, has every tile's K schedule cut at unit
boundaries into equal shares taken by different CTAs; the last CTA to finish
a tile's rows adds the other shares' partial residues (marked gpu).  The
result must still equal the oracle bit for bit, for both triangles, two and
three digits per residue (and a 2×2 Y for p = 131071), one level of
Algorithm 2 (five products sharing the launch), and repeated calls (the
per-tile counters must be back at zero for the next launch).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2001_04109_gb300 import ffsyrk, inputs
from parity_util import SENTINEL, check_against_oracle, residues

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def run_timed(A_host, p, levels, uplo, calls=2):
    n, k = A_host.shape
    dev = torch.device("cuda")
    A = A_host.to(dev)
    plan = ffsyrk.Plan(p, n, k, leaf="tc", levels=levels, tile_ctas=1)  # the split is a one-SM-tile feature
    plan.set_timing(True)
    outs = []
    for _ in range(calls):
        C = torch.full((n, n), SENTINEL, dtype=torch.int32, device=dev)
        plan(A, C, uplo=uplo)
        plan.sync_status()
        outs.append(C.cpu().numpy().view(np.uint32))
    t = plan.timing()
    plan.close()
    return outs, t


@pytest.mark.parametrize("n,k,p,levels,uplo", [
    # ≥ 256 k-blocks of digit products per tile: with Karatsuba digits
    # (3 products for p = 65521, 6 for 8388593) and schoolbook (4 for 131071)
    (1000, 7000, 65521, 0, "lower"),
    (1000, 7000, 65521, 0, "upper"),
    (700, 4097, 131071, 0, "lower"),
    (300, 3000, 8388593, 0, "upper"),
    (1536, 12288, 65521, 1, "lower"),
])
def test_split_matches_oracle(n, k, p, levels, uplo):
    A = residues(n, k, p, seed=n + k + p % 97)
    outs, t = run_timed(A, p, levels, uplo)
    assert t["split_tiles"] > 0, t
    assert t["leaf_entries"] > t["leaf_tiles"], t
    for C in outs:
        check_against_oracle(A, p, C, uplo=uplo)
    assert np.array_equal(outs[0], outs[1])


def test_no_split_for_a_full_wave():
    # 272 tiles of A 4096×4096 keep every SM busy: no tile is shared
    n, k, p = 4096, 512, 65521
    A = residues(n, k, p, seed=3)
    _, t = run_timed(A, p, 0, "lower", calls=1)
    assert t["split_tiles"] == 0 and t["leaf_entries"] == t["leaf_tiles"] == 272, t


def test_no_split_for_short_tiles():
    # few tiles, but each only 4·16 = 64 k-blocks of MMAs: not worth sharing
    n, k, p = 600, 1024, 65521
    A = residues(n, k, p, seed=4)
    outs, t = run_timed(A, p, 0, "lower", calls=1)
    assert t["split_tiles"] == 0, t
    check_against_oracle(A, p, outs[0])


@pytest.mark.parametrize("n,cut", [(2560, False), (3072, True), (3584, True), (4096, False),
                                   (4608, True)])
def test_pair_tiles_balanced_last_waves(n, cut):
    # SM-pair tiles: the lower 256×256 tiles of n² leave a last wave on the
    # 76 pairs that is 3 % (3072: 78 tiles), 38 % (3584) or 25 % (4608) full,
    # so the last two waves are cut into equal shares; 2560 (55 tiles) and
    # 4096 (1.79 waves) stay whole.  The result stays exact, also for the update.
    p = 65521
    k = 1100
    A = inputs.uniform_residues(n, k, p, seed=n)
    plan = ffsyrk.Plan(p, n, k, leaf="tc", levels=0, tile_ctas=2)
    C = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    plan.set_timing(True)
    plan(A.cuda(), C)
    plan.sync_status()
    assert (plan.timing()["split_tiles"] > 0) == cut, plan.timing()
    plan.set_timing(False)
    rows = np.array(sorted({0, 1, 255, 256, 511, n // 2, n - 257, n - 256, n - 1} |
                           set(np.random.default_rng(n).integers(0, n, 24).tolist())), dtype=np.int64)
    want = oracle.syrk_rows(A.numpy(), p, rows)
    got = C[torch.from_numpy(rows).cuda()].cpu().numpy().view(np.uint32)
    for t, r in enumerate(rows):
        assert np.array_equal(got[t, : r + 1], want[t, : r + 1]), f"row {r}"
    C0 = inputs.uniform_residues(n, n, p, seed=1).cuda()
    C1 = C0.clone()
    plan(A.cuda(), C1, alpha=5, beta=7)
    plan.sync_status()
    old = C0.cpu().numpy().view(np.uint32)[rows].astype(np.uint64)
    got = C1[torch.from_numpy(rows).cuda()].cpu().numpy().view(np.uint32)
    w2 = (5 * want.astype(np.uint64) + 7 * old) % p
    for t, r in enumerate(rows):
        assert np.array_equal(got[t, : r + 1], w2[t, : r + 1].astype(np.uint32)), f"update row {r}"
    plan.close()
