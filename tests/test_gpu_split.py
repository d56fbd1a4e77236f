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

from paper_2001_04109_gb300 import ffsyrk
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
    (1000, 5000, 65521, 0, "lower"),
    (1000, 5000, 65521, 0, "upper"),
    (700, 4097, 131071, 0, "lower"),
    (300, 3000, 8388593, 0, "upper"),
    (1536, 8192, 65521, 1, "lower"),
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
