"""The primes where the digit scheme changes, against the oracle (marked gpu).

509 is the last prime with one digit (|digit| ≤ 254, chunks of 4 k-blocks),
521 the first with two (digit bounds 128 and 1), 131321 the last with two
balanced base-362 digits and 131357 the first with three (bounds 128, 128,
1).  Each runs at depths 0–2 on both leaves with a ragged K, on forced
SM-pair tiles, and with every entry at the residue whose digits all sit at
their bounds, so that every K-chunk sum of the depth-0 product reaches its
exactness limit.
"""
import numpy as np
import pytest
import torch

from parity_util import check_against_oracle, gpu_syrk, residues

pytestmark = pytest.mark.gpu

# (p, symmetric residue whose digits all sit at their bounds)
EDGES = [(509, 254), (521, 128), (131321, 65341), (131357, 32640)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("leaf", ["i64", "tc"])
@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("p", [p for p, _ in EDGES])
def test_edge_primes(p, levels, leaf):
    A = residues(389, 1100, p, seed=p % 977 + levels)
    C, info = gpu_syrk(A, p, leaf=leaf, levels=levels)
    check_against_oracle(A, p, C)


@pytest.mark.parametrize("levels", [0, 1])
@pytest.mark.parametrize("p", [p for p, _ in EDGES])
def test_edge_primes_pair_tiles(p, levels):
    A = residues(511, 1030, p, seed=p % 991)
    C, _ = gpu_syrk(A, p, leaf="tc", levels=levels, tile_ctas=2)
    check_against_oracle(A, p, C)


@pytest.mark.parametrize("p,s", EDGES)
def test_edge_primes_at_digit_bounds(p, s):
    n, k = 300, 4096 + 64
    C, _ = gpu_syrk(torch.full((n, k), s % p, dtype=torch.int32), p, leaf="tc", levels=0)
    check_against_oracle(torch.full((n, k), s % p, dtype=torch.int32), p, C)
    sign = np.where((np.arange(n)[:, None] + np.arange(k)[None, :]) % 2 == 0, 1, -1)
    B = torch.from_numpy(((sign * s) % p).astype(np.int32))
    C, _ = gpu_syrk(B, p, leaf="tc", levels=1)
    check_against_oracle(B, p, C)
