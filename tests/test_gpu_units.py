"""Accumulator units from the operands' digits (marked gpu).

With unit_bounds "data" (the default) a pass before the tensor-core leaf
bounds each unit's partial sums by Cauchy–Schwarz on the digit planes' row
sums of squares and merges the worst-case schedule's units where that bound
stays ≤ 2^24.  These tests check that the result stays bit-exact against the
oracle on inputs where merging happens (uniform residues), where it must not
(every digit at its bound, with perturbations so that an FP32 sum past 2^24
would lose low bits), and where it may happen over only part of K; and that
the unit counts move the way the bound says.  Sizes where the counts are
asserted have enough output tiles that no tile is cut into pieces (a piece
starts a unit, whatever its bound).
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


def run(A_host, p, levels, unit_bounds=None, digit_products=None, tile_ctas=None):
    n, k = A_host.shape
    A = A_host.cuda()
    C = torch.full((n, n), SENTINEL, dtype=torch.int32, device="cuda")
    plan = ffsyrk.Plan(p, n, k, leaf="tc", levels=levels, unit_bounds=unit_bounds,
                       digit_products=digit_products, tile_ctas=tile_ctas)
    plan(A, C)
    plan.sync_status()
    units = plan.units()
    plan.close()
    return C.cpu().numpy().view(np.uint32), units


# the symmetric residue whose byte digits all sit at their bounds for p = 8388593:
# (−128, −128, 64), so the digit-sum plane X0 + X1 is −256 everywhere
S_BOUND = 4161408


def bound_matrix(n, k, p, seed):
    """Every digit at its bound, except a sparse set of entries one less in magnitude
    (odd sums: an FP32 accumulation past 2^24 would round them)."""
    rng = np.random.default_rng(seed)
    s = np.full((n, k), S_BOUND, dtype=np.int64)
    s[rng.random((n, k)) < 0.05] -= 1
    s *= np.where(rng.random((n, 1)) < 0.5, 1, -1)  # row signs
    return torch.from_numpy((s % p).astype(np.int32))


@pytest.mark.parametrize("p", [8388593, 65521, 131071])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_uniform_residues_exact_and_merged(p, levels):
    n, k = 2560 + 96, 2048 + 192
    A = residues(n, k, p, seed=levels + p % 97)
    C, (host_units, units) = run(A, p, levels)
    check_against_oracle(A, p, C)
    assert units <= host_units
    if p != 131071:  # byte digits with Karatsuba sum planes: the digit sums merge
        assert units < host_units


@pytest.mark.parametrize("levels", [0, 1])
def test_digits_at_their_bounds_stay_exact(levels):
    p = 8388593
    n, k = 640, 8192 + 64
    A = bound_matrix(n, k, p, seed=3)
    C, (host_units, units) = run(A, p, levels)
    check_against_oracle(A, p, C)
    if levels == 0:
        # every row block near its largest sum of squares: nothing to merge
        assert units == host_units


def test_bound_digits_over_half_of_k():
    """Digits at their bounds in the first half of K, uniform residues after: units
    merge in the second half only, and the result stays exact."""
    p = 8388593
    n, k = 2560, 8192
    A = bound_matrix(n, k, p, seed=5)
    A[:, k // 2:] = residues(n, k - k // 2, p, seed=6)
    C, (host_units, units) = run(A, p, 0)
    check_against_oracle(A, p, C)
    assert units < host_units


@pytest.mark.parametrize("digit_products", ["schoolbook", "karatsuba"])
@pytest.mark.parametrize("tile_ctas", [1, 2])
def test_schoolbook_and_pairs(digit_products, tile_ctas):
    p = 8388593
    n, k = 1500, 3000
    A = residues(n, k, p, seed=11)
    C, (host_units, units) = run(A, p, 1, digit_products=digit_products, tile_ctas=tile_ctas)
    check_against_oracle(A, p, C)
    assert units <= host_units


def test_worst_case_option_keeps_the_host_schedule():
    p = 8388593
    A = residues(700, 2048, p, seed=13)
    C, (host_units, units) = run(A, p, 1, unit_bounds="worst")
    check_against_oracle(A, p, C)
    assert units == host_units


def test_replay_follows_new_data():
    """A plan replays its captured launches for a repeated call; the unit pass runs
    in every call, so new operands in the same buffer get their own units."""
    p = 8388593
    n, k = 2560, 2048
    A1 = residues(n, k, p, seed=21)
    A2 = bound_matrix(n, k, p, seed=22)
    A = A1.cuda()
    C = torch.full((n, n), SENTINEL, dtype=torch.int32, device="cuda")
    plan = ffsyrk.Plan(p, n, k, leaf="tc", levels=0)
    for _ in range(2):
        plan(A, C)
    h1, u1 = plan.units()
    check_against_oracle(A1, p, C.cpu().numpy().view(np.uint32))
    A.copy_(A2.cuda())
    plan(A, C)
    h2, u2 = plan.units()
    check_against_oracle(A2, p, C.cpu().numpy().view(np.uint32))
    plan.close()
    assert u1 < h1 and u2 == h2
