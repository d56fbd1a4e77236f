"""INT8 leaf (mma.sync u8/s8 → s32): tiles, exactness at the int32 unit bound (marked gpu).

The INT8 leaf splits a residue's symmetric representative into the bytes of
its two's complement (unsigned low digits, a signed top digit) and
accumulates every weight class of digit pairs in int32 over units whose
worst-case sum is at most 2^30.  These inputs put every byte at its largest
magnitude with one sign, so that the units reach that bound: an overflow or
a wrong operand type (u8 read as s8, or the reverse) would show up here.
"""
import numpy as np
import pytest
import torch

from paper_2001_04109_gb300 import ffsyrk
from parity_util import check_against_oracle, gpu_syrk, residues

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_single_tile_and_info():
    p = 65521
    A = residues(128, 128, p, seed=1)
    C, info = gpu_syrk(A, p, leaf="i8", levels=0)
    assert info["leaf"] == ffsyrk.LEAF_I8 and info["digits"] == 2
    assert all(c % 128 == 0 for c in info["chunk_k"][:2])
    check_against_oracle(A, p, C)


@pytest.mark.parametrize("n,k", [(129, 127), (256, 384), (300, 200), (517, 1000)])
def test_small_classical(n, k):
    for p in [65521, 8388593, 131071]:
        A = residues(n, k, p, seed=n + k + p % 97)
        C, _ = gpu_syrk(A, p, leaf="i8", levels=0)
        check_against_oracle(A, p, C)


# (p, symmetric residue whose two's-complement bytes all sit at their bounds,
#  k that makes one unit of the heaviest weight class reach 2^30)
BOUND_CASES = [
    (65521, -32513, 16384),      # bytes (255, −128); class 1 unit 2·128·128·255·128 ≈ 0.996·2^30
    (8388593, -4128769, 38400),  # bytes (255, 255, −64); class 1 unit fills 2^30 to one k-block
    (131071, -1, 38400),         # bytes (255, 255, −1)
]


@pytest.mark.parametrize("p,s,k", BOUND_CASES)
def test_exact_at_int32_unit_bound(p, s, k):
    D = len(ffsyrk.i8_digit_bounds(p))
    bytes_ = [(s >> (8 * t)) & 255 for t in range(D)]
    bounds = ffsyrk.i8_digit_bounds(p)
    assert all(b == bd for b, bd in zip(bytes_[:-1], bounds[:-1]))
    assert abs(((bytes_[-1] + 128) % 256) - 128) == bounds[-1]
    n = 300
    x = s % p
    A = torch.full((n, k), x, dtype=torch.int32)
    C, _ = gpu_syrk(A, p, leaf="i8", levels=0)
    check_against_oracle(A, p, C)
    # mixed signs: rows alternate s and −s, columns alternate too
    sign = np.where((np.arange(n)[:, None] + np.arange(k)[None, :]) % 2 == 0, 1, -1)
    B = torch.from_numpy(((sign * s) % p).astype(np.int32))
    C, _ = gpu_syrk(B, p, leaf="i8", levels=1)
    check_against_oracle(B, p, C)


@pytest.mark.parametrize("levels", [1, 2])
def test_winograd_levels_on_the_int8_leaf(levels):
    p = 8388593
    n, k = 700, 650
    A = residues(n, k, p, seed=levels)
    plan = ffsyrk.Plan(p, n, k, leaf="i8", levels=levels + 1, winograd=levels)
    C = torch.full((n, n), -559038737, dtype=torch.int32, device="cuda")
    plan(A.cuda(), C)
    plan.sync_status()
    assert plan.info()["winograd"][0] == levels
    plan.close()
    check_against_oracle(A, p, C.cpu().numpy().view(np.uint32))


def test_update_on_the_int8_leaf():
    import oracle
    p = 131071
    n, k = 333, 444
    A = residues(n, k, p, seed=4)
    C0 = residues(n, n, p, seed=5)
    for levels in [0, 1]:
        plan = ffsyrk.Plan(p, n, k, leaf="i8", levels=levels)
        C = C0.clone().cuda()
        plan(A.cuda(), C, alpha=12345, beta=678)
        plan.sync_status()
        plan.close()
        want = oracle.syrk_update(A.numpy(), p, 12345, C0.numpy(), 678)
        assert np.array_equal(C.cpu().numpy().view(np.uint32), want)
