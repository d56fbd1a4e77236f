"""Tensor-core leaf on CTA pairs (tcgen05 cta_group::2, 256×256 tiles), marked gpu.

Each test forces the pair variant and compares with the oracle bit-exactly:
a single pair tile first, ragged shapes that leave partial tiles in both
dimensions, the fast path at several depths, the FP32-bound inputs, and the
upper triangle with padded strides.
"""
import numpy as np
import pytest
import torch

from parity_util import check_against_oracle, gpu_syrk, residues

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_single_pair_tile():
    p = 65521
    A = residues(256, 64, p, seed=1)
    C, info = gpu_syrk(A, p, leaf="tc", levels=0, tile_ctas=2)
    check_against_oracle(A, p, C)


@pytest.mark.parametrize("n,k", [(300, 200), (511, 1030), (1024, 1024), (777, 333), (129, 4100)])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_pair_shapes(n, k, levels):
    p = 131071
    A = residues(n, k, p, seed=n * 7 + k)
    C, _ = gpu_syrk(A, p, leaf="tc", levels=levels, tile_ctas=2)
    check_against_oracle(A, p, C)


@pytest.mark.parametrize("p,s", [(65521, 32640), (131071, 65341), (8388593, 4161408)])
def test_pair_exact_at_fp32_bound(p, s):
    n, k = 520, 4096 + 64
    sign = np.where((np.arange(n)[:, None] + np.arange(k)[None, :]) % 3 == 0, -1, 1)
    A = torch.from_numpy(((sign * s) % p).astype(np.int32))
    C, _ = gpu_syrk(A, p, leaf="tc", levels=1, tile_ctas=2)
    check_against_oracle(A, p, C)


def test_pair_upper_strides():
    p = 8388593
    A = residues(600, 700, p, seed=4)
    C, _ = gpu_syrk(A, p, leaf="tc", levels=1, uplo="upper", lda_pad=3, ldc_pad=5, tile_ctas=2)
    check_against_oracle(A, p, C, uplo="upper")
