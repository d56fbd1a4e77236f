"""Tensor-core leaf: a single tile first, then exactness at the FP32 bound (marked gpu).

The leaf accumulates bf16 digit products in FP32 over K-chunks sized so that
|partial sum| ≤ 2^24.  These inputs put every digit at its largest magnitude
with one sign, so every chunk sum reaches its unit's limit (exactly ±2^24
for byte digits at p = 65521): any loss of integer precision in the
tensor-core accumulation would show up here.
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


def test_single_tile_classical():
    p = 65521
    A = residues(128, 64, p, seed=1)
    C, info = gpu_syrk(A, p, leaf="tc", levels=0)
    assert info["leaf"] == 1
    check_against_oracle(A, p, C)


@pytest.mark.parametrize("n,k", [(128, 128), (256, 64), (300, 200), (129, 1000)])
def test_small_classical(n, k):
    p = 65521
    A = residues(n, k, p, seed=n + k)
    C, _ = gpu_syrk(A, p, leaf="tc", levels=0)
    check_against_oracle(A, p, C)


# (p, symmetric residue whose signed digits, in the base the library takes for p,
# all sit at their bounds: 131071 uses the balanced base 362, digits (−181, 181))
BOUND_CASES = [(65521, 32640), (131071, 65341), (8388593, 4161408)]


@pytest.mark.parametrize("p,s", BOUND_CASES)
@pytest.mark.parametrize("levels", [0, 1])
def test_exact_at_fp32_bound(p, s, levels):
    n, k = 300, 4096 + 64
    x = s % p
    A = torch.full((n, k), x, dtype=torch.int32)
    C, info = gpu_syrk(A, p, leaf="tc", levels=levels)
    check_against_oracle(A, p, C)
    # mixed signs: rows alternate s and −s, columns alternate too
    sign = np.where((np.arange(n)[:, None] + np.arange(k)[None, :]) % 2 == 0, 1, -1)
    B = torch.from_numpy(((sign * s) % p).astype(np.int32))
    C, _ = gpu_syrk(B, p, leaf="tc", levels=levels)
    check_against_oracle(B, p, C)


def test_chunks_match_plan_info():
    from paper_2001_04109_gb300 import ffsyrk
    for p, D in [(65521, 2), (131071, 2), (8388593, 3), (251, 1)]:
        plan = ffsyrk.Plan(p, 8, 8, leaf="tc", levels=0)
        info = plan.info()
        plan.close()
        assert info["digits"] == D
        ck = info["chunk_k"]
        for i in range(D):
            for j in range(D):
                assert ck[i * 3 + j] % 64 == 0 and ck[i * 3 + j] >= 256


def _run(A_host, p, levels, digit_products, tile_ctas=None, uplo="lower"):
    from paper_2001_04109_gb300 import ffsyrk
    n, k = A_host.shape
    plan = ffsyrk.Plan(p, n, k, leaf="tc", levels=levels, digit_products=digit_products,
                       tile_ctas=tile_ctas)
    C = torch.full((n, n), -559038737, dtype=torch.int32, device="cuda")
    plan(A_host.cuda(), C, uplo=uplo)
    plan.sync_status()
    info = plan.info()
    plan.close()
    return C.cpu().numpy().view(np.uint32), info


# residues whose balanced byte digits are all 127 with one sign, so that the
# Karatsuba sum planes reach 254 (p = 65521: s = 127·257; p = 8388593:
# s = 127 + 127·256 + 63·256², sums 254, 190, 190)
KS_BOUND_CASES = [(65521, 32639, 2), (8388593, 4161407, 3)]


@pytest.mark.parametrize("p,s,D", KS_BOUND_CASES)
@pytest.mark.parametrize("levels", [0, 1])
@pytest.mark.parametrize("tile_ctas", [1, 2])
def test_karatsuba_exact_at_fp32_bound(p, s, D, levels, tile_ctas):
    n, k = 300, 4096 + 64
    A = torch.full((n, k), s % p, dtype=torch.int32)
    C, info = _run(A, p, levels, "karatsuba", tile_ctas)
    assert info["products"] == D * (D + 1) // 2 and info["planes"] == D * (D + 1) // 2
    check_against_oracle(A, p, C)
    sign = np.where((np.arange(n)[:, None] + np.arange(k)[None, :]) % 2 == 0, 1, -1)
    B = torch.from_numpy(((sign * s) % p).astype(np.int32))
    C, _ = _run(B, p, levels, "karatsuba", tile_ctas)
    check_against_oracle(B, p, C)


@pytest.mark.parametrize("p", [65521, 8388593, 16777213, 521])
@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("dp", ["schoolbook", "karatsuba"])
def test_digit_products_both_ways(p, levels, dp):
    n, k = 389, 517
    A = residues(n, k, p, seed=p % 1000 + levels)
    C, info = _run(A, p, levels, dp)
    D = info["digits"]
    assert info["products"] == (D * D if dp == "schoolbook" else D * (D + 1) // 2)
    check_against_oracle(A, p, C)
    C, _ = _run(A, p, levels, dp, uplo="upper")
    check_against_oracle(A, p, C, uplo="upper")


def test_karatsuba_does_not_apply_to_balanced_base():
    # p = 131071's balanced digits reach 181: a sum could exceed 256, so the
    # plan keeps the schoolbook products whatever it is asked
    _, info = _run(residues(64, 64, 131071, seed=1), 131071, 0, "karatsuba")
    assert info["products"] == 4 and info["planes"] == 2
