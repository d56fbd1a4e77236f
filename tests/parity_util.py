"""Shared helpers of the GPU parity tests (the oracle is the reference)."""
import numpy as np
import torch

import oracle
from paper_2001_04109_gb300 import ffsyrk, inputs

SENTINEL = -559038737  # 0xDEADBEEF as int32: marks entries that must stay untouched


def gpu_syrk(A_host: torch.Tensor, p: int, leaf=None, levels=None, uplo="lower", lda_pad=0,
             ldc_pad=0, tile_ctas=None):
    """Run the library on a host int32 matrix; returns (C as uint32 numpy, plan info)."""
    n, k = A_host.shape
    dev = torch.device("cuda")
    Abig = torch.full((n, k + lda_pad), 7, dtype=torch.int32, device=dev)
    Abig[:, :k] = A_host.to(dev)
    A = Abig[:, :k]
    Cbig = torch.full((n, n + ldc_pad), SENTINEL, dtype=torch.int32, device=dev)
    C = Cbig[:, :n]
    plan = ffsyrk.Plan(p, max(n, 1), max(k, 1), leaf=leaf, levels=levels, tile_ctas=tile_ctas)
    plan(A, C, uplo=uplo)
    plan.sync_status()
    info = plan.info()
    plan.close()
    out = Cbig.cpu().numpy().view(np.uint32)
    if ldc_pad:
        assert np.all(out[:, n:] == np.uint32(SENTINEL & 0xFFFFFFFF)), "wrote past the last column"
    return out[:, :n], info


def check_against_oracle(A_host: torch.Tensor, p: int, C: np.ndarray, uplo="lower"):
    n = A_host.shape[0]
    want = oracle.syrk(A_host.numpy(), p, uplo)
    mask = np.tril(np.ones((n, n), dtype=bool)) if uplo == "lower" else np.triu(np.ones((n, n), dtype=bool))
    sent = np.uint32(SENTINEL & 0xFFFFFFFF)
    bad = np.argwhere(C[mask] != want[mask])
    assert bad.size == 0, f"{bad.size} of {mask.sum()} entries differ from the oracle"
    assert np.all(C[~mask] == sent), "the other strict triangle was written"


def residues(n, k, p, seed):
    return inputs.uniform_residues(n, k, p, seed)
