"""Autotuned plans: the chosen depth and tile variant are valid, results stay
bit-exact, and the tuning cache file is written and reused (marked gpu)."""
import os

import numpy as np
import pytest
import torch

from paper_2001_04109_gb300 import ffsyrk
from parity_util import check_against_oracle, residues

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_autotune_choice_and_cache(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("FFSYRK_TUNE_CACHE", str(cache))
    p, n, k = 131071, 2100, 1900
    plan = ffsyrk.Plan(p, n, k, autotune=True)
    info = plan.info()
    assert info["autotuned"] == 1 and info["tuned_ms"] > 0
    assert 0 <= info["levels"] <= 2 and info["tile_ctas"] in (1, 2)
    A = residues(n, k, p, seed=21)
    C = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    plan(A.cuda(), C)
    plan.sync_status()
    check_against_oracle(A, p, np.where(np.tril(np.ones((n, n), bool)),
                                        C.cpu().numpy().view(np.uint32), np.uint32(0xDEADBEEF)))
    plan.close()
    lines = cache.read_text().split("\n")
    assert any(f"|n{n}|k{k}|" in ln for ln in lines)
    # the second plan for the same problem takes the cached choice
    again = ffsyrk.Plan(p, n, k, autotune=True).info()
    assert again["levels"] == info["levels"] and again["tile_ctas"] == info["tile_ctas"]
    assert abs(again["tuned_ms"] - info["tuned_ms"]) < 1e-3
