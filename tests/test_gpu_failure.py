"""Failure detection without a GPU fault (marked gpu).

A device-side wait that runs out must end its kernel normally, be reported
to the host as FFSYRK_ERR_TIMEOUT through the plan, and leave the plan and
the CUDA context usable.  The wait is made to run out on a barrier that
nothing signals, with a 10 ms limit.
"""
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


def test_timeout_is_reported_and_recoverable():
    p, n, k = 65521, 300, 200
    plan = ffsyrk.Plan(p, n, k, leaf="tc", levels=1)
    plan.selftest_timeout(10_000_000)
    with pytest.raises(ffsyrk.FfsyrkError) as ei:
        plan.sync_status()
    assert ei.value.code == ffsyrk.ERR_TIMEOUT
    plan.sync_status()  # cleared once reported
    A = residues(n, k, p, seed=77)
    C = torch.full((n, n), -559038737, dtype=torch.int32, device="cuda")
    plan(A.cuda(), C)
    plan.sync_status()
    check_against_oracle(A, p, C.cpu().numpy().view(np.uint32))
    plan.close()


def test_pending_timeout_blocks_the_next_call():
    p = 65521
    plan = ffsyrk.Plan(p, 64, 64, leaf="tc", levels=0)
    plan.selftest_timeout(5_000_000)
    torch.cuda.synchronize()
    A = residues(64, 64, p, seed=1).cuda()
    with pytest.raises(ffsyrk.FfsyrkError) as ei:
        plan(A)
    assert ei.value.code == ffsyrk.ERR_TIMEOUT
    with pytest.raises(ffsyrk.FfsyrkError):
        plan.sync_status()
    plan(A)
    plan.sync_status()
    plan.close()
