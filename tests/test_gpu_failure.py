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


def _cached_syrk(A, p, C):
    n, k = A.shape
    rc = ffsyrk.lib().ffsyrk(0, n, k, p, A.data_ptr(), k, C.data_ptr(), n,
                             torch.cuda.current_stream().cuda_stream)
    return rc


def test_injected_workspace_failure_reports_err_alloc():
    """A plan whose workspace allocation fails returns FFSYRK_ERR_ALLOC and keeps no memory."""
    p = 65521
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert ffsyrk.inject_alloc_failure(0, 1) == 0
    with pytest.raises(ffsyrk.FfsyrkError) as ei:
        ffsyrk.Plan(p, 2048, 2048, leaf="tc", levels=1)
    assert ei.value.code == ffsyrk.ERR_ALLOC
    assert ffsyrk.inject_alloc_failure(0, 0) == 0  # the one failure was used
    torch.cuda.synchronize()
    # the workspace alone is 50 MB: less than 8 MB gone means it was released
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20), "the failed plan kept device memory"
    # the shared-tile slots fail after the workspace succeeded: the same outcome
    ffsyrk.inject_alloc_failure(1, 1)
    with pytest.raises(ffsyrk.FfsyrkError) as ei:
        ffsyrk.Plan(p, 2048, 2048, leaf="tc", levels=0)
    assert ei.value.code == ffsyrk.ERR_ALLOC
    assert ffsyrk.inject_alloc_failure(0, 0) == 0
    # and the next plan works
    A = residues(300, 200, p, seed=5)
    plan = ffsyrk.Plan(p, 300, 200, leaf="tc", levels=1)
    C = torch.full((300, 300), -559038737, dtype=torch.int32, device="cuda")
    plan(A.cuda(), C)
    plan.sync_status()
    check_against_oracle(A, p, C.cpu().numpy().view(np.uint32))
    plan.close()


def test_plan_cache_releases_and_retries_once():
    """The cache behind ffsyrk() frees this device's plans and retries once after ERR_ALLOC."""
    p = 65521
    # fill the cache with a few plans
    for n, k in [(256, 128), (320, 96), (384, 64)]:
        A = residues(n, k, p, seed=n).cuda()
        C = torch.zeros((n, n), dtype=torch.int32, device="cuda")
        assert _cached_syrk(A, p, C) == ffsyrk.SUCCESS
    torch.cuda.synchronize()
    plans0, rel0 = ffsyrk.cache_info()
    assert plans0 >= 3
    # the next new plan's first workspace allocation fails: the cache releases
    # its plans, tries once more and succeeds
    A_host = residues(500, 300, p, seed=8)
    C = torch.full((500, 500), -559038737, dtype=torch.int32, device="cuda")
    ffsyrk.inject_alloc_failure(0, 1)
    assert _cached_syrk(A_host.cuda(), p, C) == ffsyrk.SUCCESS
    torch.cuda.synchronize()
    assert ffsyrk.inject_alloc_failure(0, 0) == 0
    plans1, rel1 = ffsyrk.cache_info()
    assert rel1 == rel0 + 1 and plans1 == 1
    check_against_oracle(A_host, p, C.cpu().numpy().view(np.uint32))
    # two failures in a row: the retry fails too and the error reaches the caller
    ffsyrk.inject_alloc_failure(0, 2)
    A2 = residues(600, 100, p, seed=9).cuda()
    C2 = torch.zeros((600, 600), dtype=torch.int32, device="cuda")
    assert _cached_syrk(A2, p, C2) == ffsyrk.ERR_ALLOC
    assert ffsyrk.inject_alloc_failure(0, 0) == 0
    torch.cuda.synchronize()
    assert torch.count_nonzero(C2).item() == 0  # nothing was enqueued
    assert _cached_syrk(A2, p, C2) == ffsyrk.SUCCESS
    torch.cuda.synchronize()


def test_two_host_threads_call_concurrently():
    """Two threads, each with its own stream, call ffsyrk() at once; both results are exact."""
    import threading
    p = 65521
    shapes = [(1000, 700), (1500, 900)]
    hosts = [residues(n, k, p, seed=40 + t) for t, (n, k) in enumerate(shapes)]
    outs = [None, None]
    errs = []
    barrier = threading.Barrier(2)

    def work(t):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                A = hosts[t].cuda()
                n = A.shape[0]
                for rep in range(3):
                    C = torch.full((n, n), -559038737, dtype=torch.int32, device="cuda")
                    if rep == 0:
                        barrier.wait()
                    rc = ffsyrk.lib().ffsyrk(0, n, A.shape[1], p, A.data_ptr(), A.shape[1],
                                             C.data_ptr(), n, s.cuda_stream)
                    assert rc == ffsyrk.SUCCESS, rc
                s.synchronize()
                outs[t] = C.cpu().numpy().view(np.uint32)
        except Exception as e:  # pragma: no cover - reported below
            errs.append(e)

    th = [threading.Thread(target=work, args=(t,)) for t in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errs, errs
    for t in range(2):
        check_against_oracle(hosts[t], p, outs[t])
