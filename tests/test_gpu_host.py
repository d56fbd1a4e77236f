"""GPU parity of the host-buffer entry point ffsyrk_host (marked gpu).

A and C live in host memory (pinned or pageable); the library copies A in,
runs the product and copies back the n × n result: the triangle, zeros in
the other strict triangle.  Checked against the oracle: both triangles,
odd shapes, padded host strides (columns past n untouched), repeated calls
on one plan with changing shapes and triangles, and a pipeline of calls on
two plans and streams.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2001_04109_gb300 import ffsyrk, inputs
from parity_util import SENTINEL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def host_case(n, k, p, uplo, pinned, lda_pad=0, ldc_pad=0, plan=None, seed=1):
    A = torch.full((n, k + lda_pad), 9, dtype=torch.int32)
    A[:, :k] = inputs.arbitrary_u32(n, k, seed=seed)
    C = torch.full((n, n + ldc_pad), SENTINEL, dtype=torch.int32)
    if pinned:
        A, C = A.pin_memory(), C.pin_memory()
    own = plan is None
    if own:
        plan = ffsyrk.Plan(p, n, k)
    plan.host(A[:, :k], C[:, :n], uplo=uplo)
    torch.cuda.synchronize()
    plan.sync_status()
    if own:
        plan.close()
    want = oracle.syrk(A[:, :k].numpy(), p, uplo)
    got = C.numpy().view(np.uint32)
    sent = np.uint32(SENTINEL & 0xFFFFFFFF)
    assert np.array_equal(got[:, :n], want)   # the oracle's other triangle is 0 too
    assert np.all(got[:, n:] == sent)


@pytest.mark.parametrize("uplo", ["lower", "upper"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_entry_triangles(uplo, pinned):
    host_case(1037, 513, 65521, uplo, pinned, lda_pad=3, ldc_pad=5)


def test_host_entry_repeated_and_pipelined():
    p = 131071
    plan = ffsyrk.Plan(p, 800, 700)
    for n, k, uplo, seed in [(800, 700, "lower", 1), (300, 77, "lower", 2), (300, 77, "upper", 4),
                             (800, 3, "upper", 5), (1, 5, "lower", 3)]:
        host_case(n, k, p, uplo, True, plan=plan, seed=seed)
    plan.close()
    # four calls over two plans on two streams, as a serving loop runs them
    n, k = 600, 400
    plans = [ffsyrk.Plan(p, n, k) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    As = [inputs.uniform_residues(n, k, p, seed=10 + i).pin_memory() for i in range(4)]
    Cs = [torch.zeros((n, n), dtype=torch.int32).pin_memory() for _ in range(4)]
    for i in range(4):
        plans[i % 2].host(As[i], Cs[i], stream=streams[i % 2])
    torch.cuda.synchronize()
    for i in range(4):
        want = oracle.syrk(As[i].numpy(), p, "lower")
        assert np.array_equal(Cs[i].numpy().view(np.uint32), want)
    for pl in plans:
        pl.sync_status()
        pl.close()
