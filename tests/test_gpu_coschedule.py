"""The persistent n = 14 kernels under co-scheduling.

The split-bf16 tensor-core kernel and the staged FP32 decompose and compose
kernels launch one grid of persistent CTAs whose jobs wait (bounded) on jobs
that other CTAs took earlier from the same in-order queue.  Their progress
argument is that a job only ever waits on jobs dequeued before it, which
belong to CTAs that are already running; it must hold when some of the grid
cannot start at once because another kernel occupies the SMs.  Here a chain
of large bf16 matrix products runs on a second stream while each persistent
kernel runs; the results must match the oracle and the status word must be
clean (a time-out would show as PTDR_ERR_TIMEOUT, not as a hang).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from helpers import TOL, dev, host, rel_err

pytestmark = pytest.mark.gpu

ptdr = pytest.importorskip("paper_2403_11644_gb300")


def setup_module(_):
    from paper_2403_11644_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def a14():
    return workloads.dense_c64_direct(14, 1414)


def busy_stream(reps=24, size=8192):
    """Enqueues `reps` bf16 products of size^3 on a new stream (tens of ms of
    full-GPU work) and returns the stream and the buffers to keep alive."""
    s = torch.cuda.Stream()
    a = torch.randn(size, size, device="cuda", dtype=torch.bfloat16)
    b = torch.randn(size, size, device="cuda", dtype=torch.bfloat16)
    c = torch.empty(size, size, device="cuda", dtype=torch.bfloat16)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(reps):
            torch.matmul(a, b, out=c)
    return s, (a, b, c)


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_decompose_n14_beside_busy_stream(a14, prec):
    Ad = dev(a14)
    C = torch.empty_like(Ad)
    xs = workloads.sample_masks(14, 1414, count=24)
    ref = oracle.fwht(a14, xs=xs)
    ptdr.decompose(Ad, precision=prec, out=C)  # first launch outside the overlap (attributes, tables)
    torch.cuda.synchronize()
    C.zero_()
    s, keep = busy_stream()
    mine = torch.cuda.Stream()
    mine.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(mine):
        for _ in range(3):
            ptdr.decompose(Ad, precision=prec, out=C)
    torch.cuda.synchronize()
    got = host(C[torch.from_numpy(xs.astype(np.int64)).cuda()])
    assert rel_err(got, ref) <= TOL[prec]
    assert ptdr.last_device_status() == 0
    del keep, s


def test_compose_n14_beside_busy_stream(a14):
    Ad = dev(a14)
    Cd = torch.empty_like(Ad)
    ptdr.decompose(Ad, precision="fp32", out=Cd)
    torch.cuda.synchronize()
    A2 = torch.empty_like(Ad)
    ptdr.compose(Cd, precision="fp32", out=A2)  # first launch outside the overlap
    torch.cuda.synchronize()
    A2.zero_()
    s, keep = busy_stream()
    mine = torch.cuda.Stream()
    mine.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(mine):
        for _ in range(3):
            ptdr.compose(Cd, precision="fp32", out=A2)
    torch.cuda.synchronize()
    # the round trip returns A (compose is the inverse of decompose)
    assert rel_err(host(A2), a14) <= TOL["fp32"]
    assert ptdr.last_device_status() == 0
    del keep, s
