"""Failure detection without a GPU fault: bounded device waits that run out, and
host-side fault injection.

The persistent n = 14 kernels wait (bounded) on counters other CTAs publish and on
their own pipeline barriers.  With the wait limit set to 1 ns (PTDR_WAIT_NS, read at
each launch) a wait that is not already satisfied gives up at once: the kernel records
PTDR_ERR_TIMEOUT, leaves its loops, waits for its own copies and tensor-core products
in flight, frees its tensor memory and returns.  The test then checks that the status
word reports the time-out and that the context still computes correct results.
PTDR_FAULT=launch makes the host fail the call before anything is enqueued.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads
from helpers import TOL, dev, host, rel_err

pytestmark = pytest.mark.gpu

ptdr = pytest.importorskip("paper_2403_11644_gb300")

TIMEOUT, CUDA_ERR = 6, 4


def setup_module(_):
    from paper_2403_11644_gb300 import build
    build.build()


class env:
    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kv}
        os.environ.update(self.kv)

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.fixture(scope="module")
def a14():
    A = workloads.dense_c64_direct(14, 614)
    xs = workloads.sample_masks(14, 614, count=2)
    return A, dev(A), xs, oracle.fwht(A, xs=xs)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_wait_limit_runs_out_and_context_survives(a14, prec):
    """Staged FP32 and split-bf16 tensor-core kernels: a 1 ns wait limit is reported as
    PTDR_ERR_TIMEOUT; the next launch with the default limit is correct again."""
    A, Ad, xs, ref = a14
    assert ptdr.last_device_status() == 0
    with env(PTDR_WAIT_NS="1"):
        ptdr.decompose(Ad, precision=prec)
        assert ptdr.last_device_status() == TIMEOUT
    C = ptdr.decompose(Ad, precision=prec)
    assert ptdr.last_device_status() == 0
    got = host(C[torch.from_numpy(xs.astype(np.int64)).cuda()])
    assert rel_err(got, ref) <= TOL[prec]


def test_wait_limit_compose_staged(a14):
    A, Ad, _, _ = a14
    with env(PTDR_WAIT_NS="1"):
        ptdr.compose(Ad, precision="fp32")
        assert ptdr.last_device_status() == TIMEOUT
    ptdr.compose(Ad, precision="fp32")
    assert ptdr.last_device_status() == 0


def test_launch_fault_injection_is_host_side():
    """PTDR_FAULT=launch: the call returns PTDR_ERR_CUDA before anything is enqueued."""
    A = workloads.dense(6, 1)
    Ad = dev(A)
    out = torch.full((64, 64), 7.0 + 7.0j, dtype=torch.complex128, device="cuda")
    with env(PTDR_FAULT="launch"):
        with pytest.raises(ptdr.PtdrError) as e:
            ptdr.decompose(Ad, precision="fp64", out=out)
        assert e.value.status == CUDA_ERR
    assert torch.all(out == 7.0 + 7.0j)  # nothing ran
    assert ptdr.last_device_status() == 0
    C = host(ptdr.decompose(Ad, precision="fp64", out=out))
    assert rel_err(C, oracle.direct(A)) <= TOL["fp64"]
