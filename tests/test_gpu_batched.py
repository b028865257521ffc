"""GPU parity of the persistent batched launch (512 matrices of uneven size)."""
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


def test_uneven_small_batch_fp64():
    rng = np.random.default_rng(3)
    ns = [1, 13, 2, 7, 7, 5, 12, 3, 1, 9]
    mats = [workloads.dense(int(n), 50 + i) for i, n in enumerate(ns)]
    outs = ptdr.decompose_batched([dev(m) for m in mats], precision="fp64", out_dtype=torch.complex128)
    for m, c in zip(mats, outs):
        assert rel_err(host(c), oracle.fwht(m)) <= TOL["fp64"]
    assert ptdr.last_device_status() == 0


def test_workload_batched_512():
    """512 seeded complex64 matrices, n ~ U{4..11}, one persistent launch."""
    ns, mats = workloads.batched(seed=4)
    outs = ptdr.decompose_batched([dev(m) for m in mats], precision="fp32")
    worst = 0.0
    for m, c in zip(mats, outs):
        worst = max(worst, rel_err(host(c), oracle.fwht(m)))
    assert worst <= TOL["fp32"]
    assert ptdr.last_device_status() == 0


def test_batched_graph_replay():
    """The launch sequence replays from a CUDA graph with new data behind the same pointers."""
    ns = [4, 6, 9, 11, 5]
    mats = [workloads.dense(n, 70 + n, dtype=np.complex64) for n in ns]
    As = [dev(m) for m in mats]
    Cs = [torch.empty_like(a) for a in As]
    plan = ptdr.BatchedPlan(As, Cs, precision="fp32")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.run()  # warm-up outside capture (sets kernel attributes)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.run()
    for rep in range(3):
        new = [workloads.dense(n, 300 + 10 * rep + n, dtype=np.complex64) for n in ns]
        for a, m in zip(As, new):
            a.copy_(dev(m))
        g.replay()
        torch.cuda.synchronize()
        for m, c in zip(new, Cs):
            assert rel_err(host(c), oracle.fwht(m)) <= TOL["fp32"]


def test_batched_fp32_unaligned_and_aligned_mixed():
    """complex64 matrices of n = 9 .. 12 whose A or C starts 8 bytes past a
    16-byte boundary take the element-wise gather; aligned ones in the same
    launch take the 16-byte piece copies.  Both match the oracle."""
    ns = [11, 10, 9, 11, 10, 9, 8, 12, 12, 12]
    mats = [workloads.dense(n, 400 + i, dtype=np.complex64) for i, n in enumerate(ns)]
    As, Cs = [], []
    for i, m in enumerate(mats):
        N = m.shape[0]
        off_a, off_c = (i % 3 == 1), (i % 3 == 2)  # 8-byte offsets on A, on C, or none
        a = torch.empty(N * N + 1, dtype=torch.complex64, device="cuda")[int(off_a):][: N * N].view(N, N)
        a.copy_(dev(m))
        c = torch.empty(N * N + 1, dtype=torch.complex64, device="cuda")[int(off_c):][: N * N].view(N, N)
        assert (a.data_ptr() % 16 == 8) == off_a and (c.data_ptr() % 16 == 8) == off_c
        As.append(a)
        Cs.append(c)
    ptdr.BatchedPlan(As, Cs, precision="fp32").run()
    torch.cuda.synchronize()
    for m, c in zip(mats, Cs):
        assert rel_err(host(c), oracle.fwht(m)) <= TOL["fp32"]
    assert ptdr.last_device_status() == 0
