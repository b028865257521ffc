"""ptdr_decompose_batched_static: the batched decomposition without a workspace.

For callers that cannot allocate device memory (their memory is owned by their
own pool, or allocation after start-up is not allowed), the library offers a variant whose scratch is a fixed array in its
device image.  Its results must match the workspace entry point's, call after
call, because every call rewrites the shared array before use.  Collected last
on purpose (file name), so a failure here comes after every other test ran.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads
from helpers import TOL, dev, host, rel_err

pytestmark = pytest.mark.gpu


def setup_module(_):
    from paper_2403_11644_gb300 import build
    build.build()


def _static_call(lib, plan_inputs, outs, prec):
    from paper_2403_11644_gb300 import _lib
    As = plan_inputs
    d = As[0].device
    h_n = np.array([a.shape[0].bit_length() - 1 for a in As], np.int32)
    d_A = torch.tensor([a.data_ptr() for a in As], dtype=torch.int64, device=d)
    d_C = torch.tensor([c.data_ptr() for c in outs], dtype=torch.int64, device=d)
    d_n = torch.from_numpy(h_n).to(d)
    code = {torch.complex64: _lib.C64, torch.complex128: _lib.C128}
    st = lib.ptdr_decompose_batched_static(
        ctypes.c_void_p(d_A.data_ptr()), ctypes.c_void_p(d_C.data_ptr()),
        ctypes.c_void_p(d_n.data_ptr()), h_n.ctypes.data_as(ctypes.c_void_p), len(As),
        code[As[0].dtype], code[outs[0].dtype], prec,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("prec_name", ["fp32", "fp64"])
def test_static_matches_workspace_entry_point_twice(prec_name):
    import paper_2403_11644_gb300 as ptdr
    from paper_2403_11644_gb300 import _lib
    lib = _lib.load()
    prec = ptdr.PRECISIONS[prec_name]
    dt = np.complex64 if prec_name == "fp32" else np.complex128
    tdt = torch.complex64 if prec_name == "fp32" else torch.complex128
    batches = [
        [1, 13, 4, 7, 11, 2, 9, 9, 5, 12],   # first call: uneven sizes
        [6, 3, 10, 8, 1, 4, 4, 11],           # second call: a different, smaller batch
    ]
    inputs, refs, outs = [], [], []
    for call, ns in enumerate(batches):
        As = [dev(workloads.dense(n, 900 + 31 * call + i, dtype=dt)) for i, n in enumerate(ns)]
        inputs.append(As)
        refs.append(ptdr.BatchedPlan(As, [torch.empty_like(a, dtype=tdt) for a in As], prec_name).run())
        outs.append([torch.full_like(a, float("nan"), dtype=tdt) for a in As])
    torch.cuda.synchronize()
    # two calls of the static entry point in a row, the second over a different batch
    for call in range(2):
        assert _static_call(lib, inputs[call], outs[call], prec) == 0
    assert ptdr.last_device_status() == 0
    for call in range(2):
        # per-matrix results do not depend on the queue order: bit for bit the
        # workspace entry point's, and within the bound of the oracle
        for a, r, o in zip(inputs[call], refs[call], outs[call]):
            assert torch.equal(o, r), (call, prec_name)
            A = host(a)
            ref = oracle.direct(A) if A.shape[0] <= 256 else oracle.fwht(A)
            assert rel_err(host(o), ref) <= TOL[prec_name], (call, prec_name)


def test_static_at_its_limit():
    """Exactly 4096 matrices (the largest batch the fixed array holds, its tables end on
    the array's last bytes), twice in a row, against the oracle."""
    from paper_2403_11644_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(4096)
    ns = rng.integers(1, 4, 4096)
    As = [dev(workloads.dense(int(n), 5000 + i, dtype=np.complex64)) for i, n in enumerate(ns)]
    for _ in range(2):
        outs = [torch.full_like(a, float("nan")) for a in As]
        assert _static_call(lib, As, outs, _lib.PREC_FP32) == 0
        import paper_2403_11644_gb300 as ptdr
        assert ptdr.last_device_status() == 0
        got = [host(o) for o in outs]
        for a, g in zip(As, got):
            assert rel_err(g, oracle.direct(host(a))) <= TOL["fp32"]


def test_static_rejects_batches_beyond_its_limit():
    from paper_2403_11644_gb300 import _lib
    lib = _lib.load()
    n = 4097
    h_n = np.full(n, 2, np.int32)
    fake = torch.zeros(n, dtype=torch.int64, device="cuda")
    st = lib.ptdr_decompose_batched_static(
        ctypes.c_void_p(fake.data_ptr()), ctypes.c_void_p(fake.data_ptr()),
        ctypes.c_void_p(fake.data_ptr()), h_n.ctypes.data_as(ctypes.c_void_p), n,
        _lib.C64, _lib.C64, _lib.PREC_FP32, None)
    assert st == 5  # PTDR_ERR_WORKSPACE
