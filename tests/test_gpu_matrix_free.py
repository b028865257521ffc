"""GPU parity of the matrix-free input (Sec. V.B: the input need not be stored).

The callback fills, block after block, the sheared tile set the library asks for; the
coefficients are compared with the oracle on the same matrix.  One generator computes
its entries from their indices (a Fourier matrix, never stored on the device); the
others gather from a stored matrix to exercise every path up to n = 15.
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


def gather_fill(Ad, n):
    """fill() that copies the sheared tile set of block xt out of a stored matrix."""
    N = 1 << n
    k = torch.arange(N, device="cuda")
    calls = []

    def fill(xt, a, S):
        calls.append(xt)
        i = torch.arange(1 << a, device="cuda")
        rows = (((k >> a) ^ xt) << a)[None, :] + i[:, None]
        S.copy_(Ad[rows, k[None, :]])
    return fill, calls


@pytest.mark.parametrize("n,prec,dt", [(1, "fp64", np.complex128), (5, "fp32", np.complex64), (9, "fp64", np.complex128),
                                       (12, "fp32", np.complex64), (14, "fp64", np.complex64),
                                       (15, "fp32", np.complex64)])
def test_matrix_free_matches_oracle(n, prec, dt):
    A = workloads.dense(n, 900 + n, dtype=dt) if n < 14 else workloads.dense_c64_direct(n, 900 + n)
    Ad = dev(A)
    fill, calls = gather_fill(Ad, n)
    C = ptdr.decompose_matrix_free(fill, n, a_dtype=Ad.dtype, precision=prec)
    a = min(7, n)
    assert calls == list(range(1 << (n - a)))  # every block once, in order
    if n <= 12:
        ref = oracle.direct(A) if n <= 8 else oracle.fwht(A)
        assert rel_err(host(C), ref) <= TOL[prec]
    else:
        xs = workloads.sample_masks(n, 900 + n, count=6)
        got = host(C[torch.from_numpy(xs.astype(np.int64)).cuda()])
        assert rel_err(got, oracle.fwht(A, xs=xs)) <= TOL[prec]
    assert ptdr.last_device_status() == 0


def test_matrix_free_fourier_never_stored():
    """A[r][c] = exp(2 pi i r c / N) / sqrt(N), computed from the indices inside fill:
    the device never holds more than 2^7 rows of it."""
    n = 10
    N = 1 << n
    k = torch.arange(N, device="cuda", dtype=torch.float64)

    def fill(xt, a, S):
        i = torch.arange(1 << a, device="cuda")
        rows = ((((torch.arange(N, device="cuda") >> a) ^ xt) << a)[None, :] + i[:, None]).double()
        S.copy_(torch.exp(2j * np.pi * ((rows * k[None, :]) % N) / N) / np.sqrt(N))

    C = host(ptdr.decompose_matrix_free(fill, n, a_dtype=torch.complex128, precision="fp64"))
    r = np.arange(N)
    F = np.exp(2j * np.pi * ((r[:, None] * r[None, :]) % N) / N) / np.sqrt(N)
    assert rel_err(C, oracle.fwht(F)) <= TOL["fp64"]


def test_matrix_free_callback_error_stops_the_call():
    def fill(xt, a, S):
        if xt == 2:
            raise RuntimeError("generator failed")
        S.zero_()
    with pytest.raises(RuntimeError, match="generator failed"):
        ptdr.decompose_matrix_free(fill, 10, a_dtype=torch.complex64, precision="fp32")
