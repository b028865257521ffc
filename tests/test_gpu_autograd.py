"""Autograd of loss = sum_P w_P |c_P|^2 through ptdr (n = 5 and n = 10)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from helpers import dev, host, rel_err

pytestmark = pytest.mark.gpu

ptdr = pytest.importorskip("paper_2403_11644_gb300")


def setup_module(_):
    from paper_2403_11644_gb300 import build
    build.build()


def loss_fn(A, w):
    c = ptdr.decompose_autograd(A, precision="fp64")
    return (w * c.abs() ** 2).sum()


def test_gradcheck_n5():
    A, w = workloads.autograd_case(5, 5)
    Ad = dev(A).requires_grad_(True)
    wd = dev(w.reshape(32, 32))
    assert torch.autograd.gradcheck(lambda a: loss_fn(a, wd), (Ad,), eps=1e-6, atol=1e-7, rtol=1e-6)


@pytest.mark.parametrize("n", [5, 10])
def test_gradient_matches_oracle(n):
    A, w = workloads.autograd_case(n, n)
    N = 2 ** n
    Ad = dev(A).requires_grad_(True)
    wd = dev(w.reshape(N, N))
    L = loss_fn(Ad, wd)
    L.backward()
    g = host(Ad.grad)
    ref = oracle.loss_grad(A, w.reshape(N, N))
    assert rel_err(g, ref) <= 1e-12


def test_finite_differences_n10():
    n = 10
    A, w = workloads.autograd_case(n, 10)
    N = 2 ** n
    Ad = dev(A).requires_grad_(True)
    wd = dev(w.reshape(N, N))
    L = loss_fn(Ad, wd)
    L.backward()
    g = Ad.grad.detach()
    rng = np.random.default_rng(10)
    h = 1e-6
    for _ in range(4):
        D = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
        Dd = dev(D)
        with torch.no_grad():
            fd = (loss_fn(Ad + h * Dd, wd) - loss_fn(Ad - h * Dd, wd)).item() / (2 * h)
        want = torch.sum(torch.conj(g) * Dd).real.item()
        assert abs(fd - want) <= 1e-6 * max(1.0, abs(want))
