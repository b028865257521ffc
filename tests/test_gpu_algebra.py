"""GPU parity of the Hermitian real-output mode (Thm 2) and of the decomposition
algebra (Sec. IV.B) against the oracle.

The algebra ops are checked against the definition: the oracle decomposes the
assembled matrix (mu A + B, the block-diagonal matrix, the augmented matrix)
directly, and the device op combines the oracle's coefficients of the parts.
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


def ref_full(A):
    n = A.shape[0].bit_length() - 1
    return oracle.direct(A) if n <= 8 else oracle.fwht(A)


# ------------------------------------------------------- Hermitian real-output mode


@pytest.mark.parametrize("n", [1, 4, 6, 10, 12, 13, 14])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fixed"])
def test_hermitian_real_output(n, prec):
    """Hermitian A: the real output type holds every coefficient (Thm 2), to the
    path's bound; the imaginary parts the oracle returns are rounding noise."""
    if n >= 13 and prec == "fp64":
        pytest.skip("FP64 n >= 13 is covered by the complex-output tests")
    adt = np.complex64 if prec == "fp32" else np.complex128
    A = workloads.dense(n, 500 + n, dtype=adt, hermitian=True)
    odt = torch.float32 if prec == "fp32" else torch.float64
    C = host(ptdr.decompose(dev(A), precision=prec, out_dtype=odt))
    ref = ref_full(A)
    tol = TOL[prec] if prec != "fixed" else TOL["fixed"]
    assert np.max(np.abs(ref.imag)) <= 1e-13 * np.max(np.abs(ref))
    err = rel_err(C, ref.real)
    print(f"Hermitian real output n={n} {prec}: rel err {err:.3e}")
    assert err <= tol
    assert ptdr.last_device_status() == 0


def test_hermitian_real_output_tensor_cores_n14():
    """The split-bf16 tensor-core kernel writes float32 real parts (half the write
    bytes) for a Hermitian n = 14 matrix: whole output against the oracle."""
    N = 1 << 14
    B = workloads.dense_c64_direct(14, 514)
    A = (0.5 * (B + B.conj().T)).astype(np.complex64)
    del B
    C = host(ptdr.decompose(dev(A), precision="bf16x3", out_dtype=torch.float32))
    assert C.shape == (N, N) and C.dtype == np.float32
    ref = oracle.fwht(A)
    err = rel_err(C, ref.real)
    print(f"Hermitian real output n=14 bf16x3: rel err {err:.3e}")
    assert err <= TOL["bf16x3"]
    assert ptdr.last_device_status() == 0


def test_real_output_of_general_matrix_is_real_part():
    """For a non-Hermitian A a real output type stores Re c_P (the documented meaning)."""
    A = workloads.dense(8, 9)
    C = host(ptdr.decompose(dev(A), precision="fp64", out_dtype=torch.float64))
    assert rel_err(C, oracle.direct(A).real) <= TOL["fp64"]


@pytest.mark.parametrize("prec,adt", [("fp64", np.float64), ("fp32", np.float32)])
def test_real_matrix_input(prec, adt):
    A = workloads.dense(9, 19).real.astype(adt)
    C = host(ptdr.decompose(dev(A), precision=prec))
    assert rel_err(C, oracle.fwht(A.astype(np.complex128))) <= TOL[prec]


@pytest.mark.parametrize("n", [3, 7, 12])
@pytest.mark.parametrize("prec", ["fp64", "fixed"])
def test_compose_real_coefficients_gives_hermitian(n, prec):
    """Real coefficients describe a Hermitian matrix (Thm 2): compose from float64
    coefficients against the oracle's inverse map."""
    rng = np.random.default_rng(70 + n)
    C = rng.standard_normal((1 << n, 1 << n))
    A = host(ptdr.compose(dev(C), precision=prec))
    assert A.dtype == np.complex128
    want = oracle.compose(C) if n <= 8 else oracle.compose_fwht(C)
    assert rel_err(A, want) <= TOL["fp64"]
    assert rel_err(A, A.conj().T) <= 1e-14


# ------------------------------------------------------------ decomposition algebra


@pytest.mark.parametrize("dt,tol", [(np.complex128, 1e-14), (np.complex64, 1e-6)])
def test_lincomb(dt, tol):
    """Sec. IV.B.3: c(mu A + B) = mu c(A) + c(B); also in place into c(B)."""
    n = 9
    A, B = workloads.dense(n, 11), workloads.dense(n, 12)
    mu = 0.75 - 1.25j
    cA, cB = dev(oracle.fwht(A).astype(dt)), dev(oracle.fwht(B).astype(dt))
    got = host(ptdr.lincomb(mu, cA, cB))
    want = oracle.fwht(mu * A + B)
    assert rel_err(got, want) <= tol
    ptdr.lincomb(mu, cA, cB, out=cB)  # in place
    assert rel_err(host(cB), want) <= tol
    assert rel_err(host(ptdr.lincomb(2.0, cA)), 2 * oracle.fwht(A)) <= tol


def test_lincomb_real_arrays():
    n = 6
    A, B = workloads.dense(n, 13, hermitian=True), workloads.dense(n, 14, hermitian=True)
    cA, cB = dev(oracle.direct(A).real.copy()), dev(oracle.direct(B).real.copy())
    got = host(ptdr.lincomb(-0.5, cA, cB))
    assert rel_err(got, oracle.direct(-0.5 * A + B).real) <= 1e-14
    with pytest.raises(ptdr.PtdrError):
        ptdr.lincomb(1j, cA, cB)  # a complex factor would leave the real arrays


def dense_block_diag(blocks):
    N = blocks[0].shape[0]
    M = np.zeros((N * len(blocks), N * len(blocks)), complex)
    for i, b in enumerate(blocks):
        M[i * N:(i + 1) * N, i * N:(i + 1) * N] = b
    return M


@pytest.mark.parametrize("n,m", [(1, 1), (3, 1), (4, 2), (3, 3), (2, 4), (10, 2)])
@pytest.mark.parametrize("dt", [np.complex128, np.complex64])
def test_block_diag_and_direct_sum(n, m, dt):
    """Sec. IV.B.1-2: the block-diagonal matrix of 2^m blocks from the blocks'
    coefficients (m = 1: the direct sum), against the oracle's decomposition of
    the assembled matrix."""
    blocks = [workloads.dense(n, 100 * n + i) for i in range(1 << m)]
    coeffs = [dev(ref_full(b).astype(dt)) for b in blocks]
    got = host(ptdr.block_diag(coeffs))
    want = ref_full(dense_block_diag(blocks))
    tol = 1e-14 if dt == np.complex128 else 1e-6
    assert rel_err(got, want) <= tol
    N = 1 << n
    assert np.all(got[N:] == 0)  # no X or Y on a top qubit


def test_direct_sum_recursive_pairing():
    """diag(A_0..A_7) = diag(A_0..A_3) (+) diag(A_4..A_7): the paper's recursive
    grouping agrees with the 8-block transform."""
    n = 3
    blocks = [workloads.dense(n, 40 + i) for i in range(8)]
    coeffs = [dev(oracle.direct(b)) for b in blocks]
    eight = host(ptdr.block_diag(coeffs))
    left, right = ptdr.block_diag(coeffs[:4]), ptdr.block_diag(coeffs[4:])
    pair = host(ptdr.block_diag([left, right]))
    assert rel_err(pair, eight) <= 1e-15


@pytest.mark.parametrize("n", [1, 5, 11])
@pytest.mark.parametrize("odt", [torch.float64, torch.complex128, torch.float32])
def test_hermitian_augmentation(n, odt):
    """Sec. IV.B.5: [[0, A^H], [A, 0]] = X (x) sum Re(alpha) P + Y (x) sum Im(alpha) P."""
    A = workloads.dense(n, 60 + n)
    N = 1 << n
    M = np.zeros((2 * N, 2 * N), complex)
    M[:N, N:] = A.conj().T
    M[N:, :N] = A
    cA = dev(ref_full(A))
    got = host(ptdr.hermitian_augment(cA, out_dtype=odt))
    want = ref_full(M)
    assert np.max(np.abs(want.imag)) <= 1e-13 * np.max(np.abs(want))  # Thm 2
    tol = 1e-6 if odt == torch.float32 else 1e-14
    assert rel_err(got, want.real if not np.iscomplexobj(got) else want) <= tol
    assert np.all(got[:N] == 0)
    assert ptdr.last_device_status() == 0
