"""GPU parity of the exact fixed-point path (PTDR_PREC_FIXED_I128) against the FP64 oracle.

The transform runs in 128-bit integers: the only roundings are the input's, below
2^-(124-n) of its largest magnitude, and one rounding of each result, so the bound
is the FP64 one (1e-12) for complex128 output, and half an ulp of the result for
complex64 output.
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


@pytest.mark.parametrize("n", range(1, 14))
@pytest.mark.parametrize("adt", [np.complex128, np.complex64])
def test_fixed_all_sizes(n, adt):
    A = workloads.dense(n, 3000 + n, dtype=adt)
    C = host(ptdr.decompose(dev(A), precision="fixed", out_dtype=torch.complex128))
    err = rel_err(C, ref_full(A))
    print(f"fixed n={n} {np.dtype(adt).name}: rel err {err:.3e}")
    assert err <= TOL["fixed"]
    assert ptdr.last_device_status() == 0


@pytest.mark.parametrize("hermitian", [False, True])
def test_fixed_workload_n6_and_n12(hermitian):
    """dense n = 6 and n = 12 complex128 workloads (general and Hermitian) at the FP64 bound."""
    for n, seed in ((6, 106 if hermitian else 6), (12, 112 if hermitian else 12)):
        A = workloads.dense(n, seed, hermitian=hermitian)
        C = host(ptdr.decompose(dev(A), precision="fixed", out_dtype=torch.complex128))
        assert rel_err(C, ref_full(A)) <= TOL["fixed"]
        if hermitian:  # Thm 2: real coefficients
            assert np.max(np.abs(C.imag)) <= TOL["fixed"] * np.max(np.abs(C))


def test_fixed_workload_n14():
    """dense n = 14 complex64 (the benchmark matrix) into complex128 at the FP64 bound."""
    A = workloads.dense_c64_direct(14, 14)
    C = host(ptdr.decompose(dev(A), precision="fixed", out_dtype=torch.complex128))
    err = rel_err(C, oracle.fwht(A))
    print(f"fixed n=14 complex64 -> complex128: rel err {err:.3e}")
    assert err <= TOL["fixed"]
    xs = workloads.sample_masks(14, 14, count=6)
    assert rel_err(C[xs.astype(np.int64)], oracle.direct(A, xs=xs)) <= TOL["fixed"]
    assert ptdr.last_device_status() == 0


def test_fixed_workload_n15_sampled():
    """dense n = 15 complex64 (first pass + one strided pass over six bits) into
    complex64: sampled rows at half an ulp of float32, against the FWHT check."""
    A = workloads.dense_c64_direct(15, 1515)
    C = ptdr.decompose(dev(A), precision="fixed", out_dtype=torch.complex64)
    xs = workloads.sample_masks(15, 1515, count=6)
    got = host(C[torch.from_numpy(xs.astype(np.int64)).cuda()])
    err = rel_err(got, oracle.fwht(A, xs=xs))
    print(f"fixed n=15 complex64 -> complex64 (sampled): rel err {err:.3e}")
    assert err <= 2.0 ** -24 * (1 + 1e-6)
    assert ptdr.last_device_status() == 0


@pytest.mark.parametrize("out_dtype", [torch.float64, torch.float32, torch.complex64])
def test_fixed_n13_hermitian_output_types(out_dtype):
    """n = 13 Hermitian complex128 (first pass + one strided pass over four bits):
    real outputs hold the whole (real, Thm 2) coefficient, complex64 the rounded one."""
    A = workloads.dense(13, 1313, hermitian=True)
    C = host(ptdr.decompose(dev(A), precision="fixed", out_dtype=out_dtype))
    ref = oracle.fwht(A)
    bound = TOL["fixed"] if out_dtype == torch.float64 else 2.0 ** -24 * (1 + 1e-6)
    assert rel_err(C, ref.real if out_dtype.is_floating_point else ref) <= bound
    assert ptdr.last_device_status() == 0


def test_fixed_n13_real_float32_input():
    """A real float32 matrix of n = 13 (the imaginary parts enter as zeros)."""
    A = np.ascontiguousarray(workloads.dense(13, 1314).real.astype(np.float32))
    C = host(ptdr.decompose(dev(A), precision="fixed", out_dtype=torch.complex128))
    assert rel_err(C, oracle.fwht(A.astype(np.complex128))) <= TOL["fixed"]
    assert ptdr.last_device_status() == 0


def test_fixed_complex64_output_rounded_once():
    """complex64 output: each coefficient is the exact sum rounded once, so the error is
    at most half an ulp of float32 (2^-24 of the largest coefficient)."""
    A = workloads.dense(11, 31, dtype=np.complex128)
    C = host(ptdr.decompose(dev(A), precision="fixed", out_dtype=torch.complex64))
    err = rel_err(C, oracle.fwht(A))
    print(f"fixed n=11 complex128 -> complex64: rel err {err:.3e}")
    assert err <= 2.0 ** -24 * (1 + 1e-6)


def test_fixed_wide_dynamic_range():
    """Entries spanning 2^-60 .. 2^40: the shared exponent keeps the small ones to
    2^-(124-n) of the largest, well inside the FP64 bound of the whole array."""
    rng = np.random.default_rng(7)
    n = 9
    A = workloads.dense(n, 8) * np.exp2(rng.integers(-60, 40, (1 << n, 1 << n)))
    C = host(ptdr.decompose(dev(A), precision="fixed", out_dtype=torch.complex128))
    assert rel_err(C, oracle.direct(A)) <= TOL["fixed"]


def test_fixed_single_operator_inputs_exact():
    """A = P_(x,z) gives exactly one unit coefficient, bit for bit (Thm 1)."""
    import itertools
    sig = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]]), "Y": np.array([[0, -1j], [1j, 0]]),
           "Z": np.diag([1, -1])}
    code = {"I": (0, 0), "X": (1, 0), "Y": (1, 1), "Z": (0, 1)}
    for s in itertools.product("IXYZ", repeat=3):
        P = np.array([[1.0 + 0j]])
        x = z = 0
        for l, ch in enumerate(reversed(s)):
            x |= code[ch][0] << l
            z |= code[ch][1] << l
        for ch in s:
            P = np.kron(P, sig[ch])
        C = host(ptdr.decompose(dev(P.astype(np.complex64)), precision="fixed", out_dtype=torch.complex128))
        want = np.zeros((8, 8), complex)
        want[x, z] = 1
        assert np.array_equal(C, want), s


@pytest.mark.parametrize("n", [1, 3, 6, 10])
def test_fixed_compose_matches_oracle(n):
    rng = np.random.default_rng(90 + n)
    N = 1 << n
    C = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    for scale in (1.0, 2.0 ** -n, -0.25, 0.3):
        got = host(ptdr.compose(dev(C), scale=scale, precision="fixed", out_dtype=torch.complex128))
        assert rel_err(got, oracle.compose(C, scale=scale)) <= TOL["fixed"], scale
    assert ptdr.last_device_status() == 0


def test_fixed_compose_n14_and_round_trip():
    """n = 14 compose (multi-pass, intermediate in L2-sized chunks) against the oracle's
    inverse FWHT, and decompose -> compose returning the matrix to the FP64 bound."""
    A = workloads.dense_c64_direct(14, 41).astype(np.complex128)
    Ad = dev(A)
    C = ptdr.decompose(Ad, precision="fixed", out_dtype=torch.complex128)
    B = host(ptdr.compose(C, precision="fixed", out_dtype=torch.complex128))
    assert rel_err(B, A) <= TOL["fixed"]
    Ch = host(C)
    want = oracle.compose_fwht(Ch)
    assert rel_err(B, want) <= TOL["fixed"]
    assert ptdr.last_device_status() == 0


def test_fixed_host_buffers():
    A = workloads.dense(9, 44)
    hc = [torch.empty((512, 512), dtype=torch.complex128)]
    ptdr.decompose_host([torch.from_numpy(A)], hc, precision="fixed")
    torch.cuda.synchronize()
    assert rel_err(hc[0].numpy(), oracle.direct(A)) <= TOL["fixed"]


def test_fixed_non_finite_input_reported():
    """A non-finite entry is an argument error found on the device: the pre-pass records
    PTDR_ERR_INVALID_ARG in the status word (the coefficients are then undefined)."""
    A = workloads.dense(5, 3)
    A[3, 7] = np.inf
    ptdr.decompose(dev(A), precision="fixed")
    assert ptdr.last_device_status() == 1
    assert ptdr.last_device_status() == 0  # read and cleared


def test_fixed_unsupported_elsewhere():
    bands = dev(workloads.tridiagonal(6, 1))
    with pytest.raises(ptdr.PtdrError):
        ptdr.decompose_structured(bands, 1, precision="fixed")
    with pytest.raises(ptdr.PtdrError):
        ptdr.decompose_batched([dev(workloads.dense(4, 1, dtype=np.complex64))], precision="fixed")
