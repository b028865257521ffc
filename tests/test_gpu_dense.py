"""GPU parity of dense decompose/compose against the CPU oracle (n = 1..15, the n = 6, 12 and 14 workloads)."""
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
@pytest.mark.parametrize("prec,adt", [("fp64", np.complex128), ("fp32", np.complex64),
                                      ("fp64", np.complex64), ("fp32", np.complex128)])
def test_all_sizes(n, prec, adt):
    A = workloads.dense(n, 1000 + n, dtype=adt)
    C = host(ptdr.decompose(dev(A), precision=prec))
    err = rel_err(C, ref_full(A))
    print(f"decompose n={n} {prec} {np.dtype(adt).name}: rel err {err:.3e}")
    assert err <= TOL[prec]
    assert ptdr.last_device_status() == 0


@pytest.mark.parametrize("hermitian", [False, True])
def test_workload_dense_n6(hermitian):
    """dense n=6 complex128, general and Hermitian, FP64 against every oracle route."""
    A = workloads.dense(6, 106 if hermitian else 6, hermitian=hermitian)
    C = host(ptdr.decompose(dev(A), precision="fp64"))
    for ref in (oracle.brute(A), oracle.direct(A), oracle.tree(A)):
        assert rel_err(C, ref) <= TOL["fp64"]
    if hermitian:  # Thm 2: real coefficients
        assert np.max(np.abs(C.imag)) <= TOL["fp64"] * np.max(np.abs(C))


@pytest.mark.parametrize("hermitian", [False, True])
@pytest.mark.parametrize("prec,adt", [("fp64", np.complex128), ("fp32", np.complex64),
                                      ("fp64", np.complex64), ("fp32", np.complex128)])
def test_workload_dense_n12(hermitian, prec, adt):
    """dense n=12, complex128/complex64, general/Hermitian, FP64 and FP32 paths."""
    A = workloads.dense(12, 112 if hermitian else 12, dtype=adt, hermitian=hermitian)
    C = host(ptdr.decompose(dev(A), precision=prec))
    assert rel_err(C, oracle.fwht(A)) <= TOL[prec]
    xs = workloads.sample_masks(12, 12, count=30)
    assert rel_err(C[xs.astype(np.int64)], oracle.direct(A, xs=xs)) <= TOL[prec]
    if hermitian:
        assert np.max(np.abs(C.imag)) <= 2 * TOL[prec] * np.max(np.abs(C))


@pytest.fixture(scope="module")
def a14():
    return workloads.dense_c64_direct(14, 14)


@pytest.fixture(scope="module")
def ref14(a14):
    return oracle.fwht(a14)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_workload_dense_n14(a14, ref14, prec):
    """dense n=14 complex64: full output against the FWHT check, sampled rows against the direct trace."""
    Ad = dev(a14)
    out_dtype = torch.complex128 if prec == "fp64" else torch.complex64
    C = host(ptdr.decompose(Ad, precision=prec, out_dtype=out_dtype))
    assert rel_err(C, ref14) <= TOL[prec]
    xs = workloads.sample_masks(14, 14, count=14)
    assert rel_err(C[xs.astype(np.int64)], oracle.direct(a14, xs=xs)) <= TOL[prec]
    assert ptdr.last_device_status() == 0


def test_workload_dense_n14_split_bf16_tc(a14, ref14):
    """dense n=14 complex64 on the split-bf16 tensor-core path: error vs the FP64 oracle <= 2e-6."""
    C = host(ptdr.decompose(dev(a14), precision="bf16x3"))
    err = rel_err(C, ref14)
    print(f"split-bf16 TC n=14 rel err {err:.3e}")
    assert err <= TOL["bf16x3"]
    xs = workloads.sample_masks(14, 14, count=6)
    assert rel_err(C[xs.astype(np.int64)], oracle.direct(a14, xs=xs)) <= TOL["bf16x3"]
    assert ptdr.last_device_status() == 0


def test_split_tc_unsupported_sizes():
    A = dev(workloads.dense(6, 1, dtype=np.complex64))
    with pytest.raises(ptdr.PtdrError):
        ptdr.decompose(A, precision="bf16x3")


def test_n14_fp64_into_c64_workspace_path(a14, ref14):
    C = host(ptdr.decompose(dev(a14), precision="fp64", out_dtype=torch.complex64))
    assert rel_err(C, ref14) <= 1e-6  # rounded to complex64 once at the end


def chunked_rel_err(got_rows, ref_rows, N, chunk=2048):
    """rel_err over all masks, computed chunk by chunk (host memory stays bounded):
    got_rows(x0, x1) and ref_rows(x0, x1) return rows x0 .. x1 - 1."""
    num = den = 0.0
    for x0 in range(0, N, chunk):
        g = got_rows(x0, x0 + chunk).astype(np.complex128)
        r = ref_rows(x0, x0 + chunk)
        num = max(num, float(np.max(np.abs(g - r))))
        den = max(den, float(np.max(np.abs(r))))
    return num / den


def test_n15_fp32_multipass():
    """dense n = 15 (rows longer than one tile: first pass + strided HBM passes): the
    whole output against the oracle's FWHT check, mask chunk by mask chunk, plus sampled
    rows against the direct trace."""
    N = 1 << 15
    A = workloads.dense_c64_direct(15, 15)
    C = host(ptdr.decompose(dev(A), precision="fp32"))
    xs = workloads.sample_masks(15, 15, count=4)
    assert rel_err(C[xs.astype(np.int64)], oracle.direct(A, xs=xs)) <= TOL["fp32"]
    A = A.astype(np.complex128)  # converted once for every chunk of the check
    err = chunked_rel_err(lambda a, b: C[a:b], lambda a, b: oracle.fwht(A, xs=np.arange(a, b)), N)
    print(f"decompose n=15 fp32 full output: rel err {err:.3e}")
    assert err <= TOL["fp32"]
    assert ptdr.last_device_status() == 0


def test_n15_fp32_generic_multipass_for_unaligned_output():
    """An output that is not 16-byte aligned takes the generic multi-pass plan (first
    pass and strided HBM passes) instead of the staged kernel: sampled rows."""
    A = workloads.dense_c64_direct(15, 152)
    Ad = dev(A)
    buf = torch.empty((1 << 30) + 1, dtype=torch.complex64, device="cuda")
    C = buf[1:].view(1 << 15, 1 << 15)  # 8-byte aligned only
    ptdr.decompose(Ad, precision="fp32", out=C)
    xs = workloads.sample_masks(15, 152, count=6)
    got = host(C[torch.from_numpy(xs.astype(np.int64)).cuda()])
    assert rel_err(got, oracle.fwht(A, xs=xs)) <= TOL["fp32"]
    assert ptdr.last_device_status() == 0


def test_compose_n15_against_oracle():
    """n = 15 compose (multi-pass), complex64 coefficients fed to both sides, against the
    oracle's inverse FWHT: every XOR-diagonal of the result, mask chunk by mask chunk."""
    N = 1 << 15
    Cq = workloads.dense_c64_direct(15, 151)
    B = host(ptdr.compose(dev(Cq), precision="fp32"))
    k = np.arange(N)

    def got(a, b):
        return np.stack([B[k ^ x, k] for x in range(a, b)])

    def ref(a, b):
        return oracle.compose_fwht(Cq[a:b], xs=np.arange(a, b))

    err = chunked_rel_err(got, ref, N)
    print(f"compose n=15 fp32: rel err {err:.3e}")
    assert err <= TOL["fp32"]
    assert ptdr.last_device_status() == 0


@pytest.mark.parametrize("n", [1, 3, 6, 9, 12])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_round_trip(n, prec):
    adt = np.complex128 if prec == "fp64" else np.complex64
    A = workloads.dense(n, 2000 + n, dtype=adt)
    Ad = dev(A)
    C = ptdr.decompose(Ad, precision=prec, out_dtype=Ad.dtype)
    B = host(ptdr.compose(C, precision=prec))
    err = rel_err(B, A)
    print(f"round trip n={n} {prec}: rel err {err:.3e}")
    assert err <= TOL[prec]


@pytest.mark.parametrize("n", [1, 4, 7])
def test_compose_matches_oracle(n):
    rng = np.random.default_rng(n)
    C = rng.standard_normal((2 ** n, 2 ** n)) + 1j * rng.standard_normal((2 ** n, 2 ** n))
    for scale in (1.0, 2.0 ** -n):
        got = host(ptdr.compose(dev(C), scale=scale, precision="fp64"))
        assert rel_err(got, oracle.compose(C, scale=scale)) <= TOL["fp64"]


@pytest.mark.parametrize("n", range(1, 14))
def test_compose_fp32_matches_oracle(n):
    """FP32 compose (complex64 coefficients fed to both sides) against the oracle's
    inverse map: the direct O(8^n) sum up to n = 10, the inverse FWHT above."""
    rng = np.random.default_rng(60 + n)
    N = 2 ** n
    C = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    for scale in (1.0, 2.0 ** -n):
        got = host(ptdr.compose(dev(C), scale=scale, precision="fp32"))
        want = oracle.compose(C, scale=scale) if n <= 10 else oracle.compose_fwht(C, scale=scale)
        err = rel_err(got, want)
        print(f"compose n={n} fp32 scale={scale:g}: rel err {err:.3e}")
        assert err <= TOL["fp32"]
    assert ptdr.last_device_status() == 0


def test_compose_n14_staged(a14, ref14):
    """dense n=14 compose (complex64, FP32): the oracle's coefficients of the seeded
    matrix are mapped back to it, and the adjoint scale 2^-14 scales it exactly."""
    Cq = ref14.astype(np.complex64)
    Cd = dev(Cq)
    want = oracle.compose_fwht(Cq)  # the same complex64 coefficients on both sides
    B = host(ptdr.compose(Cd, precision="fp32"))
    err = rel_err(B, want)
    print(f"compose n=14 staged fp32: rel err {err:.3e} vs oracle, {rel_err(B, a14):.3e} vs A")
    assert err <= TOL["fp32"]
    assert rel_err(B, a14) <= TOL["fp32"]
    Bs = host(ptdr.compose(Cd, scale=2.0 ** -14, precision="fp32"))
    assert rel_err(Bs * 2.0 ** 14, want) <= TOL["fp32"]
    assert ptdr.last_device_status() == 0


def test_compose_n14_round_trip_and_linearity(a14):
    Ad = dev(a14)
    C = ptdr.decompose(Ad, precision="fp32")
    B = host(ptdr.compose(C, precision="fp32"))
    err = rel_err(B, a14)
    print(f"round trip n=14 fp32: rel err {err:.3e}")
    assert err <= TOL["fp32"]
    # single Pauli operators X..X (x = all ones, z = 0) and Z..Z (x = 0, z = all ones)
    Cs = torch.zeros((1 << 14, 1 << 14), dtype=torch.complex64, device="cuda")
    Cs[(1 << 14) - 1, 0] = 1.0
    Cs[0, (1 << 14) - 1] = 2.0
    P = host(ptdr.compose(Cs, precision="fp32"))
    k = np.arange(1 << 14)
    want_x = np.zeros_like(P)
    want_x[k ^ ((1 << 14) - 1), k] = 1.0                      # X..X: ones on the anti-diagonal
    want_z = np.zeros_like(P)
    want_z[k, k] = 2.0 * (-1.0) ** np.array([bin(v).count("1") for v in k])  # 2 Z..Z: diagonal signs
    assert np.array_equal(P, (want_x + want_z).astype(P.dtype))


@pytest.mark.parametrize("n,prec,dt", [(10, "fp32", np.complex64), (6, "fp64", np.complex128),
                                      (14, "bf16x3", np.complex64)])
def test_decompose_host_buffers(n, prec, dt):
    """Host-buffer entry point: three matrices copied in, decomposed and copied out with
    overlapped transfers; each against the oracle."""
    As = [workloads.dense(n, 300 + i, dtype=dt) if n < 14 else workloads.dense_c64_direct(14, 300 + i)
          for i in range(3 if n < 14 else 2)]
    ha = [torch.from_numpy(a).pin_memory() for a in As]
    hc = [torch.empty_like(a).pin_memory() for a in ha]
    ptdr.decompose_host(ha, hc, precision=prec)
    torch.cuda.synchronize()
    for a, c in zip(As, hc):
        ref = oracle.fwht(a) if n > 8 else oracle.direct(a)
        assert rel_err(c.numpy(), ref) <= TOL[prec]
    assert ptdr.last_device_status() == 0


def test_decompose_host_single_pageable():
    A = workloads.dense(8, 77, dtype=np.complex64)
    hc = [torch.empty((256, 256), dtype=torch.complex64)]
    ptdr.decompose_host([torch.from_numpy(A)], hc, precision="fp32")
    torch.cuda.synchronize()
    assert rel_err(hc[0].numpy(), oracle.direct(A)) <= TOL["fp32"]


def test_single_operator_inputs_exact():
    import itertools
    sig = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]]), "Y": np.array([[0, -1j], [1j, 0]]),
           "Z": np.diag([1, -1])}
    code = {"I": (0, 0), "X": (1, 0), "Y": (1, 1), "Z": (0, 1)}
    n = 3
    for s in itertools.product("IXYZ", repeat=n):
        P = np.array([[1.0 + 0j]])
        x = z = 0
        for l, ch in enumerate(reversed(s)):
            x |= code[ch][0] << l
            z |= code[ch][1] << l
        for ch in s:
            P = np.kron(P, sig[ch])
        C = host(ptdr.decompose(dev(P.astype(np.complex128)), precision="fp64"))
        want = np.zeros((8, 8), complex)
        want[x, z] = 1
        assert np.array_equal(C, want), s


def test_deterministic():
    A = dev(workloads.dense(12, 77, dtype=np.complex64))
    a = host(ptdr.decompose(A, precision="fp32"))
    b = host(ptdr.decompose(A, precision="fp32"))
    assert np.array_equal(a, b)


def test_parseval_n12():
    A = workloads.dense(12, 99)
    C = host(ptdr.decompose(dev(A), precision="fp64"))
    lhs = np.sum(np.abs(A) ** 2)
    assert abs(lhs - 4096 * np.sum(np.abs(C) ** 2)) / lhs < 1e-13


def test_checked_build_small():
    """Bounds-checked build: same results, and the status word stays clean."""
    import ctypes
    from paper_2403_11644_gb300 import _lib, build
    build.build(checked=True)
    L = _lib.load(checked=True)
    for n in (3, 8, 15):
        A = dev(workloads.dense(n, 5, dtype=np.complex64) if n < 15 else workloads.dense_c64_direct(15, 5))
        C = torch.empty_like(A)
        wsb = ptdr.workspace_size("decompose", n, A.dtype, C.dtype, "fp32")
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device="cuda")
        st = L.ptdr_decompose(ctypes.c_void_p(A.data_ptr()), _lib.C64, ctypes.c_void_p(C.data_ptr()),
                              _lib.C64, n, _lib.PREC_FP32, ctypes.c_void_p(ws.data_ptr()), wsb,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0
        assert L.ptdr_last_device_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
        ref = host(ptdr.decompose(A, precision="fp32"))
        assert np.array_equal(host(C), ref)
