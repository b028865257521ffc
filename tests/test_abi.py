"""The C ABI without a GPU: symbols, host-only entry points, argument checks.

None of these calls launch work.  Argument errors are detected before any CUDA
call; with valid arguments and no usable device every compute entry point
returns PTDR_ERR_NO_DEVICE (there is no CPU fallback).
"""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_2403_11644_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HAVE_GPU = torch.cuda.is_available()

OK, INVALID, UNSUPPORTED, NO_DEVICE, CUDA, WORKSPACE, TIMEOUT, INTERNAL = range(8)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def header_functions():
    with open(os.path.join(ROOT, "include", "ptdr.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ptdr_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.lib_file()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (ptdr_\w+)", out))
    assert set(names) <= exported
    assert exported <= set(names), f"undeclared exports: {exported - set(names)}"


def test_status_strings(lib):
    for code, name in _lib.STATUS_NAMES.items():
        assert lib.ptdr_status_string(code).decode() == name
    assert lib.ptdr_status_string(99).decode() == "PTDR_ERR_UNKNOWN"
    assert lib.ptdr_version() >= 100


@pytest.mark.parametrize("n", range(1, 11))
def test_structured_masks_match_oracle(lib, n):
    for s in range(0, 7):
        if s >= 2 ** n:
            continue
        cnt = ctypes.c_size_t(0)
        assert lib.ptdr_structured_masks(n, s, None, ctypes.byref(cnt)) == OK
        out = np.zeros(cnt.value, np.uint64)
        assert lib.ptdr_structured_masks(n, s, out.ctypes.data_as(ctypes.c_void_p),
                                         ctypes.byref(cnt)) == OK
        assert np.array_equal(out, oracle.band_masks(n, s)), (n, s)


def test_structured_masks_capacity_and_args(lib):
    cnt = ctypes.c_size_t(2)
    out = np.zeros(2, np.uint64)
    assert lib.ptdr_structured_masks(8, 1, out.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(cnt)) == INVALID
    assert cnt.value == 9
    assert lib.ptdr_structured_masks(0, 1, None, ctypes.byref(cnt)) == INVALID
    assert lib.ptdr_structured_masks(8, -1, None, ctypes.byref(cnt)) == INVALID
    assert lib.ptdr_structured_masks(8, 1, None, None) == INVALID


def ws_size(lib, op, n, a, c, p):
    out = ctypes.c_size_t(123)
    st = lib.ptdr_workspace_size(op, n, a, c, p, ctypes.byref(out))
    return st, out.value


def test_workspace_sizes(lib):
    C64, C128 = _lib.C64, _lib.C128
    assert ws_size(lib, 0, 12, C64, C64, _lib.PREC_FP32) == (OK, 0)
    st, b = ws_size(lib, 0, 14, C64, C64, _lib.PREC_FP32)  # clustered kernel's exchange scratch
    assert st == OK and 0 < b <= 128 << 20
    assert ws_size(lib, 0, 14, C128, C64, _lib.PREC_FP32) == (OK, 0)
    assert ws_size(lib, 0, 12, C64, C64, _lib.PREC_SPLIT_BF16_TC)[0] == UNSUPPORTED
    assert ws_size(lib, 0, 14, C64, C64, 4)[0] == INVALID  # no precision 4
    # n = 15 complex64: the staged kernel's three 32 MiB staging slots (the generic
    # multi-pass plan, taken for unaligned buffers, keeps its intermediate in C)
    assert ws_size(lib, 0, 15, C64, C64, _lib.PREC_FP32) == (OK, 4096 + (96 << 20))
    assert ws_size(lib, 0, 15, C128, C64, _lib.PREC_FP32) == (OK, 0)
    st, b = ws_size(lib, 0, 14, C64, C64, _lib.PREC_FP64)  # FP64 intermediate, C64 out
    assert st == OK and b > 0
    assert ws_size(lib, 0, 14, C64, C128, _lib.PREC_FP64) == (OK, 0)
    # fixed point: a 256-byte header (exponent word), plus one L2-sized chunk of
    # 32-byte intermediate rows once a row no longer fits one tile (n >= 13)
    assert ws_size(lib, 0, 12, C64, C128, _lib.PREC_FIXED_I128) == (OK, 256)
    assert ws_size(lib, 1, 10, C128, C128, _lib.PREC_FIXED_I128) == (OK, 256)
    assert ws_size(lib, 0, 14, C64, C128, _lib.PREC_FIXED_I128) == (OK, 256 + (128 << 20))
    assert ws_size(lib, 1, 15, C128, C64, _lib.PREC_FIXED_I128) == (OK, 256 + (128 << 20))
    st, b = ws_size(lib, 1, 15, C64, C64, _lib.PREC_FP32)  # compose multi-pass
    assert st == OK and b > 0
    assert ws_size(lib, 0, 0, C64, C64, _lib.PREC_FP32)[0] == INVALID
    assert ws_size(lib, 0, 16, C64, C64, _lib.PREC_FP32)[0] == INVALID
    assert ws_size(lib, 7, 4, C64, C64, _lib.PREC_FP32)[0] == INVALID
    assert lib.ptdr_workspace_size(0, 4, C64, C64, 1, None) == INVALID


FAKE_A = 0x7F0000000000
FAKE_C = 0x7F0100000000


def decompose(lib, A, a_t, C, c_t, n, prec, ws=0, wsb=0):
    return lib.ptdr_decompose(ctypes.c_void_p(A), a_t, ctypes.c_void_p(C), c_t, n, prec,
                              ctypes.c_void_p(ws), wsb, None)


def test_decompose_argument_errors(lib):
    C64, C128 = _lib.C64, _lib.C128
    P32, TC = _lib.PREC_FP32, _lib.PREC_SPLIT_BF16_TC
    assert decompose(lib, 0, C64, FAKE_C, C64, 4, P32) == INVALID
    assert decompose(lib, FAKE_A, C64, 0, C64, 4, P32) == INVALID
    assert decompose(lib, FAKE_A, C64, FAKE_C, C64, 0, P32) == INVALID
    assert decompose(lib, FAKE_A, C64, FAKE_C, C64, 16, P32) == INVALID
    assert decompose(lib, FAKE_A, 9, FAKE_C, C64, 4, P32) == INVALID
    assert decompose(lib, FAKE_A, C64, FAKE_C, C64, 4, 9) == INVALID
    # real matrices and real (Hermitian-mode) outputs pass validation; the fake
    # pointers then fail the device check (GPU) or there is no device (CPU)
    ND = INVALID if HAVE_GPU else NO_DEVICE
    assert decompose(lib, FAKE_A, _lib.F32, FAKE_C, C64, 4, P32) == ND
    assert decompose(lib, FAKE_A, C64, FAKE_C, _lib.F64, 4, P32) == ND
    assert decompose(lib, FAKE_A, C128, FAKE_C, C64, 4, TC) == UNSUPPORTED
    assert decompose(lib, FAKE_A, C64, FAKE_C, _lib.F64, 14, TC) == UNSUPPORTED  # TC real output is F32
    # compose: real coefficients in (Hermitian A), but never a real A out
    st = lib.ptdr_compose(ctypes.c_void_p(FAKE_C), _lib.F32, ctypes.c_void_p(FAKE_A), C64, 4, 1.0, P32,
                          None, 0, None)
    assert st == ND
    st = lib.ptdr_compose(ctypes.c_void_p(FAKE_C), C64, ctypes.c_void_p(FAKE_A), _lib.F32, 4, 1.0, P32,
                          None, 0, None)
    assert st == UNSUPPORTED
    assert decompose(lib, FAKE_A + 4, C64, FAKE_C, C64, 4, P32) == INVALID  # misaligned
    assert decompose(lib, FAKE_A, C64, FAKE_A + 64, C64, 4, P32) == INVALID  # overlap
    # FP64 arithmetic into a complex64 output at n = 14 needs a workspace
    assert decompose(lib, FAKE_A, C64, FAKE_C, C64, 14, _lib.PREC_FP64) == WORKSPACE
    st = lib.ptdr_compose(ctypes.c_void_p(FAKE_C), C64, ctypes.c_void_p(FAKE_A), C64, 4, 1.0, TC,
                          None, 0, None)
    assert st == UNSUPPORTED
    st = lib.ptdr_compose(ctypes.c_void_p(FAKE_C), C64, ctypes.c_void_p(FAKE_A), C64, 4,
                          float("nan"), P32, None, 0, None)
    assert st == INVALID


@pytest.mark.skipif(HAVE_GPU, reason="checks the no-device path")
def test_no_device_no_fallback(lib):
    C64 = _lib.C64
    assert decompose(lib, FAKE_A, C64, FAKE_C, C64, 6, _lib.PREC_FP32) == NO_DEVICE
    assert decompose(lib, FAKE_A, C64, FAKE_C, C64, 6, _lib.PREC_FP64) == NO_DEVICE
    st = lib.ptdr_compose(ctypes.c_void_p(FAKE_C), C64, ctypes.c_void_p(FAKE_A), C64, 6, 1.0,
                          _lib.PREC_FP32, None, 0, None)
    assert st == NO_DEVICE
    assert lib.ptdr_last_device_status(None) == NO_DEVICE


def test_structured_argument_errors(lib):
    masks = np.array([0, 1, 3], np.uint64)
    mp = masks.ctypes.data_as(ctypes.c_void_p)

    def call(bands, b_t, n, s, masks_p, count, c, c_t, prec):
        return lib.ptdr_decompose_structured(ctypes.c_void_p(bands), b_t, n, s, masks_p, count,
                                             ctypes.c_void_p(c), c_t, prec, None, 0, None)

    F64, C128 = _lib.F64, _lib.C128
    assert call(0, F64, 6, 1, mp, 3, FAKE_C, F64, 0) == INVALID
    assert call(FAKE_A, F64, 6, 1, None, 3, FAKE_C, F64, 0) == INVALID
    assert call(FAKE_A, F64, 31, 1, mp, 3, FAKE_C, F64, 0) == INVALID
    assert call(FAKE_A, F64, 6, 64, mp, 3, FAKE_C, F64, 0) == INVALID  # s >= 2^n
    assert call(FAKE_A, C128, 6, 1, mp, 3, FAKE_C, F64, 0) == UNSUPPORTED  # complex in, real out
    assert call(FAKE_A, F64, 6, 1, mp, 3, FAKE_C, F64, _lib.PREC_SPLIT_BF16_TC) == UNSUPPORTED
    bad = np.array([0, 64], np.uint64)
    assert call(FAKE_A, F64, 6, 1, bad.ctypes.data_as(ctypes.c_void_p), 2, FAKE_C, F64, 0) == INVALID
    # valid arguments but no workspace
    assert call(FAKE_A, F64, 6, 1, mp, 3, FAKE_C, F64, 0) == WORKSPACE


def test_batched_argument_errors(lib):
    ns = np.array([4, 5, 14], np.int32)
    sz = ctypes.c_size_t(0)
    assert lib.ptdr_batched_workspace_size(ns.ctypes.data_as(ctypes.c_void_p), 3, _lib.C64, _lib.C64,
                                           _lib.PREC_FP32, ctypes.byref(sz)) == INVALID
    ns = np.array([4, 5, 11], np.int32)
    assert lib.ptdr_batched_workspace_size(ns.ctypes.data_as(ctypes.c_void_p), 3, _lib.C64, _lib.C64,
                                           _lib.PREC_FP32, ctypes.byref(sz)) == OK
    assert sz.value >= 16 + 2 * 12
    st = lib.ptdr_decompose_batched(ctypes.c_void_p(FAKE_A), ctypes.c_void_p(FAKE_C),
                                    ctypes.c_void_p(FAKE_A + 4096), ns.ctypes.data_as(ctypes.c_void_p),
                                    3, _lib.C64, _lib.C64, _lib.PREC_FP32, None, 0, None)
    assert st == WORKSPACE


def test_host_entry_point_argument_errors(lib):
    """ptdr_decompose_host: sizes and argument checks before any device work."""
    C64, P32 = _lib.C64, _lib.PREC_FP32
    sz = ctypes.c_size_t(0)
    assert lib.ptdr_decompose_host_scratch_size(10, C64, C64, P32, ctypes.byref(sz)) == OK
    assert sz.value >= 4 * (8 << 20)  # two input and two output buffers of 2^20 complex64
    assert lib.ptdr_decompose_host_scratch_size(16, C64, C64, P32, ctypes.byref(sz)) == INVALID
    assert lib.ptdr_decompose_host_scratch_size(10, _lib.F32, C64, P32, ctypes.byref(sz)) == OK  # real matrix
    host_a = np.zeros((2, 16, 16), np.complex64)
    host_c = np.zeros((2, 16, 16), np.complex64)
    ha = (ctypes.c_void_p * 2)(host_a[0].ctypes.data, host_a[1].ctypes.data)
    hc = (ctypes.c_void_p * 2)(host_c[0].ctypes.data, host_c[1].ctypes.data)

    def call(a, c, count, n, scratch, nbytes, prec=P32):
        return lib.ptdr_decompose_host(ctypes.cast(a, ctypes.c_void_p) if a is not None else None,
                                       ctypes.cast(c, ctypes.c_void_p) if c is not None else None,
                                       count, C64, C64, n, prec, ctypes.c_void_p(scratch), nbytes, None)

    assert call(None, hc, 2, 4, FAKE_A, 1 << 20) == INVALID
    assert call(ha, hc, 0, 4, FAKE_A, 1 << 20) == INVALID
    assert call(ha, hc, 2, 0, FAKE_A, 1 << 20) == INVALID
    assert call(ha, hc, 2, 4, 0, 0) == WORKSPACE
    assert call(ha, hc, 2, 4, FAKE_A, 16) == WORKSPACE
    assert call(ha, hc, 2, 4, FAKE_A + 64, 1 << 20) == INVALID  # scratch not 256-byte aligned
    same = (ctypes.c_void_p * 2)(host_a[0].ctypes.data, host_a[0].ctypes.data)
    assert call(ha, same, 2, 4, FAKE_A, 1 << 20) == INVALID  # output overlaps its input
    if not HAVE_GPU:
        assert call(ha, hc, 2, 4, FAKE_A, 1 << 20) == NO_DEVICE


def test_fault_injection_plan_is_host_side():
    """PTDR_FAULT=plan makes the entry point fail on the host before any launch."""
    code = (
        "import ctypes; from paper_2403_11644_gb300 import _lib; L=_lib.load();"
        f"print(L.ptdr_decompose(ctypes.c_void_p({FAKE_A}),0,ctypes.c_void_p({FAKE_C}),0,6,1,None,0,None))"
    )
    env = dict(os.environ, PTDR_FAULT="plan", PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         check=True).stdout
    assert out.strip() == str(INTERNAL)


def test_python_api_rejects_cpu_tensors():
    from paper_2403_11644_gb300 import decompose as dec
    with pytest.raises(ValueError, match="CUDA"):
        dec(torch.zeros(4, 4, dtype=torch.complex64))


def test_structured_workspace_covers_concurrent_masks(lib):
    """The band masks run as independent chains on up to eight streams, each
    chain with its own V region: one mask needs exactly its V rows; many
    masks need at least the largest V and at most every V (256-aligned)."""
    def ws(n, s, masks, b_t, prec):
        arr = np.asarray(masks, np.uint64)
        out = ctypes.c_size_t(0)
        st = lib.ptdr_structured_workspace_size(n, s, arr.ctypes.data_as(ctypes.c_void_p), len(arr), b_t,
                                                b_t, prec, ctypes.byref(out))
        return st, out.value

    def vbytes(n, s, x, elem):
        pairs = [t for t in range(x + 1) if (t & ~x) == 0 and abs(x - 2 * t) <= s] if x else [0]
        return len(pairs) * (1 << (n - bin(x).count("1"))) * elem

    assert ws(26, 0, [0], _lib.F64, _lib.PREC_FP64) == (OK, 8 << 26)
    masks = [int(m) for m in oracle.band_masks(22, 1)]
    st, b = ws(22, 1, masks, _lib.F64, _lib.PREC_FP64)
    each = [vbytes(22, 1, x, 8) for x in masks]
    assert st == OK and max(each) < b <= sum((v + 255) // 256 * 256 for v in each)
    st, b = ws(10, 3, [int(m) for m in oracle.band_masks(10, 3)], _lib.C128, _lib.PREC_FP64)
    assert st == OK and b > 0


@pytest.mark.parametrize("n,s", [(1, 0), (3, 0), (4, 1), (5, 2), (6, 3), (6, 5)])
def test_antistructured_masks_brute_force(lib, n, s):
    """Anti-band masks (Remark 1 of Sec. IV.A) against a brute-force enumeration of the
    XOR r ^ c over every entry with |r + c - (2^n - 1)| <= s."""
    N = 1 << n
    want = sorted({r ^ c for r in range(N) for c in range(N) if abs(r + c - (N - 1)) <= s})
    cnt = ctypes.c_size_t(0)
    assert lib.ptdr_antistructured_masks(n, s, None, ctypes.byref(cnt)) == OK
    out = np.zeros(cnt.value, np.uint64)
    assert lib.ptdr_antistructured_masks(n, s, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)) == OK
    assert out.tolist() == want
    if s == 0:
        assert want == [N - 1]  # anti-diagonal: X or Y on every qubit


def test_select_and_algebra_argument_errors(lib):
    sz = ctypes.c_size_t(0)
    assert lib.ptdr_select_workspace_size(ctypes.byref(sz)) == OK and sz.value > 0
    st = lib.ptdr_coeff_select(4, ctypes.c_void_p(FAKE_C), _lib.C64, -1.0, 0, None, None, 0,
                               ctypes.c_void_p(FAKE_A), ctypes.c_void_p(FAKE_A + 8), ctypes.c_void_p(FAKE_A + 4096),
                               sz.value, None)
    assert st == INVALID  # negative threshold
    st = lib.ptdr_coeff_select(4, ctypes.c_void_p(FAKE_C), _lib.C64, 0.0, 0, None, None, 10,
                               ctypes.c_void_p(FAKE_A), ctypes.c_void_p(FAKE_A + 8), ctypes.c_void_p(FAKE_A + 4096),
                               sz.value, None)
    assert st == INVALID  # capacity without output arrays
    st = lib.ptdr_coeff_select(4, ctypes.c_void_p(FAKE_C), _lib.C64, 0.0, 0, None, None, 0,
                               ctypes.c_void_p(FAKE_A), ctypes.c_void_p(FAKE_A + 8), None, 0, None)
    assert st == WORKSPACE
    assert lib.ptdr_coeff_lincomb(4, 1.0, 2.0, ctypes.c_void_p(FAKE_A), None, ctypes.c_void_p(FAKE_C), _lib.F64,
                                  None) == UNSUPPORTED  # a complex factor on real arrays
    assert lib.ptdr_coeff_lincomb(4, float("inf"), 0.0, ctypes.c_void_p(FAKE_A), None, ctypes.c_void_p(FAKE_C),
                                  _lib.C64, None) == INVALID
    blocks = (ctypes.c_void_p * 2)(FAKE_A, FAKE_A + (1 << 20))
    assert lib.ptdr_coeff_block_diag(4, 0, ctypes.cast(blocks, ctypes.c_void_p), ctypes.c_void_p(FAKE_C), _lib.C64,
                                     None) == INVALID  # m = 0
    assert lib.ptdr_coeff_block_diag(14, 2, ctypes.cast(blocks, ctypes.c_void_p), ctypes.c_void_p(FAKE_C), _lib.C64,
                                     None) == INVALID  # n + m > 15
    assert lib.ptdr_coeff_hermitian_augment(15, ctypes.c_void_p(FAKE_A), _lib.C64, ctypes.c_void_p(FAKE_C), _lib.F32,
                                            None) == INVALID
