"""CPU FP64 oracle for the Pauli decomposition (arXiv 2403.11644).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the CPU-baseline leg of the benchmark, never by the library.  It shares
no code with the CUDA path.  The arithmetic lives in ``ptdr_oracle.c`` (plain
C, double precision, Neumaier-compensated sums); this module only marshals
numpy arrays.

Conventions (Sec. II.B, PauliComposer notation): P = sigma_{n-1} (x) ... (x)
sigma_0, qubit l <-> index bit l.  Operator (x, z): x_l = d(sigma_l) (1 for X,
Y), z_l = 1 for Y, Z.  Output ``C[x, z] = 2^-n tr(P_{x,z} A)`` (Sec. II.A).

Parity status of every function: pinned (see the oracle tests).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_u64p = ctypes.POINTER(ctypes.c_uint64)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        vp, i, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
        lib.oracle_brute.argtypes = [i, vp, vp]
        lib.oracle_direct.argtypes = [i, vp, vp, u64, vp, i]
        lib.oracle_tree.argtypes = [i, vp, vp, i, u64, u64, i]
        lib.oracle_compose.argtypes = [i, vp, ctypes.c_double, vp, i]
        lib.oracle_compose_fwht.argtypes = [i, vp, vp, u64, ctypes.c_double, vp, i]
        lib.oracle_fwht.argtypes = [i, vp, vp, u64, vp, i]
        lib.oracle_band_direct.argtypes = [i, i, vp, vp, u64, vp, i]
        lib.oracle_band_fwht.argtypes = [i, i, vp, vp, u64, vp, i]
        lib.oracle_band_masks.argtypes = [i, i, vp, u64, _u64p]
        for f in ("oracle_brute", "oracle_direct", "oracle_tree", "oracle_compose", "oracle_compose_fwht",
                  "oracle_fwht",
                  "oracle_band_direct", "oracle_band_fwht", "oracle_band_masks", "oracle_max_threads"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _nof(A):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    N = A.shape[0]
    if A.ndim != 2 or A.shape[1] != N or N < 2 or N & (N - 1):
        raise ValueError("A must be a square 2^n x 2^n matrix")
    return A, N.bit_length() - 1


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def _masks(xs, N):
    if xs is None:
        return None, N
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    return xs, len(xs)


def max_threads() -> int:
    return _load().oracle_max_threads()


def brute(A):
    """Straightforward method (Sec. II.A): explicit Kronecker products, n <= 6."""
    A, n = _nof(A)
    C = np.zeros((1 << n, 1 << n), np.complex128)
    _check(_load().oracle_brute(n, _ptr(A), _ptr(C)), "brute")
    return C


def direct(A, xs=None, threads=0):
    """O(2^n) sparse trace per coefficient (Sec. II.A).  Rows = masks ``xs`` (all if None)."""
    A, n = _nof(A)
    xs, nx = _masks(xs, 1 << n)
    C = np.zeros((nx, 1 << n), np.complex128)
    _check(_load().oracle_direct(n, _ptr(A), _ptr(xs), nx, _ptr(C), threads), "direct")
    return C


def tree(A, cut=4, subtrees=None, threads=0):
    """Algorithms 1-4 (Sec. III) with the forest split of Sec. V.B.

    ``subtrees=(t0, t1)`` walks only that range of the 4^min(cut, n) subtrees
    (numbered by their label path in base 4, digit l = label of qubit l);
    unwalked coefficients are returned as NaN.
    """
    A, n = _nof(A)
    L = min(cut, n)
    t0, t1 = (0, 1 << (2 * L)) if subtrees is None else subtrees
    C = np.full((1 << n, 1 << n), np.nan, np.complex128)
    _check(_load().oracle_tree(n, _ptr(A), _ptr(C), cut, t0, t1, threads), "tree")
    return C


def compose(C, scale=1.0, threads=0):
    """Inverse map A = scale * sum_P c_P P (Sec. II.A); direct O(8^n)."""
    C = np.ascontiguousarray(C, dtype=np.complex128)
    N = C.shape[0]
    n = N.bit_length() - 1
    A = np.zeros((N, N), np.complex128)
    _check(_load().oracle_compose(n, _ptr(C), float(scale), _ptr(A), threads), "compose")
    return A


def compose_fwht(C, scale=1.0, xs=None, threads=0):
    """Inverse map A = scale * sum_P c_P P for large n: per mask, phase i^{|x&z|},
    textbook FWHT over z, XOR-scatter (pinned against ``compose``).

    ``xs=None``: C is the whole coefficient array; returns A.  Otherwise C holds
    one row of coefficients per mask in ``xs`` and row i of the result is the
    XOR-diagonal ``A[k ^ xs[i], k]`` over k (a few masks of a large matrix)."""
    C = np.ascontiguousarray(C, dtype=np.complex128)
    N = C.shape[1]
    if C.ndim != 2 or N < 2 or N & (N - 1) or (xs is None and C.shape[0] != N):
        raise ValueError("C must hold rows of 2^n coefficients")
    n = N.bit_length() - 1
    if xs is not None:
        xs = np.ascontiguousarray(xs, dtype=np.uint64)
        if len(xs) != C.shape[0]:
            raise ValueError("one coefficient row per mask")
    out = np.zeros((N if xs is None else len(xs), N), np.complex128)
    _check(_load().oracle_compose_fwht(n, _ptr(C), _ptr(xs), 0 if xs is None else len(xs), float(scale),
                                       _ptr(out), threads), "compose_fwht")
    return out


def fwht(A, xs=None, threads=0):
    """Auxiliary full check: per-mask gather + textbook FWHT + phase + scale."""
    A, n = _nof(A)
    xs, nx = _masks(xs, 1 << n)
    C = np.zeros((nx, 1 << n), np.complex128)
    _check(_load().oracle_fwht(n, _ptr(A), _ptr(xs), nx, _ptr(C), threads), "fwht")
    return C


def _bands(bands, s):
    bands = np.ascontiguousarray(bands, dtype=np.complex128)
    if bands.ndim != 2 or bands.shape[0] != 2 * s + 1:
        raise ValueError("bands must have shape (2s+1, 2^n)")
    N = bands.shape[1]
    return bands, N.bit_length() - 1


def band_direct(bands, s, xs, threads=0):
    """Direct sparse trace over band storage bands[d+s, c] = A[c+d, c] (Sec. IV.A)."""
    bands, n = _bands(bands, s)
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    C = np.zeros((len(xs), 1 << n), np.complex128)
    _check(_load().oracle_band_direct(n, s, _ptr(bands), _ptr(xs), len(xs), _ptr(C), threads),
           "band_direct")
    return C


def band_fwht(bands, s, xs, threads=0):
    """Dense-gather FWHT over band storage (auxiliary full check for large n)."""
    bands, n = _bands(bands, s)
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    C = np.zeros((len(xs), 1 << n), np.complex128)
    _check(_load().oracle_band_fwht(n, s, _ptr(bands), _ptr(xs), len(xs), _ptr(C), threads),
           "band_fwht")
    return C


def band_masks(n, s):
    """Masks x reachable by some in-band entry (r, c), |r - c| <= s, r XOR c = x (brute force)."""
    cnt = ctypes.c_uint64(0)
    _load().oracle_band_masks(n, s, None, 0, ctypes.byref(cnt))
    out = np.zeros(cnt.value, np.uint64)
    _check(_load().oracle_band_masks(n, s, _ptr(out), cnt.value, ctypes.byref(cnt)), "band_masks")
    return out


def bands_to_dense(bands, s):
    """Expands band storage to the dense matrix (entries outside the matrix ignored)."""
    bands = np.asarray(bands)
    N = bands.shape[1]
    A = np.zeros((N, N), bands.dtype)
    for d in range(-s, s + 1):
        c = np.arange(max(0, -d), min(N, N - d))
        A[c + d, c] = bands[d + s, c]
    return A


def loss_grad(A, w):
    """Gradient of L = sum_P w_P |c_P|^2 in PyTorch's convention (2 dL/d conj(A)).

    c = D(A) is linear with D(A)_P = 2^-n <P, A>, so dL/d conj(A) =
    2^-n sum_P w_P c_P P and the gradient is 2^(1-n) * compose(w * c).
    """
    A, n = _nof(A)
    c = fwht(A)
    return compose(np.asarray(w).reshape(c.shape) * c, scale=2.0 ** (1 - n))
