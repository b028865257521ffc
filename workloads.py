"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers and nothing else: it holds none of the Pauli
decomposition's arithmetic, so both the oracle side and the CUDA side can use
it without sharing any of the method.

Recipes (numpy PCG64 via ``default_rng(seed)``; the paper's workloads are
generic dense complex matrices with no structure, Sec. V):
  dense(n, seed)          real parts drawn first, then imaginary parts, both
                          i.i.d. N(0, 1) in float64; complex64 is a cast of the
                          same draws.  ``hermitian=True`` returns (B + B^H)/2.
  dense_c64_direct(n, s)  complex64 drawn directly in float32 (real block then
                          imaginary block), used at n = 14 where a float64
                          intermediate of 4 GiB would dominate set-up time.
  diagonal(n, seed)       real float64 entries U(-1, 1).
  tridiagonal(n, seed)    real symmetric: main diagonal N(0,1)[2^n], then the
                          off-diagonal N(0,1)[2^n - 1]; returned in band layout
                          bands[d + 1, c] = A[c + d, c], d in {-1, 0, 1}.
  batched_ns(seed)        512 sizes n ~ U{4..11} (integers(4, 12)), then each
                          matrix drawn as complex64 N(0,1) in draw order.
  autograd_case(n, seed)  complex128 N(0,1) matrix, then weights U(0,1)[4^n].
"""
import numpy as np


def dense(n: int, seed: int, dtype=np.complex128, hermitian: bool = False) -> np.ndarray:
    N = 1 << n
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((N, N))
    im = rng.standard_normal((N, N))
    A = re + 1j * im
    if hermitian:
        A = 0.5 * (A + A.conj().T)
    return np.ascontiguousarray(A.astype(dtype))


def dense_c64_direct(n: int, seed: int) -> np.ndarray:
    N = 1 << n
    rng = np.random.default_rng(seed)
    out = np.empty((N, N), np.complex64)
    f = out.view(np.float32).reshape(N, N, 2)
    f[:, :, 0] = rng.standard_normal((N, N), dtype=np.float32)
    f[:, :, 1] = rng.standard_normal((N, N), dtype=np.float32)
    return out


def diagonal(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, 1 << n)


def tridiagonal(n: int, seed: int) -> np.ndarray:
    N = 1 << n
    rng = np.random.default_rng(seed)
    main = rng.standard_normal(N)
    off = rng.standard_normal(N - 1)
    # band layout bands[d + 1, c] = A[c + d, c]; symmetric, A[i, i+1] = A[i+1, i] = off[i]:
    #   d = -1 holds A[c - 1, c] for c = 1 .. N-1  -> off[c - 1]
    #   d = +1 holds A[c + 1, c] for c = 0 .. N-2  -> off[c]
    bands = np.zeros((3, N))
    bands[1] = main
    bands[0, 1:] = off
    bands[2, : N - 1] = off
    return bands


def random_bands(n: int, s: int, seed: int, complex_: bool = True) -> np.ndarray:
    """General (non-symmetric) band matrix of half-width s in band layout."""
    N = 1 << n
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((2 * s + 1, N))
    b = re + 1j * rng.standard_normal((2 * s + 1, N)) if complex_ else re
    for d in range(-s, s + 1):  # zero the slots that fall outside the matrix
        c = np.arange(N)
        b[d + s, (c + d < 0) | (c + d >= N)] = 0
    return b


def batched_ns(seed: int = 4, count: int = 512, lo: int = 4, hi: int = 11) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, count)


def batched(seed: int = 4, count: int = 512, lo: int = 4, hi: int = 11):
    rng = np.random.default_rng(seed)
    ns = rng.integers(lo, hi + 1, count)
    mats = []
    for n in ns:
        N = 1 << int(n)
        m = np.empty((N, N), np.complex64)
        f = m.view(np.float32).reshape(N, N, 2)
        f[:, :, 0] = rng.standard_normal((N, N), dtype=np.float32)
        f[:, :, 1] = rng.standard_normal((N, N), dtype=np.float32)
        mats.append(m)
    return ns, mats


def autograd_case(n: int, seed: int):
    rng = np.random.default_rng(seed)
    N = 1 << n
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    w = rng.uniform(0.0, 1.0, N * N)
    return A, w


def sample_masks(n: int, seed: int, count: int = 254) -> np.ndarray:
    """Masks 0 and 2^n - 1 plus ``count`` distinct seeded random masks (sorted)."""
    N = 1 << n
    rng = np.random.default_rng(seed + 1000)
    k = min(count, max(0, N - 2))
    rest = rng.choice(np.arange(1, N - 1), size=k, replace=False) if k else np.array([], np.int64)
    xs = np.unique(np.concatenate([[0, N - 1], rest]))
    return xs.astype(np.uint64)
