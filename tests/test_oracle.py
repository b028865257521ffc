"""Pins the CPU oracle to things other than itself (CPU only).

Each check is chosen so that a plausible slip in the oracle (a transposed
operand, a wrong phase sign, a reversed bit order, a dropped 2^-n, an
off-by-one in the tree's update rules) fails at least one of them:
  * the hand-worked n = 1 fixture (Sec. I tables, Sec. II.A definition);
  * numpy.kron + numpy.trace on every operator for n <= 4 (library routine);
  * single-operator inputs give exactly one unit coefficient (Thm 1);
  * Hermitian inputs give real coefficients (Thm 2); real symmetric inputs
    have no terms with an odd number of Y;
  * diagonal inputs give only I/Z terms (Sec. IV.A.1) equal to a
    Sylvester-Hadamard product from scipy;
  * Parseval, exact reconstruction, linearity, direct sum (Sec. IV.B.1),
    Hermitian augmentation (Sec. IV.B.5), the product table (Sec. IV.B.4);
  * band masks against Thm 3 and Thm 4 term counts (Sec. IV.A.2-3);
  * the loss gradient against central finite differences.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SIG = {
    "I": np.array([[1, 0], [0, 1]], complex),
    "X": np.array([[0, 1], [1, 0]], complex),
    "Y": np.array([[0, -1j], [1j, 0]], complex),
    "Z": np.array([[1, 0], [0, -1]], complex),
}
XZ = {"I": (0, 0), "X": (1, 0), "Y": (1, 1), "Z": (0, 1)}


def label_masks(s):
    """Pauli string sigma_{n-1} ... sigma_0 -> (x, z); character -1 is qubit 0."""
    x = z = 0
    for l, ch in enumerate(reversed(s)):
        x |= XZ[ch][0] << l
        z |= XZ[ch][1] << l
    return x, z


def kron_op(s):
    P = np.array([[1.0 + 0j]])
    for ch in s:  # leftmost factor first: sigma_{n-1} (x) ... (x) sigma_0
        P = np.kron(P, SIG[ch])
    return P


def rel_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def rand_c(n, seed):
    return workloads.dense(n, seed)


# --------------------------------------------------------------------------- fixtures


def test_hand_worked_n1():
    A = np.zeros((2, 2), complex)
    want = {}
    with open(os.path.join(GOLDEN, "pauli_n1_hand.txt")) as f:
        for line in f:
            p = line.split()
            if not p or p[0].startswith("#"):
                continue
            if p[0] == "A":
                A[int(p[1]), int(p[2])] = float(p[3]) + 1j * float(p[4])
            elif p[0] == "C":
                want[(int(p[2]), int(p[3]))] = float(p[4]) + 1j * float(p[5])
    for method in (oracle.brute, oracle.direct, oracle.tree, oracle.fwht):
        C = method(A)
        for (x, z), v in want.items():
            assert abs(C[x, z] - v) < 1e-15, (method.__name__, x, z, C[x, z], v)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_brute_against_numpy_kron(n):
    A = rand_c(n, 100 + n)
    C = oracle.brute(A)
    for s in itertools.product("IXYZ", repeat=n):
        s = "".join(s)
        x, z = label_masks(s)
        ref = np.trace(kron_op(s) @ A) / 2 ** n
        assert abs(C[x, z] - ref) < 1e-13, s


@pytest.mark.parametrize("n", range(1, 7))
def test_methods_agree_small(n):
    A = rand_c(n, 200 + n)
    ref = oracle.brute(A)
    for method in (oracle.direct, oracle.tree, oracle.fwht):
        assert rel_err(method(A), ref) < 1e-14, method.__name__


@pytest.mark.parametrize("n", [7, 8, 9])
def test_tree_direct_fwht_agree(n):
    A = rand_c(n, 300 + n)
    ref = oracle.direct(A)
    assert rel_err(oracle.tree(A), ref) < 1e-14
    assert rel_err(oracle.fwht(A), ref) < 1e-13


def test_tree_forest_threads_bitwise():
    """Sec. V.B: the forest split adds no error; 1 thread == many threads bit for bit."""
    A = rand_c(7, 7)
    a = oracle.tree(A, cut=4, threads=1)
    b = oracle.tree(A, cut=4, threads=max(2, oracle.max_threads()))
    c = oracle.tree(A, cut=0, threads=1)  # whole tree walked by one recursion
    assert np.array_equal(a, b)
    assert np.array_equal(a, c)


def test_tree_subtree_range_covers_disjointly():
    A = rand_c(5, 55)
    full = oracle.tree(A, cut=2)
    parts = [oracle.tree(A, cut=2, subtrees=(t, t + 1)) for t in range(16)]
    got = np.full_like(full, np.nan)
    for p in parts:
        m = ~np.isnan(p.real)
        assert np.all(np.isnan(got[m].real)), "subtrees overlap"
        got[m] = p[m]
    assert np.array_equal(got, full)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_single_operator_inputs(n):
    for s in itertools.product("IXYZ", repeat=n):
        s = "".join(s)
        x, z = label_masks(s)
        want = np.zeros((2 ** n, 2 ** n), complex)
        want[x, z] = 1.0
        A = kron_op(s)
        for method in (oracle.brute, oracle.direct, oracle.tree, oracle.fwht):
            assert np.max(np.abs(method(A) - want)) < 1e-15, (method.__name__, s)


def test_single_operator_random_large():
    n = 8
    rng = np.random.default_rng(8)
    for _ in range(4):
        s = "".join(rng.choice(list("IXYZ"), n))
        x, z = label_masks(s)
        C = oracle.fwht(kron_op(s))
        want = np.zeros_like(C)
        want[x, z] = 1
        assert np.max(np.abs(C - want)) < 1e-15
        assert np.max(np.abs(oracle.direct(kron_op(s), xs=[x]) - want[[x]])) < 1e-15


@pytest.mark.parametrize("n", [3, 6])
def test_hermitian_real(n):
    A = workloads.dense(n, 106, hermitian=True)
    for method in (oracle.brute if n <= 6 else oracle.direct, oracle.tree, oracle.fwht):
        C = method(A)
        assert np.max(np.abs(C.imag)) <= 1e-15 * np.max(np.abs(C)), method.__name__


def test_real_symmetric_no_odd_y():
    n = 5
    B = np.random.default_rng(1).standard_normal((32, 32))
    A = B + B.T
    C = oracle.direct(A)
    x, z = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    ny = np.vectorize(lambda v: bin(v).count("1"))(x & z)
    assert np.max(np.abs(C[ny % 2 == 1])) < 1e-14
    assert np.max(np.abs(C.imag)) < 1e-15


@pytest.mark.parametrize("n", [4, 9])
def test_diagonal_iz_only_and_hadamard(n):
    d = workloads.diagonal(n, 26) + 1j * workloads.diagonal(n, 27)
    A = np.diag(d)
    C = oracle.fwht(A) if n > 6 else oracle.brute(A)
    assert np.max(np.abs(C[1:])) == 0.0
    H = scipy.linalg.hadamard(2 ** n)  # Sylvester order: H[z, k] = (-1)^{popcount(z & k)}
    assert rel_err(C[0], H @ d / 2 ** n) < 1e-15
    assert rel_err(oracle.direct(A, xs=[0])[0], H @ d / 2 ** n) < 1e-14


@pytest.mark.parametrize("n", [2, 6, 10])
def test_parseval(n):
    """||A||_F^2 = 2^n sum |c|^2 (the basis is orthogonal with <P,P> = 2^n, Thm 1)."""
    A = rand_c(n, 400 + n)
    C = oracle.fwht(A) if n > 6 else oracle.direct(A)
    lhs = np.sum(np.abs(A) ** 2)
    rhs = 2 ** n * np.sum(np.abs(C) ** 2)
    assert abs(lhs - rhs) / lhs < 1e-13


@pytest.mark.parametrize("n", [1, 3, 7])
def test_round_trip(n):
    A = rand_c(n, 500 + n)
    C = oracle.direct(A)
    assert rel_err(oracle.compose(C), A) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 3])
def test_compose_against_numpy_kron(n):
    rng = np.random.default_rng(n)
    C = rng.standard_normal((2 ** n, 2 ** n)) + 1j * rng.standard_normal((2 ** n, 2 ** n))
    ref = np.zeros((2 ** n, 2 ** n), complex)
    for s in itertools.product("IXYZ", repeat=n):
        s = "".join(s)
        x, z = label_masks(s)
        ref += C[x, z] * kron_op(s)
    assert rel_err(oracle.compose(C, scale=1.0), ref) < 1e-14
    assert rel_err(oracle.compose(C, scale=0.25), 0.25 * ref) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 5, 8, 10])
def test_compose_fwht_matches_direct_compose(n):
    """The FWHT inverse (large-n compose check) against the direct O(8^n) sum,
    itself pinned to numpy.kron above; both scales."""
    rng = np.random.default_rng(40 + n)
    C = rng.standard_normal((2 ** n, 2 ** n)) + 1j * rng.standard_normal((2 ** n, 2 ** n))
    for scale in (1.0, 2.0 ** -n):
        assert rel_err(oracle.compose_fwht(C, scale=scale), oracle.compose(C, scale=scale)) < 1e-13


def test_compose_fwht_round_trip_and_single_operator():
    """compose_fwht inverts fwht (n = 11) and maps a unit coefficient to its operator."""
    A = rand_c(11, 77)
    c = oracle.fwht(A)
    assert rel_err(oracle.compose_fwht(c), A) < 1e-13
    xs = np.array([0, 5, 2047], np.uint64)  # the XOR-diagonal form for a few masks
    k = np.arange(2048)
    want = np.stack([A[k ^ int(x), k] for x in xs])
    assert rel_err(oracle.compose_fwht(c[xs.astype(np.int64)], xs=xs), want) < 1e-13
    C = np.zeros((8, 8), complex)
    x, z = label_masks("YXZ")
    C[x, z] = 1.0
    assert np.array_equal(oracle.compose_fwht(C), kron_op("YXZ"))


def test_linearity():
    n = 6
    A, B = rand_c(n, 1), rand_c(n, 2)
    mu = 0.3 - 1.7j
    assert rel_err(oracle.fwht(mu * A + B), mu * oracle.fwht(A) + oracle.fwht(B)) < 1e-14


def test_direct_sum():
    """Sec. IV.B.1: A (+) B = I (x) (A+B)/2 + Z (x) (A-B)/2."""
    n = 4
    A, B = rand_c(n, 3), rand_c(n, 4)
    N = 2 ** n
    M = np.zeros((2 * N, 2 * N), complex)
    M[:N, :N], M[N:, N:] = A, B
    cA, cB, cM = oracle.direct(A), oracle.direct(B), oracle.direct(M)
    # new top qubit n: I -> (x_n, z_n) = (0, 0), Z -> (0, 1)
    want = np.zeros_like(cM)
    want[:N, :N] = (cA + cB) / 2
    want[:N, N:] = (cA - cB) / 2
    assert rel_err(cM, want) < 1e-14


def test_hermitian_augmentation():
    """Sec. IV.B.5: [[0, A^*], [A, 0]] = X (x) sum Re(alpha) P + Y (x) sum Im(alpha) P."""
    n = 4
    A = rand_c(n, 5)
    N = 2 ** n
    M = np.zeros((2 * N, 2 * N), complex)
    M[:N, N:] = A.conj().T
    M[N:, :N] = A
    cA, cM = oracle.direct(A), oracle.direct(M)
    want = np.zeros_like(cM)
    want[N:, :N] = cA.real  # top qubit X: x_n = 1, z_n = 0
    want[N:, N:] = cA.imag  # top qubit Y: x_n = 1, z_n = 1
    assert rel_err(cM, want) < 1e-14


def test_product_table():
    """Sec. IV.B.4: decomposition of A B from those of A and B via Pauli products."""
    n = 2
    A, B = rand_c(n, 6), rand_c(n, 7)
    cA, cB = oracle.brute(A), oracle.brute(B)
    strings = ["".join(s) for s in itertools.product("IXYZ", repeat=n)]
    want = np.zeros((4, 4), complex)
    for s in strings:
        for t in strings:
            prod = kron_op(s) @ kron_op(t)  # a Pauli operator times a phase
            want += cA[label_masks(s)] * cB[label_masks(t)] * oracle.brute(prod)
    assert rel_err(oracle.brute(A @ B), want) < 1e-14


# --------------------------------------------------------------------------- bands


def c_of_s(s):
    f = int(np.floor(np.log2(s)))
    return s * (f + 1) - 2 ** (f + 1)


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n", [4, 6, 7])
def test_band_mask_counts(n, s):
    """Thm 3 (s = 1): (n+1) masks; Thm 4: (s n - c(s)) masks of 2^n terms each."""
    masks = oracle.band_masks(n, s)
    assert len(masks) == s * n - c_of_s(s)
    if s == 1:
        assert len(masks) == n + 1
        assert sorted(masks.tolist()) == sorted([0] + [2 ** m - 1 for m in range(1, n + 1)])


def test_band_masks_diagonal():
    assert oracle.band_masks(9, 0).tolist() == [0]


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_band_direct_matches_dense(s):
    n = 6
    bands = workloads.random_bands(n, s, seed=10 + s)
    A = oracle.bands_to_dense(bands, s)
    masks = oracle.band_masks(n, s)
    dense = oracle.direct(A)
    # Only the band's masks can carry nonzero terms (Sec. IV.A).
    other = np.setdiff1d(np.arange(2 ** n), masks.astype(np.int64))
    assert np.max(np.abs(dense[other])) == 0.0
    assert rel_err(oracle.band_direct(bands, s, masks), dense[masks.astype(np.int64)]) < 1e-14
    assert rel_err(oracle.band_fwht(bands, s, masks), dense[masks.astype(np.int64)]) < 1e-13


def test_tridiagonal_workload_symmetric():
    bands = workloads.tridiagonal(5, 22)
    A = oracle.bands_to_dense(bands, 1)
    assert np.array_equal(A, A.T)
    C = oracle.band_fwht(bands, 1, oracle.band_masks(5, 1))
    assert np.max(np.abs(C.imag)) < 1e-15  # Thm 2


# --------------------------------------------------------------------------- gradient


def test_loss_gradient_finite_differences():
    n = 3
    A, w = workloads.autograd_case(n, 5)
    w = w.reshape(2 ** n, 2 ** n)
    g = oracle.loss_grad(A, w)

    def loss(M):
        return float(np.sum(w * np.abs(oracle.brute(M)) ** 2))

    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(6):
        r, c = rng.integers(0, 2 ** n, 2)
        for unit in (1.0, 1j):
            E = np.zeros_like(A)
            E[r, c] = unit * h
            fd = (loss(A + E) - loss(A - E)) / (2 * h)
            # PyTorch convention: dL along direction u equals Re(conj(g) u)
            want = (np.conj(g[r, c]) * unit).real
            assert abs(fd - want) < 1e-7 * max(1.0, abs(want))
