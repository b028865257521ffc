"""GPU parity of the band-diagonal path (tridiagonal n = 22, diagonal n = 26 and general bands)."""
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


@pytest.mark.parametrize("s", [0, 1, 2, 3, 5])
@pytest.mark.parametrize("n", [1, 4, 7, 10])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_general_complex_bands(n, s, prec):
    if s >= 2 ** n:
        pytest.skip("band wider than the matrix")
    bands = workloads.random_bands(n, s, seed=100 * n + s)
    masks = ptdr.structured_masks(n, s)
    assert np.array_equal(masks, oracle.band_masks(n, s))
    bd = dev(bands if prec == "fp64" else bands.astype(np.complex64))
    C = host(ptdr.decompose_structured(bd, s, masks=masks, precision=prec))
    ref = oracle.band_direct(bands if prec == "fp64" else bands.astype(np.complex64), s, masks)
    assert rel_err(C, ref) <= TOL[prec]


def test_unreachable_and_repeated_masks_give_oracle_rows():
    n, s = 8, 2
    bands = workloads.random_bands(n, s, seed=7)
    # 5 (2^2 - 1 = 3 > s) and 128 (2^7 - 0 > s) are out of the band's reach; 255 is reachable
    masks = np.array([5, 0, 255, 3, 3, 128], np.uint64)
    reach = set(oracle.band_masks(n, s).tolist())
    assert 5 not in reach and 128 not in reach and 255 in reach
    C = host(ptdr.decompose_structured(dev(bands), s, masks=masks, precision="fp64"))
    ref = oracle.band_direct(bands, s, masks)
    assert rel_err(C, ref) <= TOL["fp64"]
    assert np.max(np.abs(C[0])) == 0 and np.max(np.abs(C[5])) == 0
    assert np.array_equal(C[3], C[4])


@pytest.mark.parametrize("n", [9, 12])
def test_real_symmetric_tridiagonal_real_output(n):
    bands = workloads.tridiagonal(n, 22)
    masks = ptdr.structured_masks(n, 1)
    C = host(ptdr.decompose_structured(dev(bands), 1, masks=masks, precision="fp64"))
    ref = oracle.band_fwht(bands, 1, masks)
    assert np.max(np.abs(ref.imag)) <= 1e-15 * np.max(np.abs(ref))  # Thm 2
    assert rel_err(C, ref.real) <= TOL["fp64"]
    dense = oracle.direct(oracle.bands_to_dense(bands, 1)) if n <= 9 else None
    if dense is not None:  # masks outside the set carry nothing (Thm 3)
        assert rel_err(C, dense[masks.astype(np.int64)].real) <= TOL["fp64"]


def test_workload_tridiagonal_n22():
    """real symmetric tridiagonal n=22 stored as 3 bands, FP64, only the n+1 masks."""
    n = 22
    bands = workloads.tridiagonal(n, 22)
    masks = ptdr.structured_masks(n, 1)
    assert len(masks) == n + 1
    C = host(ptdr.decompose_structured(dev(bands), 1, masks=masks, precision="fp64"))
    ref = oracle.band_fwht(bands, 1, masks)
    assert rel_err(C, ref.real) <= TOL["fp64"]
    assert ptdr.last_device_status() == 0


def test_workload_diagonal_n26():
    """real diagonal n=26 (U(-1,1)), FP64: only mask 0."""
    n = 26
    d = workloads.diagonal(n, 26)
    masks = ptdr.structured_masks(n, 0)
    assert masks.tolist() == [0]
    C = host(ptdr.decompose_structured(dev(d[None, :]), 0, masks=masks, precision="fp64"))
    ref = oracle.band_fwht(d[None, :], 0, masks)
    assert rel_err(C, ref.real) <= TOL["fp64"]
    assert ptdr.last_device_status() == 0
