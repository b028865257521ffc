"""GPU: the autotuner picks a schedule for the strided HBM passes, caches it under this
GPU's name, and later calls run it with results at the path's bound."""
import json
import os

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


def test_autotune_fp64_n14_and_tuned_calls(tmp_path, monkeypatch):
    """FP64 n = 14 (rows of 256 KiB: a first pass and strided passes): tune, check the
    cache file entry, and check a later decomposition against the oracle."""
    path = tmp_path / "tune.json"
    monkeypatch.setenv("PTDR_TUNE_CACHE", str(path))
    A = workloads.dense_c64_direct(14, 714)
    Ad = dev(A)
    C = torch.empty((1 << 14, 1 << 14), dtype=torch.complex128, device="cuda")
    best = ptdr.autotune("decompose", Ad, C, "fp64")
    print("autotuned FP64 n=14:", best)
    assert 15 <= best["tile_log2"] <= 17 and best["threads"] in (256, 512) and best["ms"] > 0
    data = json.loads(path.read_text())
    key = f"{torch.cuda.get_device_name()}|decompose|n=14|c64|c128|fp64"
    assert key in data and data[key]["tile_log2"] == best["tile_log2"]
    C.fill_(0)
    ptdr.decompose(Ad, precision="fp64", out=C)
    xs = workloads.sample_masks(14, 714, count=4)
    got = host(C[torch.from_numpy(xs.astype(np.int64)).cuda()])
    assert rel_err(got, oracle.fwht(A, xs=xs)) <= TOL["fp64"]
    assert ptdr.last_device_status() == 0


def test_autotune_rejects_plans_without_strided_passes():
    A = dev(workloads.dense(10, 1, dtype=np.complex64))
    with pytest.raises(ptdr.PtdrError):
        ptdr.autotune("decompose", A, torch.empty_like(A), "fp32")
