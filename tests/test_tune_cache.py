"""The autotuner's cache on the host (no GPU): store, reload in a fresh process, key
mismatch, malformed lines.  The cache file is the one PTDR_TUNE_CACHE names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROG = r"""
import ctypes, json, sys
sys.path.insert(0, {root!r})
from paper_2403_11644_gb300 import _lib, build
build.build()
lib = _lib.load()

class P(ctypes.Structure):
    _fields_ = [("tile_log2", ctypes.c_int), ("masks_log2", ctypes.c_int), ("pass_tile_log2", ctypes.c_int),
                ("threads", ctypes.c_int), ("ms", ctypes.c_double)]

def look(gpu, op, n, a, c, prec):
    p = P()
    st = lib.ptdr_tune_lookup(gpu.encode(), op, n, a, c, prec, ctypes.byref(p))
    return st, (p.tile_log2, p.masks_log2, p.pass_tile_log2, p.threads, p.ms)

mode = sys.argv[1]
if mode == "store":
    p = P(17, 1, 15, 256, 12.5)
    print(json.dumps(lib.ptdr_tune_store(b"Test GPU", 0, 14, _lib.C64, _lib.C128, _lib.PREC_FP64, ctypes.byref(p))))
else:
    out = {{
        "hit": look("Test GPU", 0, 14, _lib.C64, _lib.C128, _lib.PREC_FP64),
        "other_gpu": look("Other GPU", 0, 14, _lib.C64, _lib.C128, _lib.PREC_FP64)[0],
        "other_n": look("Test GPU", 0, 15, _lib.C64, _lib.C128, _lib.PREC_FP64)[0],
        "other_op": look("Test GPU", 1, 14, _lib.C64, _lib.C128, _lib.PREC_FP64)[0],
        "other_prec": look("Test GPU", 0, 14, _lib.C64, _lib.C128, _lib.PREC_FP32)[0],
    }}
    print(json.dumps(out))
"""


def run(mode, path):
    env = dict(os.environ, PTDR_TUNE_CACHE=str(path))
    r = subprocess.run([sys.executable, "-c", PROG.format(root=ROOT), mode], capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_tune_cache_round_trip_and_keys(tmp_path):
    path = tmp_path / "tune.json"
    assert run("store", path) == 0
    text = path.read_text()
    data = json.loads(text)  # the file is valid JSON
    (key, entry), = data.items()
    assert key == "Test GPU|decompose|n=14|c64|c128|fp64"
    assert entry == {"tile_log2": 17, "masks_log2": 1, "pass_tile_log2": 15, "threads": 256, "ms": 12.5}
    got = run("lookup", path)  # a fresh process loads the file
    assert got["hit"][0] == 0 and got["hit"][1] == [17, 1, 15, 256, 12.5]
    UNSUPPORTED = 2
    assert got["other_gpu"] == got["other_n"] == got["other_op"] == got["other_prec"] == UNSUPPORTED


def test_tune_cache_ignores_malformed_lines(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text('{\n  "garbage": 12,\n  "Test GPU|decompose|n=14|c64|c128|fp64": {"tile_log2": 16, '
                    '"masks_log2": 2, "pass_tile_log2": 16, "threads": 512, "ms": 3.0}\n}\n')
    got = run("lookup", path)
    assert got["hit"][0] == 0 and got["hit"][1] == [16, 2, 16, 512, 3.0]


def test_tune_cache_missing_file_is_empty(tmp_path):
    got = run("lookup", tmp_path / "absent.json")
    assert got["hit"][0] == 2
