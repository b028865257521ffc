"""Benchmark: Pauli coefficients/s of the dense n=14 decomposition on GB300.

One step = one decomposition of a seeded 16384 x 16384 complex64 matrix (all
268,435,456 coefficients): XOR-diagonal gather, Walsh-Hadamard transform,
phase and scale, through the library's C ABI.  The input (2 GiB) and output
(2 GiB) are each larger than the 129 MB L2, so no flush is needed between
steps.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P]
  python bench.py --impl reference ...   # the CPU oracle on the host cores

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the decomposition has no exchange step across matrices), "scaling": "weak",
value = coefficients of all ranks / max time over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_QUBITS = 14
SEED = 14
METRIC = "Pauli coeffs/s and HBM GB/s at n=14, split-BF16 TC vs FP64 plain"

# DRAM bytes (read + write) per launch of the dominant kernel of each n = 14
# path, from one ncu capture each (summaries under profiles/).  A figure is
# reported only while the sources it was taken from are unchanged.
NCU_TRAFFIC = {
    "fp32": {"kernel": "k_dense_staged", "bytes": 2_147_561_472 + 2_123_435_520,
             "sources": {"paper_2403_11644_gb300/csrc/k_dense14s.cu":
                         "48307cc6b4e0cced6ac086cc997693b4d822e88f7174f517680b8de24971c4f0",
                         "paper_2403_11644_gb300/csrc/common.cuh":
                         "0b8af7566a7fe16e8503406413c2ad8e3700521db352a206df357200a0645186"}},
    "bf16x3": {"kernel": "k_tc14_pipe", "bytes": 2_148_103_168 + 2_117_208_064,
               "sources": {"paper_2403_11644_gb300/csrc/k_tc14p.cu":
                           "fac413e7ad250256122c5ce63f7bfeb02adc1343dabc06324a7e9732336c9481",
                           "paper_2403_11644_gb300/csrc/common.cuh":
                           "0b8af7566a7fe16e8503406413c2ad8e3700521db352a206df357200a0645186"}},
}


def ncu_traffic(prec, n):
    """(kernel, bytes per launch) from the capture table, bytes None if stale."""
    import hashlib
    e = NCU_TRAFFIC.get(prec)
    if e is None or n != 14:
        return ({"bf16x3": "k_tc14_pipe", "fp32": "k_dense_staged"}.get(prec) if n == 14 else None), None
    for rel, sha in e["sources"].items():
        path = os.path.join(ROOT, rel)
        if not os.path.exists(path):
            return e["kernel"], None
        with open(path, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != sha:
                return e["kernel"], None
    return e["kernel"], e["bytes"]


# Relative max-abs error bounds against the FP64 oracle, per arithmetic path.
TOLERANCE = {"fp64": 1e-12, "fp32": 1e-5, "bf16x3": 2e-6, "fixed": 1e-12}


def fp64_add_rate(dev, stream, reps=3):
    """FP64 adds/s of this GPU, measured now with the library's add-chain probe
    (8 independent chains per thread, 8 CTAs of 256 threads per SM): the bound
    of the FP64 transforms."""
    import ctypes
    import torch
    from paper_2403_11644_gb300 import _lib
    lib = _lib.load()
    blocks = torch.cuda.get_device_properties(dev).multi_processor_count * 8
    sink = torch.zeros(blocks, dtype=torch.float64, device=dev)
    adds = ctypes.c_double(0)
    sp = ctypes.c_void_p(stream.cuda_stream)

    def run():
        _lib.check(lib.ptdr_probe_fp64_adds(ctypes.c_void_p(sink.data_ptr()), blocks, 256, 4096,
                                            ctypes.byref(adds), sp), "ptdr_probe_fp64_adds")
    run()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        run()
    b.record(stream)
    torch.cuda.synchronize(dev)
    return reps * adds.value / (a.elapsed_time(b) * 1e-3)


def _timed(fn, stream, reps=3, flush=None):
    """Mean CUDA-event time (ms) of fn() over reps, after one warm-up call."""
    import torch
    fn()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(reps):
        if flush is not None:
            flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
    return tot / reps


def measure_rows(dev, stream, hbm_peak, fp64_rate, only="all", batched_count=512):
    """Throughput of the other hot-path rows on their workloads (rank 0, N = 1).

    The band inputs are the seeded workloads of the GPU tests; the dense and
    batched inputs are seeded draws made on the device (timing only; their
    parity is covered by the GPU tests).  Each entry reports its own bound:
    HBM bytes against the measured copy bandwidth, or FP64 adds against the
    FP64 add rate.
    """
    import torch
    import paper_2403_11644_gb300 as ptdr
    g = torch.Generator(device=dev)
    rows = {}
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def flush():
        flush_buf.fill_(1)

    def hbm(ms, nbytes):
        gbs = nbytes / ms / 1e6
        return {"bound": "hbm", "achieved_gbs": gbs, "frac": gbs / hbm_peak}

    def fp64(ms, adds):
        r = adds / (ms * 1e-3)
        return {"bound": "fp64_alu", "achieved_ops_per_s": r, "frac": r / fp64_rate}

    def entry(name, fn, work):
        if only != "all" and name not in only.split(","):
            return
        try:
            rows[name] = fn()
            rows[name].update(work(rows[name]["ms"]))
        except Exception as e:  # report, never hide
            rows[name] = {"error": str(e)}

    # a6: diagonal n = 26 (mask 0 only) and tridiagonal n = 22 (23 masks), FP64.
    # Real bands are transformed in real arithmetic: the FP64 work is the pruned
    # transforms' adds plus the expansion (one add per pair and one scale per output).
    def band_fp64_ops(n, s):
        """FP64 operations of a real band: per mask, |T_x| transforms of 2^f
        values (f 2^f adds each), the 2^-n applied once per band value, and
        |T_x| - 1 adds per coefficient in the expansion."""
        ops = 0
        for x in ptdr.structured_masks(n, s):
            x = int(x)
            f = n - bin(x).count("1")
            pairs = [t for t in range(x + 1) if (t & ~x) == 0 and abs(x - 2 * t) <= s] if x else [0]
            ops += len(pairs) * (f + 1) * (1 << f) + max(len(pairs) - 1, 0) * (1 << n)
        return ops

    def diag():
        import workloads
        bands = torch.from_numpy(workloads.diagonal(26, 26)).reshape(1, -1).to(dev)
        out = torch.empty((1, 1 << 26), dtype=torch.float64, device=dev)
        ms = _timed(lambda: ptdr.decompose_structured(bands, 0, out=out), stream)
        return {"workload": "diagonal n=26 float64", "ms": ms, "coeffs_per_s": (1 << 26) / (ms * 1e-3),
                "algorithmic_bytes": 2 * 8 << 26, "fp64_ops": band_fp64_ops(26, 0)}
    entry("diagonal_n26_fp64", diag, lambda ms: fp64(ms, rows["diagonal_n26_fp64"]["fp64_ops"]))

    def tri():
        import workloads
        bands = torch.from_numpy(workloads.tridiagonal(22, 22)).to(dev)
        nm = len(ptdr.structured_masks(22, 1))
        out = torch.empty((nm, 1 << 22), dtype=torch.float64, device=dev)
        ms = _timed(lambda: ptdr.decompose_structured(bands, 1, out=out), stream)
        nbytes = 3 * 8 << 22
        nbytes += nm * 8 << 22
        return {"workload": "tridiagonal n=22 float64", "ms": ms, "coeffs_per_s": nm * (1 << 22) / (ms * 1e-3),
                "algorithmic_bytes": nbytes, "fp64_ops": band_fp64_ops(22, 1)}
    entry("tridiagonal_n22_fp64", tri, lambda ms: fp64(ms, rows["tridiagonal_n22_fp64"]["fp64_ops"]))

    # a7: 512 matrices of uneven size in one persistent launch, FP32
    def batched():
        import workloads
        ns = workloads.batched_ns(4)[:batched_count]
        g.manual_seed(4)
        As = [torch.randn((1 << int(n), 1 << int(n)), generator=g, device=dev, dtype=torch.complex64) for n in ns]
        Cs = [torch.empty_like(a) for a in As]
        plan = ptdr.BatchedPlan(As, Cs, "fp32")
        coeffs = int(sum(4 ** int(n) for n in ns))
        ms = _timed(plan.run, stream, flush=flush)
        return {"workload": f"{len(ns)} matrices, n ~ U{{4..11}}, complex64 (seed 4)", "ms": ms,
                "coeffs_per_s": coeffs / (ms * 1e-3), "algorithmic_bytes": 16 * coeffs}
    entry("batched_512_fp32", batched, lambda ms: hbm(ms, rows["batched_512_fp32"]["algorithmic_bytes"]))

    # a8: compose (inverse map) n = 14, FP32
    def comp():
        g.manual_seed(114)
        Cc = torch.randn((1 << 14, 1 << 14), generator=g, device=dev, dtype=torch.complex64)
        Ao = torch.empty_like(Cc)
        ms = _timed(lambda: ptdr.compose(Cc, out=Ao), stream)
        return {"workload": "compose n=14 complex64", "ms": ms, "coeffs_per_s": (1 << 28) / (ms * 1e-3),
                "algorithmic_bytes": 16 << 28}
    entry("compose_n14_fp32", comp, lambda ms: hbm(ms, 16 << 28))

    # a4: n = 15 (rows too long for one tile: strided HBM passes), FP32
    def n15():
        g.manual_seed(15)
        A15 = torch.randn((1 << 15, 1 << 15), generator=g, device=dev, dtype=torch.complex64)
        C15 = torch.empty_like(A15)
        ms = _timed(lambda: ptdr.decompose(A15, precision="fp32", out=C15), stream, reps=2)
        return {"workload": "dense n=15 complex64", "ms": ms, "coeffs_per_s": (1 << 30) / (ms * 1e-3),
                "algorithmic_bytes": 16 << 30}
    entry("dense_n15_fp32", n15, lambda ms: hbm(ms, 16 << 30))

    # dense n = 12 (L2 flushed between repetitions)
    def n12(prec, odt):
        def f():
            g.manual_seed(12)
            A12 = torch.randn((1 << 12, 1 << 12), generator=g, device=dev, dtype=torch.complex128)
            C12 = torch.empty_like(A12, dtype=odt)
            ms = _timed(lambda: ptdr.decompose(A12, precision=prec, out=C12), stream, flush=flush)
            return {"workload": f"dense n=12 complex128 -> {str(odt).split('.')[-1]} {prec}", "ms": ms,
                    "coeffs_per_s": (1 << 24) / (ms * 1e-3),
                    "algorithmic_bytes": (16 + C12.element_size()) << 24}
        return f
    entry("dense_n12_fp64", n12("fp64", torch.complex128), lambda ms: fp64(ms, 2 * 12 * (1 << 24)))
    entry("dense_n12_fp32", n12("fp32", torch.complex64),
          lambda ms: hbm(ms, rows["dense_n12_fp32"]["algorithmic_bytes"]))
    del flush_buf
    torch.cuda.empty_cache()
    return rows


def max_over_ranks(v: float, world: int, device) -> float:
    """The largest value of v over the ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(total_ms: float, steps: int, units_per_rank: int, world: int, device):
    """(ms per step, whole-job units/s): every rank processes units_per_rank per step
    (weak scaling) and the job takes as long as its slowest rank."""
    ms = max_over_ranks(total_ms, world, device) / steps
    return ms, world * units_per_rank / (ms * 1e-3)


def host_link(h_in, h_out, d_in, d_out, dev, reps=5):
    """The host link as the host-buffer path sees it: ms per copy of the input
    alone (host -> device), of the output alone (device -> host), and of both at
    the same time on two streams, plus the GB/s each way of the last.  A step of
    the host-buffer path moves its input in and its output out, so no step can
    take less than the slower of the two alone (the bound reported); a run near
    the sum of the two did not overlap them.  Whole-buffer copies in both
    directions at once have measured anywhere from the bound to well above the
    sum on these hosts (the host memory is shared with other jobs), so that
    figure is reported as context, not as the bound.  Each figure is the best
    of several copies timed one by one."""
    import torch
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def timed(fn):
        # best of `reps` copies timed one by one: the host memory is shared with
        # other jobs, so single copies can run several times slower than the link
        fn()
        torch.cuda.synchronize(dev)
        best = float("inf")
        for _ in range(reps):
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize(dev)
            best = min(best, (time.perf_counter() - t) * 1e3)
        return best

    def up_only():
        with torch.cuda.stream(up):
            d_in.copy_(h_in, non_blocking=True)

    def down_only():
        with torch.cuda.stream(down):
            h_out.copy_(d_out, non_blocking=True)

    def both():
        up_only()
        down_only()

    ms_up, ms_down, ms_both = timed(up_only), timed(down_only), timed(both)
    nbytes = min(h_in.numel() * h_in.element_size(), h_out.numel() * h_out.element_size())
    return {"up_ms": ms_up, "down_ms": ms_down, "both_ms": ms_both, "gbs_each_way": nbytes / (ms_both * 1e-3) / 1e9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, help="fp32 | fp64 | bf16x3 | fixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra-paths", action="store_true")
    ap.add_argument("--rows", default="all",
                    help="comma-separated context rows to measure (e.g. batched_512_fp32); "
                         "given explicitly, they run even with --no-extra-paths")
    ap.add_argument("--n", type=int, default=14, help="matrix size 2^n (profiling of smaller cases)")
    ap.add_argument("--batched-count", type=int, default=512,
                    help="matrices of the batched row: the first K of the seeded 512 (profiling of smaller cases)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _tree_rate(A, threads, seconds, cut=9):
    """Coefficients/s of the oracle's tree walk (Algorithms 1-4) over whole subtrees of
    the forest cut at level `cut`, `threads` subtrees per round, for about `seconds`."""
    import oracle
    n = A.shape[0].bit_length() - 1
    per_tree = 4 ** (n - cut)
    done, t0, nxt = 0, time.perf_counter(), 0
    while True:
        oracle.tree(A, cut=cut, subtrees=(nxt, nxt + threads), threads=threads)
        nxt += threads
        done += threads
        el = time.perf_counter() - t0
        if el >= seconds or nxt >= 4 ** cut:
            break
    return done * per_tree / el, done, el


def _direct_rate(A, threads, seconds):
    """Coefficients/s of the oracle's direct sparse trace (Sec. II.A) over whole mask
    rows (2^n coefficients each), `threads` masks per round, for about `seconds`."""
    import oracle
    N = A.shape[0]
    done, t0, nxt = 0, time.perf_counter(), 1
    while True:
        xs = (np.arange(nxt, nxt + threads) % N).astype(np.uint64)
        oracle.direct(A, xs=xs, threads=threads)
        nxt += threads
        done += threads
        el = time.perf_counter() - t0
        if el >= seconds or done >= N:
            break
    return done * N / el, done, el


def cpu_baseline(seconds=12.0):
    """The oracle on the host cores, on bounded samples of the n=14 workload.

    The headline value is the tree walk (Algorithms 1-4, forest split) on all
    cores; beside it, the same walk on one core, the direct sparse trace on all
    cores and on one core, and (labelled extra) the textbook FWHT check over the
    whole matrix."""
    import oracle
    import workloads

    A = workloads.dense_c64_direct(N_QUBITS, SEED).astype(np.complex128)
    threads = oracle.max_threads()
    v, done, el = _tree_rate(A, threads, seconds)
    v1, done1, el1 = _tree_rate(A, 1, seconds / 4)
    dv, ddone, del_ = _direct_rate(A, threads, seconds / 3)
    dv1, ddone1, del1 = _direct_rate(A, 1, seconds / 4)
    t0 = time.perf_counter()
    oracle.fwht(A, threads=threads)
    fw = time.perf_counter() - t0
    return {"value": v, "unit": "coeffs/s", "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{done} of {4 ** 9} subtrees (cut at level 9) of the n=14 tree walk, "
                      f"{done * 4 ** (N_QUBITS - 9)} coefficients in {el:.1f} s on {threads} threads",
            "modes": {
                "tree_all_cores": {"coeffs_per_s": v, "threads": threads, "seconds": el, "subtrees": done},
                "tree_1_core": {"coeffs_per_s": v1, "threads": 1, "seconds": el1, "subtrees": done1},
                "direct_all_cores": {"coeffs_per_s": dv, "threads": threads, "seconds": del_, "masks": ddone},
                "direct_1_core": {"coeffs_per_s": dv1, "threads": 1, "seconds": del1, "masks": ddone1},
                "fwht_check_all_cores_extra": {"coeffs_per_s": (1 << (2 * N_QUBITS)) / fw, "threads": threads,
                                               "seconds": fw, "note": "textbook FWHT check (not the paper's "
                                                                      "method), whole n=14 matrix"}}}


def path_accuracy(A_h, rows, xs):
    """Max relative error of each path's coefficients against the FP64 oracle on the
    sampled masks xs: max|c - c_ref| / max|c_ref| over those rows.  Runs after every
    GPU measurement, in the same host-side leg as the CPU baseline."""
    import oracle
    ref = oracle.fwht(A_h, xs=xs)
    den = float(np.max(np.abs(ref)))
    out = {}
    for p, got in rows.items():
        err = float(np.max(np.abs(got.astype(np.complex128) - ref))) / den
        out[p] = {"max_rel_err": err, "tolerance": TOLERANCE[p], "within": err <= TOLERANCE[p],
                  "masks": len(xs), "reference": "oracle FWHT check in FP64 on the same complex64 input"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = []
    base = None
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(seconds=4.0)
        if i >= args.warmup:
            steps.append(r["value"])
        base = r
    v = float(np.median(steps))
    base["value"] = v
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "coeffs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 2 ** (2 * N_QUBITS) / v * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "dense n=14 16384x16384 complex64 N(0,1), seed 14", "n": N_QUBITS,
                   "l2": "inputs larger than L2"},
        "cpu_baseline": base,
        "e2e": {"value": v, "unit": "coeffs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2403_11644_gb300 as ptdr
    import workloads
    from paper_2403_11644_gb300 import build as lib_build

    lib_build.build()
    global N_QUBITS
    N_QUBITS = args.n
    prec = args.precision or "bf16x3"
    out_dtype = torch.complex128 if prec in ("fp64", "fixed") else torch.complex64
    A_h = workloads.dense_c64_direct(N_QUBITS, (SEED if N_QUBITS == 14 else N_QUBITS) + rank)
    A = torch.from_numpy(A_h).to(dev)
    C = torch.empty((1 << N_QUBITS, 1 << N_QUBITS), dtype=out_dtype, device=dev)
    ncoef = 1 << (2 * N_QUBITS)
    stream = torch.cuda.current_stream(dev)
    ws_bytes = ptdr.workspace_size("decompose", N_QUBITS, A.dtype, out_dtype, prec)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)

    def step():
        ptdr.decompose(A, precision=prec, out=C, workspace=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
    total_ms = t0.elapsed_time(t1)
    # sampled rows of every path's output, checked against the oracle at the end
    xs = workloads.sample_masks(N_QUBITS, SEED, count=126)
    xs_t = torch.from_numpy(xs.astype(np.int64)).to(dev)
    acc_rows = {prec: C[xs_t].cpu().numpy()}
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = float(np.mean(launch_ms))
    ms_per_step, value = job_throughput(total_ms, args.steps, ncoef, world, dev)

    in_b = A.element_size() * A.numel()
    out_b = C.element_size() * C.numel()
    alg_bytes = in_b + out_b
    hbm_peak, peak_kind = peaks()
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    # our kernels per step: the n = 14 complex64 paths are one persistent launch
    # (plus a 4 KiB memset of the work-queue counters)
    launches_per_step = 1 if (N_QUBITS == 14 and prec in ("fp32", "bf16x3")) else None
    kernel_name, traffic = ncu_traffic(prec, N_QUBITS)

    result = None
    if rank == 0:
        result = {
            "metric": METRIC, "value": value, "unit": "coeffs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "bf16x3": "bf16x3->f32", "fixed": "i128"}[prec],
            "data": "synthetic",
            "config": {"workload": f"dense n={N_QUBITS} {1 << N_QUBITS}x{1 << N_QUBITS} complex64 N(0,1), "
                                   f"seed {SEED if N_QUBITS == 14 else N_QUBITS} (+rank)",
                       "n": N_QUBITS, "precision": prec, "output": str(out_dtype).split(".")[-1],
                       "l2": "inputs larger than L2 (2 GiB in, 2 GiB out), no flush",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "peak_source": peak_kind,
                         "traffic": traffic, "kernel": kernel_name,
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "kernel_ms": kern_ms},
            "clocks": clk.summary(),
            "gpu_launches": None if launches_per_step is None else launches_per_step * args.steps,
        }

    # end to end through the C ABI with host buffers (ptdr_decompose_host): every step
    # copies its matrix in from pinned host memory and its coefficients out; the call
    # overlaps the transfers of neighbouring steps
    if not args.no_e2e:
        A_pin = torch.from_numpy(A_h).pin_memory()
        C_pins = [torch.empty(C.shape, dtype=C.dtype).pin_memory() for _ in range(2)]
        # the host link this process sees (A is rewritten with its own values)
        link = host_link(A_pin, C_pins[0], A, C, dev)
        e2e_steps = max(3, min(args.steps, 20))  # the first upload and the last download are not overlapped
        scratch = torch.empty(ptdr.host_scratch_size(N_QUBITS, A.dtype, out_dtype, prec), dtype=torch.uint8,
                              device=dev)
        As = [A_pin] * e2e_steps
        Cs = [C_pins[i & 1] for i in range(e2e_steps)]
        ptdr.decompose_host(As[:2], Cs[:2], precision=prec, device=dev, scratch=scratch)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ptdr.decompose_host(As, Cs, precision=prec, device=dev, scratch=scratch)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e_ms, e_value = job_throughput(e0.elapsed_time(e1), e2e_steps, ncoef, world, dev)
        if rank == 0:
            result["e2e"] = {"value": e_value, "unit": "coeffs/s",
                             "h2d_bytes_per_step": in_b, "d2h_bytes_per_step": out_b,
                             "ms_per_step": e_ms, "steps": e2e_steps,
                             "link_gbs_each_way": link["gbs_each_way"],
                             "link_bound_ms_per_step": max(link["up_ms"], link["down_ms"]),
                             "link_up_alone_ms": link["up_ms"], "link_down_alone_ms": link["down_ms"],
                             "link_both_at_once_ms": link["both_ms"],
                             "link_serial_ms_per_step": link["up_ms"] + link["down_ms"],
                             "api": "ptdr_decompose_host (C ABI, host buffers, transfers overlapped across steps)"}
        del scratch

    # the other arithmetic paths on the same input, for context
    if rank == 0 and not args.no_extra_paths:
        extra = {prec: {"coeffs_per_s": ncoef / (kern_ms * 1e-3), "ms": kern_ms, "algorithmic_gbs": achieved,
                        "note": "the headline path, timed above"}}
        for p2, od in (("fp64", torch.complex128), ("fp32", torch.complex64), ("bf16x3", torch.complex64),
                       ("fixed", torch.complex128)):
            if p2 == prec:
                continue
            try:
                C2 = torch.empty(C.shape, dtype=od, device=dev)
                wsb = ptdr.workspace_size("decompose", N_QUBITS, A.dtype, od, p2)
                ws2 = torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev)
                def time_path():
                    for _ in range(2):
                        ptdr.decompose(A, precision=p2, out=C2, workspace=ws2)
                    torch.cuda.synchronize(dev)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    reps = 3
                    a.record(stream)
                    for _ in range(reps):
                        ptdr.decompose(A, precision=p2, out=C2, workspace=ws2)
                    b.record(stream)
                    torch.cuda.synchronize(dev)
                    return a.elapsed_time(b) / reps
                ms = time_path()
                extra[p2] = {"coeffs_per_s": ncoef / (ms * 1e-3), "ms": ms,
                             "algorithmic_gbs": (in_b + C2.element_size() * C2.numel()) / ms / 1e6}
                if p2 == "fp64":
                    # its rows (256 KiB) take a first pass and strided HBM passes: autotune
                    # their schedule on these buffers, then time the tuned plan
                    tuned = ptdr.autotune("decompose", A, C2, p2, workspace=ws2)
                    ms_t = time_path()
                    extra[p2].update({"ms_default_schedule": ms, "ms": ms_t, "schedule": tuned,
                                      "coeffs_per_s": ncoef / (ms_t * 1e-3),
                                      "algorithmic_gbs": (in_b + C2.element_size() * C2.numel()) / ms_t / 1e6})
                acc_rows[p2] = C2[xs_t].cpu().numpy()
                del C2, ws2
            except Exception as e:  # report, never hide
                extra[p2] = {"error": str(e)}
        result["paths"] = extra
        fp64_rate = fp64_add_rate(dev, stream)
        result["fp64_add_rate"] = {"adds_per_s": fp64_rate, "source": "measured in this run "
                                   "(ptdr_probe_fp64_adds: 8 add chains per thread, 8 CTAs x 256 threads per SM)"}
        result["rows"] = measure_rows(dev, stream, hbm_peak, fp64_rate, args.rows, args.batched_count)
    elif rank == 0 and args.rows != "all":
        fp64_rate = fp64_add_rate(dev, stream)
        result["rows"] = measure_rows(dev, stream, hbm_peak, fp64_rate, args.rows, args.batched_count)

    # host-side oracle leg (after every GPU measurement): accuracy of each path on
    # the sampled masks, then the CPU baseline
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        acc = path_accuracy(A_h, acc_rows, xs)
        result["accuracy"] = acc
        result["roofline"]["max_rel_err"] = acc[prec]["max_rel_err"]
        for p2, e in acc.items():
            if p2 in result.get("paths", {}):
                result["paths"][p2].update({"max_rel_err": e["max_rel_err"], "tolerance": e["tolerance"]})
        if N_QUBITS == 14:
            result["cpu_baseline"] = cpu_baseline()

    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
