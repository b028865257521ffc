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
    "fp32": {"kernel": "k_dense14_staged", "bytes": 2_157_797_000 + 2_158_074_000,
             "sources": {"paper_2403_11644_gb300/csrc/k_dense14s.cu":
                         "0ca9f8674df9a8b43490c448728f48d96a7bc33a9cbd206e4409619055ad01be",
                         "paper_2403_11644_gb300/csrc/common.cuh":
                         "f41af31f86534a7bc1c1c9a73b10f6d27e738589ae7e9bb8fe5f42eb0a9e6cc1"}},
}


def ncu_traffic(prec, n):
    """(kernel, bytes per launch) from the capture table, bytes None if stale."""
    import hashlib
    e = NCU_TRAFFIC.get(prec)
    if e is None or n != 14:
        return ({"bf16x3": "k_tc14_pipe"}.get(prec) if n == 14 else None), None
    for rel, sha in e["sources"].items():
        path = os.path.join(ROOT, rel)
        if not os.path.exists(path):
            return e["kernel"], None
        with open(path, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != sha:
                return e["kernel"], None
    return e["kernel"], e["bytes"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, help="fp32 | fp64 | bf16x3 | fp16x2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra-paths", action="store_true")
    ap.add_argument("--n", type=int, default=14, help="matrix size 2^n (profiling of smaller cases)")
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


def cpu_baseline(seconds=12.0):
    """The oracle's tree walk (Algorithms 1-4, forest split) on a bounded sample of the
    n=14 workload: whole subtrees of the forest cut at level 9 (1,024 coefficients each,
    every coefficient an O(2^14) trace), one subtree per core per round, as many rounds
    as fit the time budget."""
    import oracle
    import workloads

    A = workloads.dense_c64_direct(N_QUBITS, SEED).astype(np.complex128)
    threads = oracle.max_threads()
    cut = 9
    per_tree = 4 ** (N_QUBITS - cut)
    done, t0, nxt = 0, time.perf_counter(), 0
    while True:
        oracle.tree(A, cut=cut, subtrees=(nxt, nxt + threads), threads=threads)
        nxt += threads
        done += threads
        el = time.perf_counter() - t0
        if el >= seconds or nxt >= 4 ** cut:
            break
    return {"value": done * per_tree / el, "unit": "coeffs/s", "cores": threads, "kind": "oracle",
            "sample": f"{done} of {4 ** cut} subtrees (cut at level {cut}) of the n=14 tree walk, "
                      f"{done * per_tree} coefficients in {el:.1f} s"}


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
    out_dtype = torch.complex128 if prec == "fp64" else torch.complex64
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
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = float(np.mean(launch_ms))
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * ncoef / (ms_per_step * 1e-3)

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
            "dtype": {"fp32": "f32", "fp64": "f64", "bf16x3": "bf16x3->f32", "fp16x2": "fp16x2->f32"}[prec],
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

    # end to end through the public API from pinned host memory
    if not args.no_e2e:
        A_pin = torch.from_numpy(A_h).pin_memory()
        C_pin = torch.empty(C.shape, dtype=C.dtype).pin_memory()
        e2e_steps = max(2, min(args.steps, 5))
        for _ in range(2):
            A.copy_(A_pin, non_blocking=True)
            step()
            C_pin.copy_(C, non_blocking=True)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            A.copy_(A_pin, non_blocking=True)
            step()
            C_pin.copy_(C, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e_ms = e0.elapsed_time(e1) / e2e_steps
        if world > 1:
            t = torch.tensor([e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_ms = float(t.item())
        if rank == 0:
            result["e2e"] = {"value": world * ncoef / (e_ms * 1e-3), "unit": "coeffs/s",
                             "h2d_bytes_per_step": in_b, "d2h_bytes_per_step": out_b,
                             "ms_per_step": e_ms}

    # the other arithmetic paths on the same input, for context
    if rank == 0 and not args.no_extra_paths:
        extra = {}
        for p2, od in (("fp64", torch.complex128), ("fp32", torch.complex64), ("bf16x3", torch.complex64)):
            if p2 == prec:
                continue
            try:
                C2 = torch.empty(C.shape, dtype=od, device=dev)
                wsb = ptdr.workspace_size("decompose", N_QUBITS, A.dtype, od, p2)
                ws2 = torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev)
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
                ms = a.elapsed_time(b) / reps
                extra[p2] = {"coeffs_per_s": ncoef / (ms * 1e-3), "ms": ms,
                             "algorithmic_gbs": (in_b + C2.element_size() * C2.numel()) / ms / 1e6}
                del C2, ws2
            except Exception as e:  # report, never hide
                extra[p2] = {"error": str(e)}
        result["paths"] = extra

    if rank == 0 and world == 1 and N_QUBITS == 14 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline()

    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
