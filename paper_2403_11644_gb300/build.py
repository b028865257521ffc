"""Builds libptdr.so in-tree (paper_2403_11644_gb300/_build/) with nvcc for sm_103a.

Each .cu translation unit compiles in parallel; the shared library links them
against the CUDA runtime.  Set PTDR_CHECKED=1 for the bounds-checked variant
(every computed global index is range-checked in device code; a bad index is
recorded in the device status word and the access skipped), built as
libptdr_checked.so.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def lib_path(checked: bool = False) -> str:
    return os.path.join(OUT, "libptdr_checked.so" if checked else "libptdr.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(HERE, "..", "include", "ptdr.h"), os.path.abspath(__file__)]


def _stamp(lib: str) -> str:
    return lib + ".sources"


def _source_list() -> str:
    return "\n".join(os.path.basename(s) for s in _sources())


def build(checked: bool = False, force: bool = False, verbose: bool = False) -> str:
    lib = lib_path(checked)
    if not force and os.path.exists(lib) and os.path.exists(_stamp(lib)):
        t = os.path.getmtime(lib)
        with open(_stamp(lib)) as f:
            same_sources = f.read() == _source_list()  # a source added or removed also rebuilds
        if same_sources and all(os.path.getmtime(d) <= t for d in _deps()):
            return lib
    os.makedirs(OUT, exist_ok=True)
    tag = "checked" if checked else "release"
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                    "-Xptxas", "-v", "-I", os.path.join(HERE, "..", "include")]
    if checked:
        flags += ["-DPTDR_CHECKED=1"]
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(OUT, f"{os.path.basename(src)[:-3]}.{tag}.o")
        log = obj + ".ptxas.txt"
        r = subprocess.run([cc, *flags, "-c", src, "-o", obj], capture_output=True, text=True)
        with open(log, "w") as f:
            f.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr[-4000:]}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = lib + ".tmp"
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "shared", "-ldl",
                           "-Xlinker", "-rpath,/usr/local/cuda/lib64"])
    os.replace(tmp, lib)
    with open(_stamp(lib), "w") as f:
        f.write(_source_list())
    if verbose:
        print(lib)
    return lib


if __name__ == "__main__":
    build(checked="--checked" in sys.argv, force="--force" in sys.argv, verbose=True)
