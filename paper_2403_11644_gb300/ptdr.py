"""PyTorch-facing API over libptdr's C ABI.

Torch supplies device memory and the current stream; every step of the
decomposition runs in libptdr's CUDA kernels.  Tensors must be CUDA tensors;
there is no CPU path.

Output layout: ``C[x, z] = c_{P(x,z)} = 2^-n tr(P A)`` with the paper's
PauliComposer masks (Sec. II.B): x_l = 1 for X/Y on qubit l, z_l = 1 for Y/Z;
qubit l is bit l of the row/column index (P = sigma_{n-1} (x) ... (x) sigma_0).
"""
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check

PRECISIONS = {
    "fp64": _lib.PREC_FP64,
    "fp32": _lib.PREC_FP32,
    "bf16x3": _lib.PREC_SPLIT_BF16_TC,
    "fixed": _lib.PREC_FIXED_I128,
}
_DT = {torch.complex64: _lib.C64, torch.complex128: _lib.C128, torch.float32: _lib.F32,
       torch.float64: _lib.F64}


def _dtype_code(t: torch.dtype) -> int:
    if t not in _DT:
        raise TypeError(f"unsupported dtype {t}")
    return _DT[t]


def _n_of(N: int) -> int:
    if N < 2 or N & (N - 1):
        raise ValueError("matrix size must be a power of two >= 2")
    return N.bit_length() - 1


def _stream(dev) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _cuda(t: torch.Tensor, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (libptdr has no CPU path)")
    return t.contiguous()


def _workspace(nbytes: int, dev) -> torch.Tensor:
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)


def _prec(precision: str) -> int:
    if precision not in PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
    return PRECISIONS[precision]


def workspace_size(op: str, n: int, a_dtype, c_dtype, precision: str) -> int:
    out = ctypes.c_size_t(0)
    code = _lib.OP_DECOMPOSE if op == "decompose" else _lib.OP_COMPOSE
    check(_lib.load().ptdr_workspace_size(code, n, _dtype_code(a_dtype), _dtype_code(c_dtype),
                                          _prec(precision), ctypes.byref(out)), "ptdr_workspace_size")
    return out.value


def decompose(A: torch.Tensor, precision: str = "fp32", out_dtype=None, out=None,
              workspace=None) -> torch.Tensor:
    """All 4^n coefficients ``C[x, z]`` of a 2^n x 2^n complex CUDA matrix."""
    A = _cuda(A, "A")
    n = _n_of(A.shape[0])
    if A.shape != (1 << n, 1 << n):
        raise ValueError("A must be square")
    if out_dtype is None:
        out_dtype = torch.complex128 if precision in ("fp64", "fixed") else torch.complex64
    C = out if out is not None else torch.empty((1 << n, 1 << n), dtype=out_dtype, device=A.device)
    ws_bytes = workspace_size("decompose", n, A.dtype, C.dtype, precision)
    ws = workspace if workspace is not None else (_workspace(ws_bytes, A.device) if ws_bytes else None)
    check(_lib.load().ptdr_decompose(
        ctypes.c_void_p(A.data_ptr()), _dtype_code(A.dtype), ctypes.c_void_p(C.data_ptr()),
        _dtype_code(C.dtype), n, _prec(precision),
        ctypes.c_void_p(ws.data_ptr() if ws is not None else 0), ws_bytes, _stream(A.device)),
        "ptdr_decompose")
    return C


def compose(C: torch.Tensor, scale: float = 1.0, precision: str = "fp32", out_dtype=None,
            out=None) -> torch.Tensor:
    """A = scale * sum_P C[P] P (the inverse of decompose for scale = 1)."""
    C = _cuda(C, "C")
    n = _n_of(C.shape[0])
    if out_dtype is None:  # real coefficients describe a Hermitian, complex A (Thm 2)
        out_dtype = {torch.float32: torch.complex64, torch.float64: torch.complex128}.get(C.dtype, C.dtype)
    A = out if out is not None else torch.empty((1 << n, 1 << n), dtype=out_dtype, device=C.device)
    ws_bytes = workspace_size("compose", n, A.dtype, C.dtype, precision)
    ws = _workspace(ws_bytes, C.device) if ws_bytes else None
    check(_lib.load().ptdr_compose(
        ctypes.c_void_p(C.data_ptr()), _dtype_code(C.dtype), ctypes.c_void_p(A.data_ptr()),
        _dtype_code(A.dtype), n, float(scale), _prec(precision),
        ctypes.c_void_p(ws.data_ptr() if ws is not None else 0), ws_bytes, _stream(C.device)),
        "ptdr_compose")
    return A


class TuneParams(ctypes.Structure):
    """ptdr_tune_params: the schedule of a multi-pass plan chosen by the autotuner."""
    _fields_ = [("tile_log2", ctypes.c_int), ("masks_log2", ctypes.c_int), ("pass_tile_log2", ctypes.c_int),
                ("threads", ctypes.c_int), ("ms", ctypes.c_double)]


def autotune(op: str, inp: torch.Tensor, out: torch.Tensor, precision: str, workspace=None) -> dict:
    """Times the candidate schedules of the strided HBM passes of decompose/compose on these
    buffers (out is overwritten) and caches the fastest for this GPU (and in the JSON file
    PTDR_TUNE_CACHE names).  Returns the chosen schedule and its time."""
    inp, out = _cuda(inp, "inp"), _cuda(out, "out")
    n = _n_of(inp.shape[0])
    code = _lib.OP_DECOMPOSE if op == "decompose" else _lib.OP_COMPOSE
    a_dt, c_dt = (inp.dtype, out.dtype) if op == "decompose" else (out.dtype, inp.dtype)
    wsb = workspace_size(op, n, a_dt, c_dt, precision)
    ws = workspace if workspace is not None else (_workspace(wsb, inp.device) if wsb else None)
    p = TuneParams()
    check(_lib.load().ptdr_autotune(
        code, n, _dtype_code(inp.dtype), _dtype_code(out.dtype), _prec(precision), ctypes.c_void_p(inp.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.data_ptr() if ws is not None else 0), wsb,
        _stream(inp.device), ctypes.byref(p)), "ptdr_autotune")
    return {"tile_log2": p.tile_log2, "masks_log2": p.masks_log2, "pass_tile_log2": p.pass_tile_log2,
            "threads": p.threads, "ms": p.ms}


def decompose_matrix_free(fill, n: int, a_dtype=torch.complex64, precision: str = "fp32", out_dtype=None,
                          device=None) -> torch.Tensor:
    """Decomposition of a 2^n x 2^n matrix that is never stored (Sec. V.B).

    ``fill(xt, a, S)`` must write into the CUDA tensor S (shape (2^a, 2^n), dtype
    a_dtype) the sheared tile set of x-block xt: S[i, k] = A[((k >> a) ^ xt) * 2^a + i, k],
    on the current stream.  Returns C[x, z]."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if out_dtype is None:
        out_dtype = torch.complex128 if precision == "fp64" else torch.complex64
    lib = _lib.load()
    wsz = ctypes.c_size_t(0)
    check(lib.ptdr_matrix_free_workspace_size(n, _dtype_code(a_dtype), _dtype_code(out_dtype), _prec(precision),
                                              ctypes.byref(wsz)), "ptdr_matrix_free_workspace_size")
    ws = torch.empty(wsz.value, dtype=torch.uint8, device=dev)
    a = min(7, n)
    S = ws[: (1 << (a + n)) * torch.empty((), dtype=a_dtype).element_size()].view(a_dtype).view(1 << a, 1 << n)
    C = torch.empty((1 << n, 1 << n), dtype=out_dtype, device=dev)
    errors = []

    def cb(_user, n_, xt, a_, d_s, _stream):
        try:
            assert d_s == S.data_ptr() and a_ == a and n_ == n
            fill(int(xt), a, S)
            return 0
        except Exception as exc:  # reported after the call
            errors.append(exc)
            return 1

    fn = _lib.TILE_FN(cb)
    st = lib.ptdr_decompose_matrix_free(n, _dtype_code(a_dtype), ctypes.cast(fn, ctypes.c_void_p), None,
                                        ctypes.c_void_p(C.data_ptr()), _dtype_code(out_dtype), _prec(precision),
                                        ctypes.c_void_p(ws.data_ptr()), wsz.value, _stream(dev))
    if errors:
        raise errors[0]
    check(st, "ptdr_decompose_matrix_free")
    return C


def host_scratch_size(n: int, a_dtype, c_dtype, precision: str) -> int:
    """Device scratch bytes that decompose_host needs (two A, two C buffers, workspace)."""
    out = ctypes.c_size_t(0)
    check(_lib.load().ptdr_decompose_host_scratch_size(n, _dtype_code(a_dtype), _dtype_code(c_dtype),
                                                       _prec(precision), ctypes.byref(out)),
          "ptdr_decompose_host_scratch_size")
    return out.value


def decompose_host(As, Cs, precision: str = "fp32", device=None, scratch=None):
    """Decomposes host (CPU) matrices As[i] into host outputs Cs[i] through the C ABI.

    The call copies each matrix in, decomposes it and copies the coefficients out,
    overlapping the transfers of neighbouring matrices; pinned tensors let the copies
    overlap.  Returns once the work is enqueued on the current stream of `device`
    (synchronise before reading Cs)."""
    if len(As) != len(Cs) or not As:
        raise ValueError("As and Cs must be non-empty lists of equal length")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    n = _n_of(As[0].shape[0])
    a_t, c_t = As[0].dtype, Cs[0].dtype
    for a, c in zip(As, Cs):
        if a.is_cuda or c.is_cuda:
            raise ValueError("decompose_host takes host tensors")
        if a.shape != (1 << n, 1 << n) or c.shape != (1 << n, 1 << n) or a.dtype != a_t or c.dtype != c_t:
            raise ValueError("all matrices must have the same size and dtypes")
        if not (a.is_contiguous() and c.is_contiguous()):
            raise ValueError("host tensors must be contiguous")
    need = host_scratch_size(n, a_t, c_t, precision)
    if scratch is None:
        scratch = torch.empty(need, dtype=torch.uint8, device=dev)
    k = len(As)
    ha = (ctypes.c_void_p * k)(*[a.data_ptr() for a in As])
    hc = (ctypes.c_void_p * k)(*[c.data_ptr() for c in Cs])
    check(_lib.load().ptdr_decompose_host(
        ctypes.cast(ha, ctypes.c_void_p), ctypes.cast(hc, ctypes.c_void_p), k, _dtype_code(a_t), _dtype_code(c_t),
        n, _prec(precision), ctypes.c_void_p(scratch.data_ptr()), scratch.numel(), _stream(dev)),
        "ptdr_decompose_host")
    return Cs


def structured_masks(n: int, s: int, anti: bool = False) -> np.ndarray:
    """Masks reachable by a band matrix of half-width s (host computation); with
    anti=True, by an anti-band matrix (the band's masks XOR 2^n - 1)."""
    lib = _lib.load()
    fn = lib.ptdr_antistructured_masks if anti else lib.ptdr_structured_masks
    cnt = ctypes.c_size_t(0)
    check(fn(n, s, None, ctypes.byref(cnt)), "ptdr_structured_masks")
    out = np.zeros(cnt.value, np.uint64)
    check(fn(n, s, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)), "ptdr_structured_masks")
    return out


def decompose_structured(bands: torch.Tensor, s: int, masks=None, precision: str = "fp64",
                         out_dtype=None, workspace=None, out=None, anti: bool = False) -> torch.Tensor:
    """Coefficients of a band matrix on its reachable masks (rows follow ``masks``).

    ``bands`` has shape (2s+1, 2^n) with bands[d+s, c] = A[c+d, c].  With anti=True
    A is anti-band and bands[d+s, c] = A[c+d, 2^n-1-c] (Remark 1 of Sec. IV.A).
    """
    bands = _cuda(bands, "bands")
    if bands.ndim != 2 or bands.shape[0] != 2 * s + 1:
        raise ValueError("bands must have shape (2s+1, 2^n)")
    n = _n_of(bands.shape[1])
    h_masks = structured_masks(n, s, anti) if masks is None else np.ascontiguousarray(masks, np.uint64)
    if out_dtype is None:
        if anti:  # anti-band coefficients are complex even for real storage
            out_dtype = torch.complex128 if precision == "fp64" else torch.complex64
        else:
            out_dtype = bands.dtype if not bands.dtype.is_complex else (
                torch.complex128 if precision == "fp64" else torch.complex64)
    C = out if out is not None else torch.empty((len(h_masks), 1 << n), dtype=out_dtype,
                                                device=bands.device)
    lib = _lib.load()
    hp = h_masks.ctypes.data_as(ctypes.c_void_p)
    wsz = ctypes.c_size_t(0)
    size_fn = lib.ptdr_antistructured_workspace_size if anti else lib.ptdr_structured_workspace_size
    check(size_fn(n, s, hp, len(h_masks), _dtype_code(bands.dtype), _dtype_code(C.dtype), _prec(precision),
                  ctypes.byref(wsz)), "ptdr_structured_workspace_size")
    ws = workspace if workspace is not None else (_workspace(wsz.value, bands.device) if wsz.value else None)
    run_fn = lib.ptdr_decompose_antistructured if anti else lib.ptdr_decompose_structured
    check(run_fn(
        ctypes.c_void_p(bands.data_ptr()), _dtype_code(bands.dtype), n, s,
        hp, len(h_masks), ctypes.c_void_p(C.data_ptr()),
        _dtype_code(C.dtype), _prec(precision),
        ctypes.c_void_p(ws.data_ptr() if ws is not None else 0), wsz.value, _stream(bands.device)),
        "ptdr_decompose_structured")
    return C


# ----------------------------------------------------------- decomposition algebra


def _coeff_n(C: torch.Tensor, name: str) -> int:
    if C.ndim != 2 or C.shape[0] != C.shape[1]:
        raise ValueError(f"{name} must be a square 2^n x 2^n coefficient array")
    return _n_of(C.shape[0])


def lincomb(mu, CA: torch.Tensor, CB: torch.Tensor = None, out=None) -> torch.Tensor:
    """Coefficients of mu A + B from those of A and B (Sec. IV.B.3): mu * CA + CB."""
    CA = _cuda(CA, "CA")
    n = _coeff_n(CA, "CA")
    if CB is not None:
        CB = _cuda(CB, "CB")
        if CB.shape != CA.shape or CB.dtype != CA.dtype:
            raise ValueError("CA and CB must have the same shape and dtype")
    C = out if out is not None else torch.empty_like(CA)
    mu = complex(mu)
    check(_lib.load().ptdr_coeff_lincomb(
        n, mu.real, mu.imag, ctypes.c_void_p(CA.data_ptr()),
        ctypes.c_void_p(CB.data_ptr() if CB is not None else 0), ctypes.c_void_p(C.data_ptr()),
        _dtype_code(CA.dtype), _stream(CA.device)), "ptdr_coeff_lincomb")
    return C


def block_diag(blocks, out=None) -> torch.Tensor:
    """Coefficients of diag(A_0, ..., A_{2^m-1}) from those of the 2^m blocks
    (Sec. IV.B.1-2; two blocks = the direct sum A (+) B)."""
    blocks = [_cuda(b, "block") for b in blocks]
    k = len(blocks)
    if k < 2 or k & (k - 1):
        raise ValueError("need 2^m blocks, m >= 1")
    m = k.bit_length() - 1
    n = _coeff_n(blocks[0], "block")
    for b in blocks:
        if b.shape != blocks[0].shape or b.dtype != blocks[0].dtype:
            raise ValueError("blocks must have the same shape and dtype")
    C = out if out is not None else torch.empty((1 << (n + m), 1 << (n + m)), dtype=blocks[0].dtype,
                                                device=blocks[0].device)
    ptrs = (ctypes.c_void_p * k)(*[b.data_ptr() for b in blocks])
    check(_lib.load().ptdr_coeff_block_diag(n, m, ctypes.cast(ptrs, ctypes.c_void_p), ctypes.c_void_p(C.data_ptr()),
                                            _dtype_code(C.dtype), _stream(C.device)), "ptdr_coeff_block_diag")
    return C


def hermitian_augment(CA: torch.Tensor, out_dtype=None, out=None) -> torch.Tensor:
    """Coefficients of [[0, A^H], [A, 0]] (n + 1 qubits) from those of A (Sec. IV.B.5)."""
    CA = _cuda(CA, "CA")
    n = _coeff_n(CA, "CA")
    if out_dtype is None:
        out_dtype = torch.float64 if CA.dtype in (torch.complex128, torch.float64) else torch.float32
    C = out if out is not None else torch.empty((2 << n, 2 << n), dtype=out_dtype, device=CA.device)
    check(_lib.load().ptdr_coeff_hermitian_augment(
        n, ctypes.c_void_p(CA.data_ptr()), _dtype_code(CA.dtype), ctypes.c_void_p(C.data_ptr()),
        _dtype_code(C.dtype), _stream(CA.device)), "ptdr_coeff_hermitian_augment")
    return C


def select(C: torch.Tensor, threshold: float = 0.0, k: int = 0):
    """Sparse form of a decomposition for an LCU block-encoding (Sec. VI).

    Returns (indices, values, l1): the indices x * 2^n + z (ascending, int64) of the
    coefficients with |c| > threshold (the k largest of them when k > 0; ties go to the
    lower index), their values, and the normaliser sum |alpha_i| over them.  With no
    k the count is read back first (one synchronisation) to size the outputs."""
    C = _cuda(C, "C")
    n = _coeff_n(C, "C")
    lib = _lib.load()
    wsz = ctypes.c_size_t(0)
    check(lib.ptdr_select_workspace_size(ctypes.byref(wsz)), "ptdr_select_workspace_size")
    ws = _workspace(wsz.value, C.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=C.device)
    l1 = torch.zeros(1, dtype=torch.float64, device=C.device)

    def run(cap, idx, val):
        check(lib.ptdr_coeff_select(
            n, ctypes.c_void_p(C.data_ptr()), _dtype_code(C.dtype), float(threshold), int(k),
            ctypes.c_void_p(idx.data_ptr() if idx is not None else 0),
            ctypes.c_void_p(val.data_ptr() if val is not None else 0), cap,
            ctypes.c_void_p(cnt.data_ptr()), ctypes.c_void_p(l1.data_ptr()),
            ctypes.c_void_p(ws.data_ptr()), wsz.value, _stream(C.device)), "ptdr_coeff_select")

    if k > 0:
        cap = min(int(k), C.numel())
    else:
        run(0, None, None)
        cap = int(cnt.item())
    idx = torch.empty(max(cap, 1), dtype=torch.int64, device=C.device)
    val = torch.empty(max(cap, 1), dtype=C.dtype, device=C.device)
    run(cap, idx, val)
    m = int(cnt.item())
    return idx[:m], val[:m], float(l1.item())


class BatchedPlan:
    """Device-side pointer/size tables and workspace for ptdr_decompose_batched.

    Built once per list of matrices; ``run()`` enqueues the persistent launch,
    so a CUDA graph can capture it and replay it with new data in the same
    buffers.
    """

    def __init__(self, As, Cs, precision: str = "fp32"):
        if len(As) != len(Cs) or not As:
            raise ValueError("need matching non-empty input/output lists")
        dev = As[0].device
        self.As, self.Cs = As, Cs
        self.h_n = np.array([_n_of(a.shape[0]) for a in As], np.int32)
        self.d_A = torch.tensor([a.data_ptr() for a in As], dtype=torch.int64, device=dev)
        self.d_C = torch.tensor([c.data_ptr() for c in Cs], dtype=torch.int64, device=dev)
        self.d_n = torch.from_numpy(self.h_n).to(dev)
        self.a_t, self.c_t = _dtype_code(As[0].dtype), _dtype_code(Cs[0].dtype)
        self.prec = _prec(precision)
        wsz = ctypes.c_size_t(0)
        check(_lib.load().ptdr_batched_workspace_size(
            self.h_n.ctypes.data_as(ctypes.c_void_p), len(As), self.a_t, self.c_t, self.prec,
            ctypes.byref(wsz)), "ptdr_batched_workspace_size")
        self.ws = _workspace(wsz.value, dev)
        self.ws_bytes = wsz.value
        self.device = dev

    def run(self):
        check(_lib.load().ptdr_decompose_batched(
            ctypes.c_void_p(self.d_A.data_ptr()), ctypes.c_void_p(self.d_C.data_ptr()),
            ctypes.c_void_p(self.d_n.data_ptr()), self.h_n.ctypes.data_as(ctypes.c_void_p),
            len(self.As), self.a_t, self.c_t, self.prec, ctypes.c_void_p(self.ws.data_ptr()),
            self.ws_bytes, _stream(self.device)), "ptdr_decompose_batched")
        return self.Cs


def decompose_batched(As, precision: str = "fp32", out_dtype=torch.complex64):
    """Decomposes a list of CUDA matrices of possibly different sizes in one launch."""
    As = [_cuda(a, "A") for a in As]
    Cs = [torch.empty_like(a, dtype=out_dtype) for a in As]
    return BatchedPlan(As, Cs, precision).run()


def last_device_status(device=None) -> int:
    """Synchronises the current stream and returns (and clears) the device status word."""
    dev = torch.device("cuda") if device is None else torch.device(device)
    return _lib.load().ptdr_last_device_status(_stream(dev))


class PtdrDecompose(torch.autograd.Function):
    """c = decompose(A); backward is the adjoint 2^-n * compose(grad_c).

    c_P = 2^-n <P, A> is linear in A, so the vector-Jacobian product of a
    gradient g (PyTorch's convention for complex tensors) is
    2^-n sum_P g_P P, i.e. ptdr_compose with scale = 2^-n.
    """

    @staticmethod
    def forward(ctx, A, precision="fp64"):
        ctx.precision = precision
        ctx.a_dtype = A.dtype
        return decompose(A, precision=precision, out_dtype=A.dtype)

    @staticmethod
    def backward(ctx, grad_c):
        n = _n_of(grad_c.shape[0])
        prec = "fp64" if ctx.precision == "fp64" else "fp32"
        gA = compose(grad_c.contiguous(), scale=2.0 ** (-n), precision=prec, out_dtype=ctx.a_dtype)
        return gA, None


def decompose_autograd(A: torch.Tensor, precision: str = "fp64") -> torch.Tensor:
    return PtdrDecompose.apply(A, precision)
