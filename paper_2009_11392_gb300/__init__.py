"""GB300 generalized Nystrom (GN) low-rank approximation -- Python binding.

A thin ctypes layer over the C ABI declared in ``include/gn.h`` (library
``_build/libgn.so``).  It only marshals torch tensors into ``gn_mat`` /
``gn_core_t`` descriptors and checks return codes; every step of the method
runs in the library's CUDA kernels.  PyTorch supplies device memory and the
stream.  There is no CPU fallback: importing the package fails when the
shared library is missing, and every call raises on a non-OK status.

Entry points (same names as the C ABI):
    quantize, sketch, core, factors, approx, error_fro2, hmt
plus ``workspace`` (sized by gn_workspace_size) and ``Core`` (the small
factors of Section 5.1 held in caller-owned tensors).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

__all__ = [
    "GNError", "Handle", "Core", "lib_path", "lib", "F64", "F32", "BF16", "BF16X2",
    "PLAIN", "SGN", "AUTO", "EPS_RELATIVE", "ABI_SYMBOLS", "mat", "round8", "padded",
]

F64, F32, BF16, BF16X2, E4M3 = 0, 1, 2, 3, 4
PLAIN, SGN, AUTO = 0, 1, 2
SVD_TRUNCATE, SVD_RAISE, RRQR_RAISE, DIAG_RAISE = 0, 1, 2, 3
EPS_RELATIVE = 0x100
CORE_DEFER = 0x200
CORE_C_GIVEN = 0x400

# Every symbol declared in include/gn.h.
ABI_SYMBOLS = (
    "gn_create", "gn_destroy", "gn_set_stream", "gn_sync_status", "gn_set_wait_limit", "gn_set_fp64_g",
    "gn_status_string", "gn_device_sm_count", "gn_workspace_size", "gn_quantize",
    "gn_sketch", "gn_core", "gn_factors", "gn_approx", "gn_error_fro2", "gn_hmt",
    "gn_kernel_launches", "gn_error_fro2_noalloc", "gn_backward_workspace_size", "gn_backward",
    "gn_forward_dense", "gn_backward_saved", "gn_batched_workspace_size", "gn_batched_prepare", "gn_batched_run",
    "gn_batched_set_policy", "gn_batched_tune", "gn_set_fp64_tc", "gn_dgemm_tc_workspace_size", "gn_dgemm_tc",
    "gn_apply_workspace_size", "gn_apply", "gn_update_workspace_size", "gn_update", "gn_resample",
    "gn_append_rows", "gn_append_cols", "gn_resample_workspace_size", "gn_core_finish",
    "gn_set_stall_test", "gn_dct_sketch", "gn_sketch_csr_countsketch", "gn_countsketch_matrix",
    "gn_countsketch_apply", "gn_set_fp64_accum", "gn_variant_workspace_size", "gn_factors_variant",
)


class GnMat(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("lo", ctypes.c_void_p), ("rows", ctypes.c_int64),
                ("cols", ctypes.c_int64), ("ld", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("scale", ctypes.c_void_p), ("data_t", ctypes.c_void_p), ("ld_t", ctypes.c_int64)]


class GnCsr(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("vals", ctypes.c_void_p),
                ("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("dtype", ctypes.c_int32)]


class GnProblem(ctypes.Structure):
    _fields_ = [("A", GnMat), ("X", GnMat), ("Y", GnMat), ("AX", GnMat), ("YtA", GnMat),
                ("Q", ctypes.c_void_p), ("R", ctypes.c_void_p), ("Q2", ctypes.c_void_p),
                ("R2", ctypes.c_void_p), ("k", ctypes.c_void_p)]


class GnCoreT(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_void_p), ("R", ctypes.c_void_p), ("Q2", ctypes.c_void_p),
                ("R2", ctypes.c_void_p), ("C", ctypes.c_void_p), ("r", ctypes.c_int64),
                ("l", ctypes.c_int64), ("k", ctypes.c_int64), ("sgn", ctypes.c_int32),
                ("rinv_est", ctypes.c_double), ("c_norm_est", ctypes.c_double),
                ("eps_abs", ctypes.c_double)]


def kernel_launches() -> int:
    """Kernels launched so far by the library in this process."""
    return int(lib.gn_kernel_launches())


def lib_path() -> str:
    return _build.LIB


def _load():
    path = _build.LIB
    if not os.path.exists(path) or _build.stale():
        if os.environ.get("GN_AUTOBUILD", "1") == "1":
            _build.build()
        if not os.path.exists(path):
            raise ImportError(f"GN CUDA library not built: {path} is missing (run the package's build.py)")
    L = ctypes.CDLL(path)
    P, I32, I64, D, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    M = ctypes.POINTER(GnMat)
    C = ctypes.POINTER(GnCoreT)
    sig = {
        "gn_create": ([ctypes.POINTER(P), P], I32),
        "gn_destroy": ([P], I32),
        "gn_set_stream": ([P, P], I32),
        "gn_sync_status": ([P], I32),
        "gn_set_wait_limit": ([P, ctypes.c_uint64], I32),
        "gn_set_stall_test": ([P, I32], I32),
        "gn_set_fp64_accum": ([P, I64], I32),
        "gn_variant_workspace_size": ([I64, I64, I64, I64, ctypes.POINTER(SZ)], I32),
        "gn_factors_variant": ([P, M, M, M, D, I32, M, M, ctypes.POINTER(I64), P, P, SZ], I32),
        "gn_dct_sketch": ([P, I64, I64, P, P, M], I32),
        "gn_sketch_csr_countsketch": ([P, ctypes.POINTER(GnCsr), P, P, P, P, M, M], I32),
        "gn_countsketch_matrix": ([P, I64, I64, P, P, M], I32),
        "gn_countsketch_apply": ([P, M, P, P, M], I32),
        "gn_set_fp64_g": ([P, I32], I32),
        "gn_status_string": ([I32], ctypes.c_char_p),
        "gn_device_sm_count": ([P], ctypes.c_int),
        "gn_workspace_size": ([I64, I64, I64, I64, I32, ctypes.POINTER(SZ)], I32),
        "gn_quantize": ([P, M, M], I32),
        "gn_sketch": ([P, M, M, M, M, M, P, SZ], I32),
        "gn_core": ([P, M, M, D, I32, C, P, SZ], I32),
        "gn_core_finish": ([P, C], I32),
        "gn_factors": ([P, M, M, C, M, M, P, SZ], I32),
        "gn_approx": ([P, M, M, M, D, I32, M, M, C, M, M, P, SZ], I32),
        "gn_error_fro2": ([P, M, M, M, P, P, SZ], I32),
        "gn_hmt": ([P, M, M, M, M, P, SZ], I32),
        "gn_kernel_launches": ([], ctypes.c_uint64),
        "gn_error_fro2_noalloc": ([P, M, M, M, P], I32),
        "gn_backward_workspace_size": ([I64, I64, I64, I64, I32, ctypes.POINTER(SZ)], I32),
        "gn_backward": ([P, M, M, M, M, M, P, SZ], I32),
        "gn_forward_dense": ([P, M, M, M, M, P, SZ], I32),
        "gn_backward_saved": ([P, M, M, M, M, P, SZ], I32),
        "gn_batched_workspace_size": ([I32, ctypes.POINTER(GnProblem), ctypes.POINTER(SZ)], I32),
        "gn_batched_prepare": ([P, I32, ctypes.POINTER(GnProblem), P, SZ], I32),
        "gn_batched_run": ([P, D, I32, P, SZ], I32),
        "gn_batched_set_policy": ([P, I32], I32),
        "gn_set_fp64_tc": ([P, I32], I32),
        "gn_apply_workspace_size": ([I64, I64, I64, I64, I64, I32, ctypes.POINTER(SZ)], I32),
        "gn_apply": ([P, M, M, C, M, M, I32, P, SZ], I32),
        "gn_update_workspace_size": ([I64, I64, I64, I64, I32, ctypes.POINTER(SZ)], I32),
        "gn_update": ([P, M, M, M, M, M, P, SZ], I32),
        "gn_resample": ([P, M, M, M, M, M, M, M, P, SZ], I32),
        "gn_resample_workspace_size": ([I64, I64, I64, I64, I32, ctypes.POINTER(SZ)], I32),
        "gn_append_rows": ([P, M, M, M, M, M, M, P, SZ], I32),
        "gn_append_cols": ([P, M, M, M, M, M, M, P, SZ], I32),
        "gn_dgemm_tc_workspace_size": ([I64, I64, I64, I32, ctypes.POINTER(SZ)], I32),
        "gn_dgemm_tc": ([P, I64, I64, I64, D, P, I32, I64, I32, P, I64, I32, D, P, I64, P, SZ], I32),
        "gn_batched_tune": ([P, I32, ctypes.POINTER(GnProblem), P, SZ, D, I32, ctypes.POINTER(I32),
                             ctypes.POINTER(D)], I32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


class GNError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.gn_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def _check(status: int, where: str):
    if status != 0:
        raise GNError(status, where)


_TORCH_DT = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}


def round8(x: int) -> int:
    return (x + 7) // 8 * 8


def mat(t, lo: torch.Tensor | None = None) -> GnMat:
    """gn_mat for a row-major 2-D CUDA tensor (stride (ld, 1)); ``lo`` makes it
    split bf16; an E4M3Mat maps to its e4m3 description."""
    if isinstance(t, E4M3Mat):
        return t.gnmat()
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("operands must be 2-D row-major (stride(1) == 1)")
    if not t.is_cuda:
        raise ValueError("operands must be CUDA tensors")
    dt = _TORCH_DT.get(t.dtype)
    if dt is None:
        raise ValueError(f"unsupported dtype {t.dtype}")
    ld = t.stride(0) if t.shape[0] > 1 else max(t.shape[1], t.stride(0))
    m = GnMat(t.data_ptr(), 0, t.shape[0], t.shape[1], ld, dt)
    if lo is not None:
        if lo.shape != t.shape or lo.stride() != t.stride() or lo.dtype != torch.bfloat16:
            raise ValueError("lo must match data in shape, stride and bf16 dtype")
        m.lo = lo.data_ptr()
        m.dtype = BF16X2
    return m


@dataclass
class E4M3Mat:
    """An e4m3 operand with one power-of-two scale per 128 x 128 tile.

    ``data`` (rows x cols) and ``data_t`` (cols x rows) hold the codes as uint8
    views with leading dimensions that are multiples of 16 (either may be None);
    ``scale`` holds one UE8M0 byte (exponent + 127) per tile, row-major over the
    tiles of the rows x cols matrix."""
    rows: int
    cols: int
    scale: torch.Tensor
    data: torch.Tensor | None = None
    data_t: torch.Tensor | None = None

    def gnmat(self) -> "GnMat":
        m = GnMat(self.data.data_ptr() if self.data is not None else 0, 0, self.rows, self.cols,
                  self.data.stride(0) if self.data is not None else 0, E4M3)
        m.scale = self.scale.data_ptr()
        if self.data_t is not None:
            m.data_t = self.data_t.data_ptr()
            m.ld_t = self.data_t.stride(0)
        return m

    def values(self) -> torch.Tensor:
        """The FP64 values code * 2^e (rows x cols) on the device, from ``data``
        or ``data_t``."""
        # 2^e exactly, from the FP64 bit pattern (a power function need not be exact)
        sc = ((self.scale.to(torch.int64) - 127 + 1023) << 52).view(torch.float64)
        sc = sc.repeat_interleave(128, 0).repeat_interleave(128, 1)[: self.rows, : self.cols]
        if self.data is not None:
            v = self.data.view(torch.float8_e4m3fn).to(torch.float64)
        else:
            v = self.data_t.view(torch.float8_e4m3fn).to(torch.float64).t()
        return (v * sc).contiguous()


def _cols(t) -> int:
    return t.cols if isinstance(t, E4M3Mat) else int(t.shape[1])


def _mat_or_empty(t, rows: int) -> GnMat:
    """gn_mat of ``t``, or for a tensor with no columns a descriptor with the
    right row count that the library does not read."""
    if not isinstance(t, E4M3Mat) and t.dim() == 2 and t.shape[1] == 0:
        return GnMat(0, 0, rows, 0, 0, _TORCH_DT.get(t.dtype, F32))
    return mat(t)


def padded(rows: int, cols: int, dtype, device) -> torch.Tensor:
    """An uninitialised rows x cols tensor whose leading dimension is a multiple
    of 8 elements (the TMA rule for bf16 operands)."""
    return torch.empty(rows, round8(cols), dtype=dtype, device=device)[:, :cols]


@dataclass
class Core:
    C: torch.Tensor
    Q: torch.Tensor
    R: torch.Tensor
    Q2: torch.Tensor
    R2: torch.Tensor
    r: int
    l: int
    k: int = 0
    sgn: int = 0
    rinv_est: float = 0.0
    c_norm_est: float = 0.0
    eps_abs: float = 0.0

    @staticmethod
    def empty(r: int, l: int, device) -> "Core":
        z = lambda a, b: torch.empty(a, b, dtype=torch.float64, device=device)
        return Core(z(r + l, r), z(r + l, r), z(r, r), z(r, r), z(r, r), r, l)

    def cstruct(self) -> GnCoreT:
        return GnCoreT(self.Q.data_ptr(), self.R.data_ptr(), self.Q2.data_ptr(), self.R2.data_ptr(),
                       self.C.data_ptr(), self.r, self.l, self.k, self.sgn, self.rinv_est,
                       self.c_norm_est, self.eps_abs)

    def update(self, c: GnCoreT):
        self.k, self.sgn, self.rinv_est = int(c.k), int(c.sgn), float(c.rinv_est)
        self.c_norm_est, self.eps_abs = float(c.c_norm_est), float(c.eps_abs)


class Handle:
    """Owns a gn_handle bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("GN needs a CUDA device; there is no CPU path")
        self.stream = stream or torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib.gn_create(ctypes.byref(h), ctypes.c_void_p(self.stream.cuda_stream)), "gn_create")
        self._h = h
        self.front_calls = 0   # gn_forward_dense / gn_backward calls (each leaves a front in its ws)

    @property
    def h(self):
        return self._h

    def close(self):
        if self._h:
            lib.gn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sm_count(self) -> int:
        return lib.gn_device_sm_count(self._h)

    def sync_status(self) -> int:
        return lib.gn_sync_status(self._h)

    def set_wait_limit(self, ns: int):
        _check(lib.gn_set_wait_limit(self._h, int(ns)), "gn_set_wait_limit")

    def set_stall_test(self, on: bool):
        """Test hook: sketch launches wait on a barrier nothing completes, so
        the bounded wait runs out (GN_ERR_TIMEOUT)."""
        _check(lib.gn_set_stall_test(self._h, 1 if on else 0), "gn_set_stall_test")

    def set_fp64_g(self, on: bool):
        """G = Q_1^T (Y^T A) in FP64 (True) or on the tensor cores (False, default) for FP32 Y^T A."""
        _check(lib.gn_set_fp64_g(self._h, 1 if on else 0), "gn_set_fp64_g")

    def set_fp64_accum(self, part_k: int):
        """FP64-level accumulation (split-BF16 sketches in stored K parts summed in
        FP64, digit-sliced C, FP64 G): part_k >= 4096 K elements per part, 0 off."""
        _check(lib.gn_set_fp64_accum(self._h, int(part_k)), "gn_set_fp64_accum")

    def set_fp64_tc(self, on: bool):
        """The factors' large FP64 products (FP32 AX) on the tensor cores by exact
        digit slicing (True, default) or on the FP64 units (False)."""
        _check(lib.gn_set_fp64_tc(self._h, 1 if on else 0), "gn_set_fp64_tc")

    def dgemm_tc(self, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor = None, alpha: float = 1.0,
                 beta: float = 0.0, ta: bool = False, tb: bool = False) -> torch.Tensor:
        """C = alpha op(A) op(B) + beta C in FP64 on the tensor cores (digit slicing).
        A: FP64 or FP32, B and C: FP64, all row-major with unit column stride."""
        if A.dtype not in (torch.float64, torch.float32) or B.dtype != torch.float64:
            raise TypeError("dgemm_tc: A FP64 or FP32, B FP64")
        if A.stride(1) != 1 or B.stride(1) != 1:
            raise ValueError("dgemm_tc: unit column stride required")
        M, K = (A.shape[1], A.shape[0]) if ta else (A.shape[0], A.shape[1])
        K2, N = (B.shape[1], B.shape[0]) if tb else (B.shape[0], B.shape[1])
        if K != K2:
            raise ValueError("dgemm_tc: inner dimensions differ")
        if C is None:
            C = torch.zeros(M, N, dtype=torch.float64, device=A.device)
        a32 = 1 if A.dtype == torch.float32 else 0
        b = ctypes.c_size_t()
        _check(lib.gn_dgemm_tc_workspace_size(M, N, K, a32, ctypes.byref(b)), "gn_dgemm_tc_workspace_size")
        with torch.cuda.stream(self.stream):   # freed in order with the handle's stream
            ws = torch.empty(int(b.value), dtype=torch.uint8, device=A.device)
        _check(lib.gn_dgemm_tc(self._h, M, N, K, float(alpha), A.data_ptr(), a32, A.stride(0), 1 if ta else 0,
                               B.data_ptr(), B.stride(0), 1 if tb else 0, float(beta), C.data_ptr(), C.stride(0),
                               ws.data_ptr(), ws.numel()), "gn_dgemm_tc")
        return C

    # ---------------------------------------------------------------- sizing
    @staticmethod
    def workspace_bytes(m, n, r, l, op_dtype) -> int:
        b = ctypes.c_size_t()
        _check(lib.gn_workspace_size(m, n, r, l, op_dtype, ctypes.byref(b)), "gn_workspace_size")
        return int(b.value)

    def workspace(self, m, n, r, l, op_dtype, device=None) -> torch.Tensor:
        nb = self.workspace_bytes(m, n, r, l, op_dtype)
        return torch.empty(nb, dtype=torch.uint8, device=device or "cuda")

    # ---------------------------------------------------------------- calls
    def quantize(self, src: torch.Tensor, split: bool = False):
        """FP64/FP32 -> bf16 (or split bf16 hi, lo) with an 8-aligned leading dimension."""
        hi = padded(src.shape[0], src.shape[1], torch.bfloat16, src.device)
        lo = padded(src.shape[0], src.shape[1], torch.bfloat16, src.device) if split else None
        d = mat(hi, lo)
        _check(lib.gn_quantize(self._h, ctypes.byref(mat(src)), ctypes.byref(d)), "gn_quantize")
        return (hi, lo) if split else hi

    def quantize_e4m3(self, src: torch.Tensor, data: bool = True, transposed: bool = True) -> E4M3Mat:
        """FP64/FP32 -> e4m3 with one power-of-two scale per 128 x 128 tile,
        row-major (``data``) and / or transposed (``data_t``) codes."""
        rows, cols = src.shape
        r16 = lambda x: (x + 15) // 16 * 16
        sc = torch.empty((rows + 127) // 128, (cols + 127) // 128, dtype=torch.uint8, device=src.device)
        d = torch.empty(rows, r16(cols), dtype=torch.uint8, device=src.device)[:, :cols] if data else None
        dt = torch.empty(cols, r16(rows), dtype=torch.uint8, device=src.device)[:, :rows] if transposed else None
        q = E4M3Mat(rows, cols, sc, d, dt)
        dst = q.gnmat()
        _check(lib.gn_quantize(self._h, ctypes.byref(mat(src)), ctypes.byref(dst)), "gn_quantize")
        return q

    def sketch(self, A, X, Y, AX, YtA, ws, A_lo=None):
        _check(lib.gn_sketch(self._h, ctypes.byref(mat(A, A_lo)), ctypes.byref(mat(X)), ctypes.byref(mat(Y)),
                             ctypes.byref(mat(AX)), ctypes.byref(mat(YtA)), ctypes.c_void_p(ws.data_ptr()),
                             ws.numel()), "gn_sketch")

    def core(self, YtA, X, eps: float, mode: int, core: Core, ws) -> Core:
        """gn_core; with CORE_DEFER in ``mode`` the host fields stay pending
        (k = -1) until ``core_finish``."""
        c = core.cstruct()
        _check(lib.gn_core(self._h, ctypes.byref(mat(YtA)), ctypes.byref(mat(X)), float(eps), int(mode),
                           ctypes.byref(c), ctypes.c_void_p(ws.data_ptr()), ws.numel()), "gn_core")
        core.update(c)
        return core

    def core_finish(self, core: Core) -> Core:
        c = core.cstruct()
        _check(lib.gn_core_finish(self._h, ctypes.byref(c)), "gn_core_finish")
        core.update(c)
        return core

    def factors(self, AX, YtA, core: Core, F, G, ws):
        c = core.cstruct()
        _check(lib.gn_factors(self._h, ctypes.byref(mat(AX)), ctypes.byref(mat(YtA)), ctypes.byref(c),
                              ctypes.byref(mat(F)), ctypes.byref(mat(G)), ctypes.c_void_p(ws.data_ptr()),
                              ws.numel()), "gn_factors")

    def apply(self, AX, YtA, core: Core, W, out=None, side: int = 0, ws=None) -> torch.Tensor:
        """Ahat W (side 0, W: n x kw -> m x kw) or W Ahat (side 1, W: kw x m ->
        kw x n) from the sketches and the core, without forming Ahat."""
        m, n = AX.shape[0], YtA.shape[1]
        kw = W.shape[1] if side == 0 else W.shape[0]
        if out is None:
            shape = (m, kw) if side == 0 else (kw, n)
            out = torch.empty(shape, dtype=torch.float64, device=W.device)
        if ws is None:
            b = ctypes.c_size_t()
            _check(lib.gn_apply_workspace_size(m, n, core.r, core.l, kw, side, ctypes.byref(b)),
                   "gn_apply_workspace_size")
            with torch.cuda.stream(self.stream):   # freed in order with the handle's stream
                ws = torch.empty(int(b.value), dtype=torch.uint8, device=W.device)
        c = core.cstruct()
        _check(lib.gn_apply(self._h, ctypes.byref(mat(AX)), ctypes.byref(mat(YtA)), ctypes.byref(c),
                            ctypes.byref(mat(W)), ctypes.byref(mat(out)), int(side),
                            ctypes.c_void_p(ws.data_ptr()), ws.numel()), "gn_apply")
        return out

    def update(self, E, X, Y, AX, YtA, ws=None, E_lo=None):
        """A <- A + E on the sketch state: AX += E X, Y^T A += Y^T E (E given as
        gn_sketch takes A)."""
        m, n = mat(E).rows, mat(E).cols
        r, rl = mat(X).cols, mat(Y).cols
        if ws is None:
            b = ctypes.c_size_t()
            _check(lib.gn_update_workspace_size(m, n, r, rl - r, mat(E, E_lo).dtype, ctypes.byref(b)),
                   "gn_update_workspace_size")
            with torch.cuda.stream(self.stream):   # freed in order with the handle's stream
                ws = torch.empty(int(b.value), dtype=torch.uint8, device=AX.device)
        _check(lib.gn_update(self._h, ctypes.byref(mat(E, E_lo)), ctypes.byref(mat(X)), ctypes.byref(mat(Y)),
                             ctypes.byref(mat(AX)), ctypes.byref(mat(YtA)), ctypes.c_void_p(ws.data_ptr()),
                             ws.numel()), "gn_update")

    def update_workspace(self, m, n, r, l, op_dtype, device=None) -> torch.Tensor:
        """Scratch for update / append_rows / append_cols on an m x n block."""
        b = ctypes.c_size_t()
        _check(lib.gn_update_workspace_size(m, n, r, l, op_dtype, ctypes.byref(b)), "gn_update_workspace_size")
        return torch.empty(int(b.value), dtype=torch.uint8, device=device or "cuda")

    def _scratch(self, nbytes, device):
        with torch.cuda.stream(self.stream):   # freed in order with the handle's stream
            return torch.empty(int(nbytes), dtype=torch.uint8, device=device)

    def resample(self, A, Xd, Yd, AX, YtA, AXn, YtAn, A_lo=None):
        """Rank r -> r + dr, oversampling l -> l + dl: AXn = [AX, A Xd],
        YtAn = [Y^T A; Yd^T A] (Xd: n x dr, Yd: m x (dr + dl); dr or dl may be 0)."""
        Am = mat(A, A_lo)
        m, n = Am.rows, Am.cols
        dr, drl = _cols(Xd), _cols(Yd)
        b = ctypes.c_size_t()
        _check(lib.gn_resample_workspace_size(m, n, dr, drl - dr, Am.dtype, ctypes.byref(b)),
               "gn_resample_workspace_size")
        ws = self._scratch(max(256, b.value), AX.device)
        _check(lib.gn_resample(self._h, ctypes.byref(Am), ctypes.byref(_mat_or_empty(Xd, n)),
                               ctypes.byref(mat(Yd)), ctypes.byref(mat(AX)), ctypes.byref(mat(YtA)),
                               ctypes.byref(_mat_or_empty(AXn, m)), ctypes.byref(mat(YtAn)),
                               ctypes.c_void_p(ws.data_ptr()), ws.numel()), "gn_resample")

    def append_rows(self, B, X, Yb, AX, YtA, AXn):
        """[A; B]: AXn = [AX; B X], Y^T A += Yb^T B."""
        mb, n, r, rl = mat(B).rows, mat(B).cols, mat(X).cols, mat(Yb).cols
        b = ctypes.c_size_t()
        _check(lib.gn_update_workspace_size(mb, n, r, rl - r, mat(B).dtype, ctypes.byref(b)),
               "gn_update_workspace_size")
        ws = self._scratch(b.value, AX.device)
        _check(lib.gn_append_rows(self._h, ctypes.byref(mat(B)), ctypes.byref(mat(X)), ctypes.byref(mat(Yb)),
                                  ctypes.byref(mat(AX)), ctypes.byref(mat(YtA)), ctypes.byref(mat(AXn)),
                                  ctypes.c_void_p(ws.data_ptr()), ws.numel()), "gn_append_rows")

    def append_cols(self, B, Xb, Y, AX, YtA, YtAn):
        """[A, B]: AX += B Xb, YtAn = [Y^T A, Y^T B]."""
        m, nb, r, rl = mat(B).rows, mat(B).cols, mat(Xb).cols, mat(Y).cols
        b = ctypes.c_size_t()
        _check(lib.gn_update_workspace_size(m, nb, r, rl - r, mat(B).dtype, ctypes.byref(b)),
               "gn_update_workspace_size")
        ws = self._scratch(b.value, AX.device)
        _check(lib.gn_append_cols(self._h, ctypes.byref(mat(B)), ctypes.byref(mat(Xb)), ctypes.byref(mat(Y)),
                                  ctypes.byref(mat(AX)), ctypes.byref(mat(YtA)), ctypes.byref(mat(YtAn)),
                                  ctypes.c_void_p(ws.data_ptr()), ws.numel()), "gn_append_cols")

    def approx(self, A, X, Y, eps, mode, AX, YtA, core: Core, F, G, ws, A_lo=None) -> Core:
        c = core.cstruct()
        _check(lib.gn_approx(self._h, ctypes.byref(mat(A, A_lo)), ctypes.byref(mat(X)), ctypes.byref(mat(Y)),
                             float(eps), int(mode), ctypes.byref(mat(AX)), ctypes.byref(mat(YtA)),
                             ctypes.byref(c), ctypes.byref(mat(F)), ctypes.byref(mat(G)),
                             ctypes.c_void_p(ws.data_ptr()), ws.numel()), "gn_approx")
        core.update(c)
        return core

    def error_fro2(self, A, F, G, out, ws, A_lo=None):
        """Writes ||A - F G||_F^2 into the 1-element float64 CUDA tensor ``out``."""
        _check(lib.gn_error_fro2(self._h, ctypes.byref(mat(A, A_lo)), ctypes.byref(mat(F)), ctypes.byref(mat(G)),
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel()),
               "gn_error_fro2")

    def error_fro2_noalloc(self, A, F, G, out, A_lo=None):
        """Like error_fro2 but without a workspace (fixed device array inside the library)."""
        _check(lib.gn_error_fro2_noalloc(self._h, ctypes.byref(mat(A, A_lo)), ctypes.byref(mat(F)),
                                         ctypes.byref(mat(G)), ctypes.c_void_p(out.data_ptr())),
               "gn_error_fro2_noalloc")

    # ------------------------------------------------------------ adjoint
    def backward_workspace(self, m, n, r, l, dtype) -> torch.Tensor:
        b = ctypes.c_size_t()
        _check(lib.gn_backward_workspace_size(m, n, r, l, dtype, ctypes.byref(b)), "gn_backward_workspace_size")
        return torch.empty(int(b.value), dtype=torch.uint8, device="cuda")

    def backward(self, A, X, Y, Gup, dA, ws):
        self.front_calls += 1
        _check(lib.gn_backward(self._h, ctypes.byref(mat(A)), ctypes.byref(mat(X)), ctypes.byref(mat(Y)),
                               ctypes.byref(mat(Gup)), ctypes.byref(mat(dA)), ctypes.c_void_p(ws.data_ptr()),
                               ws.numel()), "gn_backward")

    def forward_dense(self, A, X, Y, Ahat, ws):
        self.front_calls += 1
        _check(lib.gn_forward_dense(self._h, ctypes.byref(mat(A)), ctypes.byref(mat(X)), ctypes.byref(mat(Y)),
                                    ctypes.byref(mat(Ahat)), ctypes.c_void_p(ws.data_ptr()), ws.numel()),
               "gn_forward_dense")

    def backward_saved(self, X, Y, Gup, dA, ws):
        """gn_backward from the front the last forward_dense / backward left in ws."""
        _check(lib.gn_backward_saved(self._h, ctypes.byref(mat(X)), ctypes.byref(mat(Y)), ctypes.byref(mat(Gup)),
                                     ctypes.byref(mat(dA)), ctypes.c_void_p(ws.data_ptr()), ws.numel()),
               "gn_backward_saved")

    # ------------------------------------------------------------ batched
    def batched_prepare(self, problems):
        """problems: list of dicts with A, X, Y (bf16), AX, YtA (f32), Q, R, Q2, R2 (f64), k (int32[1]).
        Returns the workspace tensor that gn_batched_run needs (keep it alive)."""
        arr = (GnProblem * len(problems))()
        for i, p in enumerate(problems):
            arr[i] = GnProblem(mat(p["A"]), mat(p["X"]), mat(p["Y"]), mat(p["AX"]), mat(p["YtA"]),
                               p["Q"].data_ptr(), p["R"].data_ptr(), p["Q2"].data_ptr(), p["R2"].data_ptr(),
                               p["k"].data_ptr())
        b = ctypes.c_size_t()
        _check(lib.gn_batched_workspace_size(len(problems), arr, ctypes.byref(b)), "gn_batched_workspace_size")
        ws = torch.empty(int(b.value), dtype=torch.uint8, device="cuda")
        _check(lib.gn_batched_prepare(self._h, len(problems), arr, ctypes.c_void_p(ws.data_ptr()), ws.numel()),
               "gn_batched_prepare")
        self._batched_arr = arr
        return ws

    def batched_set_policy(self, policy: int):
        _check(lib.gn_batched_set_policy(self._h, int(policy)), "gn_batched_set_policy")

    def batched_tune(self, eps, mode, ws):
        """Time every tile policy on the prepared batch, keep the fastest;
        returns (policy, ms per run)."""
        arr = self._batched_arr
        best = ctypes.c_int32()
        ms = ctypes.c_double()
        _check(lib.gn_batched_tune(self._h, len(arr), arr, ctypes.c_void_p(ws.data_ptr()), ws.numel(), float(eps),
                                   int(mode), ctypes.byref(best), ctypes.byref(ms)), "gn_batched_tune")
        return int(best.value), float(ms.value)

    def batched_run(self, eps, mode, ws):
        _check(lib.gn_batched_run(self._h, float(eps), int(mode), ctypes.c_void_p(ws.data_ptr()), ws.numel()),
               "gn_batched_run")

    def dct_sketch(self, n: int, signs: torch.Tensor, cols: torch.Tensor, dtype=torch.bfloat16) -> torch.Tensor:
        """The subsampled DCT sketch D C^T S (n x len(cols)) from its draws (signs:
        n float64, cols: int64), made on the device; bf16 with an 8-aligned ld."""
        r = int(cols.numel())
        dev = self.stream.device
        s = signs.to(device=dev, dtype=torch.float64).contiguous()
        c = cols.to(device=dev, dtype=torch.int64).contiguous()
        X = padded(n, r, dtype, dev) if dtype == torch.bfloat16 else torch.empty(n, r, dtype=dtype, device=dev)
        _check(lib.gn_dct_sketch(self._h, n, r, ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                 ctypes.byref(mat(X))), "gn_dct_sketch")
        return X

    def sketch_csr_countsketch(self, crow, col, vals, shape, bx, sx, by, sy, AX, YtA):
        """AX, Y^T A of a CSR matrix (crow int64, col int32, vals f64/f32 device
        tensors, shape (m, n)) with CountSketch X (bx, sx) and Y (by, sy)."""
        m, n = shape
        dt = _TORCH_DT[vals.dtype]
        A = GnCsr(crow.data_ptr(), col.data_ptr(), vals.data_ptr(), m, n, int(vals.numel()), dt)
        keep = [t.contiguous() for t in (bx, sx, by, sy)]
        _check(lib.gn_sketch_csr_countsketch(self._h, ctypes.byref(A), *[ctypes.c_void_p(t.data_ptr()) for t in keep],
                                             ctypes.byref(mat(AX)), ctypes.byref(mat(YtA))), "gn_sketch_csr_countsketch")

    def countsketch_apply(self, B, bx, sx, out):
        """out (FP64) = B X for the CountSketch X of (bx, sx)."""
        b, s = bx.contiguous(), sx.contiguous()
        _check(lib.gn_countsketch_apply(self._h, ctypes.byref(mat(B)), ctypes.c_void_p(b.data_ptr()),
                                        ctypes.c_void_p(s.data_ptr()), ctypes.byref(mat(out))), "gn_countsketch_apply")
        return out

    def countsketch_matrix(self, n: int, r: int, buckets, signs, dtype=torch.float64) -> torch.Tensor:
        X = torch.empty(n, r, dtype=dtype, device=self.stream.device)
        b, s = buckets.contiguous(), signs.contiguous()
        _check(lib.gn_countsketch_matrix(self._h, n, r, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                         ctypes.byref(mat(X))), "gn_countsketch_matrix")
        return X

    def factors_variant(self, AX, YtA, X, eps: float, variant: int, F, G, sv=None) -> int:
        """Section 5.1.1's perturbed cores and SGN with the SVD eps-pseudoinverse:
        F, G (first k columns / rows) from the sketch state; returns k."""
        m, r = AX.shape
        rl, n = YtA.shape
        b = ctypes.c_size_t()
        _check(lib.gn_variant_workspace_size(m, n, r, rl - r, ctypes.byref(b)), "gn_variant_workspace_size")
        ws = self._scratch(b.value, AX.device)
        k = ctypes.c_int64()
        _check(lib.gn_factors_variant(self._h, ctypes.byref(mat(AX)), ctypes.byref(mat(YtA)), ctypes.byref(mat(X)),
                                      float(eps), int(variant), ctypes.byref(mat(F)), ctypes.byref(mat(G)),
                                      ctypes.byref(k), ctypes.c_void_p(sv.data_ptr() if sv is not None else 0),
                                      ctypes.c_void_p(ws.data_ptr()), ws.numel()), "gn_factors_variant")
        return int(k.value)

    def hmt(self, A, X, Q, B, ws):
        _check(lib.gn_hmt(self._h, ctypes.byref(mat(A)), ctypes.byref(mat(X)), ctypes.byref(mat(Q)),
                          ctypes.byref(mat(B)), ctypes.c_void_p(ws.data_ptr()), ws.numel()), "gn_hmt")


_DT = {torch.float64: F64, torch.float32: F32}


class GNApprox(torch.autograd.Function):
    """A -> A_hat = (AX)(Y^T A X)^+(Y^T A) (plain GN) with X, Y fixed, as a
    differentiable torch op.  forward: gn_forward_dense, whose workspace keeps
    the sketches, the core's QR and F; backward: gn_backward_saved from them when
    no other forward_dense / backward ran on the handle since (the handle keeps
    one front), else gn_backward, which forms them again from A."""

    @staticmethod
    def forward(ctx, A, X, Y, handle):
        m, n = A.shape
        r, l = X.shape[1], Y.shape[1] - X.shape[1]
        ws = handle.backward_workspace(m, n, r, l, _DT[A.dtype])
        Ahat = torch.empty_like(A)
        handle.forward_dense(A, X, Y, Ahat, ws)
        ctx.save_for_backward(A, X, Y)
        ctx.handle = handle
        ctx.ws = ws
        ctx.front = handle.front_calls
        return Ahat

    @staticmethod
    def backward(ctx, grad):
        A, X, Y = ctx.saved_tensors
        m, n = A.shape
        r, l = X.shape[1], Y.shape[1] - X.shape[1]
        dA = torch.empty_like(A)
        if ctx.handle.front_calls == ctx.front:
            ctx.handle.backward_saved(X, Y, grad.contiguous(), dA, ctx.ws)
        else:
            ws = ctx.handle.backward_workspace(m, n, r, l, _DT[A.dtype])
            ctx.handle.backward(A, X, Y, grad.contiguous(), dA, ws)
        ctx.ws = None
        return dA, None, None, None


def gn_approx_dense(A, X, Y, handle):
    """Differentiable plain-GN approximant of A (FP64 or FP32 CUDA tensors)."""
    return GNApprox.apply(A, X, Y, handle)
