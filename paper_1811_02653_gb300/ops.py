"""Thin Python binding of liboversketch.so (argument marshalling only).

Every function here has the name of the C entry point it calls (without the
``oversketch_`` prefix), passes device pointers of torch tensors and the
current torch CUDA stream, and raises ``OverSketchError`` on a non-OK status.
Tensors are allocated with torch (device memory is plumbing); every step of
the computation runs in the library's kernels.  There is no fallback: if the
library is missing or fails to load, the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboversketch.so")

F32, BF16, FP8, TF32X2 = 0, 1, 2, 3
_DT = {torch.float32: F32, torch.bfloat16: BF16}
if hasattr(torch, "float8_e4m3fn"):
    _DT[torch.float8_e4m3fn] = FP8
_TORCH_DT = {F32: torch.float32, BF16: torch.bfloat16, FP8: getattr(torch, "float8_e4m3fn", None),
             TF32X2: torch.float32}
DTYPE_NAMES = {"f32": F32, "fp32": F32, "bf16": BF16, "fp8": FP8, "fp8e4m3": FP8, "tf32x2": TF32X2}
FROB_WORKSPACE_BYTES = 12288

_lib = None
_lock = threading.Lock()


class OverSketchError(RuntimeError):
    pass


class _Opts(ctypes.Structure):
    _fields_ = [("gemm_dtype", ctypes.c_int), ("col_scale", ctypes.c_void_p),
                ("symmetric", ctypes.c_int32), ("flags", ctypes.c_int32)]

OPT_SPARSE_A = 1


class _Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("l", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64),
                ("plan", ctypes.c_void_p), ("mask", ctypes.c_uint64)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("branches", ctypes.c_int32), ("tile_n", ctypes.c_int32),
                ("total_tiles", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("operand_bytes", ctypes.c_size_t), ("workspace_bytes", ctypes.c_size_t),
                ("tuned_ms", ctypes.c_float)]


def load_library(path: str | None = None):
    """Load liboversketch.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise OverSketchError(f"{p} is missing; build it with paper_1811_02653_gb300.build.build()")
        lib = ctypes.CDLL(p)
        vp, i64, i32, u64, f32, sz = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_uint64, ctypes.c_float, ctypes.c_size_t)
        st, pp = ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)
        sigs = {
            "oversketch_status_string": (ctypes.c_char_p, [st]),
            "oversketch_last_cuda_error": (ctypes.c_char_p, []),
            "oversketch_plan": (st, [i64, i32, i32, i32, u64, vp, pp]),
            "oversketch_plan_from_tables": (st, [i64, i32, i32, i32, vp, vp, vp, pp]),
            "oversketch_plan_get_tables": (st, [vp, vp, vp, vp, vp]),
            "oversketch_plan_info": (st, [vp, vp, vp, vp, vp]),
            "oversketch_plan_destroy": (st, [vp]),
            "oversketch_sketch_workspace": (st, [vp, i64, st, ctypes.POINTER(sz)]),
            "oversketch_sketch_left": (st, [vp, vp, st, i64, i64, vp, st, i64, vp, vp, u64, vp, sz, vp]),
            "oversketch_sketch_right": (st, [vp, vp, st, i64, i64, vp, st, i64, vp, vp, u64, vp, sz, vp]),
            "oversketch_gemm_masked": (st, [vp, vp, i64, vp, vp, i64, vp, st, i64, i64, u64, f32, f32,
                                            vp, i64, vp]),
            "oversketch_workspace_size": (st, [vp, i64, i64, st, st, ctypes.POINTER(_Opts), ctypes.POINTER(sz)]),
            "oversketch_matmul": (st, [vp, vp, st, i64, vp, st, i64, vp, i64, i64, i64, i64, u64,
                                       ctypes.POINTER(_Opts), vp, sz, vp]),
            "oversketch_unsketch_cols": (st, [vp, vp, i64, i64, u64, f32, vp, st, i64, vp]),
            "oversketch_unsketch_rows": (st, [vp, vp, i64, i64, u64, f32, vp, st, i64, vp]),
            "oversketch_frob": (st, [vp, i64, vp, i64, i64, i64, vp, vp, sz, vp]),
            "oversketch_device_status": (st, [vp, ctypes.POINTER(i32), i32]),
            "oversketch_sketch_left_noalloc": (st, [vp, vp, st, i64, i64, vp, st, i64, vp, vp, u64, vp]),
            "oversketch_gemm_bf16": (st, [vp, i64, vp, i64, i64, i64, i64, f32, f32, vp, i64, vp]),
            "oversketch_select_transpose": (st, [vp, st, i64, i64, i64, u64, i32, vp, st, i64, vp]),
            "oversketch_cast": (st, [vp, st, i64, i64, i64, vp, st, i64, vp]),
            "oversketch_sketch_left_sparse": (st, [vp, vp, st, i64, i64, vp, st, i64, vp, vp, u64, vp]),
            "oversketch_matmul_host_workspace_size": (st, [vp, i64, i64, st, st, ctypes.POINTER(_Opts),
                                                           ctypes.POINTER(sz)]),
            "oversketch_matmul_host": (st, [vp, vp, st, i64, vp, st, i64, vp, i64, i64, i64, i64, u64,
                                            ctypes.POINTER(_Opts), vp, sz, vp]),
            "oversketch_gemm_masked_blocks": (st, [vp, vp, i64, vp, i64, i64, i64, vp, i64, i64, f32, vp,
                                                   i64, vp]),
            "oversketch_sketch_size": (st, [ctypes.c_double, ctypes.c_double, i32, ctypes.c_double, i32,
                                            ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "oversketch_batch_create": (st, [ctypes.POINTER(_Problem), i32, st, st, st, sz, i32, vp, pp]),
            "oversketch_batch_run": (st, [vp, vp]),
            "oversketch_batch_info": (st, [vp, ctypes.POINTER(_BatchInfo)]),
            "oversketch_batch_destroy": (st, [vp]),
            "oversketch_test_wait_timeout": (st, [u64, i32]),
            "oversketch_matmul_batched_workspace_size": (st, [i32, vp, vp, vp, vp, st, st, ctypes.POINTER(_Opts),
                                                              ctypes.POINTER(sz)]),
            "oversketch_matmul_batched": (st, [i32, vp, vp, vp, vp, vp, vp, vp, st, st, vp, ctypes.POINTER(_Opts), vp,
                                               sz, vp]),
            "oversketch_matmul_backward_workspace_size": (st, [vp, i64, i64, u64, i32, i32, ctypes.POINTER(sz)]),
            "oversketch_matmul_backward": (st, [vp, vp, i64, vp, i64, vp, i64, i64, i64, u64, vp, st, i64, vp, st,
                                                i64, vp, sz, vp]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def exported_symbols() -> list[str]:
    return sorted(n for n in _sigs_names())


def _sigs_names():
    return ["oversketch_status_string", "oversketch_last_cuda_error", "oversketch_plan",
            "oversketch_plan_from_tables", "oversketch_plan_get_tables", "oversketch_plan_info",
            "oversketch_plan_destroy", "oversketch_sketch_workspace", "oversketch_sketch_left",
            "oversketch_sketch_right", "oversketch_gemm_masked", "oversketch_workspace_size",
            "oversketch_matmul", "oversketch_unsketch_cols", "oversketch_unsketch_rows",
            "oversketch_frob", "oversketch_device_status", "oversketch_sketch_left_noalloc",
            "oversketch_gemm_bf16", "oversketch_select_transpose", "oversketch_cast",
            "oversketch_batch_create", "oversketch_batch_run", "oversketch_batch_info",
            "oversketch_batch_destroy", "oversketch_sketch_left_sparse",
            "oversketch_matmul_host_workspace_size", "oversketch_matmul_host", "oversketch_sketch_size",
            "oversketch_gemm_masked_blocks", "oversketch_matmul_backward_workspace_size", "oversketch_test_wait_timeout",
            "oversketch_matmul_batched_workspace_size", "oversketch_matmul_batched",
            "oversketch_matmul_backward"]


def _check(status: int, what: str):
    if status != 0:
        lib = load_library()
        msg = lib.oversketch_status_string(status).decode()
        if status == 5:
            msg += " (" + lib.oversketch_last_cuda_error().decode() + ")"
        raise OverSketchError(f"{what}: {msg}")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _dt(t: torch.Tensor) -> int:
    if t.dtype not in _DT:
        raise OverSketchError(f"unsupported dtype {t.dtype}")
    return _DT[t.dtype]


def _dtype_code(d) -> int:
    if isinstance(d, str):
        return DTYPE_NAMES[d.lower()]
    if isinstance(d, torch.dtype):
        return _DT[d]
    return int(d)


def _rowmajor_host(t: torch.Tensor, name: str):
    if t.dim() != 2 or t.stride(1) != 1:
        raise OverSketchError(f"{name} must be a row-major 2-D tensor")
    if t.is_cuda:
        raise OverSketchError(f"{name} must live in host memory")
    return t.stride(0)


def _rowmajor(t: torch.Tensor, name: str):
    if t.dim() != 2 or t.stride(1) != 1:
        raise OverSketchError(f"{name} must be a row-major 2-D tensor")
    if not t.is_cuda:
        raise OverSketchError(f"{name} must live on a CUDA device")
    return t.stride(0)


def _pad_ld(cols: int, dtype_code: int) -> int:
    el = 16 // (4 if dtype_code == F32 else (2 if dtype_code == BF16 else 1))
    return (cols + el - 1) // el * el


class Plan:
    """The sketch S of Eq. 3 on the device (oversketch_plan)."""

    def __init__(self, n: int, b: int, N: int, e: int, seed: int = 0, stream=None,
                 tables=None):
        lib = load_library()
        h = ctypes.c_void_p()
        if tables is None:
            _check(lib.oversketch_plan(n, b, N, e, seed & (2 ** 64 - 1), _stream(stream),
                                       ctypes.byref(h)), "oversketch_plan")
        else:
            hh, ss = tables
            hh = np.ascontiguousarray(hh, dtype=np.uint32)
            ss = np.ascontiguousarray(ss, dtype=np.int8)
            assert hh.shape == (N + e, n) and ss.shape == (N + e, n)
            _check(lib.oversketch_plan_from_tables(n, b, N, e, hh.ctypes.data_as(ctypes.c_void_p),
                                                   ss.ctypes.data_as(ctypes.c_void_p),
                                                   _stream(stream), ctypes.byref(h)),
                   "oversketch_plan_from_tables")
        self._h = h
        self.n, self.b, self.N, self.e, self.seed = n, b, N, e, seed
        self.P = N + e
        self.z = self.P * b

    @property
    def handle(self):
        return self._h

    def tables(self):
        """(h, sigma, perm, offs) copied to host numpy arrays."""
        lib = load_library()
        h = np.empty((self.P, self.n), np.uint32)
        s = np.empty((self.P, self.n), np.int8)
        perm = np.empty((self.P, self.n), np.uint32)
        offs = np.empty((self.P, self.b + 1), np.uint32)
        _check(lib.oversketch_plan_get_tables(self._h, h.ctypes.data_as(ctypes.c_void_p),
                                              s.ctypes.data_as(ctypes.c_void_p),
                                              perm.ctypes.data_as(ctypes.c_void_p),
                                              offs.ctypes.data_as(ctypes.c_void_p)),
               "oversketch_plan_get_tables")
        return h, s, perm, offs

    def destroy(self):
        if self._h:
            load_library().oversketch_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def plan(n, b, N, e, seed=0, stream=None) -> Plan:
    return Plan(n, b, N, e, seed, stream)


def sketch_size(eps: float, theta: float, b: int, straggler_fraction: float = 0.0, r: int = 1):
    """(N, e) for an (eps, theta)-accurate product with blocks of width b (Thm. 4.1):
    N = ceil(r * 2/(eps*theta) / b), e = smallest e >= p (N + e)."""
    N, e = ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().oversketch_sketch_size(eps, theta, b, straggler_fraction, r, ctypes.byref(N),
                                                 ctypes.byref(e)), "oversketch_sketch_size")
    return N.value, e.value


def plan_from_tables(h, sigma, b, N, e, stream=None) -> Plan:
    P, n = np.asarray(h).shape
    return Plan(n, b, N, e, 0, stream, tables=(h, sigma))


def _fp8_scales_shape(rows, z):
    # slice-major: [t, r] for slice t of z/128 and row r, rows padded to a multiple of 4
    return ((z + 127) // 128, (rows + 3) // 4 * 4)


def fp8_scales_by_row(scales: torch.Tensor, rows: int) -> torch.Tensor:
    """View of slice-major FP8 scales as rows x (z/128) (entry [r, t])."""
    return scales[:, :rows].t()


def sketch_workspace(p: Plan, free_extent: int, in_dtype=torch.float32) -> int:
    """Bytes of the packed-strip workspace for a sketch with this free extent."""
    out = ctypes.c_size_t()
    _check(load_library().oversketch_sketch_workspace(p.handle, free_extent, _dtype_code(in_dtype),
                                                      ctypes.byref(out)), "oversketch_sketch_workspace")
    return out.value


def _alloc_out(rows, ld, z, od, device):
    """Sketch output: rows x z view (row pitch ld); for TF32X2 the hi plane of a
    (2, rows, ld) buffer whose lo plane follows it."""
    if od == TF32X2:
        return torch.empty((2, rows, ld), dtype=torch.float32, device=device)[0, :, :z]
    return torch.empty((rows, ld), dtype=_TORCH_DT[od], device=device)[:, :z]


def tf32_planes(t):
    """(hi, lo) views of a TF32X2 sketch output."""
    base = t.as_strided((2, t.shape[0], t.shape[1]), (t.shape[0] * t.stride(0), t.stride(0), 1))
    return base[0], base[1]


def _workspace(p, F, dtype, device, workspace):
    if workspace is None:
        workspace = torch.empty(sketch_workspace(p, F, dtype), dtype=torch.uint8, device=device)
    return workspace


def sketch_left(p: Plan, A: torch.Tensor, out_dtype="f32", col_scale=None, out=None,
                scales=None, workspace=None, block_mask=0, stream=None):
    """A~ = A diag(col_scale) S (m x z, K-major); returns (At, scales or None)."""
    lda = _rowmajor(A, "A")
    m = A.shape[0]
    od = _dtype_code(out_dtype)
    ld = _pad_ld(p.z, od)
    if out is None:
        out = _alloc_out(m, ld, p.z, od, A.device)
    if od == FP8 and scales is None:
        scales = torch.empty(_fp8_scales_shape(m, p.z), dtype=torch.float32, device=A.device)
    workspace = _workspace(p, m, A.dtype, A.device, workspace)
    _check(load_library().oversketch_sketch_left(
        p.handle, _ptr(A), _dt(A), m, lda, _ptr(out), od, out.stride(0), _ptr(scales),
        _ptr(col_scale), block_mask, _ptr(workspace), workspace.numel(), _stream(stream)),
        "oversketch_sketch_left")
    return out, scales


def sketch_left_sparse(p: Plan, A: torch.Tensor, out_dtype="f32", col_scale=None, out=None,
                       scales=None, block_mask=0, stream=None):
    """A~ = A diag(col_scale) S for a sparse A stored dense (only the nonzeros are
    routed; no workspace); returns (At, scales or None)."""
    lda = _rowmajor(A, "A")
    m = A.shape[0]
    od = _dtype_code(out_dtype)
    ld = _pad_ld(p.z, od)
    if out is None:
        out = _alloc_out(m, ld, p.z, od, A.device)
    if od == FP8 and scales is None:
        scales = torch.empty(_fp8_scales_shape(m, p.z), dtype=torch.float32, device=A.device)
    _check(load_library().oversketch_sketch_left_sparse(
        p.handle, _ptr(A), _dt(A), m, lda, _ptr(out), od, out.stride(0), _ptr(scales),
        _ptr(col_scale), block_mask, _stream(stream)), "oversketch_sketch_left_sparse")
    return out, scales


def sketch_right(p: Plan, B: torch.Tensor, out_dtype="f32", out=None, scales=None, block_mask=0,
                 workspace=None, stream=None, row_scale=None):
    """B~^T = (S^T diag(row_scale) B)^T (l x z, K-major); returns (BtT, scales or None)."""
    ldb = _rowmajor(B, "B")
    l = B.shape[1]
    od = _dtype_code(out_dtype)
    ld = _pad_ld(p.z, od)
    if out is None:
        out = _alloc_out(l, ld, p.z, od, B.device)
    if od == FP8 and scales is None:
        scales = torch.empty(_fp8_scales_shape(l, p.z), dtype=torch.float32, device=B.device)
    workspace = _workspace(p, l, B.dtype, B.device, workspace)
    _check(load_library().oversketch_sketch_right(
        p.handle, _ptr(B), _dt(B), l, ldb, _ptr(out), od, out.stride(0), _ptr(scales), _ptr(row_scale),
        block_mask, _ptr(workspace), workspace.numel(), _stream(stream)), "oversketch_sketch_right")
    return out, scales


def gemm_masked(p: Plan, At, BtT, mask: int, alpha=1.0, beta=0.0, C=None, a_scales=None,
                b_scales=None, dtype=None, stream=None):
    """C = (alpha/k) * sum_{j in mask} At_j BtT_j^T (+ beta C), k = popcount(mask)
    applied by the library (alpha = 1: the OverSketch product).
    ``dtype`` overrides the operand dtype (e.g. "tf32x2" for hi/lo planes)."""
    m, l = At.shape[0], BtT.shape[0]
    if C is None:
        C = torch.empty((m, l), dtype=torch.float32, device=At.device)
    _check(load_library().oversketch_gemm_masked(
        p.handle, _ptr(At), At.stride(0), _ptr(a_scales), _ptr(BtT), BtT.stride(0), _ptr(b_scales),
        _dtype_code(dtype) if dtype is not None else _dt(At), m, l, mask, alpha, beta, _ptr(C), C.stride(0),
        _stream(stream)), "oversketch_gemm_masked")
    return C


def gemm_masked_blocks(p: Plan, At, BtT, block_masks, bm: int, bn: int, beta=0.0, C=None, stream=None):
    """C with Alg. 3's termination rule per bm x bn block of C: block (i, j) sums its
    own kept sketch blocks block_masks[i, j] (int64 CUDA tensor of bit masks), 1/k_ij."""
    m, l = At.shape[0], BtT.shape[0]
    if C is None:
        C = torch.empty((m, l), dtype=torch.float32, device=At.device)
    bmask = block_masks.contiguous()
    _check(load_library().oversketch_gemm_masked_blocks(
        p.handle, _ptr(At), At.stride(0), _ptr(BtT), BtT.stride(0), m, l, _ptr(bmask), bm, bn, beta, _ptr(C),
        C.stride(0), _stream(stream)), "oversketch_gemm_masked_blocks")
    return C


def _opts(gemm_dtype, col_scale=None, symmetric=False, sparse_a=False):
    return _Opts(_dtype_code(gemm_dtype), col_scale.data_ptr() if col_scale is not None else None,
                 1 if symmetric else 0, OPT_SPARSE_A if sparse_a else 0)


def workspace_size(p: Plan, m: int, l: int, a_dtype=torch.float32, gemm_dtype="f32",
                   symmetric=False, b_dtype=torch.float32) -> int:
    out = ctypes.c_size_t()
    o = _opts(gemm_dtype, None, symmetric)
    _check(load_library().oversketch_workspace_size(p.handle, m, l, _dtype_code(a_dtype),
                                                    _dtype_code(b_dtype), ctypes.byref(o),
                                                    ctypes.byref(out)),
           "oversketch_workspace_size")
    return out.value


def matmul(p: Plan, A, B, mask: int, gemm_dtype="f32", col_scale=None, symmetric=False, C=None,
           workspace=None, stream=None, sparse_a=False):
    """The whole OverSketch product (A S)(S^T B)/k over the kept blocks.
    ``sparse_a``: A is sparse (stored dense); its sketch routes only the nonzeros."""
    lda = _rowmajor(A, "A")
    m, n = A.shape
    if symmetric:
        l, ldb, bt, bp = m, 0, F32, None
    else:
        ldb = _rowmajor(B, "B")
        l, bt, bp = B.shape[1], _dt(B), _ptr(B)
    if C is None:
        C = torch.empty((m, l), dtype=torch.float32, device=A.device)
    o = _opts(gemm_dtype, col_scale, symmetric, sparse_a)
    if workspace is None:
        workspace = torch.empty(workspace_size(p, m, l, A.dtype, gemm_dtype, symmetric,
                                               B.dtype if B is not None else torch.float32),
                                dtype=torch.uint8, device=A.device)
    _check(load_library().oversketch_matmul(
        p.handle, _ptr(A), _dt(A), lda, bp, bt, ldb, _ptr(C), C.stride(0), m, n, l, mask,
        ctypes.byref(o), _ptr(workspace), workspace.numel(), _stream(stream)), "oversketch_matmul")
    return C


def matmul_host_workspace(p: Plan, m: int, l: int, a_dtype=torch.float32, b_dtype=torch.float32,
                          gemm_dtype="f32", symmetric=False, sparse_a=False) -> int:
    out = ctypes.c_size_t()
    o = _opts(gemm_dtype, None, symmetric, sparse_a)
    _check(load_library().oversketch_matmul_host_workspace_size(
        p.handle, m, l, _dtype_code(a_dtype), _dtype_code(b_dtype), ctypes.byref(o), ctypes.byref(out)),
        "oversketch_matmul_host_workspace_size")
    return out.value


def matmul_host(p: Plan, A, B, mask: int, gemm_dtype="f32", C=None, col_scale=None, symmetric=False,
                sparse_a=False, workspace=None, stream=None):
    """(A S)(S^T B)/k with A, B and C in host memory (CPU tensors, ideally pinned):
    the transfers overlap the kernels (oversketch_matmul_host).  Returns C on the
    host; it is complete once `stream` is synchronised."""
    lda = _rowmajor_host(A, "A")
    m, n = A.shape
    if symmetric:
        l, ldb, bt, bp = m, 0, _dt(A), None
    else:
        ldb = _rowmajor_host(B, "B")
        l, bt, bp = B.shape[1], _dt(B), _ptr(B)
    if C is None:
        C = torch.empty((m, l), dtype=torch.float32).pin_memory()
    _rowmajor_host(C, "C")
    o = _opts(gemm_dtype, col_scale, symmetric, sparse_a)
    if workspace is None:
        workspace = torch.empty(matmul_host_workspace(p, m, l, A.dtype, B.dtype if B is not None else A.dtype,
                                                      gemm_dtype, symmetric, sparse_a),
                                dtype=torch.uint8, device="cuda")
    _check(load_library().oversketch_matmul_host(
        p.handle, _ptr(A), _dt(A), lda, bp, bt, ldb, _ptr(C), C.stride(0), m, n, l, mask, ctypes.byref(o),
        _ptr(workspace), workspace.numel(), _stream(stream)), "oversketch_matmul_host")
    return C


def matmul_backward_workspace(p: Plan, m: int, l: int, mask: int, need_dx=True, need_dg=True) -> int:
    out = ctypes.c_size_t()
    _check(load_library().oversketch_matmul_backward_workspace_size(p.handle, m, l, mask, 1 if need_dx else 0,
                                                                    1 if need_dg else 0, ctypes.byref(out)),
           "oversketch_matmul_backward_workspace_size")
    return out.value


def matmul_backward(p: Plan, At, BtT, dC, mask: int, x_dtype=torch.float32, g_dtype=torch.float32,
                    need_dx=True, need_dg=True, workspace=None, stream=None):
    """(dX, dG) of C = (1/k)(A S_sel)(S_sel^T B) for the upstream gradient dC (FP32
    m x l), from the forward pass's BF16 sketches At (m x z) and BtT (l x z);
    the library applies 1/k.  A side not needed comes back as None."""
    m, l = dC.shape
    lddc = _rowmajor(dC, "dC")
    dX = torch.empty((m, p.n), dtype=x_dtype, device=dC.device) if need_dx else None
    dG = torch.empty((p.n, l), dtype=g_dtype, device=dC.device) if need_dg else None
    if workspace is None:
        workspace = torch.empty(matmul_backward_workspace(p, m, l, mask, need_dx, need_dg), dtype=torch.uint8,
                                device=dC.device)
    _check(load_library().oversketch_matmul_backward(
        p.handle, _ptr(At), At.stride(0) if At is not None else 0, _ptr(BtT), BtT.stride(0) if BtT is not None else 0,
        _ptr(dC), lddc, m, l, mask, _ptr(dX), _dt(dX) if dX is not None else F32, dX.stride(0) if dX is not None else 0,
        _ptr(dG), _dt(dG) if dG is not None else F32, dG.stride(0) if dG is not None else 0, _ptr(workspace),
        workspace.numel(), _stream(stream)), "oversketch_matmul_backward")
    return dX, dG


def unsketch_cols(p: Plan, T, mask: int, scale: float, out_dtype="f32", out=None, stream=None):
    m = T.shape[0]
    od = _dtype_code(out_dtype)
    if out is None:
        out = torch.empty((m, p.n), dtype=_TORCH_DT[od], device=T.device)
    _check(load_library().oversketch_unsketch_cols(
        p.handle, _ptr(T), m, T.stride(0), mask, scale, _ptr(out), od, out.stride(0), _stream(stream)),
        "oversketch_unsketch_cols")
    return out


def unsketch_rows(p: Plan, U, mask: int, scale: float, out_dtype="f32", out=None, stream=None):
    l = U.shape[1]
    od = _dtype_code(out_dtype)
    if out is None:
        out = torch.empty((p.n, l), dtype=_TORCH_DT[od], device=U.device)
    _check(load_library().oversketch_unsketch_rows(
        p.handle, _ptr(U), l, U.stride(0), mask, scale, _ptr(out), od, out.stride(0), _stream(stream)),
        "oversketch_unsketch_rows")
    return out


def frob(X, Y=None, stream=None):
    """(sum (X-Y)^2, sum Y^2, sum X*Y) in FP64 on the device (Def. 4.1's norms)."""
    out = torch.empty(3, dtype=torch.float64, device=X.device)
    ws = torch.empty(FROB_WORKSPACE_BYTES, dtype=torch.uint8, device=X.device)
    _check(load_library().oversketch_frob(
        _ptr(X), X.stride(0), _ptr(Y), Y.stride(0) if Y is not None else 0, X.shape[0], X.shape[1],
        _ptr(out), _ptr(ws), ws.numel(), _stream(stream)), "oversketch_frob")
    return out


def device_status(reset=True, stream=None) -> int:
    """0 (OS_OK) or 6 (OS_ERR_TIMEOUT) from the tensor-core kernels' status word."""
    out = ctypes.c_int32()
    _check(load_library().oversketch_device_status(_stream(stream), ctypes.byref(out), 1 if reset else 0),
           "oversketch_device_status")
    return out.value


def test_wait_timeout(limit_ns: int, skip_kb: int):
    """Test hook: the next one-CTA tensor-core GEMM launch leaves K step skip_kb of
    its first tile unloaded and gives up after limit_ns (skip_kb < 0 withdraws it)."""
    _check(load_library().oversketch_test_wait_timeout(limit_ns, skip_kb), "oversketch_test_wait_timeout")


def sketch_left_noalloc(p: Plan, A: torch.Tensor, out: torch.Tensor, out_dtype="f32", col_scale=None,
                        scales=None, block_mask=0, stream=None):
    """A~ into the caller's `out` using the library's fixed 32 MiB scratch array
    instead of a workspace: for callers that cannot allocate device memory.
    Raises OverSketchError (OS_ERR_WORKSPACE) when the packed operand does not
    fit."""
    lda = _rowmajor(A, "A")
    od = _dtype_code(out_dtype)
    _check(load_library().oversketch_sketch_left_noalloc(
        p.handle, _ptr(A), _dt(A), A.shape[0], lda, _ptr(out), od, out.stride(0), _ptr(scales),
        _ptr(col_scale), block_mask, _stream(stream)), "oversketch_sketch_left_noalloc")
    return out


def gemm_bf16(A, B, alpha=1.0, beta=0.0, C=None, stream=None):
    """C = alpha * A . B^T (+ beta C) on the tensor cores; A m x K, B n x K, BF16 K-major."""
    lda, ldb = _rowmajor(A, "A"), _rowmajor(B, "B")
    m, K = A.shape
    n = B.shape[0]
    if C is None:
        C = torch.empty((m, n), dtype=torch.float32, device=A.device)
    _check(load_library().oversketch_gemm_bf16(_ptr(A), lda, _ptr(B), ldb, m, n, K, alpha, beta, _ptr(C),
                                               C.stride(0), _stream(stream)), "oversketch_gemm_bf16")
    return C


def select_transpose(X, out_dtype=None, block_mask=0, b=0, out=None, stream=None):
    """Y = X[:, selected columns]^T with an optional dtype conversion."""
    ldx = _rowmajor(X, "X")
    rows, cols = X.shape
    od = _dtype_code(out_dtype) if out_dtype is not None else _dt(X)
    ocols = cols if not block_mask else bin(block_mask).count("1") * b
    if out is None:
        out = torch.empty((ocols, _pad_ld(rows, od)), dtype=_TORCH_DT[od], device=X.device)[:, :rows]
    _check(load_library().oversketch_select_transpose(_ptr(X), _dt(X), rows, cols, ldx, block_mask, b, _ptr(out),
                                                      od, out.stride(0), _stream(stream)),
           "oversketch_select_transpose")
    return out


def cast(X, out_dtype, out=None, stream=None):
    ldx = _rowmajor(X, "X")
    rows, cols = X.shape
    od = _dtype_code(out_dtype)
    if out is None:
        out = torch.empty((rows, _pad_ld(cols, od)), dtype=_TORCH_DT[od], device=X.device)[:, :cols]
    _check(load_library().oversketch_cast(_ptr(X), _dt(X), rows, cols, ldx, _ptr(out), od, out.stride(0),
                                          _stream(stream)), "oversketch_cast")
    return out


def _batched_arrays(plans, ms, ns, ls):
    cnt = len(plans)
    P = (ctypes.c_void_p * cnt)(*[p.handle.value for p in plans])
    M = (ctypes.c_int64 * cnt)(*ms)
    Nn = (ctypes.c_int64 * cnt)(*ns)
    Lr = (ctypes.c_int64 * cnt)(*ls)
    return P, M, Nn, Lr


def matmul_batched_workspace(plans, ms, ns, ls, a_dtype=torch.float32, b_dtype=torch.float32) -> int:
    P, M, Nn, Lr = _batched_arrays(plans, ms, ns, ls)
    out = ctypes.c_size_t()
    o = _opts("bf16")
    _check(load_library().oversketch_matmul_batched_workspace_size(
        len(plans), P, M, Nn, Lr, _dtype_code(a_dtype), _dtype_code(b_dtype), ctypes.byref(o), ctypes.byref(out)),
        "oversketch_matmul_batched_workspace_size")
    return out.value


def matmul_batched(plans, As, Bs, Cs, masks, workspace=None, stream=None):
    """C_p = (1/k_p)(A_p S_p)(S_p^T B_p) for every p in one call (BF16 GEMM),
    the kept blocks of product p read from masks[p] on the device when the work
    runs (masks: int64 CUDA tensor of len(plans) words).  A_p, B_p: row-major
    CUDA tensors (one dtype per side), C_p: FP32 m_p x l_p, all contiguous."""
    cnt = len(plans)
    ms = [A.shape[0] for A in As]
    ns = [A.shape[1] for A in As]
    ls = [B.shape[1] for B in Bs]
    a_t, b_t = _dt(As[0]), _dt(Bs[0])
    for A, B, C in zip(As, Bs, Cs):
        if not (A.is_contiguous() and B.is_contiguous() and C.is_contiguous()):
            raise OverSketchError("matmul_batched: A, B and C must be contiguous")
        if _dt(A) != a_t or _dt(B) != b_t or C.dtype != torch.float32:
            raise OverSketchError("matmul_batched: one dtype per operand side, FP32 C")
    P, M, Nn, Lr = _batched_arrays(plans, ms, ns, ls)
    Ap = (ctypes.c_void_p * cnt)(*[A.data_ptr() for A in As])
    Bp = (ctypes.c_void_p * cnt)(*[B.data_ptr() for B in Bs])
    Cp = (ctypes.c_void_p * cnt)(*[C.data_ptr() for C in Cs])
    if workspace is None:
        workspace = torch.empty(matmul_batched_workspace(plans, ms, ns, ls, As[0].dtype, Bs[0].dtype),
                                dtype=torch.uint8, device=As[0].device)
    o = _opts("bf16")
    _check(load_library().oversketch_matmul_batched(
        cnt, P, Ap, Bp, Cp, M, Nn, Lr, a_t, b_t, _ptr(masks), ctypes.byref(o), _ptr(workspace), workspace.numel(),
        _stream(stream)), "oversketch_matmul_batched")
    return Cs


class Batch:
    """Many independent products run as one CUDA graph (oversketch_batch_*).

    ``problems``: list of (A, B, C, plan, mask) with A (m x n) and B (n x l)
    row-major CUDA tensors (FP32 or BF16, one dtype per side for the whole
    batch) and C (m x l) FP32.  The tensors are captured by address: keep
    them alive and in place while the batch exists.
    """

    def __init__(self, problems, gemm_dtype="bf16", workspace_limit=0, tune=False, stream=None):
        lib = load_library()
        arr = (_Problem * len(problems))()
        a_t = b_t = None
        self._keep = []
        for i, (A, B, C, plan, mask) in enumerate(problems):
            m, n = A.shape
            l = B.shape[1]
            arr[i] = _Problem(m, n, l, A.data_ptr(), _rowmajor(A, "A"), B.data_ptr(), _rowmajor(B, "B"),
                              C.data_ptr(), _rowmajor(C, "C"), plan.handle.value, mask)
            a_t = _dt(A) if a_t is None else a_t
            b_t = _dt(B) if b_t is None else b_t
            if _dt(A) != a_t or _dt(B) != b_t:
                raise OverSketchError("Batch: one dtype per operand side")
            self._keep.append((A, B, C, plan))
        h = ctypes.c_void_p()
        _check(lib.oversketch_batch_create(arr, len(problems), a_t, b_t, _dtype_code(gemm_dtype),
                                           workspace_limit, 1 if tune else 0, _stream(stream), ctypes.byref(h)),
               "oversketch_batch_create")
        self.handle = h

    def run(self, stream=None):
        _check(load_library().oversketch_batch_run(self.handle, _stream(stream)), "oversketch_batch_run")

    def info(self) -> dict:
        inf = _BatchInfo()
        _check(load_library().oversketch_batch_info(self.handle, ctypes.byref(inf)), "oversketch_batch_info")
        return {f: getattr(inf, f) for f, _ in _BatchInfo._fields_}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load_library().oversketch_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
