"""Python binding of libh2.so (ctypes).

Argument marshalling only: every step of the product and of the solve runs in
the CUDA library.  Functions keep the C names (``h2_build``, ``h2_matmul``,
``h2_matmul_transposed``, ``h2_block_cg``, ...).  Dense blocks are torch
tensors (device or host) or numpy arrays (host), float64, n×m with unit column
stride; PyTorch only supplies the memory and the stream.  If the compiled
library is missing the import of any entry point raises: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libh2.so")

H2_OK = 0
H2_E_BADARG = -1
H2_E_CUDA = -2
H2_E_NOCONVERGE = -3
H2_E_BREAKDOWN = -4
H2_E_TIMEOUT = -5
H2_E_OOM = -6
H2_E_UNSUPPORTED = -7

H2_F64, H2_F32, H2_BF16, H2_F32_MF = 0, 1, 2, 3
DTYPES = {"f64": H2_F64, "f32": H2_F32, "bf16": H2_BF16}  # also the precisions a build can add
# product dtypes: "f32mf" is the FP32 tensor-core product with the matrix-free coupling
PRODUCT_DTYPES = dict(DTYPES, f32mf=H2_F32_MF)
H2_CG_COLUMNWISE = 0
H2_CG_GRAM = 1
VARIANTS = {"columnwise": H2_CG_COLUMNWISE, "gram": H2_CG_GRAM}
H2_PRECOND_NONE = 0
H2_PRECOND_BLOCK_JACOBI = 1
PRECONDS = {None: H2_PRECOND_NONE, "none": H2_PRECOND_NONE, "block_jacobi": H2_PRECOND_BLOCK_JACOBI}

_STATUS = {0: "ok", -1: "badarg", -2: "cuda", -3: "noconverge", -4: "breakdown", -5: "timeout", -6: "oom",
           -7: "unsupported"}


class H2Error(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(code, code)} ({code}): {msg}")
        self.code = code


H2_KERNEL_EXP, H2_KERNEL_HELMHOLTZ = 0, 1
KERNELS = {"exp": H2_KERNEL_EXP, "helmholtz": H2_KERNEL_HELMHOLTZ}


class BuildParams(C.Structure):
    _fields_ = [("q", C.c_int32), ("leaf_size", C.c_int32), ("eta", C.c_double), ("length", C.c_double),
                ("sigma", C.c_double), ("precisions", C.c_uint32), ("stream", C.c_void_p),
                ("kernel", C.c_int32), ("kappa", C.c_double), ("delta", C.c_double)]


class Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("k", C.c_int64), ("n_clusters", C.c_int64), ("n_leaves", C.c_int64),
                ("n_adm", C.c_int64), ("n_near", C.c_int64), ("nnz_near", C.c_int64), ("depth", C.c_int32),
                ("q", C.c_int32), ("bytes_f64", C.c_int64), ("bytes_f32", C.c_int64), ("bytes_bf16", C.c_int64),
                ("flops_per_col", C.c_double), ("launches", C.c_int32), ("launches_tc", C.c_int32),
                ("kernel", C.c_int32), ("hybrid", C.c_int32), ("n_above_cut", C.c_int64)]


class CGParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("variant", C.c_int32),
                ("dtype", C.c_int32), ("refine", C.c_int32), ("inner_tol", C.c_double),
                ("max_outer", C.c_int32), ("check_every", C.c_int32), ("transposed", C.c_int32),
                ("precond", C.c_int32), ("stream", C.c_void_p)]


class GMRESParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("restart", C.c_int32), ("dtype", C.c_int32),
                ("precond", C.c_int32), ("transposed", C.c_int32), ("stream", C.c_void_p)]


class CGResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("outer_steps", C.c_int32),
                ("h2mm_calls", C.c_int32), ("col_iterations", C.POINTER(C.c_int32)),
                ("rel_residual", C.POINTER(C.c_double)), ("seconds", C.c_double)]


class TuneResult(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("m", C.c_int32), ("path", C.c_int32), ("stages", C.c_int32),
                ("up_target", C.c_int32), ("down_target", C.c_int32), ("n_candidates", C.c_int32),
                ("ms_best", C.c_double), ("ms", C.c_double * 16), ("cand_path", C.c_int32 * 16),
                ("cand_stages", C.c_int32 * 16), ("cand_up", C.c_int32 * 16), ("cand_down", C.c_int32 * 16)]


#: product paths of h2_autotune_ex
TUNE_PATHS = {1: "tensor cores, CUDA-core transfer passes", 2: "tensor cores, tensor-core transfer passes",
              3: "tensor cores, transfer passes fused with coupling and leaf phases", 4: "CUDA cores",
              5: "tensor cores, CUDA-core subtree passes, clusters above the upward cut in the coupling launch"}


class TreeView(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_clusters", C.c_int64), ("n_adm", C.c_int64), ("n_near", C.c_int64),
                ("depth", C.c_int32),
                ("perm", C.POINTER(C.c_int64)), ("cl_offset", C.POINTER(C.c_int64)),
                ("cl_size", C.POINTER(C.c_int64)), ("cl_level", C.POINTER(C.c_int32)),
                ("cl_parent", C.POINTER(C.c_int32)), ("cl_son0", C.POINTER(C.c_int32)),
                ("cl_son1", C.POINTER(C.c_int32)), ("cl_box", C.POINTER(C.c_double)),
                ("adm_rowptr", C.POINTER(C.c_int64)), ("adm_col", C.POINTER(C.c_int32)),
                ("near_rowptr", C.POINTER(C.c_int64)), ("near_col", C.POINTER(C.c_int32))]


#: every symbol include/h2.h declares
EXPORTS = ["h2_build", "h2_free", "h2_info", "h2_matmul", "h2_matmul_transposed", "h2_matmul_noalloc",
           "h2_matmul_complex", "h2_block_cg", "h2_block_gmres",
           "h2_timing_enable", "h2_timing_query", "h2_coupling_get", "h2_coupling_set", "h2_shift_set",
           "h2_adjoint_grads", "h2_batch_create", "h2_batch_free", "h2_batch_matmul", "h2_batch_block_cg",
           "h2_autotune", "h2_autotune_ex",
           "h2_tree_build", "h2_tree_view_get", "h2_tree_free", "h2_tree_schedule", "h2_set_alloc_limit",
           "h2_alloc_bytes", "h2_set_wait_limit", "h2_last_error_string", "h2_version"]
H2_NPHASE = 8
PHASES = ["gather", "leaf_fwd", "up", "coupling", "down", "leaf_bwd_near", "coupling_kernel"]

_lib = None


def lib() -> C.CDLL:
    """Load libh2.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    L.h2_build.argtypes = [C.POINTER(BuildParams), vp, i64, C.POINTER(vp)]
    L.h2_free.argtypes = [vp]
    L.h2_info.argtypes = [vp, C.POINTER(Info)]
    for f in (L.h2_matmul, L.h2_matmul_transposed, L.h2_matmul_noalloc):
        f.argtypes = [vp, dbl, vp, i64, vp, i64, i64, i32, vp]
    L.h2_matmul_complex.argtypes = [vp, dbl, dbl, vp, i64, vp, i64, i64, i32, vp]
    L.h2_block_cg.argtypes = [vp, vp, i64, vp, i64, i64, C.POINTER(CGParams), C.POINTER(CGResult)]
    L.h2_block_gmres.argtypes = [vp, vp, i64, vp, i64, i64, C.POINTER(GMRESParams), C.POINTER(CGResult)]
    L.h2_coupling_get.argtypes = [vp, vp, vp]
    L.h2_coupling_set.argtypes = [vp, vp, vp]
    L.h2_shift_set.argtypes = [vp, dbl]
    L.h2_adjoint_grads.argtypes = [vp, vp, i64, vp, i64, i64, vp, C.POINTER(C.c_double), vp]
    L.h2_batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(vp)]
    L.h2_batch_free.argtypes = [vp]
    L.h2_batch_matmul.argtypes = [vp, dbl, C.POINTER(vp), C.POINTER(i64), C.POINTER(vp), C.POINTER(i64),
                                  C.POINTER(i64), i32, vp]
    L.h2_batch_block_cg.argtypes = [vp, C.POINTER(vp), C.POINTER(i64), C.POINTER(vp), C.POINTER(i64),
                                    C.POINTER(i64), C.POINTER(CGParams), C.POINTER(CGResult)]
    L.h2_autotune.argtypes = [vp, i64, vp, C.POINTER(C.c_double)]
    L.h2_autotune_ex.argtypes = [vp, i64, i32, vp, C.POINTER(TuneResult)]
    L.h2_timing_enable.argtypes = [vp, i32]
    L.h2_timing_query.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), i32]
    L.h2_tree_build.argtypes = [C.POINTER(BuildParams), vp, i64, C.POINTER(vp)]
    L.h2_tree_view_get.argtypes = [vp, C.POINTER(TreeView)]
    L.h2_tree_free.argtypes = [vp]
    L.h2_tree_schedule.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), vp, vp]
    L.h2_set_alloc_limit.argtypes = [i64]
    L.h2_alloc_bytes.argtypes = [C.POINTER(i64)]
    L.h2_set_wait_limit.argtypes = [i64]
    L.h2_last_error_string.restype = C.c_char_p
    L.h2_version.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("h2_last_error_string", "h2_version"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(rc: int, where: str, ok=(0,)):
    if rc not in ok:
        raise H2Error(rc, where, lib().h2_last_error_string().decode())
    return rc


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr_ld(a, name: str, want_rows: int | None = None, writable=False):
    """(pointer, leading dimension, m, keepalive) of a float64 n×m block."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if a.dtype != torch.float64:
            raise TypeError(f"{name} must be float64")
        if a.dim() == 1:
            a = a.view(-1, 1)
        if a.dim() != 2 or (a.shape[1] > 1 and a.stride(1) != 1):
            raise ValueError(f"{name} must be 2-D with unit column stride")
        ld = a.stride(0) if a.shape[0] > 1 else a.shape[1]
        if want_rows is not None and a.shape[0] != want_rows:
            raise ValueError(f"{name} must have {want_rows} rows")
        return a.data_ptr(), int(ld), int(a.shape[1]), a
    arr = np.asarray(a)
    if arr.dtype != np.float64:
        raise TypeError(f"{name} must be float64")
    if arr.ndim == 1:
        arr = arr.reshape(-1, 1)
    if writable and not arr.flags.writeable:
        raise ValueError(f"{name} must be writable")
    if arr.strides[1] != 8 and arr.shape[1] > 1:
        raise ValueError(f"{name} must have unit column stride")
    if want_rows is not None and arr.shape[0] != want_rows:
        raise ValueError(f"{name} must have {want_rows} rows")
    ld = arr.strides[0] // 8 if arr.shape[0] > 1 else arr.shape[1]
    return arr.ctypes.data, int(ld), int(arr.shape[1]), arr


# ---------------------------------------------------------------------------
# C-named entry points
# ---------------------------------------------------------------------------
def h2_build(points, q=3, leaf_size=64, eta=2.0, length=0.5, sigma=1e-2, precisions=("f32",), stream=None,
             kernel="exp", kappa=1.0, delta=0.05):
    """Build the H² matrix of a point cloud; returns an opaque handle (int).
    kernel "exp": exp(-r/length); "helmholtz": exp(i·kappa·r)/(4π·sqrt(r² + delta²))
    (complex; multiply with h2_matmul_complex)."""
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64))
    if pts.ndim != 2 or pts.shape[1] != 3:
        raise ValueError("points must be n×3")
    mask = 0
    for p in precisions:
        mask |= 1 << DTYPES[p]
    bp = BuildParams(q, leaf_size, eta, length, sigma, mask, _stream_ptr(stream), KERNELS[kernel], kappa, delta)
    h = C.c_void_p()
    _check(lib().h2_build(C.byref(bp), pts.ctypes.data, pts.shape[0], C.byref(h)), "h2_build")
    return h.value


def h2_free(handle) -> None:
    lib().h2_free(handle)


def h2_info(handle) -> dict:
    info = Info()
    _check(lib().h2_info(handle, C.byref(info)), "h2_info")
    return {f: getattr(info, f) for f, _ in Info._fields_}


def _mm(fn, where, handle, alpha, X, Y, dtype, stream):
    info_n = h2_info(handle)["n"]
    xp, ldx, m, kx = _ptr_ld(X, "X", info_n)
    yp, ldy, my, ky = _ptr_ld(Y, "Y", info_n, writable=True)
    if my != m:
        raise ValueError("X and Y must have the same number of columns")
    dt = PRODUCT_DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    _check(fn(handle, float(alpha), xp, ldx, yp, ldy, m, dt, _stream_ptr(stream)), where)
    return Y


def h2_matmul(handle, alpha, X, Y, dtype="f64", stream=None):
    """Y += alpha·A·X (Y is updated in place and returned)."""
    return _mm(lib().h2_matmul, "h2_matmul", handle, alpha, X, Y, dtype, stream)


def _ptr_ld_complex(a, name: str, want_rows: int, writable=False):
    """(pointer, leading dimension in complex elements, m, keepalive) of a complex128 n×m block."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if a.dtype != torch.complex128:
            raise TypeError(f"{name} must be complex128")
        if a.dim() == 1:
            a = a.view(-1, 1)
        if a.dim() != 2 or (a.shape[1] > 1 and a.stride(1) != 1):
            raise ValueError(f"{name} must be 2-D with unit column stride")
        if a.shape[0] != want_rows:
            raise ValueError(f"{name} must have {want_rows} rows")
        ld = a.stride(0) if a.shape[0] > 1 else a.shape[1]
        return a.data_ptr(), int(ld), int(a.shape[1]), a
    arr = np.asarray(a)
    if arr.dtype != np.complex128:
        raise TypeError(f"{name} must be complex128")
    if arr.ndim == 1:
        arr = arr.reshape(-1, 1)
    if writable and not arr.flags.writeable:
        raise ValueError(f"{name} must be writable")
    if arr.strides[1] != 16 and arr.shape[1] > 1:
        raise ValueError(f"{name} must have unit column stride")
    if arr.shape[0] != want_rows:
        raise ValueError(f"{name} must have {want_rows} rows")
    ld = arr.strides[0] // 16 if arr.shape[0] > 1 else arr.shape[1]
    return arr.ctypes.data, int(ld), int(arr.shape[1]), arr


def h2_matmul_complex(handle, alpha, X, Y, dtype="f64", stream=None):
    """Y += alpha·A·X over C for a matrix built with kernel="helmholtz"; X, Y complex128
    (torch tensors on the device or host, or numpy arrays), alpha complex."""
    n = h2_info(handle)["n"]
    xp, ldx, m, kx = _ptr_ld_complex(X, "X", n)
    yp, ldy, my, ky = _ptr_ld_complex(Y, "Y", n, writable=True)
    if my != m:
        raise ValueError("X and Y must have the same number of columns")
    a = complex(alpha)
    dt = PRODUCT_DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    _check(lib().h2_matmul_complex(handle, a.real, a.imag, xp, ldx, yp, ldy, m, dt, _stream_ptr(stream)),
           "h2_matmul_complex")
    return Y


def h2_matmul_transposed(handle, alpha, X, Y, dtype="f64", stream=None):
    """Y += alpha·Aᵀ·X."""
    return _mm(lib().h2_matmul_transposed, "h2_matmul_transposed", handle, alpha, X, Y, dtype, stream)


def h2_timing_enable(handle, enable: bool = True) -> None:
    _check(lib().h2_timing_enable(handle, 1 if enable else 0), "h2_timing_enable")


def h2_timing_query(handle, reset: bool = False):
    """(dict phase -> accumulated ms, number of recorded products)."""
    ms = (C.c_double * H2_NPHASE)()
    calls = C.c_int64()
    _check(lib().h2_timing_query(handle, ms, C.byref(calls), 1 if reset else 0), "h2_timing_query")
    return {p: ms[i] for i, p in enumerate(PHASES)}, calls.value


def h2_matmul_noalloc(handle, alpha, X, Y, dtype="f64", stream=None):
    """Y += alpha·A·X without any device allocation (scratch is a fixed 32 MiB
    array inside the library; X and Y must be CUDA tensors).  For callers that
    cannot allocate at call time; see include/h2.h for the size limit and the
    rules on concurrent calls."""
    return _mm(lib().h2_matmul_noalloc, "h2_matmul_noalloc", handle, alpha, X, Y, dtype, stream)


def h2_set_alloc_limit(nbytes: int) -> None:
    """Cap the device bytes the process's matrices hold for their stored data (0: no cap)."""
    _check(lib().h2_set_alloc_limit(int(nbytes)), "h2_set_alloc_limit")


def h2_alloc_bytes() -> int:
    """Device bytes the live matrices hold for their stored data."""
    v = C.c_int64()
    _check(lib().h2_alloc_bytes(C.byref(v)), "h2_alloc_bytes")
    return v.value


def h2_set_wait_limit(polls: int) -> None:
    """Poll limit of the device-side flag waits (0: default; < 0: give up at once)."""
    _check(lib().h2_set_wait_limit(int(polls)), "h2_set_wait_limit")


def h2_coupling_get(handle, out=None):
    """FP64 coupling matrices S_b in admissible-list order, shape (n_adm, k, k)."""
    info = h2_info(handle)
    shape = (info["n_adm"], info["k"], info["k"])
    if out is None:
        out = np.zeros(shape)
    ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
    _check(lib().h2_coupling_get(handle, ptr, _stream_ptr(None)), "h2_coupling_get")
    return out


def h2_coupling_set(handle, S):
    """Replace the coupling matrices (FP64, shape (n_adm, k, k), host or device, contiguous)."""
    if hasattr(S, "data_ptr"):
        if not S.is_contiguous() or S.dtype.itemsize != 8:
            raise ValueError("S must be a contiguous float64 tensor")
        ptr = S.data_ptr()
    else:
        S = np.ascontiguousarray(S, dtype=np.float64)
        ptr = S.ctypes.data
    _check(lib().h2_coupling_set(handle, ptr, _stream_ptr(None)), "h2_coupling_set")


def h2_shift_set(handle, sigma: float):
    _check(lib().h2_shift_set(handle, float(sigma)), "h2_shift_set")


def h2_adjoint_grads(handle, L, X, dS=None, want_dsigma=True, stream=None):
    """(dS, dsigma) of a loss through X = A⁻¹B, given Λ = A⁻ᵀ ∂L/∂X (CUDA tensors).
    dS has shape (n_adm, k, k) on the device; pass dS=False to skip it."""
    import torch
    n = h2_info(handle)["n"]
    lp, ldl, m, kl = _ptr_ld(L, "L", n)
    xp, ldx, mx, kx = _ptr_ld(X, "X", n)
    if mx != m:
        raise ValueError("L and X must have the same number of columns")
    info = h2_info(handle)
    if dS is None:
        dS = torch.empty((info["n_adm"], info["k"], info["k"]), dtype=torch.float64, device=X.device)
    dsp = dS.data_ptr() if dS is not False else None
    ds = C.c_double(0.0)
    _check(lib().h2_adjoint_grads(handle, lp, ldl, xp, ldx, m, dsp, C.byref(ds) if want_dsigma else None,
                                  _stream_ptr(stream)), "h2_adjoint_grads")
    return (dS if dS is not False else None), (ds.value if want_dsigma else None)


@dataclass
class SolveResult:
    status: int
    iterations: int
    outer_steps: int
    h2mm_calls: int
    col_iterations: np.ndarray
    rel_residual: np.ndarray
    seconds: float

    @property
    def status_name(self) -> str:
        return _STATUS.get(self.status, str(self.status))


def h2_block_cg(handle, B, X, tol=1e-8, max_iter=20000, dtype="f64", refine=True, inner_tol=1e-4,
                max_outer=30, check_every=1, variant=H2_CG_COLUMNWISE, transposed=False, precond=None,
                stream=None) -> SolveResult:
    """Solve A X = B (X: initial guess in, solution out).  ``dtype`` is the
    precision of the product; with a low precision and ``refine`` the solve is
    an FP64 iterative refinement around low-precision block CG.  Returns the
    result; non-convergence and breakdown are reported in ``status``, not raised."""
    n = h2_info(handle)["n"]
    bp, ldb, m, kb = _ptr_ld(B, "B", n)
    xp, ldx, mx, kx = _ptr_ld(X, "X", n, writable=True)
    if mx != m:
        raise ValueError("B and X must have the same number of columns")
    it = np.zeros(max(m, 1), dtype=np.int32)
    rel = np.zeros(max(m, 1), dtype=np.float64)
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    pc = PRECONDS[precond] if precond is None or isinstance(precond, str) else int(precond)
    prm = CGParams(tol, max_iter, variant, dt, int(refine), inner_tol, max_outer, check_every,
                   1 if transposed else 0, pc, _stream_ptr(stream))
    res = CGResult(0, 0, 0, 0, it.ctypes.data_as(C.POINTER(C.c_int32)), rel.ctypes.data_as(C.POINTER(C.c_double)),
                   0.0)
    rc = lib().h2_block_cg(handle, bp, ldb, xp, ldx, m, C.byref(prm), C.byref(res))
    _check(rc, "h2_block_cg", ok=(H2_OK, H2_E_NOCONVERGE, H2_E_BREAKDOWN))
    return SolveResult(res.status, res.iterations, res.outer_steps, res.h2mm_calls, it[:m].copy(), rel[:m].copy(),
                       res.seconds)


def h2_block_gmres(handle, B, X, tol=1e-8, max_iter=20000, restart=30, dtype="f64", precond=None,
                   transposed=False, stream=None) -> SolveResult:
    """Block GMRES (restarted, per column, left-preconditioned): solve A X = B
    for device B and X (X: initial guess in, solution out).  Non-convergence is
    reported in ``status``, not raised."""
    n = h2_info(handle)["n"]
    bp, ldb, m, kb = _ptr_ld(B, "B", n)
    xp, ldx, mx, kx = _ptr_ld(X, "X", n, writable=True)
    if mx != m:
        raise ValueError("B and X must have the same number of columns")
    it = np.zeros(max(m, 1), dtype=np.int32)
    rel = np.zeros(max(m, 1), dtype=np.float64)
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    pc = PRECONDS[precond] if precond is None or isinstance(precond, str) else int(precond)
    prm = GMRESParams(tol, max_iter, restart, dt, pc, 1 if transposed else 0, _stream_ptr(stream))
    res = CGResult(0, 0, 0, 0, it.ctypes.data_as(C.POINTER(C.c_int32)), rel.ctypes.data_as(C.POINTER(C.c_double)),
                   0.0)
    rc = lib().h2_block_gmres(handle, bp, ldb, xp, ldx, m, C.byref(prm), C.byref(res))
    _check(rc, "h2_block_gmres", ok=(H2_OK, H2_E_NOCONVERGE))
    return SolveResult(res.status, res.iterations, res.outer_steps, res.h2mm_calls, it[:m].copy(), rel[:m].copy(),
                       res.seconds)


def h2_autotune(handle, m: int, stream=None):
    """Time the FP32 product on the tensor cores and on the CUDA cores and keep
    the faster; returns (ms tensor-core, ms CUDA-core)."""
    ms = (C.c_double * 2)()
    _check(lib().h2_autotune(handle, int(m), _stream_ptr(stream), ms), "h2_autotune")
    return ms[0], ms[1]


def h2_autotune_ex(handle, m: int, dtype="f32", stream=None) -> dict:
    """Tune the product of m columns in dtype for this matrix (path, stage count,
    transfer-pass cuts); returns the choice and every candidate's time."""
    r = TuneResult()
    _check(lib().h2_autotune_ex(handle, int(m), DTYPES[dtype], _stream_ptr(stream), C.byref(r)), "h2_autotune_ex")
    cands = [dict(path=r.cand_path[i], stages=r.cand_stages[i], up_target=r.cand_up[i], down_target=r.cand_down[i],
                  ms=r.ms[i]) for i in range(r.n_candidates)]
    return dict(path=r.path, path_name=TUNE_PATHS.get(r.path, "?"), stages=r.stages, up_target=r.up_target,
                down_target=r.down_target, ms=r.ms_best, candidates=cands)


class H2Batch:
    """Independent systems whose products and block-CG iterations run as one
    CUDA graph launch (h2_batch_*).  Holds references to the matrices."""

    def __init__(self, mats):
        self.mats = list(mats)
        arr = (C.c_void_p * len(self.mats))(*[mm.handle for mm in self.mats])
        h = C.c_void_p()
        _check(lib().h2_batch_create(arr, len(self.mats), C.byref(h)), "h2_batch_create")
        self.handle = h.value

    def _ptrs(self, blocks, name, writable=False):
        cnt = len(self.mats)
        ps, lds, ms, keep = (C.c_void_p * cnt)(), (C.c_int64 * cnt)(), (C.c_int64 * cnt)(), []
        for i, (mm, b) in enumerate(zip(self.mats, blocks)):
            p, ld, m, k = _ptr_ld(b, f"{name}[{i}]", mm.n, writable)
            ps[i], lds[i], ms[i] = p, ld, m
            keep.append(k)
        return ps, lds, ms, keep

    def matmul(self, Xs, Ys, alpha=1.0, dtype="f64", stream=None):
        xp, lx, mx, kx = self._ptrs(Xs, "X")
        yp, ly, my, ky = self._ptrs(Ys, "Y", True)
        dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        _check(lib().h2_batch_matmul(self.handle, float(alpha), xp, lx, yp, ly, mx, dt, _stream_ptr(stream)),
               "h2_batch_matmul")
        return Ys

    def block_cg(self, Bs, Xs, tol=1e-8, max_iter=20000, dtype="f32", inner_tol=0.1, check_every=4,
                 variant="columnwise", stream=None):
        bp, lb, mb, kb = self._ptrs(Bs, "B")
        xp, lx, mx, kx = self._ptrs(Xs, "X", True)
        cnt = len(self.mats)
        dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        var = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        prm = CGParams(tol, max_iter, var, dt, 2, inner_tol, 0, check_every, 0, H2_PRECOND_NONE,
                       _stream_ptr(stream))
        its = [np.zeros(max(int(mb[i]), 1), dtype=np.int32) for i in range(cnt)]
        rels = [np.zeros(max(int(mb[i]), 1)) for i in range(cnt)]
        res = (CGResult * cnt)()
        for i in range(cnt):
            res[i].col_iterations = its[i].ctypes.data_as(C.POINTER(C.c_int32))
            res[i].rel_residual = rels[i].ctypes.data_as(C.POINTER(C.c_double))
        rc = lib().h2_batch_block_cg(self.handle, bp, lb, xp, lx, mb, C.byref(prm), res)
        _check(rc, "h2_batch_block_cg", ok=(H2_OK, H2_E_NOCONVERGE, H2_E_BREAKDOWN))
        return [SolveResult(res[i].status, res[i].iterations, res[i].outer_steps, res[i].h2mm_calls,
                            its[i][: mb[i]].copy(), rels[i][: mb[i]].copy(), res[i].seconds) for i in range(cnt)]

    def close(self):
        if self.handle:
            lib().h2_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def h2_tree_build(points, leaf_size=64, eta=2.0, q=3) -> dict:
    """Host-only topology (no GPU): numpy copies of the trees and block lists."""
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64))
    bp = BuildParams(q, leaf_size, eta, 0.5, 0.0, 0, None)
    h = C.c_void_p()
    _check(lib().h2_tree_build(C.byref(bp), pts.ctypes.data, pts.shape[0], C.byref(h)), "h2_tree_build")
    try:
        v = TreeView()
        _check(lib().h2_tree_view_get(h, C.byref(v)), "h2_tree_view_get")
        nc = v.n_clusters

        def arr(ptr, count):
            return np.ctypeslib.as_array(ptr, shape=(count,)).copy() if count > 0 else np.zeros(0)

        return dict(
            n=v.n, n_clusters=nc, n_adm=v.n_adm, n_near=v.n_near, depth=v.depth,
            perm=arr(v.perm, v.n), offset=arr(v.cl_offset, nc), size=arr(v.cl_size, nc),
            level=arr(v.cl_level, nc), parent=arr(v.cl_parent, nc), son0=arr(v.cl_son0, nc),
            son1=arr(v.cl_son1, nc), box=arr(v.cl_box, 6 * nc).reshape(nc, 6),
            adm_rowptr=arr(v.adm_rowptr, nc + 1), adm_col=arr(v.adm_col, v.n_adm),
            near_rowptr=arr(v.near_rowptr, nc + 1), near_col=arr(v.near_col, v.n_near),
        )
    finally:
        lib().h2_tree_free(h)


def h2_tree_schedule(points, which, leaf_size=64, eta=2.0, q=3) -> dict:
    """Host-only: the FP32/BF16 transfer-pass schedule of the tree of `points`
    (which = "down" or "up"): task_ptr [ntasks+1], steps [nsteps, 4] and the
    stack depth, as h2_build uses them."""
    w = {"down": 0, "up": 1}[which]
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64))
    bp = BuildParams(q, leaf_size, eta, 0.5, 0.0, 0, None)
    h = C.c_void_p()
    _check(lib().h2_tree_build(C.byref(bp), pts.ctypes.data, pts.shape[0], C.byref(h)), "h2_tree_build")
    try:
        nt, ns, ent = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().h2_tree_schedule(h, w, C.byref(nt), C.byref(ns), C.byref(ent), None, None), "h2_tree_schedule")
        ptr = np.zeros(nt.value + 1, dtype=np.int32)
        steps = np.zeros((ns.value, 4), dtype=np.int32)
        _check(lib().h2_tree_schedule(h, w, C.byref(nt), C.byref(ns), C.byref(ent), ptr.ctypes.data,
                                      steps.ctypes.data), "h2_tree_schedule")
        return dict(task_ptr=ptr, steps=steps, entries=ent.value)
    finally:
        lib().h2_tree_free(h)


class H2Matrix:
    """Owning wrapper around an h2_matrix handle."""

    def __init__(self, points, q=3, leaf_size=64, eta=2.0, length=0.5, sigma=1e-2, precisions=("f32",),
                 stream=None, kernel="exp", kappa=1.0, delta=0.05):
        self.handle = h2_build(points, q, leaf_size, eta, length, sigma, precisions, stream, kernel, kappa, delta)
        self.kernel = kernel
        self.info = h2_info(self.handle)
        self.n = self.info["n"]

    def matmul(self, X, Y, alpha=1.0, dtype="f64", stream=None):
        return h2_matmul(self.handle, alpha, X, Y, dtype, stream)

    def matmul_transposed(self, X, Y, alpha=1.0, dtype="f64", stream=None):
        return h2_matmul_transposed(self.handle, alpha, X, Y, dtype, stream)

    def matmul_complex(self, X, Y, alpha=1.0, dtype="f64", stream=None):
        return h2_matmul_complex(self.handle, alpha, X, Y, dtype, stream)

    def block_cg(self, B, X, **kw) -> SolveResult:
        return h2_block_cg(self.handle, B, X, **kw)

    def block_gmres(self, B, X, **kw) -> SolveResult:
        return h2_block_gmres(self.handle, B, X, **kw)

    def flops(self, m: int) -> float:
        return self.info["flops_per_col"] * m

    def close(self):
        if self.handle:
            h2_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
