"""Python binding of the C ABI in include/kk_spgemm.h (argument marshalling only).

Every function named ``kk_*`` here calls the C function of the same name in
``libkk_spgemm.so`` with raw device pointers taken from torch tensors; all
computation runs in the library's CUDA kernels.  Loading fails loudly when the
library is missing: there is no CPU fallback.

Higher-level helpers (``DeviceCSR``, ``SpGEMM``, ``spgemm``) allocate C's arrays
with torch between the symbolic and numeric phases, as the two-phase method
requires (Kokkos Kernels paper, Sec. "Standard SpGEMM Kernel": row pointers
first, symbolic, then column indices and values of size nnz(C), numeric).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libkk_spgemm.so")
_lock = threading.Lock()
_lib = None

KK_OK = 0
STATUS_NAMES = {
    0: "KK_OK", 1: "KK_ERR_INVALID_ARG", 2: "KK_ERR_CUDA", 3: "KK_ERR_OOM",
    4: "KK_ERR_STRUCTURE_MISMATCH", 5: "KK_ERR_CAPACITY", 6: "KK_ERR_TIMEOUT",
    7: "KK_ERR_NOT_SYMBOLIC", 8: "KK_ERR_BAD_INDEX",
}
KK_ARITH_AUTO, KK_ARITH_FP64, KK_ARITH_DF32 = 0, 1, 2


class KKError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {detail}")


class KkCsr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p), ("vals", ctypes.c_void_p)]


class KkOptions(ctypes.Structure):
    _fields_ = [("arith", ctypes.c_int32), ("debug_checks", ctypes.c_int32),
                ("timing", ctypes.c_int32), ("force_tier", ctypes.c_int32),
                ("team_vec_min_len", ctypes.c_int32), ("sym_team_max_flop", ctypes.c_int32),
                ("sym_cta_max_flop", ctypes.c_int32), ("num_team_max_nnz", ctypes.c_int32),
                ("num_cta_max_nnz", ctypes.c_int32), ("use_window", ctypes.c_int32),
                ("batched_graph", ctypes.c_int32), ("sym_load_pct", ctypes.c_int32),
                ("num_load_pct", ctypes.c_int32), ("structure_cache", ctypes.c_int32),
                ("wide_cache_mb", ctypes.c_int32), ("batched_mode", ctypes.c_int32),
                ("batched_learned", ctypes.c_int32), ("stage_long_rows", ctypes.c_int32),
                ("small_max_rows", ctypes.c_int32)]


# exported symbol -> (restype, argtypes)
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_SIGS = {
    "kk_spgemm_options_default": (_I32, [ctypes.POINTER(KkOptions)]),
    "kk_spgemm_handle_create": (_I32, [ctypes.POINTER(_P), ctypes.POINTER(KkOptions), _P]),
    "kk_spgemm_set_stream": (_I32, [_P, _P]),
    "kk_spgemm_symbolic": (_I32, [_P, ctypes.POINTER(KkCsr), ctypes.POINTER(KkCsr), _P,
                                  ctypes.POINTER(ctypes.c_int64)]),
    "kk_spgemm_numeric": (_I32, [_P, ctypes.POINTER(KkCsr), ctypes.POINTER(KkCsr), _P, _P, _P]),
    "kk_spgemm_sync": (_I32, [_P]),
    "kk_spgemm_destroy": (_I32, [_P]),
    "kk_status_string": (ctypes.c_char_p, [_I32]),
    "kk_spgemm_last_error": (ctypes.c_char_p, [_P]),
    "kk_spgemm_last_arith": (_I32, [_P]),
    "kk_spgemm_kernel_times": (_I32, [_P, _I32, ctypes.POINTER(ctypes.c_char_p),
                                      ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_I32), _I32]),
    "kk_spgemm_stats": (_I32, [_P, ctypes.POINTER(ctypes.c_int64)]),
    # result download helper (include/kk_copy.h)
    "kk_copy_to_host": (_I32, [_P, _P, _P, ctypes.c_size_t]),
    # sparse matrix addition (include/kk_spadd.h)
    "kk_spadd_symbolic": (_I32, [_P, ctypes.POINTER(KkCsr), ctypes.POINTER(KkCsr), _P,
                                 ctypes.POINTER(ctypes.c_int64)]),
    "kk_spadd_numeric": (_I32, [_P, ctypes.c_double, ctypes.POINTER(KkCsr), ctypes.c_double,
                                ctypes.POINTER(KkCsr), _P, _P, _P]),
    # Jacobi-fused numeric phase (include/kk_jacobi.h)
    "kk_spgemm_jacobi_numeric": (_I32, [_P, ctypes.c_double, ctypes.POINTER(KkCsr),
                                        ctypes.POINTER(KkCsr), _P, _P, _P]),
    # learned form (include/kk_learned.h)
    "kk_spgemm_row_features": (_I32, [_P, ctypes.POINTER(KkCsr), ctypes.POINTER(KkCsr), _P]),
    "kk_capacity_classes": (_I32, [_P, _I32, _P, _P]),
    "kk_mlp_init": (_I32, [_P, _P, ctypes.c_uint64]),
    "kk_mlp_loss_grad": (_I32, [_P, _I32, _P, _P, _P, _P, _P]),
    "kk_mlp_adam": (_I32, [_P, _P, _P, _P, _P, _I32, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, ctypes.c_float]),
    "kk_mlp_train": (_I32, [_P, _I32, _P, _P, _P, _I32, _I32, ctypes.c_float, ctypes.c_uint64,
                            ctypes.POINTER(ctypes.c_float)]),
    "kk_mlp_predict": (_I32, [_P, _I32, _P, _P, ctypes.c_float, _P]),
    "kk_spgemm_set_predictor": (_I32, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_float]),
    "kk_spgemm_learned_symbolic": (_I32, [_P, ctypes.POINTER(KkCsr), ctypes.POINTER(KkCsr), _P,
                                          ctypes.POINTER(ctypes.c_int64)]),
    "kk_spgemm_learned_numeric": (_I32, [_P, ctypes.POINTER(KkCsr), ctypes.POINTER(KkCsr), _P, _P,
                                         _P]),
}
MLP_FEATURES, MLP_CLASSES, MLP_NUM_PARAMS = 8, 16, 1872


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libkk_spgemm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(
                    f"{_LIB_PATH} is missing: build it with paper_2103_11991_gb300._build.build() "
                    "(nvcc, sm_103a); there is no CPU fallback")
            lib = ctypes.CDLL(_LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status: int, handle=None):
    if status != KK_OK:
        detail = ""
        if handle:
            raw = load_library().kk_spgemm_last_error(handle)
            detail = raw.decode() if raw else ""
        raise KKError(status, detail)


# ----------------------------------------------------------------------------
# Same-name wrappers of the C ABI
# ----------------------------------------------------------------------------
def kk_spgemm_options_default() -> KkOptions:
    o = KkOptions()
    _check(load_library().kk_spgemm_options_default(ctypes.byref(o)))
    return o


def kk_spgemm_handle_create(opt: KkOptions | None = None, stream=None):
    """Returns an opaque handle (int).  ``stream``: a torch.cuda.Stream, a raw
    cudaStream_t int, or None for torch's current stream."""
    import torch
    h = _P()
    if stream is None:
        stream = torch.cuda.current_stream()
    raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(load_library().kk_spgemm_handle_create(ctypes.byref(h),
                                                  ctypes.byref(opt) if opt is not None else None,
                                                  ctypes.c_void_p(raw)))
    return h.value


def kk_spgemm_set_stream(h, stream):
    raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(load_library().kk_spgemm_set_stream(h, ctypes.c_void_p(raw)), h)


def kk_spgemm_symbolic(h, A: "DeviceCSR", B: "DeviceCSR", c_rowptr) -> int:
    nnz = ctypes.c_int64(0)
    a, b = A.abi(), B.abi()
    _check(load_library().kk_spgemm_symbolic(h, ctypes.byref(a), ctypes.byref(b),
                                             ctypes.c_void_p(c_rowptr.data_ptr()),
                                             ctypes.byref(nnz)), h)
    return int(nnz.value)


def kk_spgemm_numeric(h, A: "DeviceCSR", B: "DeviceCSR", c_rowptr, c_colind, c_vals):
    a, b = A.abi(), B.abi()
    _check(load_library().kk_spgemm_numeric(h, ctypes.byref(a), ctypes.byref(b),
                                            ctypes.c_void_p(c_rowptr.data_ptr()),
                                            ctypes.c_void_p(c_colind.data_ptr()),
                                            ctypes.c_void_p(c_vals.data_ptr())), h)


def kk_spgemm_jacobi_numeric(h, omega: float, A: "DeviceCSR", B: "DeviceCSR", c_rowptr, c_colind,
                             c_vals):
    a, b = A.abi(), B.abi()
    _check(load_library().kk_spgemm_jacobi_numeric(h, ctypes.c_double(float(omega)), ctypes.byref(a),
                                                   ctypes.byref(b),
                                                   ctypes.c_void_p(c_rowptr.data_ptr()),
                                                   ctypes.c_void_p(c_colind.data_ptr()),
                                                   ctypes.c_void_p(c_vals.data_ptr())), h)


def kk_spadd_symbolic(h, A: "DeviceCSR", B: "DeviceCSR", c_rowptr) -> int:
    a, b = A.abi(), B.abi()
    nnz = ctypes.c_int64(0)
    _check(load_library().kk_spadd_symbolic(h, ctypes.byref(a), ctypes.byref(b),
                                            ctypes.c_void_p(c_rowptr.data_ptr()), ctypes.byref(nnz)), h)
    return int(nnz.value)


def kk_spadd_numeric(h, alpha: float, A: "DeviceCSR", beta: float, B: "DeviceCSR", c_rowptr, c_colind,
                     c_vals):
    a, b = A.abi(), B.abi()
    _check(load_library().kk_spadd_numeric(h, ctypes.c_double(float(alpha)), ctypes.byref(a),
                                           ctypes.c_double(float(beta)), ctypes.byref(b),
                                           ctypes.c_void_p(c_rowptr.data_ptr()),
                                           ctypes.c_void_p(c_colind.data_ptr()),
                                           ctypes.c_void_p(c_vals.data_ptr())), h)


def kk_copy_to_host(dst, src, stream=None):
    """Copy device tensor ``src`` into page-locked host tensor ``dst`` (same
    number of bytes) with the library's streaming kernel on ``stream`` (a
    torch.cuda.Stream; default torch's current stream).  Asynchronous."""
    import torch
    nbytes = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() < nbytes:
        raise ValueError("destination smaller than source")
    if stream is None:
        stream = torch.cuda.current_stream()
    raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(load_library().kk_copy_to_host(ctypes.c_void_p(raw), ctypes.c_void_p(dst.data_ptr()),
                                          ctypes.c_void_p(src.data_ptr()), ctypes.c_size_t(nbytes)))


def kk_spgemm_sync(h):
    _check(load_library().kk_spgemm_sync(h), h)


def kk_spgemm_destroy(h):
    _check(load_library().kk_spgemm_destroy(h))


def kk_status_string(s: int) -> str:
    return load_library().kk_status_string(s).decode()


def kk_spgemm_last_arith(h) -> int:
    return int(load_library().kk_spgemm_last_arith(h))


def kk_spgemm_kernel_times(h, reset: bool = False) -> dict:
    lib = load_library()
    n = 64
    names = (ctypes.c_char_p * n)()
    ms = (ctypes.c_double * n)()
    launches = (ctypes.c_int64 * n)()
    count = _I32(0)
    _check(lib.kk_spgemm_kernel_times(h, n, names, ms, launches, ctypes.byref(count), int(reset)), h)
    return {names[i].decode(): (ms[i], launches[i]) for i in range(min(count.value, n))}


def kk_spgemm_stats(h) -> dict:
    arr = (ctypes.c_int64 * 32)()
    _check(load_library().kk_spgemm_stats(h, arr), h)
    keys = ["sym_team_rows", "sym_cta_rows", "sym_dense_rows", "num_team_rows", "num_cta_rows",
            "num_dense_rows", "flops", "b_sorted", "launches_sym", "launches_num",
            "sym_window_rows", "num_window_rows", "onepass_rows", "overflow_rows", "heavy_rows",
            "staging_entries", "num_team_c", "num_cta_c", "num_dense_c", "num_window_c",
            "num_team_a", "num_cta_a", "num_dense_a", "num_window_a", "kept_structure_rows",
            "compressed_b_pairs", "num_team_f", "num_cta_f", "num_dense_f", "num_window_f",
            "small_path_rows"]
    return {k: int(arr[i]) for i, k in enumerate(keys)}


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def kk_spgemm_row_features(h, A: "DeviceCSR", B: "DeviceCSR", features):
    a, b = A.abi(), B.abi()
    _check(load_library().kk_spgemm_row_features(h, ctypes.byref(a), ctypes.byref(b),
                                                 ctypes.c_void_p(features.data_ptr())), h)


def kk_capacity_classes(m: int, c_rowptr, cls, stream=None):
    _check(load_library().kk_capacity_classes(_stream_ptr(stream), int(m),
                                              ctypes.c_void_p(c_rowptr.data_ptr()),
                                              ctypes.c_void_p(cls.data_ptr())))


def kk_mlp_init(params, seed: int, stream=None):
    _check(load_library().kk_mlp_init(_stream_ptr(stream), ctypes.c_void_p(params.data_ptr()),
                                      ctypes.c_uint64(seed)))


def kk_mlp_loss_grad(X, y, params, grad, loss, stream=None):
    _check(load_library().kk_mlp_loss_grad(_stream_ptr(stream), int(X.shape[0]),
                                           ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                           ctypes.c_void_p(params.data_ptr()),
                                           ctypes.c_void_p(grad.data_ptr()),
                                           ctypes.c_void_p(loss.data_ptr())))


def kk_mlp_adam(grad, params, m1, m2, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load_library().kk_mlp_adam(_stream_ptr(stream), ctypes.c_void_p(grad.data_ptr()),
                                      ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(m1.data_ptr()),
                                      ctypes.c_void_p(m2.data_ptr()), int(step), lr, beta1, beta2, eps))


def kk_mlp_train(X, y, params, epochs=20, batch=4096, lr=3e-3, seed=0, stream=None) -> float:
    out = ctypes.c_float(0.0)
    _check(load_library().kk_mlp_train(_stream_ptr(stream), int(X.shape[0]), ctypes.c_void_p(X.data_ptr()),
                                       ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(params.data_ptr()),
                                       int(epochs), int(batch), float(lr), ctypes.c_uint64(seed),
                                       ctypes.byref(out)))
    return float(out.value)


def kk_mlp_predict(X, params, cls, quantile=0.0, stream=None):
    _check(load_library().kk_mlp_predict(_stream_ptr(stream), int(X.shape[0]), ctypes.c_void_p(X.data_ptr()),
                                         ctypes.c_void_p(params.data_ptr()), float(quantile),
                                         ctypes.c_void_p(cls.data_ptr())))


def kk_spgemm_set_predictor(h, params_host, quantile: float = 0.95):
    if params_host is None:
        _check(load_library().kk_spgemm_set_predictor(h, None, float(quantile)), h)
        return
    arr = np.ascontiguousarray(params_host, dtype=np.float32)
    if arr.size != MLP_NUM_PARAMS:
        raise ValueError("predictor needs %d parameters" % MLP_NUM_PARAMS)
    _check(load_library().kk_spgemm_set_predictor(h, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                  float(quantile)), h)


def kk_spgemm_learned_symbolic(h, A: "DeviceCSR", B: "DeviceCSR", c_rowptr) -> int:
    nnz = ctypes.c_int64(0)
    a, b = A.abi(), B.abi()
    _check(load_library().kk_spgemm_learned_symbolic(h, ctypes.byref(a), ctypes.byref(b),
                                                     ctypes.c_void_p(c_rowptr.data_ptr()),
                                                     ctypes.byref(nnz)), h)
    return int(nnz.value)


def kk_spgemm_learned_numeric(h, A: "DeviceCSR", B: "DeviceCSR", c_rowptr, c_colind, c_vals):
    a, b = A.abi(), B.abi()
    _check(load_library().kk_spgemm_learned_numeric(h, ctypes.byref(a), ctypes.byref(b),
                                                    ctypes.c_void_p(c_rowptr.data_ptr()),
                                                    ctypes.c_void_p(c_colind.data_ptr()),
                                                    ctypes.c_void_p(c_vals.data_ptr())), h)


# ----------------------------------------------------------------------------
# Device CSR and a small object API on top of the C ABI
# ----------------------------------------------------------------------------
class DeviceCSR:
    """A CSR matrix in device memory (torch tensors).  rowptr int32 (int64 for
    outputs of the product), colind int32, vals float64."""

    def __init__(self, m, n, rowptr, colind, vals):
        self.m, self.n = int(m), int(n)
        self.rowptr, self.colind, self.vals = rowptr, colind, vals

    @property
    def nnz(self) -> int:
        return int(self.colind.numel())

    @classmethod
    def from_host(cls, M, device="cuda", non_blocking=False):
        import torch
        rp = torch.from_numpy(np.ascontiguousarray(M.rowptr, dtype=np.int32)).to(device, non_blocking=non_blocking)
        ci = torch.from_numpy(np.ascontiguousarray(M.colind, dtype=np.int32)).to(device, non_blocking=non_blocking)
        va = torch.from_numpy(np.ascontiguousarray(M.vals, dtype=np.float64)).to(device, non_blocking=non_blocking)
        return cls(M.m, M.n, rp, ci, va)

    def abi(self) -> KkCsr:
        if self.rowptr.dtype.itemsize != 4:
            raise TypeError("the C ABI takes int32 row pointers for A and B")
        return KkCsr(self.m, self.n, self.nnz, self.rowptr.data_ptr(),
                     self.colind.data_ptr() if self.nnz else None,
                     self.vals.data_ptr() if (self.vals is not None and self.nnz) else None)

    def to_host(self):
        from paper_2103_11991_gb300.inputs import CSR
        return CSR(self.m, self.n, self.rowptr.cpu().numpy(), self.colind.cpu().numpy(),
                   self.vals.cpu().numpy())


def make_options(**kw) -> KkOptions:
    o = kk_spgemm_options_default()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, int(v))
    return o


class SpGEMM:
    """Owns a handle; ``symbolic`` returns C's int64 row pointers and nnz(C),
    ``numeric`` fills freshly allocated (or given) colind / vals."""

    def __init__(self, stream=None, **options):
        self.opt = make_options(**options)
        self.h = kk_spgemm_handle_create(self.opt, stream)

    def symbolic(self, A: DeviceCSR, B: DeviceCSR):
        import torch
        rowptr = torch.empty(A.m + 1, dtype=torch.int64, device=A.rowptr.device)
        nnz = kk_spgemm_symbolic(self.h, A, B, rowptr)
        return rowptr, nnz

    def numeric(self, A: DeviceCSR, B: DeviceCSR, rowptr, nnz, colind=None, vals=None):
        import torch
        dev = A.rowptr.device
        if colind is None:
            colind = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
        if vals is None:
            vals = torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)
        kk_spgemm_numeric(self.h, A, B, rowptr, colind, vals)
        return colind[:nnz], vals[:nnz]

    def spadd_symbolic(self, A: DeviceCSR, B: DeviceCSR):
        """Structure of C = alpha A + beta B: (int64 row pointers, nnz(C))."""
        import torch
        rowptr = torch.empty(A.m + 1, dtype=torch.int64, device=A.rowptr.device)
        return rowptr, kk_spadd_symbolic(self.h, A, B, rowptr)

    def spadd_numeric(self, alpha: float, A: DeviceCSR, beta: float, B: DeviceCSR, rowptr, nnz,
                      colind=None, vals=None):
        import torch
        dev = A.rowptr.device
        if colind is None:
            colind = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
        if vals is None:
            vals = torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)
        kk_spadd_numeric(self.h, alpha, A, beta, B, rowptr, colind, vals)
        return colind[:nnz], vals[:nnz]

    def jacobi_numeric(self, A: DeviceCSR, B: DeviceCSR, rowptr, nnz, omega: float, colind=None,
                       vals=None):
        """C = (I - omega D^-1 A) B on the structure of the last symbolic call
        of (A, B) on this handle."""
        import torch
        dev = A.rowptr.device
        if colind is None:
            colind = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
        if vals is None:
            vals = torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)
        kk_spgemm_jacobi_numeric(self.h, omega, A, B, rowptr, colind, vals)
        return colind[:nnz], vals[:nnz]

    def __call__(self, A: DeviceCSR, B: DeviceCSR) -> DeviceCSR:
        rowptr, nnz = self.symbolic(A, B)
        colind, vals = self.numeric(A, B, rowptr, nnz)
        return DeviceCSR(A.m, B.n, rowptr, colind, vals)

    def set_predictor(self, params, quantile: float = 0.95):
        kk_spgemm_set_predictor(self.h, params, quantile)

    def learned_symbolic(self, A: DeviceCSR, B: DeviceCSR):
        import torch
        rowptr = torch.empty(A.m + 1, dtype=torch.int64, device=A.rowptr.device)
        nnz = kk_spgemm_learned_symbolic(self.h, A, B, rowptr)
        return rowptr, nnz

    def learned_numeric(self, A: DeviceCSR, B: DeviceCSR, rowptr, nnz, colind=None, vals=None):
        import torch
        dev = A.rowptr.device
        if colind is None:
            colind = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
        if vals is None:
            vals = torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)
        kk_spgemm_learned_numeric(self.h, A, B, rowptr, colind, vals)
        return colind[:nnz], vals[:nnz]

    def sync(self):
        kk_spgemm_sync(self.h)

    def kernel_times(self, reset=False):
        return kk_spgemm_kernel_times(self.h, reset)

    def stats(self):
        return kk_spgemm_stats(self.h)

    def last_arith(self):
        return kk_spgemm_last_arith(self.h)

    def close(self):
        if self.h:
            kk_spgemm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spgemm(A: DeviceCSR, B: DeviceCSR, **options) -> DeviceCSR:
    """C = A*B on the GPU (symbolic, allocate, numeric, sync)."""
    with SpGEMM(**options) as op:
        C = op(A, B)
        op.sync()
    return C


# ----------------------------------------------------------------------------
# Batched form (include/kk_batched.h)
# ----------------------------------------------------------------------------
_SIGS.update({
    "kk_spgemm_batched_symbolic": (_I32, [_P, _I32, ctypes.POINTER(KkCsr), ctypes.POINTER(KkCsr), _P,
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "kk_spgemm_batched_numeric": (_I32, [_P, _I32, ctypes.POINTER(KkCsr), ctypes.POINTER(KkCsr), _P, _P, _P]),
})


def _csr_array(mats):
    arr = (KkCsr * max(1, len(mats)))()
    for k, M in enumerate(mats):
        arr[k] = M.abi()
    return arr


def kk_spgemm_batched_symbolic(h, As, Bs, c_rowptr):
    """Returns (offsets as a numpy int64[count + 1], total nnz)."""
    lib = load_library()
    count = len(As)
    a, b = _csr_array(As), _csr_array(Bs)
    off = np.zeros(count + 1, dtype=np.int64)
    total = ctypes.c_int64(0)
    _check(lib.kk_spgemm_batched_symbolic(h, count, a, b,
                                          ctypes.c_void_p(c_rowptr.data_ptr()) if c_rowptr is not None else None,
                                          off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                          ctypes.byref(total)), h)
    return off, int(total.value)


def kk_spgemm_batched_numeric(h, As, Bs, c_rowptr, c_colind, c_vals):
    lib = load_library()
    a, b = _csr_array(As), _csr_array(Bs)
    _check(lib.kk_spgemm_batched_numeric(h, len(As), a, b, ctypes.c_void_p(c_rowptr.data_ptr()),
                                         ctypes.c_void_p(c_colind.data_ptr()),
                                         ctypes.c_void_p(c_vals.data_ptr())), h)


class BatchedSpGEMM:
    """Batched products C_k = A_k * B_k on one handle (stream: a non-default
    torch.cuda.Stream enables CUDA-graph capture and replay)."""

    def __init__(self, stream=None, **options):
        self.opt = make_options(**options)
        self.stream = stream
        self.h = kk_spgemm_handle_create(self.opt, stream)

    def set_predictor(self, params, quantile: float = 0.95):
        """Predictor for the learned form of the packed batch (option
        ``batched_learned=1``)."""
        kk_spgemm_set_predictor(self.h, params, quantile)

    def symbolic(self, As, Bs):
        import torch
        R = sum(A.m for A in As)
        dev = As[0].rowptr.device if As else "cuda"
        rowptr = torch.empty(R + 1, dtype=torch.int64, device=dev)
        off, total = kk_spgemm_batched_symbolic(self.h, As, Bs, rowptr)
        return rowptr, off, total

    def numeric(self, As, Bs, rowptr, total, colind=None, vals=None):
        import torch
        dev = rowptr.device
        if colind is None:
            colind = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
        if vals is None:
            vals = torch.empty(max(total, 1), dtype=torch.float64, device=dev)
        kk_spgemm_batched_numeric(self.h, As, Bs, rowptr, colind, vals)
        return colind, vals

    def sync(self):
        kk_spgemm_sync(self.h)

    def stats(self):
        return kk_spgemm_stats(self.h)

    def kernel_times(self, reset=False):
        return kk_spgemm_kernel_times(self.h, reset)

    def close(self):
        if self.h:
            kk_spgemm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# Symbolic phase without allocation (include/kk_noalloc.h)
# ----------------------------------------------------------------------------
_SIGS.update({
    "kk_spgemm_symbolic_noalloc": (_I32, [ctypes.POINTER(KkCsr), ctypes.POINTER(KkCsr), _P,
                                          ctypes.POINTER(ctypes.c_int64), _P]),
})
NOALLOC_MAX_ROWS = 1 << 20


def kk_spgemm_symbolic_noalloc(A: "DeviceCSR", B: "DeviceCSR", c_rowptr, stream=None) -> int:
    """Row pointers of C = A*B into c_rowptr (int64[A.m + 1]) using only the
    library's fixed device scratch; returns nnz(C)."""
    lib = load_library()
    nnz = ctypes.c_int64(0)
    a, b = A.abi(), B.abi()
    _check(lib.kk_spgemm_symbolic_noalloc(ctypes.byref(a), ctypes.byref(b),
                                          ctypes.c_void_p(c_rowptr.data_ptr()), ctypes.byref(nnz),
                                          _stream_ptr(stream)))
    return int(nnz.value)
