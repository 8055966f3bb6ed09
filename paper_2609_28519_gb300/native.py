"""Thin ctypes binding of ``libbdct.so`` (argument marshalling only).

Every function here maps one-to-one onto an ``include/bdct.h`` entry point:
it checks tensor dtypes and shapes, passes raw device pointers and the
current CUDA stream, and turns a non-zero status into ``BdctError``.  No
step of a transform runs in Python, and there is no fallback: if the library
is missing the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbdct.so")

# kinds, norms, paths, statuses (mirrors include/bdct.h)
FORWARD, INVERSE, ROUNDTRIP, SPECTRAL = 1, 2, 4, 8
NORM_ORTHO, NORM_NONE = 0, 1
PATH_AUTO, PATH_FP32, PATH_SPLIT_TC, PATH_SPLIT_HILO, PATH_BF16 = 0, 1, 2, 3, 4
PATHS = {"auto": PATH_AUTO, "fp32": PATH_FP32, "split_tc": PATH_SPLIT_TC,
         "split_hilo": PATH_SPLIT_HILO, "bf16": PATH_BF16}
NORMS = {"ortho": NORM_ORTHO, "none": NORM_NONE}
KINDS = {"forward": FORWARD, "inverse": INVERSE, "roundtrip": ROUNDTRIP, "spectral": SPECTRAL}
STATUS = {0: "OK", 1: "ERR_INVALID_ARG", 2: "ERR_UNSUPPORTED_SHAPE", 3: "ERR_KIND",
          4: "ERR_ALIGN", 5: "ERR_ALIAS", 6: "ERR_CUDA", 7: "ERR_ARCH",
          8: "ERR_DEVICE_TIMEOUT", 9: "ERR_NO_MEMORY", 10: "ERR_PATH"}

# every symbol the header declares, in declaration order
EXPORTS = [
    "bdct_plan_create", "bdct_plan_set_spectral", "bdct_plan_set_range_protection", "bdct_plan_destroy", "bdct_forward", "bdct_inverse", "bdct_roundtrip",
    "bdct_execute", "bdct_execute_tiled", "bdct_plan_set_host_staging", "bdct_execute_host",
    "bdct_execute_tiled_host", "bdct_plan_get_info", "bdct_plan_set_chunk_bytes", "bdct_plan_device_status",
    "bdct_ragged_create", "bdct_ragged_execute", "bdct_ragged_destroy", "bdct_ragged_num_classes",
    "bdct_ragged_class_info", "bdct_execute_noalloc", "bdct_selftest_wait_timeout", "bdct_status_string",
    "bdct_last_cuda_error", "bdct_version",
]


class BdctError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        self.code = STATUS.get(status, str(status))
        detail = ""
        if status == 6 and _lib is not None:
            detail = f" (cuda error {_lib.bdct_last_cuda_error()})"
        msg = _lib.bdct_status_string(status).decode() if _lib is not None else self.code
        super().__init__(f"{where}: {self.code}: {msg}{detail}")


class PlanInfo(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int), ("cols", ctypes.c_int), ("kind", ctypes.c_uint),
                ("norm", ctypes.c_int), ("path", ctypes.c_int), ("variant", ctypes.c_int),
                ("workspace_bytes", ctypes.c_size_t), ("table_bytes", ctypes.c_size_t)]


class RaggedClass(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int), ("cols", ctypes.c_int), ("count", ctypes.c_size_t),
                ("path", ctypes.c_int), ("variant", ctypes.c_int), ("tuned_us_per_array", ctypes.c_double),
                ("chunk_bytes", ctypes.c_size_t)]


_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Load ``libbdct.so`` (built by ``build.build()``); raise if it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library missing: {LIB_PATH}; run "
                                   "paper_2609_28519_gb300.build.build() first")
            L = ctypes.CDLL(LIB_PATH)
            vp, sz, ci, cu = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint
            L.bdct_plan_create.argtypes = [ctypes.POINTER(vp), ci, ci, cu, ci, ci]
            L.bdct_plan_destroy.argtypes = [vp]
            L.bdct_plan_set_spectral.argtypes = [vp, vp]
            L.bdct_plan_set_range_protection.argtypes = [vp, ci]
            for name in ("bdct_forward", "bdct_inverse", "bdct_roundtrip"):
                getattr(L, name).argtypes = [vp, vp, vp, sz, vp]
            L.bdct_execute.argtypes = [vp, cu, vp, vp, sz, vp]
            L.bdct_execute_tiled.argtypes = [vp, cu, vp, vp, ci, ci, sz, sz, vp]
            L.bdct_plan_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
            L.bdct_plan_set_host_staging.argtypes = [vp, sz]
            L.bdct_execute_host.argtypes = [vp, vp, ci, vp, vp, sz, vp]
            L.bdct_execute_tiled_host.argtypes = [vp, vp, ci, vp, vp, ci, ci, vp]
            L.bdct_plan_device_status.argtypes = [vp, ci]
            L.bdct_plan_set_chunk_bytes.argtypes = [vp, sz]
            L.bdct_selftest_wait_timeout.argtypes = [cu]
            L.bdct_execute_noalloc.argtypes = [ci, ci, cu, ci, vp, vp, sz, vp]
            L.bdct_ragged_create.argtypes = [ctypes.POINTER(vp), sz, vp, vp, vp, vp, cu, ci, ci]
            L.bdct_ragged_execute.argtypes = [vp, cu, vp, vp, vp]
            L.bdct_ragged_destroy.argtypes = [vp]
            L.bdct_ragged_num_classes.argtypes = [vp]
            L.bdct_ragged_class_info.argtypes = [vp, ci, ctypes.POINTER(RaggedClass)]
            L.bdct_status_string.argtypes = [ci]
            L.bdct_status_string.restype = ctypes.c_char_p
            L.bdct_last_cuda_error.restype = ci
            L.bdct_version.restype = ci
            _lib = L
    return _lib


def _check(status: int, where: str) -> None:
    if status != 0:
        raise BdctError(status, where)


def _stream_of(t, stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A plan for rows x cols arrays (``bdct_plan_create``)."""

    def __init__(self, rows: int, cols: int, kind=FORWARD | INVERSE | ROUNDTRIP | SPECTRAL,
                 norm="ortho", path="auto"):
        L = lib()
        self.rows, self.cols = int(rows), int(cols)
        self.norm = NORMS[norm] if isinstance(norm, str) else int(norm)
        self.path_requested = PATHS[path] if isinstance(path, str) else int(path)
        self.kind = int(kind)
        h = ctypes.c_void_p()
        _check(L.bdct_plan_create(ctypes.byref(h), self.rows, self.cols, self.kind, self.norm,
                                  self.path_requested), "bdct_plan_create")
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("plan destroyed")
        return self._h

    def info(self) -> PlanInfo:
        inf = PlanInfo()
        _check(lib().bdct_plan_get_info(self.handle, ctypes.byref(inf)), "bdct_plan_get_info")
        return inf

    def set_chunk_bytes(self, nbytes: int) -> None:
        """Chunk of whole arrays per two-pass round of the separable routes
        (bdct_plan_set_chunk_bytes)."""
        _check(lib().bdct_plan_set_chunk_bytes(self.handle, int(nbytes)), "bdct_plan_set_chunk_bytes")

    def device_status(self, clear: bool = True) -> int:
        """Synchronize and return the plan's device status (0, or 8 after a
        bounded device wait expired); raises on host errors."""
        st = lib().bdct_plan_device_status(self.handle, 1 if clear else 0)
        if st not in (0, 8):
            _check(st, "bdct_plan_device_status")
        return st

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.bdct_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _batch(self, x) -> int:
        import torch
        if x.dtype != torch.float32 or not x.is_cuda:
            raise TypeError("expected a CUDA float32 tensor")
        if x.dim() < 2 or x.shape[-2] != self.rows or x.shape[-1] != self.cols:
            raise ValueError(f"trailing shape must be ({self.rows}, {self.cols}), got {tuple(x.shape)}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.numel() // (self.rows * self.cols)

    def execute(self, kind: int, x, out=None, stream=None):
        import torch
        kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        b = self._batch(x)
        if out is None:
            out = torch.empty_like(x)
        elif self._batch(out) != b:
            raise ValueError("out batch differs from input batch")
        _check(lib().bdct_execute(self.handle, kind, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), b, _stream_of(x, stream)),
               "bdct_execute")
        return out

    def forward(self, x, out=None, stream=None):
        return self.execute(FORWARD, x, out, stream)

    def inverse(self, x, out=None, stream=None):
        return self.execute(INVERSE, x, out, stream)

    def roundtrip(self, x, out=None, stream=None):
        return self.execute(ROUNDTRIP, x, out, stream)

    def set_spectral(self, lam) -> None:
        """The rows x cols diagonal of the spectral direction (numpy, any float
        dtype; passed as row-major float64 to bdct_plan_set_spectral)."""
        import numpy as np
        a = np.ascontiguousarray(lam, dtype=np.float64)
        if a.shape != (self.rows, self.cols):
            raise ValueError(f"diagonal must be ({self.rows}, {self.cols}), got {a.shape}")
        _check(lib().bdct_plan_set_spectral(self.handle, ctypes.c_void_p(a.ctypes.data)), "bdct_plan_set_spectral")

    def set_range_protection(self, on: bool = True) -> None:
        """Per-array power-of-two pre-scaling around every call
        (bdct_plan_set_range_protection)."""
        _check(lib().bdct_plan_set_range_protection(self.handle, 1 if on else 0), "bdct_plan_set_range_protection")

    def spectral(self, x, out=None, stream=None):
        return self.execute(SPECTRAL, x, out, stream)

    def set_host_staging(self, chunk_bytes: int = 8 << 20) -> None:
        _check(lib().bdct_plan_set_host_staging(self.handle, int(chunk_bytes)), "bdct_plan_set_host_staging")

    @staticmethod
    def _kinds(kinds):
        ks = [KINDS[k] if isinstance(k, str) else int(k) for k in kinds]
        return (ctypes.c_uint * len(ks))(*ks), len(ks)

    def execute_host(self, kinds, h_in, h_out, stream=None):
        """Host (CPU, ideally pinned) float32 tensors in and out; the directions
        in `kinds` are applied in order on the device (bdct_execute_host)."""
        import torch
        arr, n = self._kinds(kinds)
        b = h_in.numel() // (self.rows * self.cols)
        s = torch.cuda.current_stream() if stream is None else stream
        _check(lib().bdct_execute_host(self.handle, arr, n, ctypes.c_void_p(h_in.data_ptr()),
                                       ctypes.c_void_p(h_out.data_ptr()), b, ctypes.c_void_p(s.cuda_stream)),
               "bdct_execute_host")
        return h_out

    def execute_tiled_host(self, kinds, h_img, h_out, stream=None):
        """Host image in and out through the tiled view (bdct_execute_tiled_host)."""
        import torch
        arr, n = self._kinds(kinds)
        s = torch.cuda.current_stream() if stream is None else stream
        _check(lib().bdct_execute_tiled_host(self.handle, arr, n, ctypes.c_void_p(h_img.data_ptr()),
                                             ctypes.c_void_p(h_out.data_ptr()), h_img.shape[0], h_img.shape[1],
                                             ctypes.c_void_p(s.cuda_stream)),
               "bdct_execute_tiled_host")
        return h_out

    def execute_tiled(self, kind: int, img, out=None, stream=None):
        """Transform every rows x cols block of a 2D image (``bdct_execute_tiled``)."""
        import torch
        kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        if img.dtype != torch.float32 or not img.is_cuda or img.dim() != 2 or img.stride(1) != 1:
            raise ValueError("expected a 2D CUDA float32 image with unit column stride")
        if out is None:
            out = torch.empty_like(img)
        _check(lib().bdct_execute_tiled(self.handle, kind, ctypes.c_void_p(img.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), img.shape[0], img.shape[1],
                                        img.stride(0), out.stride(0), _stream_of(img, stream)),
               "bdct_execute_tiled")
        return out


class Ragged:
    """A ragged batch of mixed shapes (``bdct_ragged_create``).

    ``shapes`` is a list of (rows, cols); arrays are packed back to back in
    that order (element offsets rounded up to multiples of 4) unless explicit
    ``in_off`` / ``out_off`` lists are given.
    """

    def __init__(self, shapes, kind=FORWARD | INVERSE | ROUNDTRIP, norm="ortho", path="auto",
                 in_off=None, out_off=None):
        import numpy as np
        L = lib()
        self.shapes = [(int(r), int(c)) for r, c in shapes]
        n = len(self.shapes)
        rows = np.array([r for r, _ in self.shapes], dtype=np.int32)
        cols = np.array([c for _, c in self.shapes], dtype=np.int32)
        if in_off is None:
            sizes = rows.astype(np.int64) * cols
            padded = (sizes + 3) // 4 * 4
            in_off = np.concatenate([[0], np.cumsum(padded)[:-1]]).astype(np.uint64)
            self.total = int(np.sum(padded))
        else:
            in_off = np.asarray(in_off, dtype=np.uint64)
            self.total = int(max(int(o) + r * c for o, (r, c) in zip(in_off, self.shapes))) if n else 0
        out_off = in_off.copy() if out_off is None else np.asarray(out_off, dtype=np.uint64)
        self.in_off, self.out_off = in_off, out_off
        norm = NORMS[norm] if isinstance(norm, str) else int(norm)
        path = PATHS[path] if isinstance(path, str) else int(path)
        h = ctypes.c_void_p()
        _check(L.bdct_ragged_create(ctypes.byref(h), n, rows.ctypes.data, cols.ctypes.data,
                                    in_off.ctypes.data, out_off.ctypes.data, int(kind), norm, path),
               "bdct_ragged_create")
        self._h = h

    def classes(self):
        L = lib()
        out = []
        for i in range(L.bdct_ragged_num_classes(self._h)):
            c = RaggedClass()
            _check(L.bdct_ragged_class_info(self._h, i, ctypes.byref(c)), "bdct_ragged_class_info")
            out.append({"rows": c.rows, "cols": c.cols, "count": c.count, "path": c.path,
                        "variant": c.variant, "tuned_us_per_array": c.tuned_us_per_array,
                        "chunk_bytes": c.chunk_bytes})
        return out

    def execute(self, kind, x, out, stream=None):
        """x, out: flat CUDA float32 tensors holding the packed arrays."""
        kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        _check(lib().bdct_ragged_execute(self._h, kind, ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), _stream_of(x, stream)),
               "bdct_ragged_execute")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.bdct_ragged_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
