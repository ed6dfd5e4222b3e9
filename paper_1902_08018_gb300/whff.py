"""ctypes binding of include/whff.h (argument marshalling only).

Vectors use the row-per-right-hand-side convention of PyTorch: x is a CUDA
float32 tensor of shape (N,) or (R, N) whose rows are the R right-hand sides
(column-major N x R with ldx = x.stride(0) in the C ABI); y is float64 (M,)
or (R, M); the state is float64 (M,).
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

from . import build as _build

FMT_ZFP = 1
FMT_BF16 = 2
FMT_FP16 = 3
FMT_FP8E4M3 = 4
FMT_FIXED_LIFT = 5
FMT_FIXED_BFP = 6
FMT_FP32 = 7
FMT_FIXED_ACC = 8

_ERRORS = {
    -1: "WHFF_EINVAL",
    -2: "WHFF_ERANGE",
    -3: "WHFF_ENONFINITE",
    -4: "WHFF_ENOMEM",
    -5: "WHFF_EFORMAT",
    -6: "WHFF_ECUDA",
    -7: "WHFF_ETIMEOUT",
    -8: "WHFF_EBUSY",
}


class WhffError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library() -> ctypes.CDLL:
    """Load libwhff.so, building it first if it is missing or stale."""
    global _lib
    if _lib is not None:
        return _lib
    so = Path(_build.OUT)
    if not _build.up_to_date():
        _build.build()
    L = ctypes.CDLL(str(so))
    P, i64, c_int, sz, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
    sigs = {
        "whff_compressed_size": (sz, [c_int, c_int, i64, i64]),
        "whff_compress": (c_int, [P, i64, i64, i64, c_int, c_int, P, sz, ctypes.POINTER(sz), c_int]),
        "whff_accuracy_max_size": (sz, [i64, i64]),
        "whff_compress_accuracy": (c_int, [P, i64, i64, i64, dbl, P, sz, ctypes.POINTER(sz), c_int]),
        "whff_accuracy_begin": (c_int, [P, sz, i64, i64, dbl]),
        "whff_compress_accuracy_band": (c_int, [P, sz, P, i64, i64, i64, c_int]),
        "whff_accuracy_seal": (c_int, [P, sz, ctypes.POINTER(sz)]),
        "whff_blob_init": (c_int, [P, sz, c_int, c_int, i64, i64]),
        "whff_compress_band": (c_int, [P, sz, P, i64, i64, i64, c_int]),
        "whff_blob_seal": (c_int, [P, sz]),
        "whff_create": (c_int, [P, sz, c_int, P, ctypes.POINTER(P)]),
        "whff_create_ex": (c_int, [P, sz, c_int, ctypes.c_uint, P, ctypes.POINTER(P)]),
        "whff_info": (c_int, [P, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(i64),
                              ctypes.POINTER(i64), ctypes.POINTER(sz)]),
        "whff_plan": (c_int, [P, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
        "whff_step": (c_int, [P, P, c_int, i64, P, i64, P, dbl, P]),
        "whff_step_host": (c_int, [P, P, c_int, i64, P, i64, P, dbl, P]),
        "whff_decompress": (c_int, [P, P, i64, P]),
        "whff_sync_status": (c_int, [P, P]),
        "whff_set_wait_limit": (c_int, [P, i64]),
        "whff_destroy": (None, [P]),
        "whff_step_noalloc": (c_int, [P, c_int, i64, i64, P, c_int, i64, P, i64, P, dbl, P]),
        "whff_graph_create": (c_int, [P, P, c_int, i64, P, i64, P, dbl, P, ctypes.POINTER(P)]),
        "whff_graph_create_host": (c_int, [P, P, c_int, i64, P, i64, P, dbl, P, ctypes.POINTER(P)]),
        "whff_graph_launch": (c_int, [P, P]),
        "whff_graph_create_rows": (c_int, [P, i64, i64, P, c_int, i64, P, i64, P, dbl, P, ctypes.POINTER(P)]),
        "whff_graph_set_rows": (c_int, [P, P, i64]),
        "whff_fields_create": (c_int, [c_int, c_int, i64, i64, c_int, c_int, ctypes.c_uint, P, ctypes.POINTER(P)]),
        "whff_fields_load": (c_int, [P, c_int, P, sz, P]),
        "whff_fields_acquire": (c_int, [P, c_int, P, ctypes.POINTER(P)]),
        "whff_fields_release": (c_int, [P, c_int, P]),
        "whff_fields_destroy": (None, [P]),
        "whff_graph_destroy": (None, [P]),
        "whff_server_create": (c_int, [sz, c_int, c_int, ctypes.POINTER(P)]),
        "whff_server_add_model": (c_int, [P, P, dbl, ctypes.POINTER(c_int)]),
        "whff_server_add_model_ex": (c_int, [P, P, dbl, ctypes.c_uint, ctypes.POINTER(c_int)]),
        "whff_server_model_state": (c_int, [P, c_int, ctypes.POINTER(c_int)]),
        "whff_server_remove_model": (c_int, [P, c_int]),
        "whff_server_reset_state": (c_int, [P, c_int]),
        "whff_server_read_state": (c_int, [P, c_int, P]),
        "whff_server_run": (c_int, [P, c_int, P, P, P, P, P, P, P, dbl, dbl]),
        "whff_server_destroy": (None, [P]),
        "whff_tune": (c_int, [P, c_int, P, ctypes.POINTER(dbl)]),
        "whff_get_config": (c_int, [P, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
        "whff_set_config": (c_int, [P, c_int, c_int, c_int]),
        "whff_get_crossover": (c_int, [P, ctypes.POINTER(c_int)]),
        "whff_step_rows": (c_int, [P, i64, i64, P, c_int, i64, P, i64, P, dbl, P]),
        "whff_set_crossover": (c_int, [P, c_int]),
        "whff_get_slice_rows": (c_int, [P, ctypes.POINTER(i64)]),
        "whff_set_slice_rows": (c_int, [P, i64]),
        "whff_read_probe": (c_int, [P, ctypes.c_size_t, P, P]),
        "whff_batch_create": (c_int, [P, P, c_int, ctypes.POINTER(P)]),
        "whff_batch_step": (c_int, [P, P, P, P, P, P, dbl, P]),
        "whff_batch_destroy": (None, [P]),
        "whff_last_error": (ctypes.c_char_p, []),
        "whff_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(code: int):
    if code != 0:
        raise WhffError(code, library().whff_last_error().decode(errors="replace"))


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def compressed_size(fmt: int, rate: int, M: int, N: int) -> int:
    return int(library().whff_compressed_size(fmt, rate, M, N))


def whff_compress(A: np.ndarray, fmt: int = FMT_ZFP, rate: int = 16, nthreads: int = 0) -> np.ndarray:
    """Offline encode of an FP64 row-major matrix -> blob (uint8 array)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    M, N = A.shape
    n = compressed_size(fmt, rate, M, N)
    if n == 0:
        raise WhffError(-1, "invalid format, rate or shape")
    out = np.empty(n, dtype=np.uint8)
    used = ctypes.c_size_t()
    _check(library().whff_compress(A.ctypes.data, M, N, N, fmt, rate, out.ctypes.data, n, ctypes.byref(used),
                                   nthreads))
    return out


def whff_compress_accuracy(A: np.ndarray, tol: float, nthreads: int = 0) -> np.ndarray:
    """Fixed-accuracy encode (WZ3) of an FP64 row-major matrix at absolute tolerance tol -> blob."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    M, N = A.shape
    cap = int(library().whff_accuracy_max_size(M, N))
    if cap == 0:
        raise WhffError(-1, "empty shape")
    out = np.empty(cap, dtype=np.uint8)
    used = ctypes.c_size_t()
    _check(library().whff_compress_accuracy(A.ctypes.data, M, N, N, float(tol), out.ctypes.data, cap,
                                            ctypes.byref(used), nthreads))
    return out[: used.value].copy()


def whff_compress_accuracy_bands(M: int, N: int, bands, tol: float, nthreads: int = 0) -> np.ndarray:
    """Fixed-accuracy encode of a matrix given as an iterable of (row0, FP64 band), bands in row order."""
    L = library()
    cap = int(L.whff_accuracy_max_size(M, N))
    if cap == 0:
        raise WhffError(-1, "empty shape")
    out = np.empty(cap, dtype=np.uint8)
    _check(L.whff_accuracy_begin(out.ctypes.data, cap, M, N, float(tol)))
    for row0, band in bands:
        band = np.ascontiguousarray(band, dtype=np.float64)
        _check(L.whff_compress_accuracy_band(out.ctypes.data, cap, band.ctypes.data, row0, band.shape[0],
                                             band.shape[1], nthreads))
    used = ctypes.c_size_t()
    _check(L.whff_accuracy_seal(out.ctypes.data, cap, ctypes.byref(used)))
    return out[: used.value].copy()


def whff_compress_bands(M: int, N: int, bands, fmt: int = FMT_ZFP, rate: int = 16, nthreads: int = 0) -> np.ndarray:
    """Encode a matrix given as an iterable of (row0, FP64 band) without holding all of it."""
    L = library()
    n = compressed_size(fmt, rate, M, N)
    if n == 0:
        raise WhffError(-1, "invalid format, rate or shape")
    out = np.empty(n, dtype=np.uint8)
    _check(L.whff_blob_init(out.ctypes.data, n, fmt, rate, M, N))
    for row0, band in bands:
        band = np.ascontiguousarray(band, dtype=np.float64)
        _check(L.whff_compress_band(out.ctypes.data, n, band.ctypes.data, row0, band.shape[0], band.shape[1],
                                    nthreads))
    _check(L.whff_blob_seal(out.ctypes.data, n))
    return out


def _vec_args(t, rows: int, name: str, dtype):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype:
        raise WhffError(-1, f"{name} must be a CUDA {dtype} tensor")
    if t.dim() == 1:
        if t.shape[0] < rows or t.stride(0) != 1:
            raise WhffError(-1, f"{name}: need {rows} contiguous entries")
        return t.data_ptr(), 1, rows
    if t.dim() != 2 or t.stride(1) != 1 or t.shape[1] < rows:
        raise WhffError(-1, f"{name}: shape (R, {rows}) with contiguous rows expected")
    # one row: its stride is arbitrary (numpy's x[None, :] has stride 0); any ld >= rows works
    return t.data_ptr(), t.shape[0], t.stride(0) if t.shape[0] > 1 else max(t.stride(0), rows)


class Handle:
    """A matrix resident on the GPU (owner of the device copy and workspace)."""

    def __init__(self, ptr: int):
        self._ptr = ctypes.c_void_p(ptr)
        f, r, m, n, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        _check(library().whff_info(self._ptr, ctypes.byref(f), ctypes.byref(r), ctypes.byref(m), ctypes.byref(n),
                                   ctypes.byref(b)))
        self.fmt, self.rate, self.M, self.N, self.device_bytes = f.value, r.value, m.value, n.value, b.value

    @property
    def ptr(self):
        return self._ptr

    def tune(self, iters: int = 20, stream=None, cache: str | None = None) -> dict:
        """Pick the fastest launch shape (WZ2); with `cache` (a JSON path) reuse / store the
        result keyed by format, rate, shape and SM count."""
        import json
        import os

        import torch

        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        key = f"fmt{self.fmt}-rate{self.rate}-{self.M}x{self.N}-sm{sms}"
        db = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                db = json.load(f)
        if key in db:
            self.set_config(db[key]["unroll"], db[key]["ctas_per_sm"], db[key].get("fold", 0))
            if "crossover" in db[key] and (self.crossover < 33 or db[key]["crossover"] == 33):
                self.crossover = db[key]["crossover"]
            return dict(db[key], cached=True)
        ms = ctypes.c_double()
        _check(library().whff_tune(self._ptr, iters, _stream_ptr(stream), ctypes.byref(ms)))
        u, c, f = self.config()
        rec = {"unroll": u, "ctas_per_sm": c, "fold": f, "crossover": self.crossover, "ms": ms.value}
        if cache:
            db[key] = rec
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            with open(cache, "w") as f:
                json.dump(db, f, indent=1)
        return dict(rec, cached=False)

    def config(self):
        """(unroll, ctas_per_sm, fold flags: 1 FP32-pair fold, 2 lane groups) of the WZ2 launch shape."""
        u, c, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(library().whff_get_config(self._ptr, ctypes.byref(u), ctypes.byref(c), ctypes.byref(r)))
        return u.value, c.value, r.value

    def set_config(self, unroll: int, ctas_per_sm: int, fold: int | None = None):
        if fold is None:
            fold = self.config()[2]
        _check(library().whff_set_config(self._ptr, unroll, ctas_per_sm, int(fold)))

    @property
    def crossover(self) -> int:
        """Fewest right-hand sides of a tensor-core pass (33: CUDA cores only)."""
        v = ctypes.c_int()
        _check(library().whff_get_crossover(self._ptr, ctypes.byref(v)))
        return v.value

    @crossover.setter
    def crossover(self, min_rhs: int):
        _check(library().whff_set_crossover(self._ptr, int(min_rhs)))

    @property
    def slice_rows(self) -> int:
        """Rows per slit when whff_step runs a pass as time slices (0: whole matrix)."""
        v = ctypes.c_int64()
        _check(library().whff_get_slice_rows(self._ptr, ctypes.byref(v)))
        return v.value

    @slice_rows.setter
    def slice_rows(self, rows: int):
        _check(library().whff_set_slice_rows(self._ptr, int(rows)))

    def plan(self):
        """(ksplit, kernel launches per pass of up to 8 right-hand sides)."""
        k, n = ctypes.c_int(), ctypes.c_int()
        _check(library().whff_plan(self._ptr, ctypes.byref(k), ctypes.byref(n)))
        return k.value, n.value

    def step(self, x, y, state=None, decay: float = 0.99, stream=None):
        whff_step(self, x, y, state, decay, stream)

    def step_rows(self, row0: int, nrows: int, x, y, state=None, decay: float = 0.99, stream=None):
        whff_step_rows(self, row0, nrows, x, y, state, decay, stream)

    def step_host(self, x_host: np.ndarray, y_host: np.ndarray, state=None, decay: float = 0.99, stream=None):
        whff_step_host(self, x_host, y_host, state, decay, stream)

    def decompress(self, out, stream=None):
        whff_decompress(self, out, stream)

    def sync_status(self, stream=None) -> int:
        return int(library().whff_sync_status(self._ptr, _stream_ptr(stream)))

    def set_wait_limit(self, polls: int):
        """Polls of the tensor-core kernels' in-loop waits (< 0: the default); for failure-detection tests."""
        _check(library().whff_set_wait_limit(self._ptr, int(polls)))

    def destroy(self):
        if self._ptr:
            library().whff_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def whff_create(blob, max_rhs: int = 32, stream=None, host_resident: bool = False) -> Handle:
    """Make a blob resident; host_resident keeps the stream in pinned host memory read over the CPU link."""
    b = np.ascontiguousarray(np.frombuffer(blob, dtype=np.uint8) if isinstance(blob, (bytes, bytearray)) else blob,
                             dtype=np.uint8)
    h = ctypes.c_void_p()
    _check(library().whff_create_ex(b.ctypes.data, b.size, max_rhs, 1 if host_resident else 0, _stream_ptr(stream),
                                    ctypes.byref(h)))
    return Handle(h.value)


def whff_step(h: Handle, x, y, state=None, decay: float = 0.99, stream=None):
    import torch

    xp, R, ldx = _vec_args(x, h.N, "x", torch.float32)
    yp, Ry, ldy = _vec_args(y, h.M, "y", torch.float64)
    if Ry != R:
        raise WhffError(-1, "x and y disagree on the number of right-hand sides")
    sp = 0
    if state is not None:
        sp, Rs, _ = _vec_args(state, h.M, "state", torch.float64)
        if Rs != 1:
            raise WhffError(-1, "state must be a vector")
    _check(library().whff_step(h.ptr, xp, R, ldx, yp, ldy, sp or None, float(decay), _stream_ptr(stream)))


def whff_step_rows(h: Handle, row0: int, nrows: int, x, y, state=None, decay: float = 0.99, stream=None):
    """A slit step: y (nrows,) or (R, nrows) = rows row0 .. row0+nrows-1 of the matrix times x."""
    import torch

    xp, R, ldx = _vec_args(x, h.N, "x", torch.float32)
    yp, Ry, ldy = _vec_args(y, nrows, "y", torch.float64)
    if Ry != R:
        raise WhffError(-1, "x and y disagree on the number of right-hand sides")
    sp = 0
    if state is not None:
        sp, Rs, _ = _vec_args(state, nrows, "state", torch.float64)
        if Rs != 1:
            raise WhffError(-1, "state must be a vector")
    _check(library().whff_step_rows(h.ptr, int(row0), int(nrows), xp, R, ldx, yp, ldy, sp or None, float(decay),
                                    _stream_ptr(stream)))


def whff_step_host(h: Handle, x_host: np.ndarray, y_host: np.ndarray, state=None, decay: float = 0.99, stream=None):
    """x_host: float32 (N,) or (R, N); y_host: float64 (M,) or (R, M); both host (ideally pinned) arrays."""
    import torch

    xh = x_host if x_host.ndim == 2 else x_host.reshape(1, -1)
    yh = y_host if y_host.ndim == 2 else y_host.reshape(1, -1)
    if xh.dtype != np.float32 or yh.dtype != np.float64 or xh.strides[1] != 4 or yh.strides[1] != 8:
        raise WhffError(-1, "x_host float32 and y_host float64 with contiguous rows expected")
    if xh.shape[1] < h.N or yh.shape[1] < h.M or yh.shape[0] < xh.shape[0]:
        raise WhffError(-1, f"x_host needs (R, {h.N}) and y_host (R, {h.M}) with the same R or more rows of y")
    sp = 0
    if state is not None:
        sp, _, _ = _vec_args(state, h.M, "state", torch.float64)
    _check(library().whff_step_host(h.ptr, xh.ctypes.data, xh.shape[0], xh.strides[0] // 4, yh.ctypes.data,
                                    yh.strides[0] // 8, sp or None, float(decay), _stream_ptr(stream)))


def whff_read_probe(buf, out, stream=None):
    """XOR of every 32-bit word of a 16-byte-aligned CUDA tensor into out (int32, 1 element, on the GPU):
    one read of the buffer at full bandwidth, the achievable-read roofline."""
    import torch

    if not isinstance(buf, torch.Tensor) or not buf.is_cuda or not buf.is_contiguous():
        raise WhffError(-1, "buf must be a contiguous CUDA tensor")
    if not isinstance(out, torch.Tensor) or not out.is_cuda or out.dtype != torch.int32 or out.numel() < 1:
        raise WhffError(-1, "out must be a CUDA int32 tensor")
    _check(library().whff_read_probe(buf.data_ptr(), buf.numel() * buf.element_size(), out.data_ptr(),
                                     _stream_ptr(stream)))


def whff_decompress(h: Handle, out, stream=None):
    import torch

    if not isinstance(out, torch.Tensor) or not out.is_cuda or out.dtype != torch.float64 or out.dim() != 2:
        raise WhffError(-1, "out must be a 2-D CUDA float64 tensor")
    if out.shape[0] < h.M or out.shape[1] < h.N or out.stride(1) != 1:
        raise WhffError(-1, "out too small or not row-contiguous")
    _check(library().whff_decompress(h.ptr, out.data_ptr(), out.stride(0), _stream_ptr(stream)))


def whff_destroy(h: Handle):
    h.destroy()


def whff_step_noalloc(stream_dev, rate: int, M: int, N: int, x, y, state=None, decay: float = 0.99, stream=None):
    """The allocation-free step: stream_dev is a CUDA uint8 tensor holding the WZ1 stream
    (the blob without its 64-byte header) in caller-owned memory."""
    import torch

    if not isinstance(stream_dev, torch.Tensor) or not stream_dev.is_cuda or stream_dev.dtype != torch.uint8:
        raise WhffError(-1, "stream_dev must be a CUDA uint8 tensor")
    # the C entry point takes no length: a short buffer would be read past its end on the device
    need = -(-int(M) // 4) * -(-int(N) // 4) * 2 * int(rate)
    if M <= 0 or N <= 0 or not stream_dev.is_contiguous() or stream_dev.numel() < need:
        raise WhffError(-1, f"stream_dev holds {stream_dev.numel()} bytes; M={M}, N={N}, rate={rate} need {need}")
    xp, R, ldx = _vec_args(x, N, "x", torch.float32)
    yp, Ry, ldy = _vec_args(y, M, "y", torch.float64)
    if Ry != R:
        raise WhffError(-1, "x and y disagree on the number of right-hand sides")
    sp = 0
    if state is not None:
        sp, _, _ = _vec_args(state, M, "state", torch.float64)
    _check(library().whff_step_noalloc(stream_dev.data_ptr(), rate, M, N, xp, R, ldx, yp, ldy, sp or None,
                                       float(decay), _stream_ptr(stream)))


class Graph:
    """A captured control step (whff_graph_create / whff_graph_create_host / whff_graph_create_rows)."""

    def __init__(self, ptr: int, keep=()):
        self._ptr = ctypes.c_void_p(ptr)
        self._keep = keep  # buffers the graph reads or writes

    def launch(self, stream=None):
        _check(library().whff_graph_launch(self._ptr, _stream_ptr(stream)))

    def set_rows(self, row0: int, h: "Handle | None" = None):
        """Move a slit graph to rows row0.. (and onto handle h, if given)."""
        _check(library().whff_graph_set_rows(self._ptr, h.ptr if h is not None else None, int(row0)))
        if h is not None:
            self._keep = tuple(self._keep) + (h,)

    def destroy(self):
        if self._ptr:
            library().whff_graph_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def whff_graph_create(h: Handle, x, y, state=None, decay: float = 0.99, stream=None) -> Graph:
    import torch

    xp, R, ldx = _vec_args(x, h.N, "x", torch.float32)
    yp, Ry, ldy = _vec_args(y, h.M, "y", torch.float64)
    if Ry != R:
        raise WhffError(-1, "x and y disagree on the number of right-hand sides")
    sp = _vec_args(state, h.M, "state", torch.float64)[0] if state is not None else 0
    g = ctypes.c_void_p()
    _check(library().whff_graph_create(h.ptr, xp, R, ldx, yp, ldy, sp or None, float(decay), _stream_ptr(stream),
                                       ctypes.byref(g)))
    return Graph(g.value, (x, y, state))


def whff_graph_create_rows(h: Handle, row0: int, nrows: int, x, y, state=None, decay: float = 0.99,
                           stream=None) -> Graph:
    """A slit graph: y (M,) or (R, M) and state (M,) are field-sized; a replay writes rows row0..row0+nrows-1."""
    import torch

    xp, R, ldx = _vec_args(x, h.N, "x", torch.float32)
    yp, Ry, ldy = _vec_args(y, h.M, "y", torch.float64)
    if Ry != R:
        raise WhffError(-1, "x and y disagree on the number of right-hand sides")
    sp = _vec_args(state, h.M, "state", torch.float64)[0] if state is not None else 0
    g = ctypes.c_void_p()
    _check(library().whff_graph_create_rows(h.ptr, int(row0), int(nrows), xp, R, ldx, yp, ldy, sp or None,
                                            float(decay), _stream_ptr(stream), ctypes.byref(g)))
    return Graph(g.value, (h, x, y, state))


def whff_graph_create_host(h: Handle, x_host: np.ndarray, y_host: np.ndarray, state=None, decay: float = 0.99,
                           stream=None) -> Graph:
    """x_host float32 (R, N) and y_host float64 (R, M): pinned host arrays the graph copies from / to."""
    import torch

    xh = x_host if x_host.ndim == 2 else x_host.reshape(1, -1)
    yh = y_host if y_host.ndim == 2 else y_host.reshape(1, -1)
    if xh.dtype != np.float32 or yh.dtype != np.float64 or xh.strides[1] != 4 or yh.strides[1] != 8:
        raise WhffError(-1, "x_host float32 and y_host float64 with contiguous rows expected")
    if xh.shape[1] < h.N or yh.shape[1] < h.M or yh.shape[0] < xh.shape[0]:
        raise WhffError(-1, f"x_host needs (R, {h.N}) and y_host (R, {h.M}) with the same R or more rows of y")
    sp = _vec_args(state, h.M, "state", torch.float64)[0] if state is not None else 0
    g = ctypes.c_void_p()
    _check(library().whff_graph_create_host(h.ptr, xh.ctypes.data, xh.shape[0], xh.strides[0] // 4, yh.ctypes.data,
                                            yh.strides[0] // 8, sp or None, float(decay), _stream_ptr(stream),
                                            ctypes.byref(g)))
    return Graph(g.value, (x_host, y_host, state))


class Server:
    """Request server over resident models (continuous batching, graph replay)."""

    def __init__(self, hbm_budget: int, max_batch: int = 8, nstreams: int = 4):
        p = ctypes.c_void_p()
        _check(library().whff_server_create(int(hbm_budget), max_batch, nstreams, ctypes.byref(p)))
        self._ptr = p
        self.models = []

    def add_model(self, h: Handle, decay: float = 0.99, wait: bool = False) -> int:
        """Admit a model; with wait=True one that does not fit waits for removals to free memory."""
        mid = ctypes.c_int()
        _check(library().whff_server_add_model_ex(self._ptr, h.ptr, float(decay), 1 if wait else 0,
                                                  ctypes.byref(mid)))
        self.models.append(h)
        return mid.value

    def model_state(self, model_id: int) -> str:
        v = ctypes.c_int()
        _check(library().whff_server_model_state(self._ptr, int(model_id), ctypes.byref(v)))
        return {0: "removed", 1: "admitted", 2: "waiting"}[v.value]

    def remove_model(self, model_id: int):
        _check(library().whff_server_remove_model(self._ptr, int(model_id)))

    def reset_state(self, model_id: int):
        _check(library().whff_server_reset_state(self._ptr, model_id))

    def read_state(self, model_id: int) -> np.ndarray:
        out = np.empty(self.models[model_id].M, dtype=np.float64)
        _check(library().whff_server_read_state(self._ptr, model_id, out.ctypes.data))
        return out

    def run(self, model, arrival_s, xs, want_y: bool = False, max_wait_s: float = 600.0,
            drop_after_s: float = 0.0, return_status: bool = False):
        """model: int array, arrival_s: float array (non-decreasing), xs: list of float32 host
        vectors.  Returns (latency_s, batch, ys or None[, status])."""
        n = len(model)
        model = np.ascontiguousarray(model, dtype=np.int32)
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        xs = [np.ascontiguousarray(v, dtype=np.float32).reshape(-1) for v in xs]
        if arr.shape != (n,) or len(xs) != n:
            raise WhffError(-1, "model, arrival_s and xs need one entry per request")
        for i in range(n):  # the server copies N floats from each x
            m = int(model[i])
            if not 0 <= m < len(self.models):
                raise WhffError(-1, f"request {i}: unknown model {m}")
            if xs[i].size < self.models[m].N:
                raise WhffError(-1, f"request {i}: x has {xs[i].size} entries, model {m} needs {self.models[m].N}")
        xptr = (ctypes.c_void_p * n)(*[v.ctypes.data for v in xs])
        ys = None
        yptr = None
        if want_y:
            ys = [np.empty(self.models[m].M, dtype=np.float64) for m in model]
            yptr = (ctypes.c_void_p * n)(*[v.ctypes.data for v in ys])
        lat = np.empty(n, dtype=np.float64)
        bat = np.empty(n, dtype=np.int32)
        st = np.empty(n, dtype=np.int32)
        _check(library().whff_server_run(self._ptr, n, model.ctypes.data, arr.ctypes.data, xptr, yptr,
                                         lat.ctypes.data, bat.ctypes.data, st.ctypes.data, float(drop_after_s),
                                         float(max_wait_s)))
        return (lat, bat, ys, st) if return_status else (lat, bat, ys)

    def destroy(self):
        if self._ptr:
            library().whff_server_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.destroy()


class Batch:
    """Many resident matrices (WZ2 of one format and rate, or one scaled format) stepped together
    (whff_batch_create / whff_batch_step); R[i] at most handle i's max_rhs."""

    def __init__(self, handles, R):
        self.handles = list(handles)
        self.R = [int(r) for r in R]
        arr = (ctypes.c_void_p * len(self.handles))(*[h.ptr.value for h in self.handles])
        rs = (ctypes.c_int * len(self.R))(*self.R)
        p = ctypes.c_void_p()
        _check(library().whff_batch_create(arr, rs, len(self.handles), ctypes.byref(p)))
        self._ptr = p

    def step(self, xs, ys, states=None, decay: float = 0.99, stream=None):
        """xs[i]: CUDA float32 (R_i, N_i); ys[i]: float64 (R_i, M_i); states[i]: float64 (M_i,) or None."""
        import torch

        n = len(self.handles)
        if len(xs) != n or len(ys) != n or (states is not None and len(states) != n):
            raise WhffError(-1, f"one x, y (and state) per matrix: {n} expected")
        xp, lx, yp, ly = [], [], [], []
        for i, h in enumerate(self.handles):
            p, R, ld = _vec_args(xs[i], h.N, "x", torch.float32)
            q, Ry, ldy = _vec_args(ys[i], h.M, "y", torch.float64)
            if R != self.R[i] or Ry != self.R[i]:
                raise WhffError(-1, f"matrix {i}: expected {self.R[i]} right-hand sides")
            xp.append(p), lx.append(ld), yp.append(q), ly.append(ldy)
        sp = None
        if states is not None:  # each a CUDA float64 vector of M_i entries, or None
            ptrs = []
            for i, (h, st) in enumerate(zip(self.handles, states)):
                if st is None:
                    ptrs.append(None)
                    continue
                p, Rs, _ = _vec_args(st, h.M, f"state {i}", torch.float64)
                if Rs != 1:
                    raise WhffError(-1, f"state {i} must be a vector")
                ptrs.append(p)
            sp = (ctypes.c_void_p * n)(*ptrs)
        _check(library().whff_batch_step(self._ptr, (ctypes.c_void_p * n)(*xp), (ctypes.c_int64 * n)(*lx),
                                         (ctypes.c_void_p * n)(*yp), (ctypes.c_int64 * n)(*ly), sp, float(decay),
                                         _stream_ptr(stream)))

    def destroy(self):
        if self._ptr:
            library().whff_batch_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.destroy()


class _SlotHandle(Handle):
    """A field pipeline's slot: owned by the pipeline, never destroyed here."""

    def destroy(self):
        self._ptr = ctypes.c_void_p()


class Fields:
    """Compressed fields streamed into nbuf resident slots (whff_fields_*)."""

    def __init__(self, fmt: int, rate: int, M: int, N: int, nbuf: int = 2, max_rhs: int = 1,
                 verify_crc: bool = False, stream=None):
        p = ctypes.c_void_p()
        _check(library().whff_fields_create(int(fmt), int(rate), int(M), int(N), int(nbuf), int(max_rhs),
                                            1 if verify_crc else 0, _stream_ptr(stream), ctypes.byref(p)))
        self._ptr = p
        self.nbuf = nbuf
        self._blobs = [None] * nbuf  # the host blob of each slot's last load (kept alive for the copy)
        self._handles = [None] * nbuf

    def load(self, slot: int, blob: np.ndarray, copy_stream=None):
        b = blob if isinstance(blob, np.ndarray) else np.frombuffer(blob, dtype=np.uint8)
        _check(library().whff_fields_load(self._ptr, int(slot), b.ctypes.data, b.size, _stream_ptr(copy_stream)))
        self._blobs[slot] = b

    def acquire(self, slot: int, stream=None) -> Handle:
        hp = ctypes.c_void_p()
        _check(library().whff_fields_acquire(self._ptr, int(slot), _stream_ptr(stream), ctypes.byref(hp)))
        if self._handles[slot] is None or self._handles[slot].ptr.value != hp.value:
            self._handles[slot] = _SlotHandle(hp.value)
        return self._handles[slot]

    def release(self, slot: int, stream=None):
        _check(library().whff_fields_release(self._ptr, int(slot), _stream_ptr(stream)))

    def destroy(self):
        if self._ptr:
            library().whff_fields_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.destroy()
