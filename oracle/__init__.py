"""CPU oracle for the compressed control-step GEMV -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The library (the CUDA path and
its host encoder) never imports, links or executes anything here, and this
package imports nothing from the library.

The arithmetic lives in plain C (``orc.c``; see ``orc.h`` for what each
function follows in the paper).  This module is argument marshalling over
ctypes plus numpy conveniences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_BUILD = _HERE / "_build"
_SO = _BUILD / "liborc.so"

FMT_ZFP = 1
FMT_BF16 = 2
FMT_FP16 = 3
FMT_FP8E4M3 = 4
FMT_FIXED_LIFT = 5
FMT_FIXED_BFP = 6
FMT_FP32 = 7
FMT_FIXED_ACC = 8
HEADER_BYTES = 64


def build(force: bool = False) -> Path:
    """Compile orc.c into oracle/_build/liborc.so with gcc (OpenMP, no FP contraction)."""
    src = _HERE / "orc.c"
    if _SO.exists() and not force and _SO.stat().st_mtime >= max(src.stat().st_mtime, (_HERE / "orc.h").stat().st_mtime):
        return _SO
    _BUILD.mkdir(exist_ok=True)
    tmp = _SO.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", str(tmp), str(src), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_SO))
        c_i64, c_int, c_sz = ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
        P = ctypes.c_void_p
        sig = {
            "orc_crc32": (ctypes.c_uint32, [P, c_sz]),
            "orc_fwd_lift4": (None, [P]),
            "orc_inv_lift4": (None, [P]),
            "orc_fwd_xform": (None, [P]),
            "orc_inv_xform": (None, [P]),
            "orc_int2nb": (ctypes.c_uint32, [ctypes.c_int32]),
            "orc_nb2int": (ctypes.c_int32, [ctypes.c_uint32]),
            "orc_sequency": (None, [P]),
            "orc_encode_planes": (c_int, [P, c_int, P, c_i64]),
            "orc_decode_planes": (c_int, [P, c_i64, c_int, P]),
            "orc_wz1_encode_block": (c_int, [P, c_int, P]),
            "orc_wz1_decode_block": (None, [P, c_int, P, P, P]),
            "orc_wz1_value": (ctypes.c_double, [ctypes.c_int32, c_int, c_int]),
            "orc_rate_ok": (c_int, [c_int]),
            "orc_blob_size": (c_sz, [c_int, c_int, c_i64, c_i64]),
            "orc_encode": (c_int, [c_int, c_int, P, c_i64, c_i64, c_i64, P, c_sz]),
            "orc_parse": (c_int, [P, c_sz, P, P, P, P]),
            "orc_decode_rows": (c_int, [P, c_sz, c_i64, c_i64, P, c_i64]),
            "orc_round_fmt": (ctypes.c_double, [c_int, ctypes.c_double, P]),
            "orc_fmt_max": (ctypes.c_double, [c_int]),
            "orc_fmt_decode": (ctypes.c_double, [c_int, ctypes.c_uint32]),
            "orc_gemv64": (None, [P, c_i64, c_i64, c_i64, P, c_int, c_i64, P, c_i64]),
            "orc_gemv_mp": (None, [P, c_i64, c_i64, c_i64, P, P]),
            "orc_state_update": (None, [P, c_i64, P, c_int, c_i64, ctypes.c_double]),
            "orc_num_threads": (c_int, []),
            "orc_wz2_width": (c_int, [c_int]),
            "orc_wz2_encode_block": (c_int, [P, c_int, c_int, P]),
            "orc_wz2_decode_block": (None, [P, c_int, c_int, P]),
            "orc_wz3_block": (c_int, [P, ctypes.c_double, c_int, P, P, P, P]),
            "orc_wz3_block_bytes": (c_int, [c_int]),
            "orc_wz3_encode_run": (c_int, [P, c_int, ctypes.c_double, c_int, P, P]),
            "orc_wz3_decode_block": (None, [P, c_int, c_int, P]),
            "orc_wz3_max_blob_size": (c_sz, [c_i64, c_i64]),
            "orc_wz3_encode_matrix": (c_int, [P, c_i64, c_i64, c_i64, ctypes.c_double, P, c_sz, P]),
            "orc_wz3_decode_matrix": (c_int, [P, c_sz, P, c_i64, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(code: int, what: str):
    if code != 0:
        raise OracleError(f"{what} failed with code {code}")


# ----------------------------------------------------------- block-level steps
def fwd_lift4(v):
    a = np.ascontiguousarray(v, dtype=np.int32).copy()
    lib().orc_fwd_lift4(_p(a))
    return a


def inv_lift4(v):
    a = np.ascontiguousarray(v, dtype=np.int32).copy()
    lib().orc_inv_lift4(_p(a))
    return a


def fwd_xform(b):
    a = np.ascontiguousarray(b, dtype=np.int32).reshape(16).copy()
    lib().orc_fwd_xform(_p(a))
    return a.reshape(4, 4)


def inv_xform(b):
    a = np.ascontiguousarray(b, dtype=np.int32).reshape(16).copy()
    lib().orc_inv_xform(_p(a))
    return a.reshape(4, 4)


def int2nb(c: int) -> int:
    return int(lib().orc_int2nb(int(c)))


def nb2int(u: int) -> int:
    return int(lib().orc_nb2int(int(u) & 0xFFFFFFFF))


def sequency() -> list[int]:
    a = np.zeros(16, dtype=np.int32)
    lib().orc_sequency(_p(a))
    return a.tolist()


def encode_planes(u, maxbits: int, nwords: int) -> tuple[np.ndarray, int]:
    uu = np.ascontiguousarray(u, dtype=np.uint32)
    w = np.zeros(nwords, dtype=np.uint64)
    used = lib().orc_encode_planes(_p(uu), int(maxbits), _p(w), 0)
    return w, used


def decode_planes(words, maxbits: int) -> tuple[np.ndarray, int]:
    w = np.ascontiguousarray(words, dtype=np.uint64)
    u = np.zeros(16, dtype=np.uint32)
    used = lib().orc_decode_planes(_p(w), 0, int(maxbits), _p(u))
    return u, used


def encode_block(a, rate: int) -> np.ndarray:
    """One 4x4 block (row-major, FP32 values) -> rate/4 little-endian uint64 words."""
    f = np.ascontiguousarray(a, dtype=np.float32).reshape(16)
    w = np.zeros(rate // 4, dtype=np.uint64)
    _check(lib().orc_wz1_encode_block(_p(f), int(rate), _p(w)), "encode_block")
    return w


def decode_block(words, rate: int):
    """-> (q int32 4x4 after the inverse transform, emax, nonzero, values FP64 4x4)."""
    w = np.ascontiguousarray(words, dtype=np.uint64)
    q = np.zeros(16, dtype=np.int32)
    emax = ctypes.c_int()
    nz = ctypes.c_int()
    lib().orc_wz1_decode_block(_p(w), int(rate), _p(q), ctypes.byref(emax), ctypes.byref(nz))
    vals = np.array([lib().orc_wz1_value(int(x), emax.value, nz.value) for x in q], dtype=np.float64)
    return q.reshape(4, 4), emax.value, nz.value, vals.reshape(4, 4)


def wz2_width(rate: int) -> int:
    return int(lib().orc_wz2_width(int(rate)))


def wz2_encode_block(a, rate: int, lift: bool) -> np.ndarray:
    f = np.ascontiguousarray(a, dtype=np.float32).reshape(16)
    w = np.zeros(rate // 4, dtype=np.uint64)
    _check(lib().orc_wz2_encode_block(_p(f), int(rate), int(bool(lift)), _p(w)), "wz2_encode_block")
    return w


def wz2_decode_block(words, rate: int, lift: bool) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint64)
    out = np.zeros(16, dtype=np.float64)
    lib().orc_wz2_decode_block(_p(w), int(rate), int(bool(lift)), _p(out))
    return out.reshape(4, 4)


def wz3_block(a, tol: float, lift: bool = True):
    """(emax, K, v[16] in sequency order, width the block needs) of the fixed-accuracy reading."""
    f = np.ascontiguousarray(a, dtype=np.float32).reshape(16)
    v = np.zeros(16, dtype=np.int64)
    e, k, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().orc_wz3_block(_p(f), float(tol), int(bool(lift)), ctypes.byref(e), ctypes.byref(k), _p(v),
                               ctypes.byref(w)), "wz3_block")
    return e.value, k.value, v, w.value


def wz3_block_bytes(W: int) -> int:
    return int(lib().orc_wz3_block_bytes(int(W)))


def wz3_encode_run(blocks, tol: float, lift: bool = True):
    """Encode up to 32 blocks (n x 4 x 4) as one run: (words, W)."""
    b = np.ascontiguousarray(blocks, dtype=np.float32).reshape(-1, 16)
    words = np.zeros(b.shape[0] * wz3_block_bytes(31) // 8, dtype=np.uint64)
    w = ctypes.c_int()
    _check(lib().orc_wz3_encode_run(_p(b), b.shape[0], float(tol), int(bool(lift)), _p(words), ctypes.byref(w)),
           "wz3_encode_run")
    return words[: b.shape[0] * wz3_block_bytes(w.value) // 8].copy(), w.value


def wz3_decode_block(words, W: int, lift: bool = True) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint64)
    out = np.zeros(16, dtype=np.float64)
    lib().orc_wz3_decode_block(_p(w), int(W), int(bool(lift)), _p(out))
    return out.reshape(4, 4)


def wz3_encode(A: np.ndarray, tol: float) -> bytes:
    """Whole matrix in the fixed-accuracy layout (with the lift): a blob of variable length."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    M, N = A.shape
    cap = int(lib().orc_wz3_max_blob_size(M, N))
    buf = np.zeros(cap, dtype=np.uint8)
    n = ctypes.c_size_t()
    _check(lib().orc_wz3_encode_matrix(_p(A), M, N, N, float(tol), _p(buf), cap, ctypes.byref(n)), "wz3_encode")
    return buf[: n.value].tobytes()


def wz3_decode(blob: bytes):
    """(decoded FP64 matrix, tolerance) of a fixed-accuracy blob."""
    b = np.frombuffer(blob, dtype=np.uint8)
    M = int(np.frombuffer(blob[16:24], dtype=np.int64)[0])
    N = int(np.frombuffer(blob[24:32], dtype=np.int64)[0])
    out = np.zeros((M, N), dtype=np.float64)
    tol = ctypes.c_double()
    _check(lib().orc_wz3_decode_matrix(_p(b), b.size, _p(out), N, ctypes.byref(tol)), "wz3_decode")
    return out, tol.value


# ---------------------------------------------------------- whole matrices
def blob_size(fmt: int, rate: int, M: int, N: int) -> int:
    return int(lib().orc_blob_size(int(fmt), int(rate), int(M), int(N)))


def encode(A: np.ndarray, fmt: int = FMT_ZFP, rate: int = 16) -> bytes:
    A = np.ascontiguousarray(A, dtype=np.float64)
    M, N = A.shape
    n = blob_size(fmt, rate, M, N)
    if n == 0:
        raise OracleError("bad format, rate or shape")
    out = np.zeros(n, dtype=np.uint8)
    _check(lib().orc_encode(int(fmt), int(rate), _p(A), M, N, N, _p(out), n), "encode")
    return out.tobytes()


def parse(blob: bytes):
    b = np.frombuffer(blob, dtype=np.uint8)
    fmt, rate = ctypes.c_int(), ctypes.c_int()
    M, N = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().orc_parse(_p(b), b.size, ctypes.byref(fmt), ctypes.byref(rate), ctypes.byref(M), ctypes.byref(N)),
           "parse")
    return fmt.value, rate.value, M.value, N.value


def decode_rows(blob: bytes, row0: int, nrows: int) -> np.ndarray:
    b = np.frombuffer(blob, dtype=np.uint8)
    N = int.from_bytes(b[24:32].tobytes(), "little")
    out = np.zeros((nrows, N), dtype=np.float64)
    _check(lib().orc_decode_rows(_p(b), b.size, int(row0), int(nrows), _p(out), N), "decode_rows")
    return out


def decode(blob: bytes) -> np.ndarray:
    _, _, M, _ = parse(blob)
    return decode_rows(blob, 0, M)


def round_fmt(fmt: int, v: float) -> tuple[float, int]:
    bits = ctypes.c_uint32()
    r = lib().orc_round_fmt(int(fmt), float(v), ctypes.byref(bits))
    return r, bits.value


def fmt_max(fmt: int) -> float:
    return float(lib().orc_fmt_max(int(fmt)))


def fmt_decode(fmt: int, bits: int) -> float:
    return float(lib().orc_fmt_decode(int(fmt), int(bits)))


# --------------------------------------------------------------------- GEMV
def gemv64(A: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Y = A @ X in FP64 with sequential j-order sums.  X: (N,) or (N, R)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    vec = X.ndim == 1
    Xc = np.asfortranarray(X.reshape(X.shape[0], -1), dtype=np.float64)
    M, N = A.shape
    R = Xc.shape[1]
    Y = np.zeros((M, R), dtype=np.float64, order="F")
    lib().orc_gemv64(_p(A), M, N, N, _p(Xc), R, N, _p(Y), M)
    return Y[:, 0].copy() if vec else Y


def gemv_mp(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(A.shape[0], dtype=np.float32)
    lib().orc_gemv_mp(_p(A), A.shape[0], A.shape[1], A.shape[1], _p(x), _p(y))
    return y


def state_update(s: np.ndarray, Y: np.ndarray, decay: float) -> np.ndarray:
    s = np.ascontiguousarray(s, dtype=np.float64).copy()
    Yc = np.asfortranarray(Y.reshape(Y.shape[0], -1), dtype=np.float64)
    lib().orc_state_update(_p(s), s.size, _p(Yc), Yc.shape[1], Yc.shape[0], float(decay))
    return s


def num_threads() -> int:
    return int(lib().orc_num_threads())


def crc32(data: bytes) -> int:
    b = np.frombuffer(data, dtype=np.uint8)
    return int(lib().orc_crc32(_p(b), b.size))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
