"""CPU-only checks of the library: it loads, exports every symbol include/whff.h
declares, and its host encoder (whff_compress, the offline step of Sec. 4.3)
produces blobs byte-identical to the oracle's, for every format, for ragged
shapes, for band-by-band encoding and for every thread count."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def W():
    import paper_1902_08018_gb300 as W

    W.library()
    return W


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "whff.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(whff_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(W):
    names = _declared_functions()
    assert len(names) >= 12
    L = W.library()
    for n in names:
        assert hasattr(L, n), n
    assert L.whff_version().startswith(b"whff")


def test_compressed_size_formula(W):
    for M, N, rate in [(1, 1, 4), (4096, 4096, 16), (32768, 32768, 16), (7, 9, 12)]:
        assert W.compressed_size(W.FMT_ZFP, rate, M, N) == 64 + -(-M // 4) * -(-N // 4) * 2 * rate
    assert W.compressed_size(W.FMT_ZFP, 6, 8, 8) == 0  # rate not a multiple of 4
    assert W.compressed_size(W.FMT_ZFP, 16, 0, 8) == 0
    assert W.compressed_size(W.FMT_BF16, 0, 200, 150) == 64 + 200 * 160 * 2 + 2 * 2 * 4
    assert W.compressed_size(W.FMT_FP32, 0, 200, 150) == 64 + 200 * 160 * 4 + 2 * 2 * 4
    assert W.compressed_size(W.FMT_FIXED_LIFT, 16, 5, 9) == 64 + 2 * 3 * 32
    assert W.compressed_size(W.FMT_FIXED_LIFT, 4, 8, 8) == 0  # WZ2 rates are 8..24
    assert W.compressed_size(W.FMT_FIXED_BFP, 28, 8, 8) == 0


@pytest.mark.parametrize("fmt,rate", [(1, 4), (1, 8), (1, 12), (1, 16), (1, 24), (1, 36), (2, 0), (3, 0), (4, 0), (7, 0),
                                      (5, 8), (5, 12), (5, 16), (5, 24), (6, 8), (6, 16), (6, 20)])
def test_encoder_byte_identical_to_oracle(W, orc, fmt, rate):
    import workloads

    rng = np.random.default_rng(40 + fmt * 100 + rate)
    mats = [
        workloads.KernelMatrix(130, 12, 130, 0.2, 7).dense()[:, :97],  # smooth, ragged
        rng.standard_normal((33, 45)) * np.exp(rng.uniform(-30, 30, size=(33, 45))),  # wild dynamic range
        np.zeros((9, 5)),
        np.where(rng.random((20, 20)) < 0.7, 0.0, rng.standard_normal((20, 20)) * 1e-35),  # tiny / subnormal
    ]
    for A in mats:
        r = rate if fmt == 1 else 16
        lib = W.whff_compress(A, fmt, r, nthreads=3)
        ref = np.frombuffer(orc.encode(A, fmt, r), dtype=np.uint8)
        assert lib.size == ref.size
        assert (lib == ref).all()


def test_encoder_byte_identical_on_a_seeded_sweep_of_shapes(W, orc):
    """60 small ragged shapes (1..70 rows and columns) in every format and a rate drawn
    for it, with smooth, wild-range, sparse and integer-valued matrices: the library's
    blob equals the oracle's byte for byte, for 1 and 3 host threads."""
    rng = np.random.default_rng(2024)
    choices = [(1, r) for r in (4, 8, 12, 16, 20, 24, 32, 48, 64)] + [(5, r) for r in (8, 12, 16, 20, 24)] + \
              [(6, r) for r in (8, 12, 16, 20, 24)] + [(2, 0), (3, 0), (4, 0), (7, 0)]
    for k in range(60):
        M, N = (int(v) for v in rng.integers(1, 71, size=2))
        fmt, rate = choices[int(rng.integers(len(choices)))]
        kind = k % 4
        if kind == 0:
            i, j = np.mgrid[0:M, 0:N]
            A = np.exp(-((i - M / 2) ** 2 + (j - N / 3) ** 2) / (0.1 * (M * M + N * N) + 1.0))
        elif kind == 1:
            A = rng.standard_normal((M, N)) * np.exp(rng.uniform(-40, 40, size=(M, N)))
        elif kind == 2:
            A = np.where(rng.random((M, N)) < 0.8, 0.0, rng.standard_normal((M, N)))
        else:
            A = rng.integers(-1000, 1000, size=(M, N)).astype(np.float64)
        ref = np.frombuffer(orc.encode(A, fmt, rate or 16), dtype=np.uint8)
        for nt in (1, 3):
            got = W.whff_compress(A, fmt, rate or 16, nthreads=nt)
            assert got.size == ref.size and (got == ref).all(), (k, M, N, fmt, rate, nt)


def test_fixed_accuracy_encoder_byte_identical_on_a_seeded_sweep(W, orc):
    """30 small ragged shapes (up to 150 columns: several runs per band) at tolerances
    from 0 to 1, smooth, wild-range and sparse matrices: the library's fixed-accuracy
    blob equals the oracle's byte for byte."""
    rng = np.random.default_rng(2025)
    for k in range(30):
        M, N = int(rng.integers(1, 40)), int(rng.integers(1, 151))
        tol = [0.0, 1e-12, 1e-7, 1e-3, 1.0][k % 5]
        kind = k % 3
        if kind == 0:
            i, j = np.mgrid[0:M, 0:N]
            A = np.cos(0.05 * i) * np.exp(-0.01 * j) + 1e-3 * rng.standard_normal((M, N))
        elif kind == 1:
            A = rng.standard_normal((M, N)) * np.exp(rng.uniform(-30, 30, size=(M, N)))
        else:
            A = np.where(rng.random((M, N)) < 0.9, 0.0, rng.standard_normal((M, N)))
        want = orc.wz3_encode(A, tol)
        got = W.whff_compress_accuracy(A, tol, nthreads=2)
        assert got.tobytes() == want, (k, M, N, tol)


def test_fixed_accuracy_encoder_at_tolerances_equal_to_an_achieved_error(W, orc):
    """Tolerances placed exactly on a shift's decoded error, and one ulp below it,
    are where a shortcut in the shift search would first differ: the library's
    one-block blobs equal the oracle's there."""
    rng = np.random.default_rng(77)
    for k in range(120):
        kind = k % 3
        if kind == 0:
            a = (1.0 + 0.1 * rng.standard_normal((4, 4))) * 2.0 ** int(rng.integers(-20, 20))
        elif kind == 1:
            a = rng.standard_normal((4, 4))
        else:
            a = np.exp(-rng.random((4, 4)) * 3.0)
        a32 = a.astype(np.float32)
        words, Wr = orc.wz3_encode_run(a32.reshape(1, 4, 4), 10.0 ** float(rng.uniform(-9, -2)))
        err = float(np.abs(orc.wz3_decode_block(words, Wr) - a32.astype(np.float64)).max())
        for tol in (err, float(np.nextafter(err, 0.0))):
            want = orc.wz3_encode(a32.astype(np.float64), tol)
            got = W.whff_compress_accuracy(a32.astype(np.float64), tol)
            assert got.tobytes() == want, (k, tol)


def test_band_encoding_and_thread_count_invariance(W, orc):
    import workloads

    km = workloads.KernelMatrix(300, 18, 300, 0.1, 9)
    A = km.dense()
    ref = np.frombuffer(orc.encode(A, 1, 12), dtype=np.uint8)
    for nt in (1, 2, 7):
        assert (W.whff_compress(A, 1, 12, nthreads=nt) == ref).all()
    bands = ((r0, A[r0:r0 + 64]) for r0 in range(0, 300, 64))
    assert (W.whff_compress_bands(300, 300, bands, 1, 12) == ref).all()
    ref2 = np.frombuffer(orc.encode(A, 3), dtype=np.uint8)
    bands = ((r0, A[r0:r0 + 128]) for r0 in range(0, 300, 128))
    assert (W.whff_compress_bands(300, 300, bands, 3) == ref2).all()


def test_encoder_errors(W):
    A = np.ones((8, 8))
    A[3, 3] = np.inf
    with pytest.raises(W.WhffError) as e:
        W.whff_compress(A)
    assert e.value.code == -3
    A[3, 3] = 3e38
    with pytest.raises(W.WhffError) as e:
        W.whff_compress(A)
    assert e.value.code == -2
    with pytest.raises(W.WhffError):
        W.whff_compress(np.ones((8, 8)), 1, 10)


def test_create_rejects_corrupt_blob_without_gpu(W):
    # header checks run before any CUDA call, so they are testable on the CPU
    blob = W.whff_compress(np.ones((8, 8)), 1, 8).copy()
    blob[70] ^= 1  # stream byte: CRC mismatch
    with pytest.raises(W.WhffError) as e:
        W.whff_create(blob, stream=0)
    assert e.value.code == -5
    blob = W.whff_compress(np.ones((8, 8)), 1, 8).copy()
    blob[0] = ord("X")
    with pytest.raises(W.WhffError) as e:
        W.whff_create(blob, stream=0)
    assert e.value.code == -5


def _reheader(blob, M, N):
    """The blob with its header's M and N replaced and the header CRC made valid again."""
    import struct
    import zlib

    b = bytearray(np.asarray(blob, dtype=np.uint8).tobytes())
    b[16:32] = struct.pack("<qq", M, N)
    b[44:48] = struct.pack("<I", zlib.crc32(bytes(b[:44])))
    return np.frombuffer(bytes(b), dtype=np.uint8).copy()


@pytest.mark.parametrize("M,N", [((1 << 61) + 4, 4), (4, (1 << 61) + 4), ((1 << 48) + 1, 4), (1 << 40, 1 << 40)])
def test_create_rejects_oversized_shapes_without_gpu(W, M, N):
    """A header whose shape would wrap the 64-bit size arithmetic is refused before any
    CUDA call: with M = 2^61 + 4 and N = 4, ceil(M/4) * 32 bytes = 2^64 + 32 wraps to
    the 32 bytes a 4 x 4 rate-16 stream holds, and the kernels would walk 2^59 blocks."""
    blob = W.whff_compress(np.ones((4, 4)), W.FMT_FIXED_LIFT, 16)
    with pytest.raises(W.WhffError) as e:
        W.whff_create(_reheader(blob, M, N), stream=0)
    assert e.value.code == -5
    acc = W.whff_compress_accuracy(np.ones((4, 4)), 0.0)
    with pytest.raises(W.WhffError) as e:
        W.whff_create(_reheader(acc, M, N), stream=0)
    assert e.value.code == -5
    assert W.compressed_size(W.FMT_FIXED_LIFT, 16, M, N) == 0
    assert W.compressed_size(W.FMT_BF16, 0, M, N) == 0
    assert W.library().whff_accuracy_max_size(M, N) == 0


def test_largest_accepted_shape_sizes():
    """The bound keeps the largest accepted shapes' sizes exact (no wrap)."""
    import paper_1902_08018_gb300 as W

    M, N = 1 << 48, 1 << 14  # 2^46 x 2^12 = 2^58 blocks: over the 2^56 bound
    assert W.compressed_size(W.FMT_FIXED_LIFT, 16, M, N) == 0
    M, N = 1 << 48, 1 << 12  # 2^46 x 2^10 = 2^56 blocks: accepted
    assert W.compressed_size(W.FMT_FIXED_LIFT, 16, M, N) == 64 + (1 << 56) * 32


@pytest.mark.parametrize("M,N", [(130, 97), (64, 260), (5, 3), (257, 1030)])
@pytest.mark.parametrize("tol", [1e-2, 1e-6, 0.0])
def test_fixed_accuracy_encoder_byte_identical_to_oracle(W, orc, M, N, tol):
    """WZ3 (fixed accuracy, Sec. 4.3 read with a per-block shift and per-run field width):
    the library's blob, index included, equals the oracle's byte for byte, for every
    thread count."""
    import workloads

    A = workloads.RectKernelMatrix(M, N, 0.05, M * 7 + N).dense()
    want = orc.wz3_encode(A, tol)
    for nt in (1, 3, 0):
        got = W.whff_compress_accuracy(A, tol, nthreads=nt)
        assert got.tobytes() == want, nt


def test_fixed_accuracy_encoder_hand_derived_matrix(W):
    """The library's WZ3 blob of the hand-derived matrix in tests/golden/wz3_blocks.txt
    (one lifted step block at K 25 and a constant at K 27 sharing a run of width 4,
    word-interleaved), whole and band by band."""
    from test_oracle_wz3 import _golden_wz3, golden_wz3_matrix

    for rec in _golden_wz3()["matrix"]:
        A, want = golden_wz3_matrix(rec)
        assert W.whff_compress_accuracy(A, float(rec[1])).tobytes() == want
        got = W.whff_compress_accuracy_bands(A.shape[0], A.shape[1], [(0, A)], float(rec[1]))
        assert got.tobytes() == want


def test_block_encoders_hand_derived_words(W):
    """The library's WZ1 and WZ2 streams of the hand-derived 4 x 4 blocks in
    tests/golden/wz1_blocks.txt and wz2_blocks.txt (a one-block matrix's stream is
    the block's words)."""
    from test_oracle_wz1 import _golden as wz1_golden
    from test_oracle_wz2 import _golden as wz2_golden

    for name, rate, block, words, _ in wz1_golden():
        got = np.frombuffer(W.whff_compress(block.astype(np.float64).reshape(4, 4), W.FMT_ZFP, rate).tobytes()[64:],
                            dtype=np.uint64)
        assert [int(x) for x in got[: len(words)]] == words and not got[len(words):].any(), name
    for name, rate, lift, block, words in wz2_golden():
        fmt = W.FMT_FIXED_LIFT if lift else W.FMT_FIXED_BFP
        got = np.frombuffer(W.whff_compress(block.reshape(4, 4), fmt, rate).tobytes()[64:], dtype=np.uint64)
        assert [int(x) for x in got[: len(words)]] == words, name


def test_scaled_encoder_hand_derived_streams(W):
    """The library's scaled-format streams of the hand-derived matrices in
    tests/golden/scaled_blobs.txt (row padding to 16 elements, tile scales after the
    payload, the FP32 scale's rounding carried into the quotients)."""
    from test_oracle_gemv_scaled import golden_scaled

    for name, fmt, A, body in golden_scaled():
        assert W.whff_compress(A, fmt, 0).tobytes()[64:] == body, name


def test_fixed_accuracy_rejections(W):
    with pytest.raises(W.WhffError):
        W.whff_compress_accuracy(np.ones((4, 4)), -1.0)
    with pytest.raises(W.WhffError):
        W.whff_compress_accuracy(np.full((4, 4), np.nan), 1e-3)


@pytest.mark.parametrize("split", [[4], [8, 120], [12, 4, 4, 100, 8], [256]])
def test_fixed_accuracy_bands_equal_whole_matrix(W, split):
    """The band interface of the fixed-accuracy format gives the whole-matrix blob byte
    for byte, for every band split (the last band ragged), and every thread count."""
    import workloads

    M, N = 259, 1030
    A = workloads.RectKernelMatrix(M, N, 0.05, 17).dense()
    want = W.whff_compress_accuracy(A, 1e-5).tobytes()
    bounds, r = [], 0
    for k in split:
        if r >= M:
            break
        bounds.append((r, min(M, r + k)))
        r += k
    if r < M:
        bounds.append((r, M))
    for nt in (1, 0):
        got = W.whff_compress_accuracy_bands(M, N, ((a, A[a:b]) for a, b in bounds), 1e-5, nthreads=nt)
        assert got.tobytes() == want, (split, nt)


def test_fixed_accuracy_bands_refusals(W):
    import ctypes

    L = W.library()
    M, N = 16, 40
    A = np.ones((M, N))
    cap = int(L.whff_accuracy_max_size(M, N))
    out = np.zeros(cap, dtype=np.uint8)
    assert L.whff_accuracy_begin(out.ctypes.data, cap, M, N, 1e-3) == 0
    band = np.ascontiguousarray(A[4:8])
    assert L.whff_compress_accuracy_band(out.ctypes.data, cap, band.ctypes.data, 4, 4, N, 1) != 0  # not the next row
    band = np.ascontiguousarray(A[0:6])
    assert L.whff_compress_accuracy_band(out.ctypes.data, cap, band.ctypes.data, 0, 6, N, 1) != 0  # 6 rows mid-matrix
    band = np.ascontiguousarray(A[0:8])
    assert L.whff_compress_accuracy_band(out.ctypes.data, cap, band.ctypes.data, 0, 8, N, 1) == 0
    used = ctypes.c_size_t()
    assert L.whff_accuracy_seal(out.ctypes.data, cap, ctypes.byref(used)) != 0  # rows 8..15 missing
    with pytest.raises(W.WhffError):
        W.whff_create(out, stream=0)  # unsealed: refused before any device work
    band = np.ascontiguousarray(A[8:16])
    assert L.whff_compress_accuracy_band(out.ctypes.data, cap, band.ctypes.data, 8, 8, N, 1) == 0
    assert L.whff_accuracy_seal(out.ctypes.data, cap, ctypes.byref(used)) == 0
    assert out[: used.value].tobytes() == W.whff_compress_accuracy(A, 1e-3).tobytes()
    small = np.zeros(70, dtype=np.uint8)
    assert L.whff_accuracy_begin(small.ctypes.data, small.size, M, N, 1e-3) != 0  # no room for the index
    # a damaged area counter of an unsealed blob: the seal refuses it instead of reading past cap
    assert L.whff_accuracy_begin(out.ctypes.data, cap, M, N, 1e-3) == 0
    band = np.ascontiguousarray(A)
    assert L.whff_compress_accuracy_band(out.ctypes.data, cap, band.ctypes.data, 0, M, N, 1) == 0
    for area in (cap, 1 << 62, (1 << 64) - 8):
        out[56:64] = np.frombuffer(np.uint64(area).tobytes(), dtype=np.uint8)
        assert L.whff_accuracy_seal(out.ctypes.data, cap, ctypes.byref(used)) != 0, area
    # and a band appended to such a blob is refused before anything is written
    assert L.whff_accuracy_begin(out.ctypes.data, cap, M, N, 1e-3) == 0
    out[56:64] = np.frombuffer(np.uint64((1 << 64) - 8).tobytes(), dtype=np.uint8)
    before = out.copy()
    assert L.whff_compress_accuracy_band(out.ctypes.data, cap, band.ctypes.data, 0, M, N, 1) != 0
    assert (out == before).all()
