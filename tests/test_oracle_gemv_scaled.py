"""Pins of the oracle's GEMV (Sec. 4.4, dot-product equation and the
sequential mixed-precision listing), its state update (stand-in for the
thermal update of Sec. 2.1) and its scaled storage formats, against exact
rational arithmetic, closed forms, numpy / torch's own conversions and hand-derived
streams (tests/golden/scaled_blobs.txt)."""
import math
from fractions import Fraction

import numpy as np
import pytest


# --------------------------------------------------------------------- GEMV
def test_gemv64_against_exact_rationals(orc):
    rng = np.random.default_rng(20)
    for M, N in [(1, 1), (3, 5), (12, 12), (7, 11)]:
        A = rng.standard_normal((M, N)) * 10.0 ** rng.integers(-3, 3, size=(M, N))
        x = rng.standard_normal(N)
        y = orc.gemv64(A, x)
        for i in range(M):
            exact = sum(Fraction(float(A[i, j])) * Fraction(float(x[j])) for j in range(N))
            scale = sum(abs(Fraction(float(A[i, j])) * Fraction(float(x[j]))) for j in range(N))
            # a sequential FP64 sum of N products: error <= N * 2^-53 * sum |terms| (first order)
            assert abs(Fraction(float(y[i])) - exact) <= Fraction(N + 1, 2 ** 53) * scale


def test_gemv64_matches_numpy_and_multi_rhs(orc):
    rng = np.random.default_rng(21)
    A = rng.standard_normal((300, 257))
    X = rng.standard_normal((257, 5))
    Y = orc.gemv64(A, X)
    ref = A @ X
    assert np.abs(Y - ref).max() <= 1e-13 * np.abs(A).sum(1).max() * np.abs(X).max()
    for r in range(5):
        assert (orc.gemv64(A, X[:, r].copy()) == Y[:, r]).all()


def test_gemv64_exact_on_integers_and_unit_vectors(orc):
    rng = np.random.default_rng(22)
    A = rng.integers(-1000, 1000, size=(40, 60)).astype(np.float64)
    x = rng.integers(-1000, 1000, size=60).astype(np.float64)
    assert (orc.gemv64(A, x) == A.astype(np.int64) @ x.astype(np.int64)).all()
    e = np.zeros(60)
    e[17] = 1.0
    assert (orc.gemv64(A, e) == A[:, 17]).all()


def test_gemv_mp_paper_rule(orc):
    # FP32 products of exactly-representable small integers are exact, so the
    # FP64 sum is exact and the FP32 result is the rounded exact dot product
    rng = np.random.default_rng(23)
    A = rng.integers(-2000, 2000, size=(20, 3000)).astype(np.float64)
    x = rng.integers(-2000, 2000, size=3000).astype(np.float64)
    exact = A.astype(np.int64) @ x.astype(np.int64)
    assert (orc.gemv_mp(A, x) == exact.astype(np.float32)).all()
    # and the product is rounded to FP32 before widening (not an FP64 product)
    a = 1.0 + 2.0 ** -12
    y = orc.gemv_mp(np.array([[a]]), np.array([a]))
    assert float(y[0]) == float(np.float32(a) * np.float32(a))


def test_state_update_closed_form(orc):
    M, decay = 9, 0.99
    y = np.arange(M, dtype=np.float64) + 1.0
    s = np.zeros(M)
    for k in range(1, 50):
        s = orc.state_update(s, y.reshape(M, 1), decay)
        closed = y * (1 - decay ** k) / (1 - decay)
        assert np.allclose(s, closed, rtol=1e-13)
    # multi-column: columns applied in order r = 0, 1, ...
    Y = np.stack([y, 2 * y, 3 * y], axis=1)
    s1 = orc.state_update(np.ones(M), Y, 0.5)
    ref = np.ones(M)
    for r in range(3):
        ref = 0.5 * ref + Y[:, r]
    assert (s1 == ref).all()


# ----------------------------------------------------------- scaled formats
def test_fp16_rounding_matches_numpy(orc):
    rng = np.random.default_rng(24)
    vals = rng.standard_normal(20000) * 10.0 ** rng.integers(-9, 5, size=20000)
    vals = np.concatenate([vals, [0.0, -0.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26, 32768.0, 1.0 + 2.0 ** -11]])
    for v in vals:
        r, bits = orc.round_fmt(orc.FMT_FP16, float(v))
        if abs(v) <= 32768.0:
            ref = np.float16(v)  # numpy rounds FP64 -> FP16 directly, ties to even
            assert r == float(ref), v
            assert bits == int(np.array(ref).view(np.uint16)), v
        else:
            assert abs(r) == 32768.0
        assert orc.fmt_decode(orc.FMT_FP16, bits) == r


def test_bf16_rounding_matches_torch_on_fp32_values(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(25)
    vals = (rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 1, size=20000)).astype(np.float32)
    vals = vals[np.abs(vals) <= 1.0]
    ref = torch.from_numpy(vals).to(torch.bfloat16)
    ref_bits = ref.view(torch.int16).numpy().astype(np.uint16)
    for v, rb, rv in zip(vals, ref_bits, ref.float().numpy()):
        r, bits = orc.round_fmt(orc.FMT_BF16, float(v))
        assert r == float(rv) and bits == int(rb), v
        assert orc.fmt_decode(orc.FMT_BF16, bits) == r


def test_e4m3_rounding_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(26)
    vals = (rng.standard_normal(20000) * 10.0 ** rng.integers(-4, 3, size=20000)).astype(np.float32)
    vals = vals[np.abs(vals) <= 448.0]
    ref = torch.from_numpy(vals).to(torch.float8_e4m3fn)
    ref_bits = ref.view(torch.uint8).numpy()
    for v, rb, rv in zip(vals, ref_bits, ref.float().numpy()):
        r, bits = orc.round_fmt(orc.FMT_FP8E4M3, float(v))
        assert r == float(rv) and bits == int(rb), v
    # every finite E4M3 pattern decodes like torch
    pats = np.array([b for b in range(256) if (b & 0x7F) != 0x7F], dtype=np.uint8)
    tv = torch.from_numpy(pats).view(torch.float8_e4m3fn).float().numpy()
    for b, t in zip(pats, tv):
        assert orc.fmt_decode(orc.FMT_FP8E4M3, int(b)) == float(t)
    # saturation instead of NaN
    assert orc.round_fmt(orc.FMT_FP8E4M3, 1e6)[0] == 448.0
    assert orc.round_fmt(orc.FMT_FP8E4M3, -500.0)[0] == -448.0


@pytest.mark.parametrize("fmt", [2, 3, 4])
def test_scaled_blob_roundtrip_properties(orc, fmt):
    rng = np.random.default_rng(27 + fmt)
    M, N = 200, 150  # ragged against the 128x128 scale tiles
    A = rng.standard_normal((M, N)) * np.exp(rng.uniform(-3, 3, size=(M, N)))
    blob = orc.encode(A, fmt)
    ld = math.ceil(N / 16) * 16
    el = 1 if fmt == 4 else 2
    assert len(blob) == 64 + M * ld * el + math.ceil(M / 128) * math.ceil(N / 128) * 4
    D = orc.decode(blob)
    fmax = orc.fmt_max(fmt)
    for ti in range(2):
        for tj in range(2):
            t = A[128 * ti:128 * ti + 128, 128 * tj:128 * tj + 128]
            d = D[128 * ti:128 * ti + 128, 128 * tj:128 * tj + 128]
            s = float(np.float32(np.abs(t).max() / fmax))
            # every decoded value is s * (a format value), the amax maps to +-FMTMAX (or
            # rounds next to it), and values exactly s*q round-trip exactly
            i = np.unravel_index(np.abs(t).argmax(), t.shape)
            assert abs(abs(d[i]) / s - fmax) <= fmax * 2.0 ** -7
            q = d / s
            for v in q.reshape(-1)[:500]:
                assert orc.round_fmt(fmt, float(v))[0] == v
            rel = {2: 2.0 ** -8, 3: 2.0 ** -11, 4: 2.0 ** -4}[fmt]
            tiny = {2: 0.0, 3: s * 2.0 ** -24, 4: s * 2.0 ** -9}[fmt]
            assert (np.abs(d - t) <= rel * np.abs(t) + tiny).all()
    # a matrix that is exactly s * q (q a format value, one entry per tile = FMTMAX)
    # decodes exactly: the tile scale comes out as s and every quotient is exact
    s = 0.5
    q = fmax * rng.choice([0.0, 0.125, -0.125, 0.25, -0.25, 0.5, -0.5, 1.0, -1.0], size=(M, N))
    q[::128, ::128] = fmax
    B = s * q
    assert (orc.decode(orc.encode(B, fmt)) == B).all()


def test_fp32_storage_is_numpy_float32(orc):
    """FP32 storage (the uncompressed comparison) decodes to exactly numpy's
    float32 rounding of A -- normal, subnormal, ties and zero entries -- with
    every tile scale 1; |a| >= 2^127 and non-finite entries are refused."""
    rng = np.random.default_rng(71)
    M, N = 150, 140
    A = rng.standard_normal((M, N)) * np.exp(rng.uniform(-100, 80, size=(M, N)))
    A[0, :8] = [0.0, -0.0, 2.0 ** -149, 2.0 ** -150 * 3, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, -(2.0 ** 126), 1e-50]
    blob = orc.encode(A, orc.FMT_FP32)
    ld = math.ceil(N / 16) * 16
    assert len(blob) == 64 + M * ld * 4 + 2 * 2 * 4
    scales = np.frombuffer(blob[64 + M * ld * 4:], dtype=np.float32)
    assert (scales == 1.0).all()
    ref = A.astype(np.float32).astype(np.float64)
    D = orc.decode(blob)
    assert (D.view(np.uint64) == ref.view(np.uint64)).all()
    for bad, code in ((2.0 ** 127, -2), (np.inf, -3), (np.nan, -3)):
        B = A.copy()
        B[5, 7] = bad
        with pytest.raises(orc.OracleError):
            orc.encode(B, orc.FMT_FP32)


def test_gemv_mp_follows_the_papers_rounding(orc):
    """The paper's mixed precision (Sec. 4.4): products rounded to FP32, their
    sum in FP64, y rounded to FP32 -- checked against the same steps in numpy
    on a small case where the FP64 sum order is the same."""
    rng = np.random.default_rng(72)
    A = rng.standard_normal((9, 31))
    x = rng.standard_normal(31)
    y = orc.gemv_mp(A, x)
    for i in range(9):
        p = A[i].astype(np.float32) * x.astype(np.float32)  # float32 products, rounded
        s = 0.0
        for v in p:
            s += float(v)
        assert y[i] == np.float32(s)


# ----------------------------------------------- hand-derived scaled streams
def _runs(field, conv):
    """Values of a fixture field: whitespace-separated, v*k for k copies."""
    out = []
    for t in field.split():
        v, _, k = t.partition("*")
        out.extend([conv(v)] * (int(k) if k else 1))
    return out


def golden_scaled():
    """Records of tests/golden/scaled_blobs.txt as (name, fmt, A, expected stream bytes).
    The stream is assembled here from the layout rule the header documents: M rows of
    roundup(N, 16) little-endian elements, the padding zero, then the FP32 tile scales."""
    import os
    import struct

    path = os.path.join(os.path.dirname(__file__), "golden", "scaled_blobs.txt")
    recs = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        fmt, name, M, N, rows, scales, qrows = [f.strip() for f in line.split("|")]
        fmt, M, N = int(fmt), int(M), int(N)
        A = np.array([_runs(r, float) for r in rows.split(";")])
        assert A.shape == (M, N), name
        eb = {2: 2, 3: 2, 4: 1, 7: 4}[fmt]
        ld = -(-N // 16) * 16
        packer = {1: "<B", 2: "<H", 4: "<I"}[eb]
        body = b""
        for r in qrows.split(";"):
            q = _runs(r, lambda v: int(v, 16))
            assert len(q) == N, name
            body += b"".join(struct.pack(packer, v) for v in q) + bytes((ld - N) * eb)
        body += b"".join(struct.pack("<I", v) for v in _runs(scales, lambda v: int(v, 16)))
        recs.append((name, fmt, A, body))
    return recs


@pytest.mark.parametrize("rec", golden_scaled(), ids=lambda r: r[0])
def test_scaled_hand_derived_streams(orc, rec):
    import struct

    name, fmt, A, body = rec
    blob = orc.encode(A, fmt)
    assert blob[64:] == body, name
    magic, ver, f, rate, M, N, sbytes = struct.unpack("<4sIIIqqQ", blob[:40])
    assert (magic, ver, f, rate, M, N, sbytes) == (b"WZ1\0", 1, fmt, 8 * {2: 2, 3: 2, 4: 1, 7: 4}[fmt],
                                                   A.shape[0], A.shape[1], len(body))
