"""Pins of the CPU oracle's WZ1 coder (Sec. 4.3, zfp-style fixed rate) against
facts that do not come from the oracle itself: closed forms of the lift,
the definition of base -2, hand-derived streams, exact round trips at full
rate, the embedded-prefix and fixed-size properties, and an independent CRC."""
import math
import os
import zlib
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "wz1_blocks.txt")
FULL_RATE = 36  # 576 bits >= 9 header + 512 plane bits + at most 48 test bits


# ------------------------------------------------------------------- lifting
def test_lift_constant_and_ramp(orc):
    for c in [0, 1, -1, 12345, -(2 ** 25), 2 ** 25 - 1]:
        assert orc.fwd_lift4([c] * 4).tolist() == [c, 0, 0, 0]
    # ramp a + b*i with even b: s is the exact mean, d = 2b, d0 = b, e = 0
    rng = np.random.default_rng(1)
    for _ in range(200):
        a = int(rng.integers(-2 ** 24, 2 ** 24))
        b = 2 * int(rng.integers(-2 ** 20, 2 ** 20))
        s, d, d0, e = orc.fwd_lift4([a, a + b, a + 2 * b, a + 3 * b]).tolist()
        assert Fraction(s) == Fraction(4 * a + 6 * b, 4)
        assert (d, d0, e) == (2 * b, b, 0)


def test_lift_is_the_linear_haar_pair_when_no_rounding(orc):
    # With all inputs multiples of 4 every halving is exact, so the lift must equal the
    # linear transform s = mean, d = ((x2+x3) - (x0+x1))/2, d0 = x1-x0, e = (x3-x2) - (x1-x0).
    rng = np.random.default_rng(2)
    for _ in range(500):
        x = (4 * rng.integers(-2 ** 22, 2 ** 22, size=4)).tolist()
        s, d, d0, e = orc.fwd_lift4(x).tolist()
        assert Fraction(s) == Fraction(sum(x), 4)
        assert Fraction(d) == Fraction(x[2] + x[3] - x[0] - x[1], 2)
        assert d0 == x[1] - x[0]
        assert e == (x[3] - x[2]) - (x[1] - x[0])


def test_lift_inverse_exhaustive_small_and_random_full_range(orc):
    import itertools

    for v in itertools.product(range(-2, 3), repeat=4):
        assert tuple(orc.inv_lift4(orc.fwd_lift4(v)).tolist()) == v
    rng = np.random.default_rng(3)
    for _ in range(3000):
        v = rng.integers(-2 ** 31, 2 ** 31, size=4, dtype=np.int64).astype(np.int32)
        assert (orc.inv_lift4(orc.fwd_lift4(v)) == v).all()
    for _ in range(300):
        b = rng.integers(-2 ** 26, 2 ** 26, size=(4, 4)).astype(np.int32)
        assert (orc.inv_xform(orc.fwd_xform(b)) == b).all()


def test_lift_growth_bound(orc):
    # |coefficient| < 2^30 for |x| < 2^26: growth at most 4x per dimension
    rng = np.random.default_rng(4)
    for _ in range(2000):
        b = rng.choice([-(2 ** 26) + 1, 2 ** 26 - 1, 0], size=(4, 4)).astype(np.int32)
        assert np.abs(orc.fwd_xform(b).astype(np.int64)).max() < 2 ** 30


# ---------------------------------------------------------------- negabinary
def _base_m2_value(u: int) -> int:
    return sum(((u >> k) & 1) * (-2) ** k for k in range(32))


def test_negabinary_is_base_minus_two(orc):
    rng = np.random.default_rng(5)
    vals = [0, 1, -1, 2, -2, 2 ** 29, -(2 ** 29), 2 ** 30 - 1, -(2 ** 30) + 1]
    vals += rng.integers(-2 ** 30 + 1, 2 ** 30, size=2000).tolist()
    for c in vals:
        u = orc.int2nb(c)
        assert _base_m2_value(u) == c
        assert orc.nb2int(u) == c


# ----------------------------------------------------------------- sequency
def test_sequency_order(orc):
    p = orc.sequency()
    assert sorted(p) == list(range(16))
    rank = [0, 1, 2, 2]
    keys = [(rank[k // 4] + rank[k % 4], max(rank[k // 4], rank[k % 4]), k // 4, k % 4) for k in p]
    assert keys == sorted(keys)
    assert p[0] == 0 and set(p[1:3]) == {1, 4}


# --------------------------------------------------------------- the coder
def _block(field):
    """One value fills the block; four are every row of it."""
    v = [float(t) for t in field.split()]
    return np.full(16, v[0], dtype=np.float32) if len(v) == 1 else np.tile(np.array(v, dtype=np.float32), 4)


def _golden():
    """(name, rate, block, leading words, decoded block)."""
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = [t.strip() for t in line.split("|")]
        name, rate, block, words = f[0], int(f[1]), _block(f[2]), [int(t, 16) for t in f[3].split()]
        dec = _block(f[4]) if len(f) > 4 else block
        rows.append((name, rate, block, words, dec))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: r[0])
def test_hand_derived_streams(orc, row):
    name, rate, block, words, dec = row
    w = orc.encode_block(block, rate)
    assert [int(x) for x in w[: len(words)]] == words
    assert not w[len(words):].any()
    q, emax, nz, vals = orc.decode_block(w, rate)
    assert (vals.reshape(16) == dec.astype(np.float64)).all()


def _bfp_truncate(a: np.ndarray) -> np.ndarray:
    """Closed form of the only loss at full rate: each value cut toward zero to the
    block's grid 2^(emax-26), emax = max frexp exponent of the block."""
    a = a.astype(np.float32).astype(np.float64)
    nz = a[a != 0]
    if nz.size == 0:
        return np.zeros_like(a)
    emax = max(math.frexp(float(v))[1] for v in nz)
    if emax <= -100:
        return np.zeros_like(a)
    step = 2.0 ** (emax - 26)
    return np.trunc(a / step) * step


def test_full_rate_exact_all_binary_patterns(orc):
    # every 0/1 pattern of a 4x4 block, at a few scales: decodes to the input exactly
    for scale in (1.0, 2.0 ** -20, 2.0 ** 40):
        for pat in range(0, 1 << 16, 7 if scale != 1.0 else 1):
            a = np.array([(pat >> i) & 1 for i in range(16)], dtype=np.float64) * scale
            _, _, _, vals = orc.decode_block(orc.encode_block(a, FULL_RATE), FULL_RATE)
            assert (vals.reshape(16) == a).all(), (scale, pat)


def test_full_rate_random_blocks_only_bfp_truncation(orc):
    rng = np.random.default_rng(6)
    for it in range(3000):
        kind = it % 3
        if kind == 0:
            a = rng.standard_normal(16) * 10.0 ** rng.integers(-30, 30)
        elif kind == 1:  # dyadic polynomial block: exact at full rate
            r, c = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
            co = rng.integers(-64, 64, size=4)
            a = ((co[0] + co[1] * r + co[2] * c + co[3] * r * c).astype(np.float64) * 2.0 ** rng.integers(-8, 8)).reshape(16)
        else:
            a = rng.standard_normal(16) * np.exp(rng.uniform(-20, 20, size=16))
        a = a.astype(np.float32).astype(np.float64)
        _, _, _, vals = orc.decode_block(orc.encode_block(a, FULL_RATE), FULL_RATE)
        assert (vals.reshape(16) == _bfp_truncate(a)).all(), it
        if kind == 1:
            assert (vals.reshape(16) == a).all()


def test_constants_exact_at_every_rate(orc):
    # a constant costs 9 header bits, <= 5 leading empty-plane tests and two bits per
    # plane below its top plane (27 planes at most): always within rate 8's 128 bits
    rng = np.random.default_rng(7)
    for _ in range(300):
        v = float(np.float32(rng.standard_normal() * 10.0 ** rng.integers(-20, 20)))
        for rate in range(8, 40, 4):
            _, _, _, vals = orc.decode_block(orc.encode_block(np.full(16, v), rate), rate)
            assert (vals.reshape(16) == _bfp_truncate(np.full(16, v))).all()


def _bits(words, nbits):
    out = []
    for b in range(nbits):
        out.append((int(words[b // 64]) >> (b % 64)) & 1)
    return out


def test_embedded_prefix_property(orc):
    # the rate-r stream of a block is the first 16r bits of its full-rate stream
    rng = np.random.default_rng(8)
    for _ in range(400):
        a = (rng.standard_normal(16) * np.exp(rng.uniform(-6, 6, size=16))).astype(np.float32)
        full = _bits(orc.encode_block(a, FULL_RATE), 16 * FULL_RATE)
        for rate in range(4, FULL_RATE, 4):
            w = orc.encode_block(a, rate)
            assert _bits(w, 16 * rate) == full[: 16 * rate]


def test_plane_coder_bit_budget(orc):
    rng = np.random.default_rng(9)
    for _ in range(2000):
        u = rng.integers(0, 2 ** 32, size=16, dtype=np.uint64) >> rng.integers(0, 32, size=16).astype(np.uint64)
        u = u.astype(np.uint32)
        maxbits = int(rng.integers(1, 600))
        w, used = orc.encode_planes(u, maxbits, 10)
        assert used <= maxbits
        dec, used2 = orc.decode_planes(w, maxbits)
        assert used2 == used
        if used < maxbits:  # the whole block fitted: lossless
            assert (dec == u).all()
        else:  # a prefix of the planes: decoded bits are a subset of the true bits
            assert ((dec & ~u) == 0).all()
    # the worst case fits in 569 bits
    # all ones: plane 31 spends a test and a bit on each of coefficients 0..14 and one
    # test on 15 (implied), 31 bits; planes 30..0 are 16 verbatim bits each
    u = np.full(16, 0xFFFFFFFF, dtype=np.uint32)
    _, used = orc.encode_planes(u, 10_000, 10)
    assert used == 31 + 31 * 16
    u = np.array([1 << 31] + [0] * 15, dtype=np.uint32)
    _, used = orc.encode_planes(u, 10_000, 10)
    assert used <= 569


def test_error_decreases_with_rate(orc):
    import workloads

    A = workloads.KernelMatrix(64, 8, 64, 0.3, 11).dense()
    errs = []
    for rate in (4, 8, 12, 16, 24, 32):
        D = orc.decode(orc.encode(A, orc.FMT_ZFP, rate))
        errs.append(np.abs(D - A).max())
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-7


# --------------------------------------------------------------------- blobs
def test_blob_layout_size_and_crc(orc):
    rng = np.random.default_rng(10)
    for (M, N, rate) in [(1, 1, 4), (5, 7, 8), (13, 4, 16), (64, 33, 12), (4, 4, 36)]:
        A = rng.standard_normal((M, N))
        blob = orc.encode(A, orc.FMT_ZFP, rate)
        assert len(blob) == 64 + math.ceil(M / 4) * math.ceil(N / 4) * 2 * rate
        assert blob[:4] == b"WZ1\x00"
        assert int.from_bytes(blob[40:44], "little") == zlib.crc32(blob[64:])
        assert int.from_bytes(blob[44:48], "little") == zlib.crc32(blob[:44])
        assert orc.parse(blob) == (1, rate, M, N)
        bad = bytearray(blob)
        bad[-1] ^= 0x10
        with pytest.raises(orc.OracleError):
            orc.parse(bytes(bad))
        D = orc.decode(blob)
        assert D.shape == (M, N)


def test_edge_blocks_replicate(orc):
    # a ragged matrix decodes the same as the replicated-padding matrix, cropped
    rng = np.random.default_rng(12)
    A = rng.standard_normal((6, 7))
    P = np.pad(A, ((0, 2), (0, 1)), mode="edge")
    Da = orc.decode(orc.encode(A, orc.FMT_ZFP, 16))
    Dp = orc.decode(orc.encode(P, orc.FMT_ZFP, 16))
    assert (Da == Dp[:6, :7]).all()


def test_rejects_nonfinite_and_range(orc):
    A = np.ones((4, 4))
    A[1, 1] = np.nan
    with pytest.raises(orc.OracleError):
        orc.encode(A)
    A[1, 1] = 2.0 ** 127
    with pytest.raises(orc.OracleError):
        orc.encode(A)


def test_crc_matches_zlib(orc):
    rng = np.random.default_rng(13)
    for n in (0, 1, 7, 64, 1000):
        b = rng.integers(0, 256, size=n, dtype=np.uint8).tobytes()
        assert orc.crc32(b) == zlib.crc32(b)
