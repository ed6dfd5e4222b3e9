"""Pins of the oracle's WZ2 (fixed-allocation) coder: hand-derived streams,
exact round trips where the coefficients fit (which pins the linear lift pair
(2G)(4F) = 8I), the closed form of the no-transform variant, the quantisation
error bound implied by the stored shift K, minimality of K, and the size rule."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "wz2_blocks.txt")


def _golden():
    """(name, rate, lift, the 16 values, expected leading words): one value fills the
    block, four are every row of it."""
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, rate, lift, val, words = [f.strip() for f in line.split("|")]
        v = [float(t) for t in val.split()]
        block = np.full(16, v[0]) if len(v) == 1 else np.tile(np.array(v), 4)
        rows.append((name, int(rate), int(lift), block, [int(t, 16) for t in words.split()]))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: r[0])
def test_wz2_hand_derived_streams(orc, row):
    name, rate, lift, block, words = row
    w = orc.wz2_encode_block(block, rate, lift)
    assert [int(x) for x in w[: len(words)]] == words
    assert (orc.wz2_decode_block(w, rate, lift).reshape(16) == block).all()


def _emax(a):
    nz = a[a != 0]
    return max(math.frexp(float(v))[1] for v in nz) if nz.size else None


def _fields(words, rate):
    W = (16 * rate - 13) // 16
    bits = 0
    for i, x in enumerate(words):
        bits |= int(x) << (64 * i)
    E = bits & 0xFF
    K = (bits >> 8) & 31
    v = [((bits >> (13 + W * k)) & ((1 << W) - 1)) - (1 << (W - 1)) for k in range(16)]
    return E, K, v, W


def test_wz2_roundtrip_exact_when_coefficients_fit(orc):
    # blocks of 11-bit integers times a power of two: q = m * 2^13, so every
    # coefficient is a multiple of 2^13 and the shift K chosen at rate 24 (W = 23)
    # rounds nothing; decoding must return the input exactly, which only holds if
    # the decoder's (2G)/8 is exactly the inverse of the encoder's 4F
    rng = np.random.default_rng(50)
    for _ in range(2000):
        m = rng.integers(-(2 ** 10), 2 ** 10, size=16).astype(np.float64)
        m[0] = 2 ** 10  # fix emax so that q = m * 2^(24-emax) stays small
        a = m * 2.0 ** int(rng.integers(-30, 30))
        for lift in (0, 1):
            w = orc.wz2_encode_block(a, 24, lift)
            assert (orc.wz2_decode_block(w, 24, lift).reshape(16) == a).all()


def test_wz2_bfp_closed_form_and_k_minimal(orc):
    rng = np.random.default_rng(51)
    for rate in (8, 12, 16, 20, 24):
        for _ in range(300):
            a = (rng.standard_normal(16) * np.exp(rng.uniform(-5, 5, 16))).astype(np.float32).astype(np.float64)
            w = orc.wz2_encode_block(a, rate, 0)
            E, K, v, W = _fields(w, rate)
            emax = _emax(a)
            assert E == emax + 127
            q = np.trunc(a * 2.0 ** (24 - emax))
            want = np.array([np.round(x / 2.0 ** K) for x in q])  # numpy rounds half to even
            assert (np.array(v) == want).all()
            lo, hi = -(2 ** (W - 1)), 2 ** (W - 1) - 1
            if K > 0:  # one shift less would not fit
                prev = np.array([np.round(x / 2.0 ** (K - 1)) for x in q])
                assert prev.min() < lo or prev.max() > hi
            dec = orc.wz2_decode_block(w, rate, 0).reshape(16)
            assert (dec == want * 2.0 ** (K + emax - 24)).all()


def test_wz2_lift_error_bound(orc):
    # every coefficient is off by at most 2^(K-1); the inverse (2G).(2G)^T/64 has
    # row sums of |entries| <= 5, so each value is off by <= 25 * 2^(K-1) * 2^(emax-30),
    # plus the truncation to 24 fraction bits
    rng = np.random.default_rng(52)
    for rate in (8, 12, 16, 20, 24):
        for _ in range(300):
            a = (rng.standard_normal(16) * np.exp(rng.uniform(-3, 3, 16))).astype(np.float32).astype(np.float64)
            w = orc.wz2_encode_block(a, rate, 1)
            E, K, v, W = _fields(w, rate)
            emax = E - 127
            dec = orc.wz2_decode_block(w, rate, 1).reshape(16)
            bound = 25 * 2.0 ** (K - 1) * 2.0 ** (emax - 30) + 2.0 ** (emax - 24)
            assert np.abs(dec - a).max() <= bound


def test_wz2_blob_and_error_by_rate(orc):
    import workloads

    A = workloads.KernelMatrix(64, 8, 64, 0.3, 11).dense()[:61, :59]
    for fmt in (orc.FMT_FIXED_LIFT, orc.FMT_FIXED_BFP):
        errs = []
        for rate in (8, 12, 16, 20, 24):
            blob = orc.encode(A, fmt, rate)
            assert len(blob) == 64 + 16 * 15 * 2 * rate
            errs.append(np.abs(orc.decode(blob) - A).max())
        assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    with pytest.raises(orc.OracleError):
        orc.encode(A, orc.FMT_FIXED_LIFT, 4)  # W = 3 too narrow: rates 8..24 only
    with pytest.raises(orc.OracleError):
        orc.encode(A, orc.FMT_FIXED_LIFT, 28)
