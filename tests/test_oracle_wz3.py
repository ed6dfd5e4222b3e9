"""Pins of the oracle's fixed-accuracy reading (WZ3, the device format for
zfp's fixed-accuracy mode, Sec. 4.3): every decoded block within the tolerance
of its FP32 input, the shift the largest that achieves it, the field width the
smallest that holds it (the run's width the largest of its blocks), the bit
layout exactly WZ2's with the width chosen per run, at WZ2's own error a WZ3
block never costs more bits than WZ2's fixed rate, and hand-derived blocks, a
run and a whole matrix (tests/golden/wz3_blocks.txt) reproduced bit for bit."""
import numpy as np
import pytest


def _blocks(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        kind = k % 4
        if kind == 0:  # smooth: a plane plus a small bump
            i, j = np.mgrid[0:4, 0:4]
            b = 1.0 + 0.1 * i + 0.05 * j + 0.01 * rng.standard_normal((4, 4))
        elif kind == 1:
            b = rng.standard_normal((4, 4))
        elif kind == 2:
            b = rng.standard_normal((4, 4)) * 2.0 ** rng.integers(-40, 40)
        else:
            b = np.exp(-rng.random((4, 4)))  # all positive, like kernel entries
        out.append(b.astype(np.float32))
    return out


def _err(orc, words, W, a, lift):
    return float(np.abs(orc.wz3_decode_block(words, W, lift) - a.astype(np.float64)).max())


_F4 = np.array([[1, 1, 1, 1], [-2, -2, 2, 2], [-4, 4, 0, 0], [4, -4, -4, 4]], dtype=np.int64)


def _floor_shift(a, lift):
    """The smallest shift whose coefficients, rounded half to even, fit 31-bit fields --
    computed here from the definition with numpy (24 fraction bits, C = (4F) Q (4F)^T)."""
    a = a.astype(np.float64)
    nz = a[a != 0]
    if nz.size == 0:
        return 0
    emax = int(np.frexp(np.abs(nz))[1].max())
    q = np.trunc(np.ldexp(a, 24 - emax)).astype(np.int64)
    c = _F4 @ q @ _F4.T if lift else q
    for K in range(28):
        v = np.rint(np.ldexp(c.astype(np.float64), -K))
        if v.min() >= -(2.0**30) and v.max() <= 2.0**30 - 1:
            return K
    return 27


@pytest.mark.parametrize("lift", [True, False])
@pytest.mark.parametrize("p", [4, 8, 12, 16, 20])
def test_decoded_block_within_tolerance_when_reachable(orc, lift, p):
    for a in _blocks(24, p):
        tol = float(np.abs(a).max()) * 2.0**-p
        emax, K, v, need = orc.wz3_block(a, tol, lift)
        words, W = orc.wz3_encode_run(a[None], tol, lift)
        assert W == need
        err = _err(orc, words, W, a, lift)
        if err > tol:  # unreachable: the floor, the finest quantisation 31-bit fields hold
            assert K == _floor_shift(a, lift)
            w0, W0 = orc.wz3_encode_run(a[None], 0.0, lift)
            assert _err(orc, w0, W0, a, lift) == err
        else:
            assert err <= tol, (K, err, tol)


@pytest.mark.parametrize("lift", [True, False])
def test_shift_is_the_largest_and_width_the_smallest(orc, lift):
    for a in _blocks(40, 7):
        tol = float(np.abs(a).max()) * 2.0**-10
        emax, K, v, need = orc.wz3_block(a, tol, lift)
        # width: v fits in `need` bits, not in need - 1
        assert v.min() >= -(2 ** (need - 1)) and v.max() <= 2 ** (need - 1) - 1
        if need > 1:
            assert v.min() < -(2 ** (need - 2)) or v.max() > 2 ** (need - 2) - 1
        # shift: the block's own error at K is its tolerance's witness; any
        # tolerance below that error forces a smaller shift
        words, W = orc.wz3_encode_run(a[None], tol, lift)
        err = _err(orc, words, W, a, lift)
        if K > 0 and err > 0:
            _, K2, _, _ = orc.wz3_block(a, np.nextafter(err, 0.0), lift)
            assert K2 < K
        _, K3, _, _ = orc.wz3_block(a, err, lift)
        assert K3 >= K


@pytest.mark.parametrize("lift", [True, False])
@pytest.mark.parametrize("rate", [8, 12, 16, 20, 24])
def test_same_layout_as_wz2_and_never_more_bits_at_its_error(orc, lift, rate):
    W2 = orc.wz2_width(rate)
    for a in _blocks(16, rate):
        w2 = orc.wz2_encode_block(a, rate, lift)
        d2 = orc.wz2_decode_block(w2, rate, lift)
        # the layouts coincide: WZ2's words read as a WZ3 block of width W2
        assert np.array_equal(orc.wz3_decode_block(w2, W2, lift), d2)
        e2 = float(np.abs(d2 - a.astype(np.float64)).max())
        emax, K, v, need = orc.wz3_block(a, e2, lift)
        words, W = orc.wz3_encode_run(a[None], e2, lift)
        assert _err(orc, words, W, a, lift) <= e2
        assert orc.wz3_block_bytes(need) <= orc.wz3_block_bytes(W2) <= 2 * rate


def test_zero_blocks_and_exact_blocks(orc):
    z = np.zeros((4, 4), dtype=np.float32)
    emax, K, v, need = orc.wz3_block(z, 1e-3)
    assert need == 0 and (v == 0).all()
    words, W = orc.wz3_encode_run(z[None], 1e-3)
    assert W == 0 and words.size == 1 and words[0] == 0
    assert (orc.wz3_decode_block(words, W) == 0).all()
    # dyadic small integers: exact at tolerance 0
    rng = np.random.default_rng(3)
    for _ in range(20):
        a = (rng.integers(-8, 8, (4, 4)) * 2.0 ** int(rng.integers(-5, 5))).astype(np.float32)
        for lift in (True, False):
            words, W = orc.wz3_encode_run(a[None], 0.0, lift)
            assert np.array_equal(orc.wz3_decode_block(words, W, lift), a.astype(np.float64))


def test_run_width_bytes_and_monotonic_tolerance(orc):
    blocks = _blocks(32, 11)
    blocks[5] = np.zeros((4, 4), dtype=np.float32)
    tol = 1e-4
    words, W = orc.wz3_encode_run(np.stack(blocks), tol)
    needs = [orc.wz3_block(b, tol)[3] for b in blocks]
    assert W == max(needs)
    nb = orc.wz3_block_bytes(W)
    assert nb == 8 * ((13 + 16 * W + 63) // 64) and words.size * 8 == 32 * nb
    for k, b in enumerate(blocks):  # every block decodes from its own slot
        d = orc.wz3_decode_block(words[k * nb // 8:(k + 1) * nb // 8], W)
        assert np.array_equal(d, orc.wz3_decode_block(orc.wz3_encode_run(b[None], tol)[0], orc.wz3_block(b, tol)[3]))
    assert (orc.wz3_decode_block(words[5 * nb // 8:6 * nb // 8], W) == 0).all()
    for b in blocks[:12]:  # a larger tolerance never takes a smaller shift or a wider field
        prev_k, prev_w = -1, 99
        for t in (1e-8, 1e-6, 1e-4, 1e-2, 1.0):
            _, K, _, need = orc.wz3_block(b, t)
            assert K >= prev_k and need <= prev_w
            prev_k, prev_w = K, need


def test_errors(orc):
    a = np.ones((4, 4), dtype=np.float32)
    with pytest.raises(RuntimeError):
        orc.wz3_block(a, -1.0)
    bad = a.copy()
    bad[0, 0] = np.inf
    with pytest.raises(RuntimeError):
        orc.wz3_block(bad, 1e-3)
    with pytest.raises(RuntimeError):
        orc.wz3_encode_run(np.ones((33, 4, 4), dtype=np.float32), 1e-3)


def _kernel_matrix(M, N, seed):
    import workloads

    n = max(M, N)
    g = int(np.ceil(np.sqrt(n)))
    return workloads.KernelMatrix(n, g, n, 0.1, seed).dense()[:M, :N]


@pytest.mark.parametrize("M,N", [(130, 97), (64, 260), (5, 3)])
def test_matrix_layout_round_trip_and_index(orc, M, N):
    A = _kernel_matrix(M, N, M + N)
    A32 = A.astype(np.float32)
    for tol in (1e-2, 1e-4, 1e-6):
        blob = orc.wz3_encode(A, tol)
        D, t = orc.wz3_decode(blob)
        assert t == tol
        assert np.abs(D - A32.astype(np.float64)).max() <= tol
        # the index, read here from the bytes: u64 per run, offset | W << 56
        BM, BN = -(-M // 4), -(-N // 4)
        RB = -(-BN // 32)
        idx = np.frombuffer(blob[64 + 8:64 + 8 + 8 * BM * RB], dtype=np.uint64)
        off, off_expect = idx & np.uint64((1 << 56) - 1), 0
        Ws = (idx >> np.uint64(56)).astype(int)
        # padded blocks replicate the last valid row, then column
        Ap = np.pad(A32, ((0, 4 * BM - M), (0, 4 * BN - N)), mode="edge")
        for I in range(BM):
            for r in range(RB):
                k = I * RB + r
                assert int(off[k]) == off_expect
                blocks = [Ap[4 * I:4 * I + 4, 4 * J:4 * J + 4] for J in range(32 * r, min(BN, 32 * r + 32))]
                assert Ws[k] == max(orc.wz3_block(b, tol)[3] for b in blocks)
                # word-interleaved: word j of block b at byte 8 (j nb + b) of the run
                nb, nw = len(blocks), orc.wz3_block_bytes(Ws[k]) // 8
                words, W = orc.wz3_encode_run(np.stack(blocks), tol)
                assert W == Ws[k]
                start = 64 + 8 + 8 * BM * RB + int(off[k])
                run = np.frombuffer(blob[start:start + 8 * nb * nw], dtype=np.uint64)
                assert np.array_equal(run.reshape(nw, nb).T.reshape(-1), words)
                off_expect += len(blocks) * orc.wz3_block_bytes(Ws[k])
        assert len(blob) == 64 + 8 + 8 * BM * RB + off_expect


def test_matrix_bytes_fall_with_the_tolerance_and_corruption_is_caught(orc):
    A = _kernel_matrix(96, 96, 3)
    sizes = [len(orc.wz3_encode(A, t)) for t in (1e-7, 1e-5, 1e-3, 1e-1)]
    assert sizes == sorted(sizes, reverse=True)
    blob = bytearray(orc.wz3_encode(A, 1e-4))
    blob[200] ^= 1
    with pytest.raises(RuntimeError):
        orc.wz3_decode(bytes(blob))


@pytest.mark.parametrize("lift", [True, False])
def test_full_scale_checkerboard_stays_within_31_bit_fields(orc, lift):
    """A near-full-scale block whose signs follow the last lift row's pattern drives one
    lifted coefficient to about 2^32: 34-bit fields at K = 0.  The floor is then the
    smallest shift that fits 31 bits, the block keeps its 64 bytes, and a whole matrix of
    such blocks fits the size bound and decodes."""
    s = np.array([1.0, -1.0, -1.0, 1.0])
    a = (np.outer(s, s) * (1.0 - 2.0**-20)).astype(np.float32)
    a[0, 1] = np.float32(-(1.0 - 2.0**-20 - 3 * 2.0**-24))  # an odd fixed-point value: not exact above K = 0
    emax, K, v, need = orc.wz3_block(a, 0.0, lift)
    assert need <= 31 and K == _floor_shift(a, lift)
    if lift:
        assert K == 2  # about 2^32 needs two shifts to fit in 31 bits
    words, W = orc.wz3_encode_run(a[None], 0.0, lift)
    assert W == need and words.size * 8 == orc.wz3_block_bytes(W) <= 64
    d = orc.wz3_decode_block(words, W, lift)
    e_floor = float(np.abs(d - a.astype(np.float64)).max())
    assert e_floor <= 2.0 ** (K - 1) * 25 * 2.0 ** (emax - 30) + 2.0 ** (emax - 24)  # the WZ2 bound at K
    if not lift:  # the matrix layout takes the lift
        return
    A = np.tile(a.astype(np.float64), (2, 2))
    blob = orc.wz3_encode(A, 0.0)
    assert len(blob) <= orc.lib().orc_wz3_max_blob_size(8, 8)
    D, _ = orc.wz3_decode(blob)
    assert np.array_equal(D[:4, :4], d)


# ------------------------------------------------ hand-derived fixtures
def _golden_wz3():
    """Records of tests/golden/wz3_blocks.txt: {kind: [fields, ...]}."""
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "wz3_blocks.txt")
    out = {"block": [], "run": [], "matrix": []}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = [x.strip() for x in line.split("|")]
        out[f[0]].append(f[1:])
    return out


def _floats(s):
    return [float(v) for v in s.split()]


def _hex_words(s):
    return [int(v, 16) for v in s.split()]


def _golden_block_input(rec):
    """The 4x4 FP32 block of a block record (every row the same)."""
    return np.tile(np.array(_floats(rec[3]), dtype=np.float32), (4, 1))


@pytest.mark.parametrize("rec", _golden_wz3()["block"], ids=lambda r: r[0])
def test_wz3_hand_derived_blocks(orc, rec):
    name, lift, tol, _, K, W, words, dec = rec
    lift, tol = bool(int(lift)), float(tol)
    a = _golden_block_input(rec)
    emax, k, _, need = orc.wz3_block(a, tol, lift)
    assert (emax, k, need) == (1, int(K), int(W)), name
    got, w = orc.wz3_encode_run(a.reshape(1, 4, 4), tol, lift)
    assert w == int(W)
    assert [int(x) for x in got] == _hex_words(words), name
    want = np.tile(np.array(_floats(dec)), (4, 1))
    assert (orc.wz3_decode_block(got, w, lift) == want).all(), name


@pytest.mark.parametrize("rec", _golden_wz3()["run"], ids=lambda r: r[0])
def test_wz3_hand_derived_run(orc, rec):
    name, lift, tol, names, W, words = rec
    blocks = {r[0]: _golden_block_input(r) for r in _golden_wz3()["block"]}
    a = np.stack([blocks[n] for n in names.split()])
    got, w = orc.wz3_encode_run(a, float(tol), bool(int(lift)))
    assert w == int(W)
    assert [int(x) for x in got] == _hex_words(words), name


def golden_wz3_matrix(rec):
    """(A, expected blob) of a matrix record; the header follows the blob layout
    (magic, version 1, format 8, rate 0, M, N, stream bytes, CRC-32 of the stream
    and of the header's first 44 bytes, the rest zero), CRCs from zlib."""
    import struct
    import zlib

    name, tol, M, N, row, words = rec
    M, N = int(M), int(N)
    A = np.tile(np.array(_floats(row)), (M, 1))
    stream = b"".join(struct.pack("<Q", w) for w in _hex_words(words))
    assert struct.unpack("<d", stream[:8])[0] == float(tol)
    head = b"WZ1\0" + struct.pack("<IIIqqQI", 1, 8, 0, M, N, len(stream), zlib.crc32(stream))
    head += struct.pack("<I", zlib.crc32(head)) + bytes(16)
    return A, head + stream


@pytest.mark.parametrize("rec", _golden_wz3()["matrix"], ids=lambda r: r[0])
def test_wz3_hand_derived_matrix(orc, rec):
    A, want = golden_wz3_matrix(rec)
    blob = orc.wz3_encode(A, float(rec[1]))
    assert blob == want
    dec, tol = orc.wz3_decode(blob)
    assert tol == float(rec[1]) and (dec == A).all()
