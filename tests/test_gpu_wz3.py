"""The fixed-accuracy format (WZ3: the lifted blocks of Sec. 4.3 with a per-block
shift chosen for an absolute tolerance and one field width per run of 32 blocks)
on the GPU, through the C ABI, against the FP64 oracle.

  * whff_decompress equals the oracle's decode bit for bit (the integer inverse
    transform and the power-of-two scale are exact in FP64);
  * the fused decode + GEMV step (1 and 8 right-hand sides per pass; R = 3 and 11
    take several passes) and the state update against the oracle GEMV on the
    decoded matrix within relative L2 1e-6, for ragged shapes, bands split over
    many column ranges, tolerances from coarse (narrow fields) to 0 (fields wider
    than 23 bits) and matrices with all-zero runs;
  * row slits and time-sliced steps (row views that start at a later band);
  * a run index that points past the stream, or a width above 31, is refused at
    create time (WHFF_EFORMAT) before anything reaches the device.
"""
import zlib

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-6
HEADER = 64


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_1902_08018_gb300 as W

    W.library()
    return W, torch


def _matrix(M, N, seed):
    import workloads

    return workloads.RectKernelMatrix(M, N, 0.05, seed).dense()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


SHAPES = [(130, 97), (1037, 4001), (5, 3), (64, 30001), (2051, 260)]


@pytest.mark.parametrize("M,N", SHAPES)
@pytest.mark.parametrize("tol", [1e-2, 1e-5, 0.0])
def test_decompress_bit_exact(env, orc, M, N, tol):
    W, torch = env
    blob = W.whff_compress_accuracy(_matrix(M, N, M + N), tol)
    Ahat, t = orc.wz3_decode(blob.tobytes())
    assert t == tol
    with W.whff_create(blob, max_rhs=1) as h:
        out = torch.full((M, N + 3), float("nan"), dtype=torch.float64, device="cuda")
        h.decompress(out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    assert np.array_equal(got[:, :N], Ahat)
    assert np.isnan(got[:, N:]).all()  # nothing written past column N


@pytest.mark.parametrize("M,N", SHAPES)
@pytest.mark.parametrize("tol", [1e-2, 1e-5, 0.0])
@pytest.mark.parametrize("R", [1, 3, 8, 11])
def test_step_against_oracle(env, orc, M, N, tol, R):
    W, torch = env
    blob = W.whff_compress_accuracy(_matrix(M, N, 3 * M + N), tol)
    Ahat, _ = orc.wz3_decode(blob.tobytes())
    rng = np.random.default_rng(R * 1000 + M)
    X = rng.standard_normal((R, N)).astype(np.float32)
    with W.whff_create(blob, max_rhs=R) as h:
        s = torch.full((M,), 0.5, dtype=torch.float64, device="cuda")
        y = torch.full((R, M), float("nan"), dtype=torch.float64, device="cuda")
        h.step(torch.from_numpy(X).cuda(), y, s, 0.9)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        got, st = y.cpu().numpy(), s.cpu().numpy()
    s_ref = np.full(M, 0.5)
    for r in range(R):  # the state takes the columns in order (Sec. 2.1, one control step per column)
        ref = orc.gemv64(Ahat, X[r].astype(np.float64))
        assert _rel(got[r], ref) <= TOL, (r, _rel(got[r], ref))
        s_ref = orc.state_update(s_ref, ref, 0.9)
    assert _rel(st, s_ref) <= TOL


def test_zero_runs_and_mixed_widths(env, orc):
    """Whole runs of zero blocks (width 0: 8 zero bytes per block), runs of tiny values next to
    runs of large ones (widths from 1 to 31 in one band)."""
    W, torch = env
    M, N = 256, 4096
    A = _matrix(M, N, 77)
    A[:, 128:640] = 0.0  # runs 1..4 of every band: all zero
    A[:64, 1024:2048] *= 1e-9  # below the tolerance: narrow fields
    A[64:128, 2048:3072] *= 1e6  # far above it: wide fields
    tol = 1e-7
    blob = W.whff_compress_accuracy(A, tol)
    Ahat, _ = orc.wz3_decode(blob.tobytes())
    RB = (N // 4 + 31) // 32
    widths = np.frombuffer(blob.tobytes()[HEADER + 8:HEADER + 8 + 8 * (M // 4) * RB], dtype=np.uint64) >> 56
    assert widths.min() == 0 and widths.max() > 23, (widths.min(), widths.max())
    X = np.random.default_rng(5).standard_normal(N).astype(np.float32)
    ref = orc.gemv64(Ahat, X.astype(np.float64))
    mag = orc.gemv64(np.abs(Ahat), np.abs(X.astype(np.float64)))
    with W.whff_create(blob, max_rhs=1) as h:
        y = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
        h.step(torch.from_numpy(X).cuda(), y)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
    # per row: FP32 products of FP64-exact fields, pairs added in TwoSum
    assert (np.abs(got - ref) <= 1e-6 * mag + 1e-300).all()


def test_slits_and_time_slices(env, orc):
    W, torch = env
    M, N = 1030, 5001
    blob = W.whff_compress_accuracy(_matrix(M, N, 11), 1e-6)
    Ahat, _ = orc.wz3_decode(blob.tobytes())
    X = np.random.default_rng(11).standard_normal(N).astype(np.float32)
    x = torch.from_numpy(X).cuda()
    full = orc.gemv64(Ahat, X.astype(np.float64))
    mag = orc.gemv64(np.abs(Ahat), np.abs(X.astype(np.float64)))
    with W.whff_create(blob, max_rhs=1) as h:
        for row0, nrows in ((0, M), (4, 37), (512, 300), (1028, 2)):
            y = torch.full((nrows,), float("nan"), dtype=torch.float64, device="cuda")
            h.step_rows(row0, nrows, x, y)
            torch.cuda.synchronize()
            got = y.cpu().numpy()
            assert (np.abs(got - full[row0:row0 + nrows]) <= 1e-6 * mag[row0:row0 + nrows]).all(), (row0, nrows)
        with pytest.raises(W.WhffError):
            h.step_rows(2, 8, x, torch.zeros(8, dtype=torch.float64, device="cuda"))  # not a band start
        for slice_rows in (4, 128, 1000):
            h.slice_rows = slice_rows
            y = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
            s = torch.zeros(M, dtype=torch.float64, device="cuda")
            h.step(x, y, s, 0.99)
            torch.cuda.synchronize()
            got = y.cpu().numpy()
            assert (np.abs(got - full) <= 1e-6 * mag).all(), slice_rows
            assert np.array_equal(s.cpu().numpy(), got)  # s = 0.99 * 0 + y
        assert h.sync_status() == 0


def _reseal(blob):
    """Recompute the stream and header CRCs of a blob whose stream was edited."""
    b = bytearray(blob)
    n = int.from_bytes(b[32:40], "little")
    b[40:44] = zlib.crc32(bytes(b[HEADER:HEADER + n])).to_bytes(4, "little")
    b[44:48] = zlib.crc32(bytes(b[:44])).to_bytes(4, "little")
    return np.frombuffer(bytes(b), dtype=np.uint8)


def test_create_refuses_bad_run_index(env):
    W, torch = env
    M, N = 64, 300  # BN = 75: 3 runs per band
    blob = W.whff_compress_accuracy(_matrix(M, N, 3), 1e-6)
    assert _reseal(blob).tobytes() == blob.tobytes()  # the CRCs are zlib's CRC-32
    with W.whff_create(blob, max_rhs=1):
        pass
    idx0 = HEADER + 8  # run 0 of band 0
    for patch in ("width", "offset"):
        b = bytearray(blob.tobytes())
        e = int.from_bytes(b[idx0:idx0 + 8], "little")
        if patch == "width":
            e = (e & ((1 << 56) - 1)) | (40 << 56)
        else:
            e = (e & ~((1 << 56) - 1)) | (len(b) * 8)
        b[idx0:idx0 + 8] = e.to_bytes(8, "little")
        with pytest.raises(W.WhffError) as err:
            W.whff_create(_reseal(b), max_rhs=1)
        assert err.value.code == -5, patch


def test_host_resident_graph_and_server(env, orc):
    """The same fixed-accuracy bytes read over the host link give the device-resident
    results bit for bit; a captured step replays to the result of whff_step; a WZ3 model
    served among WZ2 ones gets what it gets alone and the oracle's state."""
    W, torch = env
    M, N = 700, 1300
    blob = W.whff_compress_accuracy(_matrix(M, N, 21), 1e-6)
    Ahat, _ = orc.wz3_decode(blob.tobytes())
    rng = np.random.default_rng(21)
    X = torch.from_numpy(rng.standard_normal((9, N)).astype(np.float32)).cuda()
    out = []
    for host in (False, True):
        with W.whff_create(blob, max_rhs=16, host_resident=host) as h:
            y = torch.zeros((9, M), dtype=torch.float64, device="cuda")
            s = torch.full((M,), 0.5, dtype=torch.float64, device="cuda")
            h.step(X, y, s, 0.9)  # a pass of 8 columns, then one of 1
            ys = torch.zeros((2, 256), dtype=torch.float64, device="cuda")
            h.step_rows(256, 256, X[:2], ys)
            D = torch.zeros((M, N), dtype=torch.float64, device="cuda")
            h.decompress(D)
            torch.cuda.synchronize()
            assert h.sync_status() == 0
            out.append((y, s, ys, D))
    for u, v in zip(*out):
        assert torch.equal(u, v)
    assert np.array_equal(out[0][3].cpu().numpy(), Ahat)

    with W.whff_create(blob, max_rhs=8) as h:
        x = torch.zeros((2, N), dtype=torch.float32, device="cuda")
        y = torch.zeros((2, M), dtype=torch.float64, device="cuda")
        s = torch.zeros(M, dtype=torch.float64, device="cuda")
        y_ref = torch.zeros((2, M), dtype=torch.float64, device="cuda")
        s_ref = torch.zeros(M, dtype=torch.float64, device="cuda")
        with W.whff_graph_create(h, x, y, s, 0.9) as g:
            for _ in range(3):
                xv = torch.from_numpy(rng.standard_normal((2, N)).astype(np.float32)).cuda()
                x.copy_(xv)
                g.launch()
                h.step(xv, y_ref, s_ref, 0.9)
                torch.cuda.synchronize()
                assert torch.equal(y, y_ref) and torch.equal(s, s_ref)

    import workloads

    other = W.whff_compress(workloads.RectKernelMatrix(512, 512, 0.05, 22).dense(), 5, 16)
    handles = [W.whff_create(blob, max_rhs=8), W.whff_create(other, max_rhs=8)]
    n_req = 60
    model = rng.integers(0, 2, size=n_req)
    arrival = np.sort(np.repeat(np.arange(n_req // 10) * 2e-3, 10))
    xs = [rng.standard_normal(handles[m].N).astype(np.float32) for m in model]
    with W.Server(hbm_budget=8 << 30, max_batch=8, nstreams=2) as srv:
        ids = [srv.add_model(h, decay=0.95) for h in handles]
        lat, bat, ys = srv.run(model, arrival, xs, want_y=True)
        state0 = srv.read_state(ids[0])
    s = np.zeros(M)
    for i in range(n_req):
        if model[i] != 0:
            continue
        ref = orc.gemv64(Ahat, xs[i].astype(np.float64))
        assert _rel(ys[i], ref) <= TOL, i
        s = orc.state_update(s, ref, 0.95)
    assert _rel(state0, s) <= TOL
    for h in handles:
        h.destroy()


def test_batch_refuses_fixed_accuracy(env):
    W, torch = env
    h = W.whff_create(W.whff_compress_accuracy(_matrix(64, 64, 5), 1e-4), max_rhs=1)
    with pytest.raises(W.WhffError):
        W.Batch([h], [1])
    h.destroy()
