"""The scan's two levels of divide and conquer (Sec. 2.1; Fig. whff_algo) through the C ABI.

  * One instantiated slit graph moved over a field: for every offset the replay's y
    rows and the slit's state rows against the FP64 oracle on the same rows of the
    decoded matrix (relative L2 1e-6), and bit for bit against whff_step_rows on the
    same slit; block and scaled formats, CUDA-core and tensor-core passes.
  * Fields streamed over the host link into two resident slots (Sec. 4.3, Fig.
    compression_cost): every slit step on a streamed field is bit-identical to the same
    step on a handle made resident by whff_create, while the next field's copy runs on
    another stream; mismatching blobs are refused.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-6


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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("fmt,rate,R", [(5, 16, 1), (6, 12, 2), (1, 16, 1), (5, 8, 8), (2, 0, 1), (2, 0, 8),
                                        (7, 0, 1)])
def test_one_graph_moves_over_every_slit(env, orc, fmt, rate, R):
    W, torch = env
    M, N, nrows = 1408, 3000, 378 if fmt in (1, 5, 6) else 256
    blob = W.whff_compress(_matrix(M, N, 11 + fmt), fmt, rate or 16)
    Ahat = orc.decode(blob.tobytes())
    rng = np.random.default_rng(fmt * 100 + R)
    align = 4 if fmt in (1, 5, 6) else 128
    offsets = [0, align * 3, (M - nrows) // align * align, align * 7, M // 2 // align * align, align]
    with W.whff_create(blob, max_rhs=8) as h:
        x = torch.zeros((R, N), dtype=torch.float32, device="cuda")
        y = torch.full((R, M), float("nan"), dtype=torch.float64, device="cuda")
        s = torch.zeros(M, dtype=torch.float64, device="cuda")
        s_ref = np.zeros(M)
        g = W.whff_graph_create_rows(h, offsets[0], nrows, x, y, s, 0.9)
        for k, row0 in enumerate(offsets):
            X = rng.standard_normal((R, N)).astype(np.float32)
            x.copy_(torch.from_numpy(X))
            g.set_rows(row0)
            s_before = s[row0:row0 + nrows].clone()
            g.launch()
            torch.cuda.synchronize()
            rows = slice(row0, row0 + nrows)
            ref = orc.gemv64(Ahat[rows], X.T.astype(np.float64))
            Y = y.cpu().numpy()[:, rows]
            for r in range(R):
                assert _rel(Y[r], ref[:, r]) <= TOL, (k, r, _rel(Y[r], ref[:, r]))
            s_ref[rows] = orc.state_update(s_ref[rows], ref, 0.9)
            assert _rel(s.cpu().numpy()[rows], s_ref[rows]) <= TOL, k
            # the same slit through the direct call: bit for bit
            y2 = torch.zeros((R, nrows), dtype=torch.float64, device="cuda")
            s2 = s_before.clone()
            h.step_rows(row0, nrows, x, y2, s2, 0.9)
            torch.cuda.synchronize()
            assert (y2.cpu().numpy() == Y).all(), k
            assert (s2.cpu().numpy() == s.cpu().numpy()[rows]).all(), k
        assert h.sync_status() == 0
        g.destroy()


def test_slit_graph_refuses_bad_offsets(env):
    W, torch = env
    blob = W.whff_compress(_matrix(64, 64, 3), 5, 16)
    with W.whff_create(blob, max_rhs=1) as h:
        x = torch.zeros(64, dtype=torch.float32, device="cuda")
        y = torch.zeros(64, dtype=torch.float64, device="cuda")
        g = W.whff_graph_create_rows(h, 0, 16, x, y)
        with pytest.raises(W.WhffError):
            g.set_rows(2)  # not on a 4-row band
        with pytest.raises(W.WhffError):
            g.set_rows(52)  # past the matrix
        other = W.whff_create(W.whff_compress(_matrix(64, 60, 4), 5, 16), max_rhs=1)
        with pytest.raises(W.WhffError):
            g.set_rows(0, other)  # another shape
        other.destroy()
        with pytest.raises(W.WhffError):
            W.whff_graph_create_rows(h, 0, 65, x, y)
        g.destroy()


@pytest.mark.parametrize("fmt,rate", [(5, 16), (1, 12), (4, 0)])
def test_streamed_fields_equal_resident_handles(env, orc, fmt, rate):
    W, torch = env
    L, N, nrows, steps = 520, 4000, 128, 5  # field rows, columns, slit rows, slit steps per field
    nfields = 4
    blobs = [W.whff_compress(_matrix(L, N, 40 + k), fmt, rate or 16) for k in range(nfields)]
    pinned = []
    for b in blobs:
        t = torch.from_numpy(b.copy()).pin_memory()
        pinned.append(t.numpy())
    rng = np.random.default_rng(fmt)
    X = rng.standard_normal((nfields * steps, N)).astype(np.float32)
    align = 4 if fmt in (1, 5, 6) else 128
    offs = [min(L - nrows, (L - nrows) * j // (steps - 1)) // align * align for j in range(steps)]
    compute = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    got = []
    with W.Fields(fmt, rate, L, N, nbuf=2, max_rhs=1) as F:
        x = torch.zeros(N, dtype=torch.float32, device="cuda")
        y = torch.zeros(L, dtype=torch.float64, device="cuda")
        s = torch.zeros(L, dtype=torch.float64, device="cuda")
        F.load(0, pinned[0], copy)
        g = None
        for f in range(nfields):
            if f + 1 < nfields:
                F.load((f + 1) % 2, pinned[f + 1], copy)  # the next field crosses the link meanwhile
            h = F.acquire(f % 2, compute)
            for j, r0 in enumerate(offs):
                x.copy_(torch.from_numpy(X[f * steps + j]).cuda())
                if g is None:
                    g = W.whff_graph_create_rows(h, r0, nrows, x, y, s, 0.99)
                else:
                    g.set_rows(r0, h)
                g.launch(compute)
                got.append(y[r0:r0 + nrows].clone())
            F.release(f % 2, compute)
        torch.cuda.synchronize()
        g.destroy()
    got = [v.cpu().numpy() for v in got]
    s_stream = s.cpu().numpy()
    # the same slits on resident handles
    s2 = torch.zeros(L, dtype=torch.float64, device="cuda")
    k = 0
    for f in range(nfields):
        with W.whff_create(blobs[f], max_rhs=1) as h:
            Ahat = orc.decode(blobs[f].tobytes())
            for j, r0 in enumerate(offs):
                xv = torch.from_numpy(X[f * steps + j]).cuda()
                y2 = torch.zeros(nrows, dtype=torch.float64, device="cuda")
                h.step_rows(r0, nrows, xv, y2, s2[r0:r0 + nrows], 0.99)
                torch.cuda.synchronize()
                assert (y2.cpu().numpy() == got[k]).all(), (f, j)
                ref = orc.gemv64(Ahat[r0:r0 + nrows], X[f * steps + j].astype(np.float64))
                assert _rel(got[k], ref) <= TOL
                k += 1
    assert (s2.cpu().numpy() == s_stream).all()


def test_fields_refuse_mismatching_blobs(env):
    W, torch = env
    with W.Fields(5, 16, 64, 64, nbuf=2) as F:
        with pytest.raises(W.WhffError):
            F.load(0, W.whff_compress(_matrix(64, 60, 1), 5, 16))  # another shape
        with pytest.raises(W.WhffError):
            F.load(0, W.whff_compress(_matrix(64, 64, 1), 5, 12))  # another rate
        with pytest.raises(W.WhffError):
            F.load(2, W.whff_compress(_matrix(64, 64, 1), 5, 16))  # no slot 2
        bad = W.whff_compress(_matrix(64, 64, 1), 5, 16)
        bad[10] ^= 1  # header CRC
        with pytest.raises(W.WhffError):
            F.load(0, bad)
    with W.Fields(5, 16, 64, 64, nbuf=2, verify_crc=True) as F:
        bad = W.whff_compress(_matrix(64, 64, 1), 5, 16)
        bad[100] ^= 1  # stream CRC, checked on request
        with pytest.raises(W.WhffError):
            F.load(0, bad)
