"""Slit steps (Sec. 2.1, divide and conquer: C_slit is a block of rows of the
resident C_field) through the C ABI: every slit's y within relative L2 1e-6
of the FP64 oracle GEMV on the same rows of the decoded matrix (slits of 64
rows and more), every entry within 1e-6 of its row's sum_j |a_ij x_j| (any
slit: a few rows can cancel more than a whole vector), its own state
following the oracle recursion, for block and scaled formats, CUDA-core and
tensor-core passes; misaligned or out-of-range slits are refused."""
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


def _matrix(M, N, seed=5):
    import workloads

    n = max(M, N)
    return workloads.KernelMatrix(n, int(np.ceil(np.sqrt(n))), n, 0.1, seed).rows(0, M)[:, :N]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("fmt,rate", [(1, 16), (5, 16), (6, 12), (2, 0), (7, 0)])
@pytest.mark.parametrize("R", [1, 3, 8])
def test_slits_match_the_oracle_rows(env, orc, fmt, rate, R):
    W, torch = env
    M, N = 1030, 2500
    blob = W.whff_compress(_matrix(M, N), fmt, rate or 16)
    Ahat = orc.decode(blob.tobytes())
    X = np.random.default_rng(fmt * 10 + R).standard_normal((R, N)).astype(np.float32)
    x = torch.from_numpy(X).cuda()
    blocked = fmt in (1, 5, 6)
    slits = [(0, M), (256, 256), (768, M - 768), (128, 3)] + ([(4, 1), (1000, 30)] if blocked else [])
    with W.whff_create(blob, max_rhs=8) as h:
        for row0, nrows in slits:
            y = torch.zeros((R, nrows), dtype=torch.float64, device="cuda")
            s = torch.full((nrows,), 0.5, dtype=torch.float64, device="cuda")
            h.step_rows(row0, nrows, x, y, s, 0.9)
            torch.cuda.synchronize()
            assert h.sync_status() == 0
            rows = Ahat[row0:row0 + nrows]
            ref = orc.gemv64(rows, X.T.astype(np.float64))
            mag = orc.gemv64(np.abs(rows), np.abs(X.T.astype(np.float64)))  # sum_j |a_ij x_j|
            Y = y.cpu().numpy()
            for r in range(R):
                assert (np.abs(Y[r] - ref[:, r]) <= TOL * mag[:, r]).all(), (row0, nrows, r)
                if nrows >= 64:
                    assert _rel(Y[r], ref[:, r]) <= TOL, (row0, nrows, r)
            s_ref = orc.state_update(np.full(nrows, 0.5), ref, 0.9)
            s_mag = orc.state_update(np.full(nrows, 0.5), mag, 0.9)
            assert (np.abs(s.cpu().numpy() - s_ref) <= TOL * s_mag).all(), (row0, nrows)


def test_slit_arguments_are_checked(env):
    W, torch = env
    M, N = 300, 200
    for fmt, bad_row0 in ((5, 2), (2, 64)):
        blob = W.whff_compress(_matrix(M, N), fmt, 16)
        with W.whff_create(blob, max_rhs=2) as h:
            x = torch.zeros(N, dtype=torch.float32, device="cuda")
            y = torch.zeros(16, dtype=torch.float64, device="cuda")
            with pytest.raises(W.WhffError):
                h.step_rows(bad_row0, 16, x, y)  # not on a band / scale-tile boundary
            with pytest.raises(W.WhffError):
                h.step_rows(256 if fmt == 2 else 296, 64, x, torch.zeros(64, dtype=torch.float64, device="cuda"))
            h.step_rows(0, 16, x, y)  # a valid slit still works
            torch.cuda.synchronize()
            assert (y.cpu().numpy() == 0).all()


@pytest.mark.parametrize("fmt,rate", [(5, 16), (1, 12), (7, 0)])
def test_time_sliced_step_is_its_slits(env, orc, fmt, rate):
    """With slice_rows set, whff_step runs the pass as consecutive slits: its
    y and state equal those of the slit steps bit for bit, meet the bar
    against the oracle, and a graph captured afterwards replays the same."""
    W, torch = env
    M, N, R = 1100, 1500, 3
    blob = W.whff_compress(_matrix(M, N, 9), fmt, rate or 16)
    Ahat = orc.decode(blob.tobytes())
    X = np.random.default_rng(fmt).standard_normal((R, N)).astype(np.float32)
    x = torch.from_numpy(X).cuda()
    ref = orc.gemv64(Ahat, X.T.astype(np.float64))
    slice_rows = 256 if fmt == 7 else 300
    with W.whff_create(blob, max_rhs=4) as h:
        assert h.slice_rows == 0
        h.slice_rows = slice_rows
        y = torch.zeros((R, M), dtype=torch.float64, device="cuda")
        s = torch.full((M,), 0.5, dtype=torch.float64, device="cuda")
        h.step(x, y, s, 0.9)
        y_sl = torch.zeros_like(y)
        s_sl = torch.full((M,), 0.5, dtype=torch.float64, device="cuda")
        for r0 in range(0, M, slice_rows):
            n = min(slice_rows, M - r0)
            ys = torch.zeros((R, n), dtype=torch.float64, device="cuda")
            ss = s_sl[r0:r0 + n].clone()
            h.step_rows(r0, n, x, ys, ss, 0.9)
            y_sl[:, r0:r0 + n] = ys
            s_sl[r0:r0 + n] = ss
        g = W.whff_graph_create(h, x, (yg := torch.zeros_like(y)))
        g.launch()
        torch.cuda.synchronize()
        assert torch.equal(y, y_sl) and torch.equal(s, s_sl) and torch.equal(yg, y)
        Y = y.cpu().numpy()
        for r in range(R):
            assert _rel(Y[r], ref[:, r]) <= TOL
        s_ref = orc.state_update(np.full(M, 0.5), ref, 0.9)
        assert _rel(s.cpu().numpy(), s_ref) <= TOL
        g.destroy()
        h.slice_rows = 0
        with pytest.raises(W.WhffError):
            h.slice_rows = 6 if fmt != 7 else 64  # not on a band / scale-tile boundary
