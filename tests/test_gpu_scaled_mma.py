"""Tensor-core (tcgen05) passes for the scaled formats (BF16, FP16, FP8 E4M3
with 128 x 128 FP32 tile scales), through the C ABI: every column within
relative L2 1e-6 of the FP64 oracle GEMV on the decoded matrix, for ragged
shapes (rows past a 128-row tile, columns past a 64-column stage and past the
stored row length), split columns, R that mixes tensor-core and CUDA-core
passes, row views and time slices; the carried state follows the oracle
recursion in column order."""
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


def _matrix(M, N, seed, length=0.1):
    import workloads

    n = max(M, N)
    g = int(np.ceil(np.sqrt(n)))
    return workloads.KernelMatrix(n, g, n, length, seed).dense()[:M, :N]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(W, torch, h, X, state=None, decay=0.95):
    x = torch.from_numpy(X).cuda()
    y = torch.zeros((X.shape[0], h.M), dtype=torch.float64, device="cuda")
    h.step(x, y, state, decay)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    return y.cpu().numpy()


@pytest.mark.parametrize("fmt", [2, 3, 4])
@pytest.mark.parametrize("M,N,R", [
    (128, 64, 16),      # one tile, one stage
    (300, 1000, 32),    # ragged rows and columns, several stages and scale tiles
    (129, 2001, 35),    # 32 on tensor cores + 2 + 1 on CUDA cores; N past the stored row
    (2050, 700, 20),    # many tiles, CTA ranges crossing tiles
    (64, 20000, 32),    # wide: a tile split between CTAs (segments)
    (5000, 330, 8),     # tall
])
def test_scaled_tensor_core_passes_match_oracle(env, orc, fmt, M, N, R):
    W, torch = env
    A = _matrix(M, N, M + 3 * N + fmt)
    blob = W.whff_compress(A, fmt, 0)
    Ahat = orc.decode(blob.tobytes())
    X = np.random.default_rng(R + fmt).standard_normal((R, N)).astype(np.float32)
    ref = orc.gemv64(Ahat, X.T.astype(np.float64))
    with W.whff_create(blob, max_rhs=64) as h:
        assert h.crossover == 4
        s = torch.full((M,), 1.0, dtype=torch.float64, device="cuda")
        Y = _run(W, torch, h, X, s, 0.95)
        S = s.cpu().numpy()
    for r in range(R):
        assert _rel(Y[r], ref[:, r]) <= TOL, (r, _rel(Y[r], ref[:, r]))
    s_ref = orc.state_update(np.ones(M), ref, 0.95)
    assert _rel(S, s_ref) <= TOL


@pytest.mark.parametrize("fmt", [2, 4])
def test_scaled_engines_agree(env, orc, fmt):
    """The same columns on the tensor cores and on the CUDA cores: both meet the
    bar against the oracle (two roundings of one sum)."""
    W, torch = env
    M, N, R = 700, 900, 8
    blob = W.whff_compress(_matrix(M, N, 41), fmt, 0)
    Ahat = orc.decode(blob.tobytes())
    X = np.random.default_rng(5).standard_normal((R, N)).astype(np.float32)
    ref = orc.gemv64(Ahat, X.T.astype(np.float64))
    with W.whff_create(blob, max_rhs=R) as h:
        Yt = _run(W, torch, h, X)
        h.crossover = 33
        Yc = _run(W, torch, h, X)
        h.crossover = 2
        Y2 = _run(W, torch, h, X[:2])
    for r in range(R):
        assert _rel(Yt[r], ref[:, r]) <= TOL, r
        assert _rel(Yc[r], ref[:, r]) <= TOL, r
    for r in range(2):
        assert _rel(Y2[r], ref[:, r]) <= TOL, r


@pytest.mark.parametrize("fmt", [2, 3])
def test_scaled_row_views_and_slices_on_tensor_cores(env, orc, fmt):
    """A slit of rows (on a 128-row scale tile boundary) and time-sliced steps
    run their tensor-core passes on the view's rows only."""
    W, torch = env
    M, N, R = 1000, 600, 16
    blob = W.whff_compress(_matrix(M, N, 77), fmt, 0)
    Ahat = orc.decode(blob.tobytes())
    X = np.random.default_rng(8).standard_normal((R, N)).astype(np.float32)
    ref = orc.gemv64(Ahat, X.T.astype(np.float64))
    with W.whff_create(blob, max_rhs=R) as h:
        row0, nrows = 256, 500
        x = torch.from_numpy(X).cuda()
        y = torch.zeros((R, nrows), dtype=torch.float64, device="cuda")
        h.step_rows(row0, nrows, x, y)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        Yv = y.cpu().numpy()
        h.slice_rows = 384
        Ys = _run(W, torch, h, X)
    for r in range(R):
        assert _rel(Yv[r], ref[row0:row0 + nrows, r]) <= TOL, r
        assert _rel(Ys[r], ref[:, r]) <= TOL, r


@pytest.mark.parametrize("host_resident", [False, True])
def test_fp16_pass_over_wide_column_ranges(env, orc, host_resident):
    """FP16 storage on the TMA-fed pass scales each column of x by a power of two before
    splitting it into FP16 pieces (and the register-fed pass of a host-resident handle
    does not): columns of very different magnitudes, a column with a wide range inside
    it and an all-zero column all meet the bar; the zero column gives exact zeros."""
    W, torch = env
    M, N = 700, 1300
    blob = W.whff_compress(_matrix(M, N, 31), 3, 0)
    Ahat = orc.decode(blob.tobytes())
    rng = np.random.default_rng(31)
    X = rng.standard_normal((8, N)).astype(np.float32)
    X[1] *= 1e-20
    X[2] *= 1e20
    X[3] = 0.0
    X[4, : N // 2] *= 1e-6
    X[4, N // 2:] *= 1e3
    X[5] = np.float32(65504.0) * 4  # above the FP16 maximum before scaling
    X[6, ::2] = 0.0
    with W.whff_create(blob, max_rhs=8, host_resident=host_resident) as h:
        assert h.crossover <= 8
        y = torch.full((8, M), float("nan"), dtype=torch.float64, device="cuda")
        h.step(torch.from_numpy(X).cuda(), y)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        Y = y.cpu().numpy()
    for r in range(8):
        ref = orc.gemv64(Ahat, X[r].astype(np.float64))
        if r == 3:
            assert (Y[r] == 0.0).all()
        else:
            assert _rel(Y[r], ref) <= TOL, (r, _rel(Y[r], ref))
