"""Tensor-core (tcgen05) passes for many right-hand sides on WZ2 matrices,
through the C ABI: every column within relative L2 1e-6 of the FP64 oracle
GEMV on the decoded matrix, for ragged shapes, split columns and R that mixes
tensor-core (>= 4 columns by default) and CUDA-core passes; the carried state follows
the oracle recursion in column order."""
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


@pytest.mark.parametrize("fmt,rate,M,N,R", [
    (5, 16, 128, 64, 16),      # one tile, one stage
    (5, 16, 260, 1000, 32),    # ragged rows and columns, several stages
    (6, 12, 300, 3001, 17),
    (5, 8, 1500, 1200, 9),
    (5, 16, 900, 1000, 35),    # 32 on tensor cores + 2 + 1 on CUDA cores
    (5, 24, 64, 20000, 32),    # wide: split columns
    (6, 20, 2050, 700, 43),    # 32 on tensor cores + 11 on tensor cores
    (5, 16, 3000, 5000, 24),   # several stages per CTA, CTA ranges crossing tiles
    (6, 8, 4100, 9000, 16),
])
def test_tensor_core_passes_match_oracle(env, orc, fmt, rate, M, N, R):
    W, torch = env
    A = _matrix(M, N, M + N)
    blob = W.whff_compress(A, fmt, rate)
    Ahat = orc.decode(blob.tobytes())
    rng = np.random.default_rng(R)
    X = rng.standard_normal((R, N)).astype(np.float32)
    ref = orc.gemv64(Ahat, X.T.astype(np.float64))
    with W.whff_create(blob, max_rhs=64) as h:
        x = torch.from_numpy(X).cuda()
        y = torch.zeros((R, M), dtype=torch.float64, device="cuda")
        s = torch.full((M,), 1.0, dtype=torch.float64, device="cuda")
        h.step(x, y, s, 0.95)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        Y = y.cpu().numpy()
    for r in range(R):
        assert _rel(Y[r], ref[:, r]) <= TOL, (r, _rel(Y[r], ref[:, r]))
    s_ref = orc.state_update(np.ones(M), ref, 0.95)
    assert _rel(s.cpu().numpy(), s_ref) <= TOL


@pytest.mark.parametrize("R", [2, 5, 8])
def test_low_crossover_matches_oracle(env, orc, R):
    """With the crossover lowered, passes of 2..8 columns run on the tensor
    cores and meet the same bar."""
    W, torch = env
    M, N = 1100, 2300
    blob = W.whff_compress(_matrix(M, N, 11), 5, 16)
    Ahat = orc.decode(blob.tobytes())
    X = np.random.default_rng(R + 100).standard_normal((R, N)).astype(np.float32)
    ref = orc.gemv64(Ahat, X.T.astype(np.float64))
    with W.whff_create(blob, max_rhs=8) as h:
        assert h.crossover == 4
        h.crossover = 2
        assert h.crossover == 2
        x = torch.from_numpy(X).cuda()
        y = torch.zeros((R, M), dtype=torch.float64, device="cuda")
        h.step(x, y)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        Y = y.cpu().numpy()
        for r in range(R):
            assert _rel(Y[r], ref[:, r]) <= TOL, r
        h.crossover = 33  # CUDA cores only: another rounding, the same bar
        y2 = torch.zeros_like(y)
        h.step(x, y2)
        torch.cuda.synchronize()
        Y2 = y2.cpu().numpy()
        for r in range(R):
            assert _rel(Y2[r], ref[:, r]) <= TOL, r


def test_crossover_needs_tensor_core_workspace(env):
    W, torch = env
    blob = W.whff_compress(_matrix(64, 64, 3), 5, 16)
    with W.whff_create(blob, max_rhs=1) as h:
        assert h.crossover == 33
        with pytest.raises(W.WhffError):
            h.crossover = 4
        h.crossover = 33
    with W.whff_create(blob, max_rhs=4) as h:
        for bad in (1, 34):
            with pytest.raises(W.WhffError):
                h.crossover = bad
    with W.whff_create(W.whff_compress(_matrix(64, 64, 3), 1, 16), max_rhs=16) as h:
        assert h.crossover == 33  # WZ1 has no tensor-core passes


@pytest.mark.parametrize("fmt", [5, 6])
def test_huge_blocks_take_the_exact_scale(env, orc, fmt):
    """Blocks near the top of the exponent range (|a| ~ 2^120) decode through
    the explicit multiply instead of the exponent trick; results are the same
    bar, relative to their magnitude."""
    W, torch = env
    M, N, R = 200, 300, 16
    A = _matrix(M, N, 5) * 2.0 ** {5: 118, 6: 121}[fmt]  # some blocks with E + K > 258, sums below 2^126
    A[:100] *= 2.0**-200  # tiny rows in the same matrix take the fast path
    blob = W.whff_compress(A, fmt, 16)
    Ahat = orc.decode(blob.tobytes())
    X = np.random.default_rng(9).standard_normal((R, N)).astype(np.float32)
    ref = orc.gemv64(Ahat, X.T.astype(np.float64))
    with W.whff_create(blob, max_rhs=R) as h:
        x = torch.from_numpy(X).cuda()
        y = torch.zeros((R, M), dtype=torch.float64, device="cuda")
        h.step(x, y)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        Y = y.cpu().numpy()
    for r in range(R):
        for rows in (slice(0, 100), slice(100, M)):
            assert _rel(Y[r, rows], ref[rows, r]) <= TOL, (r, rows)
