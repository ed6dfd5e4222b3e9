"""GPU parity of the library against the CPU oracle, through the C ABI.

  * whff_decompress (Sec. 5.2's decode) is bit-identical to the oracle decoder;
  * whff_step (Sec. 4.4 GEMV on the decoded matrix, Sec. 2.1 state update) is
    within relative L2 error 1e-6 of the FP64 oracle GEMV on the same decoded
    matrix, per right-hand side;
  * A*e_j reproduces decoded column j exactly; multi-RHS columns equal the
    single-RHS results bit for bit; steps are deterministic.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-6  # relative L2, per right-hand side


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_1902_08018_gb300 as W

    W.library()
    return W, torch


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def smooth(M, N, seed=3, length=0.15):
    import workloads

    n = max(M, N)
    g = int(np.ceil(np.sqrt(n)))
    return workloads.KernelMatrix(n, g, n, length, seed).rows(0, M)[:, :N]


def run_step(W, torch, h, X, state=None, decay=0.99):
    """X: (R, N) float32 numpy -> y (R, M) float64 numpy."""
    x = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    y = torch.zeros((X.shape[0], h.M), dtype=torch.float64, device="cuda")
    h.step(x, y, state, decay)
    torch.cuda.synchronize()
    return y.cpu().numpy()


CASES = [
    (1, 8, 64, 64),
    (1, 12, 130, 97),
    (1, 16, 257, 513),
    (1, 16, 16, 20000),   # wide: split-K
    (1, 8, 3001, 40),     # tall
    (1, 16, 1, 5),
    (2, 0, 300, 301),
    (3, 0, 257, 500),
    (4, 0, 129, 1000),
    (4, 0, 24, 9000),     # wide scaled: split-K
    (5, 16, 257, 513),
    (5, 8, 130, 97),
    (5, 24, 16, 20000),   # wide WZ2: split-K
    (6, 12, 301, 300),
    (7, 0, 300, 301),     # FP32 storage, the paper's mixed precision
    (7, 0, 16, 20000),    # wide FP32
    (7, 0, 3001, 40),     # tall FP32
    (2, 0, 3001, 378),    # tall BF16: 8-lane groups per band
    (4, 0, 2050, 700),    # tall FP8
    (6, 20, 3001, 40),
]


@pytest.mark.parametrize("fmt,rate,M,N", CASES)
def test_decompress_bit_exact(env, orc, fmt, rate, M, N):
    W, torch = env
    A = smooth(M, N)
    blob = W.whff_compress(A, fmt, rate or 16)
    ref = orc.decode(blob.tobytes())
    with W.whff_create(blob) as h:
        out = torch.full((M, N + 3), np.nan, dtype=torch.float64, device="cuda")
        h.decompress(out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    assert (got[:, :N].view(np.uint64) == ref.view(np.uint64)).all()
    assert np.isnan(got[:, N:]).all()  # nothing written past N


@pytest.mark.parametrize("fmt,rate", [(1, 4), (1, 20), (1, 36), (1, 64), (5, 12), (5, 20), (6, 8), (6, 24)])
def test_decompress_other_rates(env, orc, fmt, rate):
    W, torch = env
    rng = np.random.default_rng(rate)
    A = rng.standard_normal((37, 41)) * np.exp(rng.uniform(-8, 8, size=(37, 41)))
    blob = W.whff_compress(A, fmt, rate)
    ref = orc.decode(blob.tobytes())
    with W.whff_create(blob) as h:
        out = torch.empty((37, 41), dtype=torch.float64, device="cuda")
        h.decompress(out)
        torch.cuda.synchronize()
        assert (out.cpu().numpy().view(np.uint64) == ref.view(np.uint64)).all()


@pytest.mark.parametrize("fmt,rate,M,N", CASES)
@pytest.mark.parametrize("R", [1, 3, 8])
def test_step_matches_fp64_oracle(env, orc, fmt, rate, M, N, R):
    W, torch = env
    A = smooth(M, N)
    blob = W.whff_compress(A, fmt, rate or 16)
    Ahat = orc.decode(blob.tobytes())
    rng = np.random.default_rng(M * 7 + N + R)
    X = rng.standard_normal((R, N)).astype(np.float32)  # FP32-exact inputs isolate the kernel error
    ref = orc.gemv64(Ahat, X.T.astype(np.float64))
    with W.whff_create(blob) as h:
        Y = run_step(W, torch, h, X)
        Y1 = run_step(W, torch, h, X[:1])
        Y2 = run_step(W, torch, h, X)
        same_engine = R < h.crossover  # R columns and 1 column both on the CUDA cores
    for r in range(R):
        assert rel_l2(Y[r], ref[:, r]) <= TOL, (r, rel_l2(Y[r], ref[:, r]))
    assert (Y == Y2).all()  # deterministic
    if same_engine:
        assert (Y1[0] == Y[0]).all()  # the first column does not depend on the others
    else:  # a tensor-core pass: another rounding of the same sum
        assert rel_l2(Y1[0], Y[0]) <= TOL


def test_unit_vectors_give_decoded_columns(env, orc):
    W, torch = env
    A = smooth(133, 70)
    blob = W.whff_compress(A, 1, 16)
    Ahat = orc.decode(blob.tobytes())
    cols = [0, 1, 33, 69]
    X = np.zeros((len(cols), 70), dtype=np.float32)
    for k, j in enumerate(cols):
        X[k, j] = 1.0
    with W.whff_create(blob) as h:
        Y = run_step(W, torch, h, X)
    for k, j in enumerate(cols):
        assert (Y[k] == Ahat[:, j]).all()


def test_state_update_over_steps(env, orc):
    W, torch = env
    A = smooth(260, 260)
    blob = W.whff_compress(A, 1, 16)
    Ahat = orc.decode(blob.tobytes())
    rng = np.random.default_rng(5)
    s_dev = torch.zeros(260, dtype=torch.float64, device="cuda")
    s_ref = np.zeros(260)
    with W.whff_create(blob) as h:
        for k in range(6):
            R = 1 + (k % 3)
            X = rng.standard_normal((R, 260)).astype(np.float32)
            run_step(W, torch, h, X, state=s_dev, decay=0.99)
            s_ref = orc.state_update(s_ref, orc.gemv64(Ahat, X.T.astype(np.float64)), 0.99)
    assert rel_l2(s_dev.cpu().numpy(), s_ref) <= TOL


def test_state_with_split_k(env, orc):
    W, torch = env
    A = smooth(12, 30000)
    blob = W.whff_compress(A, 1, 12)
    Ahat = orc.decode(blob.tobytes())
    X = np.random.default_rng(6).standard_normal((3, 30000)).astype(np.float32)
    s_dev = torch.ones(12, dtype=torch.float64, device="cuda")
    with W.whff_create(blob) as h:
        Y = run_step(W, torch, h, X, state=s_dev, decay=0.5)
    ref = orc.gemv64(Ahat, X.T.astype(np.float64))
    s_ref = orc.state_update(np.ones(12), ref, 0.5)
    assert rel_l2(Y.T, ref) <= TOL
    assert rel_l2(s_dev.cpu().numpy(), s_ref) <= TOL


def test_fp64_input_rounding_within_tolerance(env, orc):
    # the GPU consumes x rounded to FP32 (Sec. 4.4: single-precision inputs); against the
    # oracle on the unrounded FP64 x the error still stays inside the tolerance
    W, torch = env
    A = smooth(512, 512)
    blob = W.whff_compress(A, 1, 16)
    Ahat = orc.decode(blob.tobytes())
    x64 = np.random.default_rng(7).standard_normal(512)
    with W.whff_create(blob) as h:
        Y = run_step(W, torch, h, x64[None, :].astype(np.float32))
    assert rel_l2(Y[0], orc.gemv64(Ahat, x64)) <= TOL


def test_step_host_equals_step(env):
    W, torch = env
    A = smooth(300, 200)
    blob = W.whff_compress(A, 1, 16)
    X = np.random.default_rng(8).standard_normal((2, 200)).astype(np.float32)
    with W.whff_create(blob) as h:
        Yd = run_step(W, torch, h, X)
        xh = torch.from_numpy(X).pin_memory()
        yh = torch.zeros((2, 300), dtype=torch.float64).pin_memory()
        h.step_host(xh.numpy(), yh.numpy())
        torch.cuda.synchronize()
        assert (yh.numpy() == Yd).all()


def test_linearity(env):
    W, torch = env
    A = smooth(200, 200)
    blob = W.whff_compress(A, 1, 8)
    rng = np.random.default_rng(9)
    x1 = rng.standard_normal(200).astype(np.float32)
    x2 = rng.standard_normal(200).astype(np.float32)
    with W.whff_create(blob) as h:
        Y = run_step(W, torch, h, np.stack([x1, x2, x1 + x2]))
    assert rel_l2(Y[2], Y[0] + Y[1]) <= 1e-6


def test_invalid_arguments(env):
    W, torch = env
    blob = W.whff_compress(np.ones((8, 8)), 1, 16)
    with W.whff_create(blob, max_rhs=2) as h:
        x = torch.zeros((3, 8), dtype=torch.float32, device="cuda")
        y = torch.zeros((3, 8), dtype=torch.float64, device="cuda")
        with pytest.raises(W.WhffError):
            h.step(x, y)  # R > max_rhs
        with pytest.raises(W.WhffError):
            h.step(torch.zeros(7, dtype=torch.float32, device="cuda"), y[0])  # x too short
        assert h.sync_status() == 0


@pytest.mark.parametrize("M,N", [(378, 9000), (5000, 378), (1000, 1000)])
def test_fp32_storage_follows_the_papers_mixed_precision(env, orc, M, N):
    """FP32 storage: every product rounded to FP32, the products summed
    without loss (Sec. 4.4).  Against the paper's rule (FP32 products, FP64
    running sum, y rounded to FP32): |y - y_mp| <= half an FP32 ulp of y_mp
    (its final rounding) + 1e-13 * sum_j |p_j| (the two sums' orders)."""
    W, torch = env
    A = smooth(M, N)
    x = np.random.default_rng(M + N).standard_normal(N).astype(np.float32)
    blob = W.whff_compress(A, W.FMT_FP32)
    y_mp = orc.gemv_mp(A, x.astype(np.float64)).astype(np.float64)
    P = np.abs(A.astype(np.float32) * x[None, :]).astype(np.float64).sum(axis=1)
    with W.whff_create(blob) as h:
        (y,) = run_step(W, torch, h, x[None, :])
    ulp = np.spacing(np.abs(y_mp).astype(np.float32)).astype(np.float64)
    assert (np.abs(y - y_mp) <= 0.5 * ulp + 1e-13 * P).all()
