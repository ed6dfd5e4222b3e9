"""Batched persistent launch over uneven matrices and the launch-shape tuner,
through the C ABI: every matrix of a batch gets y within relative L2 1e-6 of
the FP64 oracle GEMV on its decoded matrix, its state follows the oracle's
recursion in column order, and tuned shapes keep the results."""
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

    n = max(M, N)
    g = int(np.ceil(np.sqrt(n)))
    return workloads.KernelMatrix(n, g, n, 0.1, seed).dense()[:M, :N]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("fmt,rate", [(5, 12), (6, 16)])
def test_batch_matches_oracle(env, orc, fmt, rate):
    W, torch = env
    shapes = [(130, 97), (1500, 1400), (16, 6000), (777, 777), (2000, 300), (64, 64)]
    Rs = [1, 3, 8, 13, 4, 32]
    rng = np.random.default_rng(fmt * 10 + rate)
    handles, blobs, X, Y, S = [], [], [], [], []
    for k, ((M, N), R) in enumerate(zip(shapes, Rs)):
        blob = W.whff_compress(_matrix(M, N, 100 + k), fmt, rate)
        blobs.append(blob)
        handles.append(W.whff_create(blob, max_rhs=32))
        X.append(torch.from_numpy(rng.standard_normal((R, N)).astype(np.float32)).cuda())
        Y.append(torch.zeros((R, M), dtype=torch.float64, device="cuda"))
        S.append(torch.full((M,), 0.25, dtype=torch.float64, device="cuda"))
    with W.Batch(handles, Rs) as b:
        b.step(X, Y, S, decay=0.9)
        torch.cuda.synchronize()
        for k, (M, N) in enumerate(shapes):
            Ahat = orc.decode(blobs[k].tobytes())
            ref = orc.gemv64(Ahat, X[k].cpu().numpy().T.astype(np.float64))
            Yk = Y[k].cpu().numpy()
            for r in range(Rs[k]):
                assert _rel(Yk[r], ref[:, r]) <= TOL, (k, r)
            s_ref = orc.state_update(np.full(M, 0.25), ref, 0.9)
            assert _rel(S[k].cpu().numpy(), s_ref) <= TOL, k
        # a second step reuses the plan: results must be reproducible
        Y2 = [torch.zeros_like(y) for y in Y]
        b.step(X, Y2, None)
        torch.cuda.synchronize()
        for k in range(len(shapes)):
            assert torch.equal(Y2[k], Y[k])
    for h in handles:
        h.destroy()


@pytest.mark.parametrize("fmt", [2, 3, 4, 7])
def test_scaled_batch_matches_oracle(env, orc, fmt):
    """One scaled format per batch (BF16, FP16, FP8, FP32; 128 x 128 scale tiles cut
    by ragged shapes): CUDA-core column groups for few columns, the matrices' own
    tensor-core passes at or above their crossover (not for FP32), states in order."""
    W, torch = env
    shapes = [(130, 97), (1500, 1400), (16, 6000), (777, 777), (2000, 300), (64, 64)]
    Rs = [1, 3, 8, 13, 4, 32]
    rng = np.random.default_rng(fmt)
    handles, blobs, X, Y, S = [], [], [], [], []
    for k, ((M, N), R) in enumerate(zip(shapes, Rs)):
        blob = W.whff_compress(_matrix(M, N, 200 + k), fmt, 0)
        blobs.append(blob)
        handles.append(W.whff_create(blob, max_rhs=32))
        X.append(torch.from_numpy(rng.standard_normal((R, N)).astype(np.float32)).cuda())
        Y.append(torch.full((R, M), float("nan"), dtype=torch.float64, device="cuda"))
        S.append(torch.full((M,), 0.25, dtype=torch.float64, device="cuda"))
    with W.Batch(handles, Rs) as b:
        b.step(X, Y, S, decay=0.9)
        torch.cuda.synchronize()
        for k, (M, N) in enumerate(shapes):
            Ahat = orc.decode(blobs[k].tobytes())
            ref = orc.gemv64(Ahat, X[k].cpu().numpy().T.astype(np.float64))
            Yk = Y[k].cpu().numpy()
            for r in range(Rs[k]):
                assert _rel(Yk[r], ref[:, r]) <= TOL, (k, r)
            s_ref = orc.state_update(np.full(M, 0.25), ref, 0.9)
            assert _rel(S[k].cpu().numpy(), s_ref) <= TOL, k
        Y2 = [torch.zeros_like(y) for y in Y]
        b.step(X, Y2, None)  # the plan is reused: the same bits
        torch.cuda.synchronize()
        for k in range(len(shapes)):
            assert torch.equal(Y2[k], Y[k])
    for h in handles:
        assert h.sync_status() == 0
        h.destroy()


def test_batch_rejects_mixed_formats_and_wide_requests(env):
    W, torch = env
    h1 = W.whff_create(W.whff_compress(_matrix(64, 64, 1), 5, 12))
    h2 = W.whff_create(W.whff_compress(_matrix(64, 64, 2), 5, 16))
    with pytest.raises(W.WhffError):
        W.Batch([h1, h2], [1, 1])
    h3 = W.whff_create(W.whff_compress(_matrix(64, 64, 3), 2, 0))  # BF16
    h4 = W.whff_create(W.whff_compress(_matrix(64, 64, 4), 3, 0))  # FP16
    for pair in ([h3, h4], [h3, h1], [h1, h3]):
        with pytest.raises(W.WhffError):
            W.Batch(pair, [1, 1])
    h5 = W.whff_create(W.whff_compress(_matrix(64, 64, 5), 2, 0), max_rhs=4)  # BF16, workspaces for 4
    with pytest.raises(W.WhffError):
        W.Batch([h5], [5])  # more columns than the handle's max_rhs
    for h in (h1, h2, h3, h4, h5):
        h.destroy()


def test_tuner_keeps_results(env, orc, tmp_path):
    W, torch = env
    A = _matrix(3000, 3000, 7)
    blob = W.whff_compress(A, 5, 16)
    Ahat = orc.decode(blob.tobytes())
    x = torch.from_numpy(np.random.default_rng(8).standard_normal(3000).astype(np.float32)).cuda()
    ref = orc.gemv64(Ahat, x.cpu().numpy().astype(np.float64))
    cache = str(tmp_path / "tune.json")
    with W.whff_create(blob) as h:
        rec = h.tune(iters=3, cache=cache)
        assert rec["unroll"] in (2, 4, 8) and rec["ctas_per_sm"] >= 1 and rec["fold"] in (0, 1, 2, 3, 4, 5)
        assert not rec["cached"]
        y = torch.zeros(3000, dtype=torch.float64, device="cuda")
        h.step(x, y)
        torch.cuda.synchronize()
        assert _rel(y.cpu().numpy(), ref) <= TOL
        y0 = y.clone()
        c, f = rec["ctas_per_sm"], rec["fold"]
        fb = f & 3  # the fold without the bulk-staging flag (4)
        for cc in (c, 1):  # blocks in flight (registers or bulk-staged) change the schedule, not the arithmetic
            ys = []
            for u, ff in ([(2, fb), (4, fb), (8, fb), (2, fb | 4)] if fb < 2 else [(2, fb)]):
                try:
                    h.set_config(u, cc, ff)
                except W.WhffError:  # more CTAs per SM than this kernel keeps resident
                    continue
                h.step(x, y)
                torch.cuda.synchronize()
                ys.append(y.clone())
            assert ys and all(torch.equal(v, ys[0]) for v in ys)
            if cc == c:
                assert torch.equal(ys[0], y0)
        for u, c2, r2 in ((2, 1, 0), (2, 1, 1), (2, c, 2), (2, c, 3), (4, c, 1 - (f & 1))):  # other partitions / folds
            h.set_config(u, c2, r2)
            assert h.config() == (u, c2, r2)
            h.step(x, y)
            torch.cuda.synchronize()
            assert _rel(y.cpu().numpy(), ref) <= TOL
        with pytest.raises(W.WhffError):
            h.set_config(1, 1)
        with pytest.raises(W.WhffError):
            h.set_config(2, 1, 8)
        with pytest.raises(W.WhffError):
            h.set_config(4, 1, 2)  # lane groups take unroll 2
        with pytest.raises(W.WhffError):
            h.set_config(8, 1, 2)
        with pytest.raises(W.WhffError):
            h.set_config(16, 1, 0)
    with W.whff_create(blob) as h2:
        rec2 = h2.tune(iters=3, cache=cache)
        assert rec2["cached"] and rec2["unroll"] == rec["unroll"]
        assert h2.config() == (rec["unroll"], rec["ctas_per_sm"], rec["fold"])


def test_batch_tensor_core_groups_match_oracle(env, orc):
    """Matrices with R at or above the crossover share one persistent
    tensor-core launch per width class; CTA ranges cross from one matrix to
    the next, and a matrix with R = 40 has passes in both classes."""
    W, torch = env
    shapes = [(1000, 2200), (3100, 900), (260, 5000), (2048, 2048), (700, 1300)]
    Rs = [5, 16, 20, 40, 32]
    rng = np.random.default_rng(77)
    handles, blobs, X, Y, S = [], [], [], [], []
    for k, ((M, N), R) in enumerate(zip(shapes, Rs)):
        blob = W.whff_compress(_matrix(M, N, 200 + k), 5, 16)
        blobs.append(blob)
        handles.append(W.whff_create(blob, max_rhs=64))
        X.append(torch.from_numpy(rng.standard_normal((R, N)).astype(np.float32)).cuda())
        Y.append(torch.zeros((R, M), dtype=torch.float64, device="cuda"))
        S.append(torch.full((M,), -0.5, dtype=torch.float64, device="cuda"))
    with W.Batch(handles, Rs) as b:
        b.step(X, Y, S, decay=0.95)
        torch.cuda.synchronize()
        for h in handles:
            assert h.sync_status() == 0
        for k, (M, N) in enumerate(shapes):
            Ahat = orc.decode(blobs[k].tobytes())
            ref = orc.gemv64(Ahat, X[k].cpu().numpy().T.astype(np.float64))
            Yk = Y[k].cpu().numpy()
            for r in range(Rs[k]):
                assert _rel(Yk[r], ref[:, r]) <= TOL, (k, r)
            s_ref = orc.state_update(np.full(M, -0.5), ref, 0.95)
            assert _rel(S[k].cpu().numpy(), s_ref) <= TOL, k
        Y2 = [torch.zeros_like(y) for y in Y]
        b.step(X, Y2, None)
        torch.cuda.synchronize()
        for k in range(len(shapes)):
            assert torch.equal(Y2[k], Y[k])
    for h in handles:
        h.destroy()
