"""The allocation-free step (whff_step_noalloc) against the CPU oracle.

whff_step_noalloc serves callers that cannot call cudaMalloc (fixed-memory
real-time controllers, code inside a private memory pool): they pass the
compressed stream, x, y and the state in memory they own, and the split-K
partials go to a static device array.  Its y and state are checked against
the FP64 oracle GEMV and state recursion on the oracle's decode of the same
blob, on two calls in a row (the second reuses the array the first one left
behind), and against the handle-based step.  This file is collected last so
that a run stopping at the first failure has already run every other test; it
also passes on its own in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-6  # relative L2, as in the other parity tests


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# (rate, M, N, R, with state): the first three split the columns (partials in the
# static array), the last two do not (ksplit 1: N <= 252 leaves one split per band)
CASES = [(12, 24, 30000, 1, True), (16, 40, 20000, 4, True), (8, 2000, 2000, 2, True), (16, 301, 200, 1, False),
         (12, 1000, 252, 8, True)]


@pytest.mark.parametrize("rate,M,N,R,with_state", CASES)
def test_noalloc_matches_oracle_on_two_calls(orc, rate, M, N, R, with_state):
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_1902_08018_gb300 as W
    import workloads

    g = int(np.ceil(np.sqrt(max(M, N))))
    A = workloads.KernelMatrix(max(M, N), g, max(M, N), 0.1, 77).dense()[:M, :N]
    blob = W.whff_compress(A, W.FMT_ZFP, rate)
    Ahat = orc.decode(blob.tobytes())
    stream_dev = torch.from_numpy(blob[64:].copy()).cuda()  # caller-owned device copy of the stream
    rng = np.random.default_rng(rate + R)
    s_ref = np.full(M, 0.5)
    s = torch.full((M,), 0.5, dtype=torch.float64, device="cuda") if with_state else None
    with W.whff_create(blob) as h:
        for call in range(2):
            X = rng.standard_normal((R, N)).astype(np.float32)
            Xd = torch.from_numpy(X).cuda()
            y = torch.full((R, M), float("nan"), dtype=torch.float64, device="cuda")
            W.whff_step_noalloc(stream_dev, rate, M, N, Xd, y, s, 0.9)
            y_h = torch.zeros((R, M), dtype=torch.float64, device="cuda")
            h.step(Xd, y_h)
            torch.cuda.synchronize()
            ref = orc.gemv64(Ahat, X.T.astype(np.float64))
            Y, Yh = y.cpu().numpy(), y_h.cpu().numpy()
            for r in range(R):
                assert _rel(Y[r], ref[:, r]) <= TOL, (call, r, _rel(Y[r], ref[:, r]))
                assert _rel(Y[r], Yh[r]) <= TOL, (call, r)
            if with_state:
                s_ref = orc.state_update(s_ref, ref, 0.9)
                assert _rel(s.cpu().numpy(), s_ref) <= TOL, call


def test_noalloc_rejects_bad_requests():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_1902_08018_gb300 as W

    stream_dev = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    x = torch.zeros((3, 16), dtype=torch.float32, device="cuda")
    y = torch.zeros((3, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(W.WhffError):  # R = 3 is not a supported pass width
        W.whff_step_noalloc(stream_dev, 16, 16, 16, x, y)
    with pytest.raises(W.WhffError):  # rate 20 is not built for the fused step
        W.whff_step_noalloc(stream_dev, 20, 16, 16, x[:1], y[:1])
    with pytest.raises(W.WhffError):  # 16 x 16 at rate 16 needs 512 bytes: 511 is short
        W.whff_step_noalloc(stream_dev[:511], 16, 16, 16, x[:1], y[:1])
