"""The allocation-free step (whff_step_noalloc) against the handle-based step.

whff_step_noalloc serves callers that cannot call cudaMalloc (fixed-memory
real-time controllers, code inside a private memory pool): they pass the
compressed stream, x, y and the state in memory they own, and the split-K
partials go to a static device array.  This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-6  # relative L2, as in the other parity tests


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("rate,M,N,R", [(12, 24, 30000, 1), (16, 40, 20000, 4), (8, 2000, 2000, 2)])
def test_noalloc_matches_step_on_two_calls(rate, M, N, R):
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_1902_08018_gb300 as W
    import workloads

    g = int(np.ceil(np.sqrt(max(M, N))))
    A = workloads.KernelMatrix(max(M, N), g, max(M, N), 0.1, 77).dense()[:M, :N]
    blob = W.whff_compress(A, W.FMT_ZFP, rate)
    stream_dev = torch.from_numpy(blob[64:].copy()).cuda()  # caller-owned device copy of the stream
    rng = np.random.default_rng(rate + R)
    with W.whff_create(blob) as h:
        for call in range(2):
            X = torch.from_numpy(rng.standard_normal((R, N)).astype(np.float32)).cuda()
            y_ref = torch.zeros((R, M), dtype=torch.float64, device="cuda")
            s_ref = torch.full((M,), 0.5, dtype=torch.float64, device="cuda")
            h.step(X, y_ref, s_ref, 0.9)
            y = torch.full((R, M), float("nan"), dtype=torch.float64, device="cuda")
            s = torch.full((M,), 0.5, dtype=torch.float64, device="cuda")
            W.whff_step_noalloc(stream_dev, rate, M, N, X, y, s, 0.9)
            torch.cuda.synchronize()
            for r in range(R):
                assert _rel(y[r].cpu().numpy(), y_ref[r].cpu().numpy()) <= TOL, (call, r)
            assert _rel(s.cpu().numpy(), s_ref.cpu().numpy()) <= TOL, call


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
