"""Failure detection on the GPU without a fault: the tensor-core passes bound every
device-side wait.  With the in-loop limit set to zero polls every such wait gives up
at once, the kernel records WHFF_ETIMEOUT in the handle's status word, its CTAs stop
at their next barrier, wait with the full limit for the MMAs and copies they started,
free their tensor memory and return.  The context stays usable: with the default limit
restored, the next step on the same handle matches the FP64 oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fmt,rate", [(5, 16), (2, 0)])
def test_expired_waits_report_a_timeout_and_leave_the_context_usable(orc, fmt, rate):
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_1902_08018_gb300 as W
    import workloads

    n, R = 256, 8
    A = workloads.KernelMatrix(n, 16, n, 0.1, 31).dense()
    blob = W.whff_compress(A, fmt, rate or 16)
    Ahat = orc.decode(blob.tobytes())
    X = np.random.default_rng(31).standard_normal((R, n)).astype(np.float32)
    x = torch.from_numpy(X).cuda()
    with W.whff_create(blob, max_rhs=8) as h:
        assert h.crossover <= R  # the pass runs on the tensor cores
        assert h.sync_status() == 0
        h.set_wait_limit(0)
        y = torch.zeros((R, n), dtype=torch.float64, device="cuda")
        h.step(x, y)
        assert h.sync_status() == -7  # WHFF_ETIMEOUT
        h.set_wait_limit(-1)
        h.step(x, y)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        ref = orc.gemv64(Ahat, X.T.astype(np.float64))
        Y = y.cpu().numpy()
        for r in range(R):
            assert np.linalg.norm(Y[r] - ref[:, r]) <= 1e-6 * np.linalg.norm(ref[:, r]), r
