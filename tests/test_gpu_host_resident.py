"""Host-resident handles (the compressed stream in pinned, mapped host memory,
read by the fused kernels over the CPU-GPU link every step -- the paper's
system moves the matrix over the host link, Sec. 4.2): the same kernels on the
same bytes give the same results bit for bit as an HBM-resident handle, for
CUDA-core and tensor-core passes, slits and decompression."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_1902_08018_gb300 as W

    W.library()
    return W, torch


@pytest.mark.parametrize("fmt,rate", [(5, 16), (6, 12), (1, 16), (2, 0), (7, 0)])
def test_host_resident_equals_device_resident(env, fmt, rate):
    import workloads

    W, torch = env
    M, N = 700, 1300
    A = workloads.KernelMatrix(1300, 37, 1300, 0.1, 12).rows(0, M)[:, :N]
    blob = W.whff_compress(A, fmt, rate or 16)
    X = torch.from_numpy(np.random.default_rng(fmt).standard_normal((9, N)).astype(np.float32)).cuda()
    out = []
    for host in (False, True):
        with W.whff_create(blob, max_rhs=16, host_resident=host) as h:
            y = torch.zeros((9, M), dtype=torch.float64, device="cuda")
            s = torch.full((M,), 0.5, dtype=torch.float64, device="cuda")
            h.step(X, y, s, 0.9)  # 9 columns: a tensor-core pass on WZ2
            y1 = torch.zeros(M, dtype=torch.float64, device="cuda")
            h.step(X[0], y1)
            ys = torch.zeros((2, 256), dtype=torch.float64, device="cuda")
            h.step_rows(256, 256, X[:2], ys)
            D = torch.zeros((M, N), dtype=torch.float64, device="cuda")
            h.decompress(D)
            torch.cuda.synchronize()
            assert h.sync_status() == 0
            out.append((y, s, y1, ys, D, h.device_bytes))
    (a, b) = out
    for u, v in zip(a[:5], b[:5]):
        assert torch.equal(u, v)
    assert a[5] - b[5] == blob.size - 64  # the stream is not in device memory
