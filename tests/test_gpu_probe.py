"""The achievable-read probe (whff_read_probe), through the C ABI: it reads every
16-byte word of the buffer once (the XOR of all 32-bit words equals numpy's, for
sizes with and without a tail past the four-loads-in-flight loop), and refuses
buffers that are not 16-byte aligned or sized."""
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


@pytest.mark.parametrize("words", [4, 1 << 10, (1 << 22) + 12, 150 * 8 * 256 * 4 * 4 + 20])
def test_probe_reads_every_word(env, words):
    W, torch = env
    a = np.random.default_rng(words).integers(0, 2**32, size=words, dtype=np.uint64).astype(np.uint32)
    buf = torch.from_numpy(a.view(np.int32)).cuda()
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    W.whff_read_probe(buf, out)
    torch.cuda.synchronize()
    assert int(out.cpu().numpy().view(np.uint32)[0]) == int(np.bitwise_xor.reduce(a))


def test_probe_rejects_unaligned(env):
    W, torch = env
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(W.WhffError):
        W.whff_read_probe(buf[4:20], out)  # 16 bytes at a 4-byte offset
    with pytest.raises(W.WhffError):
        W.whff_read_probe(buf[:20], out)  # 20 bytes
