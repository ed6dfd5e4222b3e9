"""The bulk-staged one-right-hand-side kernel (WHFF_CONFIG_BULK: each warp's block range
streamed through a shared-memory ring by cp.async.bulk) against the register-fed kernel
and the FP64 oracle, through the C ABI.

  * Same partition (CTAs per SM) and fold: y and the state bit for bit equal to the
    register-fed kernel, for every WZ2 rate (16- to 48-byte blocks), with and without
    the lift, ragged shapes, bands shared by several warp ranges;
  * slits whose first block is not 16-byte aligned (24- and 40-byte blocks, odd blocks
    per band) take the aligned-down copy and still match bit for bit;
  * against the oracle on the decoded matrix within relative L2 1e-6.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-6
BULK = 4  # WHFF_CONFIG_BULK


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

    return workloads.RectKernelMatrix(M, N, 0.05, seed).dense()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("fmt,rate", [(5, 8), (5, 12), (5, 16), (5, 20), (5, 24), (6, 8), (6, 12)])
@pytest.mark.parametrize("M,N", [(1037, 4001), (130, 30001)])
def test_bulk_equals_register_fed_bit_for_bit(env, orc, fmt, rate, M, N):
    W, torch = env
    blob = W.whff_compress(_matrix(M, N, M + rate), fmt, rate)
    Ahat = orc.decode(blob.tobytes())
    X = np.random.default_rng(rate).standard_normal(N).astype(np.float32)
    x = torch.from_numpy(X).cuda()
    ref = orc.gemv64(Ahat, X.astype(np.float64))
    with W.whff_create(blob, max_rhs=1) as h:
        fold0 = h.config()[2] & 1
        for c in (1, 2):
            outs = []
            for flags in (fold0, fold0 | BULK):
                h.set_config(2, c, flags)
                assert h.config()[1:] == (c, flags)
                y = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
                s = torch.full((M,), 0.25, dtype=torch.float64, device="cuda")
                h.step(x, y, s, 0.5)
                torch.cuda.synchronize()
                outs.append((y.cpu().numpy(), s.cpu().numpy()))
            assert np.array_equal(outs[0][0], outs[1][0]), (c, "y")
            assert np.array_equal(outs[0][1], outs[1][1]), (c, "state")
            assert _rel(outs[1][0], ref) <= TOL
        assert h.sync_status() == 0


@pytest.mark.parametrize("rate", [12, 20, 8])
def test_bulk_slits_with_unaligned_starts(env, orc, rate):
    W, torch = env
    M, N = 600, 1001  # 251 blocks per band: every other band starts 8 bytes off a 16-byte boundary
    blob = W.whff_compress(_matrix(M, N, 9), 5, rate)
    Ahat = orc.decode(blob.tobytes())
    X = np.random.default_rng(9).standard_normal(N).astype(np.float32)
    x = torch.from_numpy(X).cuda()
    with W.whff_create(blob, max_rhs=1) as h:
        for row0, nrows in ((4, 37), (12, 300), (0, M), (596, 4)):
            outs = []
            for flags in (1, 1 | BULK):
                h.set_config(2, 2, flags)
                y = torch.zeros(nrows, dtype=torch.float64, device="cuda")
                h.step_rows(row0, nrows, x, y)
                torch.cuda.synchronize()
                outs.append(y.cpu().numpy())
            assert np.array_equal(outs[0], outs[1]), (row0, nrows)
            ref = orc.gemv64(Ahat[row0:row0 + nrows], X.astype(np.float64))
            mag = orc.gemv64(np.abs(Ahat[row0:row0 + nrows]), np.abs(X.astype(np.float64)))
            assert (np.abs(outs[1] - ref) <= 1e-6 * mag).all()
        assert h.sync_status() == 0


def test_bulk_flag_rules(env):
    W, torch = env
    blob = W.whff_compress(_matrix(64, 64, 1), 5, 16)
    with W.whff_create(blob, max_rhs=1) as h:
        with pytest.raises(W.WhffError):
            h.set_config(2, 1, BULK | 2)  # not with lane groups
        with pytest.raises(W.WhffError):
            h.set_config(2, 99, BULK)  # more CTAs than the staged kernel keeps resident
        h.set_config(2, 1, BULK)
        assert h.config() == (2, 1, BULK)
