"""Parity in the control loop's own regime (32768 x 32768 at 16 bits/value, WZ2 with
the lift, one right-hand side, the FP64 state s <- 0.99 s + y of Sec. 2.1).

  * A band-shaped slice with the full loop's band length: 1021 x 32765 (ragged in
    both directions), 8192 blocks per 4-row band, stepped under the launch shape the
    tuner picks on GB300 for the full matrix (4 blocks in flight, 3 CTAs per SM, the
    FP32-pair lane fold) and under the default shape; every entry of y and of the
    state against the FP64 oracle on the oracle's decode of the same blob.
  * The full 32768 x 32768 matrix itself, in the launch configuration the benchmark
    times (whff_tune on the handle), on sampled bands of rows that the oracle decodes
    and multiplies one by one: the first, the last and six seeded ones in between.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-6  # relative L2 against the FP64 oracle GEMV on the decoded matrix


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_1902_08018_gb300 as W

    W.library()
    return W, torch


@pytest.fixture(scope="module")
def band_slice(orc):
    import workloads

    M, N = 1021, 32765
    km = workloads.KernelMatrix(32768, 181, 181 * 181, 0.05, workloads.SEED_BASE + 2)
    A = np.ascontiguousarray(km.rows(0, M)[:, :N])
    return M, N, A


@pytest.mark.parametrize("shape", ["tuned", "default"])
def test_full_width_bands(env, orc, band_slice, shape):
    W, torch = env
    M, N, A = band_slice
    blob = W.whff_compress(A, W.FMT_FIXED_LIFT, 16)
    Ahat = orc.decode(blob.tobytes())
    rng = np.random.default_rng(32765)
    s_ref = np.zeros(M)
    with W.whff_create(blob, max_rhs=1) as h:
        if shape == "tuned":  # 4 blocks in flight, the most CTAs per SM it keeps resident (3 or 2), FP32 pairs
            for c in (3, 2):
                try:
                    h.set_config(4, c, 1)  # WHFF_FOLD_FP32_PAIRS
                    break
                except W.WhffError:
                    continue
            assert h.config()[0] == 4 and h.config()[2] == 1
        else:
            assert h.config()[0] == 2 and h.config()[2] == 0  # 8192 blocks per band: FP64 fold
        s = torch.zeros(M, dtype=torch.float64, device="cuda")
        for step in range(3):
            x = rng.standard_normal(N).astype(np.float32)
            y = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
            h.step(torch.from_numpy(x).cuda(), y, s, 0.99)
            torch.cuda.synchronize()
            ref = orc.gemv64(Ahat, x.astype(np.float64))
            got = y.cpu().numpy()
            assert rel_l2(got, ref) <= TOL, (step, rel_l2(got, ref))
            s_ref = orc.state_update(s_ref, ref, 0.99)
            assert rel_l2(s.cpu().numpy(), s_ref) <= TOL, step
        assert h.sync_status() == 0


def test_full_size_control_loop_sampled_rows(env, orc):
    """The 32768^2 control-loop matrix, compressed band by band like the benchmark,
    stepped in the tuned launch shape (and the default one) with the heat loads of
    control steps 0 and 1; sampled bands of y and of the state against the oracle."""
    W, torch = env
    import workloads

    cfg = workloads.config(2)
    km = cfg.matrix
    order = km.order
    blob = W.whff_compress_bands(order, order, km.bands(2048), W.FMT_FIXED_LIFT, 16)
    X = workloads.heat_loads(km.g, km.n_valid, order, 2).T.astype(np.float32)  # (2, N)
    rng = np.random.default_rng(2000)
    bands = sorted({0, order // 4 - 1, *rng.choice(order // 4, size=6, replace=False).tolist()})
    rows = np.concatenate([np.arange(4 * b, 4 * b + 4) for b in bands])
    D = np.concatenate([orc.decode_rows(blob, 4 * b, 4) for b in bands])  # (len(rows), N)
    refs = [orc.gemv64(D, X[k].astype(np.float64)) for k in range(2)]
    s_ref = orc.state_update(orc.state_update(np.zeros(len(rows)), refs[0], 0.99), refs[1], 0.99)
    for shape in ("tuned", "default"):
        h = W.whff_create(blob, max_rhs=1)
        if shape == "tuned":
            h.tune(iters=3)
        with h:
            s = torch.zeros(order, dtype=torch.float64, device="cuda")
            for k in range(2):
                y = torch.full((order,), float("nan"), dtype=torch.float64, device="cuda")
                h.step(torch.from_numpy(X[k]).cuda(), y, s, 0.99)
                torch.cuda.synchronize()
                got = y.cpu().numpy()
                assert not np.isnan(got).any()
                assert rel_l2(got[rows], refs[k]) <= TOL, (shape, k, rel_l2(got[rows], refs[k]))
            assert rel_l2(s.cpu().numpy()[rows], s_ref) <= TOL, shape
            assert h.sync_status() == 0
