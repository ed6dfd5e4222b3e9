"""Graph-captured steps and the request server, through the C ABI.

  * a captured step replays to exactly the result of whff_step;
  * served requests get exactly the y they would get alone when their pass
    ran on the same engine (CUDA cores below the handle's crossover), and y
    within relative L2 1e-6 of it when a wide pass ran on the tensor cores;
  * the carried state after a bursty trace equals the oracle's recursion
    s <- decay*s + y over the requests in arrival order;
  * models beyond the device-memory budget are refused (WHFF_EBUSY).
"""
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


def _matrix(n, seed):
    import workloads

    g = int(np.ceil(np.sqrt(n)))
    return workloads.KernelMatrix(n, g, n, 0.1, seed).dense()


def _same_as_alone(y, alone, batch, h):
    """Bit-exact when the pass used the CUDA cores like the single step, else
    within the accuracy bar (another rounding)."""
    if batch < h.crossover:
        return (y == alone).all()
    return np.linalg.norm(y - alone) <= 1e-6 * np.linalg.norm(alone)


def _step_alone(W, torch, h, x):
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    y = torch.zeros(h.M, dtype=torch.float64, device="cuda")
    h.step(xt, y, None, 0.99)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("fmt,rate", [(1, 16), (5, 16), (6, 12)])
def test_graph_replay_equals_step(env, fmt, rate):
    W, torch = env
    A = _matrix(600, 21)
    blob = W.whff_compress(A, fmt, rate)
    rng = np.random.default_rng(3)
    with W.whff_create(blob) as h:
        x = torch.zeros((2, 600), dtype=torch.float32, device="cuda")
        y = torch.zeros((2, 600), dtype=torch.float64, device="cuda")
        s = torch.zeros(600, dtype=torch.float64, device="cuda")
        s_ref = torch.zeros(600, dtype=torch.float64, device="cuda")
        y_ref = torch.zeros((2, 600), dtype=torch.float64, device="cuda")
        with W.whff_graph_create(h, x, y, s, 0.9) as g:
            for it in range(4):
                xv = torch.from_numpy(rng.standard_normal((2, 600)).astype(np.float32)).cuda()
                x.copy_(xv)
                g.launch()
                h.step(xv, y_ref, s_ref, 0.9)
                torch.cuda.synchronize()
                assert torch.equal(y, y_ref)
                assert torch.equal(s, s_ref)


def test_host_graph_replay(env):
    W, torch = env
    A = _matrix(500, 22)
    blob = W.whff_compress(A, 5, 16)
    rng = np.random.default_rng(4)
    with W.whff_create(blob) as h:
        xh = torch.zeros((4, 500), dtype=torch.float32).pin_memory()
        yh = torch.zeros((4, 500), dtype=torch.float64).pin_memory()
        with W.whff_graph_create_host(h, xh.numpy(), yh.numpy()) as g:
            for it in range(3):
                X = rng.standard_normal((4, 500)).astype(np.float32)
                xh.numpy()[:] = X
                g.launch()
                torch.cuda.synchronize()
                for r in range(4):  # a 4-column pass may run on the tensor cores
                    assert _same_as_alone(yh.numpy()[r], _step_alone(W, torch, h, X[r]), 4, h)


def test_server_batches_give_the_results_of_single_service(env, orc):
    W, torch = env
    sizes = [(256, 1, 16), (777, 5, 16), (1024, 6, 8)]
    handles, blobs = [], []
    for n, fmt, rate in sizes:
        blob = W.whff_compress(_matrix(n, n), fmt, rate)
        blobs.append(blob)
        handles.append(W.whff_create(blob, max_rhs=8))
    rng = np.random.default_rng(5)
    # bursts: many requests arrive at once, so passes are batched 1..8 wide
    n_req = 120
    model = rng.integers(0, len(sizes), size=n_req)
    arrival = np.sort(np.repeat(np.arange(n_req // 10) * 2e-3, 10))
    xs = [rng.standard_normal(sizes[m][0]).astype(np.float32) for m in model]
    with W.Server(hbm_budget=8 << 30, max_batch=8, nstreams=3) as srv:
        ids = [srv.add_model(h, decay=0.95) for h in handles]
        lat, bat, ys = srv.run(model, arrival, xs, want_y=True)
        states = [srv.read_state(i) for i in ids]
    assert bat.max() > 1  # some passes were batched
    assert (lat > 0).all()
    for i in range(n_req):
        h = handles[model[i]]
        assert _same_as_alone(ys[i], _step_alone(W, torch, h, xs[i]), bat[i], h), i
    for m, (n, fmt, rate) in enumerate(sizes):
        Ahat = orc.decode(blobs[m].tobytes())
        s = np.zeros(n)
        for i in np.nonzero(model == m)[0]:  # arrival order
            s = orc.state_update(s, orc.gemv64(Ahat, xs[i].astype(np.float64)).reshape(n, 1), 0.95)
        assert np.linalg.norm(states[m] - s) <= 1e-6 * np.linalg.norm(s)
    for h in handles:
        h.destroy()


def test_server_admission_by_footprint(env):
    W, torch = env
    blob = W.whff_compress(_matrix(512, 1), 5, 16)
    h1 = W.whff_create(blob, max_rhs=8)
    h2 = W.whff_create(blob, max_rhs=8)
    # room for one model (its matrix, workspace and staging) but not for two
    with W.Server(hbm_budget=int(h1.device_bytes * 1.6), max_batch=8, nstreams=1) as srv:
        srv.add_model(h1)
        with pytest.raises(W.WhffError) as e:
            srv.add_model(h2)
        assert e.value.code == -8  # WHFF_EBUSY
    h1.destroy()
    h2.destroy()


def test_firm_mode_drops_expired_requests(env, orc):
    # firm real time: a request whose deadline passed while queued is discarded; the
    # state then follows only the served requests, still in arrival order
    W, torch = env
    n = 2048
    blob = W.whff_compress(_matrix(n, 9), 5, 16)
    h = W.whff_create(blob, max_rhs=8)
    rng = np.random.default_rng(6)
    n_req = 200
    arrival = np.zeros(n_req)  # everything at once: most requests expire in the queue
    xs = [rng.standard_normal(n).astype(np.float32) for _ in range(n_req)]
    with W.Server(hbm_budget=8 << 30, max_batch=8, nstreams=1) as srv:
        mid = srv.add_model(h, decay=0.9)
        lat, bat, ys, status = srv.run(np.zeros(n_req, dtype=np.int32), arrival, xs, want_y=True,
                                       drop_after_s=20e-6, return_status=True)
        state = srv.read_state(mid)
    assert set(np.unique(status)) <= {0, 1, 2}
    assert (status == 2).any() and (status != 2).any()
    assert (bat[status == 2] == 0).all() and (bat[status != 2] > 0).all()
    Ahat = orc.decode(blob.tobytes())
    s = np.zeros(n)
    for i in np.nonzero(status != 2)[0]:
        assert _same_as_alone(ys[i], _step_alone(W, torch, h, xs[i]), bat[i], h), i
        s = orc.state_update(s, orc.gemv64(Ahat, xs[i].astype(np.float64)).reshape(n, 1), 0.9)
    assert np.linalg.norm(state - s) <= 1e-6 * np.linalg.norm(s)
    h.destroy()


def test_waiting_model_admitted_once_memory_frees(env, orc):
    """North star's serving rule: a model that does not fit waits and is admitted as
    memory frees up (whff_server_remove_model); meanwhile its requests are refused
    (status 3), afterwards they are served and its state follows the oracle."""
    W, torch = env
    blob = W.whff_compress(_matrix(512, 1), 5, 16)
    h1 = W.whff_create(blob, max_rhs=8)
    h2 = W.whff_create(blob, max_rhs=8)
    Ahat = orc.decode(blob.tobytes())
    rng = np.random.default_rng(7)
    xs = [rng.standard_normal(512).astype(np.float32) for _ in range(6)]
    with W.Server(hbm_budget=int(h1.device_bytes * 1.6), max_batch=8, nstreams=1) as srv:
        a = srv.add_model(h1, decay=0.9)
        b = srv.add_model(h2, decay=0.9, wait=True)  # over the budget: waits instead of WHFF_EBUSY
        assert (srv.model_state(a), srv.model_state(b)) == ("admitted", "waiting")
        with pytest.raises(W.WhffError) as e:  # without waiting, still refused
            srv.add_model(h2)
        assert e.value.code == -8
        lat, bat, _, status = srv.run(np.array([a, b, a], dtype=np.int32), np.zeros(3), xs[:3],
                                      return_status=True)
        assert list(status) == [0, 3, 0] and bat[1] == 0
        srv.remove_model(a)  # frees the budget: b is admitted
        assert (srv.model_state(a), srv.model_state(b)) == ("removed", "admitted")
        lat, bat, ys, status = srv.run(np.array([b, b, b], dtype=np.int32), np.array([0.0, 1e-3, 2e-3]), xs[3:],
                                       want_y=True, return_status=True)
        assert (status != 3).all() and (status != 2).all()  # no firm deadline: all served
        state = srv.read_state(b)
        with pytest.raises(W.WhffError):  # a removed model has no state
            srv.read_state(a)
    s = np.zeros(512)
    for i in range(3):
        ref = orc.gemv64(Ahat, xs[3 + i].astype(np.float64))
        assert np.linalg.norm(ys[i] - ref) <= 1e-6 * np.linalg.norm(ref)
        s = orc.state_update(s, ref.reshape(512, 1), 0.9)
    assert np.linalg.norm(state - s) <= 1e-6 * np.linalg.norm(s)
    h1.destroy()
    h2.destroy()
