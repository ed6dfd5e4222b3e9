"""Host-side argument checks of the Python binding that need no GPU: they run
before any call into the library."""


def test_server_run_checks_requests_before_the_c_call():
    """The server binding refuses mismatched request arrays, unknown models and short x
    vectors before the C call, which copies N floats from every x."""
    import types

    import numpy as np
    import pytest

    import paper_1902_08018_gb300 as W

    srv = object.__new__(W.Server)  # no device: the checks run before any library call
    srv._ptr = None
    srv.models = [types.SimpleNamespace(M=8, N=16)]
    x = np.zeros(16, dtype=np.float32)
    with pytest.raises(W.WhffError):
        srv.run([0, 0], [0.0], [x, x])  # one arrival for two requests
    with pytest.raises(W.WhffError):
        srv.run([1], [0.0], [x])  # no model 1
    with pytest.raises(W.WhffError):
        srv.run([0], [0.0], [np.zeros(15, dtype=np.float32)])  # 15 < N


def test_step_host_checks_shapes_before_the_c_call():
    """whff_step_host copies R columns of N floats in and R columns of M doubles out:
    y with fewer rows than x, or rows shorter than N / M, are refused first."""
    import types

    import numpy as np
    import pytest

    import paper_1902_08018_gb300 as W

    h = types.SimpleNamespace(M=8, N=16, ptr=None)
    x = np.zeros((4, 16), dtype=np.float32)
    with pytest.raises(W.WhffError):
        W.whff_step_host(h, x, np.zeros((1, 8)))  # one row of y for four columns
    with pytest.raises(W.WhffError):
        W.whff_step_host(h, x[:, :15], np.zeros((4, 8)))  # rows shorter than N
    with pytest.raises(W.WhffError):
        W.whff_step_host(h, x, np.zeros((4, 7)))  # rows shorter than M


def test_host_graph_checks_shapes_before_the_c_call():
    import types

    import numpy as np
    import pytest

    import paper_1902_08018_gb300 as W

    h = types.SimpleNamespace(M=8, N=16, ptr=None)
    with pytest.raises(W.WhffError):
        W.whff_graph_create_host(h, np.zeros((4, 16), dtype=np.float32), np.zeros((2, 8)))


def test_batch_step_checks_its_lists_before_the_c_call():
    """Batch.step refuses lists whose lengths differ from the batch's before any library
    call (the per-tensor checks need CUDA tensors and run on the GPU)."""
    import types

    import pytest

    import paper_1902_08018_gb300 as W

    b = object.__new__(W.Batch)
    b._ptr = None
    b.handles = [types.SimpleNamespace(M=8, N=16), types.SimpleNamespace(M=4, N=4)]
    b.R = [1, 1]
    with pytest.raises(W.WhffError):
        b.step([None], [None, None])
    with pytest.raises(W.WhffError):
        b.step([None, None], [None, None], states=[None])
