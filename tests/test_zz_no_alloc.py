"""frnn_build_graph_noalloc, the entry point for callers that may not
allocate device memory (for example code inside a framework that owns all
device memory and forbids cudaMalloc after start-up).  It keeps its scratch in
a fixed array in device memory, so the tests check that two calls in a row,
with different events, each give exactly what the plan-based entry point
gives, and that sizes beyond its limits are refused.  Collected last so that
a run stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2202_06929_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2202_06929_b300 as frnn  # noqa: E402


def _entry():
    fn = frnn.load().frnn_build_graph_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _reference(x, r, k):
    n, d = x.shape
    with frnn.Plan(n_max=n, d_max=d, k_max_cap=k) as plan:
        host = plan.build(torch.from_numpy(x).cuda(), r, k).to_host()
        assert plan.last_status() == frnn.FRNN_OK
    return host


def test_noalloc_matches_plan_build_on_two_calls_in_a_row():
    fn = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(synth.make_event("c1"), 0.1, 64),
             (synth.clustered_grid(30000, 12, 5, 2500, 0.03, 0.15), 0.12, 40)]
    for x, r, k in cases:
        n, d = x.shape
        ref = _reference(x, r, k)
        xt = torch.from_numpy(x).cuda()
        row_ptr = torch.full((n + 1,), -7, dtype=torch.int32, device="cuda")
        col = torch.full((n * k,), -7, dtype=torch.int32, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rc = fn(xt.data_ptr(), n, d, r, k, row_ptr.data_ptr(), col.data_ptr(), col.numel(),
                status.data_ptr(), stream)
        assert rc == frnn.FRNN_OK, frnn.status_string(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == frnn.FRNN_OK
        rp = row_ptr.cpu().numpy()
        np.testing.assert_array_equal(rp, ref["row_ptr"])
        np.testing.assert_array_equal(col[: int(rp[-1])].cpu().numpy(), ref["col"])


def test_noalloc_refuses_sizes_beyond_its_limits():
    fn = _entry()
    x = torch.zeros((40000, 4), device="cuda")
    rp = torch.zeros(40001, dtype=torch.int32, device="cuda")
    col = torch.zeros(16, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    for n, d, k in [(32769, 4, 8), (100, 17, 8), (100, 4, 65)]:
        rc = fn(x.data_ptr(), n, d, 0.1, k, rp.data_ptr(), col.data_ptr(), 16, st.data_ptr(), None)
        assert rc == frnn.FRNN_ERR_CAPACITY


def test_noalloc_device_status_outputs_and_empty_event():
    """The device-side outcomes: more edges than col_capacity gives OVERFLOW,
    a NaN gives NONFINITE_INPUT with empty rows, and n = 0 gives row_ptr[0] = 0
    with status OK."""
    fn = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    x = synth.make_event("c1")
    n, d = x.shape
    ref = _reference(x, 0.1, 64)
    xt = torch.from_numpy(x).cuda()
    row_ptr = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(n * 64, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    small = int(ref["row_ptr"][-1]) - 1
    rc = fn(xt.data_ptr(), n, d, 0.1, 64, row_ptr.data_ptr(), col.data_ptr(), small, status.data_ptr(), stream)
    assert rc == frnn.FRNN_OK
    torch.cuda.synchronize()
    assert int(status.item()) == frnn.FRNN_ERR_OVERFLOW
    bad = x.copy()
    bad[5, 1] = np.nan
    bt = torch.from_numpy(bad).cuda()
    rc = fn(bt.data_ptr(), n, d, 0.1, 64, row_ptr.data_ptr(), col.data_ptr(), col.numel(), status.data_ptr(), stream)
    assert rc == frnn.FRNN_OK
    torch.cuda.synchronize()
    assert int(status.item()) == frnn.FRNN_ERR_NONFINITE_INPUT
    assert int(row_ptr[-1].item()) == 0
    row_ptr.fill_(-3)
    status.fill_(-1)
    rc = fn(xt.data_ptr(), 0, d, 0.1, 64, row_ptr.data_ptr(), col.data_ptr(), col.numel(), status.data_ptr(), stream)
    assert rc == frnn.FRNN_OK
    torch.cuda.synchronize()
    assert int(row_ptr[0].item()) == 0 and int(status.item()) == frnn.FRNN_OK
    # and the next call is exact again
    rc = fn(xt.data_ptr(), n, d, 0.1, 64, row_ptr.data_ptr(), col.data_ptr(), col.numel(), status.data_ptr(), stream)
    assert rc == frnn.FRNN_OK
    torch.cuda.synchronize()
    assert int(status.item()) == frnn.FRNN_OK
    np.testing.assert_array_equal(row_ptr.cpu().numpy(), ref["row_ptr"])
    np.testing.assert_array_equal(col[: int(ref["row_ptr"][-1])].cpu().numpy(), ref["col"])
