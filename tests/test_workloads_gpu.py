"""The remaining workloads at full size: the batched stand-in (64 events of
N ~ U[40k, 140k], K=64), the pile-up-scale event (N=1,000,000, D=12, r=0.15,
K=128) and its cap-binding variant, with sampled rows checked exactly against
the oracle; and the autotuner, which may change speed but never the result."""
import numpy as np
import pytest

import oracle
from paper_2202_06929_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2202_06929_b300 as frnn  # noqa: E402


def _sampled_equal(x, r, k, rp, col, n_q, seed):
    n = x.shape[0]
    q = np.unique(np.concatenate([np.random.default_rng(seed).choice(n, size=min(n_q, n), replace=False),
                                  [0, n - 1]]))
    orp, ocol = oracle.radius_graph(x, r, k, queries=q)
    for qi, i in enumerate(q):
        np.testing.assert_array_equal(col[rp[i]:rp[i + 1]], ocol[orp[qi]:orp[qi + 1]], err_msg=f"row {i}")
    return q, np.diff(orp)


def test_c3_batched_events():
    w = synth.WORKLOADS["c3"]
    evs = [synth.make_event("c3", e) for e in range(64)]
    off = np.concatenate([[0], np.cumsum([e.shape[0] for e in evs])]).astype(np.int64)
    assert all(40_000 <= e.shape[0] <= 140_000 for e in evs)
    with frnn.Plan(n_max=int(off[-1]), d_max=w.d, k_max_cap=w.k, events_max=64, use_graph=True) as plan:
        csr = plan.build_batched(torch.from_numpy(np.concatenate(evs)).cuda(), off, w.r, w.k)
        host = csr.to_host()
        assert plan.last_status() == 0
    for b in range(0, 64, 8):
        rp, col = csr.event_rows(host, b)
        _sampled_equal(evs[b], w.r, w.k, rp, col, 300, b)


@pytest.mark.parametrize("name", ["c5", "c5b"])
def test_pileup_scale_event(name):
    w = synth.WORKLOADS[name]
    x = synth.make_event(name)
    assert x.shape == (1_000_000, 12)
    with frnn.Plan(n_max=x.shape[0], d_max=w.d, k_max_cap=w.k, edge_capacity=x.shape[0] * w.k) as plan:
        host = plan.build(torch.from_numpy(x).cuda(), w.r, w.k).to_host()
        assert plan.last_status() == 0
    rp = host["row_ptr"].astype(np.int64)
    q, lens = _sampled_equal(x, w.r, w.k, rp, host["col"], 2000, 77)
    capped = np.mean(lens == w.k)
    if name == "c5b":
        assert capped > 0.5, capped     # the cap binds for most rows
    else:
        assert capped < 0.01, capped


def test_autotune_keeps_result():
    evs = [synth.make_event("c2", e, n=30_000) for e in range(4)]
    off = np.concatenate([[0], np.cumsum([e.shape[0] for e in evs])]).astype(np.int64)
    xt = torch.from_numpy(np.concatenate(evs)).cuda()
    with frnn.Plan(n_max=int(off[-1]), d_max=8, k_max_cap=256, events_max=4, cells_per_point=32) as plan:
        ref = plan.build_batched(xt, off, 0.1, 256).to_host()
        g, scale, ms = plan.autotune(xt, off, 0.1, 256)
        assert g in (2, 3, 4, 5, 6) and scale in (1.0, 1.25, 1.5, 2.0) and ms > 0
        assert plan.get_tuning() == (g, scale)
        got = plan.build_batched(xt, off, 0.1, 256).to_host()
        assert plan.last_status() == 0
    np.testing.assert_array_equal(got["row_ptr"], ref["row_ptr"])
    np.testing.assert_array_equal(got["col"], ref["col"])
