"""Track labeling on the GPU (weakly connected components of the edges that
pass a d2 cut): labels equal the oracle's (smallest index of each component),
for single and batched builds and several cuts."""
import numpy as np
import pytest

import oracle
from paper_2202_06929_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2202_06929_b300 as frnn  # noqa: E402


@pytest.mark.parametrize("cut", [1.0, 0.6, 0.3])
def test_labels_equal_oracle(cut):
    x = synth.clustered_grid(6000, 8, 17, 400, 0.03, 0.2)
    r, k = 0.1, 8
    d2_max = float(np.float32(cut * cut * r * r))
    with frnn.Plan(n_max=x.shape[0], d_max=8, k_max_cap=k, emit_d2=True) as plan:
        plan.build(torch.from_numpy(x).cuda(), r, k)
        labels = plan.label_components(d2_max).cpu().numpy()
        assert plan.last_status() == 0
    np.testing.assert_array_equal(labels, oracle.track_labels(x, r, k, d2_max))


def test_labels_batched_and_replayed():
    sizes = [3000, 0, 1, 5000, 2500]
    evs = [synth.clustered_grid(n, 8, 60 + i, max(n // 15, 1), 0.03, 0.2) for i, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    xt = torch.from_numpy(np.concatenate(evs)).cuda()
    with frnn.Plan(n_max=int(off[-1]), d_max=8, k_max_cap=16, events_max=8, use_graph=True) as plan:
        for _ in range(2):
            plan.build_batched(xt, off, 0.1, 16)
            labels = plan.label_components().cpu().numpy()
            assert plan.last_status() == 0
            for b, x in enumerate(evs):
                want = oracle.track_labels(x, 0.1, 16, float("inf"))
                np.testing.assert_array_equal(labels[off[b]:off[b + 1]], want)


def test_cut_below_radius_needs_d2():
    x = torch.from_numpy(synth.uniform_grid(500, 3, 2, -30, 30)).cuda()
    with frnn.Plan(n_max=500, d_max=3, k_max_cap=8) as plan:
        with pytest.raises(frnn.FrnnError):
            plan.label_components(0.001)          # no build yet
        plan.build(x, 0.1, 8)
        with pytest.raises(frnn.FrnnError) as ei:
            plan.label_components(0.001)          # needs FRNN_EMIT_D2
        assert ei.value.status == frnn.FRNN_ERR_INVALID_ARG
        plan.label_components(1.0)                # every edge kept: fine
        assert plan.last_status() == 0


def test_edge_features_in_chunks_equal_oracle():
    """[x_i, x_j, d2] per edge, produced in fixed-size chunks as the filter
    stage consumes them, equal the oracle's graph gathered on the host."""
    sizes = [4000, 2500]
    evs = [synth.clustered_grid(n, 8, 70 + i, n // 12, 0.03, 0.15) for i, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    x_all = np.concatenate(evs)
    r, k = 0.1, 16
    xt = torch.from_numpy(x_all).cuda()
    with frnn.Plan(n_max=int(off[-1]), d_max=8, k_max_cap=k, events_max=2) as plan:
        csr = plan.build_batched(xt, off, r, k)
        e_tot = csr.n_edges()
        chunk = 7001
        feats = torch.cat([plan.edge_features(xt, a, min(a + chunk, e_tot)) for a in range(0, e_tot, chunk)])
        assert plan.last_status() == 0
    feats = feats.cpu().numpy()
    want = []
    for b, x in enumerate(evs):
        rp, col, d2 = oracle.radius_graph(x, r, k, with_d2=True)
        src = np.repeat(np.arange(x.shape[0]), np.diff(rp))
        want.append(np.concatenate([x[src], x[col], d2[:, None]], axis=1))
    want = np.concatenate(want)
    assert feats.shape == want.shape == (e_tot, 17)
    np.testing.assert_array_equal(feats.view(np.uint32), want.astype(np.float32).view(np.uint32))
