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
