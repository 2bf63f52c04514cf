"""The walk's one-byte key filter may only skip pairs farther than r.

A host-side restatement of the bound the planning step relies on (the
filter keys and threshold of FiltPlan): keys q_t = floor(fl(fl(x_t - lo_t) *
inv_h)) with inv_h = fl(254 / w) in float32, and for every pair whose float32
squared distance (summed in dim order, each operation rounded once) is at
most fl(r * r), sum_t |q_t - q'_t| <= thr = floor((2 sqrt(r2) inv_h + 4)
(1 + 2^-10)).  Checked on random, clustered and adversarial inputs: partners
placed within a few ulps of r along the filter dims, extents that make the
key step coarse or fine, and the degenerate ranges that switch the filter
off.  No GPU: this pins the arithmetic of the bound, not the kernel.
"""
import numpy as np
import pytest

F = np.float32


def keys(x, dims, lo, inv_h):
    a = ((x[:, dims] - lo[dims]).astype(F) * F(inv_h)).astype(F)
    return np.where(a < F(255), np.floor(a), 255).astype(np.int64)


def threshold(r2, inv_h):
    b = (2.0 * np.sqrt(np.float64(r2)) * np.float64(inv_h) + 4.0) * (1.0 + 2.0 ** -10)
    return int(np.floor(b))


def d2_seq(a, b):
    s = F(0)
    for t in range(a.shape[0]):
        d = F(a[t] - b[t])
        s = F(s + F(d * d))
    return s


def check(x, r, dims):
    x = x.astype(F)
    r2 = F(F(r) * F(r))
    lo = x.min(axis=0)
    w = (x.max(axis=0) - lo).astype(F)
    wmax = F(max(w[dims].max(), 0))
    assert wmax >= 2.0 ** -90 and r2 >= 2.0 ** -100  # the filter is on
    inv_h = F(F(254.0) / wmax)
    q = keys(x, dims, lo, inv_h)
    thr = threshold(r2, inv_h)
    n = x.shape[0]
    # every pair within r (float32 sequential sum) passes the key test
    diff = x[:, None, :] - x[None, :, :]
    close = np.argwhere((diff.astype(np.float64) ** 2).sum(-1) <= 1.01 * float(r2))
    checked = 0
    for i, j in close:
        if i == j or d2_seq(x[i], x[j]) > r2:
            continue
        assert np.abs(q[i] - q[j]).sum() <= thr, (i, j)
        checked += 1
    return checked


@pytest.mark.parametrize("seed", range(4))
def test_partners_at_the_radius(seed):
    rng = np.random.default_rng(seed)
    d, r = 8, 0.1
    base = rng.uniform(-1, 1, size=(150, d))
    parts = [base]
    for scale in (1 - 2 ** -22, 1.0, 1 + 2 ** -22, 1 - 2 ** -14):
        u = rng.normal(size=(150, d))
        u[:, :4] = 0.0  # displaced along the filter dims only
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        parts.append(base + r * scale * u)
    x = np.concatenate(parts)
    assert check(x, r, np.array([4, 5, 6, 7])) > 300


@pytest.mark.parametrize("extent", [0.05, 2.0, 300.0])
def test_coarse_and_fine_key_steps(extent):
    rng = np.random.default_rng(11)
    d = 6
    x = rng.uniform(0, extent, size=(400, d))
    r = extent * 0.08
    x[200:300] = x[:100] + rng.normal(0, r / 3, size=(100, d))
    assert check(x, r, np.array([2, 3, 4, 5])) > 50


def test_clustered_on_the_grid():
    rng = np.random.default_rng(5)
    c = rng.uniform(-1, 1, size=(30, 8))
    x = np.rint((np.repeat(c, 12, axis=0) + rng.normal(0, 0.03, size=(360, 8))) * 256) / 256
    x = np.clip(x, -1, 1)
    assert check(x, 0.1, np.array([0, 2, 5, 7])) > 500


def test_threshold_examples():
    # the N=120k workload's numbers: extent 2 over the filter dims, r = 0.1
    inv_h = F(F(254.0) / F(2.0))
    assert threshold(F(F(0.1) * F(0.1)), inv_h) == 29
    # a point's key never exceeds 254 when w is the largest extent
    x = np.array([[0.0], [2.0]], dtype=F)
    assert keys(x, np.array([0]), x.min(axis=0), inv_h).max() == 254
