"""Seeded synthetic inputs for the fixed-radius nearest-neighbour graph build.

The paper measures graph building on embedded TrackML spacepoints (Sec. 2 and
Table 1).  Neither the dataset nor the trained embedding network is available,
so every input here is synthetic: points in a D-dimensional latent space that
look like the embedding's output, i.e. tight groups of points (one group per
particle track) plus isolated points.  Coordinates are quantised onto the grid
u = 1/256 inside [-1, 1], so every squared distance between two points is an
integer multiple of u^2 that float32 represents exactly.

This module only draws random numbers.  It holds none of the graph-building
arithmetic and imports neither the CUDA library nor the CPU oracle, so both
sides of every parity test can share it.

Workloads (sizes, radius and neighbour cap are not stated in the paper; these
are the build's stand-ins):

    c1   N=2,000, D=8, 200 isotropic clusters x 10 points, sigma=0.03, no noise;
         r=0.1, K=64
    c2   N=120,000, D=8, track-like clusters of U{5..20} points (sigma 0.02 along
         a random direction, 0.005 across) plus round(0.15 N) uniform noise
         points; r=0.1, K=256
    c3   batched events, N ~ U[40k, 140k] per event, the c1 generator with
         N/10 clusters of 10; r=0.1, K=64
    c4   served events, N ~ U[20k, 200k] per event, the c2 generator; r=0.1, K=256
    c5   N=1,000,000, D=12, track-like clusters of U{5..30} plus 25% noise;
         r=0.15, K=128
    c5b  as c5, but every cluster centre and noise point has dims 0-3 uniform in
         [-0.9, 0.9] and dims 4-11 ~ N(0, 0.01^2), so the K cap binds for most
         points

Seed of event e of workload c: 2202069290 + 1000 * c + e (c5b uses c = 6).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GRID = 256  # grid steps per unit length: coordinates are m / 256, |m| <= 256
SEED_BASE = 2202069290


@dataclass(frozen=True)
class Workload:
    name: str
    index: int          # used in the seed
    d: int
    r: float
    k: int
    n: int | None       # fixed N, or None when N is drawn per event
    n_range: tuple[int, int] | None


WORKLOADS = {
    "c1": Workload("c1", 1, 8, 0.1, 64, 2000, None),
    "c2": Workload("c2", 2, 8, 0.1, 256, 120_000, None),
    "c3": Workload("c3", 3, 8, 0.1, 64, None, (40_000, 140_000)),
    "c4": Workload("c4", 4, 8, 0.1, 256, None, (20_000, 200_000)),
    "c5": Workload("c5", 5, 12, 0.15, 128, 1_000_000, None),
    "c5b": Workload("c5b", 6, 12, 0.15, 128, 1_000_000, None),
}


def seed_of(workload: str, event: int) -> int:
    return SEED_BASE + 1000 * WORKLOADS[workload].index + int(event)


def quantise(x: np.ndarray) -> np.ndarray:
    """Round onto the 1/256 grid (half to even), clip to [-1, 1], as float32."""
    m = np.clip(np.rint(x * GRID), -GRID, GRID)
    return (m / GRID).astype(np.float32)


def assert_on_grid(x: np.ndarray) -> None:
    m = x.astype(np.float64) * GRID
    if not (np.all(m == np.rint(m)) and np.all(np.abs(m) <= GRID)):
        raise AssertionError("coordinates are not on the 1/256 grid in [-1, 1]")


def _isotropic_clusters(rng, n_clusters, size, d, sigma):
    centres = rng.uniform(-1.0, 1.0, size=(n_clusters, d))
    pts = centres[:, None, :] + rng.normal(0.0, sigma, size=(n_clusters, size, d))
    return pts.reshape(-1, d)


def _track_like(rng, sizes, d, centres, s_along=0.02, s_across=0.005):
    """Elongated groups: centre + s_along*t*u + (I - u u^T)(s_across*n)."""
    out = []
    for c, m in zip(centres, sizes):
        u = rng.normal(size=d)
        u /= np.linalg.norm(u)
        t = rng.normal(size=(m, 1))
        nn = rng.normal(size=(m, d)) * s_across
        nn -= (nn @ u)[:, None] * u[None, :]
        out.append(c[None, :] + s_along * t * u[None, :] + nn)
    return np.concatenate(out, axis=0) if out else np.zeros((0, d))


def _cluster_sizes(rng, total, lo, hi):
    sizes = []
    left = total
    while left > 0:
        m = int(rng.integers(lo, hi + 1))
        m = min(m, left)
        sizes.append(m)
        left -= m
    return sizes


def _trackml_shaped(rng, n, d, noise_frac, size_lo, size_hi, centre_fn):
    n_noise = int(round(noise_frac * n))
    sizes = _cluster_sizes(rng, n - n_noise, size_lo, size_hi)
    centres = centre_fn(rng, len(sizes))
    pts = _track_like(rng, sizes, d, centres)
    noise = centre_fn(rng, n_noise)
    return np.concatenate([pts, noise], axis=0)


def make_event(workload: str, event: int = 0, n: int | None = None) -> np.ndarray:
    """One event of a named workload: float32 [N, D] on the 1/256 grid.

    ``n`` overrides the point count (the generator keeps its shape)."""
    w = WORKLOADS[workload]
    rng = np.random.default_rng(seed_of(workload, event))
    if n is None:
        n = w.n if w.n is not None else int(rng.integers(w.n_range[0], w.n_range[1] + 1))
    d = w.d
    if workload in ("c1", "c3"):
        n_cl = n // 10
        pts = _isotropic_clusters(rng, n_cl, 10, d, 0.03)
        rest = n - pts.shape[0]
        if rest:
            pts = np.concatenate([pts, _isotropic_clusters(rng, 1, rest, d, 0.03)])
    elif workload in ("c2", "c4"):
        uni = lambda g, m: g.uniform(-1.0, 1.0, size=(m, d))
        pts = _trackml_shaped(rng, n, d, 0.15, 5, 20, uni)
    elif workload == "c5":
        uni = lambda g, m: g.uniform(-1.0, 1.0, size=(m, d))
        pts = _trackml_shaped(rng, n, d, 0.25, 5, 30, uni)
    elif workload == "c5b":
        def slab(g, m):
            c = np.empty((m, d))
            c[:, :4] = g.uniform(-0.9, 0.9, size=(m, 4))
            c[:, 4:] = g.normal(0.0, 0.01, size=(m, d - 4))
            return c
        pts = _trackml_shaped(rng, n, d, 0.25, 5, 30, slab)
    else:  # pragma: no cover
        raise KeyError(workload)
    pts = pts[rng.permutation(pts.shape[0])]
    x = quantise(pts)
    assert x.shape == (n, d)
    return x


def event_sizes(workload: str, n_events: int, first: int = 0) -> list[int]:
    """Per-event N of a workload with drawn sizes, without generating points."""
    w = WORKLOADS[workload]
    if w.n is not None:
        return [w.n] * n_events
    out = []
    for e in range(first, first + n_events):
        rng = np.random.default_rng(seed_of(workload, e))
        out.append(int(rng.integers(w.n_range[0], w.n_range[1] + 1)))
    return out


# --- small generic generators used by the tests -------------------------------

def uniform_grid(n: int, d: int, seed: int, lo: int = -GRID, hi: int = GRID) -> np.ndarray:
    """Uniform points with integer grid coordinates m in [lo, hi], as m/256."""
    rng = np.random.default_rng(seed)
    return (rng.integers(lo, hi + 1, size=(n, d)) / GRID).astype(np.float32)


def clustered_grid(n: int, d: int, seed: int, n_clusters: int, sigma: float,
                   noise_frac: float = 0.0) -> np.ndarray:
    """Isotropic clusters plus uniform noise, quantised to the grid."""
    rng = np.random.default_rng(seed)
    n_noise = int(round(noise_frac * n))
    n_cl = n - n_noise
    lab = rng.integers(0, max(n_clusters, 1), size=n_cl)
    centres = rng.uniform(-1.0, 1.0, size=(max(n_clusters, 1), d))
    pts = centres[lab] + rng.normal(0.0, sigma, size=(n_cl, d))
    noise = rng.uniform(-1.0, 1.0, size=(n_noise, d))
    x = np.concatenate([pts, noise])[rng.permutation(n)]
    return quantise(x)


def uniform_float(n: int, d: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Off-grid float32 points (arbitrary mantissas), uniform in [-scale, scale]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=(n, d)).astype(np.float32)


def duplicates(n: int, d: int, seed: int, n_distinct: int) -> np.ndarray:
    """n points drawn from only n_distinct grid locations (many exact duplicates)."""
    rng = np.random.default_rng(seed)
    base = uniform_grid(n_distinct, d, seed + 1, -8, 8)
    return base[rng.integers(0, n_distinct, size=n)].copy()
