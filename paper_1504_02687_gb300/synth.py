"""Seeded synthetic graphs shaped like the paper's benchmark graphs.

The paper times public graphs (UF sparse-matrix layouts, US migration,
airlines, yeast); none are available here, so these seeded generators stand in
for them with the same sizes (edges, groups, samples per edge) and structure
(clustered layouts, pattern-like lattices, k-means groups on origin and
destination, as in Sec. 5). This module holds graph generation only, none of
the bundling arithmetic; the CUDA path and the CPU oracle both consume its
output.

Every workload returns world coordinates in [0, 1]^2 (float32), int32 group
ids and optional int32 weights, plus the bundling parameters of that workload.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1504


@dataclass
class Workload:
    name: str
    src_xy: np.ndarray          # float32 [E, 2], world coordinates
    dst_xy: np.ndarray          # float32 [E, 2]
    group: np.ndarray           # int32 [E]
    n_groups: int
    weight: np.ndarray | None   # int32 [E] or None (all ones)
    grid: tuple[int, int]       # (W, H)
    radius: int
    passes: int
    n_fixed: int
    n_max: int
    delta: float
    iters: int
    extra: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.src_xy.shape[0])


def _distinct_pairs(rng, n_nodes, n_edges):
    s = rng.integers(0, n_nodes, n_edges)
    t = rng.integers(0, n_nodes - 1, n_edges)
    t = t + (t >= s)  # never a self-loop
    return s, t


def kmeans_groups(feat: np.ndarray, k: int, seed: int, steps: int = 20) -> np.ndarray:
    """Seeded k-means++ initialisation and `steps` Lloyd iterations (Sec. 5's grouping
    criterion); returns int32 labels. Used only to make group ids for synthetic inputs."""
    rng = np.random.default_rng(seed)
    x = np.ascontiguousarray(feat, np.float32)
    n = x.shape[0]
    sample = x if n <= 200_000 else x[rng.choice(n, 200_000, replace=False)]
    cent = [sample[rng.integers(sample.shape[0])]]
    d2 = ((sample - cent[0]) ** 2).sum(1)
    for _ in range(1, k):
        p = d2 / d2.sum()
        c = sample[rng.choice(sample.shape[0], p=p)]
        cent.append(c)
        d2 = np.minimum(d2, ((sample - c) ** 2).sum(1))
    cent = np.stack(cent).astype(np.float32)
    labels = np.zeros(n, np.int32)
    chunk = 1 << 20
    for _ in range(steps):
        for i in range(0, n, chunk):
            xc = x[i:i + chunk]
            d = (xc * xc).sum(1)[:, None] - 2 * xc @ cent.T + (cent * cent).sum(1)[None]
            labels[i:i + chunk] = d.argmin(1)
        for j in range(k):
            m = labels == j
            if m.any():
                cent[j] = x[m].mean(0)
    return labels


def small(seed: int = SEED_BASE + 1, n_edges: int = 2000, n_nodes: int = 500) -> Workload:
    """Plain method, small: straight edges between nodes uniform in [0, 1]^2, one group,
    256 x 256 grid, r = 4, 3 passes, 32 samples per edge, 10 iterations."""
    rng = np.random.default_rng(seed)
    nodes = rng.uniform(0, 1, (n_nodes, 2)).astype(np.float32)
    s, t = _distinct_pairs(rng, n_nodes, n_edges)
    return Workload("small-2k-edges-1-group", nodes[s], nodes[t], np.zeros(n_edges, np.int32), 1,
                    None, (256, 256), 4, 3, 32, 64, 2.0, 10)


def clustered(seed: int = SEED_BASE + 2, n_edges: int = 1_000_000, n_nodes: int = 100_000,
              n_comp: int = 20, sigma: float = 0.03, intra: float = 0.7, grid=(512, 512),
              radius: int = 8, passes: int = 3, n_groups: int = 1, iters: int = 20) -> Workload:
    """Spatial-only, large: nodes from a Gaussian mixture (centres uniform in [0.1, 0.9]^2),
    uniform sources, targets in the source's component with probability `intra`."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.1, 0.9, (n_comp, 2))
    comp = rng.integers(0, n_comp, n_nodes)
    nodes = np.clip(centres[comp] + rng.normal(0, sigma, (n_nodes, 2)), 0, 1).astype(np.float32)
    members = [np.flatnonzero(comp == c) for c in range(n_comp)]
    s = rng.integers(0, n_nodes, n_edges)
    t = rng.integers(0, n_nodes, n_edges)
    same = rng.random(n_edges) < intra
    for c in range(n_comp):
        m = np.flatnonzero(same & (comp[s] == c))
        if len(members[c]) > 1 and len(m):
            t[m] = members[c][rng.integers(0, len(members[c]), len(m))]
    loops = s == t
    t[loops] = (t[loops] + 1) % n_nodes
    group = np.zeros(n_edges, np.int32)
    if n_groups > 1:
        feat = np.concatenate([nodes[s], nodes[t]], 1)
        group = kmeans_groups(feat, n_groups, seed)
    return Workload(f"clustered-{n_edges}-edges-{n_groups}-groups", nodes[s], nodes[t], group,
                    n_groups, None, grid, radius, passes, 0, 64, 2.0, iters)


def lattice_pattern(seed: int = SEED_BASE + 3, n_edges: int = 5_000_000, side: int = 2048,
                    n_groups: int = 8, grid=(1024, 1024), radius: int = 12, passes: int = 4,
                    iters: int = 30, kmeans_steps: int = 20) -> Workload:
    """Criteria-driven: nodes on a perturbed side x side lattice; each edge joins a uniform
    source to the lattice node at a log-uniform offset (1..256 lattice units) along one of 8
    pattern directions +-5 degrees; groups from k-means on (origin, destination)."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, side, n_edges)
    j = rng.integers(0, side, n_edges)
    ell = np.exp(rng.uniform(0.0, math.log(256.0), n_edges))
    ang = (rng.integers(0, 8, n_edges) * (math.pi / 4)
           + np.deg2rad(rng.uniform(-5.0, 5.0, n_edges)))
    ti = np.rint(i + ell * np.cos(ang)).astype(np.int64)
    tj = np.rint(j + ell * np.sin(ang)).astype(np.int64)
    # reflect targets that leave the lattice back inside it
    ti = np.where(ti < 0, -ti, ti)
    ti = np.where(ti >= side, 2 * (side - 1) - ti, ti)
    tj = np.where(tj < 0, -tj, tj)
    tj = np.where(tj >= side, 2 * (side - 1) - tj, tj)
    same = (ti == i) & (tj == j)
    ti[same] = np.where(i[same] + 1 < side, i[same] + 1, i[same] - 1)

    def node_xy(a, b, r):
        jit = rng.normal(0.0, 0.3 / side, (a.shape[0], 2))
        return np.column_stack([(a + 0.5) / side, (b + 0.5) / side]) + jit

    src = node_xy(i, j, rng).astype(np.float32)
    dst = node_xy(ti, tj, rng).astype(np.float32)
    group = np.zeros(n_edges, np.int32)
    if n_groups > 1:
        group = kmeans_groups(np.concatenate([src, dst], 1), n_groups, seed, kmeans_steps)
    return Workload(f"lattice-pattern-{n_edges}-edges-{n_groups}-groups", src, dst, group,
                    n_groups, None, grid, radius, passes, 0, 64, 2.0, iters)


def tiny(seed: int, n_edges: int, n_groups: int = 1, grid=(96, 80), radius: int = 3,
         passes: int = 3, n_fixed: int = 0, n_max: int = 24, delta: float = 2.0,
         weighted: bool = False, iters: int = 3) -> Workload:
    """Small uniform random graph for parity tests (several tiles plus a ragged tail)."""
    rng = np.random.default_rng(seed)
    src = rng.uniform(0, 1, (n_edges, 2)).astype(np.float32)
    dst = rng.uniform(0, 1, (n_edges, 2)).astype(np.float32)
    group = rng.integers(0, n_groups, n_edges).astype(np.int32)
    weight = rng.integers(1, 5, n_edges).astype(np.int32) if weighted else None
    return Workload(f"tiny-{n_edges}-{n_groups}", src, dst, group, n_groups, weight, grid, radius,
                    passes, n_fixed, n_max, delta, iters)


def batch(seed: int = SEED_BASE + 5, n_graphs: int = 64, e_lo: int = 10_000,
          e_hi: int = 500_000) -> list[Workload]:
    """Batched form: graphs with log-uniform edge counts, 1..16 groups, grids 256^2 / 512^2 /
    1024^2 and radius 4..12, each from the clustered generator with its own seed."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_graphs):
        e = int(math.exp(rng.uniform(math.log(e_lo), math.log(e_hi))))
        g = int(rng.integers(1, 17))
        side = int(rng.choice([256, 512, 1024]))
        r = int(rng.integers(4, 13))
        w = clustered(seed=seed * 1000 + k, n_edges=e, n_nodes=max(1000, e // 10),
                      grid=(side, side), radius=r, passes=3, n_groups=g, iters=20)
        w.name = f"batch{k}-{e}-edges-{g}-groups-{side}"
        out.append(w)
    return out


def by_name(name: str) -> Workload:
    return {"small": small, "clustered": clustered, "lattice": lattice_pattern}[name]()
