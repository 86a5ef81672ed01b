"""Parity at the benchmark's full sizes, in the launch configuration `bench.py` times (a
dedicated stream, steady iterations replayed as CUDA graphs):

 - the graph-captured fused iterations give the same bits as one-iteration calls (separate
   launches, split advect / resample), on the whole graph;
 - one more iteration in lockstep with the oracle: the whole histogram (every splatted point),
   the whole smoothed-sum stack and the whole density stack against the oracle's; resampling
   and advection on a seeded sample of edges (the oracle recomputes those polylines one by
   one from the GPU's inputs), with the same tolerances and near-tie rules as the small cases;
 - the batched form: sampled member graphs of the 64-graph batch equal their single-graph
   runs bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected only on GPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1504_02687_gb300 as pkg  # noqa: E402
from paper_1504_02687_gb300 import synth  # noqa: E402

from parity import (advect_mismatch, fetch_px, params_for, resample_mismatch,  # noqa: E402
                    rho_as_f64, step_h, sums_as_i64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_02687_gb300 import build

    build.build()
    oracle.build()


def _sub(off, xy, idx):
    """Polylines idx of a CSR set, as their own CSR set."""
    n = np.diff(off)[idx]
    sub_off = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    sub_xy = np.concatenate([xy[off[e]:off[e + 1]] for e in idx])
    return sub_off, sub_xy


WORKLOADS = {
    # configuration 3: 5M edges, 8 k-means groups, 8 x 1024^2 int64 stack, r = 12, k = 4
    "lattice-5M-8groups": lambda: synth.lattice_pattern(),
    # configuration 2: 1M edges, Gaussian-mixture nodes, 1 group, 512^2, r = 8, k = 3
    "clustered-1M": lambda: synth.clustered(),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_full_size_graph_path_and_lockstep(name):
    w = WORKLOADS[name]()
    p = params_for(w)
    stream = torch.cuda.Stream()
    ctx_g = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight, stream=stream)
    ctx_s = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight, stream=stream)
    try:
        pkg.bundle_iterate(ctx_g, 4)          # fused iterations replayed as graphs
        for _ in range(4):
            pkg.bundle_iterate(ctx_s, 1)      # split launches, one call per iteration
        og, xg = pkg.bundle_fetch(ctx_g, pixels=True)
        os_, xs = pkg.bundle_fetch(ctx_s, pixels=True)
        np.testing.assert_array_equal(og, os_)
        np.testing.assert_array_equal(xg, xs)
        for which in (pkg.DENSITY_HIST, pkg.DENSITY_SUMS, pkg.DENSITY_RHO):
            np.testing.assert_array_equal(pkg.bundle_fetch_density(ctx_g, which),
                                          pkg.bundle_fetch_density(ctx_s, which))
        del og, xg, os_, xs
        pkg.bundle_destroy(ctx_g)
        ctx_g = None

        # one more iteration in lockstep with the oracle
        info = pkg.bundle_get_info(ctx_s)
        it = info.iteration
        off0, P0 = fetch_px(ctx_s)
        pkg.bundle_iterate(ctx_s, 1)
        offR, R = fetch_px(ctx_s, resampled=True)
        off1, P1 = fetch_px(ctx_s)
        hist = pkg.bundle_fetch_density(ctx_s, pkg.DENSITY_HIST).astype(np.int64)
        S = sums_as_i64(ctx_s)
        rho = rho_as_f64(ctx_s)
        G, H, W = hist.shape
        extent = max(W, H)
        print(f"{name}: {len(R)} resampled points, {len(P1)} points")
        # every point of the whole graph: histogram, sums, density
        np.testing.assert_array_equal(hist, oracle.splat(offR, R, w.group, w.weight, G, H, W))
        np.testing.assert_array_equal(S, oracle.smooth(hist, p.radius, p.passes))
        rho_o = oracle.combine(S, p.radius, p.passes, p.alpha_num, p.alpha_den)
        np.testing.assert_array_less(np.abs(rho - rho_o), 2.0 ** -21 * np.abs(rho_o) + 1e-35)
        del S, rho_o
        # a seeded sample of edges: resampling and advection recomputed by the oracle
        rng = np.random.default_rng(2024)
        idx = np.sort(rng.choice(w.n_edges, size=20_000, replace=False))
        s_off0, s_P0 = _sub(off0, P0, idx)
        s_offR, s_R = _sub(offR, R, idx)
        s_off1, s_P1 = _sub(off1, P1, idx)
        n_cnt, n_cnt_bad, worst = resample_mismatch(s_off0, s_P0, s_offR, s_R, p, 0)
        assert n_cnt_bad == 0
        assert worst <= 8 * max(p.n_fixed, p.n_max) * 2.0 ** -23 * extent, worst
        grp = w.group[idx] if w.group is not None else None
        h = step_h(p, it)
        n_bad, n_unexp, _ = advect_mismatch(s_offR, s_R, grp, rho, h, p, s_P1, 1e-5 * extent)
        print(f"{name}: sample of {len(idx)} edges, {len(s_R)} points: {n_cnt} count ties, "
              f"{n_bad} advection near-ties")
        assert n_unexp == 0, (n_bad, n_unexp)
        assert n_bad <= max(3, 1e-3 * len(s_R))
        np.testing.assert_array_equal(P1[off1[:-1]], P0[off0[:-1]])   # endpoints never move
        np.testing.assert_array_equal(P1[off1[1:] - 1], P0[off0[1:] - 1])
    finally:
        if ctx_g is not None:
            pkg.bundle_destroy(ctx_g)
        pkg.bundle_destroy(ctx_s)


def test_full_size_batch_members():
    """Configuration 5: the 64-graph batch (one graph launch per iteration); members 0, 31 and
    the largest equal their single-graph runs bit for bit after 4 iterations."""
    ws = synth.batch(n_graphs=64)
    ps = [params_for(w) for w in ws]
    stream = torch.cuda.Stream()
    descs = [dict(src_xy=w.src_xy, dst_xy=w.dst_xy, group=w.group, n_groups=w.n_groups,
                  weight=w.weight) for w in ws]
    b = pkg.bundle_init_batch(descs, ps, stream=stream)
    try:
        pkg.bundle_iterate(b, 4)
        pkg.bundle_sync(b)
        largest = int(np.argmax([w.n_edges for w in ws]))
        for k in sorted({0, 31, largest}):
            m = pkg.bundle_batch_member(b, k)
            c = pkg.bundle_init(ps[k], ws[k].src_xy, ws[k].dst_xy, ws[k].group, ws[k].n_groups,
                                ws[k].weight, stream=stream)
            try:
                pkg.bundle_iterate(c, 4)
                o1, x1 = pkg.bundle_fetch(m, pixels=True)
                o2, x2 = pkg.bundle_fetch(c, pixels=True)
                np.testing.assert_array_equal(o1, o2)
                np.testing.assert_array_equal(x1, x2)
                np.testing.assert_array_equal(pkg.bundle_fetch_density(m, pkg.DENSITY_SUMS),
                                              pkg.bundle_fetch_density(c, pkg.DENSITY_SUMS))
            finally:
                pkg.bundle_destroy(c)
    finally:
        pkg.bundle_destroy(b)
