"""CUDA path vs the FP64 oracle, through the C ABI, on seeded synthetic graphs.

Sizes span many blocks of up to 32 edges (one warp each) plus a ragged tail and finish in seconds on the
oracle. Integer stages are bit-exact; floating-point stages are within the stated bounds:
 - density rho: one rounding of an exact integer to FP32 plus one FP32 division,
   |rho_gpu - rho| <= 4 ulp(rho) (relative 2^-21);
 - positions in lockstep: 1e-5 of the grid extent, with every larger difference traced to a
   verified near-tie decision (see parity.advect_mismatch);
 - free-running positions: RMS within 1e-4 of the layout extent (the stated FP32 tolerance), the
   maximum reported.
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

from parity import (advect_mismatch, fetch_px, oracle_params, params_for,  # noqa: E402
                    resample_mismatch, rho_as_f64, step_h, sums_as_i64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_02687_gb300 import build

    build.build()
    oracle.build()


WORKLOADS = {
    "g1-fixed32": dict(seed=11, n_edges=1000, n_groups=1, grid=(96, 80), radius=3, passes=3,
                       n_fixed=32),
    "g3-bylength-weighted": dict(seed=12, n_edges=777, n_groups=3, grid=(128, 96), radius=4,
                                 passes=3, n_fixed=0, n_max=24, weighted=True),
    "g5-bylength-r2k4": dict(seed=13, n_edges=300, n_groups=5, grid=(64, 64), radius=2, passes=4,
                             n_fixed=0, n_max=16, delta=1.5),
}


def _make(name, **over):
    w = synth.tiny(**WORKLOADS[name])
    p = params_for(w, **over)
    ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    return w, p, ctx


def test_grid_map_matches_oracle_bit_for_bit():
    w, p, ctx = _make("g3-bylength-weighted")
    try:
        off, xy = pkg.bundle_fetch(ctx, pixels=True)
        W, H, mp, sp, dp = oracle.grid_map(w.src_xy, w.dst_xy, w.grid[0], w.grid[1],
                                           margin=p.radius)
        np.testing.assert_array_equal(np.diff(off), 2)
        np.testing.assert_array_equal(xy[0::2], sp)
        np.testing.assert_array_equal(xy[1::2], dp)
        info = pkg.bundle_get_info(ctx)
        assert list(info.map) == list(mp)
        # world coordinates come back through the inverse map
        off2, xyw = pkg.bundle_fetch(ctx)
        np.testing.assert_allclose(xyw[0::2], w.src_xy, atol=1e-5)
    finally:
        pkg.bundle_destroy(ctx)


def _lockstep_once(ctx, w, p, max_bad_frac=1e-3, M=None):
    """One GPU iteration from the GPU's current state, every stage checked against the oracle."""
    info = pkg.bundle_get_info(ctx)
    it = info.iteration
    off0, P0 = fetch_px(ctx)
    pkg.bundle_iterate(ctx, 1)
    offR, R = fetch_px(ctx, resampled=True)
    hist = pkg.bundle_fetch_density(ctx, pkg.DENSITY_HIST).astype(np.int64)
    S = sums_as_i64(ctx)
    rho = rho_as_f64(ctx)
    off1, P1 = fetch_px(ctx)
    G, H, W = hist.shape
    extent = max(W, H)
    # resampling (Sec. 2.1): counts exact up to verified ties, positions to FP32 rounding
    dpx = float(p.directed_offset) * extent if it == 0 else 0.0
    n_cnt, n_cnt_bad, worst = resample_mismatch(off0, P0, offR, R, p, 0, dpx, (W, H))
    assert n_cnt_bad == 0
    # FP32 arc-length sums: a few ulps of the extent per point of the polyline
    assert worst <= 8 * max(p.n_fixed, p.n_max) * 2.0 ** -23 * extent, worst
    # histogram of the GPU's resampled points (Eq. 1, Eq. 3): bit for bit
    group = w.group
    if p.flags & pkg.FLAG_SEGMENT_HIST:
        np.testing.assert_array_equal(hist, oracle.splat_segments(offR, R, group, w.weight,
                                                                  G, H, W))
    else:
        np.testing.assert_array_equal(hist, oracle.splat(offR, R, group, w.weight, G, H, W))
        assert hist.sum() == (np.diff(offR) * (w.weight if w.weight is not None else 1)).sum()
    # box passes (Sec. 3.1): bit for bit
    np.testing.assert_array_equal(S, oracle.smooth(hist, p.radius, p.passes))
    # layer mix (Eq. 3, Eq. 4): exact integer numerator, one FP32 rounding and division
    if M is None:
        rho_o = oracle.combine(S, p.radius, p.passes, p.alpha_num, p.alpha_den)
    else:
        rho_o = oracle.combine_matrix(S, p.radius, p.passes, M)
    rel, absl = {pkg.RHO_F32: (2.0 ** -21, 1e-35), pkg.RHO_BF16: (2.0 ** -8, 1e-35),
                 pkg.RHO_F16: (2.0 ** -10, 2.0 ** -24)}[info.rho_dtype]
    np.testing.assert_array_less(np.abs(rho - rho_o), rel * np.abs(rho_o) + absl)
    # advection + Laplacian (Eq. 5, Sec. 3.3) from the GPU's R and rho
    h = step_h(p, it)
    n_bad, n_unexp, P_o = advect_mismatch(offR, R, group, rho, h, p, P1, 1e-5 * extent)
    assert n_unexp == 0, (n_bad, n_unexp)
    assert n_bad <= max(3, max_bad_frac * len(R))
    np.testing.assert_array_equal(np.diff(off1), np.diff(offR))
    # endpoints never move
    np.testing.assert_array_equal(P1[off1[:-1]], P0[off0[:-1]])
    np.testing.assert_array_equal(P1[off1[1:] - 1], P0[off0[1:] - 1])
    return n_bad, n_cnt


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_lockstep_stages(name):
    w, p, ctx = _make(name)
    try:
        _lockstep_once(ctx, w, p)          # iteration 0, from straight edges
        pkg.bundle_iterate(ctx, 2)
        _lockstep_once(ctx, w, p)          # iteration 3, from bundled polylines
    finally:
        pkg.bundle_destroy(ctx)


@pytest.mark.parametrize("rho_dtype", [pkg.RHO_BF16, pkg.RHO_F16])
def test_lockstep_reduced_precision_density(rho_dtype):
    """BF16/FP16 storage of rho: the integer stages stay bit-exact; the stored density is the
    exact value rounded once more to the storage type; advection is checked from it."""
    w, p, ctx = _make("g3-bylength-weighted", rho_dtype=rho_dtype)
    try:
        pkg.bundle_iterate(ctx, 1)
        S = sums_as_i64(ctx)
        rho = rho_as_f64(ctx)
        rho_o = oracle.combine(S, p.radius, p.passes, p.alpha_num, p.alpha_den)
        rel, absl = (2.0 ** -8, 1e-35) if rho_dtype == pkg.RHO_BF16 else (2.0 ** -10, 2.0 ** -24)
        np.testing.assert_array_less(np.abs(rho - rho_o), rel * np.abs(rho_o) + absl)
        _lockstep_once(ctx, w, p)
    finally:
        pkg.bundle_destroy(ctx)


def test_fused_sequence_equals_split_and_resume():
    """The fused advect -> resample -> splat kernel used inside one bundle_iterate(n) gives the
    same bits as n single iterations, and as a context resumed from fetched polylines."""
    w = synth.tiny(**WORKLOADS["g3-bylength-weighted"])
    p = params_for(w)
    a = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    b = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    try:
        pkg.bundle_iterate(a, 2)
        mid_off, mid_xy = pkg.bundle_fetch(a, pixels=True)
        pkg.bundle_iterate(a, 3)
        for _ in range(5):
            pkg.bundle_iterate(b, 1)
        oa, xa = pkg.bundle_fetch(a, pixels=True)
        ob, xb = pkg.bundle_fetch(b, pixels=True)
        np.testing.assert_array_equal(oa, ob)
        np.testing.assert_array_equal(xa, xb)
        for which in (pkg.DENSITY_HIST, pkg.DENSITY_SUMS, pkg.DENSITY_RHO):
            np.testing.assert_array_equal(pkg.bundle_fetch_density(a, which),
                                          pkg.bundle_fetch_density(b, which))
        info = pkg.bundle_get_info(a)
        c = pkg.bundle_init_polylines(params_for(w), mid_off, mid_xy, w.group, w.n_groups,
                                      w.weight, map5=np.array(info.map), iteration=2)
        try:
            pkg.bundle_iterate(c, 3)
            oc, xc = pkg.bundle_fetch(c, pixels=True)
            np.testing.assert_array_equal(oc, oa)
            np.testing.assert_array_equal(xc, xa)
        finally:
            pkg.bundle_destroy(c)
    finally:
        pkg.bundle_destroy(a)
        pkg.bundle_destroy(b)


def _ulp_perturbed(xy, seed):
    """Move every coordinate by -1, 0 or +1 FP32 ulp (seeded)."""
    rng = np.random.default_rng(seed)
    x32 = xy.astype(np.float32)
    d = rng.integers(-1, 2, x32.shape)
    up, dn = np.nextafter(x32, np.float32(1e9)), np.nextafter(x32, np.float32(-1e9))
    return np.where(d > 0, up, np.where(d < 0, dn, x32)).astype(np.float64)


def test_free_running_small_config():
    """The small configuration (2,000 edges, 256^2, r = 4, k = 3, 32 points, 10 iterations),
    GPU FP32 vs FP64 oracle from the same start.

    After one iteration the RMS position error is within 1e-4 of the extent. Over many
    iterations the method itself amplifies ulp-level differences through its discrete
    decisions (cell of a point, accepted step): two FP64 oracle runs whose endpoints differ
    by +-1 FP32 ulp drift apart by ~2e-3 of the extent RMS after 10 iterations. The GPU must
    stay inside that envelope of the method's own sensitivity."""
    w = synth.small()
    p = params_for(w)
    ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    try:
        off0, P0 = fetch_px(ctx)
        pkg.bundle_iterate(ctx, 1)
        off1, P1 = fetch_px(ctx)
        pkg.bundle_iterate(ctx, w.iters - 1)
        off, P = fetch_px(ctx)
    finally:
        pkg.bundle_destroy(ctx)
    prm = oracle_params(p)
    one = oracle.run(off0, P0, w.group, w.weight, 1, 256, 256, prm, 0, 1)
    err1 = np.hypot(*(P1 - one.xy).T) / 256.0
    rms1 = float(np.sqrt((err1 ** 2).mean()))
    assert rms1 <= 1e-4, rms1
    res = oracle.run(off0, P0, w.group, w.weight, 1, 256, 256, prm, 0, w.iters)
    np.testing.assert_array_equal(off, res.off)
    err = np.hypot(*(P - res.xy).T) / 256.0
    rms = float(np.sqrt((err ** 2).mean()))
    env_rms, env_max = [], []
    for seed in (0, 1):
        alt = oracle.run(off0, _ulp_perturbed(P0, seed), w.group, w.weight, 1, 256, 256, prm, 0,
                         w.iters)
        e = np.hypot(*(alt.xy - res.xy).T) / 256.0
        env_rms.append(float(np.sqrt((e ** 2).mean())))
        env_max.append(float(e.max()))
    print(f"free-running small: 1 iteration rms {rms1:.2e} max {err1.max():.2e}; "
          f"{w.iters} iterations rms {rms:.2e} max {err.max():.2e}; FP64 +-1ulp envelope rms "
          f"{env_rms} max {env_max} (units of the extent)")
    assert rms <= 1.5 * max(env_rms)
    assert err.max() <= 1.5 * max(env_max)


def test_edge_cases():
    # one edge; an edge on the border; maximum radius; 64 groups with few edges; int64 sums
    # forced on a small case; zero weights
    rng = np.random.default_rng(99)
    cases = []
    cases.append((np.array([[0.1, 0.2]], np.float32), np.array([[0.9, 0.7]], np.float32), None,
                  1, None, dict(grid_w=32, grid_h=32, radius=2, n_fixed=8)))
    E = 130
    s = rng.uniform(0, 1, (E, 2)).astype(np.float32)
    d = rng.uniform(0, 1, (E, 2)).astype(np.float32)
    s[:10, 0] = 0.0
    d[:10, 0] = 0.0
    cases.append((s, d, (np.arange(E) % 64).astype(np.int32), 64, None,
                  dict(grid_w=40, grid_h=24, radius=23, margin_px=0, n_fixed=0, n_max=12)))
    wts = rng.integers(0, 3, E).astype(np.int32)
    cases.append((s, d, None, 1, wts, dict(grid_w=50, grid_h=70, radius=3, sum_bits=64,
                                           n_fixed=6)))
    for (src, dst, g, G, wt, over) in cases:
        p = pkg.default_params(**over)
        ctx = pkg.bundle_init(p, src, dst, g, G, wt)
        try:
            class Wk:
                group, weight = g, wt
            # a radius near the grid size makes the density almost flat: many directions are
            # ill-conditioned in FP32; each such mismatch must still be a verified ambiguity
            _lockstep_once(ctx, Wk, p, max_bad_frac=0.05)
            _lockstep_once(ctx, Wk, p, max_bad_frac=0.05)
        finally:
            pkg.bundle_destroy(ctx)


def test_degenerate_and_maximum_sizes():
    """Zero-length and duplicate edges; the largest grid (4096^2: the generic row pass and the
    narrowest column strip) with the largest polylines (64 points); a ragged, odd-sized grid
    (4093 x 61: element-wise copies in both filter passes)."""
    rng = np.random.default_rng(7)

    class Wk:
        group = weight = None

    E = 500
    s = rng.uniform(0, 1, (E, 2)).astype(np.float32)
    d = s.copy()                                  # every edge has zero length ...
    d[::3] = rng.uniform(0, 1, (len(d[::3]), 2))  # ... except one in three
    s[100:150] = s[100]                           # 50 duplicates of one edge
    d[100:150] = d[100]
    cases = [(s, d, dict(grid_w=96, grid_h=96, radius=3, n_fixed=0, n_max=16)),
             (rng.uniform(0, 1, (2000, 2)).astype(np.float32),
              rng.uniform(0, 1, (2000, 2)).astype(np.float32),
              dict(grid_w=4096, grid_h=4096, radius=4, passes=3, n_fixed=64)),
             (rng.uniform(0, 1, (1500, 2)).astype(np.float32),
              rng.uniform(0, 1, (1500, 2)).astype(np.float32),
              dict(grid_w=4093, grid_h=61, radius=5, passes=3, n_fixed=0, n_max=64))]
    for src, dst, over in cases:
        p = pkg.default_params(**over)
        ctx = pkg.bundle_init(p, src, dst)
        try:
            _lockstep_once(ctx, Wk, p, max_bad_frac=0.01)
            _lockstep_once(ctx, Wk, p, max_bad_frac=0.01)
            off, xy = pkg.bundle_fetch(ctx, pixels=True)
            n = np.diff(off)
            zero = np.flatnonzero((src == dst).all(axis=1))
            if len(zero) and p.n_fixed == 0:
                assert (n[zero] == 2).all()        # L = 0: two points, both on the source
        finally:
            pkg.bundle_destroy(ctx)


def test_device_inputs_and_outputs():
    w = synth.tiny(**WORKLOADS["g1-fixed32"])
    p = params_for(w)
    dev = torch.device("cuda:0")
    ctx_h = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    ctx_d = pkg.bundle_init(p, torch.from_numpy(w.src_xy).to(dev), torch.from_numpy(w.dst_xy).to(dev),
                            torch.from_numpy(w.group).to(dev), w.n_groups, None,
                            stream=torch.cuda.current_stream())
    try:
        pkg.bundle_iterate(ctx_h, 2)
        pkg.bundle_iterate(ctx_d, 2)
        off_h, xy_h = pkg.bundle_fetch(ctx_h)
        info = pkg.bundle_get_info(ctx_d)
        off_d = torch.zeros(info.n_edges + 1, dtype=torch.int64, device=dev)
        xy_d = torch.zeros((info.n_points, 2), dtype=torch.float32, device=dev)
        pkg.bundle_fetch(ctx_d, off=off_d, xy=xy_d)
        np.testing.assert_array_equal(off_d.cpu().numpy(), off_h)
        np.testing.assert_array_equal(xy_d.cpu().numpy(), xy_h)
    finally:
        pkg.bundle_destroy(ctx_h)
        pkg.bundle_destroy(ctx_d)


def test_variants_fixed_step_directed_offset():
    """KDEEB's fixed step (Sec. 3.3) and the directed-graph normal offset (Sec. 3), checked
    stage by stage against the oracle's variants."""
    for over in (dict(flags=pkg.FLAG_FIXED_STEP), dict(directed_offset=0.004)):
        w, p, ctx = _make("g3-bylength-weighted", **over)
        try:
            _lockstep_once(ctx, w, p)
            _lockstep_once(ctx, w, p)
        finally:
            pkg.bundle_destroy(ctx)


@pytest.mark.parametrize("name", ["g1-fixed32", "g3-bylength-weighted"])
def test_segment_histogram_lockstep(name):
    """Histogram by Bresenham segments (Eq. 1 as rasterised in Sec. 4): every stage of two
    iterations from straight edges and one from bundled polylines against the oracle."""
    w, p, ctx = _make(name, flags=pkg.FLAG_SEGMENT_HIST)
    try:
        _lockstep_once(ctx, w, p)
        _lockstep_once(ctx, w, p)
        pkg.bundle_iterate(ctx, 2)
        _lockstep_once(ctx, w, p)
        pkg.bundle_sync(ctx)
    finally:
        pkg.bundle_destroy(ctx)


def test_segment_histogram_mass_overflow_is_reported():
    """With r = 3 and k = 16 the int64 sums hold no segment mass at all: the device check
    flags the first iteration and the next sync reports it (sums wrap modulo 2^64 on the
    device, nothing faults)."""
    w, p, ctx = _make("g1-fixed32", flags=pkg.FLAG_SEGMENT_HIST, radius=3, passes=16)
    try:
        pkg.bundle_iterate(ctx, 1)
        with pytest.raises(pkg.BundleError, match="segment histogram") as ei:
            pkg.bundle_sync(ctx)
        assert ei.value.status == pkg.BUNDLE_EOVERFLOW
    finally:
        pkg.bundle_destroy(ctx)


def test_ink_record_matches_histograms():
    """The convergence record (occupied cells per iteration) equals the counts of the fetched
    histogram at every iteration, and the captured-graph path records the same numbers."""
    for flags in (pkg.FLAG_INK_STATS, pkg.FLAG_INK_STATS | pkg.FLAG_SEGMENT_HIST):
        w, p, ctx = _make("g3-bylength-weighted", flags=flags)
        w2, p2, ctx2 = _make("g3-bylength-weighted", flags=flags)
        try:
            expect = []
            for _ in range(4):
                pkg.bundle_iterate(ctx, 1)
                expect.append(oracle.ink(pkg.bundle_fetch_density(ctx, pkg.DENSITY_HIST)))
            np.testing.assert_array_equal(pkg.bundle_fetch_ink(ctx, 0, 4), np.array(expect))
            pkg.bundle_iterate(ctx2, 4)          # one call: steady iterations through graphs
            np.testing.assert_array_equal(pkg.bundle_fetch_ink(ctx2, 0, 4), np.array(expect))
            with pytest.raises(pkg.BundleError) as ei:
                pkg.bundle_fetch_ink(ctx2, 2, 3)
            assert ei.value.status == pkg.BUNDLE_EINVAL
        finally:
            pkg.bundle_destroy(ctx)
            pkg.bundle_destroy(ctx2)
    w, p, ctx = _make("g1-fixed32")
    try:
        pkg.bundle_iterate(ctx, 1)
        with pytest.raises(pkg.BundleError) as ei:
            pkg.bundle_fetch_ink(ctx, 0, 1)
        assert ei.value.status == pkg.BUNDLE_ESTATE
    finally:
        pkg.bundle_destroy(ctx)


def test_optimised_step_converges_in_fewer_iterations():
    """Sec. 3.3 / Fig. 3 on the CUDA path: the ink of the segment-rasterised drawing falls
    faster with the density test than with KDEEB's fixed step (1,000-edge uniform graph)."""
    w = synth.small(n_edges=1000)
    ink = {}
    for fixed in (0, pkg.FLAG_FIXED_STEP):
        p = params_for(w, flags=fixed | pkg.FLAG_SEGMENT_HIST | pkg.FLAG_INK_STATS)
        ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
        try:
            pkg.bundle_iterate(ctx, 10)
            ink[fixed] = pkg.bundle_fetch_ink(ctx, 0, 10)[:, 0]
        finally:
            pkg.bundle_destroy(ctx)
    opt, fix = ink[0], ink[pkg.FLAG_FIXED_STEP]
    print("ink optimised", opt.tolist(), "fixed", fix.tolist())
    assert opt[0] == fix[0]
    assert (opt[1:] < fix[1:]).all()
    assert np.flatnonzero(opt <= fix[-1])[0] <= 8


def _state(ctx):
    off, xy = pkg.bundle_fetch(ctx, pixels=True)
    return [off, xy] + [pkg.bundle_fetch_density(ctx, k) for k in
                        (pkg.DENSITY_HIST, pkg.DENSITY_SUMS, pkg.DENSITY_RHO)]


def test_every_tile_choice_gives_the_same_bits():
    """Edges per block, row-pass variant and column-pass strip change only the schedule: after
    3 iterations (graph path included) every combination equals the default bit for bit."""
    w = synth.tiny(seed=21, n_edges=900, n_groups=3, grid=(256, 240), radius=5, passes=3,
                   n_fixed=0, n_max=32, weighted=True)
    p = params_for(w)
    ref = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    try:
        pkg.bundle_iterate(ref, 3)
        expect = _state(ref)
    finally:
        pkg.bundle_destroy(ref)
    for eb in (4, 8, 16, 32):
        for row in (1, 2):
            for strip in (2, 4, 8, 16):
                ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
                try:
                    pkg.bundle_set_tiles(ctx, eb, row, strip)
                    info = pkg.bundle_get_info(ctx)
                    assert (info.tile_eb, info.tile_row, info.tile_strip) == (eb, row, strip)
                    pkg.bundle_iterate(ctx, 3)
                    for a, b in zip(_state(ctx), expect):
                        np.testing.assert_array_equal(a, b)
                finally:
                    pkg.bundle_destroy(ctx)


def test_autotune_keeps_results_and_states():
    w = synth.tiny(seed=22, n_edges=1200, n_groups=2, grid=(256, 256), radius=4, passes=3,
                   n_fixed=0, n_max=24)
    p = params_for(w, flags=pkg.FLAG_INK_STATS)
    a = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    b = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    try:
        pkg.bundle_autotune(b)
        info = pkg.bundle_get_info(b)
        print("autotuned tiles:", info.tile_eb, info.tile_row, info.tile_strip)
        assert info.iteration == 0 and info.points_processed == 0
        assert info.tile_eb in (4, 8, 16, 32) and info.tile_strip in (2, 4, 8, 16)
        pkg.bundle_iterate(a, 4)
        pkg.bundle_iterate(b, 4)
        for x, y in zip(_state(a), _state(b)):
            np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(pkg.bundle_fetch_ink(a, 0, 4), pkg.bundle_fetch_ink(b, 0, 4))
        with pytest.raises(pkg.BundleError) as ei:   # only before the first iteration
            pkg.bundle_autotune(b)
        assert ei.value.status == pkg.BUNDLE_ESTATE
        with pytest.raises(pkg.BundleError) as ei:
            pkg.bundle_set_tiles(b, 32, 0, 0)
        assert ei.value.status == pkg.BUNDLE_ESTATE
    finally:
        pkg.bundle_destroy(a)
        pkg.bundle_destroy(b)
    # a batch tunes each graph on its own edges; results equal the untuned batch
    ws = [synth.tiny(seed=30 + k, n_edges=n, n_groups=g, grid=(128, 128), radius=3, passes=3)
          for k, (n, g) in enumerate([(300, 1), (1500, 3), (700, 2)])]
    descs = [dict(src_xy=x.src_xy, dst_xy=x.dst_xy, group=x.group, n_groups=x.n_groups,
                  weight=x.weight) for x in ws]
    ps = [params_for(x) for x in ws]
    b1 = pkg.bundle_init_batch(descs, ps)
    b2 = pkg.bundle_init_batch(descs, ps)
    try:
        pkg.bundle_autotune(b2)
        pkg.bundle_iterate(b1, 3)
        pkg.bundle_iterate(b2, 3)
        for k in range(len(ws)):
            for x, y in zip(_state(pkg.bundle_batch_member(b1, k)),
                            _state(pkg.bundle_batch_member(b2, k))):
                np.testing.assert_array_equal(x, y)
    finally:
        pkg.bundle_destroy(b1)
        pkg.bundle_destroy(b2)


def test_optimised_step_never_lowers_density():
    """Sec. 3.3: the halving step guarantees every advected point a density not lower than
    before; KDEEB's fixed step does not (beta = 0 so the advected points are the output)."""
    dec = {}
    for flags in (0, pkg.FLAG_FIXED_STEP):
        w, p, ctx = _make("g1-fixed32", laplace_beta=0.0, flags=flags)
        try:
            pkg.bundle_iterate(ctx, 2)
            pkg.bundle_iterate(ctx, 1)
            offR, R = fetch_px(ctx, resampled=True)
            rho = rho_as_f64(ctx)
            off1, P1 = fetch_px(ctx)
        finally:
            pkg.bundle_destroy(ctx)
        r0, _ = oracle.density_at(rho[0], R)
        r1, _ = oracle.density_at(rho[0], P1)
        interior = np.ones(len(R), bool)
        interior[offR[:-1]] = False
        interior[offR[1:] - 1] = False
        drop = (r1 < r0 - 1e-5 * np.abs(r0) - 1e-30) & interior
        dec[flags] = int(drop.sum())
    assert dec[0] == 0
    assert dec[pkg.FLAG_FIXED_STEP] > 0


def test_interaction_matrix():
    """Eq. 4 written as a general matrix reproduces the default mix bit for bit; an ordinal
    matrix (Sec. 3.2) is checked against the oracle's matrix mix."""
    w, p, ctx = _make("g3-bylength-weighted")
    w2, p2, ctx2 = _make("g3-bylength-weighted")
    try:
        G = w.n_groups
        num = np.full((G, G), -1, np.int64)  # alpha = 1/4, B - 1 = 2: -1/8 off the diagonal
        np.fill_diagonal(num, 8)
        pkg.bundle_set_interaction(ctx2, num, 8)
        pkg.bundle_iterate(ctx, 3)
        pkg.bundle_iterate(ctx2, 3)
        np.testing.assert_array_equal(pkg.bundle_fetch_density(ctx, pkg.DENSITY_RHO),
                                      pkg.bundle_fetch_density(ctx2, pkg.DENSITY_RHO))
        np.testing.assert_array_equal(pkg.bundle_fetch(ctx, pixels=True)[1],
                                      pkg.bundle_fetch(ctx2, pixels=True)[1])
        ordinal = np.array([[4, 2, -1], [2, 4, 2], [-1, 2, 4]], np.int64)
        pkg.bundle_set_interaction(ctx2, ordinal, 4)
        _lockstep_once(ctx2, w2, p2, M=ordinal / 4.0)
    finally:
        pkg.bundle_destroy(ctx)
        pkg.bundle_destroy(ctx2)


def test_graph_path_equals_separate_launches():
    """Steady-state iterations run as CUDA graphs unless per-kernel profiling is on; both
    paths give the same bits."""
    w = synth.tiny(**WORKLOADS["g5-bylength-r2k4"])
    p = params_for(w)
    a = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    b = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    try:
        pkg.bundle_profile_enable(b, True)
        pkg.bundle_iterate(a, 6)
        pkg.bundle_iterate(b, 6)
        np.testing.assert_array_equal(pkg.bundle_fetch(a, pixels=True)[1],
                                      pkg.bundle_fetch(b, pixels=True)[1])
        np.testing.assert_array_equal(pkg.bundle_fetch_density(a, pkg.DENSITY_RHO),
                                      pkg.bundle_fetch_density(b, pkg.DENSITY_RHO))
        assert pkg.bundle_get_info(a).iteration == 6
    finally:
        pkg.bundle_destroy(a)
        pkg.bundle_destroy(b)


def test_batch_members_equal_single_runs():
    """A batch of graphs with different grids, groups and parameters gives, for each graph,
    the same bits as that graph bundled alone -- through the batch graph (one CUDA graph per
    iteration for all members) and through separate launches (profiling on)."""
    names = ["g1-fixed32", "g3-bylength-weighted", "g5-bylength-r2k4"]
    ws = [synth.tiny(**WORKLOADS[n]) for n in names]
    ps = [params_for(w) for w in ws]
    descs = [dict(src_xy=w.src_xy, dst_xy=w.dst_xy, group=w.group, n_groups=w.n_groups,
                  weight=w.weight) for w in ws]
    for profiled in (False, True):
        batch = pkg.bundle_init_batch(descs, ps)
        singles = [pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
                   for w, p in zip(ws, ps)]
        try:
            assert pkg.bundle_batch_size(batch) == 3
            if profiled:
                pkg.bundle_profile_enable(batch, True)
            pkg.bundle_iterate(batch, 3)
            pkg.bundle_iterate(batch, 2)
            total = 0
            for k, c in enumerate(singles):
                pkg.bundle_iterate(c, 5)
                m = pkg.bundle_batch_member(batch, k)
                om, xm = pkg.bundle_fetch(m, pixels=True)
                oc, xc = pkg.bundle_fetch(c, pixels=True)
                np.testing.assert_array_equal(om, oc)
                np.testing.assert_array_equal(xm, xc)
                np.testing.assert_array_equal(pkg.bundle_fetch_density(m, pkg.DENSITY_SUMS),
                                              pkg.bundle_fetch_density(c, pkg.DENSITY_SUMS))
                total += pkg.bundle_get_info(c).points_processed
            assert pkg.bundle_get_info(batch).points_processed == total
            with pytest.raises(pkg.BundleError):
                pkg.bundle_iterate(pkg.bundle_batch_member(batch, 0), 1)
        finally:
            pkg.bundle_destroy(batch)
            for c in singles:
                pkg.bundle_destroy(c)


def test_profile_counts_launches():
    w, p, ctx = _make("g1-fixed32")
    try:
        pkg.bundle_profile_enable(ctx, True)
        pkg.bundle_iterate(ctx, 3)
        prof = pkg.bundle_profile_read(ctx)
        assert prof["resample"][1] == 1
        assert prof["advect_resample"][1] == 2
        assert prof["advect"][1] == 1
        assert prof["rowbox"][1] == prof["colbox"][1] == prof["mix_quads"][1] == 3
        assert all(ms >= 0 for ms, _ in prof.values())
    finally:
        pkg.bundle_destroy(ctx)


@pytest.mark.parametrize("width,radius", [(512, 1), (512, 8), (512, 15), (1024, 4), (1024, 16)])
def test_row_pass_variants_give_the_oracle_sums(width, radius):
    """Every row-pass variant (register rows, shared-memory rows, windows in registers with
    shuffled borders) gives the oracle's box sums (Sec. 3.1) bit for bit, at the widths and
    radii the shuffled-border variant covers (its border spans up to a whole lane chunk)."""
    w = synth.tiny(seed=60 + radius, n_edges=700, n_groups=2, grid=(width, 40), radius=radius,
                   passes=3, n_fixed=0, n_max=32, weighted=True)
    p = params_for(w)
    for mode in (1, 2, 3):
        ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
        try:
            pkg.bundle_set_tiles(ctx, 0, mode, 0)
            pkg.bundle_iterate(ctx, 2)
            hist = pkg.bundle_fetch_density(ctx, pkg.DENSITY_HIST).astype(np.int64)
            sums = pkg.bundle_fetch_density(ctx, pkg.DENSITY_SUMS).astype(np.int64)
        finally:
            pkg.bundle_destroy(ctx)
        np.testing.assert_array_equal(sums, oracle.smooth(hist, radius, 3), err_msg=f"mode {mode}")


@pytest.mark.parametrize("sum_bits", [32, 64])
@pytest.mark.parametrize("grid,radius", [((512, 512), 1), ((512, 512), 15), ((1024, 512), 7),
                                         ((512, 1024), 12), ((1024, 1024), 16)])
def test_banded_passes_give_the_oracle_sums(grid, radius, sum_bits):
    """The banded path (row mode 4: the row passes over the histogram written transposed,
    then the column passes as row passes over that, written back) gives the oracle's box
    sums (Sec. 3.1) bit for bit, with 32- and 64-bit sums, on square and oblong grids and
    at the radii its register windows cover; sums and densities equal the shared-memory
    path's. 32-bit sums need a small mass (the library admits them only where the sum
    bound fits)."""
    small = sum_bits == 32
    w = synth.tiny(seed=80 + radius, n_edges=20 if small else 1500, n_groups=3, grid=grid,
                   radius=radius, passes=3, n_fixed=0, n_max=8 if small else 32,
                   weighted=not small)
    p = pkg.default_params(grid_w=grid[0], grid_h=grid[1], radius=radius, passes=3, n_fixed=0,
                           n_max=8 if small else 32, sum_bits=sum_bits)
    out = {}
    for mode in (2, 4):
        ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
        try:
            pkg.bundle_set_tiles(ctx, 0, mode, 0)
            pkg.bundle_iterate(ctx, 3)  # a middle iteration clears the histogram in its row pass
            info = pkg.bundle_get_info(ctx)
            assert info.tile_row == mode and info.sum_bits == sum_bits
            out[mode] = (pkg.bundle_fetch_density(ctx, pkg.DENSITY_HIST).astype(np.int64),
                         pkg.bundle_fetch_density(ctx, pkg.DENSITY_SUMS),
                         pkg.bundle_fetch_density(ctx, pkg.DENSITY_RHO))
        finally:
            pkg.bundle_destroy(ctx)
    hist, sums, rho = out[4]
    assert hist.sum() > 0
    np.testing.assert_array_equal(sums.astype(np.int64), oracle.smooth(hist, radius, 3))
    np.testing.assert_array_equal(out[2][1], sums)
    np.testing.assert_array_equal(out[2][2], rho)


def test_banded_path_rejected_where_it_does_not_fit():
    """Row mode 4 needs both sides of 512 or 1024 cells and a radius its windows cover."""
    w = synth.tiny(seed=5, n_edges=200, n_groups=2, grid=(512, 40), radius=4, passes=2,
                   n_fixed=0, n_max=16, weighted=False)
    ctx = pkg.bundle_init(params_for(w), w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    try:
        with pytest.raises(pkg.BundleError) as ei:
            pkg.bundle_set_tiles(ctx, 0, 4, 0)
        assert ei.value.status == pkg.BUNDLE_EINVAL
    finally:
        pkg.bundle_destroy(ctx)


@pytest.mark.parametrize("rho_dtype", [pkg.RHO_F32, pkg.RHO_BF16, pkg.RHO_F16])
def test_texture_gathers_equal_load_gathers(rho_dtype):
    """The advection's density gathers through the texture view of the quad map (the default)
    and through the load path (FLAG_LOAD_GATHERS) give the same polylines, histograms and
    densities bit for bit, for every density storage type, in single runs and in a batch."""
    w = synth.tiny(**WORKLOADS["g3-bylength-weighted"])
    w2 = synth.tiny(**WORKLOADS["g5-bylength-r2k4"])
    res = []
    for flags in (0, pkg.FLAG_LOAD_GATHERS):
        p = params_for(w, rho_dtype=rho_dtype, flags=flags)
        ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
        try:
            pkg.bundle_iterate(ctx, 4)
            off, xy = pkg.bundle_fetch(ctx, pixels=True)
            res.append([off, xy, pkg.bundle_fetch_density(ctx, pkg.DENSITY_HIST),
                        pkg.bundle_fetch_density(ctx, pkg.DENSITY_RHO)])
        finally:
            pkg.bundle_destroy(ctx)
        ps = [params_for(v, rho_dtype=rho_dtype, flags=flags) for v in (w, w2)]
        descs = [dict(src_xy=v.src_xy, dst_xy=v.dst_xy, group=v.group, n_groups=v.n_groups,
                      weight=v.weight) for v in (w, w2)]
        b = pkg.bundle_init_batch(descs, ps)
        try:
            pkg.bundle_iterate(b, 4)
            for k in range(2):
                res[-1].extend(pkg.bundle_fetch(pkg.bundle_batch_member(b, k), pixels=True))
        finally:
            pkg.bundle_destroy(b)
    for x, y in zip(res[0], res[1]):
        np.testing.assert_array_equal(x, y)
