"""Precision form: the density stack stored in FP32, BF16 and FP16 for the gradient gather
(histograms and sums stay integer, positions and gradients FP32), against the FP64 oracle
after 30 iterations of the criteria-driven configuration (lattice pattern, 8 k-means groups,
8 x 1024^2 stack, r = 12, k = 4, <= 64 samples per edge).

The oracle runs the whole loop in FP64 from the same FP32 start. Because discrete decisions
amplify ulp-level differences (the cell a point falls in, the accepted trial, the resampled
count flip on near-ties), each form is compared with the
FP64 method's own drift under a +-1 FP32 ulp perturbation of the start. The edge count is
20,000 by default so the oracle finishes in seconds; PRECISION_EDGES raises it.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected only on GPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1504_02687_gb300 as pkg  # noqa: E402
from paper_1504_02687_gb300 import build, synth  # noqa: E402

from parity import fetch_px, oracle_params  # noqa: E402

ITERS = 30


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()


def _ulp_perturbed(xy, seed):
    rng = np.random.default_rng(seed)
    x32 = xy.astype(np.float32)
    d = rng.integers(-1, 2, x32.shape)
    up, dn = np.nextafter(x32, np.float32(1e9)), np.nextafter(x32, np.float32(-1e9))
    return np.where(d > 0, up, np.where(d < 0, dn, x32)).astype(np.float64)


def test_precision_forms_after_30_iterations():
    E = int(os.environ.get("PRECISION_EDGES", "20000"))
    w = synth.lattice_pattern(n_edges=E, kmeans_steps=10)
    W, H = w.grid
    results = {}
    start = None
    for name, dt in (("f32", pkg.RHO_F32), ("bf16", pkg.RHO_BF16), ("f16", pkg.RHO_F16)):
        p = pkg.default_params(grid_w=W, grid_h=H, radius=w.radius, passes=w.passes,
                               n_fixed=w.n_fixed, n_max=w.n_max, delta_px=w.delta, rho_dtype=dt)
        ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
        try:
            off0, P0 = fetch_px(ctx)
            if start is None:
                start = (off0, P0, p)
            np.testing.assert_array_equal(P0, start[1])
            pkg.bundle_iterate(ctx, ITERS)
            results[name] = fetch_px(ctx)
        finally:
            pkg.bundle_destroy(ctx)
    off0, P0, p = start
    prm = oracle_params(p)
    ref = oracle.run(off0, P0, w.group, w.weight, w.n_groups, H, W, prm, 0, ITERS)
    extent = float(max(W, H))

    def err_resampled(off, xy):
        # resampled counts may differ after a near-tie decision, so compare polyline shapes:
        # both re-spaced to 9 points at uniform arc length (endpoints included)
        o1, r1 = oracle.resample(off, xy, 9, 64, 2.0)
        o2, r2 = oracle.resample(ref.off, ref.xy, 9, 64, 2.0)
        e = np.hypot(*(r1 - r2).T) / extent
        return float(e.max()), float(np.sqrt((e ** 2).mean()))

    report = {"edges": E, "iterations": ITERS, "extent_px": extent}
    for name, (off, xy) in results.items():
        report[name] = {"max_rms_vs_fp64": err_resampled(off, xy),
                        "same_counts": bool(np.array_equal(off, ref.off))}
    env = []
    for seed in (0, 1):
        alt = oracle.run(off0, _ulp_perturbed(P0, seed), w.group, w.weight, w.n_groups, H, W,
                         prm, 0, ITERS)
        env.append(err_resampled(alt.off, alt.xy))
    report["fp64_ulp_envelope"] = env
    print("precision report: " + json.dumps(report))
    env_rms = max(e[1] for e in env)
    env_max = max(e[0] for e in env)
    # FP32 stays inside the FP64 method's own envelope. The 16-bit forms are measured and
    # reported (their rounding of the density is far above an ulp of FP32, so they leave the
    # envelope); they must stay bundled drawings of the same graph: RMS within 1 % of the extent
    assert report["f32"]["max_rms_vs_fp64"][1] <= 1.5 * env_rms
    assert report["f32"]["max_rms_vs_fp64"][0] <= 1.5 * env_max
    for name in ("bf16", "f16"):
        assert report[name]["max_rms_vs_fp64"][1] <= 1e-2, name
