"""Headless renderer (Sec. 3.4) on the CUDA path against the oracle's drawing of the same
polylines and density (the GPU's own, fetched): the integer accumulators are equal except at
pixels the oracle marks as near a coverage threshold (a position, width or projection within
1e-4 of deciding the other way, which FP32 may decide either way), and the 8-bit colours of
the pixels whose accumulators agree differ by at most one step (FP32 vs FP64 resolve)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected only on GPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1504_02687_gb300 as pkg  # noqa: E402
from paper_1504_02687_gb300 import synth  # noqa: E402

from parity import fetch_px, params_for, rho_as_f64  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1504_02687_gb300 import build

    build.build()
    oracle.build()


def _ctx(seed=12, n_edges=777, n_groups=3, iters=3, rho_dtype=pkg.RHO_F32):
    w = synth.tiny(seed=seed, n_edges=n_edges, n_groups=n_groups, grid=(128, 96), radius=4,
                   passes=3, n_fixed=0, n_max=24, weighted=True)
    p = params_for(w, rho_dtype=rho_dtype)
    ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    pkg.bundle_iterate(ctx, iters)
    return w, ctx


def _compare(ctx, w, **kw):
    pal = pkg.hue_palette(w.n_groups)
    acc = np.zeros((w.grid[1] * kw.get("scale", 1), w.grid[0] * kw.get("scale", 1), 4), np.int64)
    rgba = pkg.bundle_render(ctx, palette=pal, accum=acc, **kw)
    off, xy = fetch_px(ctx)
    rho = rho_as_f64(ctx)
    o_acc, amb, o_rgba = oracle.render(off, xy, w.group, w.weight, rho, pal, **kw)
    diff = (acc != o_acc).any(axis=2)
    assert not (diff & ~amb).any(), int((diff & ~amb).sum())
    same = ~diff
    d = np.abs(rgba.astype(int) - o_rgba.astype(int))
    assert d[same].max() <= 1
    assert acc[..., 0].astype(bool).sum() > 1000   # the drawing is not empty
    return rgba, acc, int(diff.sum()), int(amb.sum())


@pytest.mark.parametrize("kw", [
    dict(scale=1, alpha=0.3, width_min=1.0, width_max=3.0),
    dict(scale=2, alpha=0.15, width_min=1.0, width_max=5.0, log_width=True,
         background=(255, 255, 255)),
    dict(scale=3, alpha=0.5, width_min=1.5, width_max=1.5, rho_ref=1e-3),
])
def test_render_matches_oracle(kw):
    w, ctx = _ctx()
    try:
        _, _, n_diff, n_amb = _compare(ctx, w, **kw)
        print(f"render {kw}: {n_diff} accumulator differences, {n_amb} near-threshold pixels")
    finally:
        pkg.bundle_destroy(ctx)


def test_render_bf16_density_and_device_output():
    w, ctx = _ctx(rho_dtype=pkg.RHO_BF16)
    try:
        rgba_h, acc_h, _, _ = _compare(ctx, w, scale=2, width_max=4.0)
        H, W = w.grid[1] * 2, w.grid[0] * 2
        rgba_d = torch.zeros((H, W, 4), dtype=torch.uint8, device="cuda")
        acc_d = torch.zeros((H, W, 4), dtype=torch.int64, device="cuda")
        pkg.bundle_render(ctx, palette=pkg.hue_palette(w.n_groups), scale=2, width_max=4.0,
                          rgba=rgba_d, accum=acc_d)
        np.testing.assert_array_equal(rgba_d.cpu().numpy(), rgba_h)
        np.testing.assert_array_equal(acc_d.cpu().numpy(), acc_h)
    finally:
        pkg.bundle_destroy(ctx)


def test_render_states_and_arguments():
    w = synth.tiny(seed=13, n_edges=300, n_groups=2, grid=(64, 64), radius=2, passes=3)
    p = params_for(w)
    ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    try:
        with pytest.raises(pkg.BundleError) as ei:   # no density before the first iteration
            pkg.bundle_render(ctx)
        assert ei.value.status == pkg.BUNDLE_ESTATE
        pkg.bundle_iterate(ctx, 1)
        for bad in (dict(scale=0), dict(alpha=1.0), dict(width_min=0.5),
                    dict(width_min=3.0, width_max=2.0), dict(width_max=65.0)):
            with pytest.raises(pkg.BundleError) as ei:
                pkg.bundle_render(ctx, **bad)
            assert ei.value.status == pkg.BUNDLE_EINVAL
        rgba = pkg.bundle_render(ctx, background=(10, 20, 30))
        assert rgba[..., 3].min() == 255 and (rgba[..., :3] != [10, 20, 30]).any(axis=-1).any()
    finally:
        pkg.bundle_destroy(ctx)
    wz = np.zeros(w.n_edges, np.int32)  # zero weights draw nothing: only the background
    ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, wz)
    try:
        pkg.bundle_iterate(ctx, 1)
        rgba = pkg.bundle_render(ctx, background=(10, 20, 30))
        assert (rgba.reshape(-1, 4) == [10, 20, 30, 255]).all()
    finally:
        pkg.bundle_destroy(ctx)
