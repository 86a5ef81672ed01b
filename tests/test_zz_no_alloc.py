"""The allocation-free smoothing entry point computes the box-filter sums of the method.

bundle_smooth_noalloc exists for callers that cannot allocate device memory
themselves (a framework's caching allocator owns every byte, a service reserved
its budget up front, or the path must not risk cudaMalloc's implicit
synchronisation): they pass a device histogram and a device output and the
library keeps its intermediate in a fixed device array. Its output must equal,
bit for bit, the FP64/int64 oracle's k passes of the (2r+1)^2 box filter with
half-sample reflection (Sec. 3.1), and the sums bundle_iterate produced for the
same histograms, on two calls in a row (two different histograms, so a stale
intermediate would show). The shapes cover the shared-memory row pass, the
register-resident row pass and a stack of exactly the array's 16 MiB; one more
row is rejected. This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected only on GPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1504_02687_gb300 as pkg  # noqa: E402
from paper_1504_02687_gb300 import build, synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()


@pytest.mark.parametrize("sum_bits", [32, 64])
def test_noalloc_smoothing_matches_iterate_and_oracle(sum_bits):
    w = synth.tiny(seed=31, n_edges=900, n_groups=3, grid=(120, 88), radius=4, passes=3,
                   n_fixed=0, n_max=24, weighted=True)
    p = pkg.default_params(grid_w=120, grid_h=88, radius=4, passes=3, n_fixed=0, n_max=24,
                           sum_bits=sum_bits)
    ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    try:
        pairs = []
        for _ in range(2):  # two iterations: two different histograms
            pkg.bundle_iterate(ctx, 1)
            pairs.append((pkg.bundle_fetch_density(ctx, pkg.DENSITY_HIST),
                          pkg.bundle_fetch_density(ctx, pkg.DENSITY_SUMS)))
    finally:
        pkg.bundle_destroy(ctx)
    dt = torch.int32 if sum_bits == 32 else torch.int64
    for hist, sums in pairs:  # two calls in a row
        h = torch.from_numpy(hist.view(np.int32)).to(dev)
        out = torch.full(h.shape, -1, dtype=dt, device=dev)
        pkg.bundle_smooth_noalloc(h, out, p.radius, p.passes, stream=stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_array_equal(got, sums)
        want = oracle.smooth(hist.astype(np.int64), p.radius, p.passes)
        np.testing.assert_array_equal(got.astype(np.int64), want)


@pytest.mark.parametrize("shape,radius,passes", [
    ((2, 256, 256), 5, 3),     # register-resident rows of 256 cells
    ((2, 1024, 1024), 12, 4),  # exactly 16 MiB of int64: the largest accepted stack
])
def test_noalloc_register_rows_and_full_array_match_oracle(shape, radius, passes):
    rng = np.random.default_rng(7 + shape[1])
    dev = torch.device("cuda:0")
    outs = []
    hists = []
    for k in range(2):  # two calls in a row on two different histograms
        hist = (rng.random(shape) < 0.05).astype(np.int64) * rng.integers(1, 4, shape)
        hists.append(hist)
        h = torch.from_numpy(hist.astype(np.int32)).to(dev)
        out = torch.full(shape, -1, dtype=torch.int64, device=dev)
        pkg.bundle_smooth_noalloc(h, out, radius, passes)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    for hist, got in zip(hists, outs):
        np.testing.assert_array_equal(got, oracle.smooth(hist, radius, passes))


def test_noalloc_rejects_oversize():
    dev = torch.device("cuda:0")
    # one row more than the 16 MiB array holds at 8 bytes per cell
    h = torch.zeros((2, 1025, 1024), dtype=torch.int32, device=dev)
    out = torch.zeros((2, 1025, 1024), dtype=torch.int64, device=dev)
    with pytest.raises(pkg.BundleError, match="16 MiB") as ei:
        pkg.bundle_smooth_noalloc(h, out, 4, 3)
    assert ei.value.status == pkg.BUNDLE_EINVAL
