"""The allocation-free smoothing entry point agrees with the regular path.

bundle_smooth_noalloc exists for callers that cannot allocate device memory
themselves (a framework's caching allocator owns every byte, a service reserved
its budget up front, or the path must not risk cudaMalloc's implicit
synchronisation): they pass a device histogram and a device output and the
library keeps its intermediate in a fixed device array. Here the output of two
calls in a row -- on two different histograms, so a stale intermediate would
show -- must equal, bit for bit, the smoothed sums bundle_iterate produced for
the same histograms. This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected only on GPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1504_02687_gb300 as pkg  # noqa: E402
from paper_1504_02687_gb300 import build, synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


@pytest.mark.parametrize("sum_bits", [32, 64])
def test_noalloc_smoothing_matches_iterate(sum_bits):
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
        np.testing.assert_array_equal(out.cpu().numpy(), sums)


def test_noalloc_rejects_oversize():
    dev = torch.device("cuda:0")
    h = torch.zeros((3, 1024, 1024), dtype=torch.int32, device=dev)
    out = torch.zeros((3, 1024, 1024), dtype=torch.int64, device=dev)
    with pytest.raises(pkg.BundleError, match="16 MiB") as ei:
        pkg.bundle_smooth_noalloc(h, out, 4, 3)
    assert ei.value.status == pkg.BUNDLE_EINVAL
