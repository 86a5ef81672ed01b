"""Host-side argument checks and integer-width bounds of bundle_init (no GPU needed: every
check runs before the library's first CUDA call)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def pkg():
    from paper_1504_02687_gb300 import build

    build.build()
    import paper_1504_02687_gb300 as p

    return p


def _edges(E, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, 1, (E, 2)).astype(np.float32), rng.uniform(0, 1, (E, 2)).astype(np.float32)


@pytest.mark.parametrize("override,needle", [
    (dict(radius=0), "radius"),
    (dict(passes=0), "passes"),
    (dict(passes=17), "passes"),
    (dict(alpha_den=0), "alpha"),
    (dict(lam=0.0), "lambda"),
    (dict(lam=1.5), "lambda"),
    (dict(n_fixed=1), "n_fixed"),
    (dict(n_fixed=0, n_max=1), "n_max"),
    (dict(n_fixed=0, delta_px=0.0), "delta"),
    (dict(laplace_beta=1.5), "laplace_beta"),
    (dict(step_tries=0), "step_tries"),
    (dict(sum_bits=16), "sum_bits"),
    (dict(rho_dtype=7), "rho_dtype"),
    (dict(grid_w=64, grid_h=0), "grid_w"),
    (dict(grid_w=8192, grid_h=64), "grid"),
    (dict(grid_w=16, grid_h=16, radius=16, margin_px=0), "radius"),
    (dict(grid_w=16, grid_h=16, radius=4, margin_px=8), "margin"),
    (dict(flags=16), "flags"),
    (dict(flags=2, sum_bits=32), "64-bit sums"),
    (dict(directed_offset=0.5), "directed_offset"),
])
def test_invalid_arguments(pkg, override, needle):
    src, dst = _edges(10)
    with pytest.raises(pkg.BundleError) as ei:
        pkg.bundle_init(pkg.default_params(**override), src, dst)
    assert ei.value.status == pkg.BUNDLE_EINVAL
    assert needle in str(ei.value)


def test_empty_input_is_rejected(pkg):
    """No edges: EINVAL before any CUDA call (there is nothing to bundle)."""
    e = np.zeros((0, 2), np.float32)
    with pytest.raises(pkg.BundleError, match="n_edges") as ei:
        pkg.bundle_init(pkg.default_params(grid_w=64, grid_h=64), e, e)
    assert ei.value.status == pkg.BUNDLE_EINVAL


def test_invalid_polylines_are_rejected(pkg):
    """bundle_init_polylines checks its host inputs before any CUDA call: point counts, the
    drawing area (a NaN is outside it) and the offsets."""
    p = pkg.default_params(grid_w=64, grid_h=64, n_fixed=0, n_max=16)
    off = np.array([0, 3, 5], np.int64)
    xy = np.array([[1, 1], [5, 5], [9, 2], [3, 3], [7, 7]], np.float32)
    bad = [
        (np.array([0, 1, 5], np.int64), xy, "points"),           # a one-point polyline
        (off, np.where(np.arange(10).reshape(5, 2) == 3, np.nan, xy), "outside"),
        (off, xy + np.array([64.0, 0.0], np.float32), "outside"),  # beyond W - 2^-10
        (np.array([1, 3, 5], np.int64), xy, "start at 0"),
    ]
    for o, x, needle in bad:
        with pytest.raises(pkg.BundleError, match=needle) as ei:
            pkg.bundle_init_polylines(p, o, x)
        assert ei.value.status == pkg.BUNDLE_EINVAL


def test_invalid_groups_and_weights(pkg):
    src, dst = _edges(10)
    p = pkg.default_params(grid_w=64, grid_h=64)
    with pytest.raises(pkg.BundleError, match="group"):
        pkg.bundle_init(p, src, dst, group=np.full(10, 3, np.int32), n_groups=3)
    with pytest.raises(pkg.BundleError, match="n_groups"):
        pkg.bundle_init(p, src, dst, n_groups=65)
    with pytest.raises(pkg.BundleError, match="negative"):
        pkg.bundle_init(p, src, dst, weight=np.array([1] * 9 + [-1], np.int32))
    src[3, 0] = np.nan
    with pytest.raises(pkg.BundleError, match="non-finite"):
        pkg.bundle_init(p, src, dst)


def test_overflow_bounds(pkg):
    """The worst case of the integer stages is checked before anything runs: a cell can be
    counted twice per axis by a reflected window, so after k passes every value is at most
    4 (2r+1)^(2(k-1)) sum(w) cap; the layer mix multiplies by q (G-1) + p."""
    E = 1000
    src, dst = _edges(E)
    # sum(w) * cap beyond uint32 histogram cells
    w = np.full(E, 40_000, np.int32)
    with pytest.raises(pkg.BundleError, match="histogram") as ei:
        pkg.bundle_init(pkg.default_params(grid_w=64, grid_h=64, n_fixed=64), src, dst, weight=w)
    assert ei.value.status == pkg.BUNDLE_EOVERFLOW
    # int32 sums requested where the bound needs 64 bits
    with pytest.raises(pkg.BundleError, match="int32") as ei:
        pkg.bundle_init(pkg.default_params(grid_w=256, grid_h=256, radius=8, passes=4,
                                           sum_bits=32), src, dst)
    assert ei.value.status == pkg.BUNDLE_EOVERFLOW
    # even int64 cannot hold 16 passes of a wide box
    with pytest.raises(pkg.BundleError, match="int64") as ei:
        pkg.bundle_init(pkg.default_params(grid_w=256, grid_h=256, radius=12, passes=16), src,
                        dst)
    assert ei.value.status == pkg.BUNDLE_EOVERFLOW
    # the layer mix of many groups tips over where one group fits
    g = (np.arange(E) % 64).astype(np.int32)
    with pytest.raises(pkg.BundleError, match="layer-mix") as ei:
        pkg.bundle_init(pkg.default_params(grid_w=256, grid_h=256, radius=12, passes=4,
                                           n_fixed=64), src, dst, group=g, n_groups=64,
                        weight=np.full(E, 1000, np.int32))
    assert ei.value.status == pkg.BUNDLE_EOVERFLOW


def test_bounds_of_the_benchmark_configs_fit(pkg):
    """The bound arithmetic the library applies, restated: the 5M-edge, 8-group, r = 12,
    k = 4, 64-point configuration needs int64 sums and fits the int64 layer mix."""
    M0 = 5_000_000 * 64
    s = 25 ** 2
    bound = 4 * s ** 3 * M0
    assert 2**31 <= bound < 2**63
    assert (4 * 7 + 1) * bound < 2**63
    # the small configuration (2000 edges, 32 points, r = 4, k = 3) fits int32 sums
    assert 4 * 81**2 * 2000 * 32 < 2**31


def test_noalloc_binding_rejects_mismatched_buffers(pkg):
    """The allocation-free smoothing call sees only raw pointers in the C ABI, so its
    binding refuses shapes, dtypes, layouts and devices that would let the kernels write
    past the caller's output, before anything reaches the library (CPU tensors here)."""
    torch = pytest.importorskip("torch")
    h = torch.zeros((2, 16, 16), dtype=torch.int32)
    cases = [
        (h, torch.zeros((2, 16, 8), dtype=torch.int64), "one shape"),
        (h.view(2, 256), torch.zeros((2, 256), dtype=torch.int64), "one shape"),
        (h, torch.zeros((2, 16, 16), dtype=torch.float32), "int32 or int64"),
        (h.to(torch.float32), torch.zeros((2, 16, 16), dtype=torch.int64), "int32 or uint32"),
        (h, torch.zeros((2, 16, 32), dtype=torch.int64)[:, :, ::2], "contiguous"),
        (h, torch.zeros((2, 16, 16), dtype=torch.int64), "CUDA tensors"),
    ]
    for hist, sums, needle in cases:
        with pytest.raises(pkg.BundleError, match=needle) as ei:
            pkg.bundle_smooth_noalloc(hist, sums, 2, 2)
        assert ei.value.status == pkg.BUNDLE_EINVAL
