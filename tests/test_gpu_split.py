"""Split form: one graph's edges divided over contexts that exchange only their histograms.

Each context runs the per-edge stages (advection, Laplacian, resampling, splat) on its own
edges; between the splat and the box passes the histograms are summed over the contexts
(the exchange step of a multi-GPU run; Sec. 4 divides a graph's edges over CPU threads the
same way). Integer addition is exact and order-free, so the run must equal one context over
all edges bit for bit: polylines, histogram, smoothed sums and density. Here two processes
on cuda:0 sum their histograms through a gloo group on host copies; neither process's
kernels wait on the other's.
"""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected only on GPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1504_02687_gb300 as pkg  # noqa: E402
from paper_1504_02687_gb300 import build, synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ITERS = 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _whole(w, p):
    """One context over all edges: its pixel-unit start, map, and state after ITERS."""
    ctx = pkg.bundle_init(p, w.src_xy, w.dst_xy, w.group, w.n_groups, w.weight)
    try:
        off0, xy0 = pkg.bundle_fetch(ctx, pixels=True)
        info = pkg.bundle_get_info(ctx)
        pkg.bundle_iterate(ctx, ITERS)
        o, x = pkg.bundle_fetch(ctx, pixels=True)
        state = dict(off=o, xy=x, hist=pkg.bundle_fetch_density(ctx, pkg.DENSITY_HIST),
                     sums=pkg.bundle_fetch_density(ctx, pkg.DENSITY_SUMS),
                     rho=pkg.bundle_fetch_density(ctx, pkg.DENSITY_RHO))
    finally:
        pkg.bundle_destroy(ctx)
    return off0, xy0, np.array(info.map), info.sum_bits, state


def _graph():
    w = synth.tiny(seed=41, n_edges=1500, n_groups=3, grid=(160, 120), radius=4, passes=3,
                   n_fixed=0, n_max=32, weighted=True)
    p = pkg.default_params(grid_w=160, grid_h=120, radius=4, passes=3, n_fixed=0, n_max=32)
    return w, p


def test_split_steps_on_one_context_equal_iterate():
    """The phase entry points with no exchange are bundle_iterate, bit for bit."""
    w, p = _graph()
    off0, xy0, map5, bits, want = _whole(w, p)
    p.sum_bits = bits
    ctx = pkg.bundle_init_polylines(p, off0, xy0, w.group, w.n_groups, w.weight, map5=map5)
    try:
        pkg.bundle_iterate_split(ctx, ITERS, lambda h: None, on_device=True)
        o, x = pkg.bundle_fetch(ctx, pixels=True)
        np.testing.assert_array_equal(o, want["off"])
        np.testing.assert_array_equal(x, want["xy"])
        for k, sel in (("hist", pkg.DENSITY_HIST), ("sums", pkg.DENSITY_SUMS),
                       ("rho", pkg.DENSITY_RHO)):
            np.testing.assert_array_equal(pkg.bundle_fetch_density(ctx, sel), want[k])
        with pytest.raises(pkg.BundleError) as ei:  # out of order: no run is open
            pkg.bundle_density_step(ctx)
        assert ei.value.status == pkg.BUNDLE_ESTATE
        pkg.bundle_points_step(ctx)
        with pytest.raises(pkg.BundleError) as ei:  # a run is open
            pkg.bundle_iterate(ctx, 1)
        assert ei.value.status == pkg.BUNDLE_ESTATE
    finally:
        pkg.bundle_destroy(ctx)


def test_split_over_two_processes_equals_one_context(tmp_path):
    w, p = _graph()
    off0, xy0, map5, bits, want = _whole(w, p)
    inp = tmp_path / "graph.npz"
    np.savez(inp, off=off0, xy=xy0, group=w.group, weight=w.weight, map5=map5, W=160, H=120,
             r=4, k=3, n_max=32, G=w.n_groups, sum_bits=bits, iters=ITERS)
    world, port = 2, _free_port()
    env = dict(os.environ, MASTER_ADDR="127.0.0.1")
    procs = [subprocess.Popen([sys.executable, os.path.join(HERE, "split_worker.py"), str(r),
                               str(world), str(port), str(inp), str(tmp_path / f"r{r}.npz")],
                              env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                              text=True) for r in range(world)]
    for pr in procs:
        out, _ = pr.communicate(timeout=300)
        assert pr.returncode == 0, out
    parts = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    # every rank holds the whole graph's histogram, sums and density
    for part in parts:
        for k in ("hist", "sums", "rho"):
            np.testing.assert_array_equal(part[k], want[k])
    # the ranks' polylines, concatenated in edge order, are the one context's
    offs, base = [parts[0]["off"]], parts[0]["off"][-1]
    for part in parts[1:]:
        offs.append(part["off"][1:] + base)
        base += part["off"][-1]
    np.testing.assert_array_equal(np.concatenate(offs), want["off"])
    np.testing.assert_array_equal(np.concatenate([part["xy"] for part in parts]), want["xy"])
