"""FP64 CPU oracle of the 3DHEB bundling iteration (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package. The product path (the CUDA
library and its binding) never imports, links or calls it, and the oracle
imports nothing from the product.

The C++ source ``oracle3dheb.cpp`` holds the arithmetic; this module compiles
it with g++ (``-ffp-contract=off`` so that x86-64 and aarch64 give the same
bits) and marshals numpy arrays. Positions are float64 pixel coordinates,
polylines are CSR (``off[E+1]`` int64, ``xy[N, 2]`` float64), histograms and
smoothed sums int64 ``[G, H, W]``, densities float64 ``[G, H, W]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle3dheb.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle3dheb.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (seconds) and return its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared",
           "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.oracle_abi_version.restype = i32
    lib.oracle_grid_map.argtypes = [i64, P, P, i32, i32, i32, i32, P, P, P, P]
    lib.oracle_grid_map.restype = i32
    lib.oracle_resample.argtypes = [i64, P, P, i32, i32, f64, P, P, i64]
    lib.oracle_resample.restype = i64
    lib.oracle_splat.argtypes = [i64, P, P, P, P, i32, i32, i32, P]
    lib.oracle_splat.restype = None
    lib.oracle_smooth.argtypes = [i32, i32, i32, i32, i32, P, P]
    lib.oracle_smooth.restype = i32
    lib.oracle_combine.argtypes = [i32, i32, i32, i32, i32, i32, i32, P, P]
    lib.oracle_combine.restype = None
    lib.oracle_density_at.argtypes = [i32, i32, P, i64, P, P, P]
    lib.oracle_density_at.restype = None
    lib.oracle_bandwidth.argtypes = [i32, i32, i32, f64, f64]
    lib.oracle_bandwidth.restype = f64
    lib.oracle_advect_laplace.argtypes = [i64, P, P, P, i32, i32, i32, P, f64, f64, i32, f64, P, P]
    lib.oracle_advect_laplace.restype = None
    lib.oracle_run.argtypes = ([i64, P, P, P, P, i32, i32, i32, i32, i32, i32, i32, f64, f64,
                                i32, i32, f64, f64, f64, i32, i32, i32, P, P, i64, P, P, P, P, P,
                                i64])
    lib.oracle_run.restype = i64
    lib.oracle_advect_laplace_mode.argtypes = [i64, P, P, P, i32, i32, i32, P, f64, f64, i32, f64,
                                               i32, P, P]
    lib.oracle_advect_laplace_mode.restype = None
    lib.oracle_combine_matrix.argtypes = [i32, i32, i32, i32, i32, P, P, P]
    lib.oracle_combine_matrix.restype = None
    lib.oracle_directed_offset.argtypes = [i64, P, P, f64, i32, i32]
    lib.oracle_directed_offset.restype = None
    lib.oracle_run_mode.argtypes = ([i64, P, P, P, P, i32, i32, i32, i32, i32, i32, i32, f64, f64,
                                     i32, i32, f64, f64, f64, i32, i32, i32, i32, f64, P, i32, P,
                                     P, i64, P, P, P, P, P, i64])
    lib.oracle_render.argtypes = [i64, P, P, P, P, i32, i32, i32, P, i32, f64, f64, f64, f64,
                                  i32, P, P, P, P, P]
    lib.oracle_render.restype = i32
    lib.oracle_splat_segments.argtypes = [i64, P, P, P, P, i32, i32, i32, P]
    lib.oracle_splat_segments.restype = None
    lib.oracle_run_mode.restype = i64
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


@dataclass
class Params:
    """Bundling parameters (names follow the paper: r, k passes, alpha, h_max, lambda)."""
    radius: int = 4
    passes: int = 3
    alpha_num: int = 1
    alpha_den: int = 4
    h_max_sigmas: float = 2.0
    lam: float = 0.9
    n_fixed: int = 0
    n_max: int = 64
    delta: float = 2.0
    beta: float = 0.5
    eps: float = 1e-9
    tries: int = 8
    fixed_step: bool = False      # KDEEB step (Sec. 3.3)
    segment_hist: bool = False    # Bresenham segment histogram (Eq. 1, Sec. 4)
    directed_offset: float = 0.0  # pixels along the edge normal after the first sampling (Sec. 3)


def grid_map(src_xy, dst_xy, grid_w=0, grid_h=0, dominant=800, margin=4):
    """World coordinates -> FP32 pixel coordinates. Returns (W, H, map5, src_px, dst_px)."""
    lib = _load()
    s = _c(src_xy, np.float32).reshape(-1, 2)
    d = _c(dst_xy, np.float32).reshape(-1, 2)
    E = s.shape[0]
    wh = np.zeros(2, np.int32)
    mp = np.zeros(5, np.float64)
    sp = np.zeros_like(s)
    dp = np.zeros_like(d)
    rc = lib.oracle_grid_map(E, _p(s), _p(d), grid_w, grid_h, dominant, margin, _p(wh), _p(mp),
                             _p(sp), _p(dp))
    if rc != 0:
        raise ValueError(f"oracle_grid_map failed ({rc})")
    return int(wh[0]), int(wh[1]), mp, sp, dp


def straight_polylines(src_px, dst_px):
    """Initial state: every edge is the 2-point polyline (source, target)."""
    s = np.asarray(src_px, np.float64).reshape(-1, 2)
    d = np.asarray(dst_px, np.float64).reshape(-1, 2)
    E = s.shape[0]
    off = np.arange(0, 2 * E + 1, 2, dtype=np.int64)
    xy = np.empty((2 * E, 2), np.float64)
    xy[0::2] = s
    xy[1::2] = d
    return off, xy


def resample(off, xy, n_fixed=0, n_max=64, delta=2.0):
    lib = _load()
    off = _c(off, np.int64)
    xy = _c(xy, np.float64).reshape(-1, 2)
    E = off.shape[0] - 1
    cap = E * (n_fixed if n_fixed > 0 else n_max)
    off_o = np.zeros(E + 1, np.int64)
    xy_o = np.zeros((max(cap, 1), 2), np.float64)
    n = lib.oracle_resample(E, _p(off), _p(xy), n_fixed, n_max, delta, _p(off_o), _p(xy_o), cap)
    if n < 0:
        raise ValueError(f"oracle_resample failed ({n})")
    return off_o, xy_o[:n].copy()


def splat(off, xy, group, weight, G, H, W):
    lib = _load()
    off = _c(off, np.int64)
    xy = _c(xy, np.float64).reshape(-1, 2)
    E = off.shape[0] - 1
    group = _c(group, np.int32)
    weight = _c(weight, np.int32)
    hist = np.zeros((G, H, W), np.int64)
    lib.oracle_splat(E, _p(off), _p(xy), _p(group), _p(weight), G, H, W, _p(hist))
    return hist


def splat_segments(off, xy, group, weight, G, H, W):
    """Bresenham segment histogram (Eq. 1 as the paper rasterised it, Sec. 4)."""
    lib = _load()
    off = _c(off, np.int64)
    xy = _c(xy, np.float64).reshape(-1, 2)
    hist = np.zeros((G, H, W), np.int64)
    lib.oracle_splat_segments(off.shape[0] - 1, _p(off), _p(xy), _p(_c(group, np.int32)),
                              _p(_c(weight, np.int32)), G, H, W, _p(hist))
    return hist


def render(off, xy, group, weight, rho, palette, scale=1, alpha=0.25, width_min=1.0,
           width_max=4.0, rho_ref=0.0, log_width=False, background=(0, 0, 0)):
    """Headless drawing of the polylines (Sec. 3.4): returns (accum int64 [Hi, Wi, 4],
    ambiguous-pixel mask bool [Hi, Wi], rgba uint8 [Hi, Wi, 4])."""
    lib = _load()
    off = _c(off, np.int64)
    xy = _c(xy, np.float64).reshape(-1, 2)
    rho = _c(rho, np.float64)
    G, H, W = rho.shape
    Hi, Wi = H * scale, W * scale
    pal = _c(palette, np.uint8).reshape(G, 3)
    bg = np.ascontiguousarray(background, np.uint8)
    acc = np.zeros((Hi, Wi, 4), np.int64)
    amb = np.zeros((Hi, Wi), np.uint8)
    rgba = np.zeros((Hi, Wi, 4), np.uint8)
    rc = lib.oracle_render(off.shape[0] - 1, _p(off), _p(xy), _p(_c(group, np.int32)),
                           _p(_c(weight, np.int32)), G, H, W, _p(rho), scale, alpha, width_min,
                           width_max, rho_ref, 1 if log_width else 0, _p(pal), _p(bg), _p(acc),
                           _p(amb), _p(rgba))
    if rc != 0:
        raise ValueError("oracle_render: invalid arguments")
    return acc, amb.astype(bool), rgba


def ink(hist):
    """Occupied cells of a [G][H][W] histogram: (cells where any group is non-zero, sum over
    groups of each group's non-zero cells). The convergence measure compared in Fig. 3's
    experiment reading (tighter bundles cover fewer cells)."""
    occ = np.asarray(hist) != 0
    return int(occ.any(axis=0).sum()), int(occ.sum())


def smooth(hist, radius, passes):
    lib = _load()
    hist = _c(hist, np.int64)
    G, H, W = hist.shape
    out = np.zeros_like(hist)
    rc = lib.oracle_smooth(G, H, W, radius, passes, _p(hist), _p(out))
    if rc != 0:
        raise OverflowError(f"oracle_smooth failed ({rc})")
    return out


def combine(sums, radius, passes, alpha_num=1, alpha_den=4):
    lib = _load()
    sums = _c(sums, np.int64)
    G, H, W = sums.shape
    rho = np.zeros((G, H, W), np.float64)
    lib.oracle_combine(G, H, W, radius, passes, alpha_num, alpha_den, _p(sums), _p(rho))
    return rho


def density_at(layer, xy):
    """Bilinear density and gradient of one [H, W] layer at points xy[n, 2]."""
    lib = _load()
    layer = _c(layer, np.float64)
    H, W = layer.shape
    xy = _c(xy, np.float64).reshape(-1, 2)
    n = xy.shape[0]
    rho = np.zeros(n, np.float64)
    grad = np.zeros((n, 2), np.float64)
    lib.oracle_density_at(H, W, _p(layer), n, _p(xy), _p(rho), _p(grad))
    return rho, grad


def bandwidth(iteration, radius, passes, h_max_sigmas=2.0, lam=0.9):
    return float(_load().oracle_bandwidth(iteration, radius, passes, h_max_sigmas, lam))


def advect_laplace(off, xy, group, rho, h, eps=1e-9, tries=8, beta=0.5, fixed_step=False):
    """Returns (new_xy, accepted) with accepted[k] = trial index, -1 none, -2 endpoint.
    fixed_step: KDEEB's step of exactly h with no density test (Sec. 3.3, Fig. 3)."""
    lib = _load()
    off = _c(off, np.int64)
    xy = _c(xy, np.float64).reshape(-1, 2)
    E = off.shape[0] - 1
    group = _c(group, np.int32)
    rho = _c(rho, np.float64)
    G, H, W = rho.shape
    out = np.zeros_like(xy)
    acc = np.zeros(xy.shape[0], np.int32)
    lib.oracle_advect_laplace_mode(E, _p(off), _p(xy), _p(group), G, H, W, _p(rho), h, eps, tries,
                                   beta, 1 if fixed_step else 0, _p(out), _p(acc))
    return out, acc


def combine_matrix(sums, radius, passes, M):
    """rho_l = sum_b M[l, b] S_b / s^k for a general G x G interaction matrix (Eq. 3)."""
    lib = _load()
    sums = _c(sums, np.int64)
    G, H, W = sums.shape
    M = _c(M, np.float64).reshape(G, G)
    rho = np.zeros((G, H, W), np.float64)
    lib.oracle_combine_matrix(G, H, W, radius, passes, _p(M), _p(sums), _p(rho))
    return rho


def directed_offset(off, xy, amount, W, H):
    """Shift interior points by `amount` px along their edge's normal (Sec. 3); returns a copy."""
    lib = _load()
    off = _c(off, np.int64)
    xy = np.array(xy, np.float64).reshape(-1, 2)
    lib.oracle_directed_offset(off.shape[0] - 1, _p(off), _p(xy), float(amount), W, H)
    return xy


@dataclass
class RunResult:
    off: np.ndarray
    xy: np.ndarray
    hist: np.ndarray | None = None
    sums: np.ndarray | None = None
    rho: np.ndarray | None = None
    res_off: np.ndarray | None = None
    res_xy: np.ndarray | None = None


def run(off, xy, group, weight, G, H, W, prm: Params, iter0=0, n_iters=1, keep_last=False,
        M=None):
    """The whole loop: n_iters iterations from polylines (off, xy) in pixel units. M: optional
    G x G interaction matrix replacing Eq. 4's."""
    lib = _load()
    off = _c(off, np.int64)
    xy = _c(xy, np.float64).reshape(-1, 2)
    E = off.shape[0] - 1
    group = _c(group, np.int32)
    weight = _c(weight, np.int32)
    n_cap = prm.n_fixed if prm.n_fixed > 0 else prm.n_max
    cap = max(E * n_cap, int(off[-1]))
    off_o = np.zeros(E + 1, np.int64)
    xy_o = np.zeros((cap, 2), np.float64)
    hist = sums = rho = res_off = res_xy = None
    if keep_last:
        hist = np.zeros((G, H, W), np.int64)
        sums = np.zeros((G, H, W), np.int64)
        rho = np.zeros((G, H, W), np.float64)
        res_off = np.zeros(E + 1, np.int64)
        res_xy = np.zeros((cap, 2), np.float64)
    Mc = None if M is None else _c(M, np.float64).reshape(G, G)
    n = lib.oracle_run_mode(E, _p(off), _p(xy), _p(group), _p(weight), G, H, W, prm.radius,
                            prm.passes, prm.alpha_num, prm.alpha_den, prm.h_max_sigmas, prm.lam,
                            prm.n_fixed, prm.n_max, prm.delta, prm.beta, prm.eps, prm.tries, iter0,
                            n_iters, 1 if prm.fixed_step else 0, float(prm.directed_offset),
                            _p(Mc), 1 if prm.segment_hist else 0, _p(off_o), _p(xy_o), cap,
                            _p(hist), _p(sums), _p(rho),
                            _p(res_off), _p(res_xy), cap)
    if n < 0:
        raise RuntimeError(f"oracle_run failed ({n})")
    out = RunResult(off_o, xy_o[:n].copy(), hist, sums, rho, res_off, None)
    if keep_last and n_iters > 0:
        out.res_xy = res_xy[: int(res_off[-1])].copy()
    return out
