"""GB300 (sm_103a) 3DHEB edge bundling: Python binding of the C ABI in include/bundle.h.

This module only marshals arguments (numpy arrays, torch tensors, streams) to
the shared library built from ``csrc/``; every step of the bundling iteration
runs in the library's CUDA kernels. There is no CPU fallback: if the library
is missing or cannot be loaded, importing the binding's functions raises.

Names follow the C ABI: ``bundle_init``, ``bundle_init_polylines``,
``bundle_iterate``, ``bundle_fetch``, ``bundle_fetch_density``,
``bundle_get_info``, ``bundle_sync``, ``bundle_destroy``; ``Bundler`` wraps a
context for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbundle3dheb.so")

BUNDLE_OK, BUNDLE_EINVAL, BUNDLE_ENOMEM, BUNDLE_ECUDA = 0, 1, 2, 3
BUNDLE_EOVERFLOW, BUNDLE_ETIMEOUT, BUNDLE_ESTATE, BUNDLE_ENOTSUP = 4, 5, 6, 7
RHO_F32, RHO_BF16, RHO_F16 = 0, 1, 2
INPUT_DEVICE = 1
FLAG_FIXED_STEP = 1
FLAG_SEGMENT_HIST = 2
FLAG_INK_STATS = 4
FLAG_LOAD_GATHERS = 8
INK_STATS_CAP = 4096
FETCH_DEVICE, FETCH_PIXELS, FETCH_RESAMPLED = 1, 2, 4
STEP_LAST = 1
DENSITY_HIST, DENSITY_SUMS, DENSITY_RHO = 0, 1, 2
PROFILE_KINDS = ("resample", "advect", "advect_resample", "rowbox", "colbox", "mix_quads",
                 "hist_clear")

EXPORTED = ("bundle_default_params", "bundle_init", "bundle_init_polylines", "bundle_iterate",
            "bundle_fetch", "bundle_fetch_density", "bundle_get_info", "bundle_sync",
            "bundle_destroy", "bundle_last_error", "bundle_status_string",
            "bundle_profile_enable", "bundle_profile_read", "bundle_smooth_noalloc",
            "bundle_init_batch", "bundle_batch_size", "bundle_batch_member",
            "bundle_set_interaction", "bundle_fetch_ink", "bundle_render", "bundle_autotune",
            "bundle_set_tiles", "bundle_points_step", "bundle_density_step",
            "bundle_set_histogram")


class BundleParams(ctypes.Structure):
    """Mirror of ``bundle_params`` (field order and types must match include/bundle.h)."""
    _fields_ = [
        ("grid_w", ctypes.c_int32), ("grid_h", ctypes.c_int32),
        ("grid_dominant", ctypes.c_int32), ("margin_px", ctypes.c_int32),
        ("radius", ctypes.c_int32), ("passes", ctypes.c_int32),
        ("alpha_num", ctypes.c_int32), ("alpha_den", ctypes.c_int32),
        ("h_max_sigmas", ctypes.c_double), ("lambda_", ctypes.c_double),
        ("n_fixed", ctypes.c_int32), ("n_max", ctypes.c_int32),
        ("delta_px", ctypes.c_float), ("laplace_beta", ctypes.c_float), ("eps", ctypes.c_float),
        ("step_tries", ctypes.c_int32), ("sum_bits", ctypes.c_int32),
        ("rho_dtype", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("directed_offset", ctypes.c_float),
    ]


class BundleInfo(ctypes.Structure):
    """Mirror of ``bundle_info``."""
    _fields_ = [
        ("n_edges", ctypes.c_int64), ("n_points", ctypes.c_int64),
        ("n_points_resampled", ctypes.c_int64),
        ("grid_w", ctypes.c_int32), ("grid_h", ctypes.c_int32), ("n_groups", ctypes.c_int32),
        ("sum_bits", ctypes.c_int32), ("rho_dtype", ctypes.c_int32),
        ("iteration", ctypes.c_int32), ("map", ctypes.c_double * 5), ("h_next", ctypes.c_double),
        ("device_bytes", ctypes.c_int64), ("points_processed", ctypes.c_int64),
        ("tile_eb", ctypes.c_int32), ("tile_row", ctypes.c_int32), ("tile_strip", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class BundleGraphDesc(ctypes.Structure):
    """Mirror of ``bundle_graph_desc``."""
    _fields_ = [
        ("n_edges", ctypes.c_int64), ("src_xy", ctypes.c_void_p), ("dst_xy", ctypes.c_void_p),
        ("group", ctypes.c_void_p), ("n_groups", ctypes.c_int32), ("weight", ctypes.c_void_p),
    ]


class BundleRenderParams(ctypes.Structure):
    """Mirror of ``bundle_render_params``."""
    _fields_ = [
        ("scale", ctypes.c_int32), ("alpha", ctypes.c_float), ("width_min", ctypes.c_float),
        ("width_max", ctypes.c_float), ("rho_ref", ctypes.c_float), ("log_width", ctypes.c_int32),
        ("background", ctypes.c_uint8 * 4),
    ]


class BundleError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built: no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"bundling library not built: {LIB_PATH} is missing "
                          "(run paper_1504_02687_gb300/build.py)")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    pp = ctypes.POINTER(BundleParams)
    L.bundle_default_params.argtypes = [pp]
    L.bundle_default_params.restype = None
    L.bundle_init.argtypes = [ctypes.POINTER(P), pp, i64, P, P, P, i32, P, i32, P]
    L.bundle_init.restype = i32
    L.bundle_init_polylines.argtypes = [ctypes.POINTER(P), pp, i64, P, P, P, i32, P, P, i32, i32,
                                        P]
    L.bundle_init_polylines.restype = i32
    L.bundle_iterate.argtypes = [P, i32]
    L.bundle_iterate.restype = i32
    L.bundle_fetch.argtypes = [P, P, P, i64, ctypes.POINTER(i64), i32]
    L.bundle_fetch.restype = i32
    L.bundle_fetch_density.argtypes = [P, i32, P, i64, i32]
    L.bundle_fetch_density.restype = i32
    L.bundle_get_info.argtypes = [P, ctypes.POINTER(BundleInfo)]
    L.bundle_get_info.restype = i32
    L.bundle_sync.argtypes = [P]
    L.bundle_sync.restype = i32
    L.bundle_destroy.argtypes = [P]
    L.bundle_destroy.restype = None
    L.bundle_last_error.argtypes = [P]
    L.bundle_last_error.restype = ctypes.c_char_p
    L.bundle_status_string.argtypes = [i32]
    L.bundle_status_string.restype = ctypes.c_char_p
    L.bundle_profile_enable.argtypes = [P, i32]
    L.bundle_profile_enable.restype = i32
    L.bundle_profile_read.argtypes = [P, P, P, i32, i32]
    L.bundle_profile_read.restype = i32
    L.bundle_smooth_noalloc.argtypes = [P, P, i32, i32, i32, i32, i32, i32, P]
    L.bundle_smooth_noalloc.restype = i32
    L.bundle_init_batch.argtypes = [ctypes.POINTER(P), i32, ctypes.POINTER(BundleGraphDesc), pp,
                                    i32, P]
    L.bundle_init_batch.restype = i32
    L.bundle_batch_size.argtypes = [P]
    L.bundle_batch_size.restype = i32
    L.bundle_batch_member.argtypes = [P, i32]
    L.bundle_batch_member.restype = P
    L.bundle_set_interaction.argtypes = [P, P, i64]
    L.bundle_set_tiles.argtypes = [P, i32, i32, i32]
    L.bundle_set_tiles.restype = i32
    L.bundle_autotune.argtypes = [P]
    L.bundle_autotune.restype = i32
    L.bundle_render.argtypes = [P, ctypes.POINTER(BundleRenderParams), P, P, P, i32]
    L.bundle_render.restype = i32
    L.bundle_fetch_ink.argtypes = [P, P, i32, i32]
    L.bundle_fetch_ink.restype = i32
    L.bundle_set_interaction.restype = i32
    L.bundle_points_step.argtypes = [P, i32]
    L.bundle_points_step.restype = i32
    L.bundle_density_step.argtypes = [P]
    L.bundle_density_step.restype = i32
    L.bundle_set_histogram.argtypes = [P, P, i32]
    L.bundle_set_histogram.restype = i32
    _lib = L
    return L


def status_string(s: int) -> str:
    return lib().bundle_status_string(int(s)).decode()


def default_params(**overrides) -> BundleParams:
    p = BundleParams()
    lib().bundle_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, "lambda_" if k == "lam" else k, v)
    return p


def _check(status: int, ctx=None):
    if status != BUNDLE_OK:
        msg = lib().bundle_last_error(ctx).decode(errors="replace")
        raise BundleError(status, msg)


def _ptr(a):
    """Pointer of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def _host(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


_CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy: the legacy default stream


def _stream_handle(stream):
    """cudaStream_t of a torch stream or a raw handle. torch's default stream has handle 0,
    which the library would read as "make your own stream"; it is passed as
    cudaStreamLegacy instead so the work really runs on the caller's stream."""
    if stream is None:
        return None
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    return ctypes.c_void_p(h if h else _CUDA_STREAM_LEGACY)


def bundle_init(params: BundleParams, src_xy, dst_xy, group=None, n_groups=1, weight=None,
                stream=None):
    """Create a context from straight edges. Arrays are numpy (host) or CUDA torch tensors
    (all on the device together). Returns the opaque context handle."""
    dev = _is_device(src_xy)
    if not dev:
        src_xy = _host(src_xy, np.float32)
        dst_xy = _host(dst_xy, np.float32)
        group = _host(group, np.int32)
        weight = _host(weight, np.int32)
    E = int(src_xy.shape[0]) if src_xy.ndim == 2 else int(src_xy.shape[0] // 2)
    ctx = ctypes.c_void_p()
    st = lib().bundle_init(ctypes.byref(ctx), ctypes.byref(params), E, _ptr(src_xy), _ptr(dst_xy),
                           _ptr(group), int(n_groups), _ptr(weight), INPUT_DEVICE if dev else 0,
                           _stream_handle(stream))
    _check(st)
    return ctx


def bundle_init_polylines(params: BundleParams, off, xy_px, group=None, n_groups=1, weight=None,
                          map5=None, iteration=0, stream=None):
    """Create a context from CSR polylines in grid pixel units (params.grid_w/h set)."""
    dev = _is_device(xy_px)
    if not dev:
        off = _host(off, np.int64)
        xy_px = _host(xy_px, np.float32)
        group = _host(group, np.int32)
        weight = _host(weight, np.int32)
    m = None if map5 is None else _host(map5, np.float64)
    E = int(off.shape[0]) - 1
    ctx = ctypes.c_void_p()
    st = lib().bundle_init_polylines(ctypes.byref(ctx), ctypes.byref(params), E, _ptr(off),
                                     _ptr(xy_px), _ptr(group), int(n_groups), _ptr(weight), _ptr(m),
                                     int(iteration), INPUT_DEVICE if dev else 0,
                                     _stream_handle(stream))
    _check(st)
    return ctx


def bundle_init_batch(graphs, params, stream=None):
    """Create a batch. graphs: list of dicts with src_xy, dst_xy, group, n_groups, weight
    (numpy, host); params: list of BundleParams (one per graph). Returns the batch handle."""
    keep = []
    descs = (BundleGraphDesc * len(graphs))()
    for d, g in zip(descs, graphs):
        arrs = [_host(g["src_xy"], np.float32), _host(g["dst_xy"], np.float32),
                _host(g.get("group"), np.int32), _host(g.get("weight"), np.int32)]
        keep.append(arrs)
        d.n_edges = int(arrs[0].shape[0])
        d.src_xy, d.dst_xy = arrs[0].ctypes.data, arrs[1].ctypes.data
        d.group = None if arrs[2] is None else arrs[2].ctypes.data
        d.weight = None if arrs[3] is None else arrs[3].ctypes.data
        d.n_groups = int(g.get("n_groups", 1))
    parr = (BundleParams * len(params))(*params)
    ctx = ctypes.c_void_p()
    st = lib().bundle_init_batch(ctypes.byref(ctx), len(graphs), descs, parr, 0,
                                 _stream_handle(stream))
    _check(st)
    return ctx


def bundle_batch_size(ctx) -> int:
    return int(lib().bundle_batch_size(ctx))


def bundle_batch_member(ctx, k: int):
    """Borrowed handle of graph k of a batch (valid until the batch is destroyed)."""
    h = lib().bundle_batch_member(ctx, int(k))
    if not h:
        raise IndexError(k)
    return ctypes.c_void_p(h)


def bundle_set_interaction(ctx, num, den: int):
    """General interaction matrix M = num / den (G x G integers, Eq. 3)."""
    n = np.ascontiguousarray(num, dtype=np.int64)
    _check(lib().bundle_set_interaction(ctx, _ptr(n), int(den)), ctx)


def bundle_fetch_ink(ctx, first: int, n: int) -> np.ndarray:
    """Convergence record (FLAG_INK_STATS): int64 [n, 2] of (cells any group occupies,
    sum over groups of each group's occupied cells) for iterations first .. first+n-1."""
    out = np.zeros((max(int(n), 0), 2), np.int64)
    _check(lib().bundle_fetch_ink(ctx, _ptr(out), int(first), int(n)), ctx)
    return out


def bundle_autotune(ctx):
    """Time the tile shapes on this (fresh) context or batch and keep the fastest."""
    _check(lib().bundle_autotune(ctx), ctx)


def bundle_set_tiles(ctx, eb: int = 0, row_mode: int = 0, col_strip: int = 0):
    """Choose the tile shapes by hand (0 keeps eb / picks row and strip by grid size)."""
    _check(lib().bundle_set_tiles(ctx, int(eb), int(row_mode), int(col_strip)), ctx)


def bundle_iterate(ctx, n_iters: int):
    _check(lib().bundle_iterate(ctx, int(n_iters)), ctx)


def bundle_points_step(ctx, last: bool = False):
    """Split form: the per-edge stages of an iteration on this context's edges (see
    include/bundle.h): the first call of a run resamples and splats; later calls advect,
    smooth, and (unless `last`) resample and splat for the next iteration."""
    _check(lib().bundle_points_step(ctx, STEP_LAST if last else 0), ctx)


def bundle_density_step(ctx):
    """Split form: box passes, layer mix and density of the open iteration's histogram."""
    _check(lib().bundle_density_step(ctx), ctx)


def bundle_set_histogram(ctx, hist):
    """Split form: replace the open iteration's histogram (uint32/int32 [G, H, W]; numpy, or
    a CUDA tensor on the context's device), e.g. by its sum over the contexts."""
    if _is_device(hist):
        if not hist.is_contiguous():
            raise BundleError(BUNDLE_EINVAL, "hist must be contiguous")
        _check(lib().bundle_set_histogram(ctx, _ptr(hist), INPUT_DEVICE), ctx)
    else:
        h = np.ascontiguousarray(hist).view(np.uint32)
        _check(lib().bundle_set_histogram(ctx, _ptr(h), 0), ctx)


def bundle_iterate_split(ctx, n_iters: int, all_reduce, on_device: bool = True):
    """n iterations of a context that holds part of a graph's edges. `all_reduce(h)` must sum
    the int32 [G, H, W] tensor h over all parts in place (e.g. torch.distributed.all_reduce:
    on_device=True hands it a CUDA tensor, for NCCL; False a CPU tensor, for gloo). The
    integer sum is exact, so every part sees the histogram of the whole graph."""
    import torch

    info = bundle_get_info(ctx)
    shape = (info.n_groups, info.grid_h, info.grid_w)
    buf = torch.empty(shape, dtype=torch.int32, device="cuda" if on_device else "cpu")
    bundle_points_step(ctx)
    for it in range(int(n_iters)):
        bundle_fetch_density(ctx, DENSITY_HIST, out=buf if on_device else buf.numpy())
        all_reduce(buf)
        bundle_set_histogram(ctx, buf if on_device else buf.numpy())
        bundle_density_step(ctx)
        bundle_points_step(ctx, last=it == n_iters - 1)


def bundle_sync(ctx):
    _check(lib().bundle_sync(ctx), ctx)


def bundle_get_info(ctx) -> BundleInfo:
    info = BundleInfo()
    _check(lib().bundle_get_info(ctx, ctypes.byref(info)), ctx)
    return info


def bundle_fetch(ctx, pixels=False, resampled=False, off=None, xy=None):
    """Return (off int64 [E+1], xy float32 [N, 2]). With `off`/`xy` given (CUDA tensors or
    numpy arrays), fills them instead and returns them."""
    info = bundle_get_info(ctx)
    flags = (FETCH_PIXELS if pixels else 0) | (FETCH_RESAMPLED if resampled else 0)
    n = ctypes.c_int64()
    if off is None:
        off = np.zeros(info.n_edges + 1, np.int64)
        N = info.n_points_resampled if resampled else info.n_points
        xy = np.zeros((max(int(N), 1), 2), np.float32)
    if _is_device(off):
        flags |= FETCH_DEVICE
    cap = int(xy.shape[0]) if xy is not None else 0
    _check(lib().bundle_fetch(ctx, _ptr(off), _ptr(xy), cap, ctypes.byref(n), flags), ctx)
    return off, xy[: n.value]


def bundle_fetch_density(ctx, which: int, out=None):
    """Return one [G, H, W] stack of the last iteration (numpy unless `out` is given)."""
    info = bundle_get_info(ctx)
    shape = (info.n_groups, info.grid_h, info.grid_w)
    if out is None:
        if which == DENSITY_HIST:
            out = np.zeros(shape, np.uint32)
        elif which == DENSITY_SUMS:
            out = np.zeros(shape, np.int32 if info.sum_bits == 32 else np.int64)
        else:
            out = np.zeros(shape, np.float32 if info.rho_dtype == RHO_F32 else np.uint16)
    nbytes = out.numel() * out.element_size() if hasattr(out, "numel") else out.nbytes
    flags = FETCH_DEVICE if _is_device(out) else 0
    _check(lib().bundle_fetch_density(ctx, int(which), _ptr(out), int(nbytes), flags), ctx)
    return out


def hue_palette(n_groups: int) -> np.ndarray:
    """Evenly spaced hues at full saturation and value: distinct colours for nominal bins
    (Sec. 3.4). uint8 [n_groups, 3]."""
    out = np.zeros((n_groups, 3), np.uint8)
    for g in range(n_groups):
        h = 6.0 * g / max(n_groups, 1)
        k = int(h) % 6
        f = h - int(h)
        rgb = [(1, f, 0), (1 - f, 1, 0), (0, 1, f), (0, 1 - f, 1), (f, 0, 1), (1, 0, 1 - f)][k]
        out[g] = [round(255 * c) for c in rgb]
    return out


def bundle_render(ctx, palette=None, scale: int = 1, alpha: float = 0.25,
                  width_min: float = 1.0, width_max: float = 4.0, rho_ref: float = 0.0,
                  log_width: bool = False, background=(0, 0, 0), rgba=None, accum=None):
    """Draw the current polylines (Sec. 3.4). Returns rgba uint8 [Hi, Wi, 4] (numpy, or the
    given device tensor); `accum` (int64 [Hi, Wi, 4], same memory kind) receives the raw
    integer accumulators when given."""
    info = bundle_get_info(ctx)
    Hi, Wi = info.grid_h * scale, info.grid_w * scale
    pal = hue_palette(info.n_groups) if palette is None else np.ascontiguousarray(palette, np.uint8)
    if pal.shape != (info.n_groups, 3):
        raise ValueError(f"palette must be uint8 [{info.n_groups}, 3]")
    if rgba is None:
        rgba = np.zeros((Hi, Wi, 4), np.uint8)
    rp = BundleRenderParams(int(scale), float(alpha), float(width_min), float(width_max),
                            float(rho_ref), 1 if log_width else 0)
    for i, v in enumerate(background[:3]):
        rp.background[i] = int(v)
    flags = FETCH_DEVICE if _is_device(rgba) else 0
    if accum is not None and _is_device(accum) != bool(flags):
        raise ValueError("rgba and accum must both be host or both device buffers")
    _check(lib().bundle_render(ctx, ctypes.byref(rp), _ptr(pal), _ptr(rgba), _ptr(accum), flags),
           ctx)
    return rgba


def bundle_profile_enable(ctx, on: bool = True):
    _check(lib().bundle_profile_enable(ctx, 1 if on else 0), ctx)


def bundle_profile_read(ctx, reset: bool = True) -> dict:
    """Per kernel kind: (total ms, launches) of the launches recorded since the last read."""
    n = len(PROFILE_KINDS)
    ms = np.zeros(n, np.float64)
    cnt = np.zeros(n, np.int64)
    _check(lib().bundle_profile_read(ctx, _ptr(ms), _ptr(cnt), n, 1 if reset else 0), ctx)
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PROFILE_KINDS)}


def _noalloc_check(hist, sums):
    """Reasons the allocation-free call must not be made (the C ABI sees neither sizes,
    dtypes nor devices, so a mismatch here would become an out-of-bounds write)."""
    import torch

    if not (isinstance(hist, torch.Tensor) and isinstance(sums, torch.Tensor)):
        return "hist and sums must be torch tensors"
    if hist.dim() != 3 or tuple(sums.shape) != tuple(hist.shape):
        return f"hist and sums must be [G, H, W] of one shape, got {tuple(hist.shape)} and " \
               f"{tuple(sums.shape)}"
    if hist.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
        return f"hist must be int32 or uint32, got {hist.dtype}"
    if sums.dtype not in (torch.int32, torch.int64):
        return f"sums must be int32 or int64, got {sums.dtype}"
    if not (hist.is_contiguous() and sums.is_contiguous()):
        return "hist and sums must be contiguous"
    if not (hist.is_cuda and sums.is_cuda):
        return "hist and sums must be CUDA tensors"
    if hist.device != sums.device:
        return f"hist and sums must be on one device, got {hist.device} and {sums.device}"
    return None


def bundle_smooth_noalloc(hist, sums, radius: int, passes: int, stream=None):
    """Box-pass smoothing of a device histogram into a caller-provided device output, with no
    allocation by the library (for callers that cannot allocate device memory themselves:
    see include/bundle.h). hist: contiguous CUDA uint32/int32 tensor [G, H, W]; sums:
    contiguous CUDA int32 or int64 tensor of the same shape on the same device (its dtype
    picks the sum width). The call runs with that device current."""
    import torch

    why = _noalloc_check(hist, sums)
    if why is not None:
        raise BundleError(BUNDLE_EINVAL, why)
    G, H, W = (int(x) for x in hist.shape)
    bits = 8 * sums.element_size()
    with torch.cuda.device(hist.device):
        _check(lib().bundle_smooth_noalloc(_ptr(hist), _ptr(sums), G, H, W, int(radius),
                                           int(passes), bits, _stream_handle(stream)))
    return sums


def bundle_destroy(ctx):
    if ctx:
        lib().bundle_destroy(ctx)


class Bundler:
    """Owning wrapper of one context."""

    def __init__(self, ctx):
        self.ctx = ctx

    @classmethod
    def from_edges(cls, src_xy, dst_xy, group=None, n_groups=1, weight=None, params=None,
                   stream=None, **overrides):
        p = params if params is not None else default_params(**overrides)
        return cls(bundle_init(p, src_xy, dst_xy, group, n_groups, weight, stream))

    @classmethod
    def from_polylines(cls, off, xy_px, grid, group=None, n_groups=1, weight=None, map5=None,
                       iteration=0, params=None, stream=None, **overrides):
        p = params if params is not None else default_params(**overrides)
        p.grid_w, p.grid_h = int(grid[0]), int(grid[1])
        return cls(bundle_init_polylines(p, off, xy_px, group, n_groups, weight, map5, iteration,
                                         stream))

    def iterate(self, n: int = 1):
        bundle_iterate(self.ctx, n)
        return self

    def sync(self):
        bundle_sync(self.ctx)

    def info(self) -> BundleInfo:
        return bundle_get_info(self.ctx)

    def fetch(self, pixels=False, resampled=False):
        return bundle_fetch(self.ctx, pixels=pixels, resampled=resampled)

    def density(self, which: int):
        return bundle_fetch_density(self.ctx, which)

    def close(self):
        bundle_destroy(self.ctx)
        self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if self.ctx:
                self.close()
        except Exception:
            pass
