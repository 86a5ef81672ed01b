"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI, run the FP64
oracle on the same inputs, and compare stage by stage.

Lockstep: the oracle restarts every stage from the GPU's own FP32 state (exact in FP64), so
the integer stages (histogram, smoothed sums) must match bit for bit, and position
differences come only from FP32 rounding -- or from a discrete decision (which trial step is
accepted, which cell a point falls in) taken on a near-tie, which `advect_mismatch` checks
point by point.
"""
from __future__ import annotations

import numpy as np

import oracle
import paper_1504_02687_gb300 as pkg

F32_ULP = 2.0 ** -23


def params_for(w, **over):
    """Library parameters of a synthetic workload."""
    p = pkg.default_params(grid_w=w.grid[0], grid_h=w.grid[1], radius=w.radius, passes=w.passes,
                           n_fixed=w.n_fixed, n_max=w.n_max, delta_px=w.delta)
    for k, v in over.items():
        setattr(p, "lambda_" if k == "lam" else k, v)
    return p


def oracle_params(p) -> oracle.Params:
    return oracle.Params(radius=p.radius, passes=p.passes, alpha_num=p.alpha_num,
                         alpha_den=p.alpha_den, h_max_sigmas=p.h_max_sigmas, lam=p.lambda_,
                         n_fixed=p.n_fixed, n_max=p.n_max, delta=float(p.delta_px),
                         beta=float(p.laplace_beta), eps=float(p.eps), tries=p.step_tries,
                         fixed_step=bool(p.flags & pkg.FLAG_FIXED_STEP),
                         segment_hist=bool(p.flags & pkg.FLAG_SEGMENT_HIST))


def fetch_px(ctx, resampled=False):
    off, xy = pkg.bundle_fetch(ctx, pixels=True, resampled=resampled)
    return off.astype(np.int64), xy.astype(np.float64)


def rho_as_f64(ctx):
    info = pkg.bundle_get_info(ctx)
    r = pkg.bundle_fetch_density(ctx, pkg.DENSITY_RHO)
    if info.rho_dtype == pkg.RHO_F32:
        return r.astype(np.float64)
    import torch

    t = torch.from_numpy(r.view(np.int16))
    dt = torch.bfloat16 if info.rho_dtype == pkg.RHO_BF16 else torch.float16
    return t.view(dt).float().numpy().astype(np.float64)


def sums_as_i64(ctx):
    return pkg.bundle_fetch_density(ctx, pkg.DENSITY_SUMS).astype(np.int64)


def step_h(p, iteration):
    """h_i as the library passes it to the kernels (computed in double, rounded to float)."""
    return float(np.float32(oracle.bandwidth(iteration, p.radius, p.passes, p.h_max_sigmas,
                                             p.lambda_)))


def edge_of_points(off):
    n = np.diff(off)
    return np.repeat(np.arange(len(n)), n), np.concatenate([np.arange(k) for k in n])


def advect_mismatch(off, R, group, rho, h, p, gpu_P, tol):
    """Compare the GPU's advected + smoothed points with the oracle's from the same inputs.

    Returns (n_mismatch, n_unexplained, oracle_P). A point whose position differs by more
    than `tol` is explained when it or a neighbour on its polyline (the Laplacian mixes
    three points) has an ambiguous advection in the oracle's own evaluation: a gradient too
    small for its direction to be resolved in FP32 (|g| <= 1e-4 |rho|), or a step test with
    |rho(x'_t) - rho(x)| within 1e-5 of the densities for a trial t up to the accepted one.
    """
    fixed = bool(p.flags & pkg.FLAG_FIXED_STEP)
    P_o, acc = oracle.advect_laplace(off, R, group, rho, h, eps=float(p.eps), tries=p.step_tries,
                                     beta=float(p.laplace_beta), fixed_step=fixed)
    err = np.hypot(*(gpu_P - P_o).T)
    bad = np.flatnonzero(err > tol)
    if len(bad) == 0:
        return 0, 0, P_o
    eidx, jidx = edge_of_points(off)
    cand = set()
    for k in bad:
        for d in (-1, 0, 1):
            q = k + d
            if 0 <= q < len(R) and eidx[q] == eidx[k]:
                cand.add(q)
    cand = np.array(sorted(cand))
    amb = np.zeros(len(R), bool)
    G, H, W = rho.shape
    for q in cand:
        if acc[q] == -2:
            continue
        layer = rho[group[eidx[q]] if group is not None else 0]
        x = R[q:q + 1]
        r0, g = oracle.density_at(layer, x)
        gn = float(np.hypot(*g[0]))
        if gn <= 1e-4 * abs(r0[0]) + 1e-30:
            amb[q] = True
            continue
        if fixed:  # no step test: only the direction can be ambiguous
            continue
        d = g[0] / max(gn, float(p.eps))
        last = acc[q] if acc[q] >= 0 else p.step_tries - 1
        for t in range(last + 1):
            m = h * 2.0 ** -t
            xt = x + m * d
            xt[0, 0] = min(max(xt[0, 0], 0.0), W - 2.0 ** -10)
            xt[0, 1] = min(max(xt[0, 1], 0.0), H - 2.0 ** -10)
            rt, _ = oracle.density_at(layer, xt)
            if abs(rt[0] - r0[0]) <= 1e-5 * (abs(rt[0]) + abs(r0[0])) + 1e-30:
                amb[q] = True
                break
    unexplained = 0
    for k in bad:
        near = [k + d for d in (-1, 0, 1) if 0 <= k + d < len(R) and eidx[k + d] == eidx[k]]
        if not amb[near].any():
            unexplained += 1
    return len(bad), unexplained, P_o


def resample_mismatch(off_in, P, off_gpu, R_gpu, p, tol, directed_px=0.0, grid=None):
    """Oracle resampling of the GPU's polylines vs the GPU's. A count that differs must come
    from an arc length within FP32 rounding of a multiple of delta (by-length mode only).
    directed_px: the directed-graph normal offset of the first sampling (Sec. 3)."""
    o_off, o_R = oracle.resample(off_in, P, p.n_fixed, p.n_max, float(p.delta_px))
    if directed_px:
        o_R = oracle.directed_offset(o_off, o_R, directed_px, grid[0], grid[1])
    cg, co = np.diff(off_gpu), np.diff(o_off)
    diff_cnt = np.flatnonzero(cg != co)
    unexplained = 0
    for e in diff_cnt:
        seg = np.diff(P[off_in[e]:off_in[e + 1]], axis=0)
        L = float(np.hypot(seg[:, 0], seg[:, 1]).sum())
        q = L / float(p.delta_px)
        n_pts = off_in[e + 1] - off_in[e]
        if p.n_fixed > 0 or abs(q - round(q)) > 1e-5 * max(q, 1.0) * n_pts:
            unexplained += 1
    same = np.flatnonzero(cg == co)
    worst = 0.0
    if len(same):
        mask_g = np.repeat(cg == co, cg)
        mask_o = np.repeat(cg == co, co)
        worst = float(np.abs(R_gpu[mask_g] - o_R[mask_o]).max())
    return len(diff_cnt), unexplained, worst
