"""Pins of the FP64 oracle against brute force, closed forms and invariants.

None of these re-types the oracle's own formula: each expected value comes
from a different route (numpy's symmetric padding, a hand-worked polyline, the
analytic derivative of a quadratic, the variance of a box filter, ...), so a
dropped term, a flipped sign or a transposed index in the oracle fails here.
"""
import math

import numpy as np
import pytest


# ----------------------------------------------------------------- grid map (Sec. 5)
def test_grid_map_unit_square(oracle_mod):
    src = np.array([[0.0, 0.0], [0.25, 0.5]], np.float32)
    dst = np.array([[1.0, 1.0], [0.75, 0.125]], np.float32)
    W, H, mp, sp, dp = oracle_mod.grid_map(src, dst, 256, 256, margin=4)
    assert (W, H) == (256, 256)
    # bbox [0,1]^2 onto [4, 252]: scale 248, offset 4
    assert mp[2] == 248.0 and mp[3] == 4.0 and mp[4] == 4.0
    np.testing.assert_array_equal(sp, [[4.0, 4.0], [66.0, 128.0]])
    np.testing.assert_array_equal(dp, [[252.0, 252.0], [190.0, 35.0]])


def test_grid_map_auto_dominant_and_centering(oracle_mod):
    # bounding box 2 x 1: dominant dimension 800 on x, 400 on y (Sec. 5)
    src = np.array([[0.0, 0.0]], np.float32)
    dst = np.array([[2.0, 1.0]], np.float32)
    W, H, mp, sp, dp = oracle_mod.grid_map(src, dst, 0, 0, dominant=800, margin=10)
    assert (W, H) == (800, 400)
    assert mp[2] == 380.0  # min(780 / 2, 380 / 1)
    # x span 760 -> offset (800 - 760) / 2 = 20; y span 380 -> offset (400 - 380) / 2 = 10
    np.testing.assert_array_equal(sp, [[20.0, 10.0]])
    np.testing.assert_array_equal(dp, [[780.0, 390.0]])
    # tall box: dominant on y
    W, H, *_ = oracle_mod.grid_map(np.array([[0, 0]], np.float32), np.array([[1, 4]], np.float32),
                                   0, 0, dominant=800, margin=4)
    assert (W, H) == (200, 800)


# ----------------------------------------------------------------- resampling (Sec. 2.1, Sec. 3)
def test_resample_L_shape_fixed_count(oracle_mod):
    off = np.array([0, 3], np.int64)
    xy = np.array([[0, 0], [4, 0], [4, 3]], np.float64)
    o, q = oracle_mod.resample(off, xy, n_fixed=8)
    assert list(o) == [0, 8]
    expect = [[0, 0], [1, 0], [2, 0], [3, 0], [4, 0], [4, 1], [4, 2], [4, 3]]
    np.testing.assert_allclose(q, expect, atol=1e-12)


def test_resample_by_length(oracle_mod):
    off = np.array([0, 3], np.int64)
    xy = np.array([[0, 0], [4, 0], [4, 3]], np.float64)
    # L = 7, delta = 2: ceil(3.5) + 1 = 5 points at arc lengths 0, 1.75, 3.5, 5.25, 7
    o, q = oracle_mod.resample(off, xy, n_fixed=0, n_max=64, delta=2.0)
    assert list(o) == [0, 5]
    np.testing.assert_allclose(q, [[0, 0], [1.75, 0], [3.5, 0], [4, 1.25], [4, 3]], atol=1e-12)
    # n_max clamps; a zero-length edge still keeps two points, both on the source
    o, q = oracle_mod.resample(off, xy, n_fixed=0, n_max=3, delta=0.1)
    assert list(o) == [0, 3]
    z_off = np.array([0, 2], np.int64)
    z = np.array([[5.5, 6.5], [5.5, 6.5]])
    o, q = oracle_mod.resample(z_off, z, n_fixed=4)
    np.testing.assert_array_equal(q, [[5.5, 6.5]] * 4)
    o, q = oracle_mod.resample(z_off, z, n_fixed=0, n_max=64, delta=2.0)
    assert list(o) == [0, 2]


def test_resample_straight_edge_is_fixed_point_and_endpoints_exact(oracle_mod):
    rng = np.random.default_rng(7)
    E = 50
    a = rng.uniform(5, 120, (E, 2))
    b = rng.uniform(5, 120, (E, 2))
    off, xy = oracle_mod.straight_polylines(a, b)
    o1, q1 = oracle_mod.resample(off, xy, n_fixed=9)
    o2, q2 = oracle_mod.resample(o1, q1, n_fixed=9)
    np.testing.assert_allclose(q2, q1, atol=1e-10)
    # endpoints copied bit for bit
    np.testing.assert_array_equal(q1[o1[:-1]], a)
    np.testing.assert_array_equal(q1[o1[1:] - 1], b)
    # equal spacing L / (n - 1) on each straight edge
    for e in range(E):
        seg = np.diff(q1[o1[e]:o1[e + 1]], axis=0)
        d = np.hypot(seg[:, 0], seg[:, 1])
        np.testing.assert_allclose(d, np.linalg.norm(b[e] - a[e]) / 8, rtol=1e-9)


# ----------------------------------------------------------------- histogram (Eq. 1, Eq. 3)
def test_splat_hand_enumerated(oracle_mod):
    off = np.array([0, 3, 5], np.int64)
    xy = np.array([[0.5, 0.5], [1.99, 0.01], [3.999, 2.5],   # edge 0, group 1, weight 2
                   [1.0, 1.0], [0.0, 2.999]], np.float64)    # edge 1, group 0, weight 3
    hist = oracle_mod.splat(off, xy, np.array([1, 0]), np.array([2, 3]), 2, 3, 4)
    expect = np.zeros((2, 3, 4), np.int64)
    expect[1, 0, 0] += 2
    expect[1, 0, 1] += 2
    expect[1, 2, 3] += 2
    expect[0, 1, 1] += 3
    expect[0, 2, 0] += 3
    np.testing.assert_array_equal(hist, expect)
    assert hist.sum() == 2 * 3 + 3 * 2  # mass = sum_e w_e n_e


# ----------------------------------------------------------------- smoothing (Sec. 3.1)
def _box_brute(X, r, k):
    """k passes of the (2r+1)^2 box sum with half-sample symmetric reflection (numpy pad)."""
    Y = X.astype(object)
    H, W = X.shape
    for _ in range(k):
        P = np.pad(Y, r, mode="symmetric")
        out = np.zeros_like(Y)
        for dv in range(2 * r + 1):
            for du in range(2 * r + 1):
                out = out + P[dv:dv + H, du:du + W]
        Y = out
    return Y.astype(np.int64)


def test_numpy_symmetric_pad_is_half_sample_reflection():
    np.testing.assert_array_equal(np.pad([1, 2, 3], 2, mode="symmetric"), [2, 1, 1, 2, 3, 3, 2])


@pytest.mark.parametrize("H,W", [(7, 5), (16, 16), (5, 9), (3, 4)])
@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_smooth_matches_brute_force(oracle_mod, H, W, r, k):
    if r >= min(H, W):
        pytest.skip("radius must stay below the grid size")
    rng = np.random.default_rng(H * 100 + W * 10 + r + k)
    X = rng.integers(0, 50, (2, H, W)).astype(np.int64)
    S = oracle_mod.smooth(X, r, k)
    for g in range(2):
        np.testing.assert_array_equal(S[g], _box_brute(X[g], r, k))
    # each pass multiplies the mass by exactly (2r+1)^2
    assert S.sum() == X.sum() * (2 * r + 1) ** (2 * k)


def test_smooth_variance_closed_form(oracle_mod):
    # impulse far from the border: each pass adds r(r+1)/3 to the variance per axis
    r, k, n = 3, 4, 64
    X = np.zeros((1, n, n), np.int64)
    X[0, n // 2, n // 2 + 1] = 1
    S = oracle_mod.smooth(X, r, k)[0].astype(np.float64)
    tot = S.sum()
    assert tot == (2 * r + 1) ** (2 * k)
    v, u = np.mgrid[0:n, 0:n]
    mu = (S * u).sum() / tot, (S * v).sum() / tot
    assert mu == (n // 2 + 1, n // 2)
    var_u = (S * (u - mu[0]) ** 2).sum() / tot
    var_v = (S * (v - mu[1]) ** 2).sum() / tot
    assert var_u == pytest.approx(k * r * (r + 1) / 3, rel=1e-12)
    assert var_v == pytest.approx(k * r * (r + 1) / 3, rel=1e-12)
    # the k-pass profile approaches a Gaussian of that sigma (Kovesi; Eq. 2 target)
    prof = S[n // 2] / S[n // 2].sum()
    sig = math.sqrt(k * r * (r + 1) / 3)
    gauss = np.exp(-0.5 * ((u[0] - mu[0]) / sig) ** 2)
    gauss /= gauss.sum()
    assert np.abs(prof - gauss).max() < 0.1 * gauss.max()


def test_smooth_impulse_approaches_gaussian(oracle_mod):
    """Sec. 3.1 (repeated averaging filters approximate a Gaussian): the k-pass response to an
    impulse, normalised by s^k, keeps unit mass and its L2 distance to the Gaussian of
    sigma^2 = k r (r+1) / 3 shrinks as k grows (central limit), below 8 % from k = 3 on."""
    r = 4
    errs = []
    for k in (1, 2, 3, 4, 6):
        n = 6 * r * k + 1
        h = np.zeros((1, n, n), np.int64)
        c = n // 2
        h[0, c, c] = 1
        S = oracle_mod.smooth(h, r, k)[0].astype(float) / float((2 * r + 1) ** (2 * k))
        assert abs(S.sum() - 1.0) < 1e-12
        x = np.arange(n) - c
        g = np.exp(-x ** 2 / (2 * k * r * (r + 1) / 3))
        g /= g.sum()
        G = np.outer(g, g)
        errs.append(np.linalg.norm(S - G) / np.linalg.norm(G))
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[2] < 0.08 and errs[-1] < 0.04


def test_smooth_mirror_symmetry(oracle_mod):
    rng = np.random.default_rng(3)
    X = rng.integers(0, 9, (1, 12, 10)).astype(np.int64)
    S = oracle_mod.smooth(X, 2, 3)
    Sm = oracle_mod.smooth(X[:, :, ::-1].copy(), 2, 3)
    np.testing.assert_array_equal(Sm, S[:, :, ::-1])
    St = oracle_mod.smooth(X[:, ::-1, :].copy(), 2, 3)
    np.testing.assert_array_equal(St, S[:, ::-1, :])


# ----------------------------------------------------------------- layer interaction (Eq. 3, Eq. 4)
def test_combine_identities(oracle_mod):
    rng = np.random.default_rng(11)
    r, k = 2, 2
    sk = float((2 * r + 1) ** (2 * k))
    S = rng.integers(0, 10**9, (4, 6, 7)).astype(np.int64)
    # one group: density = S / s^k
    np.testing.assert_allclose(oracle_mod.combine(S[:1], r, k)[0], S[0] / sk, rtol=1e-15)
    # alpha = 0: M is the identity, layers independent
    np.testing.assert_allclose(oracle_mod.combine(S, r, k, 0, 1), S / sk, rtol=1e-15)
    # two groups, alpha = 1/4: rho_0 = (S_0 - S_1 / 4) / s^k  (B - 1 = 1)
    rho2 = oracle_mod.combine(S[:2], r, k, 1, 4)
    np.testing.assert_allclose(rho2[0], (S[0] - 0.25 * S[1]) / sk, rtol=1e-12)
    np.testing.assert_allclose(rho2[1], (S[1] - 0.25 * S[0]) / sk, rtol=1e-12)
    # four groups: each column of M sums to 1 - alpha
    rho4 = oracle_mod.combine(S, r, k, 1, 4)
    np.testing.assert_allclose(rho4.sum(0), 0.75 * S.sum(0) / sk, rtol=1e-12)
    # a group whose histogram is empty is pushed below zero where others are dense
    S2 = S.copy()
    S2[2] = 0
    assert (oracle_mod.combine(S2, r, k, 1, 4)[2] <= 0).all()


# ----------------------------------------------------------------- density and gradient (Eq. 5)
def test_density_uniform_and_linear(oracle_mod):
    H, W = 12, 16
    pts = np.array([[0.0, 0.0], [3.3, 4.7], [15.99, 11.99], [8.5, 6.5]])
    rho, grad = oracle_mod.density_at(np.full((H, W), 2.5), pts)
    np.testing.assert_allclose(rho, 2.5)
    np.testing.assert_array_equal(grad, 0.0)
    # linear ramp in cell values: rho(a, b) = 3a + 2b (a column, b row)
    b, a = np.mgrid[0:H, 0:W]
    ramp = 3.0 * a + 2.0 * b
    inner = np.array([[3.3, 4.7], [8.5, 6.5], [10.2, 2.9]])
    rho, grad = oracle_mod.density_at(ramp, inner)
    np.testing.assert_allclose(rho, 3 * (inner[:, 0] - 0.5) + 2 * (inner[:, 1] - 0.5), atol=1e-12)
    np.testing.assert_allclose(grad, np.tile([3.0, 2.0], (3, 1)), atol=1e-12)
    # at the centre of a border cell the reflected map gives a half central difference
    _, g = oracle_mod.density_at(ramp, np.array([[0.5, 5.5]]))
    np.testing.assert_allclose(g, [[1.5, 2.0]], atol=1e-12)


def test_gradient_of_quadratic_is_analytic_derivative(oracle_mod):
    H, W = 20, 24
    b, a = np.mgrid[0:H, 0:W]
    cu, cv = 11.3, 8.6
    q = -((a - cu) ** 2) - 2.0 * (b - cv) ** 2
    pts = np.array([[6.1, 5.2], [12.7, 9.9], [17.25, 14.5]])
    _, g = oracle_mod.density_at(q, pts)
    u, v = pts[:, 0] - 0.5, pts[:, 1] - 0.5
    np.testing.assert_allclose(g[:, 0], -2 * (u - cu), atol=1e-9)
    np.testing.assert_allclose(g[:, 1], -4 * (v - cv), atol=1e-9)


def test_bandwidth_schedule(oracle_mod):
    r, k = 8, 3
    sig = math.sqrt(k * r * (r + 1) / 3)
    assert oracle_mod.bandwidth(0, r, k, 2.0, 0.9) == pytest.approx(2 * sig, rel=1e-15)
    assert oracle_mod.bandwidth(5, r, k, 2.0, 0.9) == pytest.approx(2 * sig * 0.9**5, rel=1e-14)


# ----------------------------------------------------------------- advection + Laplacian (Sec. 3.3)
def test_advect_ramp_closed_form(oracle_mod):
    H, W = 40, 40
    b, a = np.mgrid[0:H, 0:W]
    rho = (3.0 * a + 2.0 * b)[None]
    off = np.array([0, 3], np.int64)
    xy = np.array([[10.0, 10.0], [20.3, 18.7], [30.0, 12.0]])
    h = 2.5
    out, acc = oracle_mod.advect_laplace(off, xy, [0], rho, h, beta=0.5)
    d = np.array([3.0, 2.0]) / math.sqrt(13)
    A1 = xy[1] + h * d
    P1 = 0.5 * A1 + 0.5 * (xy[0] + xy[2]) / 2
    np.testing.assert_allclose(out[1], P1, atol=1e-12)
    np.testing.assert_array_equal(out[[0, 2]], xy[[0, 2]])
    assert list(acc) == [-2, 0, -2]


@pytest.mark.parametrize("delta0,h,expect_t", [(0.7, 4.0, 2), (1.0, 2.0, 0), (0.2, 4.0, 4),
                                               (0.001, 4.0, -1)])
def test_advect_halving_closed_form(oracle_mod, delta0, h, expect_t):
    # rho(a) = -(a - c)^2 along x only; the bilinear map is symmetric about u = c, so a
    # trial u + m is accepted iff m <= 2 * delta0 (ties accepted)
    H, W, c = 8, 32, 15
    b, a = np.mgrid[0:H, 0:W]
    rho = (-((a - c) ** 2)).astype(np.float64)[None]
    u = c - delta0
    px = u + 0.5
    off = np.array([0, 3], np.int64)
    xy = np.array([[2.0, 4.0], [px, 4.5], [30.0, 4.0]])
    out, acc = oracle_mod.advect_laplace(off, xy, [0], rho, h, tries=8, beta=0.0)
    assert acc[1] == expect_t
    moved = h * 2.0 ** -expect_t if expect_t >= 0 else 0.0
    np.testing.assert_allclose(out[1], [px + moved, 4.5], atol=1e-12)


def test_advect_accepted_moves_never_lower_density(oracle_mod):
    rng = np.random.default_rng(5)
    H, W = 32, 48
    rho = oracle_mod.smooth(rng.integers(0, 5, (1, H, W)), 2, 2).astype(np.float64)
    E, n = 30, 6
    off = np.arange(0, E * n + 1, n, dtype=np.int64)
    xy = np.column_stack([rng.uniform(0, W - 0.01, E * n), rng.uniform(0, H - 0.01, E * n)])
    out, acc = oracle_mod.advect_laplace(off, xy, np.zeros(E, np.int32), rho, 3.0, beta=0.0)
    r0, _ = oracle_mod.density_at(rho[0], xy)
    r1, _ = oracle_mod.density_at(rho[0], out)
    assert (r1 >= r0).all()
    moved = acc >= 0
    assert moved.sum() > E  # most interior points do move
    np.testing.assert_array_equal(out[acc == -1], xy[acc == -1])


def test_advect_clamps_to_drawing_area(oracle_mod):
    H, W = 16, 16
    b, a = np.mgrid[0:H, 0:W]
    rho = (1.0 * a)[None]  # rises towards the right border
    off = np.array([0, 3], np.int64)
    xy = np.array([[2.0, 8.0], [15.5, 8.5], [3.0, 8.0]])
    out, acc = oracle_mod.advect_laplace(off, xy, [0], rho, 5.0, beta=0.0)
    assert out[1, 0] == W - 2.0**-10


# ----------------------------------------------------------------- whole loop (Sec. 3, Fig. 2)
def _tiny_graph(seed, E, G, W=64, H=48):
    rng = np.random.default_rng(seed)
    a = np.column_stack([rng.uniform(4, W - 4, E), rng.uniform(4, H - 4, E)])
    b = np.column_stack([rng.uniform(4, W - 4, E), rng.uniform(4, H - 4, E)])
    g = rng.integers(0, G, E).astype(np.int32)
    return a, b, g


def test_run_mass_endpoints_and_single_group(oracle_mod):
    a, b, g = _tiny_graph(1, 40, 3)
    off, xy = oracle_mod.straight_polylines(a, b)
    prm = oracle_mod.Params(radius=2, passes=3, n_fixed=0, n_max=16, delta=3.0)
    w = np.arange(1, 41, dtype=np.int32)
    res = oracle_mod.run(off, xy, g, w, 3, 48, 64, prm, n_iters=3, keep_last=True)
    counts = np.diff(res.res_off)
    assert res.hist.sum() == (w * counts).sum()
    np.testing.assert_array_equal(res.xy[res.off[:-1]], a)
    np.testing.assert_array_equal(res.xy[res.off[1:] - 1], b)
    assert res.sums.sum() == res.hist.sum() * 25**3
    # with one group alpha plays no part (Eq. 4 has no off-diagonal)
    z = np.zeros(40, np.int32)
    r1 = oracle_mod.run(off, xy, z, w, 1, 48, 64, prm, n_iters=3)
    prm2 = oracle_mod.Params(**{**prm.__dict__, "alpha_num": 3, "alpha_den": 5})
    r2 = oracle_mod.run(off, xy, z, w, 1, 48, 64, prm2, n_iters=3)
    np.testing.assert_array_equal(r1.xy, r2.xy)


def test_run_alpha_zero_decouples_groups(oracle_mod):
    # M = identity: a G-group run equals G independent single-group runs, bit for bit
    a, b, g = _tiny_graph(2, 60, 3)
    off, xy = oracle_mod.straight_polylines(a, b)
    prm = oracle_mod.Params(radius=2, passes=2, alpha_num=0, alpha_den=1, n_fixed=8)
    full = oracle_mod.run(off, xy, g, None, 3, 48, 64, prm, n_iters=3)
    for grp in range(3):
        sel = np.flatnonzero(g == grp)
        o2, x2 = oracle_mod.straight_polylines(a[sel], b[sel])
        part = oracle_mod.run(o2, x2, np.zeros(len(sel), np.int32), None, 1, 48, 64, prm, n_iters=3)
        mine = np.concatenate([full.xy[full.off[e]:full.off[e + 1]] for e in sel])
        np.testing.assert_array_equal(part.xy, mine)


def test_run_mirror_symmetry(oracle_mod):
    W, H = 64, 48
    a, b, g = _tiny_graph(3, 30, 2, W, H)
    off, xy = oracle_mod.straight_polylines(a, b)
    am, bm = a.copy(), b.copy()
    am[:, 0] = W - a[:, 0]
    bm[:, 0] = W - b[:, 0]
    offm, xym = oracle_mod.straight_polylines(am, bm)
    prm = oracle_mod.Params(radius=3, passes=3, n_fixed=10)
    r = oracle_mod.run(off, xy, g, None, 2, H, W, prm, n_iters=2, keep_last=True)
    rm = oracle_mod.run(offm, xym, g, None, 2, H, W, prm, n_iters=2, keep_last=True)
    np.testing.assert_array_equal(rm.hist, r.hist[:, :, ::-1])
    np.testing.assert_array_equal(rm.sums, r.sums[:, :, ::-1])
    np.testing.assert_allclose(W - rm.xy[:, 0], r.xy[:, 0], atol=1e-9)
    np.testing.assert_allclose(rm.xy[:, 1], r.xy[:, 1], atol=1e-9)


def test_run_parallel_edges_attract(oracle_mod):
    # two close parallel edges (gap 3.4 px, below sigma) are pulled together (Sec. 2.1): with a
    # step below the gap the gap shrinks every iteration until it is within one cell
    W, H = 96, 64
    a = np.array([[10.0, 30.3], [10.0, 33.7]])
    b = np.array([[86.0, 30.3], [86.0, 33.7]])
    off, xy = oracle_mod.straight_polylines(a, b)
    prm = oracle_mod.Params(radius=3, passes=3, n_fixed=20, h_max_sigmas=0.2)
    gaps = []
    for it in range(1, 6):
        r = oracle_mod.run(off, xy, None, None, 1, H, W, prm, n_iters=it)
        mid0, mid1 = r.xy[r.off[0] + 10], r.xy[r.off[1] + 10]
        gaps.append(mid1[1] - mid0[1])
    assert 3.4 > gaps[0] > gaps[1] > 0
    assert max(abs(g) for g in gaps[2:]) < 0.5


def test_run_single_edge_on_centre_row_stays(oracle_mod):
    W, H = 64, 32
    off, xy = oracle_mod.straight_polylines([[5.0, 16.5]], [[60.0, 16.5]])
    prm = oracle_mod.Params(radius=2, passes=3, n_fixed=12)
    r = oracle_mod.run(off, xy, None, None, 1, H, W, prm, n_iters=4)
    np.testing.assert_allclose(r.xy[:, 1], 16.5, atol=1e-12)


# ----------------------------------------------------------------- variants (Sec. 3, Sec. 3.2, Sec. 3.3)
def test_fixed_step_moves_by_h_even_downhill(oracle_mod):
    # KDEEB's step (Sec. 3.3, Fig. 3): magnitude h, no density test -- on the quadratic
    # bump a point 0.2 px below the peak with h = 4 overshoots to a lower density
    H, W, c = 8, 32, 15
    b, a = np.mgrid[0:H, 0:W]
    rho = (-((a - c) ** 2)).astype(np.float64)[None]
    px = c - 0.2 + 0.5
    off = np.array([0, 3], np.int64)
    xy = np.array([[2.0, 4.0], [px, 4.5], [30.0, 4.0]])
    out, acc = oracle_mod.advect_laplace(off, xy, [0], rho, 4.0, beta=0.0, fixed_step=True)
    np.testing.assert_allclose(out[1], [px + 4.0, 4.5], atol=1e-12)
    r0, _ = oracle_mod.density_at(rho[0], xy[1:2])
    r1, _ = oracle_mod.density_at(rho[0], out[1:2])
    assert r1[0] < r0[0]
    opt, _ = oracle_mod.advect_laplace(off, xy, [0], rho, 4.0, beta=0.0)
    assert abs(opt[1, 0] - px) < 0.5  # the optimised step only takes a small, uphill move


def test_combine_matrix_routes_agree(oracle_mod):
    rng = np.random.default_rng(21)
    r, k = 2, 3
    sk = float((2 * r + 1) ** (2 * k))
    S = rng.integers(0, 10**8, (3, 5, 6)).astype(np.int64)
    np.testing.assert_allclose(oracle_mod.combine_matrix(S, r, k, np.eye(3)), S / sk, rtol=1e-15)
    # Eq. 4 as a matrix equals the alpha form
    alpha = 0.25
    M = np.full((3, 3), -alpha / 2)
    np.fill_diagonal(M, 1.0)
    np.testing.assert_allclose(oracle_mod.combine_matrix(S, r, k, M),
                               oracle_mod.combine(S, r, k, 1, 4), rtol=1e-12)
    # an ordinal interaction (neighbouring bins attract half as much) on two groups
    Mo = np.array([[1.0, 0.5], [0.5, 1.0]])
    rho = oracle_mod.combine_matrix(S[:2], r, k, Mo)
    np.testing.assert_allclose(rho[0], (S[0] + 0.5 * S[1]) / sk, rtol=1e-12)


def test_directed_offset_separates_opposite_edges(oracle_mod):
    # Sec. 3: interior points move along the normal (-dy, dx)/|d| of their edge, so the
    # same segment drawn in opposite directions splits into two lines 2 * amount apart
    off, xy = oracle_mod.straight_polylines([[10.0, 20.0], [50.0, 20.0]],
                                            [[50.0, 20.0], [10.0, 20.0]])
    r_off, r_xy = oracle_mod.resample(off, xy, n_fixed=9)
    moved = oracle_mod.directed_offset(r_off, r_xy, 0.75, 64, 48)
    a, b = moved[r_off[0]:r_off[1]], moved[r_off[1]:r_off[2]]
    np.testing.assert_allclose(a[1:-1, 1], 20.75)
    np.testing.assert_allclose(b[1:-1, 1], 19.25)
    np.testing.assert_array_equal(a[[0, -1]], r_xy[[0, 8]])
    np.testing.assert_array_equal(b[[0, -1]], r_xy[[9, 17]])
    np.testing.assert_allclose(a[1:-1, 0], r_xy[1:8, 0])


# ----------------------------------------------------------------- segment histogram (Eq. 1, Sec. 4)
def _cells(hist):
    return sorted(zip(*np.nonzero(hist[0])))


def test_segment_histogram_hand_enumerated(oracle_mod):
    H, W = 12, 16
    # horizontal, vertical and 45-degree segments: every cell between the end cells
    for a, b, cells in [((1.5, 2.5), (6.2, 2.9), [(2, x) for x in range(1, 7)]),
                        ((3.1, 9.9), (3.7, 4.0), [(y, 3) for y in range(4, 10)]),
                        ((0.5, 0.5), (4.5, 4.5), [(i, i) for i in range(5)])]:
        off, xy = oracle_mod.straight_polylines([a], [b])
        assert _cells(oracle_mod.splat_segments(off, xy, None, None, 1, H, W)) == cells
    # a shallow line: one cell per column (the major axis), rows from the Bresenham rule
    off, xy = oracle_mod.straight_polylines([[0.5, 0.5]], [[8.5, 3.5]])
    hist = oracle_mod.splat_segments(off, xy, None, None, 1, H, W)
    assert hist.sum() == 9 and (hist[0].sum(0)[:9] == 1).all()
    assert _cells(hist)[0] == (0, 0) and _cells(hist)[-1] == (3, 8)


def test_segment_histogram_joints_and_weights(oracle_mod):
    # an L-shaped polyline: the corner cell is the joint of two segments and counts once;
    # a zero-length segment (both points in one cell) adds nothing
    off = np.array([0, 4], np.int64)
    xy = np.array([[1.2, 1.2], [5.7, 1.4], [5.9, 1.9], [5.5, 6.1]])
    hist = oracle_mod.splat_segments(off, xy, None, np.array([3], np.int32), 1, 8, 8)
    expect = {(1, x) for x in range(1, 6)} | {(y, 5) for y in range(1, 7)}
    assert set(_cells(hist)) == expect
    assert (hist[hist > 0] == 3).all() and hist.sum() == 3 * len(expect)
    # a polyline whose points are all in one cell counts that cell once
    off = np.array([0, 3], np.int64)
    xy = np.array([[2.1, 2.1], [2.5, 2.9], [2.9, 2.2]])
    assert oracle_mod.splat_segments(off, xy, None, None, 1, 8, 8).sum() == 1


# ------------------------------------------------- convergence: optimised vs fixed step (Fig. 3)
def test_ink_counts_occupied_cells(oracle_mod):
    hist = np.zeros((2, 3, 4), np.int64)
    hist[0, 0, 0] = hist[0, 1, 2] = 5
    hist[1, 1, 2] = hist[1, 2, 3] = hist[1, 0, 1] = 1
    # union {(0,0), (1,2), (2,3), (0,1)}; group 0 has 2 cells, group 1 has 3; (1,2) is shared
    assert oracle_mod.ink(hist) == (4, 5)
    assert oracle_mod.ink(np.zeros((3, 2, 2), np.int64)) == (0, 0)


def test_optimised_step_converges_in_fewer_iterations(oracle_mod):
    """Sec. 3.3 / Fig. 3: with the density test the bundling tightens faster than with KDEEB's
    fixed step. Measured as the ink (occupied cells of the segment-rasterised drawing) entering
    each iteration, on the 1,000-edge uniform graph (256^2, r = 4, k = 3): the optimised step is
    tighter at every iteration after the first and reaches the fixed step's 10-iteration ink in
    at most 8 iterations."""
    from paper_1504_02687_gb300 import synth

    w = synth.small(n_edges=1000)
    W, H = w.grid
    _, _, _, sp, dp = oracle_mod.grid_map(w.src_xy, w.dst_xy, W, H, margin=w.radius)
    off, xy = oracle_mod.straight_polylines(sp, dp)
    ink = {}
    for fixed in (False, True):
        prm = oracle_mod.Params(radius=w.radius, passes=w.passes, n_fixed=w.n_fixed,
                                n_max=w.n_max, delta=w.delta, fixed_step=fixed, segment_hist=True)
        o, P, row = off, xy, []
        for i in range(10):
            r = oracle_mod.run(o, P, w.group, w.weight, 1, H, W, prm, i, 1, keep_last=True)
            row.append(oracle_mod.ink(r.hist)[0])
            o, P = r.off, r.xy
        ink[fixed] = np.array(row)
    assert ink[False][0] == ink[True][0]          # the same straight drawing enters iteration 0
    assert (ink[False][1:] < ink[True][1:]).all()
    assert np.flatnonzero(ink[False] <= ink[True][-1])[0] <= 8
    assert (np.diff(ink[False]) < 0).all()        # and the ink falls every iteration


# ----------------------------------------------------------- headless rendering (Sec. 3.4)
TAU_04 = 535639  # llround(-ln(1 - 0.4) * 2^20)


def _render(oracle_mod, pts, G=1, group=None, weight=None, rho=None, H=8, W=10, **kw):
    off = np.cumsum([0] + [len(p) for p in pts]).astype(np.int64)
    xy = np.concatenate([np.asarray(p, float) for p in pts])
    rho = np.zeros((G, H, W)) if rho is None else rho
    pal = np.array([[255, 0, 0], [0, 0, 255], [0, 255, 0]][:G], np.uint8)
    kw.setdefault("alpha", 0.4)
    kw.setdefault("width_min", 1.0)
    kw.setdefault("width_max", 1.0)
    return oracle_mod.render(off, xy, group, weight, rho, pal, **kw)


def _covered(acc):
    return sorted(zip(*np.nonzero(acc[..., 0])))


def test_render_single_segment(oracle_mod):
    acc, amb, rgba = _render(oracle_mod, [[(2.5, 3.5), (7.5, 3.5)]])
    assert _covered(acc) == [(3, x) for x in range(2, 8)]
    assert (acc[3, 2:8, 0] == TAU_04).all() and (acc[3, 2:8, 1] == 255 * TAU_04).all()
    assert not amb.any()
    # opacity 1 - exp(-tau) = 0.4 over black: red 0.4 * 255 = 102
    assert (rgba[3, 2:8] == [102, 0, 0, 255]).all()
    assert (rgba[0, 0] == [0, 0, 0, 255]).all()


def test_render_crossing_joint_and_weight(oracle_mod):
    # red horizontal and blue vertical edge cross at pixel (3, 5): twice the depth, mixed colour
    acc, amb, rgba = _render(oracle_mod, [[(2.5, 3.5), (7.5, 3.5)], [(5.5, 0.5), (5.5, 7.5)]],
                             G=2, group=np.array([0, 1], np.int32))
    assert acc[3, 5, 0] == 2 * TAU_04 and acc[3, 5, 1] == acc[3, 5, 3] == 255 * TAU_04
    # A = 1 - 0.6^2 = 0.64 of the mean colour (127.5, 0, 127.5): 81.6 -> 82
    assert (rgba[3, 5] == [82, 0, 82, 255]).all()
    # an L-shaped polyline: the corner pixel is the end of one segment and the start of the
    # next, and is drawn once
    acc, amb, _ = _render(oracle_mod, [[(2.5, 2.5), (6.5, 2.5), (6.5, 6.5)]])
    expect = {(2, x) for x in range(2, 7)} | {(y, 6) for y in range(2, 7)}
    assert set(_covered(acc)) == expect and (acc[acc[..., 0] > 0, 0] == TAU_04).all()
    # weight 2 draws like two unit edges on top of each other
    a2, _, r2 = _render(oracle_mod, [[(2.5, 3.5), (7.5, 3.5)]], weight=np.array([2], np.int32))
    a11, _, r11 = _render(oracle_mod, [[(2.5, 3.5), (7.5, 3.5)]] * 2)
    np.testing.assert_array_equal(a2, a11)
    np.testing.assert_array_equal(r2, r11)


def test_render_width_from_density_and_scale(oracle_mod):
    seg = [[(2.5, 3.5), (7.5, 3.5)]]
    rho = np.ones((1, 8, 10))
    # uniform density at the reference: full width 3 (radius 1.5): rows 2..4, columns 1..8
    acc, amb, _ = _render(oracle_mod, seg, rho=rho, width_max=3.0)
    assert _covered(acc) == [(y, x) for y in range(2, 5) for x in range(1, 9)]
    assert not amb.any()
    # u = 0.6 of the reference: width 1 + 2 * 0.6 = 2.2 (radius 1.1): the caps lose corners
    acc, amb, _ = _render(oracle_mod, seg, rho=rho, width_max=3.0, rho_ref=1 / 0.6)
    assert set(_covered(acc)) == ({(3, x) for x in range(1, 9)} | {(2, x) for x in range(2, 8)}
                                  | {(4, x) for x in range(2, 8)})
    # log scale: u = 0.5 of the reference gives log2(1.5) = 0.585, width 1 + 2 * 0.585 = 2.17
    # (radius 1.085): the same 20 pixels as radius 1.1, and none of them near the threshold
    acc, amb, _ = _render(oracle_mod, seg, rho=rho, width_max=3.0, rho_ref=2.0, log_width=True)
    assert set(_covered(acc)) == ({(3, x) for x in range(1, 9)} | {(2, x) for x in range(2, 8)}
                                  | {(4, x) for x in range(2, 8)})
    assert not amb.any()
    # scale 2: the segment spans image x 5..15 on row 7.0; width 1.5 covers rows 6 and 7
    acc, amb, _ = _render(oracle_mod, seg, scale=2, width_max=1.5, width_min=1.5)
    assert acc.shape == (16, 20, 4)
    assert _covered(acc) == [(y, x) for y in (6, 7) for x in range(4, 16)]
