/*
 * FP64 CPU oracle for one iteration loop of 3D-density-histogram edge bundling
 * (3DHEB, "3D Density Histograms for Criteria-driven Edge Bundling", Moura).
 *
 * TEST INFRASTRUCTURE ONLY. The test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the product path never
 * does. It shares no source, header, table or helper with the CUDA path.
 *
 * Plain, single-threaded, slow on purpose: positions and densities are double,
 * histograms and smoothed sums are int64, and integral images are __int128 so
 * that no intermediate can wrap. Every function restates one step of the
 * paper's loop (Sec. 3, Fig. 2): resample -> histogram -> smooth -> combine
 * layers -> advect with the optimised step -> Laplacian smoothing.
 *
 * Readings of passages the paper leaves open (each is a parameter or a fixed
 * choice here, listed in the design notes):
 *  - histogram: every sample point adds its edge weight to the cell it falls
 *    in (Eq. 1 / Eq. 3 read as a point splat), or, as an option, every cell
 *    that the integer Bresenham line of a polyline segment visits (Sec. 4),
 *    joints counted once;
 *  - smoothing boundary: half-sample symmetric reflection (-1 -> 0, W -> W-1);
 *  - layer interaction applied after smoothing (smoothing is linear, Sec. 3.2);
 *  - gradient: central differences of the reflection-extended density at the
 *    four cell centres around the point, interpolated bilinearly;
 *  - step test: a trial is accepted when its density is not lower (ties pass);
 *    "until m is zero" becomes a fixed number of halvings;
 *  - Laplacian smoothing: one Jacobi pass with weight beta, endpoints fixed;
 *  - resampling: uniform arc-length spacing with a fixed count or
 *    clamp(ceil(L / delta) + 1, 2, n_max) points;
 *  - rendering (Sec. 3.4): capsule segments with a width from the density,
 *    order-free alpha accumulation as integer optical depth (oracle_render).
 *
 * Pinning: each function is checked by the non-GPU tests against brute force,
 * closed forms or invariants (see tests/test_oracle_*.py). The absolute
 * positions of a whole multi-iteration run have no independent pin (the paper
 * prints none): parity unpinned for oracle_run beyond those invariants.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <limits>
#include <vector>

namespace {

/* Half-sample symmetric reflection into [0, n): -1 -> 0, -2 -> 1, n -> n-1.
 * Valid for -n <= i < 2n. */
inline int64_t reflect_index(int64_t i, int64_t n) {
    if (i < 0) return -1 - i;
    if (i >= n) return 2 * n - 1 - i;
    return i;
}

/* Density of one layer on the reflection-extended plane, column a, row b. */
inline double ext_density(const double* layer, int64_t H, int64_t W, int64_t a, int64_t b) {
    return layer[reflect_index(b, H) * W + reflect_index(a, W)];
}

/* Cell-centre frame: cell (a, b) has its centre at (a + 0.5, b + 0.5). */
inline void cell_frame(double px, double py, int64_t* a0, int64_t* b0, double* fu, double* fv) {
    double u = px - 0.5, v = py - 0.5;
    double fa = std::floor(u), fb = std::floor(v);
    *a0 = (int64_t)fa;
    *b0 = (int64_t)fb;
    *fu = u - fa;
    *fv = v - fb;
}

/* Bilinear density at (px, py), pixel units. */
double bilinear_density(const double* layer, int64_t H, int64_t W, double px, double py) {
    int64_t a0, b0;
    double fu, fv;
    cell_frame(px, py, &a0, &b0, &fu, &fv);
    double e00 = ext_density(layer, H, W, a0, b0);
    double e10 = ext_density(layer, H, W, a0 + 1, b0);
    double e01 = ext_density(layer, H, W, a0, b0 + 1);
    double e11 = ext_density(layer, H, W, a0 + 1, b0 + 1);
    return (1 - fu) * (1 - fv) * e00 + fu * (1 - fv) * e10 + (1 - fu) * fv * e01 + fu * fv * e11;
}

/* Gradient of the density (Eq. 5's nabla rho): central differences at the four
 * surrounding cell centres, interpolated with the same bilinear weights. */
void bilinear_gradient(const double* layer, int64_t H, int64_t W, double px, double py,
                       double* gx, double* gy) {
    int64_t a0, b0;
    double fu, fv;
    cell_frame(px, py, &a0, &b0, &fu, &fv);
    double wx[4] = {(1 - fu) * (1 - fv), fu * (1 - fv), (1 - fu) * fv, fu * fv};
    int64_t ca[4] = {a0, a0 + 1, a0, a0 + 1};
    int64_t cb[4] = {b0, b0, b0 + 1, b0 + 1};
    double sx = 0, sy = 0;
    for (int c = 0; c < 4; ++c) {
        double dx = (ext_density(layer, H, W, ca[c] + 1, cb[c]) -
                     ext_density(layer, H, W, ca[c] - 1, cb[c])) / 2;
        double dy = (ext_density(layer, H, W, ca[c], cb[c] + 1) -
                     ext_density(layer, H, W, ca[c], cb[c] - 1)) / 2;
        sx += wx[c] * dx;
        sy += wx[c] * dy;
    }
    *gx = sx;
    *gy = sy;
}

/* Upper bound of the drawing area for positions: W - 2^-10 (exact in FP32). */
inline double clamp_pos(double v, int64_t n) {
    double hi = (double)n - 1.0 / 1024.0;
    if (v < 0) return 0;
    if (v > hi) return hi;
    return v;
}

}  // namespace

extern "C" {

int32_t oracle_abi_version(void) { return 1; }

/*
 * Bounding box -> histogram grid (Sec. 5: the dominant dimension is fixed, the
 * other follows the aspect ratio of the graph's bounding box). Explicit
 * grid_w, grid_h > 0 override the automatic size. A margin of `margin` pixels
 * is kept on every side; the scale is isotropic and the drawing is centred.
 * Pixel coordinates are computed in double and rounded to float once.
 * map_out = {xmin, ymin, scale, ox, oy}: px = (x - xmin) * scale + ox.
 * Returns 0, or 1..3 for empty input / half-specified grid / no room.
 */
int32_t oracle_grid_map(int64_t n_edges, const float* src_xy, const float* dst_xy,
                        int32_t grid_w, int32_t grid_h, int32_t dominant, int32_t margin,
                        int32_t* wh_out, double* map_out, float* src_px, float* dst_px) {
    if (n_edges <= 0) return 1;
    const double inf = std::numeric_limits<double>::infinity();
    double xmin = inf, ymin = inf, xmax = -inf, ymax = -inf;
    for (int64_t e = 0; e < n_edges; ++e) {
        const float* ends[2] = {src_xy + 2 * e, dst_xy + 2 * e};
        for (const float* q : ends) {
            double x = q[0], y = q[1];
            xmin = std::min(xmin, x);
            xmax = std::max(xmax, x);
            ymin = std::min(ymin, y);
            ymax = std::max(ymax, y);
        }
    }
    double sx = xmax - xmin, sy = ymax - ymin;
    int64_t W = grid_w, H = grid_h;
    if (W <= 0 && H <= 0) {
        int64_t lo = 2 * (int64_t)margin + 2;
        if (sx >= sy) {
            W = dominant;
            H = sx > 0 ? (int64_t)std::llround(dominant * (sy / sx)) : dominant;
        } else {
            H = dominant;
            W = (int64_t)std::llround(dominant * (sx / sy));
        }
        W = std::max(W, lo);
        H = std::max(H, lo);
    } else if (W <= 0 || H <= 0) {
        return 2;
    }
    if (W - 2 * (int64_t)margin <= 0 || H - 2 * (int64_t)margin <= 0) return 3;
    double kx = sx > 0 ? ((double)W - 2.0 * margin) / sx : inf;
    double ky = sy > 0 ? ((double)H - 2.0 * margin) / sy : inf;
    double scale = std::min(kx, ky);
    if (!(scale < inf)) scale = 1.0;
    double ox = ((double)W - scale * sx) / 2.0;
    double oy = ((double)H - scale * sy) / 2.0;
    for (int64_t e = 0; e < n_edges; ++e) {
        const float* in[2] = {src_xy + 2 * e, dst_xy + 2 * e};
        float* out[2] = {src_px + 2 * e, dst_px + 2 * e};
        for (int s = 0; s < 2; ++s) {
            double px = ((double)in[s][0] - xmin) * scale + ox;
            double py = ((double)in[s][1] - ymin) * scale + oy;
            out[s][0] = (float)clamp_pos((double)(float)px, W);
            out[s][1] = (float)clamp_pos((double)(float)py, H);
        }
    }
    wh_out[0] = (int32_t)W;
    wh_out[1] = (int32_t)H;
    map_out[0] = xmin;
    map_out[1] = ymin;
    map_out[2] = scale;
    map_out[3] = ox;
    map_out[4] = oy;
    return 0;
}

/*
 * Edge resampling (Sec. 2.1: sample points equally spaced along each edge;
 * Sec. 3: every iteration starts by re-spacing the points). For each polyline
 * the arc length L is summed segment by segment from the source; the new
 * point count is n_fixed when positive, else clamp(ceil(L / delta) + 1, 2,
 * n_max). Point j sits at arc length j * L / (n - 1) on the old polyline; the
 * first and last points are copied exactly, and L = 0 puts every point on the
 * source. Returns the number of output points, -1 if `cap` is too small, -2
 * for a polyline with fewer than two points.
 */
int64_t oracle_resample(int64_t n_edges, const int64_t* off, const double* xy,
                        int32_t n_fixed, int32_t n_max, double delta,
                        int64_t* off_out, double* xy_out, int64_t cap) {
    int64_t o = 0;
    off_out[0] = 0;
    std::vector<double> cum;
    for (int64_t e = 0; e < n_edges; ++e) {
        int64_t n = off[e + 1] - off[e];
        if (n < 2) return -2;
        const double* P = xy + 2 * off[e];
        cum.assign((size_t)n, 0.0);
        double L = 0;
        for (int64_t s = 1; s < n; ++s) {
            double dx = P[2 * s] - P[2 * s - 2], dy = P[2 * s + 1] - P[2 * s - 1];
            L += std::sqrt(dx * dx + dy * dy);
            cum[(size_t)s] = L;
        }
        int64_t m;
        if (n_fixed > 0) {
            m = n_fixed;
        } else {
            double c = std::ceil(L / delta) + 1;
            m = c > (double)n_max ? (int64_t)n_max : (int64_t)c;
            if (m < 2) m = 2;
        }
        if (o + m > cap) return -1;
        double* Q = xy_out + 2 * o;
        Q[0] = P[0];
        Q[1] = P[1];
        for (int64_t j = 1; j + 1 < m; ++j) {
            if (L == 0) {
                Q[2 * j] = P[0];
                Q[2 * j + 1] = P[1];
                continue;
            }
            double t = ((double)j * L) / (double)(m - 1);
            int64_t s = 1;
            while (s < n - 1 && !(cum[(size_t)s] > t)) ++s;
            double seg = cum[(size_t)s] - cum[(size_t)s - 1];
            double f = seg > 0 ? (t - cum[(size_t)s - 1]) / seg : 0.0;
            f = std::min(1.0, std::max(0.0, f));
            Q[2 * j] = P[2 * (s - 1)] + f * (P[2 * s] - P[2 * (s - 1)]);
            Q[2 * j + 1] = P[2 * (s - 1) + 1] + f * (P[2 * s + 1] - P[2 * (s - 1) + 1]);
        }
        Q[2 * (m - 1)] = P[2 * (n - 1)];
        Q[2 * (m - 1) + 1] = P[2 * (n - 1) + 1];
        o += m;
        off_out[e + 1] = o;
    }
    return o;
}

/*
 * Histogram of edge occurrence (Eq. 1, stacked per group as in Eq. 3 before
 * interaction): H[g][v][u] = sum of the weights w_e of sample points of edges
 * of group g that fall in cell (u, v), u = floor(x), v = floor(y), clamped to
 * the grid. Layout [G][H][W], row-major.
 */
void oracle_splat(int64_t n_edges, const int64_t* off, const double* xy, const int32_t* group,
                  const int32_t* weight, int32_t G, int32_t H, int32_t W, int64_t* hist) {
    std::fill(hist, hist + (int64_t)G * H * W, (int64_t)0);
    for (int64_t e = 0; e < n_edges; ++e) {
        int64_t g = group ? group[e] : 0;
        int64_t w = weight ? weight[e] : 1;
        for (int64_t k = off[e]; k < off[e + 1]; ++k) {
            int64_t cx = (int64_t)std::floor(xy[2 * k]);
            int64_t cy = (int64_t)std::floor(xy[2 * k + 1]);
            cx = std::min<int64_t>(std::max<int64_t>(cx, 0), W - 1);
            cy = std::min<int64_t>(std::max<int64_t>(cy, 0), H - 1);
            hist[(g * H + cy) * W + cx] += w;
        }
    }
}

/*
 * Histogram of edge occurrence by segment rasterisation (Eq. 1 with the paper's
 * Sec. 4 implementation: Bresenham lines written into the accumulation array).
 * Each segment P_{j-1} -> P_j of a polyline is walked from the cell of P_{j-1} to
 * the cell of P_j with the integer Bresenham line algorithm (8-connected, one cell
 * per step of the major axis), and every cell on the walk gains w_e; the first
 * cell of segments j >= 2 is the previous segment's last cell and is not counted
 * again. Cells are floor() of the positions, clamped to the grid.
 */
void oracle_splat_segments(int64_t n_edges, const int64_t* off, const double* xy,
                           const int32_t* group, const int32_t* weight, int32_t G, int32_t H,
                           int32_t W, int64_t* hist) {
    std::fill(hist, hist + (int64_t)G * H * W, (int64_t)0);
    auto cell = [&](double v, int64_t n) {
        int64_t c = (int64_t)std::floor(v);
        return std::min<int64_t>(std::max<int64_t>(c, 0), n - 1);
    };
    for (int64_t e = 0; e < n_edges; ++e) {
        int64_t* layer = hist + (int64_t)(group ? group[e] : 0) * H * W;
        int64_t w = weight ? weight[e] : 1;
        for (int64_t k = off[e] + 1; k < off[e + 1]; ++k) {
            int64_t x = cell(xy[2 * (k - 1)], W), y = cell(xy[2 * (k - 1) + 1], H);
            const int64_t x1 = cell(xy[2 * k], W), y1 = cell(xy[2 * k + 1], H);
            const int64_t dx = std::llabs(x1 - x), dy = -std::llabs(y1 - y);
            const int64_t sx = x < x1 ? 1 : -1, sy = y < y1 ? 1 : -1;
            int64_t err = dx + dy;
            bool first = true;
            for (;;) {
                if (!(first && k > off[e] + 1)) layer[y * W + x] += w;
                first = false;
                if (x == x1 && y == y1) break;
                const int64_t e2 = 2 * err;
                if (e2 >= dy) {
                    err += dy;
                    x += sx;
                }
                if (e2 <= dx) {
                    err += dx;
                    y += sy;
                }
            }
        }
    }
}

/*
 * Density smoothing by repeated averaging filters computed with integral
 * images (Sec. 3.1, after Kovesi's almost-Gaussian filtering and Viola-Jones
 * integral images): `passes` times, each layer X is replaced by its
 * (2r+1) x (2r+1) box sum, unnormalised, on the half-sample-reflected plane.
 * One pass builds the integral image of the reflection-extended layer
 * ((H + 2r) x (W + 2r)) and takes the four-corner difference per cell.
 * Returns 0, 1 if a box sum does not fit int64, 2 if r >= min(H, W).
 */
int32_t oracle_smooth(int32_t G, int32_t H, int32_t W, int32_t r, int32_t passes,
                      const int64_t* hist, int64_t* sums) {
    if (r < 0 || r >= H || r >= W) return 2;
    const int64_t He = (int64_t)H + 2 * r, We = (int64_t)W + 2 * r;
    const int64_t C = (int64_t)H * W;
    std::vector<__int128> I((size_t)((He + 1) * (We + 1)));
    std::vector<int64_t> X((size_t)C), Y((size_t)C);
    for (int64_t g = 0; g < G; ++g) {
        std::copy(hist + g * C, hist + (g + 1) * C, X.begin());
        for (int32_t p = 0; p < passes; ++p) {
            std::fill(I.begin(), I.end(), (__int128)0);
            for (int64_t b = 0; b < He; ++b) {
                for (int64_t a = 0; a < We; ++a) {
                    __int128 x = X[(size_t)(reflect_index(b - r, H) * W + reflect_index(a - r, W))];
                    I[(size_t)((b + 1) * (We + 1) + a + 1)] =
                        x + I[(size_t)(b * (We + 1) + a + 1)] + I[(size_t)((b + 1) * (We + 1) + a)] -
                        I[(size_t)(b * (We + 1) + a)];
                }
            }
            const int64_t d = 2 * r + 1;
            for (int64_t v = 0; v < H; ++v) {
                for (int64_t u = 0; u < W; ++u) {
                    __int128 s = I[(size_t)((v + d) * (We + 1) + u + d)] -
                                 I[(size_t)(v * (We + 1) + u + d)] -
                                 I[(size_t)((v + d) * (We + 1) + u)] + I[(size_t)(v * (We + 1) + u)];
                    if (s > (__int128)std::numeric_limits<int64_t>::max() ||
                        s < (__int128)std::numeric_limits<int64_t>::min())
                        return 1;
                    Y[(size_t)(v * W + u)] = (int64_t)s;
                }
            }
            X.swap(Y);
        }
        std::copy(X.begin(), X.end(), sums + g * C);
    }
    return 0;
}

/*
 * Layer interaction (Eq. 3 with Eq. 4), applied to the smoothed layers: since
 * smoothing is linear, smoothing each group's histogram and then mixing the
 * layers with M equals mixing first (Sec. 3.2 smooths each layer of the mixed
 * stack). M(l, b) = 1 on the diagonal and -alpha / (B - 1) elsewhere, with
 * alpha = alpha_num / alpha_den; with one group only the diagonal exists.
 * The result is normalised by s^passes, s = (2r+1)^2, i.e. expressed as
 * smoothed weight per cell.
 */
void oracle_combine(int32_t G, int32_t H, int32_t W, int32_t r, int32_t passes,
                    int32_t alpha_num, int32_t alpha_den, const int64_t* sums, double* rho) {
    const int64_t C = (int64_t)H * W;
    double s = (double)(2 * r + 1) * (double)(2 * r + 1);
    double sk = 1;
    for (int32_t p = 0; p < passes; ++p) sk *= s;
    double alpha = (double)alpha_num / (double)alpha_den;
    for (int64_t l = 0; l < G; ++l) {
        for (int64_t c = 0; c < C; ++c) {
            double acc = 0;
            for (int64_t b = 0; b < G; ++b) {
                double m = (l == b) ? 1.0 : -alpha / (double)(G - 1);
                acc += m * (double)sums[b * C + c];
            }
            rho[l * C + c] = acc / sk;
        }
    }
}

/*
 * Layer interaction with a general matrix (Eq. 3): rho_l = sum_b M(l, b) S_b / s^passes,
 * M given row-major as G x G doubles (Sec. 3.2: ordinal, modular or nominal bins can
 * use other matrices than Eq. 4's).
 */
void oracle_combine_matrix(int32_t G, int32_t H, int32_t W, int32_t r, int32_t passes,
                           const double* M, const int64_t* sums, double* rho) {
    const int64_t C = (int64_t)H * W;
    double s = (double)(2 * r + 1) * (double)(2 * r + 1);
    double sk = 1;
    for (int32_t p = 0; p < passes; ++p) sk *= s;
    for (int64_t l = 0; l < G; ++l)
        for (int64_t c = 0; c < C; ++c) {
            double acc = 0;
            for (int64_t b = 0; b < G; ++b) acc += M[l * G + b] * (double)sums[b * C + c];
            rho[l * C + c] = acc / sk;
        }
}

/*
 * Directed graphs (Sec. 3): interior sample points are translated by `amount`
 * pixels along the normal of their edge, (-dy, dx) / |d| for the direction d from
 * source to target, so edges of opposite directions separate. Applied in place
 * to polylines after their first sampling; endpoints stay.
 */
void oracle_directed_offset(int64_t n_edges, const int64_t* off, double* xy, double amount,
                            int32_t W, int32_t H) {
    for (int64_t e = 0; e < n_edges; ++e) {
        int64_t a = off[e], b = off[e + 1] - 1;
        double dx = xy[2 * b] - xy[2 * a], dy = xy[2 * b + 1] - xy[2 * a + 1];
        double len = std::sqrt(dx * dx + dy * dy);
        if (!(len > 0)) continue;
        double nx = -dy / len, ny = dx / len;
        for (int64_t k = a + 1; k < b; ++k) {
            xy[2 * k] = clamp_pos(xy[2 * k] + amount * nx, W);
            xy[2 * k + 1] = clamp_pos(xy[2 * k + 1] + amount * ny, H);
        }
    }
}

/* Bilinear density and gradient of one layer at n points (xy interleaved). */
void oracle_density_at(int32_t H, int32_t W, const double* layer, int64_t n, const double* xy,
                       double* rho_out, double* grad_out) {
    for (int64_t i = 0; i < n; ++i) {
        if (rho_out) rho_out[i] = bilinear_density(layer, H, W, xy[2 * i], xy[2 * i + 1]);
        if (grad_out)
            bilinear_gradient(layer, H, W, xy[2 * i], xy[2 * i + 1], grad_out + 2 * i,
                              grad_out + 2 * i + 1);
    }
}

/* Kernel bandwidth schedule (Sec. 2.1, Sec. 3.3): h_i = lambda^i * h_max with
 * h_max = h_max_sigmas * sigma, sigma = sqrt(passes * r (r + 1) / 3) being the
 * standard deviation of `passes` box filters of width 2r+1. */
double oracle_bandwidth(int32_t iteration, int32_t r, int32_t passes, double h_max_sigmas,
                        double lambda) {
    double sigma = std::sqrt((double)((int64_t)passes * r * (r + 1)) / 3.0);
    double h = h_max_sigmas * sigma;
    for (int32_t t = 0; t < iteration; ++t) h *= lambda;
    return h;
}

/*
 * Advection with the optimised step (Eq. 5 and Sec. 3.3), then Laplacian
 * smoothing (Sec. 2.1, Sec. 3.3). Each interior point x of edge e moves along
 * d = grad / max(|grad|, eps) of its own group's layer. The magnitude starts
 * at h and halves until the density at the clamped trial position is not
 * lower than at x; after `tries` sizes (h, h/2, ..., h / 2^(tries-1)) the
 * point stays. Endpoints never move. Then each interior point becomes
 * (1 - beta) A_j + beta (A_{j-1} + A_{j+1}) / 2 from the advected points A.
 * `accepted` (nullable) receives, per point, the accepted trial index, -1 when
 * none was accepted and -2 for endpoints.
 */
void oracle_advect_laplace_mode(int64_t n_edges, const int64_t* off, const double* xy_in,
                                const int32_t* group, int32_t G, int32_t H, int32_t W,
                                const double* rho, double h, double eps, int32_t tries,
                                double beta, int32_t fixed_step, double* xy_out,
                                int32_t* accepted);

void oracle_advect_laplace(int64_t n_edges, const int64_t* off, const double* xy_in,
                           const int32_t* group, int32_t G, int32_t H, int32_t W,
                           const double* rho, double h, double eps, int32_t tries, double beta,
                           double* xy_out, int32_t* accepted) {
    oracle_advect_laplace_mode(n_edges, off, xy_in, group, G, H, W, rho, h, eps, tries, beta, 0,
                               xy_out, accepted);
}

/*
 * As oracle_advect_laplace; with fixed_step != 0 every interior point moves by
 * exactly h along d with no density test: the original KDEEB advection that
 * Sec. 3.3 and Fig. 3 compare the optimised step against.
 */
void oracle_advect_laplace_mode(int64_t n_edges, const int64_t* off, const double* xy_in,
                                const int32_t* group, int32_t G, int32_t H, int32_t W,
                                const double* rho, double h, double eps, int32_t tries,
                                double beta, int32_t fixed_step, double* xy_out,
                                int32_t* accepted) {
    (void)G;
    const int64_t C = (int64_t)H * W;
    std::vector<double> A;
    for (int64_t e = 0; e < n_edges; ++e) {
        int64_t n = off[e + 1] - off[e];
        const double* P = xy_in + 2 * off[e];
        const double* layer = rho + (group ? (int64_t)group[e] : 0) * C;
        A.assign(P, P + 2 * n);
        for (int64_t j = 0; j < n; ++j)
            if (accepted) accepted[off[e] + j] = (j == 0 || j == n - 1) ? -2 : -1;
        for (int64_t j = 1; j + 1 < n; ++j) {
            double x = P[2 * j], y = P[2 * j + 1];
            double gx, gy;
            bilinear_gradient(layer, H, W, x, y, &gx, &gy);
            double den = std::max(std::sqrt(gx * gx + gy * gy), eps);
            double dx = gx / den, dy = gy / den;
            if (fixed_step) {
                A[2 * j] = clamp_pos(x + h * dx, W);
                A[2 * j + 1] = clamp_pos(y + h * dy, H);
                if (accepted) accepted[off[e] + j] = 0;
                continue;
            }
            double r0 = bilinear_density(layer, H, W, x, y);
            for (int32_t t = 0; t < tries; ++t) {
                double m = std::ldexp(h, -t);
                double xn = clamp_pos(x + m * dx, W), yn = clamp_pos(y + m * dy, H);
                if (bilinear_density(layer, H, W, xn, yn) >= r0) {
                    A[2 * j] = xn;
                    A[2 * j + 1] = yn;
                    if (accepted) accepted[off[e] + j] = t;
                    break;
                }
            }
        }
        double* Q = xy_out + 2 * off[e];
        Q[0] = A[0];
        Q[1] = A[1];
        Q[2 * (n - 1)] = A[2 * (n - 1)];
        Q[2 * (n - 1) + 1] = A[2 * (n - 1) + 1];
        for (int64_t j = 1; j + 1 < n; ++j) {
            Q[2 * j] = (1 - beta) * A[2 * j] + beta * (A[2 * (j - 1)] + A[2 * (j + 1)]) / 2;
            Q[2 * j + 1] =
                (1 - beta) * A[2 * j + 1] + beta * (A[2 * (j - 1) + 1] + A[2 * (j + 1) + 1]) / 2;
        }
    }
}

/*
 * The bundling loop (Sec. 3, Fig. 2): n_iters times, resample, build the
 * per-group histogram, smooth, combine layers, advect with h_{iter0 + i} and
 * smooth the polylines. Input and output are polylines in pixel units (CSR
 * offsets plus interleaved xy). The last iteration's histogram, smoothed sums,
 * density and resampled points are copied out when the pointers are non-null.
 * Returns the number of output points, or a negative error:
 * -1 capacity, -2 degenerate polyline, -3 smoothing overflow / radius.
 */
int64_t oracle_run_mode(int64_t n_edges, const int64_t* off_in, const double* xy_in,
                        const int32_t* group, const int32_t* weight, int32_t G, int32_t H,
                        int32_t W, int32_t r, int32_t passes, int32_t alpha_num, int32_t alpha_den,
                        double h_max_sigmas, double lambda, int32_t n_fixed, int32_t n_max,
                        double delta, double beta, double eps, int32_t tries, int32_t iter0,
                        int32_t n_iters, int32_t fixed_step, double directed_offset,
                        const double* M, int32_t segment_hist, int64_t* off_out,
                        double* xy_out, int64_t cap, int64_t* last_hist, int64_t* last_sums,
                        double* last_rho, int64_t* last_res_off, double* last_res_xy,
                        int64_t res_cap);

int64_t oracle_run(int64_t n_edges, const int64_t* off_in, const double* xy_in,
                   const int32_t* group, const int32_t* weight, int32_t G, int32_t H, int32_t W,
                   int32_t r, int32_t passes, int32_t alpha_num, int32_t alpha_den,
                   double h_max_sigmas, double lambda, int32_t n_fixed, int32_t n_max,
                   double delta, double beta, double eps, int32_t tries, int32_t iter0,
                   int32_t n_iters, int64_t* off_out, double* xy_out, int64_t cap,
                   int64_t* last_hist, int64_t* last_sums, double* last_rho,
                   int64_t* last_res_off, double* last_res_xy, int64_t res_cap) {
    return oracle_run_mode(n_edges, off_in, xy_in, group, weight, G, H, W, r, passes, alpha_num,
                           alpha_den, h_max_sigmas, lambda, n_fixed, n_max, delta, beta, eps,
                           tries, iter0, n_iters, 0, 0.0, nullptr, 0, off_out, xy_out, cap,
                           last_hist, last_sums, last_rho, last_res_off, last_res_xy, res_cap);
}

/*
 * The loop with its variants: fixed_step (KDEEB step, Sec. 3.3), directed_offset
 * (pixels, applied after the first sampling of iteration 0, Sec. 3), M (a G x G
 * interaction matrix replacing Eq. 4's; NULL keeps Eq. 4 with alpha) and
 * segment_hist (Bresenham segment histogram instead of the point splat).
 */
int64_t oracle_run_mode(int64_t n_edges, const int64_t* off_in, const double* xy_in,
                   const int32_t* group, const int32_t* weight, int32_t G, int32_t H, int32_t W,
                   int32_t r, int32_t passes, int32_t alpha_num, int32_t alpha_den,
                   double h_max_sigmas, double lambda, int32_t n_fixed, int32_t n_max,
                   double delta, double beta, double eps, int32_t tries, int32_t iter0,
                   int32_t n_iters, int32_t fixed_step, double directed_offset,
                   const double* M, int32_t segment_hist, int64_t* off_out, double* xy_out,
                   int64_t cap,
                   int64_t* last_hist, int64_t* last_sums, double* last_rho,
                   int64_t* last_res_off, double* last_res_xy, int64_t res_cap) {
    const int64_t C = (int64_t)H * W;
    const int64_t pts_cap = n_edges * (int64_t)(n_fixed > 0 ? n_fixed : n_max);
    std::vector<int64_t> P_off(off_in, off_in + n_edges + 1);
    std::vector<double> P_xy(xy_in, xy_in + 2 * off_in[n_edges]);
    std::vector<int64_t> R_off((size_t)n_edges + 1);
    std::vector<double> R_xy((size_t)(2 * pts_cap));
    std::vector<int64_t> hist((size_t)(G * C)), sums((size_t)(G * C));
    std::vector<double> rho((size_t)(G * C));
    for (int32_t it = 0; it < n_iters; ++it) {
        int64_t n = oracle_resample(n_edges, P_off.data(), P_xy.data(), n_fixed, n_max, delta,
                                    R_off.data(), R_xy.data(), pts_cap);
        if (n < 0) return n;
        if (directed_offset != 0 && iter0 + it == 0)
            oracle_directed_offset(n_edges, R_off.data(), R_xy.data(), directed_offset, W, H);
        if (segment_hist)
            oracle_splat_segments(n_edges, R_off.data(), R_xy.data(), group, weight, G, H, W,
                                  hist.data());
        else
            oracle_splat(n_edges, R_off.data(), R_xy.data(), group, weight, G, H, W,
                         hist.data());
        if (oracle_smooth(G, H, W, r, passes, hist.data(), sums.data()) != 0) return -3;
        if (M)
            oracle_combine_matrix(G, H, W, r, passes, M, sums.data(), rho.data());
        else
            oracle_combine(G, H, W, r, passes, alpha_num, alpha_den, sums.data(), rho.data());
        double h = oracle_bandwidth(iter0 + it, r, passes, h_max_sigmas, lambda);
        P_xy.assign((size_t)(2 * n), 0.0);
        oracle_advect_laplace_mode(n_edges, R_off.data(), R_xy.data(), group, G, H, W,
                                   rho.data(), h, eps, tries, beta, fixed_step, P_xy.data(),
                                   nullptr);
        P_off = R_off;
    }
    int64_t n = P_off[(size_t)n_edges];
    if (n > cap) return -1;
    std::copy(P_off.begin(), P_off.end(), off_out);
    std::copy(P_xy.begin(), P_xy.begin() + 2 * n, xy_out);
    if (n_iters > 0) {
        if (last_hist) std::copy(hist.begin(), hist.end(), last_hist);
        if (last_sums) std::copy(sums.begin(), sums.end(), last_sums);
        if (last_rho) std::copy(rho.begin(), rho.end(), last_rho);
        if (last_res_off && last_res_xy) {
            int64_t nr = R_off[(size_t)n_edges];
            if (nr > res_cap) return -1;
            std::copy(R_off.begin(), R_off.end(), last_res_off);
            std::copy(R_xy.begin(), R_xy.begin() + 2 * nr, last_res_xy);
        }
    }
    return n;
}

/*
 * Headless rendering of the bundled drawing (Sec. 3.4): polylines drawn as
 * line segments coloured by bin, edge weight shown by alpha accumulation and by
 * a line width that follows the density at the sample points. The paper draws
 * with OpenGL; this restates what the drawing shows, as a definition:
 *  - image = (W * scale) x (H * scale) pixels; pixel (px, py) has its centre at
 *    (px + 0.5, py + 0.5) in image units, i.e. grid position / scale;
 *  - segment j of edge e (points x_j, x_{j+1}, scaled to image units) has width
 *    w = width_min + (width_max - width_min) u, u = clamp(rho_bar / rho_ref, 0, 1)
 *    (log2(1 + u) with log_width), rho_bar the mean of the bilinear density of
 *    the edge's own layer at x_j and x_{j+1}; rho_ref <= 0 means the maximum of
 *    rho over the stack;
 *  - the segment covers the pixels whose centre lies within w / 2 of it; a pixel
 *    whose nearest point on segment j is its far end (t >= 1) belongs to segment
 *    j + 1 instead (joints are drawn once), except on the last segment;
 *  - alpha accumulation, order-free: every covered pixel gains the optical depth
 *    tau_e = w_e * llround(-ln(1 - alpha) * 2^20) and tau_e times the bin's RGB;
 *    the pixel's opacity is A = 1 - exp(-sum tau / 2^20) (what repeated "over"
 *    with alpha gives) and its colour the tau-weighted mean of the edges' colours;
 *  - final RGB = A * colour + (1 - A) * background, rounded half up to 8 bits,
 *    alpha 255.
 * accum: int64 [Hi][Wi][4] (sum tau, sum tau R, sum tau G, sum tau B); amb: 1
 * where some coverage decision is within 1e-4 of its threshold (a float of lower
 * precision may decide it either way); rgba: uint8 [Hi][Wi][4].
 * Returns 0, or -1 for invalid arguments.
 */
int32_t oracle_render(int64_t n_edges, const int64_t* off, const double* xy, const int32_t* group,
                      const int32_t* weight, int32_t G, int32_t H, int32_t W, const double* rho,
                      int32_t scale, double alpha, double width_min, double width_max,
                      double rho_ref, int32_t log_width, const uint8_t* palette,
                      const uint8_t* background, int64_t* accum, uint8_t* amb, uint8_t* rgba) {
    if (scale < 1 || !(alpha > 0 && alpha < 1) || !(width_min > 0) || width_max < width_min)
        return -1;
    const int64_t Wi = (int64_t)W * scale, Hi = (int64_t)H * scale;
    const int64_t tau1 = std::llround(-std::log1p(-alpha) * 1048576.0);
    if (rho_ref <= 0) {
        rho_ref = 0;
        for (int64_t i = 0; i < (int64_t)G * H * W; ++i) rho_ref = std::max(rho_ref, rho[i]);
    }
    std::fill(accum, accum + Hi * Wi * 4, (int64_t)0);
    std::fill(amb, amb + Hi * Wi, (uint8_t)0);
    for (int64_t e = 0; e < n_edges; ++e) {
        const int g = group ? group[e] : 0;
        const int64_t tau = (weight ? weight[e] : 1) * tau1;
        const double* layer = rho + (int64_t)g * H * W;
        const int64_t n = off[e + 1] - off[e];
        const double* P = xy + 2 * off[e];
        for (int64_t j = 0; j + 1 < n; ++j) {
            const bool last = j + 2 == n;
            double rb = (bilinear_density(layer, H, W, P[2 * j], P[2 * j + 1]) +
                         bilinear_density(layer, H, W, P[2 * j + 2], P[2 * j + 3])) / 2;
            double u = rho_ref > 0 ? std::min(std::max(rb / rho_ref, 0.0), 1.0) : 0.0;
            if (log_width) u = std::log2(1 + u);
            const double r = (width_min + (width_max - width_min) * u) / 2;
            const double ax = P[2 * j] * scale, ay = P[2 * j + 1] * scale;
            const double bx = P[2 * j + 2] * scale, by = P[2 * j + 3] * scale;
            const double dx = bx - ax, dy = by - ay, L2 = dx * dx + dy * dy;
            const int64_t x0 = std::max<int64_t>(0, (int64_t)std::floor(std::min(ax, bx) - r) - 1);
            const int64_t x1 = std::min<int64_t>(Wi - 1, (int64_t)std::ceil(std::max(ax, bx) + r) + 1);
            const int64_t y0 = std::max<int64_t>(0, (int64_t)std::floor(std::min(ay, by) - r) - 1);
            const int64_t y1 = std::min<int64_t>(Hi - 1, (int64_t)std::ceil(std::max(ay, by) + r) + 1);
            for (int64_t py = y0; py <= y1; ++py)
                for (int64_t px = x0; px <= x1; ++px) {
                    const double cx = px + 0.5, cy = py + 0.5;
                    const double t = L2 > 0 ? ((cx - ax) * dx + (cy - ay) * dy) / L2 : 0.0;
                    const double tc = std::min(std::max(t, 0.0), 1.0);
                    const double qx = ax + tc * dx - cx, qy = ay + tc * dy - cy;
                    const double d2 = qx * qx + qy * qy;
                    const bool near_r = std::fabs(d2 - r * r) <= 1e-4 * std::max(r * r, 1.0);
                    const bool near_t = !last && std::fabs(t - 1) <= 1e-4;
                    if ((near_r || near_t) && d2 <= r * r * (1 + 1e-3) + 1e-4)
                        amb[py * Wi + px] = 1;
                    if (d2 > r * r || (!last && t >= 1)) continue;
                    int64_t* a = accum + 4 * (py * Wi + px);
                    a[0] += tau;
                    for (int c = 0; c < 3; ++c) a[1 + c] += tau * palette[3 * g + c];
                }
        }
    }
    for (int64_t i = 0; i < Hi * Wi; ++i) {
        const int64_t* a = accum + 4 * i;
        const double A = 1 - std::exp(-(double)a[0] / 1048576.0);
        for (int c = 0; c < 3; ++c) {
            const double col = a[0] > 0 ? (double)a[1 + c] / (double)a[0] : 0.0;
            const double v = A * col + (1 - A) * background[c];
            rgba[4 * i + c] = (uint8_t)std::min(255.0, std::max(0.0, std::floor(v + 0.5)));
        }
        rgba[4 * i + 3] = 255;
    }
    return 0;
}

}  // extern "C"
