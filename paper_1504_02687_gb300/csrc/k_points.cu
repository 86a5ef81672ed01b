// Point-side kernels of the bundling iteration: advection with the halving
// step and Laplacian smoothing (Eq. 5, Sec. 3.3), resampling (Sec. 2.1,
// Sec. 3) and the per-group histogram splat (Eq. 1, Eq. 3), fused into one
// pass over the block layout of the polylines.
//
// Every floating-point step is written with explicit round-to-nearest
// intrinsics so that the fused and the split launch sequences produce the same
// bits regardless of how the compiler contracts expressions.
#include "density.cuh"

namespace heb {
namespace {

// Direction and starting density of one interior point (Eq. 5): the direction
// is the bilinear interpolation of central differences at the four surrounding
// cell centres on the reflection-extended map, normalised by max(|g|, eps).
struct Dir {
    float dx, dy, rho0;
};

template <typename T, bool TEX>
__device__ __forceinline__ Dir direction(float2 p, const QuadMap<T, TEX>& Q, int W, int H,
                                         float eps) {
    Frame f = frame_of(p.x, p.y, W, H);
    const int64_t Wq = W + kQuadPad;
    const int64_t c = (int64_t)(f.b0 + 2) * Wq + (f.a0 + 2);
    // quads at (a0, b0-1), (a0-1, b0), (a0+1, b0), (a0, b0+1): the 12-cell stencil
    const float4 up = Q.at(c - Wq), lf = Q.at(c - 1);
    const float4 rt = Q.at(c + 1), dn = Q.at(c + Wq);
    // E(a0,b0) = up.z, E(a0+1,b0) = up.w, E(a0,b0+1) = dn.x, E(a0+1,b0+1) = dn.y
    // central differences (E(a+1) - E(a-1)) / 2 at the four cell centres, interpolated;
    // halving commutes exactly with the interpolation (a power-of-two scaling), so it is
    // applied once at the end
    float gx = lerp_rn(lerp_rn(__fsub_rn(rt.x, lf.x), __fsub_rn(rt.y, lf.y), f.fu),
                       lerp_rn(__fsub_rn(rt.z, lf.z), __fsub_rn(rt.w, lf.w), f.fu), f.fv);
    float gy = lerp_rn(lerp_rn(__fsub_rn(dn.x, up.x), __fsub_rn(dn.y, up.y), f.fu),
                       lerp_rn(__fsub_rn(dn.z, up.z), __fsub_rn(dn.w, up.w), f.fu), f.fv);
    gx = __fmul_rn(gx, 0.5f);
    gy = __fmul_rn(gy, 0.5f);
    Dir d;
    d.rho0 = lerp_rn(lerp_rn(up.z, up.w, f.fu), lerp_rn(dn.x, dn.y, f.fu), f.fv);
    // d = g / max(|g|, eps): one reciprocal square root (direction only)
    const float n2 = __fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy));
    const float inv = n2 > eps * eps ? rsqrtf(n2) : __frcp_rn(eps);
    d.dx = __fmul_rn(gx, inv);
    d.dy = __fmul_rn(gy, inv);
    return d;
}

// The position a step of size m along (dx, dy) reaches, clamped to the drawing area.
__device__ __forceinline__ float2 moved(float px, float py, float m, float dx, float dy, int W,
                                        int H) {
    return make_float2(clamp_pos(__fmaf_rn(m, dx, px), W), clamp_pos(__fmaf_rn(m, dy, py), H));
}

// Segment length (the arc length sums these; an approximate square root is enough).
__device__ __forceinline__ float seg_len(float2 a, float2 b) {
    float dx = __fsub_rn(b.x, a.x), dy = __fsub_rn(b.y, a.y);
    float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    return d2 > 0.0f ? __fmul_rn(d2, rsqrtf(d2)) : 0.0f;
}

// Point count after resampling (Sec. 2.1: spacing delta; fixed count if set).
__device__ __forceinline__ int new_count(float L, const StepArgs& a) {
    if (a.n_fixed > 0) return a.n_fixed;
    float q = __fdiv_rn(L, a.delta);
    if (!(q < (float)a.n_max)) return a.n_max;  // also catches NaN
    int n = (int)ceilf(q) + 1;
    return n < 2 ? 2 : (n > a.n_max ? a.n_max : n);
}

// Inclusive warp scan of floats (Hillis-Steele order; the same order everywhere).
__device__ __forceinline__ float warp_scan_incl(float x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = __fadd_rn(x, y);
    }
    return x;
}

constexpr unsigned kFull = 0xffffffffu;

// Segment histogram (Eq. 1 as rasterised in Sec. 4): the cells from the cell of A to
// the cell of B by the integer Bresenham line algorithm, each gaining w (the first
// one skipped for segments after the first: it closed the previous segment).
// Returns the number of cells counted.
__device__ __forceinline__ int raster_segment(uint32_t* hl, int W, int H, float2 A, float2 B,
                                              bool skip_first, unsigned w) {
    int x = min(max((int)floorf(A.x), 0), W - 1), y = min(max((int)floorf(A.y), 0), H - 1);
    const int x1 = min(max((int)floorf(B.x), 0), W - 1), y1 = min(max((int)floorf(B.y), 0), H - 1);
    const int dx = abs(x1 - x), dy = -abs(y1 - y);
    const int sx = x < x1 ? 1 : -1, sy = y < y1 ? 1 : -1;
    int err = dx + dy, count = 0;
    bool first = true;
    for (;;) {
        if (!(first && skip_first)) {
            atomicAdd(hl + (size_t)y * W + x, w);
            ++count;
        }
        first = false;
        if (x == x1 && y == y1) break;
        const int e2 = 2 * err;
        if (e2 >= dy) {
            err += dy;
            x += sx;
        }
        if (e2 <= dx) {
            err += dx;
            y += sy;
        }
    }
    return count;
}

// Write one resampled point and splat it: it adds its edge weight to its group's cell
// (Eq. 1, Eq. 3) in one of the histogram copies.
__device__ __forceinline__ void emit(const StepArgs& a, uint32_t* hl, float2* dst, float2 R,
                                     int w) {
    *dst = R;
    if (w != 0 && !a.seg_hist) {
        const int cx = min(max(__float2int_rd(R.x), 0), a.W - 1);
        const int cy = min(max(__float2int_rd(R.y), 0), a.H - 1);
        atomicAdd(hl + (size_t)cy * a.W + cx, (unsigned)w);
    }
}

// Shared staging of one warp: a sub-batch of whole polylines of its block, and the
// per-slot values the warp reads uniformly (one vector load instead of a shuffle each).
struct StepSmem {
    float2 pts[kStage];               // the sub-batch's points
    float cum[kStage];                // arc lengths
    int4 meta[kMaxEdgesPerWarp];      // per slot: first point in the region, count, group, weight
    int4 outm[kMaxEdgesPerWarp];      // per slot of the sub-batch: new count, its first output,
                                      // spacing (float bits)
    unsigned char pe[kStage];         // slot (within the block) of each staged point
};

// Advection of the staged interior points (Eq. 5, Sec. 3.3), one thread per point:
// the direction, then step trials of size h, h/2, ... until the density at the
// moved position is not lower than at the point (none accepted: the point stays).
template <typename T, bool TEX>
__device__ __forceinline__ void advect_staged(const StepArgs& a, StepSmem& S, int np, int p0,
                                              const T* quads, int64_t QC4, float h) {
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < np; c += 32) {
        const int k = c + lane;
        const int4 md = S.meta[k < np ? S.pe[k] : 0];
        const int q = md.x - p0, n = md.y, g = md.z;
        const int j = k - q;
        if (k < np && j > 0 && j < n - 1) {
            const QuadMap<T, TEX> Q{quads + (int64_t)g * QC4, a.qtex, (int64_t)g * (QC4 / 4)};
            const float2 p = S.pts[k];
            const Dir d = direction(p, Q, a.W, a.H, a.eps);
            if (a.fixed_step) {  // KDEEB's step (Sec. 3.3): h whatever the density there
                S.pts[k] = moved(p.x, p.y, h, d.dx, d.dy, a.W, a.H);
                continue;
            }
            float m = h;
            for (int t = 0; t < a.tries; ++t) {
                const float2 x1 = moved(p.x, p.y, m, d.dx, d.dy, a.W, a.H);
                if (density_at(Q, a.W, a.H, x1.x, x1.y) >= d.rho0) {
                    S.pts[k] = x1;
                    break;
                }
                m = __fmul_rn(m, 0.5f);
            }
        }
    }
    __syncwarp();
}

// The work of one warp on its block of eb slots (blk: the block's index in the
// layout). The warp stages sub-batches of whole polylines in its own shared
// memory and works through them alone, with warp-level synchronisation only:
//  1. load the sub-batch's points (coalesced) and tag each with its slot;
//  2. advection, one thread per point, in place (a point reads only itself);
//  3. per polyline, two consecutive points per lane: Laplacian smoothing
//     (Jacobi), then the arc lengths by a warp scan;
//  4. new point counts and spacings (one lane per polyline) and their offsets
//     (a warp scan); then per polyline the uniformly re-spaced points, two per
//     lane, written out and splatted.
template <int MODE, typename T>
__device__ __forceinline__ void step_warp(const StepArgs& a, int64_t blk, StepSmem& S) {
    const int lane = threadIdx.x & 31;
    const int64_t e0 = blk * a.eb;
    if (e0 >= a.E) return;
    const int nb = (int)min((int64_t)a.eb, a.E - e0);
    const int64_t region = blk * a.eb * (int64_t)a.cap;
    const float2* __restrict__ pin = a.pts_in + region;
    float2* __restrict__ pout = a.pts_out + region;
    const int64_t QC4 = quad_elems(a.W, a.H) * 4;
    const T* quads = static_cast<const T*>(a.quads);
    uint32_t* hist = a.hist + (size_t)(blk % kHistCopies) * a.G * (size_t)a.W * a.H;
    const float h = a.h_sched ? __ldg(a.h_sched + __ldg(a.iter)) : a.h;

    // lane i holds slot e0 + i: its point count, group, weight and, after the scan, the
    // offset of its first point in the block's region
    int cnt = 0, grp = 0, wgt = 0;
    if (lane < nb) {
        cnt = a.cnt_in[e0 + lane];
        grp = a.group[e0 + lane];
        wgt = a.weight[e0 + lane];
    }
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    const int loc = inc - cnt;
    if (lane < nb) S.meta[lane] = make_int4(loc, cnt, grp, wgt);
    __syncwarp();

    int out_base = 0;
    for (int b0 = 0; b0 < nb;) {
        // polylines [b0, b1): the longest run from b0 that fits the staging buffer
        const int p0 = __shfl_sync(kFull, loc, b0);
        const int b1 =
            b0 + __popc(__ballot_sync(kFull, lane >= b0 && lane < nb && inc - p0 <= kStage));
        const int np = __shfl_sync(kFull, inc, b1 - 1) - p0;
        for (int k = lane; k < np; k += 32) S.pts[k] = pin[p0 + k];
        if (MODE & kModeAdvect) {
            for (int i = b0; i < b1; ++i) {
                const int4 md = S.meta[i];
                for (int j = lane; j < md.y; j += 32) S.pe[md.x - p0 + j] = (unsigned char)i;
            }
        }
        __syncwarp();

        if (MODE & kModeAdvect)
            advect_staged<T, (MODE & kModeTexGather) != 0>(a, S, np, p0, quads, QC4, h);

        // one polyline at a time, two consecutive points per lane (j = 2 lane, 2 lane + 1;
        // a polyline has at most 64 points): Laplacian smoothing, then the arc lengths. The
        // neighbours across lanes come by shuffles, so a lane writes only its own points.
        for (int i = b0; i < b1; ++i) {
            const int4 md = S.meta[i];
            const int q = md.x - p0, n = md.y;
            if (n == 2) {
                // end points only (a quarter of a bundled layout's edges are this short):
                // nothing to smooth, one segment; the same values as the general path
                if (MODE & kModeResample) {
                    if (lane == 0) {
                        S.cum[q] = 0.0f;
                        S.cum[q + 1] = seg_len(S.pts[q], S.pts[q + 1]);
                    }
                } else {
                    if (lane < 2) pout[p0 + q + lane] = S.pts[q + lane];
                    if (lane == 0) a.cnt_out[e0 + i] = n;
                }
                continue;
            }
            const int j0 = 2 * lane, j1 = j0 + 1;
            float2 A0 = j0 < n ? S.pts[q + j0] : make_float2(0.0f, 0.0f);
            float2 A1 = j1 < n ? S.pts[q + j1] : make_float2(0.0f, 0.0f);
            if (MODE & kModeAdvect) {
                // point j0 - 1 is the previous lane's second, j1 + 1 the next lane's first
                const float lx = __shfl_up_sync(kFull, A1.x, 1);
                const float ly = __shfl_up_sync(kFull, A1.y, 1);
                const float rx = __shfl_down_sync(kFull, A0.x, 1);
                const float ry = __shfl_down_sync(kFull, A0.y, 1);
                float2 B0 = A0, B1 = A1;
                if (j0 > 0 && j0 < n - 1) {
                    B0.x = __fmaf_rn(a.lap_half_beta, __fadd_rn(lx, A1.x), __fmul_rn(a.lap_keep, A0.x));
                    B0.y = __fmaf_rn(a.lap_half_beta, __fadd_rn(ly, A1.y), __fmul_rn(a.lap_keep, A0.y));
                }
                if (j1 < n - 1) {
                    B1.x = __fmaf_rn(a.lap_half_beta, __fadd_rn(A0.x, rx), __fmul_rn(a.lap_keep, A1.x));
                    B1.y = __fmaf_rn(a.lap_half_beta, __fadd_rn(A0.y, ry), __fmul_rn(a.lap_keep, A1.y));
                }
                A0 = B0;
                A1 = B1;
                if (MODE & kModeResample) {
                    if (j0 < n) S.pts[q + j0] = A0;
                    if (j1 < n) S.pts[q + j1] = A1;
                } else {
                    if (j0 < n) pout[p0 + q + j0] = A0;
                    if (j1 < n) pout[p0 + q + j1] = A1;
                    if (lane == 0) a.cnt_out[e0 + i] = n;
                }
            }
            if (MODE & kModeResample) {
                // cum[j]: lengths of the segments up to point j, by a warp scan of the lanes'
                // pair sums
                const float px = __shfl_up_sync(kFull, A1.x, 1);
                const float py = __shfl_up_sync(kFull, A1.y, 1);
                const float s0 = (j0 >= 1 && j0 < n) ? seg_len(make_float2(px, py), A0) : 0.0f;
                const float s1 = j1 < n ? seg_len(A0, A1) : 0.0f;
                const float incl = warp_scan_incl(__fadd_rn(s0, s1), lane);
                float ex = __shfl_up_sync(kFull, incl, 1);
                if (lane == 0) ex = 0.0f;
                const float c0 = __fadd_rn(ex, s0);
                if (j0 < n) S.cum[q + j0] = c0;
                if (j1 < n) S.cum[q + j1] = __fadd_rn(c0, s1);
            }
        }
        __syncwarp();

        if (MODE & kModeResample) {
            // new point count and spacing of polyline `lane`, and its first output offset
            int mc = 0;
            float sp = 0.0f;
            if (lane >= b0 && lane < b1) {
                const float L = S.cum[loc - p0 + cnt - 1];
                mc = new_count(L, a);
                sp = __fdiv_rn(L, (float)(mc - 1));
            }
            int minc = mc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, minc, o);
                if (lane >= o) minc += y;
            }
            if (lane >= b0 && lane < b1)
                S.outm[lane] = make_int4(mc, out_base + minc - mc, __float_as_int(sp), 0);
            __syncwarp();
            for (int i = b0; i < b1; ++i) {
                const int4 md = S.meta[i], mo = S.outm[i];
                const int q = md.x - p0, n = md.y, g = md.z, w = md.w;
                const int m = mo.x, ob = mo.y;
                if (m == 2 && !a.seg_hist) {
                    // the two end points, copied and splatted (one lane each)
                    if (lane < 2)
                        emit(a, hist + (size_t)g * a.W * a.H, pout + ob + lane,
                             S.pts[q + (lane == 0 ? 0 : n - 1)], w);
                    if (lane == 0) a.cnt_out[e0 + i] = m;
                    continue;
                }
                const float spi = __int_as_float(mo.z);
                const float L = S.cum[q + n - 1];
                uint32_t* hl = hist + (size_t)g * a.W * a.H;
                // directed graphs (Sec. 3): interior points shift along the edge normal
                float ox = 0.0f, oy = 0.0f;
                if (a.dir_amount != 0.0f) {
                    const float2 P0 = S.pts[q], P1 = S.pts[q + n - 1];
                    const float ddx = __fsub_rn(P1.x, P0.x), ddy = __fsub_rn(P1.y, P0.y);
                    const float len = sqrtf(__fadd_rn(__fmul_rn(ddx, ddx), __fmul_rn(ddy, ddy)));
                    if (len > 0.0f) {
                        ox = -a.dir_amount * ddy / len;
                        oy = a.dir_amount * ddx / len;
                    }
                }
                // two consecutive outputs per lane, j = 2 lane and 2 lane + 1 (m <= 64).
                // Endpoints are copied; an edge of zero length puts every point on its
                // source. Interior output j sits at arc length t_j = j * L / (m - 1) on
                // segment s, the first with cum[s] > t_j: six halvings find it for the first
                // output, and the second steps on from there.
                int lo = 1;
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int j = 2 * lane + h2;
                    if (j >= m) break;
                    float2 R;
                    if (j == m - 1) {
                        R = S.pts[q + n - 1];
                    } else if (j == 0 || L == 0.0f) {
                        R = S.pts[q];
                    } else {
                        const float t = __fmul_rn((float)j, spi);
                        if (h2 == 0) {
                            int pos = 0;  // the last k in [0, n-2] with cum[k] <= t
#pragma unroll
                            for (int step = 32; step > 0; step >>= 1) {
                                const int c = pos + step;
                                if (c <= n - 2 && !(S.cum[q + c] > t)) pos = c;
                            }
                            lo = pos + 1;
                        } else {
                            while (lo < n - 1 && !(S.cum[q + lo] > t)) ++lo;
                        }
                        const float c0 = S.cum[q + lo - 1];
                        const float seg = __fsub_rn(S.cum[q + lo], c0);
                        float fr = seg > 0.0f ? __fdividef(__fsub_rn(t, c0), seg) : 0.0f;
                        fr = fminf(fmaxf(fr, 0.0f), 1.0f);
                        const float2 A = S.pts[q + lo - 1], B = S.pts[q + lo];
                        R = make_float2(lerp_rn(A.x, B.x, fr), lerp_rn(A.y, B.y, fr));
                        if (ox != 0.0f || oy != 0.0f)
                            R = make_float2(clamp_pos(__fadd_rn(R.x, ox), a.W),
                                            clamp_pos(__fadd_rn(R.y, oy), a.H));
                    }
                    emit(a, hl, pout + ob + j, R, w);
                }
                if (a.seg_hist && w != 0) {
                    // segments of the new polyline (its points were written by this warp)
                    __syncwarp();
                    unsigned long long cells = 0;
                    for (int j = 1 + lane; j < m; j += 32)
                        cells += raster_segment(hl, a.W, a.H, pout[ob + j - 1], pout[ob + j],
                                                j >= 2, (unsigned)w);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) cells += __shfl_xor_sync(kFull, cells, o);
                    if (lane == 0 && a.mass) atomicAdd(a.mass, cells * (unsigned long long)w);
                }
                if (lane == 0) a.cnt_out[e0 + i] = m;
            }
            out_base += __shfl_sync(kFull, minc, 31);
        }
        __syncwarp();  // the next sub-batch overwrites the staging
        b0 = b1;
    }
    if ((MODE & kModeResample) && lane == 0 && a.n_splat)
        atomicAdd(a.n_splat, (unsigned long long)out_base);
}

// CTAs per SM the step kernels are compiled for, a register budget of 65536 / (128 x n):
// 10 (48 registers) where the gathers take the texture path, 9 (56) elsewhere -- the
// load-path and resample-only forms spill at 48 (measured fastest of 8 to 11).
template <int MODE>
constexpr int step_min_ctas() { return (MODE & kModeTexGather) ? 10 : 9; }

template <int MODE, typename T>
__global__ void __launch_bounds__(kStepThreads, step_min_ctas<MODE>()) k_step(const __grid_constant__ StepArgs a) {
    __shared__ StepSmem smem[kStepWarps];
    const int warp = threadIdx.x >> 5;
    step_warp<MODE, T>(a, (int64_t)blockIdx.x * kStepWarps + warp, smem[warp]);
}

// Many graphs in one launch: CTA blockIdx.x belongs to graph m with
// blk[m] <= blockIdx.x < blk[m + 1] and is that graph's CTA blockIdx.x - blk[m].
template <int MODE, typename T>
__global__ void __launch_bounds__(kStepThreads, step_min_ctas<MODE>()) k_step_batch(const __grid_constant__ BatchStepArgs P) {
    __shared__ StepSmem smem[kStepWarps];
    int lo = 0, hi = P.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.blk[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const int warp = threadIdx.x >> 5;
    step_warp<MODE, T>(P.a[lo], (int64_t)((int)blockIdx.x - P.blk[lo]) * kStepWarps + warp,
                       smem[warp]);
}

__global__ void k_advance_batch(const __grid_constant__ BatchStepArgs P) {
    const int m = threadIdx.x;
    if (m < P.n) *const_cast<int32_t*>(P.a[m].iter) += 1;
}

template <typename T>
cudaError_t launch_step_batch_t(int mode, const BatchStepArgs& P, cudaStream_t st) {
    const int total = P.blk[P.n];
    if (total <= 0) return cudaSuccess;
    for (int m = 0; m < P.n; ++m)
        if (P.a[m].eb < 1 || P.a[m].eb > kMaxEdgesPerWarp) return cudaErrorInvalidValue;
    // gathers through the texture views when every graph has one
    bool tex = true;
    for (int m = 0; m < P.n; ++m) tex = tex && P.a[m].qtex != 0;
    switch (mode | ((mode & kModeAdvect) && tex ? kModeTexGather : 0)) {
        case kModeResample: k_step_batch<kModeResample, T><<<total, kStepThreads, 0, st>>>(P); break;
        case kModeAdvect: k_step_batch<kModeAdvect, T><<<total, kStepThreads, 0, st>>>(P); break;
        case kModeAdvectResample:
            k_step_batch<kModeAdvectResample, T><<<total, kStepThreads, 0, st>>>(P);
            break;
        case kModeAdvect | kModeTexGather:
            k_step_batch<kModeAdvect | kModeTexGather, T><<<total, kStepThreads, 0, st>>>(P);
            break;
        case kModeAdvectResample | kModeTexGather:
            k_step_batch<kModeAdvectResample | kModeTexGather, T><<<total, kStepThreads, 0, st>>>(P);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step_t(int mode, const StepArgs& a, cudaStream_t st) {
    if (a.E <= 0) return cudaSuccess;
    if (a.eb < 1 || a.eb > kMaxEdgesPerWarp) return cudaErrorInvalidValue;
    dim3 grid((unsigned)step_ctas(a.E, a.eb));
    switch (mode | ((mode & kModeAdvect) && a.qtex ? kModeTexGather : 0)) {
        case kModeResample: k_step<kModeResample, T><<<grid, kStepThreads, 0, st>>>(a); break;
        case kModeAdvect: k_step<kModeAdvect, T><<<grid, kStepThreads, 0, st>>>(a); break;
        case kModeAdvectResample:
            k_step<kModeAdvectResample, T><<<grid, kStepThreads, 0, st>>>(a);
            break;
        case kModeAdvect | kModeTexGather:
            k_step<kModeAdvect | kModeTexGather, T><<<grid, kStepThreads, 0, st>>>(a);
            break;
        case kModeAdvectResample | kModeTexGather:
            k_step<kModeAdvectResample | kModeTexGather, T><<<grid, kStepThreads, 0, st>>>(a);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- init / fetch helpers

// Spatial key of an edge: group, then the Morton index of its midpoint's cell
// on a 64 x 64 tiling of the grid. Sorting by it gives each block of slots
// nearby edges of one group (locality for the density gathers and the splat).
__global__ void k_edge_keys(const float2* __restrict__ src, const float2* __restrict__ dst,
                            const int32_t* __restrict__ group, int64_t E, int32_t W, int32_t H,
                            uint32_t* key, uint32_t* bucket_cnt) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    float mx = 0.5f * (src[e].x + dst[e].x), my = 0.5f * (src[e].y + dst[e].y);
    uint32_t tx = (uint32_t)min(max((int)(mx * 64.0f / (float)W), 0), 63);
    uint32_t ty = (uint32_t)min(max((int)(my * 64.0f / (float)H), 0), 63);
    uint32_t m = 0;
    for (int b = 0; b < 6; ++b) m |= (((tx >> b) & 1u) << (2 * b)) | (((ty >> b) & 1u) << (2 * b + 1));
    uint32_t k = (uint32_t)group[e] * 4096u + m;
    key[e] = k;
    atomicAdd(bucket_cnt + k, 1u);
}

// In-place exclusive scan of n bucket counts by one block of 1024 threads.
__global__ void k_bucket_scan(uint32_t* cnt, int32_t n) {
    __shared__ uint32_t s_part[1024];
    const int tid = threadIdx.x;
    const int per = (n + 1023) / 1024;
    const int lo = min(n, tid * per), hi = min(n, lo + per);
    uint32_t s = 0;
    for (int i = lo; i < hi; ++i) s += cnt[i];
    s_part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        uint32_t run = 0;
        for (int t = 0; t < 1024; ++t) {
            uint32_t v = s_part[t];
            s_part[t] = run;
            run += v;
        }
    }
    __syncthreads();
    uint32_t run = s_part[tid];
    for (int i = lo; i < hi; ++i) {
        uint32_t v = cnt[i];
        cnt[i] = run;
        run += v;
    }
}

__global__ void k_edge_scatter(const uint32_t* __restrict__ key, int64_t E, uint32_t* cursor,
                               int32_t* perm) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    uint32_t slot = atomicAdd(cursor + key[e], 1u);
    perm[slot] = (int32_t)e;
}

__global__ void k_gather_edges(const int32_t* __restrict__ perm, int64_t E,
                               const int32_t* __restrict__ group_in,
                               const int32_t* __restrict__ weight_in, int32_t* group_out,
                               int32_t* weight_out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= E) return;
    int32_t e = perm[s];
    group_out[s] = group_in ? group_in[e] : 0;
    weight_out[s] = weight_in ? weight_in[e] : 1;
}

// Straight edges (2 points each) into the block layout.
__global__ void k_straight_layout(const int32_t* __restrict__ perm, int64_t E,
                                  const float2* __restrict__ src, const float2* __restrict__ dst,
                                  int32_t eb, int32_t cap, int32_t* cnt, float2* pts) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= E) return;
    int32_t e = perm[s];
    int64_t b = s / eb, i = s % eb;
    float2* q = pts + b * eb * (int64_t)cap + 2 * i;
    q[0] = src[e];
    q[1] = dst[e];
    cnt[s] = 2;
}

// Caller CSR polylines into the block layout: one block of slots per CTA.
__global__ void k_polyline_layout(const int32_t* __restrict__ perm, int64_t E,
                                  const int64_t* __restrict__ off, const float2* __restrict__ xy,
                                  int32_t eb, int32_t cap, int32_t* cnt, float2* pts) {
    __shared__ int s_n[kEdgesPerBlock];
    __shared__ int s_o[kEdgesPerBlock + 1];
    __shared__ int s_wtot[32];
    const int64_t s0 = (int64_t)blockIdx.x * eb;
    const int nb = (int)min((int64_t)eb, E - s0);
    const int tid = threadIdx.x;
    if (tid < nb) {
        int32_t e = perm[s0 + tid];
        s_n[tid] = (int)(off[e + 1] - off[e]);
    }
    __syncthreads();
    block_scan_excl(s_n, s_o, nb, s_wtot);
    if (tid < nb) {
        int32_t e = perm[s0 + tid];
        float2* q = pts + (int64_t)blockIdx.x * eb * cap + s_o[tid];
        for (int j = 0; j < s_n[tid]; ++j) q[j] = xy[off[e] + j];
        cnt[s0 + tid] = s_n[tid];
    }
}

__global__ void k_counts_to_caller(const int32_t* __restrict__ perm,
                                   const int32_t* __restrict__ cnt, int64_t E, int64_t* off) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < E) off[perm[s]] = cnt[s];
    if (s == 0) off[E] = 0;
}

// Three-phase exclusive scan of off[0..E] (int64) in place: block sums, scan of
// the block sums by one block, then per-block scans.
constexpr int kScanBlock = 1024;

__device__ long long block_scan_ll(long long v, long long* tmp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long t = lane < (int)(blockDim.x >> 5) ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        tmp[lane] = t;
    }
    __syncthreads();
    long long r = (wid > 0 ? tmp[wid - 1] : 0) + x;  // inclusive
    __syncthreads();
    return r;
}

__global__ void k_scan_sums(const int64_t* __restrict__ v, int64_t n, int64_t* sums) {
    __shared__ long long tmp[32];
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    long long x = i < n ? v[i] : 0;
    long long inc = block_scan_ll(x, tmp);
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = inc;
}

__global__ void k_scan_partials(int64_t* sums, int64_t nblk) {
    __shared__ long long tmp[32];
    long long carry = 0;
    for (int64_t base = 0; base < nblk; base += kScanBlock) {
        int64_t i = base + threadIdx.x;
        long long x = i < nblk ? sums[i] : 0;
        long long inc = block_scan_ll(x, tmp);
        if (i < nblk) sums[i] = carry + inc - x;
        __shared__ long long s_last;
        if (threadIdx.x == kScanBlock - 1) s_last = inc;
        __syncthreads();
        carry += s_last;
        __syncthreads();
    }
}

__global__ void k_scan_apply(int64_t* v, int64_t n, const int64_t* sums) {
    __shared__ long long tmp[32];
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    long long x = i < n ? v[i] : 0;
    long long inc = block_scan_ll(x, tmp);
    if (i < n) v[i] = sums[blockIdx.x] + inc - x;
}

__global__ void k_layout_to_caller(const int32_t* __restrict__ perm,
                                   const int32_t* __restrict__ cnt,
                                   const float2* __restrict__ pts, int64_t E, int32_t eb,
                                   int32_t cap,
                                   const int64_t* __restrict__ off, float2* xy, int32_t to_world,
                                   float ox, float oy, float inv_scale, float xmin, float ymin) {
    __shared__ int s_n[kEdgesPerBlock];
    __shared__ int s_o[kEdgesPerBlock + 1];
    __shared__ int s_wtot[32];
    const int64_t s0 = (int64_t)blockIdx.x * eb;
    const int nb = (int)min((int64_t)eb, E - s0);
    const int tid = threadIdx.x;
    if (tid < nb) s_n[tid] = cnt[s0 + tid];
    __syncthreads();
    block_scan_excl(s_n, s_o, nb, s_wtot);
    if (tid < nb) {
        int32_t e = perm[s0 + tid];
        const float2* q = pts + (int64_t)blockIdx.x * eb * cap + s_o[tid];
        float2* d = xy + off[e];
        for (int j = 0; j < s_n[tid]; ++j) {
            float2 p = q[j];
            if (to_world) {
                // presentation transform back to world units (not part of the method)
                p.x = (p.x - ox) * inv_scale + xmin;
                p.y = (p.y - oy) * inv_scale + ymin;
            }
            d[j] = p;
        }
    }
}

__global__ void k_sum_counts(const int32_t* __restrict__ cnt, int64_t E,
                             unsigned long long* total) {
    unsigned long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E;
         i += (int64_t)gridDim.x * blockDim.x)
        s += (unsigned)cnt[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(total, s);
}

__global__ void k_set_iter(int32_t* iter, int32_t value) { *iter = value; }
__global__ void k_relayout_pairs(const float2* __restrict__ src, int32_t eb_src, int32_t cap_src,
                                 float2* __restrict__ dst, int32_t eb_dst, int32_t cap_dst,
                                 int32_t* cnt_dst, int64_t E) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= E) return;
    const int64_t i = (s / eb_src) * eb_src * cap_src + 2 * (s % eb_src);
    const int64_t o = (s / eb_dst) * eb_dst * cap_dst + 2 * (s % eb_dst);
    dst[o] = src[i];
    dst[o + 1] = src[i + 1];
    if (cnt_dst) cnt_dst[s] = 2;
}
__global__ void k_check_mass(const unsigned long long* mass, unsigned long long allowed,
                             int32_t* flag) {
    if (*mass > allowed) *flag = 1;
}
__global__ void k_advance_iter(int32_t* iter) { *iter += 1; }

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_step_batch(int mode, int rho_dtype, const BatchStepArgs& P, cudaStream_t st) {
    if (P.n < 1 || P.n > kBatchLaunch) return cudaErrorInvalidValue;
    switch (rho_dtype) {
        case 0: return launch_step_batch_t<float>(mode, P, st);
        case 1: return launch_step_batch_t<__nv_bfloat16>(mode, P, st);
        case 2: return launch_step_batch_t<__half>(mode, P, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_advance_batch(const BatchStepArgs& P, cudaStream_t st) {
    k_advance_batch<<<1, kBatchLaunch, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_step(int mode, int rho_dtype, const StepArgs& a, cudaStream_t st) {
    switch (rho_dtype) {
        case 0: return launch_step_t<float>(mode, a, st);
        case 1: return launch_step_t<__nv_bfloat16>(mode, a, st);
        case 2: return launch_step_t<__half>(mode, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_edge_keys(const float2* src, const float2* dst, const int32_t* group,
                             int64_t E, int32_t W, int32_t H, uint32_t* key, uint32_t* bucket_cnt,
                             cudaStream_t st) {
    k_edge_keys<<<blocks_for(E, 256), 256, 0, st>>>(src, dst, group, E, W, H, key, bucket_cnt);
    return cudaGetLastError();
}

cudaError_t launch_bucket_scan(uint32_t* cnt, int32_t n_buckets, cudaStream_t st) {
    k_bucket_scan<<<1, 1024, 0, st>>>(cnt, n_buckets);
    return cudaGetLastError();
}

cudaError_t launch_edge_scatter(const uint32_t* key, int64_t E, uint32_t* cursor, int32_t* perm,
                                cudaStream_t st) {
    k_edge_scatter<<<blocks_for(E, 256), 256, 0, st>>>(key, E, cursor, perm);
    return cudaGetLastError();
}

cudaError_t launch_gather_edges(const int32_t* perm, int64_t E, const int32_t* group_in,
                                const int32_t* weight_in, int32_t* group_out,
                                int32_t* weight_out, cudaStream_t st) {
    k_gather_edges<<<blocks_for(E, 256), 256, 0, st>>>(perm, E, group_in, weight_in, group_out,
                                                       weight_out);
    return cudaGetLastError();
}

cudaError_t launch_straight_layout(const int32_t* perm, int64_t E, const float2* src,
                                   const float2* dst, int32_t eb, int32_t cap, int32_t* cnt,
                                   float2* pts, cudaStream_t st) {
    k_straight_layout<<<blocks_for(E, 256), 256, 0, st>>>(perm, E, src, dst, eb, cap, cnt, pts);
    return cudaGetLastError();
}

cudaError_t launch_polyline_layout(const int32_t* perm, int64_t E, const int64_t* off,
                                   const float2* xy, int32_t eb, int32_t cap, int32_t* cnt,
                                   float2* pts, cudaStream_t st) {
    k_polyline_layout<<<blocks_for(E, eb), kEdgesPerBlock, 0, st>>>(perm, E, off, xy, eb, cap,
                                                                  cnt, pts);
    return cudaGetLastError();
}

cudaError_t launch_counts_to_caller(const int32_t* perm, const int32_t* cnt, int64_t E,
                                    int64_t* off_out, cudaStream_t st) {
    k_counts_to_caller<<<blocks_for(E, 256), 256, 0, st>>>(perm, cnt, E, off_out);
    return cudaGetLastError();
}

size_t scan_offsets_tmp_elems(int64_t E) { return (size_t)((E + 1 + kScanBlock - 1) / kScanBlock); }

cudaError_t launch_scan_offsets(int64_t* off, int64_t E, int64_t* tmp, cudaStream_t st) {
    int64_t n = E + 1;
    int64_t nblk = (n + kScanBlock - 1) / kScanBlock;
    k_scan_sums<<<(unsigned)nblk, kScanBlock, 0, st>>>(off, n, tmp);
    k_scan_partials<<<1, kScanBlock, 0, st>>>(tmp, nblk);
    k_scan_apply<<<(unsigned)nblk, kScanBlock, 0, st>>>(off, n, tmp);
    return cudaGetLastError();
}

cudaError_t launch_layout_to_caller(const int32_t* perm, const int32_t* cnt, const float2* pts,
                                    int64_t E, int32_t eb, int32_t cap, const int64_t* off,
                                    float2* xy_out, int32_t to_world, float ox, float oy,
                                    float inv_scale, float xmin, float ymin, cudaStream_t st) {
    k_layout_to_caller<<<blocks_for(E, eb), kEdgesPerBlock, 0, st>>>(
        perm, cnt, pts, E, eb, cap, off, xy_out, to_world, ox, oy, inv_scale, xmin, ymin);
    return cudaGetLastError();
}

cudaError_t launch_set_iter(int32_t* iter, int32_t value, cudaStream_t st) {
    k_set_iter<<<1, 1, 0, st>>>(iter, value);
    return cudaGetLastError();
}

cudaError_t launch_relayout_pairs(const float2* src, int32_t eb_src, int32_t cap_src, float2* dst,
                                  int32_t eb_dst, int32_t cap_dst, int32_t* cnt_dst, int64_t E,
                                  cudaStream_t st) {
    if (E <= 0) return cudaSuccess;
    k_relayout_pairs<<<(unsigned)((E + 255) / 256), 256, 0, st>>>(src, eb_src, cap_src, dst, eb_dst,
                                                                  cap_dst, cnt_dst, E);
    return cudaGetLastError();
}

cudaError_t launch_check_mass(const unsigned long long* mass, unsigned long long allowed,
                              int32_t* flag, cudaStream_t st) {
    k_check_mass<<<1, 1, 0, st>>>(mass, allowed, flag);
    return cudaGetLastError();
}

cudaError_t launch_advance_iter(int32_t* iter, cudaStream_t st) {
    k_advance_iter<<<1, 1, 0, st>>>(iter);
    return cudaGetLastError();
}

cudaError_t launch_sum_counts(const int32_t* cnt, int64_t E, unsigned long long* total,
                              cudaStream_t st) {
    unsigned nblk = blocks_for(E, 256);
    k_sum_counts<<<nblk < 1024u ? nblk : 1024u, 256, 0, st>>>(cnt, E, total);
    return cudaGetLastError();
}

}  // namespace heb
