/*
 * bundle.h - C ABI of the GB300 (sm_103a) 3DHEB edge-bundling library.
 *
 * The library runs the per-iteration loop of "3D Density Histograms for
 * Criteria-driven Edge Bundling" (Moura), Sec. 3 / Fig. 2, on one GPU:
 *   resample every polyline (Sec. 2.1, Sec. 3) ->
 *   per-group integer histogram of the sample points (Eq. 1, Eq. 3) ->
 *   repeated box filters per layer, integer and exact (Sec. 3.1) ->
 *   layer interaction M (Eq. 3, Eq. 4) -> density rho ->
 *   advection along the bilinear density gradient with the halving step
 *   (Eq. 5, Sec. 3.3) -> Laplacian smoothing of the polylines (Sec. 3.3).
 *
 * Units. After bundle_init every position lives in grid pixel units: cell
 * (u, v) covers [u, u+1) x [v, v+1), x is the column, y the row. World
 * coordinates are mapped once at init (Sec. 5: a fixed dominant grid size, the
 * other from the bounding box's aspect ratio) and mapped back by bundle_fetch.
 *
 * Conventions for every call:
 *  - Every call returns a bundle_status; none aborts, traps or exits. The
 *    context keeps a message for the last failure (bundle_last_error).
 *  - Ownership: the library copies every input array at init into device
 *    buffers it owns; the caller keeps ownership of all pointers it passes and
 *    may free them once the call returns. Output buffers belong to the caller.
 *  - Pointers are host pointers unless a *_DEVICE flag says they are device
 *    pointers on the context's GPU.
 *  - Streams: `stream` is a cudaStream_t (NULL: the library creates its own
 *    non-blocking stream). bundle_iterate is asynchronous on that stream; the
 *    fetches synchronise it.
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef BUNDLE_3DHEB_H
#define BUNDLE_3DHEB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BUNDLE_OK = 0,
    BUNDLE_EINVAL = 1,    /* an argument is out of range or inconsistent */
    BUNDLE_ENOMEM = 2,    /* a device or host allocation failed */
    BUNDLE_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    BUNDLE_EOVERFLOW = 4, /* the integer widths cannot hold the worst-case bound */
    BUNDLE_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    BUNDLE_ESTATE = 6,    /* the call is not valid in the context's current state */
    BUNDLE_ENOTSUP = 7    /* a requested mode is not supported by this build */
} bundle_status;

/* Storage type of the density stack rho read by the gradient gather. */
typedef enum { BUNDLE_RHO_F32 = 0, BUNDLE_RHO_BF16 = 1, BUNDLE_RHO_F16 = 2 } bundle_rho_dtype;

/* Parameters. Fill with bundle_default_params, then override. */
typedef struct {
    int32_t grid_w, grid_h;   /* histogram size; both 0 => automatic (Sec. 5) */
    int32_t grid_dominant;    /* automatic size of the dominant axis (Sec. 5: 800) */
    int32_t margin_px;        /* free border kept by the world->grid map; -1 => radius */
    int32_t radius;           /* box radius r: each pass sums (2r+1)^2 cells (Sec. 3.1) */
    int32_t passes;           /* number of box passes k (Sec. 3.1: 3) */
    int32_t alpha_num;        /* repulsion alpha = alpha_num / alpha_den (Eq. 4: 1/4) */
    int32_t alpha_den;
    double h_max_sigmas;      /* h_max = h_max_sigmas * sigma_k (Sec. 3.3, Fig. 3: 2) */
    double lambda;            /* h_i = lambda^i h_max (Sec. 2.1: 0.5..0.9; Fig. 3: 0.9) */
    int32_t n_fixed;          /* > 0: points per polyline; 0: by length (below) */
    int32_t n_max;            /* by length: clamp(ceil(L / delta_px) + 1, 2, n_max) */
    float delta_px;           /* sampling step delta in pixels (Sec. 2.1) */
    float laplace_beta;       /* Laplacian weight beta (Sec. 3.3 leaves it open: 0.5) */
    float eps;                /* epsilon of Eq. 5 (density units: weight per cell) */
    int32_t step_tries;       /* step sizes tried: h, h/2, ..., h/2^(tries-1) (Sec. 3.3) */
    int32_t sum_bits;         /* width of the smoothed sums: 0 auto, 32 or 64 */
    int32_t rho_dtype;        /* bundle_rho_dtype */
    int32_t flags;            /* BUNDLE_FLAG_* */
    float directed_offset;    /* directed graphs (Sec. 3): after the first sampling, interior
                                 points move this fraction of max(W, H) along the normal
                                 (-dy, dx)/|d| of their edge; 0 = off (paper: 0.001..0.005) */
} bundle_params;

/* bundle_params.flags */
#define BUNDLE_FLAG_FIXED_STEP 1 /* KDEEB's advection (Sec. 3.3, Fig. 3): step exactly h, no
                                    density test -- the baseline the optimised step improves */
#define BUNDLE_FLAG_SEGMENT_HIST 2 /* histogram by Bresenham segments (Eq. 1 as rasterised in
                                      Sec. 4): every cell on a polyline segment gains w_e, joints
                                      counted once; default: every sample point adds w_e to its
                                      cell. The sums' int64 bound is then checked on the device
                                      each iteration; exceeding it makes the next sync, fetch or
                                      info call return BUNDLE_EOVERFLOW. */
#define BUNDLE_FLAG_INK_STATS 4 /* record, per iteration, the ink of the drawing entering it
                                   (occupied histogram cells): the convergence measure of
                                   bundle_fetch_ink (Sec. 3.3, Fig. 3 compares convergence of
                                   the two steps; fewer occupied cells = tighter bundles) */
#define BUNDLE_FLAG_LOAD_GATHERS 8 /* the advection's density gathers read the quad map through
                                      the load path; default: through a texture view of the same
                                      map (point sampled, the same bits), where the map's quads
                                      fit a 1D texture (the device's 1D linear texture width
                                      limit, in quads) and the texture can be made. Results
                                      are identical; only the speed differs. */

/* Result of bundle_get_info. */
typedef struct {
    int64_t n_edges;
    int64_t n_points;           /* points of the current polylines (after the last iteration) */
    int64_t n_points_resampled; /* points splatted by the last iteration */
    int32_t grid_w, grid_h, n_groups;
    int32_t sum_bits;           /* 32 or 64 */
    int32_t rho_dtype;
    int32_t iteration;          /* index i of the next iteration (h_i) */
    double map[5];              /* {xmin, ymin, scale, ox, oy}: px = (x - xmin) * scale + ox */
    double h_next;              /* h of the next iteration */
    int64_t device_bytes;       /* device memory owned by the context */
    int64_t points_processed;   /* sample points resampled and splatted since init: the sum
                                   over iterations of the points each iteration advects */
    int32_t tile_eb;            /* edges per block of the point kernels */
    int32_t tile_row;           /* row-pass variant: 0 by shape, 1 register rows, 2 shared rows,
                                   3 register windows with shuffled borders, 4 banded passes
                                   for both axes */
    int32_t tile_strip;         /* column-pass strip: 0 by shape, else 16 (TMA), 8, 4 or 2 */
    int32_t reserved;
} bundle_info;

typedef struct bundle_ctx bundle_ctx;

/* bundle_init / bundle_init_polylines flags */
#define BUNDLE_INPUT_DEVICE 1 /* input arrays are device pointers */

/* bundle_fetch flags */
#define BUNDLE_FETCH_DEVICE 1    /* off / xy are device pointers */
#define BUNDLE_FETCH_PIXELS 2    /* return grid pixel units instead of world coordinates */
#define BUNDLE_FETCH_RESAMPLED 4 /* the last iteration's resampled points (the splat input) */

/* bundle_fetch_density selectors */
#define BUNDLE_DENSITY_HIST 0 /* uint32 [G][H][W]: histogram of the last iteration (Eq. 1/3) */
#define BUNDLE_DENSITY_SUMS 1 /* int32/int64 [G][H][W]: k box passes, unnormalised (Sec. 3.1) */
#define BUNDLE_DENSITY_RHO 2  /* f32/bf16/f16 [G][H][W]: combined density (Eq. 3, Eq. 4) */

/* Defaults: the paper's values where it gives them (k = 3, alpha = 1/4,
 * h_max = 2 sigma, lambda = 0.9, dominant size 800), the readings for the
 * rest (r = 4, delta = 2 px, n_max = 64, beta = 0.5, eps = 1e-9, 8 tries). */
void bundle_default_params(bundle_params* p);

/*
 * Create a context from straight edges (Sec. 3.1: e = (x_s, x_t, w)).
 *  src_xy, dst_xy: float [2 * n_edges], interleaved (x, y), world coordinates.
 *  group: int32 [n_edges], group (bin) b_e in [0, n_groups) (Sec. 3.2); NULL => all 0.
 *  weight: int32 [n_edges], w_e >= 0 (Eq. 1); NULL => all 1.
 *  n_groups: 1..64 (Sec. 6 reports up to 64 groups).
 *  flags: BUNDLE_INPUT_DEVICE when the four arrays are device pointers.
 * The world->grid map is computed on the host in double and rounded to float
 * once. Returns EINVAL for bad sizes, EOVERFLOW when the integer histogram,
 * sums or layer mix cannot hold their worst-case bound, ENOMEM, ECUDA.
 * On failure *out is NULL and bundle_last_error(NULL) describes the cause.
 */
bundle_status bundle_init(bundle_ctx** out, const bundle_params* p, int64_t n_edges,
                          const float* src_xy, const float* dst_xy, const int32_t* group,
                          int32_t n_groups, const int32_t* weight, int32_t flags, void* stream);

/*
 * Create a context from polylines already in grid pixel units (resume from a
 * fetched state, or start from a chosen configuration).
 *  off: int64 [n_edges + 1] CSR offsets; every polyline has 2..cap points,
 *       cap = n_fixed if > 0 else n_max.
 *  xy_px: float [2 * off[n_edges]], interleaved, inside [0, W) x [0, H).
 *  p->grid_w, p->grid_h must be > 0. map5: the world map to report and to
 *  invert in bundle_fetch (NULL: identity, scale 1). iteration: index i of the
 *  first iteration to run (sets h_i).
 */
bundle_status bundle_init_polylines(bundle_ctx** out, const bundle_params* p, int64_t n_edges,
                                    const int64_t* off, const float* xy_px, const int32_t* group,
                                    int32_t n_groups, const int32_t* weight, const double* map5,
                                    int32_t iteration, int32_t flags, void* stream);

/*
 * Run n_iters iterations of the loop (Sec. 3, Fig. 2) asynchronously on the
 * context's stream. Iteration i uses h_i = lambda^i h_max (Sec. 2.1, Sec. 3.3).
 * Returns EINVAL for n_iters < 0, ECUDA if a launch fails.
 */
bundle_status bundle_iterate(bundle_ctx* ctx, int32_t n_iters);

/*
 * Copy the current polylines out (synchronises the stream).
 *  off: int64 [n_edges + 1] CSR offsets, in the caller's edge order.
 *  xy: float [2 * cap], interleaved; n_points receives the point count.
 *  flags: BUNDLE_FETCH_DEVICE, BUNDLE_FETCH_PIXELS, BUNDLE_FETCH_RESAMPLED.
 * Returns EINVAL when cap is smaller than the point count (n_points is still
 * set), ESTATE for RESAMPLED before any iteration.
 */
bundle_status bundle_fetch(bundle_ctx* ctx, int64_t* off, float* xy, int64_t cap,
                           int64_t* n_points, int32_t flags);

/*
 * Copy one [G][H][W] stack of the last iteration (synchronises the stream).
 * which: BUNDLE_DENSITY_HIST (uint32), _SUMS (int32 or int64 per sum_bits),
 * _RHO (per rho_dtype). dst_bytes must be at least G*H*W*element size.
 * flags: BUNDLE_FETCH_DEVICE when dst is a device pointer.
 */
bundle_status bundle_fetch_density(bundle_ctx* ctx, int32_t which, void* dst, int64_t dst_bytes,
                                   int32_t flags);

/*
 * Batched form: many independent graphs bundled together. Each graph has its
 * own edges, groups, grid and parameters (the paper bundles one graph at a
 * time; batching serves many small graphs at once). The batch context owns one
 * member context per graph (own buffers and stream); bundle_iterate on the
 * batch runs every member, and each steady-state iteration of all members is
 * one CUDA graph launch with one branch per member, so small graphs run side
 * by side on the GPU. Fetch results through bundle_batch_member.
 */
typedef struct {
    int64_t n_edges;
    const float* src_xy;   /* float [2 * n_edges], world coordinates */
    const float* dst_xy;
    const int32_t* group;  /* nullable */
    int32_t n_groups;
    const int32_t* weight; /* nullable */
} bundle_graph_desc;

/* Create a batch of n_graphs (1..4096) graphs; params holds one bundle_params per
 * graph. flags as bundle_init (applies to every graph). On failure *out is NULL and
 * bundle_last_error(NULL) names the graph. */
bundle_status bundle_init_batch(bundle_ctx** out, int32_t n_graphs,
                                const bundle_graph_desc* graphs, const bundle_params* params,
                                int32_t flags, void* stream);

/* Number of graphs of a batch (0 for a single-graph context). */
int32_t bundle_batch_size(const bundle_ctx* ctx);

/* Borrowed handle of graph k of a batch (NULL if out of range), valid until the
 * batch is destroyed: bundle_fetch, bundle_fetch_density and bundle_get_info work
 * on it; bundle_iterate on a member returns ESTATE, bundle_destroy ignores it. */
bundle_ctx* bundle_batch_member(bundle_ctx* ctx, int32_t k);

/*
 * General layer interaction (Eq. 3): replace Eq. 4's matrix by
 * M(l, b) = num[l * G + b] / den (row-major G x G, den > 0), e.g. for ordinal or
 * modular bins (Sec. 3.2). The mix stays exact: rho_l = (sum_b num[l,b] S_b) /
 * (den s^k) with an int64 numerator. Returns EOVERFLOW when
 * max_l sum_b |num[l,b]| times the smoothed-sum bound does not fit int64, EINVAL
 * for den <= 0 or a batch context. num is copied; applies from the next iteration.
 */
bundle_status bundle_set_interaction(bundle_ctx* ctx, const int64_t* num, int64_t den);

/*
 * Convergence record (needs BUNDLE_FLAG_INK_STATS): for iterations first .. first+n-1
 * (each < the context's iteration count and < BUNDLE_INK_STATS_CAP) writes
 * out[2 i] = cells where any group's histogram is non-zero (the ink of the drawing
 * entering iteration first+i, at grid resolution), out[2 i + 1] = the sum over groups of
 * each group's non-zero cells (minus out[2 i]: cells shared by several groups, the
 * overlaps between groups that Sec. 3.3 sees fall as bundling proceeds). With
 * BUNDLE_FLAG_SEGMENT_HIST the histogram is the rasterised drawing itself (Sec. 4).
 * out: host int64 [2 n]. Synchronises the stream. EINVAL for a range outside the record,
 * ESTATE without the flag or for a batch context (ask its members).
 */
#define BUNDLE_INK_STATS_CAP 4096
bundle_status bundle_fetch_ink(bundle_ctx* ctx, int64_t* out, int32_t first, int32_t n);

/*
 * Headless rendering of the current drawing (Sec. 3.4): polylines drawn as line
 * segments coloured by bin, bundle weight shown by alpha accumulation and by a line
 * width that follows the density at the sample points. OpenGL is not used; the
 * image is a device computation:
 *  - image: (grid_w * scale) x (grid_h * scale) pixels, pixel (px, py) centred at
 *    (px + 0.5, py + 0.5) / scale in grid units;
 *  - segment j of an edge has width w = width_min + (width_max - width_min) u, with
 *    u = clamp(rho_bar / rho_ref, 0, 1) (log2(1 + u) when log_width), rho_bar the
 *    mean of the bilinear density of the edge's own layer (the last iteration's map)
 *    at its two points; rho_ref <= 0: the largest density of the stack;
 *  - it covers the pixels whose centre is within w / 2 of it; a pixel nearest to a
 *    segment's far end (projection t >= 1) is left to the next segment, so joints
 *    are drawn once (the last segment keeps its end);
 *  - each covered pixel gains the optical depth tau_e = w_e * llround(-ln(1 - alpha)
 *    * 2^20) and tau_e times the bin's RGB (integer sums: independent of order); the
 *    pixel's opacity is 1 - exp(-sum tau / 2^20), its colour the tau-weighted mean,
 *    composited over the background and rounded to 8 bits, alpha 255.
 */
typedef struct {
    int32_t scale;         /* 1..16 */
    float alpha;           /* opacity of one unit-weight edge, 0 < alpha < 1 */
    float width_min;       /* image pixels, 1 <= width_min <= width_max <= 64 */
    float width_max;
    float rho_ref;         /* density drawn at width_max; <= 0: the stack's maximum */
    int32_t log_width;     /* 0: linear in u; 1: log2(1 + u) */
    uint8_t background[4]; /* RGB, the fourth byte unused */
} bundle_render_params;

/*
 * palette: host uint8 [n_groups][3] RGB per bin (nominal bins: distinct colours;
 * ordinal: a sequential table; Sec. 3.4). rgba: uint8 [Hi][Wi][4], host, or device
 * with BUNDLE_FETCH_DEVICE. accum: optional int64 [Hi][Wi][4] (sum tau, sum tau R,
 * sum tau G, sum tau B), same memory kind as rgba. Needs one finished iteration
 * (ESTATE otherwise, and for a batch context: render its members). Allocates
 * n_groups * Hi * Wi * 8 bytes of device workspace for the call (one depth map per
 * bin; at most 2^30 cells, and Hi * Wi <= 2^28: EINVAL beyond); synchronises the
 * stream.
 */
bundle_status bundle_render(bundle_ctx* ctx, const bundle_render_params* params,
                            const uint8_t* palette, uint8_t* rgba, int64_t* accum,
                            int32_t flags);

/*
 * Autotuner for the tile shapes (the paper has no counterpart; its CPU threads need
 * none). On a context fresh from bundle_init (or a batch of them, each graph tuned on
 * its own edges), times on the GPU: the edges per block of the point kernels (4, 8,
 * 16, 32 -- one warp works through each block; each candidate resamples, splats and filters the straight edges, then
 * the fused advect + resample step is timed), the row-pass variant and the column-pass
 * strip, then the banded path (row mode 4, both passes) against the fastest pair, and
 * keeps the fastest of each (bundle_info.tile_*). Results do not depend on
 * the tiles: every choice gives the same bits. The context returns to its fresh state
 * (iteration 0). ESTATE after an iteration, for bundle_init_polylines contexts and for
 * batch members; synchronises the stream; allocates E * 32 bytes while it runs.
 */
bundle_status bundle_autotune(bundle_ctx* ctx);

/* Set the tiles by hand (e.g. those an earlier bundle_autotune chose for the same
 * shape): eb 0 (keep) or 4, 8, 16, 32 edges per warp-owned block of the point
 * layout -- only on a fresh bundle_init context;
 * row_mode 0 (by shape), 1 (register rows, widths of 225..256, 481..512 or 993..1024
 * cells), 2 (shared-memory rows), 3 (windows in registers with borders exchanged by
 * shuffles: widths of exactly 512 (radius <= 15) or 1024 (radius <= 16)), 4 (the banded
 * path for both passes: the row passes stream bands of 8 rows through shared memory
 * and write the result transposed, the column passes then run the same way over that
 * -- widths and heights of exactly 512 (radius <= 15) or 1024 (radius <= 16); the
 * default where it applies, 3 where only the width fits; col_strip is then unused);
 * col_strip 0 (by shape), 16 (strips staged by the
 * tensor memory accelerator: heights up to 1024, width x sum bytes a multiple of 16),
 * 2, 4 or 8 (strips copied with cp.async, when the strip's column fits in shared
 * memory; 8 is the default up to height 1024). EINVAL for a choice that does not exist,
 * ESTATE for eb on an iterated context or for batches. */
bundle_status bundle_set_tiles(bundle_ctx* ctx, int32_t eb, int32_t row_mode, int32_t col_strip);

/* Sizes, widths, map, schedule and point counts of a context (synchronises the stream).
 * For a batch: sums of the counts over its graphs; sizes and map of graph 0. */
bundle_status bundle_get_info(const bundle_ctx* ctx, bundle_info* out);

/*
 * Per-kernel timing with CUDA events recorded on the context's stream around
 * every launch of bundle_iterate (a tracing aid; off by default, adds two event
 * records per launch). Kinds, in order: 0 resample+splat, 1 advect+Laplacian,
 * 2 advect+Laplacian+resample+splat, 3 row box passes, 4 column box passes,
 * 5 layer mix into the density quad map, 6 histogram clear.
 */
#define BUNDLE_PROFILE_KINDS 7
bundle_status bundle_profile_enable(bundle_ctx* ctx, int32_t on);

/*
 * Synchronise and report, per kind, the summed event time in ms and the
 * launch count of everything recorded since the last reset. ms and launches
 * hold n entries (n <= BUNDLE_PROFILE_KINDS is read; extra entries are zeroed).
 * reset != 0 clears the records.
 */
bundle_status bundle_profile_read(bundle_ctx* ctx, double* ms, int64_t* launches, int32_t n,
                                  int32_t reset);

/*
 * Box-pass smoothing that allocates no memory (the paper has no counterpart;
 * it is an integration aid). Some callers cannot call cudaMalloc: code running
 * under a framework whose caching allocator owns all device memory, services
 * that reserve their memory budget up front, or paths that must avoid the
 * implicit synchronisation cudaMalloc/cudaFree can cause. This entry point
 * runs the same row and column box passes as bundle_iterate with its
 * intermediate stack in a fixed 16 MiB device array compiled into the library
 * (every GPU that loads the library holds it until exit).
 *  hist: device uint32 [n_groups][grid_h][grid_w] histogram (input).
 *  sums: device [n_groups][grid_h][grid_w] int32 (sum_bits 32) or int64
 *        (sum_bits 64) output: `passes` unnormalised (2r+1)^2 box sums with
 *        half-sample reflection, exactly as BUNDLE_DENSITY_SUMS.
 *  sum_bits must hold 4 (2r+1)^(2(passes-1)) times the histogram's total; the
 *  call does not check this bound (bundle_init does, for its own contexts).
 *  hist and sums must both live on the current device: the launches and the
 *  fixed array are those of the current device. The C ABI cannot see their
 *  sizes; a sums buffer smaller than the stack is written past its end.
 *  stream: cudaStream_t, NULL for the legacy default stream; asynchronous.
 * Returns EINVAL when n_groups * grid_h * grid_w * sum_bits / 8 exceeds
 * 16 MiB or an argument is out of range (message via bundle_last_error(NULL)),
 * ECUDA on a launch failure. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture. The address is cached per device and CUDA context, so the
 * first call after a reset of the device looks it up again. All calls share the one array and it keeps the last call's
 * contents; nothing in it needs clearing (the row passes overwrite every cell
 * the column passes read), but calls that overlap on the GPU race on it.
 */
bundle_status bundle_smooth_noalloc(const uint32_t* hist, void* sums, int32_t n_groups,
                                    int32_t grid_h, int32_t grid_w, int32_t radius,
                                    int32_t passes, int32_t sum_bits, void* stream);

/*
 * Split form: one graph's edges divided over several contexts -- one per process or
 * GPU -- that together give exactly the run of one context over all edges (Sec. 4
 * divides a graph's edges over CPU threads the same way). Every per-edge stage runs
 * on a context's own edges; the histogram, the only state that couples edges, is
 * summed over the contexts between the splat and the box passes (an integer sum:
 * exact and order-free, e.g. an all-reduce). The contexts must share the grid map:
 * create them with bundle_init_polylines from pixel-unit polylines and one map, and
 * set params.sum_bits to the width the whole graph needs (a context sizes its
 * integers for its own edges otherwise, too small for the summed histogram).
 * A run of n iterations on each context:
 *   bundle_points_step(ctx, 0)                     resample + splat (opens the run)
 *   repeat n times:
 *     fetch BUNDLE_DENSITY_HIST, sum it over the contexts, bundle_set_histogram
 *     bundle_density_step(ctx)                     box passes, layer mix, density
 *     bundle_points_step(ctx, last ? BUNDLE_STEP_LAST : 0)
 *                                                  advect + Laplacian (+ resample +
 *                                                  splat for the next iteration)
 * With one context and no exchange this is bundle_iterate(ctx, n), bit for bit.
 * ESTATE when a call comes out of this order; bundle_iterate refuses while a run is
 * open. Asynchronous on the context's stream (host-memory histograms synchronise).
 */
#define BUNDLE_STEP_LAST 1 /* bundle_points_step: the last iteration of the run */
bundle_status bundle_points_step(bundle_ctx* ctx, int32_t flags);
bundle_status bundle_density_step(bundle_ctx* ctx);
/* Replace the splatted histogram of the open iteration by src (uint32 [G][H][W],
 * flags BUNDLE_INPUT_DEVICE for a device pointer), e.g. its sum over the contexts. */
bundle_status bundle_set_histogram(bundle_ctx* ctx, const uint32_t* src, int32_t flags);

/* Wait for the context's stream; reports a deferred kernel error as ECUDA. */
bundle_status bundle_sync(bundle_ctx* ctx);

/* Free every resource of the context (synchronises first). NULL is a no-op. */
void bundle_destroy(bundle_ctx* ctx);

/* Message of the last failure of ctx (NULL: of the last failed init on this thread). */
const char* bundle_last_error(const bundle_ctx* ctx);

/* Name of a status code. */
const char* bundle_status_string(bundle_status s);

#ifdef __cplusplus
}
#endif

#endif /* BUNDLE_3DHEB_H */
