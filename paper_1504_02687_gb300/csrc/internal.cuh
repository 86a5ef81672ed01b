// Internal declarations shared by the kernel translation units and the host
// side of the bundling library. Nothing here is part of the C ABI.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace heb {

// Point layout. Edges live in blocks of `eb` consecutive (spatially sorted)
// slots, eb <= kMaxEdgesPerWarp chosen per context; block b owns the point region
// [b * eb * cap, (b+1) * eb * cap) of a float2 buffer, and packs its edges'
// polylines back to back inside it, in slot order. Only the per-slot point
// counts are stored: the warp that owns a block recovers its edges' offsets with
// one warp scan. Buffers are sized for blocks of kEdgesPerBlock slots, which
// covers every eb that divides it.
constexpr int kEdgesPerBlock = 128;
constexpr int kMaxEdgesPerWarp = 32;  // one slot per lane
constexpr int kStepWarps = 4;         // warps per CTA of the step kernel, one block each
constexpr int kStepThreads = 32 * kStepWarps;
constexpr int kStage = 192;           // points of whole polylines staged per warp
constexpr int kMaxCap = 64;           // largest polyline (n_fixed or n_max): two points per lane
constexpr float kEdgeGuard = 0.0009765625f;  // positions stay below W - 2^-10
// CTAs of one step launch over E edges in blocks of eb.
__host__ __device__ inline int64_t step_ctas(int64_t E, int eb) {
    const int64_t blocks = (E + eb - 1) / eb;
    return (blocks + kStepWarps - 1) / kStepWarps;
}
// The splat writes into kHistCopies copies of the histogram (block b into copy
// b mod kHistCopies) and the row-pass kernel sums them as it reads: bundled
// polylines put many points on the same cells, and atomics on one address
// serialise in L2, so spreading them over copies shortens those queues.
constexpr int kHistCopies = 2;

enum StepMode : int {
    kModeResample = 2,                // resample + splat the input polylines
    kModeAdvect = 1,                  // advect + Laplacian, write polylines
    kModeAdvectResample = 3,          // advect + Laplacian + resample + splat
    kModeTexGather = 4,               // (with kModeAdvect) density gathers via StepArgs::qtex
};

struct StepArgs {
    const int32_t* cnt_in;   // [E] points per slot (input layout)
    const float2* pts_in;    // input polylines (block layout)
    int32_t* cnt_out;        // [E] points per slot (output layout)
    float2* pts_out;         // output polylines (block layout)
    const int32_t* group;    // [E] per slot
    const int32_t* weight;   // [E] per slot
    const void* quads;       // [G][H+3][W+3] density quads (see below), rho type x 4
    unsigned long long qtex; // the same quads as a 1D texture (texel i = quad i), or 0: the
                             // gathers then read `quads` through the load path
    uint32_t* hist;          // [G][H][W] histogram accumulated by the splat
    unsigned long long* n_splat;  // running count of splatted points
    int64_t E;
    int32_t eb;              // edges per block (<= kMaxEdgesPerWarp)
    int32_t cap;             // points per slot of the region (n_fixed or n_max)
    int32_t W, H, G;
    float h;                 // step magnitude h_i (used when h_sched is null)
    const float* h_sched;    // device schedule h_0, h_1, ... (graph-captured launches)
    const int32_t* iter;     // device index of the current iteration into h_sched
    float eps;               // Eq. 5 epsilon
    int32_t tries;           // step sizes tried
    float lap_keep;          // 1 - beta
    float lap_half_beta;     // beta / 2
    int32_t n_fixed, n_max;
    float delta;
    int32_t fixed_step;      // KDEEB step: exactly h, no density test
    float dir_amount;        // directed graphs: normal offset (px) of interior resampled points
    int32_t seg_hist;        // histogram by Bresenham segments instead of points
    unsigned long long* mass;  // total weight splatted by this launch (segment mode)
};

struct RenderArgs {
    const int32_t* cnt;      // [E] points per slot of the current polylines
    const float2* pts;       // current polylines (block layout)
    const int32_t* group;    // [E] per slot
    const int32_t* weight;   // [E] per slot
    const void* quads;       // density quads of the last iteration (rho type x 4)
    unsigned long long* depth;  // [G][Hi][Wi]: optical depth per bin (2^-20 units)
    unsigned int* rho_ref;   // density mapped to the full width, as float bits
    int64_t E;
    int32_t eb, cap, W, H, G;
    int32_t scale, Wi, Hi;   // image = grid x scale
    unsigned long long tau1; // optical depth of one unit-weight edge, 2^-20 units
    float width_min, width_max;
    int32_t log_width;
};

// One launch of the step kernel over many graphs (the batched form): graph m owns the
// CTAs [blk[m], blk[m + 1]) and its own arguments. Passed by value (kernel parameter
// space): kBatchLaunch graphs per launch.
constexpr int kBatchLaunch = 96;
struct BatchStepArgs {
    int32_t n;
    int32_t blk[kBatchLaunch + 1];
    StepArgs a[kBatchLaunch];
};

struct FilterArgs {
    const uint32_t* hist;  // [copies][G][H][W]: the histogram is the sum of the copies
    int32_t hist_copies;
    void* Y;               // [G][H][W] row-filtered workspace (sum type)
    void* S;               // [G][H][W] smoothed sums (sum type)
    void* rho;             // [G][H][W] density (rho type), filled from the quads on demand
    void* quads;           // [G][H+3][W+3] density quads (rho type x 4)
    int32_t G, H, W, r, passes;
    const int64_t* mix;    // optional G x G integer interaction numerators (row-major)
    int64_t mix_self;      // q (G - 1) + p : weight of a group's own layer
    int64_t mix_all;       // p : weight of the all-groups sum
    float inv_den_f;       // unused (kept for a future reciprocal form)
    float den_f;           // q (G - 1) s^k (or s^k for one group), rounded to float
    int32_t strip;         // column-pass strip: 16 (TMA-staged), 8, 4 or 2 (0: by shape)
    int32_t row_mode;      // row pass: 0 by shape, 1 register-resident rows, 2 shared-memory
                           // rows, 3 windows in registers with shuffled borders, 4 banded
                           // rows for both passes (Y holds the transposed stack)
    int32_t* err_flag;     // sticky device error word (2: a TMA copy did not land in time)
    int32_t clear_hist;    // 1: the row pass leaves the histogram zero where it can (the
                           // banded path); filter_clears_hist tells whether it does
};

// Density quads. The gather side of the iteration reads each layer's density through
// a quad map: entry (a, b), for a in [-2, W] and b in [-2, H], holds the four values
// {E(a,b), E(a+1,b), E(a,b+1), E(a+1,b+1)} of the reflection-extended map
// E(a, b) = rho(refl(a), refl(b)) at quad index (b + 2) * (W + 3) + (a + 2). One
// quad is the whole 2x2 footprint of a bilinear lookup (one 16-byte load for FP32
// densities, 8 bytes for 16-bit ones); four quads hold the 12 cells of the gradient
// stencil. No index reflection happens on the gather side.
constexpr int kQuadPad = 3;
__host__ __device__ inline int64_t quad_elems(int W, int H) {
    return (int64_t)(W + kQuadPad) * (H + kQuadPad);
}

// Launchers (return the launch status; nothing here synchronises).
cudaError_t launch_step(int mode, int rho_dtype, const StepArgs& a, cudaStream_t st);
cudaError_t launch_step_batch(int mode, int rho_dtype, const BatchStepArgs& P, cudaStream_t st);
// Advance the iteration counter of every graph of P.
cudaError_t launch_advance_batch(const BatchStepArgs& P, cudaStream_t st);
cudaError_t launch_rowbox(int sum_bits, const FilterArgs& a, cudaStream_t st);
cudaError_t launch_colbox(int sum_bits, const FilterArgs& a, cudaStream_t st);
// Layer mix (Eq. 3 / Eq. 4) of the sums straight into the density quad map.
cudaError_t launch_mix_quads(int sum_bits, int rho_dtype, const FilterArgs& a, cudaStream_t st);
// The density stack [G][H][W] (a.rho) from the quad map (for fetches and the renderer).
cudaError_t launch_rho_from_quads(int rho_dtype, const FilterArgs& a, cudaStream_t st);
// Fold histogram copies 1.. into copy 0 (their sum is unchanged), n cells per copy.
cudaError_t launch_fold_hist(uint32_t* hist, int64_t n, int copies, cudaStream_t st);
// Renderer: capsule fragments into the accumulators (after the stack maximum of rho
// into *rho_ref when want_max), then the RGBA8 resolve.
cudaError_t launch_render(int rho_dtype, const RenderArgs& a, const void* rho, int64_t rho_n,
                          bool want_max, int n_sm, cudaStream_t st);
cudaError_t launch_render_resolve(const unsigned long long* depth, int G, int64_t n_pixels,
                                  const int32_t* palette, const unsigned char* bg, void* rgba,
                                  void* accum, cudaStream_t st);
// Ink statistics of the histogram into stats[2 * (*iter)] (skipped past stats_cap).
cudaError_t launch_ink(const uint32_t* hist, int64_t cells, int G, int copies,
                       unsigned long long* stats, const int32_t* iter, int32_t stats_cap,
                       int n_sm, cudaStream_t st);

// Init / fetch helpers (point layout <-> caller order).
cudaError_t launch_edge_keys(const float2* src, const float2* dst, const int32_t* group,
                             int64_t E, int32_t W, int32_t H, uint32_t* key, uint32_t* bucket_cnt,
                             cudaStream_t st);
cudaError_t launch_bucket_scan(uint32_t* cnt, int32_t n_buckets, cudaStream_t st);
cudaError_t launch_edge_scatter(const uint32_t* key, int64_t E, uint32_t* cursor, int32_t* perm,
                                cudaStream_t st);
cudaError_t launch_gather_edges(const int32_t* perm, int64_t E, const int32_t* group_in,
                                const int32_t* weight_in, int32_t* group_out,
                                int32_t* weight_out, cudaStream_t st);
cudaError_t launch_straight_layout(const int32_t* perm, int64_t E, const float2* src,
                                   const float2* dst, int32_t eb, int32_t cap, int32_t* cnt,
                                   float2* pts, cudaStream_t st);
cudaError_t launch_polyline_layout(const int32_t* perm, int64_t E, const int64_t* off,
                                   const float2* xy, int32_t eb, int32_t cap, int32_t* cnt,
                                   float2* pts, cudaStream_t st);
cudaError_t launch_counts_to_caller(const int32_t* perm, const int32_t* cnt, int64_t E,
                                    int64_t* off_out, cudaStream_t st);
cudaError_t launch_scan_offsets(int64_t* off, int64_t E, int64_t* tmp, cudaStream_t st);
cudaError_t launch_layout_to_caller(const int32_t* perm, const int32_t* cnt, const float2* pts,
                                    int64_t E, int32_t eb, int32_t cap, const int64_t* off,
                                    float2* xy_out,
                                    int32_t to_world, float ox, float oy, float inv_scale,
                                    float xmin, float ymin, cudaStream_t st);
cudaError_t launch_sum_counts(const int32_t* cnt, int64_t E, unsigned long long* total,
                              cudaStream_t st);
// Device iteration counter used with the device schedule of h (graph-friendly).
cudaError_t launch_set_iter(int32_t* iter, int32_t value, cudaStream_t st);
// Copy two-point polylines (the straight edges of a fresh context) from one block layout
// to another: slot s sits at (s / eb) * eb * cap + 2 * (s % eb); cnt_dst (if set) gets 2.
cudaError_t launch_relayout_pairs(const float2* src, int32_t eb_src, int32_t cap_src, float2* dst,
                                  int32_t eb_dst, int32_t cap_dst, int32_t* cnt_dst, int64_t E,
                                  cudaStream_t st);
// Whether a row-pass / column-pass tile choice exists for this grid.
bool rowbox_mode_valid(int mode, int W, int H, int r);
// The k passes of the box filter along every row of a [G][NR][L] stack (L = 512 with
// r <= 15, or 1024 with r <= 16), written transposed to [G][L][NR]. in: the histogram
// (32-bit, `copies` copies copy_stride cells apart, summed) or, with sum_input, a sum
// stack of the sum type; in 16-byte aligned, out 8-byte aligned. zero: null, or the
// histogram itself (not with sum_input), whose rows are left zero once read.
bool band_rows_fits(int L, int r);
cudaError_t launch_band_rows(int sum_bits, bool sum_input, const void* in, int copies,
                             int64_t copy_stride, void* out, int G, int NR, int L, int r,
                             int passes, uint32_t* zero, cudaStream_t st);
// Whether launch_rowbox with these arguments leaves the histogram zero (clear_hist set
// and the banded path taken).
bool filter_clears_hist(const FilterArgs& a);
bool colbox_strip_valid(int strip, int W, int H, int r, int sum_bytes);
// Sticky overflow flag: set when *mass > allowed.
cudaError_t launch_check_mass(const unsigned long long* mass, unsigned long long allowed,
                              int32_t* flag, cudaStream_t st);
cudaError_t launch_advance_iter(int32_t* iter, cudaStream_t st);
size_t scan_offsets_tmp_elems(int64_t E);

// Message returned by bundle_last_error(NULL) on this thread.
void set_thread_error(const char* msg);

}  // namespace heb
