// Grid-side kernels of the bundling iteration: the repeated box filters of
// Sec. 3.1 and the layer interaction of Eq. 3 / Eq. 4.
//
// A (2r+1) x (2r+1) box sum is separable: it equals a (2r+1)-wide running sum
// along every row followed by one along every column, and with per-axis
// half-sample reflection the row and column passes commute. k passes of the 2D
// box therefore equal k row passes followed by k column passes, computed here
// by two kernels that each keep a whole row (or a strip of columns) in shared
// memory. Each 1D pass is the difference form of a 1D integral image kept as a
// running window sum. All sums are unsigned integers: modular wrap-around
// cancels exactly, so every box sum that fits its type is exact.
#include <cuda.h>  // CUtensorMap (the encoder is fetched through the runtime)

#include "box.cuh"
#include "internal.cuh"

namespace heb {
namespace {

__device__ __forceinline__ int reflect_index(int i, int n) {
    return i < 0 ? -1 - i : (i >= n ? 2 * n - 1 - i : i);
}

// ------------------------------------------------------------------ row passes
// One warp per row, `rows` warps per CTA. Lane l owns the contiguous chunk
// [l*c, (l+1)*c) of the row; the shared row is padded after every chunk so the
// 32 lanes walking their chunks in lockstep hit distinct banks.
template <typename TS>
__global__ void k_rowbox(const uint32_t* __restrict__ hist, int copies, TS* __restrict__ Y, int G,
                         int H, int W, int r, int passes, int rows, int c, int pad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.y;
    const int v = blockIdx.x * rows + warp;
    if (v >= H) return;
    const int stride = W + 32 * pad;
    TS* src = reinterpret_cast<TS*>(smem_raw) + (size_t)warp * 2 * stride;
    TS* dst = src + stride;
    const size_t base = ((size_t)g * H + v) * W;
    const size_t stride_copy = (size_t)G * H * W;
    if ((W & 3) == 0) {
        // 16-byte loads of every copy, all issued before they are summed
        const uint4* h0 = reinterpret_cast<const uint4*>(hist + base);
        for (int x4 = lane; x4 < (W >> 2); x4 += 32) {
            uint4 v = __ldg(h0 + x4);
            for (int k = 1; k < copies; ++k) {
                const uint4 u = __ldg(reinterpret_cast<const uint4*>(hist + k * stride_copy + base) + x4);
                v.x += u.x;
                v.y += u.y;
                v.z += u.z;
                v.w += u.w;
            }
            const int x = 4 * x4;
            src[x + (x / c) * pad] = (TS)v.x;
            src[x + 1 + ((x + 1) / c) * pad] = (TS)v.y;
            src[x + 2 + ((x + 2) / c) * pad] = (TS)v.z;
            src[x + 3 + ((x + 3) / c) * pad] = (TS)v.w;
        }
    } else {
        for (int x = lane; x < W; x += 32) {
            TS v = (TS)hist[base + x];
            for (int k = 1; k < copies; ++k) v += (TS)hist[k * stride_copy + base + x];
            src[x + (x / c) * pad] = v;
        }
    }
    __syncwarp();
    const int i0 = lane * c, i1 = min(i0 + c, W);
    for (int p = 0; p < passes; ++p) {
        if (i0 < i1) {
            TS s = 0;
            for (int t = i0 - 1 - r; t <= i0 - 1 + r; ++t) {
                int q = reflect_index(t, W);
                s += src[q + (q / c) * pad];
            }
            for (int i = i0; i < i1; ++i) {
                int qa = reflect_index(i + r, W), qs = reflect_index(i - r - 1, W);
                s += src[qa + (qa / c) * pad] - src[qs + (qs / c) * pad];
                dst[i + (i / c) * pad] = s;
            }
        }
        __syncwarp();
        TS* t = src;
        src = dst;
        dst = t;
    }
    for (int x = lane; x < W; x += 32) Y[base + x] = src[x + (x / c) * pad];
}

// Row passes for rows whose lane chunk c = ceil(W / 32) is C (8, 16 or 32): lane l
// owns [l*C, l*C + C) and keeps a pass's outputs in registers until the warp has
// read the pass's input, so a row needs one shared buffer. The buffer holds the row
// with a border of `halo` >= r + 1 cells on each side filled with the reflected
// values (refreshed after every pass), so every window reads its cells directly,
// with no index reflection. A slot is skipped after every C cells, so the 32 lanes,
// C apart, hit different banks.
constexpr int kRowWarps = 8;

template <int C>
__host__ __device__ __forceinline__ int padded(int k) { return k + k / C; }

template <typename TS, int C>
__global__ void __launch_bounds__(32 * kRowWarps)
    k_rowbox_reg(const uint32_t* __restrict__ hist, int copies, TS* __restrict__ Y, int G, int H,
                 int W, int r, int passes, int halo) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int LG = C == 8 ? 3 : C == 16 ? 4 : 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int stride = padded<C>(W + 2 * halo) + 1;
    TS* buf = reinterpret_cast<TS*>(smem_raw) + (size_t)warp * stride;
    const int g = blockIdx.y;
    const int v = blockIdx.x * kRowWarps + warp;
    if (v >= H) return;
    // cell t (t in [-halo, W + halo)) lives in slot padded(t + halo)
    auto slot = [&](int t) { return padded<C>(t + halo); };
    const size_t base = ((size_t)g * H + v) * W;
    const size_t stride_copy = (size_t)G * H * W;
    if ((W & 3) == 0 && copies == 2) {
        // every 16-byte load of both copies in flight before the first is summed
        constexpr int kIt = C / 4;  // W <= 32 C: at most C / 4 loads of 4 cells per lane
        const uint4* h0 = reinterpret_cast<const uint4*>(hist + base);
        const uint4* h1 = reinterpret_cast<const uint4*>(hist + stride_copy + base);
        uint4 u[kIt], w[kIt];
#pragma unroll
        for (int it = 0; it < kIt; ++it) {
            const int x4 = lane + 32 * it;
            if (x4 < (W >> 2)) {
                u[it] = __ldg(h0 + x4);
                w[it] = __ldg(h1 + x4);
            }
        }
#pragma unroll
        for (int it = 0; it < kIt; ++it) {
            const int x4 = lane + 32 * it;
            if (x4 < (W >> 2)) {
                const int x = 4 * x4;
                buf[slot(x)] = (TS)(u[it].x + w[it].x);
                buf[slot(x + 1)] = (TS)(u[it].y + w[it].y);
                buf[slot(x + 2)] = (TS)(u[it].z + w[it].z);
                buf[slot(x + 3)] = (TS)(u[it].w + w[it].w);
            }
        }
    } else if ((W & 3) == 0) {
        const uint4* h0 = reinterpret_cast<const uint4*>(hist + base);
        for (int x4 = lane; x4 < (W >> 2); x4 += 32) {
            uint4 u = __ldg(h0 + x4);
            for (int k = 1; k < copies; ++k) {
                const uint4 w = __ldg(reinterpret_cast<const uint4*>(hist + k * stride_copy + base) + x4);
                u.x += w.x;
                u.y += w.y;
                u.z += w.z;
                u.w += w.w;
            }
            const int x = 4 * x4;
            buf[slot(x)] = (TS)u.x;
            buf[slot(x + 1)] = (TS)u.y;
            buf[slot(x + 2)] = (TS)u.z;
            buf[slot(x + 3)] = (TS)u.w;
        }
    } else {
        for (int x = lane; x < W; x += 32) {
            TS u = (TS)hist[base + x];
            for (int k = 1; k < copies; ++k) u += (TS)hist[k * stride_copy + base + x];
            buf[slot(x)] = u;
        }
    }
    // the reflected border: cells -r-1 .. -1 and W .. W+r
    auto refresh_border = [&]() {
        __syncwarp();
        for (int k = lane; k < 2 * (r + 1); k += 32) {
            const int t = k <= r ? -1 - k : W + (k - r - 1);
            buf[slot(t)] = buf[slot(reflect_index(t, W))];
        }
        __syncwarp();
    };
    refresh_border();
    const int i0 = lane * C;
    const int len = max(0, min(C, W - i0));
    // lane's chunk: cell i0 + x is bl[x + floor(x / C)] (i0 + halo is a multiple of C)
    TS* bl = buf + slot(i0);
    TS out[C];
    for (int p = 0; p < passes; ++p) {
        if (len > 0) {
            TS s = 0;
            for (int x = -1 - r; x <= -1 + r; ++x) s += bl[x + (x >> LG)];
#pragma unroll
            for (int q = 0; q < C; ++q) {
                if (q < len) {
                    const int xa = q + r, xs = q - r - 1;
                    s += bl[xa + (xa >> LG)] - bl[xs + (xs >> LG)];
                    out[q] = s;
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < C; ++q)
            if (q < len) bl[q + (q >> LG)] = out[q];
        refresh_border();
    }
    for (int x = lane; x < W; x += 32) Y[base + x] = buf[slot(x)];
}

// Row passes with the window in registers, for whole rows of 32 C cells and a radius R
// known at compile time (R <= 16, R <= C). Lane l keeps E[0 .. C+2R]: cells
// l*C - R - 1 .. l*C + C + R - 1 of the pass's input, its own chunk at E[R+1 .. R+C].
// A pass fills the border -- the previous lane's last R+1 cells and the next lane's first
// R, by shuffles; the row's two ends reflect the lane's own cells -- then runs the window
// sum in registers, writing each output over the cell that just left the window, and
// shifts the outputs back into place. Shared memory carries only the row's load and
// store; the passes touch none, so a pass costs the L1 data pipe 2R+1 shuffles (two per
// 64-bit value) instead of a shared load for every cell that enters or leaves a window.
template <typename TS, int C, int R>
__global__ void __launch_bounds__(32 * kRowWarps)
    k_rowbox_shfl(const uint32_t* __restrict__ hist, int copies, TS* __restrict__ Y, int G,
                  int H, int passes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int W = 32 * C;
    constexpr int N = C + 2 * R + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    TS* buf = reinterpret_cast<TS*>(smem_raw) + (size_t)warp * (padded<C>(W) + 1);
    const int g = blockIdx.y;
    const int v = blockIdx.x * kRowWarps + warp;
    if (v >= H) return;
    const size_t base = ((size_t)g * H + v) * W;
    const size_t stride_copy = (size_t)G * H * W;
    // the row (copies summed) into shared memory, coalesced; then each lane's chunk
    const uint4* h0 = reinterpret_cast<const uint4*>(hist + base);
#pragma unroll
    for (int it = 0; it < C / 4; ++it) {
        const int x4 = lane + 32 * it;
        uint4 u = __ldg(h0 + x4);
        for (int k = 1; k < copies; ++k) {
            const uint4 w = __ldg(reinterpret_cast<const uint4*>(hist + k * stride_copy + base) + x4);
            u.x += w.x;
            u.y += w.y;
            u.z += w.z;
            u.w += w.w;
        }
        const int x = 4 * x4;
        buf[padded<C>(x)] = (TS)u.x;
        buf[padded<C>(x + 1)] = (TS)u.y;
        buf[padded<C>(x + 2)] = (TS)u.z;
        buf[padded<C>(x + 3)] = (TS)u.w;
    }
    __syncwarp();
    TS E[N];
    const TS* mine = buf + padded<C>(lane * C);
#pragma unroll
    for (int q = 0; q < C; ++q) E[R + 1 + q] = mine[q];
    box_passes_shfl<TS, C, R>(E, lane, passes);
    __syncwarp();
    TS* own = buf + padded<C>(lane * C);
#pragma unroll
    for (int q = 0; q < C; ++q) own[q] = E[R + 1 + q];
    __syncwarp();
    for (int x = lane; x < W; x += 32) Y[base + x] = buf[padded<C>(x)];
}

// The shuffle row pass exists for whole rows of 512 or 1024 cells and radii below the
// lane's chunk, up to 16.
inline bool rowbox_shfl_fits(int W, int r) {
    return (W == 512 && r >= 1 && r <= 15) || (W == 1024 && r >= 1 && r <= 16);
}

template <typename TS, int C, int R>
cudaError_t rowbox_shfl_launch(const FilterArgs& a, cudaStream_t st) {
    const size_t smem = (size_t)kRowWarps * (padded<C>(32 * C) + 1) * sizeof(TS);
    auto kern = k_rowbox_shfl<TS, C, R>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    dim3 grid((unsigned)((a.H + kRowWarps - 1) / kRowWarps), (unsigned)a.G);
    kern<<<grid, 32 * kRowWarps, smem, st>>>(a.hist, a.hist_copies < 1 ? 1 : a.hist_copies,
                                              static_cast<TS*>(a.Y), a.G, a.H, a.passes);
    return cudaGetLastError();
}

// Dispatch on the radius: R runs from RMAX down to 1.
template <typename TS, int C, int R>
cudaError_t rowbox_shfl_r(const FilterArgs& a, cudaStream_t st) {
    if constexpr (R < 1) {
        return cudaErrorInvalidValue;
    } else {
        if (a.r == R) return rowbox_shfl_launch<TS, C, R>(a, st);
        return rowbox_shfl_r<TS, C, R - 1>(a, st);
    }
}

template <typename TS>
cudaError_t rowbox_shfl_t(const FilterArgs& a, cudaStream_t st) {
    if (!rowbox_shfl_fits(a.W, a.r) || (a.W & 3)) return cudaErrorInvalidValue;
    return a.W == 1024 ? rowbox_shfl_r<TS, 32, 16>(a, st) : rowbox_shfl_r<TS, 16, 15>(a, st);
}

// border width of the register row pass: r + 1 rounded up to a whole chunk
inline int row_halo(int r, int C) { return (r + 1 + C - 1) / C * C; }

template <typename TS, int C>
cudaError_t rowbox_reg_t(const FilterArgs& a, cudaStream_t st) {
    const int halo = row_halo(a.r, C);
    const size_t smem = (size_t)kRowWarps * (padded<C>(a.W + 2 * halo) + 1) * sizeof(TS);
    auto kern = k_rowbox_reg<TS, C>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    dim3 grid((unsigned)((a.H + kRowWarps - 1) / kRowWarps), (unsigned)a.G);
    kern<<<grid, 32 * kRowWarps, smem, st>>>(a.hist, a.hist_copies < 1 ? 1 : a.hist_copies,
                                              static_cast<TS*>(a.Y), a.G, a.H, a.W, a.r,
                                              a.passes, halo);
    return cudaGetLastError();
}

// --------------------------------------------------------------- column passes
// One CTA per strip of STRIP columns of one layer, the whole column height in
// shared memory with a border of `halo` >= r + 1 rows on each side holding the
// reflected rows (refreshed after every pass), so every window reads its rows
// directly. Thread (j, ch) owns column j and the 16-row chunk ch; its 16 outputs of
// a pass stay in registers until the whole CTA has read the pass's input. A pad row
// after every chunk spreads the chunks over the banks. The strip narrows (8, 4, 2
// columns) as the height grows so that a CTA keeps its threads and the strip fits
// in shared memory.
constexpr int kChunk = 16;
constexpr int kColThreads = 512;

// border rows of the column pass: r + 1 rounded up to a whole chunk
inline int col_halo(int r) { return (r + 1 + kChunk - 1) / kChunk * kChunk; }
inline size_t colbox_smem(int H, int r, int strip, int sum_bytes) {
    const int rows = H + 2 * col_halo(r);
    return (size_t)(rows + rows / kChunk + 1) * strip * sum_bytes;
}

template <typename TS, int STRIP>
__global__ void __launch_bounds__(kColThreads)
    k_colbox(const TS* __restrict__ Y, TS* __restrict__ S, int G, int H, int W, int r,
             int passes, int halo) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TS* buf = reinterpret_cast<TS*>(smem_raw);
    const int g = blockIdx.y;
    const int x0 = blockIdx.x * STRIP;
    const int j = threadIdx.x % STRIP, ch = threadIdx.x / STRIP;
    const size_t lay = (size_t)g * H * W;
    // row t (t in [-halo, H + halo)) of the strip starts at element prow(t) * STRIP
    auto prow = [&](int t) { const int k = t + halo; return k + k / kChunk; };
    // the strip's rows are copied asynchronously straight into shared memory, all in
    // flight at once: 16-byte pieces when rows and strips are 16-byte aligned, else one
    // element per copy; columns past the width are zero-filled
    constexpr int kPiece = 16 / (int)sizeof(TS);
    constexpr int kPer = STRIP % kPiece == 0 ? STRIP / kPiece : 1;  // pieces per row of the strip
    if (STRIP % kPiece == 0 && W % kPiece == 0) {
        for (int idx = threadIdx.x; idx < H * kPer; idx += blockDim.x) {
            const int row = idx / kPer, col = (idx % kPer) * kPiece, x = x0 + col;
            const unsigned dst = (unsigned)__cvta_generic_to_shared(buf + prow(row) * STRIP + col);
            const TS* src = Y + lay + (size_t)row * W + (x < W ? x : 0);
            const int bytes = x < W ? 16 : 0;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                         "r"(bytes));
        }
    } else {
        for (int idx = threadIdx.x; idx < H * STRIP; idx += blockDim.x) {
            const int row = idx / STRIP, col = idx % STRIP, x = x0 + col;
            const unsigned dst = (unsigned)__cvta_generic_to_shared(buf + prow(row) * STRIP + col);
            const TS* src = Y + lay + (size_t)row * W + (x < W ? x : 0);
            const int bytes = x < W ? (int)sizeof(TS) : 0;
            if constexpr (sizeof(TS) == 8)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src),
                             "r"(bytes));
            else
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src),
                             "r"(bytes));
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    // the reflected border: rows -r-1 .. -1 and H .. H+r of every column of the strip
    auto refresh_border = [&]() {
        __syncthreads();
        for (int k = threadIdx.x; k < 2 * (r + 1) * STRIP; k += blockDim.x) {
            const int e = k / STRIP, c = k % STRIP;
            const int t = e <= r ? -1 - e : H + (e - r - 1);
            buf[prow(t) * STRIP + c] = buf[prow(reflect_index(t, H)) * STRIP + c];
        }
        __syncthreads();
    };
    refresh_border();
    const int i0 = ch * kChunk;
    const int len = max(0, min(kChunk, H - i0));
    // row i0 + x of column j: col[(x + floor(x / 16)) * STRIP] (i0 + halo is a whole chunk)
    TS* col = buf + (size_t)prow(i0) * STRIP + j;
    TS out[kChunk];
    for (int p = 0; p < passes; ++p) {
        if (len > 0) {
            TS s = 0;
            for (int x = -1 - r; x <= -1 + r; ++x) s += col[(x + (x >> 4)) * STRIP];
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                if (q < len) {
                    const int xa = q + r, xs = q - r - 1;
                    s += col[(xa + (xa >> 4)) * STRIP] - col[(xs + (xs >> 4)) * STRIP];
                    out[q] = s;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kChunk; ++q)
            if (q < len) col[q * STRIP] = out[q];
        refresh_border();
    }
    for (int idx = threadIdx.x; idx < H * STRIP; idx += blockDim.x) {
        int row = idx / STRIP, c = idx % STRIP, x = x0 + c;
        if (x < W) S[lay + (size_t)row * W + x] = buf[prow(row) * STRIP + c];
    }
}

// --------------------------------------------- column passes, TMA-staged strips
// The same passes on strips of 16 columns staged by the tensor memory accelerator:
// one thread issues a 2D box copy (16 columns x 16 rows) per chunk of the strip, the
// CTA waits for the bytes on an mbarrier. A row of the strip is 16 columns wide (128 B
// for 64-bit sums), so a warp -- 16 columns of 2 chunks -- reads one row of each chunk
// without bank conflicts, and the rows need no padding (every box lands 128-byte
// aligned). 1024 threads cover 64 chunks: heights up to 1024.
constexpr int kTmaStrip = 16;
constexpr int kTmaThreads = kTmaStrip * 64;
constexpr unsigned kTmaWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Wait (bounded) for phase `parity` of the mbarrier at shared address `bar`.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned limit) {
    for (unsigned it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n"
            " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

inline int tma_halo(int r) { return (r + 1 + kChunk - 1) / kChunk * kChunk; }
inline size_t colbox_tma_smem(int H, int r, int sum_bytes) {
    // the strip with its border rows, 128 bytes of alignment slack, the mbarrier
    return (size_t)(H + 2 * tma_halo(r)) * kTmaStrip * sum_bytes + 128 + 16;
}

template <typename TS>
__global__ void __launch_bounds__(kTmaThreads)
    k_colbox_tma(const __grid_constant__ CUtensorMap ymap, TS* __restrict__ S, int G, int H,
                 int W, int r, int passes, int halo, int32_t* err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    TS* buf = reinterpret_cast<TS*>(base);  // row t (t in [-halo, H + halo)): buf[(halo + t) * 16]
    const int rows = H + 2 * halo;
    const uint32_t bar = smem_u32(base + (size_t)rows * kTmaStrip * sizeof(TS));
    const int g = blockIdx.y, x0 = blockIdx.x * kTmaStrip;
    const int j = threadIdx.x % kTmaStrip, ch = threadIdx.x / kTmaStrip;
    const int nch = (H + kChunk - 1) / kChunk;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // every box is counted whole, rows past the height included (they arrive zero-filled
        // and land in the border, which is rewritten below)
        const uint32_t bytes = (uint32_t)(nch * kChunk * kTmaStrip * sizeof(TS));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                     : "memory");
        for (int c = 0; c < nch; ++c) {
            const uint32_t dst = smem_u32(buf + (size_t)(halo + kChunk * c) * kTmaStrip);
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
                "l"(reinterpret_cast<uint64_t>(&ymap)), "r"(x0), "r"(kChunk * c), "r"(g), "r"(bar)
                : "memory");
        }
    }
    const bool ok = mbar_wait(bar, 0, kTmaWaitLimit);
    if (__syncthreads_or(!ok)) {
        // the copies did not land in time: report it, let any copy still in flight finish
        // (bounded again) before the CTA's shared memory is released, leave S untouched
        if (threadIdx.x == 0 && err) atomicExch(err, 2);
        mbar_wait(bar, 0, kTmaWaitLimit);
        return;
    }
    auto refresh_border = [&]() {
        __syncthreads();
        for (int k = threadIdx.x; k < 2 * (r + 1) * kTmaStrip; k += blockDim.x) {
            const int e = k / kTmaStrip, c = k % kTmaStrip;
            const int t = e <= r ? -1 - e : H + (e - r - 1);
            buf[(size_t)(halo + t) * kTmaStrip + c] =
                buf[(size_t)(halo + reflect_index(t, H)) * kTmaStrip + c];
        }
        __syncthreads();
    };
    refresh_border();
    const int i0 = ch * kChunk;
    const int len = max(0, min(kChunk, H - i0));
    TS* col = buf + (size_t)(halo + i0) * kTmaStrip + j;  // row i0 + x: col[x * 16]
    TS out[kChunk];
    for (int p = 0; p < passes; ++p) {
        if (len > 0) {
            TS s = 0;
            for (int x = -1 - r; x <= -1 + r; ++x) s += col[x * kTmaStrip];
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                if (q < len) {
                    s += col[(q + r) * kTmaStrip] - col[(q - r - 1) * kTmaStrip];
                    out[q] = s;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kChunk; ++q)
            if (q < len) col[q * kTmaStrip] = out[q];
        refresh_border();
    }
    const size_t lay = (size_t)g * H * W;
    for (int idx = threadIdx.x; idx < H * kTmaStrip; idx += blockDim.x) {
        const int row = idx / kTmaStrip, c = idx % kTmaStrip, x = x0 + c;
        if (x < W) S[lay + (size_t)row * W + x] = buf[(size_t)(halo + row) * kTmaStrip + c];
    }
}

// -------------------------------------------------------------- layer mixing
// Eq. 3 / Eq. 4 after smoothing: with alpha = p / q and B groups,
//   rho_l = (S_l - alpha / (B - 1) * sum_{b != l} S_b) / s^k
//         = ((q (B-1) + p) S_l - p T) / (q (B-1) s^k),  T = sum_b S_b,
// whose numerator is an exact int64; one rounding gives the stored density. A
// general interaction matrix (Eq. 3) gives rho_l = (sum_b num[l, b] S_b) / (den s^k),
// its numerator exact as well.
template <typename R>
__device__ __forceinline__ R to_rho(float v);
template <>
__device__ __forceinline__ float to_rho<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_rho<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __half to_rho<__half>(float v) { return __float2half_rn(v); }

// ------------------------------------------------ layer mix into the density quads
// The layer mix is computed straight into the quad map the gather side reads, with no
// density stack in between. A CTA takes a tile of kMqX x kMqY quads (quad (a, b), a in
// [-2, W], b in [-2, H]) of every layer. First one thread per cell of the tile's
// footprint -- cells a0 .. a0 + kMqX and b0 .. b0 + kMqY of the reflection-extended
// grid -- mixes all layers at its source cell (exact integer numerator, one rounding)
// into shared memory; then the tile's quads of every layer are assembled from there and
// written as whole vectors. The density stack itself is extracted from the quads only
// when fetched.
constexpr int kMqX = 32, kMqY = 8, kMqThreads = 256;
constexpr int kMqFX = kMqX + 1, kMqF = kMqFX * (kMqY + 1);

template <typename R>
__device__ __forceinline__ uint32_t pack2(R lo, R hi) {
    unsigned short l = *reinterpret_cast<unsigned short*>(&lo);
    unsigned short h = *reinterpret_cast<unsigned short*>(&hi);
    return (uint32_t)l | ((uint32_t)h << 16);
}

inline size_t mix_quads_smem(int G, bool matrix, int rho_bytes) {
    const size_t rho = ((size_t)G * kMqF * rho_bytes + 15) / 16 * 16;
    return rho + (matrix ? (size_t)G * G * sizeof(long long) : 0);
}

template <typename TS, typename R>
__global__ void __launch_bounds__(kMqThreads)
    k_mix_quads(const TS* __restrict__ S, R* __restrict__ quads, int G, int H, int W,
                int64_t mix_self, int64_t mix_all, const int64_t* __restrict__ mix, float den) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* s_rho = reinterpret_cast<R*>(smem_raw);  // [G][kMqF]
    long long* s_num = reinterpret_cast<long long*>(
        smem_raw + ((size_t)G * kMqF * sizeof(R) + 15) / 16 * 16);  // G x G (general matrix)
    const int tid = threadIdx.x;
    const int a0 = -2 + (int)blockIdx.x * kMqX, b0 = -2 + (int)blockIdx.y * kMqY;
    const int64_t C = (int64_t)H * W;
    if (mix)
        for (int k = tid; k < G * G; k += blockDim.x) s_num[k] = mix[k];
    __syncthreads();
    for (int f = tid; f < kMqF; f += blockDim.x) {
        // footprint cell -> its source cell (cells past the last quad are clamped onto it:
        // computed, never used)
        const int a = min(a0 + f % kMqFX, W + 1), b = min(b0 + f / kMqFX, H + 1);
        const int64_t c = (int64_t)reflect_index(b, H) * W + reflect_index(a, W);
        if (mix) {
            for (int l = 0; l < G; ++l) {
                long long acc = 0;
                for (int g = 0; g < G; ++g)
                    acc += s_num[l * G + g] * (long long)S[(size_t)g * C + c];
                s_rho[l * kMqF + f] = to_rho<R>(__fdiv_rn(__ll2float_rn(acc), den));
            }
        } else if (G == 1) {
            s_rho[f] = to_rho<R>(__fdiv_rn(__ll2float_rn((long long)S[c]), den));
        } else {
            long long T = 0;
            for (int g = 0; g < G; ++g) T += (long long)S[(size_t)g * C + c];
            for (int l = 0; l < G; ++l) {
                const long long num = mix_self * (long long)S[(size_t)l * C + c] - mix_all * T;
                s_rho[l * kMqF + f] = to_rho<R>(__fdiv_rn(__ll2float_rn(num), den));
            }
        }
    }
    __syncthreads();
    const int64_t Wq = W + kQuadPad, QC = Wq * (H + kQuadPad);
    for (int e = tid; e < G * kMqX * kMqY; e += blockDim.x) {
        const int l = e / (kMqX * kMqY), qq = e % (kMqX * kMqY);
        const int qx = qq % kMqX, qy = qq / kMqX;
        const int a = a0 + qx, b = b0 + qy;
        if (a > W || b > H) continue;
        const R* r = s_rho + l * kMqF + qy * kMqFX + qx;
        const R e00 = r[0], e10 = r[1], e01 = r[kMqFX], e11 = r[kMqFX + 1];
        const int64_t idx = (int64_t)l * QC + (int64_t)(b + 2) * Wq + (a + 2);
        if constexpr (sizeof(R) == 4) {
            reinterpret_cast<float4*>(quads)[idx] = make_float4(e00, e10, e01, e11);
        } else {
            reinterpret_cast<uint2*>(quads)[idx] = make_uint2(pack2(e00, e10), pack2(e01, e11));
        }
    }
}

template <typename TS, typename R>
cudaError_t mix_quads_t(const FilterArgs& a, cudaStream_t st) {
    dim3 grid((unsigned)((a.W + kQuadPad + kMqX - 1) / kMqX),
              (unsigned)((a.H + kQuadPad + kMqY - 1) / kMqY));
    const size_t smem = mix_quads_smem(a.G, a.mix != nullptr, (int)sizeof(R));
    auto kern = k_mix_quads<TS, R>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<grid, kMqThreads, smem, st>>>(static_cast<const TS*>(a.S), static_cast<R*>(a.quads),
                                         a.G, a.H, a.W, a.mix_self, a.mix_all, a.mix, a.den_f);
    return cudaGetLastError();
}

// The density stack from the quads: rho(g, v, u) is the first value of quad (u, v).
template <typename R>
__global__ void k_rho_from_quads(const R* __restrict__ quads, R* __restrict__ rho, int G, int H,
                                 int W) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t C = (int64_t)H * W;
    if (idx >= (int64_t)G * C) return;
    const int64_t g = idx / C, rem = idx % C;
    const int v = (int)(rem / W), u = (int)(rem % W);
    const int64_t Wq = W + kQuadPad, QC = Wq * (H + kQuadPad);
    rho[idx] = quads[(g * QC + (int64_t)(v + 2) * Wq + (u + 2)) * 4];
}

template <typename R>
cudaError_t rho_from_quads_t(const FilterArgs& a, cudaStream_t st) {
    const int64_t n = (int64_t)a.G * a.H * a.W;
    k_rho_from_quads<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        static_cast<const R*>(a.quads), static_cast<R*>(a.rho), a.G, a.H, a.W);
    return cudaGetLastError();
}

template <typename TS>
cudaError_t rowbox_t(const FilterArgs& a, cudaStream_t st) {
    const int c = (a.W + 31) / 32;
    const int pad = (c % 2 == 0) ? 1 : 2;
    // mode 3 (and the default where it fits): the window in registers, borders by shuffles
    if (a.row_mode == 3 || (a.row_mode == 0 && rowbox_shfl_fits(a.W, a.r)))
        return rowbox_shfl_t<TS>(a, st);
    if (a.row_mode != 2) {  // register-resident rows where a template exists for the width
        if (c == 32) return rowbox_reg_t<TS, 32>(a, st);
        if (c == 16) return rowbox_reg_t<TS, 16>(a, st);
        if (c == 8) return rowbox_reg_t<TS, 8>(a, st);
    }
    const size_t per_row = (size_t)2 * (a.W + 32 * pad) * sizeof(TS);
    size_t fit = (200u * 1024u) / per_row;
    int rows = (int)(fit < 4 ? fit : 4);
    if (rows < 1) return cudaErrorInvalidValue;
    size_t smem = per_row * rows;
    auto kern = k_rowbox<TS>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    dim3 grid((unsigned)((a.H + rows - 1) / rows), (unsigned)a.G);
    kern<<<grid, 32 * rows, smem, st>>>(a.hist, a.hist_copies < 1 ? 1 : a.hist_copies,
                                        static_cast<TS*>(a.Y), a.G, a.H, a.W, a.r, a.passes,
                                        rows, c, pad);
    return cudaGetLastError();
}

template <typename TS, int STRIP>
cudaError_t colbox_strip(const FilterArgs& a, cudaStream_t st) {
    const int nch = (a.H + kChunk - 1) / kChunk;
    if (STRIP * nch > kColThreads) return cudaErrorInvalidValue;
    const size_t smem = colbox_smem(a.H, a.r, STRIP, sizeof(TS));
    auto kern = k_colbox<TS, STRIP>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    dim3 grid((unsigned)((a.W + STRIP - 1) / STRIP), (unsigned)a.G);
    kern<<<grid, kColThreads, smem, st>>>(static_cast<const TS*>(a.Y), static_cast<TS*>(a.S),
                                          a.G, a.H, a.W, a.r, a.passes, col_halo(a.r));
    return cudaGetLastError();
}

// The driver's tensor-map encoder, fetched through the runtime once (null if unavailable).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder() {
    static const EncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Whether the TMA-staged strip applies: heights up to 1024 (64 chunks of 16 rows per CTA),
// rows of the tensor a multiple of 16 bytes, the strip in shared memory, an encoder.
bool colbox_tma_fits(int W, int H, int r, int sum_bytes) {
    return H >= 1 && H <= 64 * kChunk && ((size_t)W * sum_bytes) % 16 == 0 &&
           colbox_tma_smem(H, r, sum_bytes) <= (size_t)227 * 1024 && tensor_map_encoder();
}

template <typename TS>
cudaError_t colbox_tma_t(const FilterArgs& a, cudaStream_t st) {
    if (!colbox_tma_fits(a.W, a.H, a.r, (int)sizeof(TS)) || (reinterpret_cast<uintptr_t>(a.Y) & 15))
        return cudaErrorInvalidValue;
    // [G][H][W] of the sum type; boxes of 16 columns x 16 rows x 1 layer; columns past W and
    // rows past H arrive as zeros
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.G};
    const cuuint64_t strides[2] = {(cuuint64_t)a.W * sizeof(TS),
                                   (cuuint64_t)a.W * a.H * sizeof(TS)};
    const cuuint32_t box[3] = {(cuuint32_t)kTmaStrip, (cuuint32_t)kChunk, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult cr = tensor_map_encoder()(
        &map, sizeof(TS) == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 3u,
        const_cast<void*>(a.Y), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const size_t smem = colbox_tma_smem(a.H, a.r, sizeof(TS));
    auto kern = k_colbox_tma<TS>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    dim3 grid((unsigned)((a.W + kTmaStrip - 1) / kTmaStrip), (unsigned)a.G);
    kern<<<grid, kTmaThreads, smem, st>>>(map, static_cast<TS*>(a.S), a.G, a.H, a.W, a.r,
                                          a.passes, tma_halo(a.r), a.err_flag);
    return cudaGetLastError();
}

// Strip 16 is the TMA-staged pass, 8, 4 and 2 the strips copied by cp.async. By default
// the 8-column strip: two of its CTAs share an SM and overlap one's copy with the other's
// passes, where the TMA strip's one 1024-thread CTA per SM cannot (61 vs 71 us at
// 8 x 1024^2, int64); the autotuner may still pick the TMA strip for a graph.
template <typename TS>
cudaError_t colbox_t(const FilterArgs& a, cudaStream_t st) {
    const int strip = a.strip ? a.strip : (a.H <= 1024 ? 8 : a.H <= 2048 ? 4 : 2);
    if (strip == kTmaStrip) return colbox_tma_t<TS>(a, st);
    if (strip == 8) return colbox_strip<TS, 8>(a, st);
    if (strip == 4) return colbox_strip<TS, 4>(a, st);
    return colbox_strip<TS, 2>(a, st);
}

}  // namespace

bool rowbox_mode_valid(int mode, int W, int H, int r) {
    const int c = (W + 31) / 32;
    if (mode == 1) return c == 8 || c == 16 || c == 32;
    if (mode == 3) return rowbox_shfl_fits(W, r);
    if (mode == 4) return band_rows_fits(W, r) && band_rows_fits(H, r);
    return mode == 0 || mode == 2;
}

// Row mode 4, the banded path: both passes run the banded row kernel, the first writing
// the row-filtered stack transposed ([G][W][H]) into Y, the second filtering Y's rows
// (the columns) and writing them transposed back into S ([G][H][W]). Chosen by hand, by
// the autotuner, or by shape when both sides fit and the buffers are aligned for it.
static bool band_path(const FilterArgs& a) {
    if (a.row_mode == 4) return true;
    if (a.row_mode != 0 || !(band_rows_fits(a.W, a.r) && band_rows_fits(a.H, a.r))) return false;
    const int copies = a.hist_copies < 1 ? 1 : a.hist_copies;
    return copies <= 2 && (reinterpret_cast<uintptr_t>(a.hist) & 15) == 0 &&
           (copies == 1 || ((int64_t)a.G * a.H * a.W * 4) % 16 == 0) &&
           (reinterpret_cast<uintptr_t>(a.Y) & 15) == 0 && (reinterpret_cast<uintptr_t>(a.S) & 7) == 0;
}

bool colbox_strip_valid(int strip, int W, int H, int r, int sum_bytes) {
    if (strip == kTmaStrip) return colbox_tma_fits(W, H, r, sum_bytes);
    const int nch = (H + kChunk - 1) / kChunk;
    return (strip == 2 || strip == 4 || strip == 8) && strip * nch <= kColThreads &&
           colbox_smem(H, r, strip, sum_bytes) <= (size_t)227 * 1024;
}

bool filter_clears_hist(const FilterArgs& a) { return a.clear_hist && band_path(a); }

cudaError_t launch_rowbox(int sum_bits, const FilterArgs& a, cudaStream_t st) {
    if (band_path(a))
        return launch_band_rows(sum_bits, false, a.hist, a.hist_copies < 1 ? 1 : a.hist_copies,
                                (int64_t)a.G * a.H * a.W, a.Y, a.G, a.H, a.W, a.r, a.passes,
                                a.clear_hist ? const_cast<uint32_t*>(a.hist) : nullptr, st);
    return sum_bits == 32 ? rowbox_t<uint32_t>(a, st) : rowbox_t<unsigned long long>(a, st);
}

cudaError_t launch_colbox(int sum_bits, const FilterArgs& a, cudaStream_t st) {
    if (band_path(a))
        return launch_band_rows(sum_bits, true, a.Y, 1, 0, a.S, a.G, a.W, a.H, a.r, a.passes,
                                nullptr, st);
    return sum_bits == 32 ? colbox_t<uint32_t>(a, st) : colbox_t<unsigned long long>(a, st);
}

__global__ void k_fold_hist(uint32_t* hist, int64_t n, int copies) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t v = hist[i];
    for (int k = 1; k < copies; ++k) {
        v += hist[k * n + i];
        hist[k * n + i] = 0;
    }
    hist[i] = v;
}

// Ink of the drawing entering an iteration, from its histogram: cells where any group
// counts something, and the sum over groups of each group's occupied cells (their
// difference counts the cells that several groups share). Row it of `stats` gets both.
__global__ void k_ink(const uint32_t* __restrict__ hist, int64_t cells, int G, int copies,
                      unsigned long long* stats, const int32_t* iter, int32_t stats_cap) {
    const int it = *iter;
    if (it < 0 || it >= stats_cap) return;
    unsigned long long any = 0, per_group = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += stride) {
        int occ = 0;
        for (int g = 0; g < G; ++g) {
            uint32_t v = 0;
            for (int k = 0; k < copies; ++k) v |= __ldg(hist + ((int64_t)k * G + g) * cells + i);
            occ += v != 0;
        }
        any += occ != 0;
        per_group += occ;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        any += __shfl_xor_sync(0xffffffffu, any, o);
        per_group += __shfl_xor_sync(0xffffffffu, per_group, o);
    }
    if ((threadIdx.x & 31) == 0 && (any | per_group)) {
        atomicAdd(stats + 2 * (int64_t)it, any);
        atomicAdd(stats + 2 * (int64_t)it + 1, per_group);
    }
}

cudaError_t launch_ink(const uint32_t* hist, int64_t cells, int G, int copies,
                       unsigned long long* stats, const int32_t* iter, int32_t stats_cap,
                       int n_sm, cudaStream_t st) {
    const int64_t want = (cells + 255) / 256;
    const int blocks = (int)(want < 4 * n_sm ? want : 4 * n_sm);
    k_ink<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(hist, cells, G, copies, stats, iter, stats_cap);
    return cudaGetLastError();
}

cudaError_t launch_fold_hist(uint32_t* hist, int64_t n, int copies, cudaStream_t st) {
    if (copies <= 1 || n <= 0) return cudaSuccess;
    k_fold_hist<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(hist, n, copies);
    return cudaGetLastError();
}

cudaError_t launch_mix_quads(int sum_bits, int rho_dtype, const FilterArgs& a, cudaStream_t st) {
    if (sum_bits == 32) {
        switch (rho_dtype) {
            case 0: return mix_quads_t<uint32_t, float>(a, st);
            case 1: return mix_quads_t<uint32_t, __nv_bfloat16>(a, st);
            case 2: return mix_quads_t<uint32_t, __half>(a, st);
        }
    } else {
        switch (rho_dtype) {
            case 0: return mix_quads_t<unsigned long long, float>(a, st);
            case 1: return mix_quads_t<unsigned long long, __nv_bfloat16>(a, st);
            case 2: return mix_quads_t<unsigned long long, __half>(a, st);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rho_from_quads(int rho_dtype, const FilterArgs& a, cudaStream_t st) {
    switch (rho_dtype) {
        case 0: return rho_from_quads_t<float>(a, st);
        case 1: return rho_from_quads_t<__nv_bfloat16>(a, st);
        case 2: return rho_from_quads_t<__half>(a, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace heb
