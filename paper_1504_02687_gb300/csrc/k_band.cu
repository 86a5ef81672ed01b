// Banded row passes: the k passes of the (2r+1)-wide box filter of Sec. 3.1 along
// every row of a [G][NR][L] stack, the result written transposed, [G][L][NR].
//
// Two runs make the whole separable (2r+1)^2 box filter, k times over: one over the
// histogram's rows (y-major, rows of W cells; its result is x-major) and one over
// that result's rows (x-major, rows of H cells, i.e. the columns; written transposed,
// the sums come back y-major). With half-sample reflection on each axis the row and
// column passes commute, so this order gives the same sums as any other. Both runs
// stream the same way and touch DRAM once per value in each direction: the column
// pass needs neither a strip of whole columns in shared memory nor a window read
// from it per cell.
//
// A CTA of kBandRows warps owns bands of kBandRows consecutive rows of one layer (warp
// w: row v0 + w), bands b = blockIdx.x, blockIdx.x + gridDim.x, ... (a persistent grid
// sized to the SMs). The rows of the next bands are in flight (cp.async, 16-byte
// pieces) while the current band is filtered: a ring of kBandStages shared-memory
// stages. A row sits in its stage with 16 bytes of padding after every lane's chunk,
// so the lanes reading their own chunks as 16-byte vectors hit distinct banks. The
// passes run in registers (box_passes_shfl). The outputs go back into the band's
// stage in transposed order, [x][band rows] with one pad element after every chunk,
// and leave as kBandRows consecutive values per x (64-byte segments for 8 rows of
// 64-bit sums).
#include <algorithm>
#include <cstdint>

#include "box.cuh"
#include "internal.cuh"

namespace heb {
namespace {

constexpr int kBandRows = 8;
constexpr int kBandThreads = 32 * kBandRows;
constexpr int kBandStages = 2;

template <typename TIn, int C>
struct BandLayout {
    static constexpr int L = 32 * C;                 // cells per row
    static constexpr int P = 16 / (int)sizeof(TIn);  // pad elements after each chunk
    static constexpr int RS = L + 32 * P;            // padded row stride, elements
};

// Bytes of one stage: the band's input rows (every copy), or its transposed outputs.
template <typename TIn, typename TS, int C>
size_t band_stage_bytes(int copies) {
    using Lay = BandLayout<TIn, C>;
    const size_t in = (size_t)kBandRows * copies * Lay::RS * sizeof(TIn);
    const size_t out = ((size_t)Lay::L * kBandRows + 32) * sizeof(TS);
    const size_t b = in > out ? in : out;
    return (b + 127) / 128 * 128;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The lane's chunk of one staged row (its copies summed) into E[R+1 .. R+C].
template <typename TIn, typename TS, int C, int R>
__device__ __forceinline__ void load_chunk(TS (&E)[C + 2 * R + 1], const TIn* row, int copies,
                                           int lane) {
    using Lay = BandLayout<TIn, C>;
    const TIn* base = row + lane * (C + Lay::P);
    if constexpr (sizeof(TIn) == 4) {
#pragma unroll
        for (int j = 0; j < C / 4; ++j) {
            uint4 u = *reinterpret_cast<const uint4*>(base + 4 * j);
            for (int k = 1; k < copies; ++k) {
                const uint4 w = *reinterpret_cast<const uint4*>(base + k * Lay::RS + 4 * j);
                u.x += w.x;
                u.y += w.y;
                u.z += w.z;
                u.w += w.w;
            }
            E[R + 1 + 4 * j] = (TS)u.x;
            E[R + 2 + 4 * j] = (TS)u.y;
            E[R + 3 + 4 * j] = (TS)u.z;
            E[R + 4 + 4 * j] = (TS)u.w;
        }
    } else {  // 64-bit sums from the first run, one copy
#pragma unroll
        for (int j = 0; j < C / 2; ++j) {
            const ulonglong2 u = *reinterpret_cast<const ulonglong2*>(base + 2 * j);
            E[R + 1 + 2 * j] = (TS)u.x;
            E[R + 2 + 2 * j] = (TS)u.y;
        }
    }
}

// in: copy k of row v of layer g at in + k * copy_stride + (g * NR + v) * L (the copies
// are summed); out: value x of row v of layer g at out + (g * L + x) * NR + v.
template <typename TIn, typename TS, int C, int R>
__global__ void __launch_bounds__(kBandThreads, 1)
    k_band_rows(const TIn* in, int copies, int64_t copy_stride, TS* __restrict__ out, int G,
                int NR, int passes, int stage_bytes, TIn* zero) {
    using Lay = BandLayout<TIn, C>;
    constexpr int L = Lay::L, P = Lay::P, RS = Lay::RS;
    constexpr int NS = kBandStages;
    constexpr int XS = kBandThreads / kBandRows;  // columns one sweep of the stores covers
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per_layer = (NR + kBandRows - 1) / kBandRows;
    const int nb = G * per_layer;
    auto stage = [&](int s) { return smem_raw + (size_t)s * stage_bytes; };
    // the copies of band b into stage s: one commit group per call (empty past the end)
    auto issue = [&](int b, int s) {
        if (b < nb) {
            const int g = b / per_layer, v0 = (b % per_layer) * kBandRows;
            const int nv = min(kBandRows, NR - v0);
            const TIn* src0 = in + ((int64_t)g * NR + v0) * L;
            TIn* dst = reinterpret_cast<TIn*>(stage(s));
            constexpr int units = L / P;  // 16-byte pieces per row
            for (int i = 0; i < nv; ++i)
                for (int cp = 0; cp < copies; ++cp) {
                    const TIn* src = src0 + cp * copy_stride + (int64_t)i * L;
                    TIn* d = dst + (i * copies + cp) * RS;
#pragma unroll
                    for (int u = threadIdx.x; u < units; u += kBandThreads)
                        cp_async16(d + u * P + (u * P / C) * P, src + u * P);
                }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) issue(blockIdx.x + s * gridDim.x, s);
    int s = 0;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        issue(b + (NS - 1) * gridDim.x, s == 0 ? NS - 1 : s - 1);
        cp_async_wait<NS - 1>();  // this thread's copies of band b have landed
        __syncthreads();          // ... and every thread's
        const int g = b / per_layer, v0 = (b % per_layer) * kBandRows;
        const int nv = min(kBandRows, NR - v0);
        const bool mine = warp < nv;
        if (zero) {  // the band's rows have landed in shared memory: clear them in `zero`
            for (int i = 0; i < nv; ++i)
                for (int cp = 0; cp < copies; ++cp) {
                    uint4* z = reinterpret_cast<uint4*>(zero + cp * copy_stride +
                                                        ((int64_t)g * NR + v0 + i) * L);
#pragma unroll
                    for (int u = threadIdx.x; u < L / P; u += kBandThreads) z[u] = make_uint4(0, 0, 0, 0);
                }
        }
        TS E[C + 2 * R + 1];
        if (mine)
            load_chunk<TIn, TS, C, R>(E, reinterpret_cast<const TIn*>(stage(s)) + warp * copies * RS,
                                      copies, lane);
        __syncthreads();  // the stage is read: it takes the outputs
        TS* T = reinterpret_cast<TS*>(stage(s));
        if (mine) {
            box_passes_shfl<TS, C, R>(E, lane, passes);
            // cell x = lane * C + q of row `warp` at T[x * kBandRows + warp + x / C]
#pragma unroll
            for (int q = 0; q < C; ++q) T[(lane * C + q) * kBandRows + warp + lane] = E[R + 1 + q];
        }
        __syncthreads();
        // thread t stores row t % kBandRows of columns t / kBandRows + XS * k: a warp writes
        // segments of kBandRows consecutive values
        const int i = threadIdx.x % kBandRows;
        if (i < nv) {
            int x = threadIdx.x / kBandRows;
            TS* op = out + ((int64_t)g * L + x) * NR + v0 + i;
            const int64_t step = (int64_t)XS * NR;
#pragma unroll 4
            for (int k = 0; k < L / XS; ++k, x += XS, op += step) *op = T[x * kBandRows + i + x / C];
        }
        __syncthreads();  // the stage is free for the copies issued next
        s = s + 1 == NS ? 0 : s + 1;
    }
    cp_async_wait<0>();
}

template <typename TIn, typename TS, int C, int R>
cudaError_t band_launch(const void* in, int copies, int64_t copy_stride, void* out, int G, int NR,
                        int passes, void* zero, cudaStream_t st) {
    const size_t sb = band_stage_bytes<TIn, TS, C>(copies);
    const size_t smem = kBandStages * sb;
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    auto kern = k_band_rows<TIn, TS, C, R>;
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBandThreads, smem);
    if (err != cudaSuccess) return err;
    const int64_t nb = (int64_t)G * ((NR + kBandRows - 1) / kBandRows);
    const int64_t grid = std::min<int64_t>(nb, (int64_t)n_sm * std::max(per_sm, 1));
    if (grid <= 0) return cudaSuccess;
    kern<<<(unsigned)grid, kBandThreads, smem, st>>>(static_cast<const TIn*>(in), copies,
                                                      copy_stride, static_cast<TS*>(out), G, NR,
                                                      passes, (int)sb, static_cast<TIn*>(zero));
    return cudaGetLastError();
}

// Dispatch on the radius: R runs from RMAX down to 1.
template <typename TIn, typename TS, int C, int R>
cudaError_t band_r(int r, const void* in, int copies, int64_t copy_stride, void* out, int G,
                   int NR, int passes, void* zero, cudaStream_t st) {
    if constexpr (R < 1) {
        return cudaErrorInvalidValue;
    } else {
        if (r == R)
            return band_launch<TIn, TS, C, R>(in, copies, copy_stride, out, G, NR, passes, zero, st);
        return band_r<TIn, TS, C, R - 1>(r, in, copies, copy_stride, out, G, NR, passes, zero, st);
    }
}

template <typename TIn, typename TS>
cudaError_t band_t(int L, int r, const void* in, int copies, int64_t copy_stride, void* out, int G,
                   int NR, int passes, void* zero, cudaStream_t st) {
    if (L == 1024)
        return band_r<TIn, TS, 32, 16>(r, in, copies, copy_stride, out, G, NR, passes, zero, st);
    return band_r<TIn, TS, 16, 15>(r, in, copies, copy_stride, out, G, NR, passes, zero, st);
}

}  // namespace

bool band_rows_fits(int L, int r) {
    return (L == 512 && r >= 1 && r <= 15) || (L == 1024 && r >= 1 && r <= 16);
}

cudaError_t launch_band_rows(int sum_bits, bool sum_input, const void* in, int copies,
                             int64_t copy_stride, void* out, int G, int NR, int L, int r,
                             int passes, uint32_t* zero, cudaStream_t st) {
    if (!band_rows_fits(L, r) || copies < 1 || copies > 2 || NR < 1 || G < 1 ||
        (copies > 1 && (copy_stride * 4) % 16 != 0) ||
        (reinterpret_cast<uintptr_t>(in) & 15) != 0 || (reinterpret_cast<uintptr_t>(out) & 7) != 0 ||
        (zero && (sum_input || zero != in)))
        return cudaErrorInvalidValue;
    if (sum_bits == 32)  // 32-bit sums: the histogram and the first run's result are both 32-bit
        return band_t<uint32_t, uint32_t>(L, r, in, copies, copy_stride, out, G, NR, passes, zero, st);
    if (sum_input)
        return band_t<unsigned long long, unsigned long long>(L, r, in, copies, copy_stride, out, G,
                                                               NR, passes, nullptr, st);
    return band_t<uint32_t, unsigned long long>(L, r, in, copies, copy_stride, out, G, NR, passes,
                                                zero, st);
}

}  // namespace heb
