// Device helpers shared by the point-side kernels (advection, resampling) and the
// renderer: density quad loads, the cell frame of a position, bilinear density,
// the drawing-area clamp and a block-wide exclusive scan.
#pragma once

#include "internal.cuh"

namespace heb {

// One density quad as four floats (see the quad map in internal.cuh).
template <typename T>
__device__ __forceinline__ float4 load_quad(const T* Q, int64_t i);
template <>
__device__ __forceinline__ float4 load_quad<float>(const float* Q, int64_t i) {
    return __ldg(reinterpret_cast<const float4*>(Q) + i);
}
template <>
__device__ __forceinline__ float4 load_quad<__nv_bfloat16>(const __nv_bfloat16* Q, int64_t i) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(Q) + i);
    __nv_bfloat162 lo = *reinterpret_cast<__nv_bfloat162*>(&u.x);
    __nv_bfloat162 hi = *reinterpret_cast<__nv_bfloat162*>(&u.y);
    float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
    return make_float4(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ float4 load_quad<__half>(const __half* Q, int64_t i) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(Q) + i);
    __half2 lo = *reinterpret_cast<__half2*>(&u.x);
    __half2 hi = *reinterpret_cast<__half2*>(&u.y);
    float2 a = __half22float2(lo), b = __half22float2(hi);
    return make_float4(a.x, a.y, b.x, b.y);
}

// The same quads through the texture path: texel i of the 1D view is quad i (16-bit
// densities come back as their bit patterns).
template <typename T>
__device__ __forceinline__ float4 fetch_quad(unsigned long long tex, int64_t i);
template <>
__device__ __forceinline__ float4 fetch_quad<float>(unsigned long long tex, int64_t i) {
    return tex1Dfetch<float4>((cudaTextureObject_t)tex, (int)i);
}
template <>
__device__ __forceinline__ float4 fetch_quad<__nv_bfloat16>(unsigned long long tex, int64_t i) {
    const ushort4 u = tex1Dfetch<ushort4>((cudaTextureObject_t)tex, (int)i);
    return make_float4(__bfloat162float(__ushort_as_bfloat16(u.x)),
                       __bfloat162float(__ushort_as_bfloat16(u.y)),
                       __bfloat162float(__ushort_as_bfloat16(u.z)),
                       __bfloat162float(__ushort_as_bfloat16(u.w)));
}
template <>
__device__ __forceinline__ float4 fetch_quad<__half>(unsigned long long tex, int64_t i) {
    const ushort4 u = tex1Dfetch<ushort4>((cudaTextureObject_t)tex, (int)i);
    return make_float4(__half2float(__ushort_as_half(u.x)), __half2float(__ushort_as_half(u.y)),
                       __half2float(__ushort_as_half(u.z)), __half2float(__ushort_as_half(u.w)));
}

// One layer of the quad map as the gathers see it: through the texture view of the whole
// map (TEX) or through the load path (the kernel is compiled for one of the two).
template <typename T, bool TEX>
struct QuadMap {
    const T* q;              // the layer's quads
    unsigned long long tex;  // texture view of the whole map
    int64_t base;            // the layer's first quad in the texture view
    __device__ __forceinline__ float4 at(int64_t i) const {
        if constexpr (TEX) return fetch_quad<T>(tex, base + i);
        else return load_quad(q, i);
    }
};

__device__ __forceinline__ float lerp_rn(float a, float b, float f) {
    return __fmaf_rn(f, __fsub_rn(b, a), a);
}

// Cell frame of a position: cell centres sit at (a + 0.5, b + 0.5). Positions stay in
// [0, W - 2^-10]; the clamp keeps every quad index on the map regardless.
struct Frame {
    int a0, b0;
    float fu, fv;
};
__device__ __forceinline__ Frame frame_of(float x, float y, int W, int H) {
    float u = __fsub_rn(x, 0.5f), v = __fsub_rn(y, 0.5f);
    float fa = floorf(u), fb = floorf(v);
    Frame f;
    f.a0 = min(max((int)fa, -1), W - 1);
    f.b0 = min(max((int)fb, -1), H - 1);
    f.fu = __fsub_rn(u, fa);
    f.fv = __fsub_rn(v, fb);
    return f;
}

// Bilinear density of the 2x2 quad q at fractions (fu, fv).
__device__ __forceinline__ float bilinear(float4 q, float fu, float fv) {
    return lerp_rn(lerp_rn(q.x, q.y, fu), lerp_rn(q.z, q.w, fu), fv);
}

// Bilinear density of one layer's quad map at (x, y).
template <typename T>
__device__ __forceinline__ float density_at(const T* __restrict__ Q, int W, int H, float x,
                                            float y) {
    Frame f = frame_of(x, y, W, H);
    return bilinear(load_quad(Q, (int64_t)(f.b0 + 2) * (W + kQuadPad) + (f.a0 + 2)), f.fu, f.fv);
}
template <typename T, bool TEX>
__device__ __forceinline__ float density_at(const QuadMap<T, TEX>& m, int W, int H, float x,
                                            float y) {
    Frame f = frame_of(x, y, W, H);
    return bilinear(m.at((int64_t)(f.b0 + 2) * (W + kQuadPad) + (f.a0 + 2)), f.fu, f.fv);
}

__device__ __forceinline__ float clamp_pos(float v, int n) {
    float hi = __fsub_rn((float)n, kEdgeGuard);
    return fminf(fmaxf(v, 0.0f), hi);
}

// Exclusive scan of in[0..n) into out[0..n] (out[n] = total), n <= blockDim.x.
__device__ inline void block_scan_excl(const int* in, int* out, int n, int* warp_tot) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    int v = tid < n ? in[tid] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive warp prefix
    }
    __syncthreads();
    int base = wid > 0 ? warp_tot[wid - 1] : 0;
    if (tid < n) out[tid] = base + x - v;
    if (tid == n - 1) out[n] = base + x;
    if (n == 0 && tid == 0) out[0] = 0;
    __syncthreads();
}


}  // namespace heb
