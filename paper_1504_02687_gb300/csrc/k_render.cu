// Headless rendering of the bundled drawing (Sec. 3.4): every polyline segment is
// drawn as a capsule whose width follows the density at its two sample points,
// coloured by the edge's bin, and overlapping edges accumulate opacity.
//
// Accumulation is order-free: each covered pixel adds the edge's integer optical
// depth tau_e to its bin's depth map with one 64-bit atomic, so the maps do not
// depend on launch order; one resolve pass sums the bins per pixel (depth and
// depth-weighted colour) and turns them into RGBA8 (opacity 1 - exp(-sum tau),
// the colour a tau-weighted mean, composited over the background).
#include "density.cuh"

namespace heb {
namespace {

// Largest density of the stack (non-negative part) as float bits: a max over
// non-negative floats is a max over their bit patterns.
template <typename T>
__global__ void k_rho_max(const T* __restrict__ rho, int64_t n, unsigned int* out) {
    float m = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        m = fmaxf(m, (float)rho[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(out, __float_as_uint(m));
}

// One block per block of eb slots (the point layout of the iteration); its
// threads take the block's segments in turn and loop over each capsule's
// bounding box.
template <typename T>
__global__ void __launch_bounds__(256) k_render_frag(RenderArgs a) {
    __shared__ int s_cnt[kEdgesPerBlock];
    __shared__ int s_loc[kEdgesPerBlock + 1];
    __shared__ int s_wtot[32];
    const int tid = threadIdx.x;
    const int64_t e0 = (int64_t)blockIdx.x * a.eb;
    const int nb = (int)min((int64_t)a.eb, a.E - e0);
    const int64_t region = (int64_t)blockIdx.x * a.eb * a.cap;
    for (int i = tid; i < nb; i += blockDim.x) s_cnt[i] = a.cnt[e0 + i];
    __syncthreads();
    block_scan_excl(s_cnt, s_loc, nb, s_wtot);
    const float rho_ref = __uint_as_float(*a.rho_ref);
    const float inv_ref = rho_ref > 0.0f ? 1.0f / rho_ref : 0.0f;
    const int64_t QC = quad_elems(a.W, a.H);
    const float sc = (float)a.scale;
    const int total = s_loc[nb];
    for (int k = tid; k < total; k += blockDim.x) {
        int lo = 0, hi = nb - 1;  // polyline of point k: the last i with s_loc[i] <= k
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_loc[mid] <= k) lo = mid; else hi = mid - 1;
        }
        const int i = lo, j = k - s_loc[i], n = s_cnt[i];
        if (j + 1 >= n) continue;
        const int g = a.group[e0 + i];
        const unsigned long long tau = (unsigned long long)a.weight[e0 + i] * a.tau1;
        if (tau == 0) continue;
        const bool last = j + 2 == n;
        const float2 P = a.pts[region + s_loc[i] + j], Pn = a.pts[region + s_loc[i] + j + 1];
        const T* Q = static_cast<const T*>(a.quads) + (int64_t)g * QC * 4;
        const float rb = 0.5f * (density_at(Q, a.W, a.H, P.x, P.y) +
                                 density_at(Q, a.W, a.H, Pn.x, Pn.y));
        float u = fminf(fmaxf(rb * inv_ref, 0.0f), 1.0f);
        if (a.log_width) u = log2f(1.0f + u);
        const float r = 0.5f * (a.width_min + (a.width_max - a.width_min) * u);
        const float r2 = r * r;
        const float ax = P.x * sc, ay = P.y * sc, bx = Pn.x * sc, by = Pn.y * sc;
        const float dx = bx - ax, dy = by - ay, L2 = dx * dx + dy * dy;
        const int x0 = max(0, (int)floorf(fminf(ax, bx) - r) - 1);
        const int x1 = min(a.Wi - 1, (int)ceilf(fmaxf(ax, bx) + r) + 1);
        const int y0 = max(0, (int)floorf(fminf(ay, by) - r) - 1);
        const int y1 = min(a.Hi - 1, (int)ceilf(fmaxf(ay, by) + r) + 1);
        unsigned long long* depth = a.depth + (int64_t)g * a.Hi * a.Wi;
        for (int py = y0; py <= y1; ++py) {
            const float ey = ay - ((float)py + 0.5f);
            for (int px = x0; px <= x1; ++px) {
                const float ex = ax - ((float)px + 0.5f);  // A - c
                const float t = L2 > 0.0f ? -(ex * dx + ey * dy) / L2 : 0.0f;
                if (!last && t >= 1.0f) continue;  // the next segment draws this pixel
                const float tc = fminf(fmaxf(t, 0.0f), 1.0f);
                const float qx = ex + tc * dx, qy = ey + tc * dy;
                if (qx * qx + qy * qy > r2) continue;
                atomicAdd(depth + (int64_t)py * a.Wi + px, tau);
            }
        }
    }
}

__global__ void k_render_resolve(const unsigned long long* __restrict__ depth, int G, int64_t n,
                                 const int32_t* __restrict__ palette, uchar4 bg,
                                 uchar4* __restrict__ rgba, unsigned long long* accum) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long t = 0, cr = 0, cg = 0, cb = 0;
    for (int g = 0; g < G; ++g) {
        const unsigned long long d = depth[(int64_t)g * n + i];
        t += d;
        cr += d * (unsigned)palette[3 * g];
        cg += d * (unsigned)palette[3 * g + 1];
        cb += d * (unsigned)palette[3 * g + 2];
    }
    if (accum) {
        reinterpret_cast<ulonglong2*>(accum)[2 * i] = make_ulonglong2(t, cr);
        reinterpret_cast<ulonglong2*>(accum)[2 * i + 1] = make_ulonglong2(cg, cb);
    }
    const float A = t ? 1.0f - expf(-(float)t * (1.0f / 1048576.0f)) : 0.0f;
    const float inv = t ? 1.0f / (float)t : 0.0f;
    const float c[3] = {(float)cr * inv, (float)cg * inv, (float)cb * inv};
    const float b[3] = {(float)bg.x, (float)bg.y, (float)bg.z};
    unsigned char o[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float v = A * c[k] + (1.0f - A) * b[k];
        o[k] = (unsigned char)fminf(255.0f, fmaxf(0.0f, floorf(v + 0.5f)));
    }
    rgba[i] = make_uchar4(o[0], o[1], o[2], 255);
}

template <typename T>
cudaError_t render_t(const RenderArgs& a, const void* rho, int64_t rho_n, bool want_max,
                     int n_sm, cudaStream_t st) {
    if (want_max) {
        int64_t blocks = (rho_n + 255) / 256;
        if (blocks > (int64_t)4 * n_sm) blocks = (int64_t)4 * n_sm;
        if (blocks < 1) blocks = 1;
        k_rho_max<T><<<(unsigned)blocks, 256, 0, st>>>(
            static_cast<const T*>(rho), rho_n, a.rho_ref);
    }
    const int64_t nblk = (a.E + a.eb - 1) / a.eb;
    if (nblk > 0) k_render_frag<T><<<(unsigned)nblk, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_render(int rho_dtype, const RenderArgs& a, const void* rho, int64_t rho_n,
                          bool want_max, int n_sm, cudaStream_t st) {
    switch (rho_dtype) {
        case 0: return render_t<float>(a, rho, rho_n, want_max, n_sm, st);
        case 1: return render_t<__nv_bfloat16>(a, rho, rho_n, want_max, n_sm, st);
        case 2: return render_t<__half>(a, rho, rho_n, want_max, n_sm, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_render_resolve(const unsigned long long* depth, int G, int64_t n_pixels,
                                  const int32_t* palette, const unsigned char* bg, void* rgba,
                                  void* accum, cudaStream_t st) {
    if (n_pixels <= 0) return cudaSuccess;
    k_render_resolve<<<(unsigned)((n_pixels + 255) / 256), 256, 0, st>>>(
        depth, G, n_pixels, palette, make_uchar4(bg[0], bg[1], bg[2], 255),
        static_cast<uchar4*>(rgba), static_cast<unsigned long long*>(accum));
    return cudaGetLastError();
}

}  // namespace heb
