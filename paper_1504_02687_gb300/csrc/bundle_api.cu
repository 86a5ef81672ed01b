// Host side of the C ABI declared in include/bundle.h: argument checks, the
// integer-width bounds, the world -> grid map, device buffers, the launch
// sequence of one bundling iteration and the fetches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <limits>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/bundle.h"
#include "internal.cuh"

using namespace heb;

struct bundle_ctx {
    bundle_params p{};
    int64_t E = 0;
    int32_t G = 1, W = 0, H = 0;
    int32_t cap = 0;
    int32_t eb = kMaxEdgesPerWarp;  // edges per block of the point layout (one warp each)
    int64_t n_blocks = 0;
    int32_t col_strip = 0;        // column-pass strip (0: by height), set by the autotuner
    int32_t row_mode = 0;         // row-pass variant (0: by width), set by the autotuner
    bool straight = false;        // points are the straight edges of bundle_init (2 per slot)
    int32_t sum_bits = 64;
    int64_t mix_self = 1, mix_all = 0;
    float den_f = 1.0f;
    double sum_bound = 0;        // worst-case smoothed sum (size_integers)
    int64_t* mix = nullptr;      // optional G x G interaction numerators (device)
    unsigned long long mass_allowed = 0;  // segment histogram: largest mass the sums can take
    int32_t* d_flag = nullptr;           // sticky overflow flag set on the device
    unsigned long long* ink = nullptr;   // [BUNDLE_INK_STATS_CAP][2] convergence record
    int n_sm = 0;
    double map[5] = {0, 0, 1, 0, 0};
    int32_t iteration = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // device state
    int32_t* perm = nullptr;      // slot -> caller edge index
    int32_t* group = nullptr;     // per slot
    int32_t* weight = nullptr;    // per slot
    int32_t* cnt[2] = {nullptr, nullptr};
    float2* pts[2] = {nullptr, nullptr};
    uint32_t* hist = nullptr;
    void* Y = nullptr;
    void* S = nullptr;
    void* rho = nullptr;
    void* quads = nullptr;   // [G][H+3][W+3] density quads
    cudaTextureObject_t qtex = 0;  // texture view of the quads (0 where it cannot be made)
    unsigned long long* counters = nullptr;  // [0] points splatted, [1] scratch sum, [2] segment mass
    int64_t* fetch_off = nullptr;
    int64_t* fetch_tmp = nullptr;
    float2* fetch_xy = nullptr;
    int64_t fetch_xy_cap = 0;
    int cur_P = 0;       // buffer holding the current polylines
    int cur_R = -1;      // buffer holding the last resampled polylines (-1: none yet)
    // split form (bundle_points_step / bundle_density_step): 0 no run open, 1 histogram of
    // the open iteration splatted (it may be replaced before the density stage), 2 density
    // of the open iteration built; split_R: buffer of the resampled polylines of the run
    int split_state = 0;
    int split_R = 0;
    bool have_density = false;
    int64_t device_bytes = 0;
    // device schedule of h and the graphs of one steady-state iteration (one per ping-pong
    // direction); launched instead of separate kernels when profiling is off
    float* h_sched = nullptr;
    int32_t h_cap = 0;
    int32_t* d_iter = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    bool use_graphs = true;
    // batch of independent graphs (bundle_init_batch): each member is a full context with
    // its own buffers and stream; a steady-state iteration of all members is one CUDA graph
    // with one branch per member
    std::vector<bundle_ctx*> members;
    bool is_member = false;
    cudaGraphExec_t bexec[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> bev;  // fork/join events
    // per-kernel event timing (bundle_profile_enable)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;  // kind of each recorded (start, stop) pair
    size_t ev_used = 0;        // events in use (2 per record)
    std::string err;
};

namespace {

thread_local std::string g_init_error;

}  // namespace

void heb::set_thread_error(const char* msg) { g_init_error = msg; }

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bundle_status fail(std::string* sink, bundle_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    *sink = buf;
    return s;
}

#define CUDA_TRY(sink, expr)                                                              \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(sink, e_ == cudaErrorMemoryAllocation ? BUNDLE_ENOMEM : BUNDLE_ECUDA, \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

template <typename T>
cudaError_t dalloc(bundle_ctx* c, T** ptr, size_t n) {
    *ptr = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), n * sizeof(T));
    if (e == cudaSuccess) c->device_bytes += (int64_t)(n * sizeof(T));
    return e;
}

void free_ctx(bundle_ctx* c) {
    if (!c) return;
    for (bundle_ctx* m : c->members) {
        m->is_member = false;
        free_ctx(m);
    }
    c->members.clear();
    if (c->device < 0) {
        delete c;
        return;
    }
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->qtex) cudaDestroyTextureObject(c->qtex);
    void* ptrs[] = {c->perm, c->group, c->weight, c->cnt[0], c->cnt[1], c->pts[0], c->pts[1],
                    c->hist, c->Y, c->S, c->rho, c->quads, c->mix, c->d_flag, c->ink, c->counters, c->fetch_off, c->fetch_tmp,
                    c->fetch_xy};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    for (cudaEvent_t ev : c->ev_pool) cudaEventDestroy(ev);
    for (cudaGraphExec_t g : c->gexec)
        if (g) cudaGraphExecDestroy(g);
    for (cudaGraphExec_t g : c->bexec)
        if (g) cudaGraphExecDestroy(g);
    for (cudaEvent_t ev : c->bev) cudaEventDestroy(ev);
    if (c->h_sched) cudaFree(c->h_sched);
    if (c->d_iter) cudaFree(c->d_iter);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int rho_bytes(int dtype) { return dtype == BUNDLE_RHO_F32 ? 4 : 2; }

// Kernel bandwidth of iteration i (Sec. 2.1, Sec. 3.3): h_i = lambda^i h_max,
// h_max = h_max_sigmas * sigma_k with sigma_k^2 = k r (r + 1) / 3, the variance
// of k box passes of width 2r+1.
double bandwidth(const bundle_params& p, int32_t i) {
    double sigma = std::sqrt((double)((int64_t)p.passes * p.radius * (p.radius + 1)) / 3.0);
    double h = p.h_max_sigmas * sigma;
    for (int32_t t = 0; t < i; ++t) h *= p.lambda;
    return h;
}

bundle_status check_params(const bundle_params& p, int32_t n_groups, std::string* e) {
    if (n_groups < 1 || n_groups > 64)
        return fail(e, BUNDLE_EINVAL, "n_groups must be in [1, 64], got %d", n_groups);
    if (p.radius < 1) return fail(e, BUNDLE_EINVAL, "radius must be >= 1, got %d", p.radius);
    if (p.passes < 1 || p.passes > 16)
        return fail(e, BUNDLE_EINVAL, "passes must be in [1, 16], got %d", p.passes);
    if (p.alpha_den <= 0 || p.alpha_num < 0)
        return fail(e, BUNDLE_EINVAL, "alpha must be p/q with p >= 0, q > 0");
    if (!(p.lambda > 0 && p.lambda <= 1) || !(p.h_max_sigmas > 0))
        return fail(e, BUNDLE_EINVAL, "need 0 < lambda <= 1 and h_max_sigmas > 0");
    if (p.n_fixed != 0 && (p.n_fixed < 2 || p.n_fixed > kMaxCap))
        return fail(e, BUNDLE_EINVAL, "n_fixed must be 0 or in [2, %d]", kMaxCap);
    if (p.n_fixed == 0 && (p.n_max < 2 || p.n_max > kMaxCap))
        return fail(e, BUNDLE_EINVAL, "n_max must be in [2, %d]", kMaxCap);
    if (p.n_fixed == 0 && !(p.delta_px > 0))
        return fail(e, BUNDLE_EINVAL, "delta_px must be > 0");
    if (!(p.laplace_beta >= 0 && p.laplace_beta <= 1))
        return fail(e, BUNDLE_EINVAL, "laplace_beta must be in [0, 1]");
    if (!(p.eps >= 0)) return fail(e, BUNDLE_EINVAL, "eps must be >= 0");
    if (p.step_tries < 1 || p.step_tries > 64)
        return fail(e, BUNDLE_EINVAL, "step_tries must be in [1, 64]");
    if (p.sum_bits != 0 && p.sum_bits != 32 && p.sum_bits != 64)
        return fail(e, BUNDLE_EINVAL, "sum_bits must be 0, 32 or 64");
    if (p.rho_dtype < 0 || p.rho_dtype > 2) return fail(e, BUNDLE_EINVAL, "bad rho_dtype");
    if (p.grid_dominant < 2 || p.grid_dominant > 4096)
        return fail(e, BUNDLE_EINVAL, "grid_dominant must be in [2, 4096]");
    if ((p.flags & ~(BUNDLE_FLAG_FIXED_STEP | BUNDLE_FLAG_SEGMENT_HIST |
                     BUNDLE_FLAG_INK_STATS | BUNDLE_FLAG_LOAD_GATHERS)) != 0)
        return fail(e, BUNDLE_EINVAL, "unknown bits in flags");
    if (!(p.directed_offset >= 0 && p.directed_offset < 0.25f))
        return fail(e, BUNDLE_EINVAL, "directed_offset must be in [0, 0.25)");
    return BUNDLE_OK;
}

// Integer widths (Eq. 1 histogram, Sec. 3.1 sums, Eq. 3-4 mix) from the
// worst case: M0 = sum_e w_e * cap points' weight. With reflection a cell can
// enter a window at most twice per axis, so after p passes every cell and
// every intermediate is at most 4 s^(p-1) M0, s = (2r+1)^2.
bundle_status size_integers(bundle_ctx* c, const int32_t* weight_host, std::string* e) {
    double M0 = 0;
    if (weight_host) {
        for (int64_t i = 0; i < c->E; ++i) {
            if (weight_host[i] < 0)
                return fail(e, BUNDLE_EINVAL, "weight[%lld] = %d is negative", (long long)i,
                            weight_host[i]);
            M0 += (double)weight_host[i];
        }
    } else {
        M0 = (double)c->E;
    }
    M0 *= c->cap;
    const double two31 = 2147483648.0, two63 = 9223372036854775808.0;
    if (M0 >= two31 * (1 - 1e-12))
        return fail(e, BUNDLE_EOVERFLOW,
                    "histogram bound sum(w)*cap = %.6g does not fit uint32 cells", M0);
    const double s = (double)(2 * c->p.radius + 1) * (double)(2 * c->p.radius + 1);
    double bound = 4.0 * M0;
    for (int p = 1; p < c->p.passes; ++p) bound *= s;
    if (c->p.flags & BUNDLE_FLAG_SEGMENT_HIST) {
        // a segment adds at most w_e to any cell, so cells stay below M0 as for points, but
        // the mass (one count per rasterised cell) has no tight static bound: 64-bit sums,
        // and the mass each iteration splats is checked on the device against what they hold
        if (c->p.sum_bits == 32)
            return fail(e, BUNDLE_EINVAL, "the segment histogram needs 64-bit sums");
        double per_mass = 4.0;
        for (int p = 1; p < c->p.passes; ++p) per_mass *= s;
        const double mix = c->G > 1 ? (double)c->p.alpha_den * (c->G - 1) + c->p.alpha_num : 1.0;
        c->mass_allowed = (unsigned long long)std::floor(two63 * (1 - 1e-12) / (per_mass * mix));
        bound = 0;  // replaced by the run-time check
    }
    int bits = c->p.sum_bits;
    if (c->p.flags & BUNDLE_FLAG_SEGMENT_HIST) bits = 64;
    if (bits == 0) bits = bound < two31 * (1 - 1e-12) ? 32 : 64;
    if (bits == 32 && !(bound < two31 * (1 - 1e-12)))
        return fail(e, BUNDLE_EOVERFLOW, "smoothed-sum bound %.6g does not fit int32", bound);
    if (!(bound < two63 * (1 - 1e-12)))
        return fail(e, BUNDLE_EOVERFLOW, "smoothed-sum bound %.6g does not fit int64", bound);
    c->sum_bits = bits;
    c->sum_bound = bound;
    double sk = 1;
    for (int p = 0; p < c->p.passes; ++p) sk *= s;
    if (c->G > 1) {
        c->mix_self = (int64_t)c->p.alpha_den * (c->G - 1) + c->p.alpha_num;
        c->mix_all = c->p.alpha_num;
        if (!((double)c->mix_self * bound < two63 * (1 - 1e-12)))
            return fail(e, BUNDLE_EOVERFLOW,
                        "layer-mix bound %.6g * %lld does not fit int64 (fewer points, passes or "
                        "groups, or a smaller radius)",
                        bound, (long long)c->mix_self);
        c->den_f = (float)((double)c->p.alpha_den * (c->G - 1) * sk);
    } else {
        c->mix_self = 1;
        c->mix_all = 0;
        c->den_f = (float)sk;
    }
    return BUNDLE_OK;
}

// World -> grid pixel map (Sec. 5): bounding box onto [m, W - m] x [m, H - m]
// with one isotropic scale, centred; computed in double, rounded to float once.
bundle_status grid_map(bundle_ctx* c, const float* src, const float* dst, std::string* e,
                       std::vector<float>* src_px, std::vector<float>* dst_px) {
    const int64_t E = c->E;
    const int margin = c->p.margin_px < 0 ? c->p.radius : c->p.margin_px;
    const double inf = std::numeric_limits<double>::infinity();
    double xmin = inf, ymin = inf, xmax = -inf, ymax = -inf;
    for (int64_t i = 0; i < E; ++i) {
        const float* q[2] = {src + 2 * i, dst + 2 * i};
        for (const float* v : q) {
            double x = v[0], y = v[1];
            if (!std::isfinite(x) || !std::isfinite(y))
                return fail(e, BUNDLE_EINVAL, "edge %lld has a non-finite coordinate",
                            (long long)i);
            xmin = std::min(xmin, x);
            xmax = std::max(xmax, x);
            ymin = std::min(ymin, y);
            ymax = std::max(ymax, y);
        }
    }
    double sx = xmax - xmin, sy = ymax - ymin;
    int64_t W = c->p.grid_w, H = c->p.grid_h;
    if (W <= 0 && H <= 0) {
        const int64_t dom = c->p.grid_dominant, lo = 2 * (int64_t)margin + 2;
        if (sx >= sy) {
            W = dom;
            H = sx > 0 ? (int64_t)std::llround(dom * (sy / sx)) : dom;
        } else {
            H = dom;
            W = (int64_t)std::llround(dom * (sx / sy));
        }
        W = std::max(W, lo);
        H = std::max(H, lo);
    } else if (W <= 0 || H <= 0) {
        return fail(e, BUNDLE_EINVAL, "grid_w and grid_h must both be > 0 or both be 0");
    }
    if (W < 2 || H < 2 || W > 4096 || H > 4096)
        return fail(e, BUNDLE_EINVAL, "grid %lld x %lld outside [2, 4096]", (long long)W,
                    (long long)H);
    if (W - 2 * (int64_t)margin <= 0 || H - 2 * (int64_t)margin <= 0)
        return fail(e, BUNDLE_EINVAL, "margin %d leaves no room on a %lld x %lld grid", margin,
                    (long long)W, (long long)H);
    double kx = sx > 0 ? ((double)W - 2.0 * margin) / sx : inf;
    double ky = sy > 0 ? ((double)H - 2.0 * margin) / sy : inf;
    double scale = std::min(kx, ky);
    if (!(scale < inf)) scale = 1.0;
    double ox = ((double)W - scale * sx) / 2.0;
    double oy = ((double)H - scale * sy) / 2.0;
    c->W = (int32_t)W;
    c->H = (int32_t)H;
    c->map[0] = xmin;
    c->map[1] = ymin;
    c->map[2] = scale;
    c->map[3] = ox;
    c->map[4] = oy;
    src_px->resize((size_t)(2 * E));
    dst_px->resize((size_t)(2 * E));
    const float hx = (float)W - kEdgeGuard, hy = (float)H - kEdgeGuard;
    auto work = [&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            const float* in[2] = {src + 2 * i, dst + 2 * i};
            float* out[2] = {src_px->data() + 2 * i, dst_px->data() + 2 * i};
            for (int s = 0; s < 2; ++s) {
                double px = ((double)in[s][0] - xmin) * scale + ox;
                double py = ((double)in[s][1] - ymin) * scale + oy;
                float fx = (float)px, fy = (float)py;
                out[s][0] = std::min(std::max(fx, 0.0f), hx);
                out[s][1] = std::min(std::max(fy, 0.0f), hy);
            }
        }
    };
    unsigned nt = std::min<unsigned>(16, std::max(1u, std::thread::hardware_concurrency()));
    if (E < 200000) nt = 1;
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back(work, E * t / nt, E * (t + 1) / nt);
    for (auto& t : th) t.join();
    return BUNDLE_OK;
}

// Device buffers sized from E, cap, G, H, W and the widths.
// The quad map's density gathers go through the texture path: a 1D texture over the
// linear quad map (one texel per quad, point sampled: the stored values bit for bit) moves
// them off the load/store data pipe, which the step kernel's shared-memory work and point
// traffic keep busy. Maps with more quads than a 1D texture holds keep the load path, and so
// does a context whose texture cannot be made (the view is a speed-up, not a requirement).
cudaError_t make_quad_texture(bundle_ctx* c) {
    const size_t n = (size_t)c->G * quad_elems(c->W, c->H);
    int max_w = 0;
    if (cudaDeviceGetAttribute(&max_w, cudaDevAttrMaxTexture1DLinearWidth, c->device) != cudaSuccess) {
        (void)cudaGetLastError();  // the launches after it check the last error
        return cudaSuccess;        // load path
    }
    if (n > (size_t)max_w || n > (size_t)INT32_MAX || (c->p.flags & BUNDLE_FLAG_LOAD_GATHERS))
        return cudaSuccess;  // load path
    cudaResourceDesc rd{};
    rd.resType = cudaResourceTypeLinear;
    rd.res.linear.devPtr = c->quads;
    rd.res.linear.desc = c->p.rho_dtype == BUNDLE_RHO_F32 ? cudaCreateChannelDesc<float4>()
                                                          : cudaCreateChannelDesc<ushort4>();
    rd.res.linear.sizeInBytes = n * 4 * rho_bytes(c->p.rho_dtype);
    cudaTextureDesc td{};
    td.readMode = cudaReadModeElementType;
    td.filterMode = cudaFilterModePoint;
    td.addressMode[0] = cudaAddressModeClamp;
    if (cudaCreateTextureObject(&c->qtex, &rd, &td, nullptr) != cudaSuccess) {
        (void)cudaGetLastError();
        c->qtex = 0;
    }
    return cudaSuccess;
}

bundle_status alloc_state(bundle_ctx* c, std::string* e) {
    const int64_t E = c->E;
    // blocks of up to 32 edges, one warp each; small graphs use smaller blocks so that at
    // least ~16 warps per SM (152 SMs) have work
    int eb = kMaxEdgesPerWarp;
    while (eb > 4 && E < (int64_t)eb * 152 * 16) eb /= 2;
    c->eb = eb;
    c->n_blocks = (E + eb - 1) / eb;
    // sized for blocks of kEdgesPerBlock whatever eb is, so that the autotuner can move the
    // points to any power-of-two block size without reallocating
    const size_t region = (size_t)((E + kEdgesPerBlock - 1) / kEdgesPerBlock) * kEdgesPerBlock * c->cap;
    const size_t C = (size_t)c->G * c->H * c->W;
    const size_t sb = c->sum_bits / 8;
    CUDA_TRY(e, dalloc(c, &c->perm, E));
    CUDA_TRY(e, dalloc(c, &c->group, E));
    CUDA_TRY(e, dalloc(c, &c->weight, E));
    for (int b = 0; b < 2; ++b) {
        CUDA_TRY(e, dalloc(c, &c->cnt[b], E));
        CUDA_TRY(e, dalloc(c, &c->pts[b], region));
    }
    CUDA_TRY(e, dalloc(c, &c->hist, C * kHistCopies));
    CUDA_TRY(e, dalloc(c, reinterpret_cast<unsigned char**>(&c->Y), C * sb));
    CUDA_TRY(e, dalloc(c, reinterpret_cast<unsigned char**>(&c->S), C * sb));
    CUDA_TRY(e, dalloc(c, reinterpret_cast<unsigned char**>(&c->rho), C * rho_bytes(c->p.rho_dtype)));
    CUDA_TRY(e, dalloc(c, reinterpret_cast<unsigned char**>(&c->quads),
                       (size_t)c->G * quad_elems(c->W, c->H) * 4 * rho_bytes(c->p.rho_dtype)));
    CUDA_TRY(e, make_quad_texture(c));
    CUDA_TRY(e, dalloc(c, &c->counters, 4));
    CUDA_TRY(e, dalloc(c, &c->d_iter, 1));
    CUDA_TRY(e, dalloc(c, &c->d_flag, 1));
    CUDA_TRY(e, cudaMemsetAsync(c->d_flag, 0, sizeof(int32_t), c->stream));
    if (c->p.flags & BUNDLE_FLAG_INK_STATS) {
        CUDA_TRY(e, dalloc(c, &c->ink, 2 * (size_t)BUNDLE_INK_STATS_CAP));
        CUDA_TRY(e, cudaMemsetAsync(c->ink, 0, 2 * sizeof(unsigned long long) * BUNDLE_INK_STATS_CAP,
                                    c->stream));
        CUDA_TRY(e, cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device));
    }
    CUDA_TRY(e, dalloc(c, &c->fetch_off, (size_t)E + 1));
    CUDA_TRY(e, dalloc(c, &c->fetch_tmp, scan_offsets_tmp_elems(E) + 1));
    CUDA_TRY(e, cudaMemsetAsync(c->hist, 0, C * kHistCopies * sizeof(uint32_t), c->stream));
    CUDA_TRY(e, cudaMemsetAsync(c->counters, 0, 4 * sizeof(unsigned long long), c->stream));
    return BUNDLE_OK;
}

// Spatial sort of the edges into slots: key = (group, Morton tile of the
// midpoint); a counting sort on the device. The bundling result does not depend
// on the slot order (every step is per edge, per point or an integer sum).
bundle_status sort_edges(bundle_ctx* c, const float2* d_src, const float2* d_dst,
                         const int32_t* d_group_in, const int32_t* d_weight_in, std::string* e) {
    const int64_t E = c->E;
    const int32_t nbk = c->G * 4096;
    uint32_t *key = nullptr, *bucket = nullptr;
    CUDA_TRY(e, cudaMalloc(&key, (size_t)E * sizeof(uint32_t)));
    cudaError_t err = cudaMalloc(&bucket, (size_t)nbk * sizeof(uint32_t));
    if (err != cudaSuccess) {
        cudaFree(key);
        CUDA_TRY(e, err);
    }
    int32_t* zero_group = nullptr;
    if (!d_group_in) {
        err = cudaMalloc(&zero_group, (size_t)E * sizeof(int32_t));
        if (err == cudaSuccess) err = cudaMemsetAsync(zero_group, 0, (size_t)E * 4, c->stream);
    }
    if (err == cudaSuccess) err = cudaMemsetAsync(bucket, 0, (size_t)nbk * 4, c->stream);
    const int32_t* gsrc = d_group_in ? d_group_in : zero_group;
    if (err == cudaSuccess)
        err = launch_edge_keys(d_src, d_dst, gsrc, E, c->W, c->H, key, bucket, c->stream);
    if (err == cudaSuccess) err = launch_bucket_scan(bucket, nbk, c->stream);
    if (err == cudaSuccess) err = launch_edge_scatter(key, E, bucket, c->perm, c->stream);
    if (err == cudaSuccess)
        err = launch_gather_edges(c->perm, E, gsrc, d_weight_in, c->group, c->weight, c->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
    cudaFree(key);
    cudaFree(bucket);
    if (zero_group) cudaFree(zero_group);
    CUDA_TRY(e, err);
    return BUNDLE_OK;
}

bundle_status make_ctx(bundle_ctx** out, const bundle_params* p, int64_t n_edges,
                       int32_t n_groups, void* stream, bundle_ctx** made, std::string* e) {
    if (!out) return fail(e, BUNDLE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!p) return fail(e, BUNDLE_EINVAL, "params is NULL");
    if (n_edges <= 0 || n_edges >= (int64_t)INT32_MAX)
        return fail(e, BUNDLE_EINVAL, "n_edges must be in [1, 2^31 - 1)");
    bundle_status s = check_params(*p, n_groups, e);
    if (s != BUNDLE_OK) return s;
    bundle_ctx* c = new (std::nothrow) bundle_ctx();
    if (!c) return fail(e, BUNDLE_ENOMEM, "host allocation failed");
    c->p = *p;
    c->E = n_edges;
    c->G = n_groups;
    c->cap = p->n_fixed > 0 ? p->n_fixed : p->n_max;
    c->stream = static_cast<cudaStream_t>(stream);
    c->device = -1;
    *made = c;
    return BUNDLE_OK;
}

// Bind the context to the current device and its stream (the first CUDA call
// of an init; host-side checks run before it).
bundle_status attach_cuda(bundle_ctx* c, std::string* e) {
    if (c->device >= 0) return BUNDLE_OK;
    cudaError_t err = cudaGetDevice(&c->device);
    if (err != cudaSuccess) {
        c->device = -1;
        return fail(e, BUNDLE_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(err));
    }
    if (!c->stream) {
        err = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (err != cudaSuccess) {
            c->stream = nullptr;
            return fail(e, BUNDLE_ECUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(err));
        }
        c->own_stream = true;
    }
    return BUNDLE_OK;
}

template <typename T>
bool to_host(const T* p, int64_t n, bool on_device, std::vector<T>* v, const T** view) {
    if (!p) {
        *view = nullptr;
        return true;
    }
    if (!on_device) {
        *view = p;
        return true;
    }
    v->resize((size_t)n);
    if (cudaMemcpy(v->data(), p, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost) != cudaSuccess)
        return false;
    *view = v->data();
    return true;
}

enum ProfileKind { kProfResample = 0, kProfAdvect, kProfAdvectResample, kProfRowbox,
                   kProfColbox, kProfMixQuads, kProfHistClear, kProfKinds };

// Launch through `fn`, bracketed by two events when profiling is on.
template <typename F>
cudaError_t timed(bundle_ctx* c, int kind, F fn) {
    if (!c->prof) return fn();
    while (c->ev_pool.size() < c->ev_used + 2) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        c->ev_pool.push_back(ev);
    }
    cudaEvent_t a = c->ev_pool[c->ev_used], b = c->ev_pool[c->ev_used + 1];
    cudaError_t e = cudaEventRecord(a, c->stream);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(b, c->stream);
    if (e == cudaSuccess) {
        c->ev_used += 2;
        c->ev_kind.push_back(kind);
    }
    return e;
}

// Arguments of one step launch of context c from buffer `in` to buffer `out`.
StepArgs make_step_args(bundle_ctx* c, int mode, int in, int out) {
    StepArgs a{};
    a.cnt_in = c->cnt[in];
    a.pts_in = c->pts[in];
    a.cnt_out = c->cnt[out];
    a.pts_out = c->pts[out];
    a.group = c->group;
    a.weight = c->weight;
    a.quads = c->quads;
    a.qtex = c->qtex;
    a.hist = c->hist;
    a.n_splat = c->counters;
    a.E = c->E;
    a.eb = c->eb;
    a.cap = c->cap;
    a.W = c->W;
    a.H = c->H;
    a.G = c->G;
    a.h = 0.0f;
    a.h_sched = c->h_sched;
    a.iter = c->d_iter;
    a.eps = c->p.eps;
    a.tries = c->p.step_tries;
    a.lap_keep = (float)(1.0 - (double)c->p.laplace_beta);
    a.lap_half_beta = (float)(0.5 * (double)c->p.laplace_beta);
    a.n_fixed = c->p.n_fixed;
    a.n_max = c->p.n_max;
    a.delta = c->p.delta_px;
    a.fixed_step = (c->p.flags & BUNDLE_FLAG_FIXED_STEP) ? 1 : 0;
    a.seg_hist = (c->p.flags & BUNDLE_FLAG_SEGMENT_HIST) ? 1 : 0;
    a.mass = a.seg_hist ? c->counters + 2 : nullptr;
    // the directed offset applies to the first sampling of the run only
    a.dir_amount = (mode == kModeResample && c->iteration == 0)
                       ? (float)((double)c->p.directed_offset * std::max(c->W, c->H))
                       : 0.0f;
    return a;
}

// hist_zero: the histogram is known to be zero already (the filter before cleared it).
bundle_status run_step(bundle_ctx* c, int mode, int in, int out, bool hist_zero = false) {
    const StepArgs a = make_step_args(c, mode, in, out);
    if ((mode & kModeResample) && !hist_zero)
        CUDA_TRY(&c->err, timed(c, kProfHistClear, [&] {
                     return cudaMemsetAsync(c->hist, 0,
                                            (size_t)kHistCopies * c->G * c->H * c->W * sizeof(uint32_t),
                                            c->stream);
                 }));
    if (a.seg_hist && (mode & kModeResample))
        CUDA_TRY(&c->err, cudaMemsetAsync(c->counters + 2, 0, sizeof(unsigned long long), c->stream));
    const int kind = mode == kModeResample ? kProfResample
                     : mode == kModeAdvect ? kProfAdvect : kProfAdvectResample;
    CUDA_TRY(&c->err, timed(c, kind, [&] { return launch_step(mode, c->p.rho_dtype, a, c->stream); }));
    if (a.seg_hist && (mode & kModeResample))
        CUDA_TRY(&c->err, launch_check_mass(c->counters + 2, c->mass_allowed, c->d_flag, c->stream));
    return BUNDLE_OK;
}

// Arguments of the grid-side kernels of context c.
FilterArgs filter_args(bundle_ctx* c) {
    FilterArgs f{};
    f.hist = c->hist;
    f.hist_copies = kHistCopies;
    f.Y = c->Y;
    f.S = c->S;
    f.rho = c->rho;
    f.quads = c->quads;
    f.G = c->G;
    f.H = c->H;
    f.W = c->W;
    f.r = c->p.radius;
    f.passes = c->p.passes;
    f.mix = c->mix;
    f.mix_self = c->mix_self;
    f.mix_all = c->mix_all;
    f.den_f = c->den_f;
    f.strip = c->col_strip;
    f.row_mode = c->row_mode;
    f.err_flag = c->d_flag;
    return f;
}

// clear: a splat follows, so the row pass may leave the histogram zero; *cleared (if
// given) says whether it did.
bundle_status run_filter(bundle_ctx* c, bool clear = false, bool* cleared = nullptr) {
    FilterArgs f = filter_args(c);
    f.clear_hist = clear ? 1 : 0;
    if (cleared) *cleared = filter_clears_hist(f);
    if (c->ink)
        CUDA_TRY(&c->err, launch_ink(c->hist, (int64_t)c->H * c->W, c->G, kHistCopies, c->ink,
                                     c->d_iter, BUNDLE_INK_STATS_CAP, c->n_sm, c->stream));
    CUDA_TRY(&c->err, timed(c, kProfRowbox, [&] { return launch_rowbox(c->sum_bits, f, c->stream); }));
    CUDA_TRY(&c->err, timed(c, kProfColbox, [&] { return launch_colbox(c->sum_bits, f, c->stream); }));
    CUDA_TRY(&c->err, timed(c, kProfMixQuads, [&] {
                 return launch_mix_quads(c->sum_bits, c->p.rho_dtype, f, c->stream);
             }));
    return BUNDLE_OK;
}

// The device schedule holds h_i for i < h_cap, filled by the same repeated
// multiplication as bandwidth(); it grows (doubling) when iterations run past it.
bundle_status ensure_schedule(bundle_ctx* c, int32_t needed) {
    if (needed <= c->h_cap && c->h_sched) return BUNDLE_OK;
    int32_t cap = c->h_cap > 0 ? c->h_cap : 1024;
    while (cap < needed) cap *= 2;
    std::vector<float> tab((size_t)cap);
    double h = bandwidth(c->p, 0);
    for (int32_t i = 0; i < cap; ++i) {
        tab[(size_t)i] = (float)h;
        h *= c->p.lambda;
    }
    float* d = nullptr;
    CUDA_TRY(&c->err, cudaMalloc(&d, (size_t)cap * sizeof(float)));
    cudaError_t e = cudaMemcpy(d, tab.data(), (size_t)cap * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        CUDA_TRY(&c->err, e);
    }
    if (c->h_sched) {
        CUDA_TRY(&c->err, cudaStreamSynchronize(c->stream));
        cudaFree(c->h_sched);
        c->device_bytes -= (int64_t)c->h_cap * 4;
    }
    c->h_sched = d;
    c->device_bytes += (int64_t)cap * 4;
    c->h_cap = cap;
    for (cudaGraphExec_t& g : c->gexec)  // the graphs hold the old pointer
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return BUNDLE_OK;
}

// One steady-state iteration: layer filter, mix into the density quads, histogram clear, the fused
// advect -> resample -> splat step from buffer R to 1 - R, then the counter advance.
bundle_status launch_iteration(bundle_ctx* c, int R) {
    bool cleared = false;
    bundle_status s = run_filter(c, true, &cleared);
    if (s != BUNDLE_OK) return s;
    s = run_step(c, kModeAdvectResample, R, 1 - R, cleared);
    if (s != BUNDLE_OK) return s;
    CUDA_TRY(&c->err, launch_advance_iter(c->d_iter, c->stream));
    return BUNDLE_OK;
}

bundle_status build_graph(bundle_ctx* c, int R) {
    if (!c->cap_stream)
        CUDA_TRY(&c->err, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaStream_t saved = c->stream;
    c->stream = c->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    bundle_status s = e == cudaSuccess ? launch_iteration(c, R) : BUNDLE_ECUDA;
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    c->stream = saved;
    if (e != cudaSuccess) return fail(&c->err, BUNDLE_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    if (s != BUNDLE_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e2 != cudaSuccess)
        return fail(&c->err, BUNDLE_ECUDA, "graph capture end: %s", cudaGetErrorString(e2));
    e = cudaGraphInstantiate(&c->gexec[R], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec[R] = nullptr;
        return fail(&c->err, BUNDLE_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return BUNDLE_OK;
}

}  // namespace

extern "C" {

void bundle_default_params(bundle_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->grid_w = 0;
    p->grid_h = 0;
    p->grid_dominant = 800;
    p->margin_px = -1;
    p->radius = 4;
    p->passes = 3;
    p->alpha_num = 1;
    p->alpha_den = 4;
    p->h_max_sigmas = 2.0;
    p->lambda = 0.9;
    p->n_fixed = 0;
    p->n_max = 64;
    p->delta_px = 2.0f;
    p->laplace_beta = 0.5f;
    p->eps = 1e-9f;
    p->step_tries = 8;
    p->sum_bits = 0;
    p->rho_dtype = BUNDLE_RHO_F32;
    p->flags = 0;
}

bundle_status bundle_init(bundle_ctx** out, const bundle_params* p, int64_t n_edges,
                          const float* src_xy, const float* dst_xy, const int32_t* group,
                          int32_t n_groups, const int32_t* weight, int32_t flags, void* stream) {
    std::string* e = &g_init_error;
    bundle_ctx* c = nullptr;
    bundle_status s = make_ctx(out, p, n_edges, n_groups, stream, &c, e);
    if (s != BUNDLE_OK) return s;
    auto bail = [&](bundle_status st) {
        free_ctx(c);
        return st;
    };
    if (!src_xy || !dst_xy) return bail(fail(e, BUNDLE_EINVAL, "src_xy and dst_xy are required"));
    const bool dev = (flags & BUNDLE_INPUT_DEVICE) != 0;
    if (dev && (s = attach_cuda(c, e)) != BUNDLE_OK) return bail(s);
    std::vector<float> hs, hd;
    std::vector<int32_t> hg, hw;
    const float *vs, *vd;
    const int32_t *vg, *vw;
    if (!to_host(src_xy, 2 * n_edges, dev, &hs, &vs) || !to_host(dst_xy, 2 * n_edges, dev, &hd, &vd) ||
        !to_host(group, n_edges, dev, &hg, &vg) || !to_host(weight, n_edges, dev, &hw, &vw))
        return bail(fail(e, BUNDLE_ECUDA, "copy of device inputs failed"));
    if (vg)
        for (int64_t i = 0; i < n_edges; ++i)
            if (vg[i] < 0 || vg[i] >= n_groups)
                return bail(fail(e, BUNDLE_EINVAL, "group[%lld] = %d outside [0, %d)",
                                 (long long)i, vg[i], n_groups));
    s = size_integers(c, vw, e);
    if (s != BUNDLE_OK) return bail(s);
    std::vector<float> spx, dpx;
    s = grid_map(c, vs, vd, e, &spx, &dpx);
    if (s != BUNDLE_OK) return bail(s);
    if (c->p.radius >= std::min(c->W, c->H))
        return bail(fail(e, BUNDLE_EINVAL, "radius %d must be below min(W, H) = %d", c->p.radius,
                         std::min(c->W, c->H)));
    if ((s = attach_cuda(c, e)) != BUNDLE_OK) return bail(s);
    DeviceGuard dg(c->device);
    s = alloc_state(c, e);
    if (s != BUNDLE_OK) return bail(s);
    // staging copies of the mapped endpoints, groups and weights
    float2 *d_src = nullptr, *d_dst = nullptr;
    int32_t *d_g = nullptr, *d_w = nullptr;
    cudaError_t err = cudaMalloc(&d_src, (size_t)n_edges * sizeof(float2));
    if (err == cudaSuccess) err = cudaMalloc(&d_dst, (size_t)n_edges * sizeof(float2));
    if (err == cudaSuccess && vg) err = cudaMalloc(&d_g, (size_t)n_edges * 4);
    if (err == cudaSuccess && vw) err = cudaMalloc(&d_w, (size_t)n_edges * 4);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(d_src, spx.data(), (size_t)n_edges * 8, cudaMemcpyHostToDevice,
                              c->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(d_dst, dpx.data(), (size_t)n_edges * 8, cudaMemcpyHostToDevice,
                              c->stream);
    if (err == cudaSuccess && vg)
        err = cudaMemcpyAsync(d_g, vg, (size_t)n_edges * 4, cudaMemcpyHostToDevice, c->stream);
    if (err == cudaSuccess && vw)
        err = cudaMemcpyAsync(d_w, vw, (size_t)n_edges * 4, cudaMemcpyHostToDevice, c->stream);
    bundle_status st = BUNDLE_OK;
    if (err == cudaSuccess) st = sort_edges(c, d_src, d_dst, d_g, d_w, e);
    if (err == cudaSuccess && st == BUNDLE_OK)
        err = launch_straight_layout(c->perm, n_edges, d_src, d_dst, c->eb, c->cap, c->cnt[0],
                                     c->pts[0], c->stream);
    if (err == cudaSuccess && st == BUNDLE_OK) err = cudaStreamSynchronize(c->stream);
    cudaFree(d_src);
    cudaFree(d_dst);
    if (d_g) cudaFree(d_g);
    if (d_w) cudaFree(d_w);
    if (st != BUNDLE_OK) return bail(st);
    if (err != cudaSuccess)
        return bail(fail(e, err == cudaErrorMemoryAllocation ? BUNDLE_ENOMEM : BUNDLE_ECUDA,
                         "init staging: %s", cudaGetErrorString(err)));
    c->cur_P = 0;
    c->cur_R = -1;
    c->straight = true;
    *out = c;
    return BUNDLE_OK;
}

bundle_status bundle_init_polylines(bundle_ctx** out, const bundle_params* p, int64_t n_edges,
                                    const int64_t* off, const float* xy_px, const int32_t* group,
                                    int32_t n_groups, const int32_t* weight, const double* map5,
                                    int32_t iteration, int32_t flags, void* stream) {
    std::string* e = &g_init_error;
    bundle_ctx* c = nullptr;
    bundle_status s = make_ctx(out, p, n_edges, n_groups, stream, &c, e);
    if (s != BUNDLE_OK) return s;
    auto bail = [&](bundle_status st) {
        free_ctx(c);
        return st;
    };
    if (!off || !xy_px) return bail(fail(e, BUNDLE_EINVAL, "off and xy_px are required"));
    if (p->grid_w < 2 || p->grid_h < 2 || p->grid_w > 4096 || p->grid_h > 4096)
        return bail(fail(e, BUNDLE_EINVAL, "grid_w and grid_h must be in [2, 4096]"));
    if (iteration < 0) return bail(fail(e, BUNDLE_EINVAL, "iteration must be >= 0"));
    c->W = p->grid_w;
    c->H = p->grid_h;
    if (c->p.radius >= std::min(c->W, c->H))
        return bail(fail(e, BUNDLE_EINVAL, "radius must be below min(W, H)"));
    const bool dev = (flags & BUNDLE_INPUT_DEVICE) != 0;
    if (dev && (s = attach_cuda(c, e)) != BUNDLE_OK) return bail(s);
    std::vector<int64_t> ho;
    std::vector<int32_t> hg, hw;
    std::vector<float> hx;
    const int64_t* vo;
    const int32_t *vg, *vw;
    const float* vx;
    if (!to_host(off, n_edges + 1, dev, &ho, &vo))
        return bail(fail(e, BUNDLE_ECUDA, "copy of device offsets failed"));
    const int64_t N = vo[n_edges];
    if (vo[0] != 0 || N <= 0) return bail(fail(e, BUNDLE_EINVAL, "off must start at 0"));
    for (int64_t i = 0; i < n_edges; ++i) {
        int64_t n = vo[i + 1] - vo[i];
        if (n < 2 || n > c->cap)
            return bail(fail(e, BUNDLE_EINVAL, "polyline %lld has %lld points, need 2..%d",
                             (long long)i, (long long)n, c->cap));
    }
    if (!to_host(xy_px, 2 * N, dev, &hx, &vx) || !to_host(group, n_edges, dev, &hg, &vg) ||
        !to_host(weight, n_edges, dev, &hw, &vw))
        return bail(fail(e, BUNDLE_ECUDA, "copy of device inputs failed"));
    const float hxm = (float)c->W - kEdgeGuard, hym = (float)c->H - kEdgeGuard;
    for (int64_t k = 0; k < N; ++k)
        if (!(vx[2 * k] >= 0 && vx[2 * k] <= hxm && vx[2 * k + 1] >= 0 && vx[2 * k + 1] <= hym))
            return bail(fail(e, BUNDLE_EINVAL, "point %lld lies outside [0, W - 2^-10] x "
                             "[0, H - 2^-10]", (long long)k));
    if (vg)
        for (int64_t i = 0; i < n_edges; ++i)
            if (vg[i] < 0 || vg[i] >= n_groups)
                return bail(fail(e, BUNDLE_EINVAL, "group[%lld] outside [0, %d)", (long long)i,
                                 n_groups));
    s = size_integers(c, vw, e);
    if (s != BUNDLE_OK) return bail(s);
    if (map5) std::memcpy(c->map, map5, sizeof c->map);
    c->iteration = iteration;
    if ((s = attach_cuda(c, e)) != BUNDLE_OK) return bail(s);
    DeviceGuard dg(c->device);
    s = alloc_state(c, e);
    if (s != BUNDLE_OK) return bail(s);
    // midpoint keys from each polyline's endpoints
    std::vector<float> ends_s((size_t)(2 * n_edges)), ends_d((size_t)(2 * n_edges));
    for (int64_t i = 0; i < n_edges; ++i) {
        ends_s[2 * i] = vx[2 * vo[i]];
        ends_s[2 * i + 1] = vx[2 * vo[i] + 1];
        ends_d[2 * i] = vx[2 * (vo[i + 1] - 1)];
        ends_d[2 * i + 1] = vx[2 * (vo[i + 1] - 1) + 1];
    }
    float2 *d_src = nullptr, *d_dst = nullptr, *d_xy = nullptr;
    int32_t *d_g = nullptr, *d_w = nullptr;
    int64_t* d_off = nullptr;
    cudaError_t err = cudaMalloc(&d_src, (size_t)n_edges * 8);
    if (err == cudaSuccess) err = cudaMalloc(&d_dst, (size_t)n_edges * 8);
    if (err == cudaSuccess) err = cudaMalloc(&d_xy, (size_t)N * 8);
    if (err == cudaSuccess) err = cudaMalloc(&d_off, (size_t)(n_edges + 1) * 8);
    if (err == cudaSuccess && vg) err = cudaMalloc(&d_g, (size_t)n_edges * 4);
    if (err == cudaSuccess && vw) err = cudaMalloc(&d_w, (size_t)n_edges * 4);
    if (err == cudaSuccess)
        err = cudaMemcpy(d_src, ends_s.data(), (size_t)n_edges * 8, cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(d_dst, ends_d.data(), (size_t)n_edges * 8, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(d_xy, vx, (size_t)N * 8, cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(d_off, vo, (size_t)(n_edges + 1) * 8, cudaMemcpyHostToDevice);
    if (err == cudaSuccess && vg)
        err = cudaMemcpy(d_g, vg, (size_t)n_edges * 4, cudaMemcpyHostToDevice);
    if (err == cudaSuccess && vw)
        err = cudaMemcpy(d_w, vw, (size_t)n_edges * 4, cudaMemcpyHostToDevice);
    bundle_status st = BUNDLE_OK;
    if (err == cudaSuccess) st = sort_edges(c, d_src, d_dst, d_g, d_w, e);
    if (err == cudaSuccess && st == BUNDLE_OK)
        err = launch_polyline_layout(c->perm, n_edges, d_off, d_xy, c->eb, c->cap, c->cnt[0],
                                     c->pts[0], c->stream);
    if (err == cudaSuccess && st == BUNDLE_OK) err = cudaStreamSynchronize(c->stream);
    cudaFree(d_src);
    cudaFree(d_dst);
    cudaFree(d_xy);
    cudaFree(d_off);
    if (d_g) cudaFree(d_g);
    if (d_w) cudaFree(d_w);
    if (st != BUNDLE_OK) return bail(st);
    if (err != cudaSuccess)
        return bail(fail(e, err == cudaErrorMemoryAllocation ? BUNDLE_ENOMEM : BUNDLE_ECUDA,
                         "init staging: %s", cudaGetErrorString(err)));
    c->cur_P = 0;
    c->cur_R = -1;
    *out = c;
    return BUNDLE_OK;
}

static bundle_status iterate_single(bundle_ctx* c, int32_t n_iters) {
    bundle_status s = ensure_schedule(c, c->iteration + n_iters);
    if (s != BUNDLE_OK) return s;
    CUDA_TRY(&c->err, launch_set_iter(c->d_iter, c->iteration, c->stream));
    // resample the current polylines and splat them (start of the first iteration)
    int src = c->cur_P, dst = 1 - c->cur_P;
    s = run_step(c, kModeResample, src, dst);
    if (s != BUNDLE_OK) return s;
    int R = dst;
    for (int32_t it = 0; it < n_iters; ++it) {
        const bool last = it == n_iters - 1;
        if (last) {
            s = run_filter(c);
            if (s == BUNDLE_OK) s = run_step(c, kModeAdvect, R, 1 - R);
            if (s != BUNDLE_OK) return s;
            CUDA_TRY(&c->err, launch_advance_iter(c->d_iter, c->stream));
            c->cur_P = 1 - R;
            c->cur_R = R;
        } else if (c->use_graphs && !c->prof) {
            if (!c->gexec[R] && (s = build_graph(c, R)) != BUNDLE_OK) return s;
            CUDA_TRY(&c->err, cudaGraphLaunch(c->gexec[R], c->stream));
            R = 1 - R;
        } else {
            if ((s = launch_iteration(c, R)) != BUNDLE_OK) return s;
            R = 1 - R;
        }
        c->iteration += 1;
    }
    c->have_density = true;
    return BUNDLE_OK;
}


// Fork: every member stream waits for the work queued so far on `from`.
static bundle_status batch_fork(bundle_ctx* c, cudaStream_t from) {
    CUDA_TRY(&c->err, cudaEventRecord(c->bev[0], from));
    for (bundle_ctx* m : c->members) CUDA_TRY(&c->err, cudaStreamWaitEvent(m->stream, c->bev[0], 0));
    return BUNDLE_OK;
}

// Join: `into` waits for every member stream.
static bundle_status batch_join(bundle_ctx* c, cudaStream_t into) {
    for (size_t k = 0; k < c->members.size(); ++k) {
        CUDA_TRY(&c->err, cudaEventRecord(c->bev[k + 1], c->members[k]->stream));
        CUDA_TRY(&c->err, cudaStreamWaitEvent(into, c->bev[k + 1], 0));
    }
    return BUNDLE_OK;
}

// One steady-state iteration of every member, each on its own branch, as one graph.
// The steady iterations of a batch run one step launch over all its graphs when they
// share the density type and need no per-graph check after the step (the segment
// histogram's mass check).
static bool batch_mergeable(const bundle_ctx* c) {
    for (const bundle_ctx* m : c->members)
        if (m->p.rho_dtype != c->members[0]->p.rho_dtype || (m->p.flags & BUNDLE_FLAG_SEGMENT_HIST))
            return false;
    return true;
}

static bundle_status build_batch_graph(bundle_ctx* c, int R) {
    if (!c->cap_stream)
        CUDA_TRY(&c->err, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    std::vector<cudaStream_t> saved;
    for (bundle_ctx* m : c->members) {
        if (!m->cap_stream)
            CUDA_TRY(&c->err, cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
    }
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(&c->err, BUNDLE_ECUDA, "batch capture: %s", cudaGetErrorString(e));
    bundle_status s = BUNDLE_OK;
    for (bundle_ctx* m : c->members) saved.push_back(m->stream);
    for (bundle_ctx* m : c->members) m->stream = m->cap_stream;
    if (s == BUNDLE_OK) s = batch_fork(c, c->cap_stream);
    if (batch_mergeable(c)) {
        // every graph's filter on its own branch, then one step launch over all graphs
        for (size_t k = 0; k < c->members.size() && s == BUNDLE_OK; ++k) {
            bundle_ctx* m = c->members[k];
            bool cleared = false;
            s = run_filter(m, true, &cleared);
            if (s == BUNDLE_OK && !cleared &&
                cudaMemsetAsync(m->hist, 0, (size_t)kHistCopies * m->G * m->H * m->W * sizeof(uint32_t),
                                m->stream) != cudaSuccess)
                s = BUNDLE_ECUDA;
            if (s != BUNDLE_OK) c->err = "member " + std::to_string(k) + ": " + m->err;
        }
        if (s == BUNDLE_OK) s = batch_join(c, c->cap_stream);
        std::unique_ptr<BatchStepArgs> P(new (std::nothrow) BatchStepArgs());
        if (!P) s = fail(&c->err, BUNDLE_ENOMEM, "host allocation failed");
        for (size_t k0 = 0; k0 < c->members.size() && s == BUNDLE_OK; k0 += kBatchLaunch) {
            const size_t n = std::min<size_t>(kBatchLaunch, c->members.size() - k0);
            P->n = (int32_t)n;
            P->blk[0] = 0;
            for (size_t j = 0; j < n; ++j) {
                bundle_ctx* m = c->members[k0 + j];
                P->a[j] = make_step_args(m, kModeAdvectResample, R, 1 - R);
                P->blk[j + 1] = P->blk[j] + (int32_t)step_ctas(m->E, m->eb);
            }
            if (launch_step_batch(kModeAdvectResample, c->members[0]->p.rho_dtype, *P,
                                  c->cap_stream) != cudaSuccess ||
                launch_advance_batch(*P, c->cap_stream) != cudaSuccess)
                s = fail(&c->err, BUNDLE_ECUDA, "batched step launch failed");
        }
    } else {
        for (size_t k = 0; k < c->members.size() && s == BUNDLE_OK; ++k) {
            s = launch_iteration(c->members[k], R);
            if (s != BUNDLE_OK) c->err = "member " + std::to_string(k) + ": " + c->members[k]->err;
        }
        if (s == BUNDLE_OK) s = batch_join(c, c->cap_stream);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    for (size_t k = 0; k < c->members.size(); ++k) c->members[k]->stream = saved[k];
    if (s != BUNDLE_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e2 != cudaSuccess)
        return fail(&c->err, BUNDLE_ECUDA, "batch capture end: %s", cudaGetErrorString(e2));
    e = cudaGraphInstantiate(&c->bexec[R], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->bexec[R] = nullptr;
        return fail(&c->err, BUNDLE_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
    }
    return BUNDLE_OK;
}

static bundle_status iterate_batch(bundle_ctx* c, int32_t n_iters) {
    bundle_status s = batch_fork(c, c->stream);
    if (s != BUNDLE_OK) return s;
    const bool graphs = c->use_graphs && !c->prof && n_iters > 1;
    if (!graphs) {
        // every member runs its own iterations on its stream, concurrently
        for (size_t k = 0; k < c->members.size(); ++k)
            if ((s = iterate_single(c->members[k], n_iters)) != BUNDLE_OK) {
                c->err = "member " + std::to_string(k) + ": " + c->members[k]->err;
                return s;
            }
        return batch_join(c, c->stream);
    }
    // members in lockstep: resample + splat on each stream, then n - 1 batch graphs, then
    // the last iteration's filter and advection on each stream
    int R = -1;
    for (size_t k = 0; k < c->members.size(); ++k) {
        bundle_ctx* m = c->members[k];
        const float* before = m->h_sched;
        if ((s = ensure_schedule(m, m->iteration + n_iters)) != BUNDLE_OK) return s;
        if (m->h_sched != before)  // the batch graphs captured the old schedule
            for (cudaGraphExec_t& g : c->bexec)
                if (g) {
                    cudaGraphExecDestroy(g);
                    g = nullptr;
                }
        CUDA_TRY(&m->err, launch_set_iter(m->d_iter, m->iteration, m->stream));
        if ((s = run_step(m, kModeResample, m->cur_P, 1 - m->cur_P)) != BUNDLE_OK) return s;
        if (R < 0) R = 1 - m->cur_P;
        if (1 - m->cur_P != R) return fail(&c->err, BUNDLE_ESTATE, "batch members out of step");
    }
    if ((s = batch_join(c, c->stream)) != BUNDLE_OK) return s;
    for (int32_t it = 0; it + 1 < n_iters; ++it) {
        if (!c->bexec[R] && (s = build_batch_graph(c, R)) != BUNDLE_OK) return s;
        CUDA_TRY(&c->err, cudaGraphLaunch(c->bexec[R], c->stream));
        R = 1 - R;
    }
    if ((s = batch_fork(c, c->stream)) != BUNDLE_OK) return s;
    for (bundle_ctx* m : c->members) {
        if ((s = run_filter(m)) == BUNDLE_OK) s = run_step(m, kModeAdvect, R, 1 - R);
        if (s != BUNDLE_OK) return s;
        CUDA_TRY(&m->err, launch_advance_iter(m->d_iter, m->stream));
        m->cur_P = 1 - R;
        m->cur_R = R;
        m->iteration += n_iters;
        m->have_density = true;
    }
    return batch_join(c, c->stream);
}

bundle_status bundle_iterate(bundle_ctx* c, int32_t n_iters) {
    if (!c) return BUNDLE_EINVAL;
    if (c->is_member)
        return fail(&c->err, BUNDLE_ESTATE, "a batch member iterates with its batch");
    if (c->split_state != 0)
        return fail(&c->err, BUNDLE_ESTATE, "a run of bundle_points_step is open: end it with "
                    "BUNDLE_STEP_LAST first");
    if (n_iters < 0) return fail(&c->err, BUNDLE_EINVAL, "n_iters must be >= 0");
    if (n_iters == 0) return BUNDLE_OK;
    DeviceGuard dg(c->device);
    if (!c->members.empty()) {
        bundle_status s = iterate_batch(c, n_iters);
        if (s == BUNDLE_OK) {
            c->iteration += n_iters;
            c->have_density = true;
        }
        return s;
    }
    return iterate_single(c, n_iters);
}

// ------------------------------------------------------------------ split form
// One graph's edges divided over several contexts (one per process or GPU): each
// context runs the per-edge stages -- advection, Laplacian smoothing, resampling and
// the splat -- on its own edges, and the histogram, the only state that couples
// edges, is summed over the contexts between the splat and the box passes. Integer
// addition is exact and order-free, so every context then holds the histogram of the
// whole graph and the run equals one context over all edges bit for bit. (Sec. 4
// splits the edges of one graph over CPU threads the same way.)

static bundle_status split_checks(bundle_ctx* c, const char* what) {
    if (!c->members.empty() || c->is_member)
        return fail(&c->err, BUNDLE_ESTATE, "%s: batches run whole iterations", what);
    return BUNDLE_OK;
}

bundle_status bundle_points_step(bundle_ctx* c, int32_t flags) {
    if (!c) return BUNDLE_EINVAL;
    if (bundle_status s = split_checks(c, "bundle_points_step")) return s;
    if (flags & ~BUNDLE_STEP_LAST)
        return fail(&c->err, BUNDLE_EINVAL, "bundle_points_step: unknown flags %d", flags);
    if (c->split_state == 1)
        return fail(&c->err, BUNDLE_ESTATE, "bundle_points_step: run bundle_density_step on the "
                    "(summed) histogram first");
    DeviceGuard dg(c->device);
    bundle_status s = ensure_schedule(c, c->iteration + 1);
    if (s != BUNDLE_OK) return s;
    if (c->split_state == 0) {
        if (flags & BUNDLE_STEP_LAST)
            return fail(&c->err, BUNDLE_EINVAL, "bundle_points_step: a run opens without "
                        "BUNDLE_STEP_LAST");
        // the start of a run: resample and splat the current polylines
        CUDA_TRY(&c->err, launch_set_iter(c->d_iter, c->iteration, c->stream));
        if ((s = run_step(c, kModeResample, c->cur_P, 1 - c->cur_P)) != BUNDLE_OK) return s;
        c->split_R = 1 - c->cur_P;
        c->split_state = 1;
        return BUNDLE_OK;
    }
    // advect on this iteration's density; resample and splat for the next one unless last
    const int R = c->split_R;
    const bool last = (flags & BUNDLE_STEP_LAST) != 0;
    if ((s = run_step(c, last ? kModeAdvect : kModeAdvectResample, R, 1 - R)) != BUNDLE_OK) return s;
    CUDA_TRY(&c->err, launch_advance_iter(c->d_iter, c->stream));
    c->iteration += 1;
    if (last) {
        c->cur_P = 1 - R;
        c->cur_R = R;
        c->split_state = 0;
    } else {
        c->split_R = 1 - R;
        c->split_state = 1;
    }
    return BUNDLE_OK;
}

bundle_status bundle_density_step(bundle_ctx* c) {
    if (!c) return BUNDLE_EINVAL;
    if (bundle_status s = split_checks(c, "bundle_density_step")) return s;
    if (c->split_state != 1)
        return fail(&c->err, BUNDLE_ESTATE, "bundle_density_step: no splatted histogram is "
                    "waiting (call bundle_points_step first)");
    DeviceGuard dg(c->device);
    bundle_status s = run_filter(c);
    if (s != BUNDLE_OK) return s;
    c->split_state = 2;
    c->have_density = true;
    return BUNDLE_OK;
}

bundle_status bundle_set_histogram(bundle_ctx* c, const uint32_t* src, int32_t flags) {
    if (!c) return BUNDLE_EINVAL;
    if (bundle_status s = split_checks(c, "bundle_set_histogram")) return s;
    if (!src) return fail(&c->err, BUNDLE_EINVAL, "bundle_set_histogram: src is NULL");
    if (flags & ~BUNDLE_INPUT_DEVICE)
        return fail(&c->err, BUNDLE_EINVAL, "bundle_set_histogram: unknown flags %d", flags);
    if (c->split_state != 1)
        return fail(&c->err, BUNDLE_ESTATE, "bundle_set_histogram: only between "
                    "bundle_points_step and bundle_density_step");
    DeviceGuard dg(c->device);
    const size_t C = (size_t)c->G * c->H * c->W;
    // copy 0 takes the histogram, the other copies are cleared: the row passes sum them
    CUDA_TRY(&c->err, cudaMemcpyAsync(c->hist, src, C * sizeof(uint32_t),
                                      (flags & BUNDLE_INPUT_DEVICE) ? cudaMemcpyDeviceToDevice
                                                                    : cudaMemcpyHostToDevice,
                                      c->stream));
    CUDA_TRY(&c->err, cudaMemsetAsync(c->hist + C, 0, (kHistCopies - 1) * C * sizeof(uint32_t),
                                      c->stream));
    if (!(flags & BUNDLE_INPUT_DEVICE)) CUDA_TRY(&c->err, cudaStreamSynchronize(c->stream));
    return BUNDLE_OK;
}

bundle_status bundle_init_batch(bundle_ctx** out, int32_t n_graphs, const bundle_graph_desc* graphs,
                                const bundle_params* params, int32_t flags, void* stream) {
    std::string* e = &g_init_error;
    if (!out) return fail(e, BUNDLE_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_graphs < 1 || n_graphs > 4096 || !graphs || !params)
        return fail(e, BUNDLE_EINVAL, "need 1..4096 graphs with their parameters");
    bundle_ctx* c = new (std::nothrow) bundle_ctx();
    if (!c) return fail(e, BUNDLE_ENOMEM, "host allocation failed");
    c->stream = static_cast<cudaStream_t>(stream);
    c->device = -1;
    bundle_status s = attach_cuda(c, e);
    if (s != BUNDLE_OK) {
        free_ctx(c);
        return s;
    }
    for (int32_t k = 0; k < n_graphs; ++k) {
        bundle_ctx* m = nullptr;
        const bundle_graph_desc& g = graphs[k];
        s = bundle_init(&m, &params[k], g.n_edges, g.src_xy, g.dst_xy, g.group, g.n_groups,
                        g.weight, flags, nullptr);
        if (s != BUNDLE_OK) {
            std::string msg = "graph " + std::to_string(k) + ": " + *e;
            free_ctx(c);
            *e = msg;
            return s;
        }
        m->is_member = true;
        c->members.push_back(m);
        c->E += m->E;
    }
    c->bev.resize(c->members.size() + 1);
    for (cudaEvent_t& ev : c->bev)
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            free_ctx(c);
            return fail(e, BUNDLE_ECUDA, "event creation failed");
        }
    c->G = c->members[0]->G;
    c->W = c->members[0]->W;
    c->H = c->members[0]->H;
    *out = c;
    return BUNDLE_OK;
}

int32_t bundle_batch_size(const bundle_ctx* c) { return c ? (int32_t)c->members.size() : 0; }

bundle_ctx* bundle_batch_member(bundle_ctx* c, int32_t k) {
    if (!c || k < 0 || k >= (int32_t)c->members.size()) return nullptr;
    return c->members[(size_t)k];
}

// ---------------------------------------------------------------- autotuner
// Elapsed milliseconds of fn() on the context's stream (events around it).
static bundle_status time_ms(bundle_ctx* c, const std::function<bundle_status()>& fn, float* ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = cudaEventRecord(a, c->stream);
    bundle_status s = e == cudaSuccess ? fn() : BUNDLE_ECUDA;
    if (s == BUNDLE_OK && e == cudaSuccess) e = cudaEventRecord(b, c->stream);
    if (s == BUNDLE_OK && e == cudaSuccess) e = cudaEventSynchronize(b);
    if (s == BUNDLE_OK && e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s != BUNDLE_OK) return s;
    CUDA_TRY(&c->err, e);
    return BUNDLE_OK;
}

// Probe state of one fresh context: its straight edges in slot order (two points per
// slot), from which any block layout can be rebuilt.
struct TuneProbe {
    float2* keep = nullptr;
    TuneProbe() = default;
    TuneProbe(const TuneProbe&) = delete;
    TuneProbe& operator=(const TuneProbe&) = delete;
    ~TuneProbe() { cudaFree(keep); }
};

static bundle_status probe_begin(bundle_ctx* c, TuneProbe* t) {
    if (!c->straight || c->iteration != 0 || c->cur_R >= 0)
        return fail(&c->err, BUNDLE_ESTATE,
                    "bundle_autotune: needs a context fresh from bundle_init (no iteration yet)");
    bundle_status s = ensure_schedule(c, 2);
    if (s != BUNDLE_OK) return s;
    CUDA_TRY(&c->err, cudaMalloc(&t->keep, (size_t)c->E * 2 * sizeof(float2)));
    CUDA_TRY(&c->err, launch_relayout_pairs(c->pts[c->cur_P], c->eb, c->cap, t->keep, 1, 2,
                                            nullptr, c->E, c->stream));
    return BUNDLE_OK;
}

// Lay the straight edges out in blocks of eb edges (buffer 0).
static bundle_status probe_layout(bundle_ctx* c, const TuneProbe& t, int32_t eb) {
    c->eb = eb;
    c->n_blocks = (c->E + eb - 1) / eb;
    CUDA_TRY(&c->err, launch_relayout_pairs(t.keep, 1, 2, c->pts[0], eb, c->cap, c->cnt[0], c->E,
                                            c->stream));
    return BUNDLE_OK;
}

// Iteration 0 up to the density (resample + splat the straight edges, filter), then the
// fused advect + resample step that is timed: the two halves, enqueued on c->stream.
static bundle_status probe_prefix(bundle_ctx* c) {
    CUDA_TRY(&c->err, launch_set_iter(c->d_iter, 0, c->stream));
    bundle_status s = run_step(c, kModeResample, 0, 1);
    return s == BUNDLE_OK ? run_filter(c) : s;
}
static bundle_status probe_step(bundle_ctx* c) { return run_step(c, kModeAdvectResample, 1, 0); }

// Row-pass variant and column-pass strip of one context, timed on its current
// histogram (best of three each), then the banded path (both passes) against the
// fastest pair.
static bundle_status tune_filter(bundle_ctx* c) {
    const int sb = c->sum_bits / 8;
    int best_row = c->row_mode, best_strip = c->col_strip;
    float best_row_ms = 3.4e38f, best_col_ms = 3.4e38f;
    FilterArgs f{};
    f.hist = c->hist;
    f.hist_copies = kHistCopies;
    f.Y = c->Y;
    f.S = c->S;
    f.G = c->G;
    f.H = c->H;
    f.W = c->W;
    f.r = c->p.radius;
    f.passes = c->p.passes;
    bundle_status s;
    for (int mode = 1; mode <= 3; ++mode) {
        if (!rowbox_mode_valid(mode, c->W, c->H, c->p.radius)) continue;
        f.row_mode = mode;
        for (int rep = 0; rep < 3; ++rep) {
            float ms = 0;
            s = time_ms(c, [&] {
                return launch_rowbox(c->sum_bits, f, c->stream) == cudaSuccess ? BUNDLE_OK : BUNDLE_ECUDA;
            }, &ms);
            if (s != BUNDLE_OK) return s;
            if (ms < best_row_ms) {
                best_row_ms = ms;
                best_row = mode;
            }
        }
    }
    for (int strip = 2; strip <= 16; strip *= 2) {
        if (!colbox_strip_valid(strip, c->W, c->H, c->p.radius, sb)) continue;
        f.strip = strip;
        for (int rep = 0; rep < 3; ++rep) {
            float ms = 0;
            s = time_ms(c, [&] {
                return launch_colbox(c->sum_bits, f, c->stream) == cudaSuccess ? BUNDLE_OK : BUNDLE_ECUDA;
            }, &ms);
            if (s != BUNDLE_OK) return s;
            if (ms < best_col_ms) {
                best_col_ms = ms;
                best_strip = strip;
            }
        }
    }
    // the banded path replaces both passes: timed as a pair against the best pair above
    if (rowbox_mode_valid(4, c->W, c->H, c->p.radius)) {
        f.row_mode = 4;
        for (int rep = 0; rep < 3; ++rep) {
            float ms = 0;
            s = time_ms(c, [&] {
                return launch_rowbox(c->sum_bits, f, c->stream) == cudaSuccess &&
                               launch_colbox(c->sum_bits, f, c->stream) == cudaSuccess
                           ? BUNDLE_OK
                           : BUNDLE_ECUDA;
            }, &ms);
            if (s != BUNDLE_OK) return s;
            if (ms < best_row_ms + best_col_ms) {
                best_row_ms = ms;
                best_col_ms = 0;
                best_row = 4;
            }
        }
    }
    c->row_mode = best_row;
    c->col_strip = best_strip;
    return BUNDLE_OK;
}

// Back to the state bundle_init leaves, with the straight edges in blocks of eb.
static bundle_status probe_end(bundle_ctx* c, const TuneProbe& t, int32_t eb) {
    bundle_status s = probe_layout(c, t, eb);
    if (s != BUNDLE_OK) return s;
    const size_t C = (size_t)c->G * c->H * c->W;
    CUDA_TRY(&c->err, cudaMemsetAsync(c->hist, 0, C * kHistCopies * sizeof(uint32_t), c->stream));
    CUDA_TRY(&c->err, cudaMemsetAsync(c->counters, 0, 4 * sizeof(unsigned long long), c->stream));
    CUDA_TRY(&c->err, cudaMemsetAsync(c->d_flag, 0, sizeof(int32_t), c->stream));
    if (c->ink)
        CUDA_TRY(&c->err, cudaMemsetAsync(c->ink, 0, 2 * sizeof(unsigned long long) *
                                                         BUNDLE_INK_STATS_CAP, c->stream));
    CUDA_TRY(&c->err, cudaStreamSynchronize(c->stream));
    c->cur_P = 0;
    c->cur_R = -1;
    c->have_density = false;
    c->ev_used = 0;
    c->ev_kind.clear();
    for (cudaGraphExec_t& g : c->gexec)  // captured with the old tiles
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return BUNDLE_OK;
}

// One graph: every eb candidate lays the straight edges out again, resamples, splats and
// filters them, and the fused step is timed (best of two); then the filter tiles.
static bundle_status autotune_one(bundle_ctx* c) {
    DeviceGuard dg(c->device);
    TuneProbe t;
    bundle_status s = probe_begin(c, &t);
    if (s != BUNDLE_OK) return s;
    int32_t best_eb = c->eb;
    float best = 3.4e38f;
    for (int32_t eb = 4; eb <= kMaxEdgesPerWarp; eb *= 2) {
        for (int rep = 0; rep < 2; ++rep) {
            if ((s = probe_layout(c, t, eb)) != BUNDLE_OK || (s = probe_prefix(c)) != BUNDLE_OK)
                return s;
            float ms = 0;
            if ((s = time_ms(c, [&] { return probe_step(c); }, &ms)) != BUNDLE_OK) return s;
            if (ms < best) {
                best = ms;
                best_eb = eb;
            }
        }
    }
    if ((s = tune_filter(c)) != BUNDLE_OK) return s;
    return probe_end(c, t, best_eb);
}

// A batch runs its graphs side by side, so the block size is chosen for the whole batch:
// each policy (every graph at its size rule, or every graph at 4, 8, 16 or 32 edges
// per block) times the fused step of all graphs together, forked from the batch stream
// and joined back (best of two). The filter tiles are then tuned per graph.
static bundle_status autotune_batch(bundle_ctx* c) {
    DeviceGuard dg(c->device);
    const size_t n = c->members.size();
    std::vector<TuneProbe> t(n);
    std::vector<int32_t> rule(n);
    bundle_status s;
    for (size_t k = 0; k < n; ++k) {
        if ((s = probe_begin(c->members[k], &t[k])) != BUNDLE_OK)
            return fail(&c->err, s, "graph %zu: %s", k, c->members[k]->err.c_str());
        rule[k] = c->members[k]->eb;
    }
    int best_policy = 0;
    float best = 3.4e38f;
    for (int policy = 0; policy <= 4; ++policy) {  // 0: size rule, 1..4: 4 << (policy - 1)
        for (int rep = 0; rep < 2; ++rep) {
            for (size_t k = 0; k < n; ++k) {
                bundle_ctx* m = c->members[k];
                const int32_t eb = policy == 0 ? rule[k] : (4 << (policy - 1));
                if ((s = probe_layout(m, t[k], eb)) != BUNDLE_OK || (s = probe_prefix(m)) != BUNDLE_OK)
                    return s;
            }
            for (bundle_ctx* m : c->members) CUDA_TRY(&c->err, cudaStreamSynchronize(m->stream));
            float ms = 0;
            s = time_ms(c, [&] {
                bundle_status r = batch_fork(c, c->stream);
                for (size_t k = 0; k < n && r == BUNDLE_OK; ++k) r = probe_step(c->members[k]);
                return r == BUNDLE_OK ? batch_join(c, c->stream) : r;
            }, &ms);
            if (s != BUNDLE_OK) return s;
            if (ms < best) {
                best = ms;
                best_policy = policy;
            }
        }
    }
    for (size_t k = 0; k < n; ++k) {
        bundle_ctx* m = c->members[k];
        if ((s = tune_filter(m)) != BUNDLE_OK) return s;
        const int32_t eb = best_policy == 0 ? rule[k] : (4 << (best_policy - 1));
        if ((s = probe_end(m, t[k], eb)) != BUNDLE_OK) return s;
    }
    for (cudaGraphExec_t& g : c->bexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return BUNDLE_OK;
}

bundle_status bundle_set_tiles(bundle_ctx* c, int32_t eb, int32_t row_mode, int32_t col_strip) {
    if (!c) return BUNDLE_EINVAL;
    if (!c->members.empty() || c->is_member)
        return fail(&c->err, BUNDLE_ESTATE, "bundle_set_tiles: set the tiles of single contexts");
    if (eb != 0 && (eb < 4 || eb > kMaxEdgesPerWarp || (eb & (eb - 1)) != 0))
        return fail(&c->err, BUNDLE_EINVAL, "bundle_set_tiles: eb must be 0, 4, 8, 16 or 32");
    if (!rowbox_mode_valid(row_mode, c->W, c->H, c->p.radius))
        return fail(&c->err, BUNDLE_EINVAL, "bundle_set_tiles: row variant %d does not exist for "
                    "width %d", row_mode, c->W);
    if (col_strip != 0 && !colbox_strip_valid(col_strip, c->W, c->H, c->p.radius, c->sum_bits / 8))
        return fail(&c->err, BUNDLE_EINVAL, "bundle_set_tiles: strip %d does not fit height %d",
                    col_strip, c->H);
    if (eb != 0 && eb != c->eb) {
        if (!c->straight || c->iteration != 0 || c->cur_R >= 0)
            return fail(&c->err, BUNDLE_ESTATE,
                        "bundle_set_tiles: eb can change only on a context fresh from bundle_init");
        DeviceGuard dg(c->device);
        float2* keep = nullptr;
        CUDA_TRY(&c->err, cudaMalloc(&keep, (size_t)c->E * 2 * sizeof(float2)));
        cudaError_t e = launch_relayout_pairs(c->pts[c->cur_P], c->eb, c->cap, keep, 1, 2, nullptr,
                                              c->E, c->stream);
        if (e == cudaSuccess)
            e = launch_relayout_pairs(keep, 1, 2, c->pts[0], eb, c->cap, c->cnt[0], c->E, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(keep);
        CUDA_TRY(&c->err, e);
        c->eb = eb;
        c->n_blocks = (c->E + eb - 1) / eb;
        c->cur_P = 0;
    }
    c->row_mode = row_mode;
    c->col_strip = col_strip;
    for (cudaGraphExec_t& g : c->gexec)  // captured with the old tiles
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return BUNDLE_OK;
}

bundle_status bundle_autotune(bundle_ctx* c) {
    if (!c) return BUNDLE_EINVAL;
    if (c->is_member)
        return fail(&c->err, BUNDLE_ESTATE, "bundle_autotune: tune the batch, not its member");
    if (c->members.empty()) return autotune_one(c);
    if (c->iteration != 0)
        return fail(&c->err, BUNDLE_ESTATE, "bundle_autotune: the batch has already iterated");
    return autotune_batch(c);
}

// Deferred device-side errors (segment histogram overflow). Synchronises the stream.
static bundle_status check_device_flag(bundle_ctx* c) {
    if (!c->d_flag) return BUNDLE_OK;
    int32_t f = 0;
    CUDA_TRY(&c->err, cudaMemcpyAsync(&f, c->d_flag, sizeof f, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(&c->err, cudaStreamSynchronize(c->stream));
    if (f == 2)
        return fail(&c->err, BUNDLE_ETIMEOUT,
                    "a tensor-memory copy of the column pass did not complete in time");
    if (f)
        return fail(&c->err, BUNDLE_EOVERFLOW,
                    "segment histogram mass exceeded %llu: the int64 smoothed sums could wrap",
                    c->mass_allowed);
    return BUNDLE_OK;
}

bundle_status bundle_fetch_ink(bundle_ctx* c, int64_t* out, int32_t first, int32_t n) {
    if (!c) return BUNDLE_EINVAL;
    if (!c->members.empty() || !c->ink)
        return fail(&c->err, BUNDLE_ESTATE,
                    "bundle_fetch_ink: the context was not created with BUNDLE_FLAG_INK_STATS "
                    "(a batch records per member)");
    if (!out || first < 0 || n < 0 || (int64_t)first + n > c->iteration ||
        (int64_t)first + n > BUNDLE_INK_STATS_CAP)
        return fail(&c->err, BUNDLE_EINVAL,
                    "bundle_fetch_ink: iterations [%d, %d) outside the record [0, %d)", first,
                    first + n, std::min<int32_t>(c->iteration, BUNDLE_INK_STATS_CAP));
    if (n == 0) return BUNDLE_OK;
    DeviceGuard dg(c->device);
    if (bundle_status fs = check_device_flag(c)) return fs;
    CUDA_TRY(&c->err, cudaMemcpyAsync(out, c->ink + 2 * (size_t)first,
                                      2 * sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost,
                                      c->stream));
    CUDA_TRY(&c->err, cudaStreamSynchronize(c->stream));
    return BUNDLE_OK;
}

bundle_status bundle_render(bundle_ctx* c, const bundle_render_params* rp,
                            const uint8_t* palette, uint8_t* rgba, int64_t* accum,
                            int32_t flags) {
    if (!c) return BUNDLE_EINVAL;
    if (!c->members.empty())
        return fail(&c->err, BUNDLE_ESTATE, "render a batch's graphs through bundle_batch_member");
    if (!rp || !palette || !rgba)
        return fail(&c->err, BUNDLE_EINVAL, "bundle_render: params, palette and rgba are required");
    if (rp->scale < 1 || rp->scale > 16 || !(rp->alpha > 0.0f && rp->alpha < 1.0f) ||
        !(rp->width_min >= 1.0f) || !(rp->width_max >= rp->width_min) ||
        !(rp->width_max <= 64.0f) || !std::isfinite(rp->rho_ref) ||
        (rp->log_width != 0 && rp->log_width != 1))
        return fail(&c->err, BUNDLE_EINVAL,
                    "bundle_render: need 1 <= scale <= 16, 0 < alpha < 1, "
                    "1 <= width_min <= width_max <= 64, finite rho_ref, log_width 0 or 1");
    const int64_t Wi = (int64_t)c->W * rp->scale, Hi = (int64_t)c->H * rp->scale;
    if (Wi * Hi > ((int64_t)1 << 28) || (int64_t)c->G * Wi * Hi > ((int64_t)1 << 30))
        return fail(&c->err, BUNDLE_EINVAL,
                    "bundle_render: image of %lld x %lld pixels x %d bins is too large "
                    "(at most 2^28 pixels and 2^30 depth cells)",
                    (long long)Wi, (long long)Hi, c->G);
    if (!c->have_density)
        return fail(&c->err, BUNDLE_ESTATE, "bundle_render: run an iteration first (no density)");
    DeviceGuard dg(c->device);
    if (bundle_status fs = check_device_flag(c)) return fs;
    const bool dev = (flags & BUNDLE_FETCH_DEVICE) != 0;
    const int64_t npx = Wi * Hi;
    unsigned long long* depth = nullptr;
    int32_t* d_pal = nullptr;
    unsigned int* d_ref = nullptr;
    void* d_rgba = nullptr;
    void* d_acc = nullptr;
    auto cleanup = [&] {
        cudaStreamSynchronize(c->stream);
        cudaFree(depth);
        cudaFree(d_pal);
        cudaFree(d_ref);
        if (!dev) {
            cudaFree(d_rgba);
            cudaFree(d_acc);
        }
    };
    std::vector<int32_t> pal((size_t)c->G * 3);
    for (size_t i = 0; i < pal.size(); ++i) pal[i] = palette[i];
    const float ref = rp->rho_ref > 0.0f ? rp->rho_ref : 0.0f;
    unsigned int ref_bits;
    std::memcpy(&ref_bits, &ref, sizeof ref_bits);
    cudaError_t e = cudaMalloc(&depth, (size_t)c->G * npx * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_pal, pal.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_ref, sizeof(unsigned int));
    if (e == cudaSuccess) {
        if (dev) {
            d_rgba = rgba;
            d_acc = accum;
        } else {
            e = cudaMalloc(&d_rgba, (size_t)npx * 4);
            if (e == cudaSuccess && accum) e = cudaMalloc(&d_acc, (size_t)npx * 32);
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(depth, 0, (size_t)c->G * npx * 8, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_pal, pal.data(), pal.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ref, &ref_bits, sizeof ref_bits, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        RenderArgs a{};
        a.cnt = c->cnt[c->cur_P];
        a.pts = c->pts[c->cur_P];
        a.group = c->group;
        a.weight = c->weight;
        a.quads = c->quads;
        a.depth = depth;
        a.rho_ref = d_ref;
        a.E = c->E;
        a.eb = c->eb;
        a.cap = c->cap;
        a.W = c->W;
        a.H = c->H;
        a.G = c->G;
        a.scale = rp->scale;
        a.Wi = (int32_t)Wi;
        a.Hi = (int32_t)Hi;
        a.tau1 = (unsigned long long)std::llround(-std::log1p(-(double)rp->alpha) * 1048576.0);
        a.width_min = rp->width_min;
        a.width_max = rp->width_max;
        a.log_width = rp->log_width;
        int n_sm = 0;
        e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device);
        if (e == cudaSuccess && !(rp->rho_ref > 0.0f))
            e = launch_rho_from_quads(c->p.rho_dtype, filter_args(c), c->stream);
        if (e == cudaSuccess)
            e = launch_render(c->p.rho_dtype, a, c->rho, (int64_t)c->G * c->H * c->W,
                              !(rp->rho_ref > 0.0f), n_sm, c->stream);
    }
    if (e == cudaSuccess)
        e = launch_render_resolve(depth, c->G, npx, d_pal, rp->background, d_rgba, d_acc,
                                  c->stream);
    if (e == cudaSuccess && !dev)
        e = cudaMemcpyAsync(rgba, d_rgba, (size_t)npx * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && !dev && accum)
        e = cudaMemcpyAsync(accum, d_acc, (size_t)npx * 32, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cleanup();
    if (e != cudaSuccess)
        return fail(&c->err, e == cudaErrorMemoryAllocation ? BUNDLE_ENOMEM : BUNDLE_ECUDA,
                    "bundle_render: %s", cudaGetErrorString(e));
    return BUNDLE_OK;
}

bundle_status bundle_sync(bundle_ctx* c) {
    if (!c) return BUNDLE_EINVAL;
    DeviceGuard dg(c->device);
    for (bundle_ctx* m : c->members) CUDA_TRY(&c->err, cudaStreamSynchronize(m->stream));
    CUDA_TRY(&c->err, cudaStreamSynchronize(c->stream));
    CUDA_TRY(&c->err, cudaGetLastError());
    for (bundle_ctx* m : c->members) {
        bundle_status s = check_device_flag(m);
        if (s != BUNDLE_OK) return fail(&c->err, s, "%s", m->err.c_str());
    }
    return check_device_flag(c);
}

bundle_status bundle_fetch(bundle_ctx* c, int64_t* off, float* xy, int64_t cap,
                           int64_t* n_points, int32_t flags) {
    if (!c) return BUNDLE_EINVAL;
    if (!c->members.empty())
        return fail(&c->err, BUNDLE_ESTATE, "fetch a batch's graphs through bundle_batch_member");
    if (!off || !n_points) return fail(&c->err, BUNDLE_EINVAL, "off and n_points are required");
    int sel = c->cur_P;
    if (flags & BUNDLE_FETCH_RESAMPLED) {
        if (c->cur_R < 0)
            return fail(&c->err, BUNDLE_ESTATE, "no iteration has run: nothing was resampled");
        sel = c->cur_R;
    }
    DeviceGuard dg(c->device);
    if (bundle_status fs = check_device_flag(c)) return fs;
    const bool dev = (flags & BUNDLE_FETCH_DEVICE) != 0;
    const bool pix = (flags & BUNDLE_FETCH_PIXELS) != 0;
    CUDA_TRY(&c->err, launch_counts_to_caller(c->perm, c->cnt[sel], c->E, c->fetch_off, c->stream));
    CUDA_TRY(&c->err, launch_scan_offsets(c->fetch_off, c->E, c->fetch_tmp, c->stream));
    int64_t N = 0;
    CUDA_TRY(&c->err, cudaMemcpyAsync(&N, c->fetch_off + c->E, sizeof N, cudaMemcpyDeviceToHost,
                                      c->stream));
    CUDA_TRY(&c->err, cudaStreamSynchronize(c->stream));
    *n_points = N;
    if (dev) {
        CUDA_TRY(&c->err, cudaMemcpyAsync(off, c->fetch_off, (size_t)(c->E + 1) * 8,
                                          cudaMemcpyDeviceToDevice, c->stream));
    } else {
        CUDA_TRY(&c->err, cudaMemcpyAsync(off, c->fetch_off, (size_t)(c->E + 1) * 8,
                                          cudaMemcpyDeviceToHost, c->stream));
    }
    if (xy) {
        if (cap < N) {
            cudaStreamSynchronize(c->stream);
            return fail(&c->err, BUNDLE_EINVAL, "xy holds %lld points, %lld needed",
                        (long long)cap, (long long)N);
        }
        float2* target = reinterpret_cast<float2*>(xy);
        if (!dev) {
            if (c->fetch_xy_cap < N) {
                if (c->fetch_xy) {
                    cudaFree(c->fetch_xy);
                    c->device_bytes -= c->fetch_xy_cap * 8;
                }
                c->fetch_xy = nullptr;
                c->fetch_xy_cap = 0;
                CUDA_TRY(&c->err, dalloc(c, &c->fetch_xy, (size_t)N));
                c->fetch_xy_cap = N;
            }
            target = c->fetch_xy;
        }
        const double inv = 1.0 / c->map[2];
        CUDA_TRY(&c->err, launch_layout_to_caller(c->perm, c->cnt[sel], c->pts[sel], c->E, c->eb, c->cap,
                                                  c->fetch_off, target, pix ? 0 : 1,
                                                  (float)c->map[3], (float)c->map[4], (float)inv,
                                                  (float)c->map[0], (float)c->map[1], c->stream));
        if (!dev)
            CUDA_TRY(&c->err, cudaMemcpyAsync(xy, target, (size_t)N * 8, cudaMemcpyDeviceToHost,
                                              c->stream));
    }
    CUDA_TRY(&c->err, cudaStreamSynchronize(c->stream));
    return BUNDLE_OK;
}

bundle_status bundle_fetch_density(bundle_ctx* c, int32_t which, void* dst, int64_t dst_bytes,
                                   int32_t flags) {
    if (!c) return BUNDLE_EINVAL;
    if (!c->members.empty())
        return fail(&c->err, BUNDLE_ESTATE, "fetch a batch's graphs through bundle_batch_member");
    if (!dst) return fail(&c->err, BUNDLE_EINVAL, "dst is NULL");
    if (!c->have_density && !(which == BUNDLE_DENSITY_HIST && c->split_state == 1))
        return fail(&c->err, BUNDLE_ESTATE, "no iteration has run");
    const size_t C = (size_t)c->G * c->H * c->W;
    const void* src;
    size_t bytes;
    switch (which) {
        case BUNDLE_DENSITY_HIST: src = c->hist; bytes = C * 4; break;
        case BUNDLE_DENSITY_SUMS: src = c->S; bytes = C * (c->sum_bits / 8); break;
        case BUNDLE_DENSITY_RHO: src = c->rho; bytes = C * rho_bytes(c->p.rho_dtype); break;
        default: return fail(&c->err, BUNDLE_EINVAL, "unknown density selector %d", which);
    }
    if (dst_bytes < (int64_t)bytes)
        return fail(&c->err, BUNDLE_EINVAL, "dst holds %lld bytes, %zu needed",
                    (long long)dst_bytes, bytes);
    DeviceGuard dg(c->device);
    if (bundle_status fs = check_device_flag(c)) return fs;
    if (which == BUNDLE_DENSITY_HIST)
        CUDA_TRY(&c->err, launch_fold_hist(c->hist, (int64_t)C, kHistCopies, c->stream));
    if (which == BUNDLE_DENSITY_RHO)
        CUDA_TRY(&c->err, launch_rho_from_quads(c->p.rho_dtype, filter_args(c), c->stream));
    CUDA_TRY(&c->err, cudaMemcpyAsync(dst, src, bytes,
                                      (flags & BUNDLE_FETCH_DEVICE) ? cudaMemcpyDeviceToDevice
                                                                    : cudaMemcpyDeviceToHost,
                                      c->stream));
    CUDA_TRY(&c->err, cudaStreamSynchronize(c->stream));
    return BUNDLE_OK;
}

bundle_status bundle_get_info(const bundle_ctx* c, bundle_info* out) {
    if (!c || !out) return BUNDLE_EINVAL;
    if (!c->members.empty()) {
        // a batch reports the sums over its graphs; sizes and map are those of graph 0
        bundle_status s = bundle_get_info(c->members[0], out);
        if (s != BUNDLE_OK) return s;
        for (size_t k = 1; k < c->members.size(); ++k) {
            bundle_info mi;
            if ((s = bundle_get_info(c->members[k], &mi)) != BUNDLE_OK) return s;
            out->n_edges += mi.n_edges;
            out->n_points += mi.n_points;
            out->n_points_resampled += mi.n_points_resampled;
            out->device_bytes += mi.device_bytes;
            out->points_processed += mi.points_processed;
        }
        out->iteration = c->iteration;
        return BUNDLE_OK;
    }
    bundle_ctx* m = const_cast<bundle_ctx*>(c);
    DeviceGuard dg(c->device);
    std::memset(out, 0, sizeof *out);
    out->n_edges = c->E;
    out->grid_w = c->W;
    out->grid_h = c->H;
    out->n_groups = c->G;
    out->sum_bits = c->sum_bits;
    out->rho_dtype = c->p.rho_dtype;
    out->iteration = c->iteration;
    std::memcpy(out->map, c->map, sizeof c->map);
    out->h_next = bandwidth(c->p, c->iteration);
    out->device_bytes = c->device_bytes;
    out->tile_eb = c->eb;
    out->tile_row = c->row_mode;
    out->tile_strip = c->col_strip;
    unsigned long long tot[2] = {0, 0};
    int sels[2] = {c->cur_P, c->cur_R};
    for (int k = 0; k < 2; ++k) {
        if (sels[k] < 0) continue;
        if (cudaMemsetAsync(m->counters + 1, 0, 8, c->stream) != cudaSuccess) return BUNDLE_ECUDA;
        if (launch_sum_counts(c->cnt[sels[k]], c->E, m->counters + 1, c->stream) != cudaSuccess)
            return BUNDLE_ECUDA;
        if (cudaMemcpyAsync(&tot[k], m->counters + 1, 8, cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return BUNDLE_ECUDA;
    }
    out->n_points = (int64_t)tot[0];
    out->n_points_resampled = (int64_t)tot[1];
    unsigned long long done = 0;
    if (cudaMemcpyAsync(&done, m->counters, 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return BUNDLE_ECUDA;
    out->points_processed = (int64_t)done;
    return BUNDLE_OK;
}

bundle_status bundle_set_interaction(bundle_ctx* c, const int64_t* num, int64_t den) {
    if (!c) return BUNDLE_EINVAL;
    if (!c->members.empty() || c->is_member)
        return fail(&c->err, BUNDLE_EINVAL, "the interaction matrix applies to single-graph contexts");
    if (!num || den <= 0) return fail(&c->err, BUNDLE_EINVAL, "need num and den > 0");
    const int G = c->G;
    double worst = 0;
    for (int l = 0; l < G; ++l) {
        double row = 0;
        for (int b = 0; b < G; ++b) row += std::fabs((double)num[l * G + b]);
        worst = std::max(worst, row);
    }
    if (!(worst * c->sum_bound < 9223372036854775808.0 * (1 - 1e-12)))
        return fail(&c->err, BUNDLE_EOVERFLOW,
                    "interaction bound %.6g x %.6g does not fit int64", worst, c->sum_bound);
    double sk = 1;
    const double s = (double)(2 * c->p.radius + 1) * (double)(2 * c->p.radius + 1);
    for (int p = 0; p < c->p.passes; ++p) sk *= s;
    DeviceGuard dg(c->device);
    if (!c->mix) CUDA_TRY(&c->err, dalloc(c, &c->mix, (size_t)G * G));
    CUDA_TRY(&c->err, cudaMemcpyAsync(c->mix, num, (size_t)G * G * sizeof(int64_t),
                                      cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(&c->err, cudaStreamSynchronize(c->stream));
    c->den_f = (float)((double)den * sk);
    for (cudaGraphExec_t& g : c->gexec)  // captured with the previous mix
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return BUNDLE_OK;
}

bundle_status bundle_profile_enable(bundle_ctx* c, int32_t on) {
    if (!c) return BUNDLE_EINVAL;
    c->prof = on != 0;
    return BUNDLE_OK;
}

bundle_status bundle_profile_read(bundle_ctx* c, double* ms, int64_t* launches, int32_t n,
                                  int32_t reset) {
    if (!c) return BUNDLE_EINVAL;
    if (n < 0 || (n > 0 && (!ms || !launches)))
        return fail(&c->err, BUNDLE_EINVAL, "ms and launches must hold n entries");
    DeviceGuard dg(c->device);
    CUDA_TRY(&c->err, cudaStreamSynchronize(c->stream));
    for (int32_t k = 0; k < n; ++k) {
        ms[k] = 0;
        launches[k] = 0;
    }
    for (size_t r = 0; r < c->ev_kind.size(); ++r) {
        float t = 0;
        CUDA_TRY(&c->err, cudaEventElapsedTime(&t, c->ev_pool[2 * r], c->ev_pool[2 * r + 1]));
        int k = c->ev_kind[r];
        if (k < n) {
            ms[k] += t;
            launches[k] += 1;
        }
    }
    if (reset) {
        c->ev_kind.clear();
        c->ev_used = 0;
    }
    return BUNDLE_OK;
}

void bundle_destroy(bundle_ctx* c) {
    if (c && c->is_member) return;  // members belong to their batch
    free_ctx(c);
}

const char* bundle_last_error(const bundle_ctx* c) {
    return c ? c->err.c_str() : g_init_error.c_str();
}

const char* bundle_status_string(bundle_status s) {
    switch (s) {
        case BUNDLE_OK: return "BUNDLE_OK";
        case BUNDLE_EINVAL: return "BUNDLE_EINVAL";
        case BUNDLE_ENOMEM: return "BUNDLE_ENOMEM";
        case BUNDLE_ECUDA: return "BUNDLE_ECUDA";
        case BUNDLE_EOVERFLOW: return "BUNDLE_EOVERFLOW";
        case BUNDLE_ETIMEOUT: return "BUNDLE_ETIMEOUT";
        case BUNDLE_ESTATE: return "BUNDLE_ESTATE";
        case BUNDLE_ENOTSUP: return "BUNDLE_ENOTSUP";
    }
    return "BUNDLE_UNKNOWN";
}

}  // extern "C"
