// Allocation-free form of the box-pass smoothing (k row passes, then k column
// passes). The row passes need an intermediate stack as large as the input;
// here it lives in one fixed device array declared at file scope, so the entry
// point never calls cudaMalloc or cudaFree.
//
// Who needs this: code that runs where the device allocator is off limits --
// inside a framework whose caching allocator owns every device byte, in a
// service that reserved its whole memory budget up front, or on a path that
// must not risk the implicit device synchronisation cudaMalloc and cudaFree can
// cause. Such callers hand in the histogram and the output buffer and get the
// smoothed sums back without the library allocating anything.
#include <mutex>

#include "../../include/bundle.h"
#include "internal.cuh"

namespace {

// Largest intermediate the array holds: 16 MiB, i.e. groups * height * width
// cells of 8 bytes (64-bit sums) or 4 bytes (32-bit sums). Every GPU that
// loads the library keeps this array until the process exits.
constexpr size_t kScratchBytes = size_t(16) << 20;
__device__ __align__(256) unsigned long long g_smooth_scratch[kScratchBytes / 8];

// In host code the array's name is only a host-side stand-in; the device
// address comes from cudaGetSymbolAddress, taken with the device current and
// cached per device together with the id of the CUDA context it was taken in.
// A context created after a reset of the device (cudaDeviceReset, or a
// framework resetting the primary context) has a new id, so the address is
// looked up again there instead of reusing one that belonged to the old one.
constexpr int kMaxDevices = 128;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Id of the calling thread's current context (driver entry points fetched
// through the runtime, so the library does not link the driver library).
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

cudaError_t current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                         cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorSymbolNotFound;
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return cudaErrorDeviceUninitialized;
    if (get_id(ctx, id) != 0) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

cudaError_t scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    unsigned long long id = 0;
    if (g_scratch_addr[dev] && current_context_id(&id) == cudaSuccess && g_scratch_ctx[dev] == id) {
        *out = g_scratch_addr[dev];
        return cudaSuccess;
    }
    // (the runtime makes the device's context current here if nothing did before)
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_smooth_scratch);
    if (e != cudaSuccess) return e;
    if ((e = current_context_id(&id)) != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = id;
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" bundle_status bundle_smooth_noalloc(const uint32_t* hist, void* sums,
                                               int32_t n_groups, int32_t grid_h,
                                               int32_t grid_w, int32_t radius, int32_t passes,
                                               int32_t sum_bits, void* stream) {
    if (!hist || !sums) {
        heb::set_thread_error("bundle_smooth_noalloc: hist and sums must be device pointers");
        return BUNDLE_EINVAL;
    }
    if (n_groups < 1 || n_groups > 64 || grid_h < 2 || grid_w < 2 || grid_h > 4096 ||
        grid_w > 4096 || radius < 1 || radius >= grid_h || radius >= grid_w || passes < 1 ||
        passes > 16 || (sum_bits != 32 && sum_bits != 64)) {
        heb::set_thread_error(
            "bundle_smooth_noalloc: need 1 <= n_groups <= 64, 2 <= H, W <= 4096, "
            "1 <= radius < min(H, W), 1 <= passes <= 16, sum_bits 32 or 64");
        return BUNDLE_EINVAL;
    }
    const size_t need = (size_t)n_groups * grid_h * grid_w * (size_t)(sum_bits / 8);
    if (need > kScratchBytes) {
        heb::set_thread_error(
            "bundle_smooth_noalloc: groups x height x width x sum bytes exceeds the 16 MiB "
            "fixed intermediate of the allocation-free entry point; use bundle_iterate");
        return BUNDLE_EINVAL;
    }
    // the launches and the scratch address belong to the current device: hist and sums
    // must live there
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        heb::set_thread_error("bundle_smooth_noalloc: no usable CUDA device");
        return BUNDLE_ECUDA;
    }
    void* Y = nullptr;
    if ((e = scratch_address(dev, &Y)) != cudaSuccess) {
        heb::set_thread_error("bundle_smooth_noalloc: device address of the fixed array not found");
        return BUNDLE_ECUDA;
    }
    heb::FilterArgs f{};
    f.hist = hist;
    f.hist_copies = 1;
    f.Y = Y;
    f.S = sums;
    f.G = n_groups;
    f.H = grid_h;
    f.W = grid_w;
    f.r = radius;
    f.passes = passes;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((e = heb::launch_rowbox(sum_bits, f, st)) != cudaSuccess ||
        (e = heb::launch_colbox(sum_bits, f, st)) != cudaSuccess) {
        heb::set_thread_error(cudaGetErrorString(e));
        return BUNDLE_ECUDA;
    }
    return BUNDLE_OK;
}
