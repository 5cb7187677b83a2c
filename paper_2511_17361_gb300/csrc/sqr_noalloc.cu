// sqr_noalloc.cu -- sq_render_fwd_noalloc: the forward render for callers that
// cannot allocate device memory when they render, and have no workspace of their
// own to lend the library.  Typical cases: a real-time perception loop that forbids
// allocation after start-up (cudaMalloc can block and synchronise the whole
// device), or a host framework / plugin interface that owns every device buffer
// and passes the library only its inputs and outputs.
//
// The scratch the forward needs (packed primitive records, padded logits, the
// ray work counter) lives in the file-scope array g_noalloc_scratch below, sized
// for SQ_NOALLOC_MAX_PRIMS primitives and SQ_MAX_CLASSES classes.  Every device
// that loads the library holds that array until the process exits.  Its device
// address is looked up with cudaGetSymbolAddress once per device, on the first
// call made while that device is current (host code must not use the symbol
// name itself as a device pointer).  All calls share the one array: two calls
// that overlap on the GPU (different streams, or the same stream from different
// host threads without ordering) race on it.  The counter that must start at zero
// is cleared by every call, on the caller's stream.
#include <mutex>

#include "sqr_common.cuh"

namespace sqr {
size_t render_workspace_size(const sq_prims_t* p);
sq_status_t render_fwd_impl(const sq_prims_t*, const sq_index_t*, const sq_grid_t*, const sq_rays_t*, float*, float*,
                            float*, void*, size_t, void*, size_t, cudaStream_t);
}  // namespace sqr

namespace {

// Per primitive the render workspace holds 64 B of record, 48 B of backward
// extras, 4 * 32 B of padded logits, 192 B of gradient accumulator and 16 B of
// packed box; plus a header (scene descriptors, ray offsets, work counter) and
// alignment padding, covered by the 64 KB allowance.
constexpr size_t kNoallocBytes = (size_t)SQ_NOALLOC_MAX_PRIMS * (64 + 48 + 4 * 32 + 192 + 16) + 64 * 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
sq_status_t noalloc_scratch(void** ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return sqr::cuda_status(e, "sq_render_fwd_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        sqr::set_last_error("sq_render_fwd_noalloc: device ordinal %d beyond %d", dev, kMaxDevices);
        return SQ_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return sqr::cuda_status(e, "sq_render_fwd_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
    return SQ_OK;
}

}  // namespace

extern "C" sq_status_t sq_render_fwd_noalloc(const sq_prims_t* prims, const sq_index_t* index, const sq_grid_t* grid,
                                             const sq_rays_t* rays, float* depth, float* sem, float* t_final,
                                             void* stream) {
    using namespace sqr;
    sq_status_t s;
    if ((s = check_prims(prims)) != SQ_OK) return s;
    if ((s = check_grid(grid)) != SQ_OK) return s;
    if ((s = check_index(index, grid, prims->n)) != SQ_OK) return s;
    if ((s = check_rays(rays)) != SQ_OK) return s;
    if ((long long)rays->n_cam * rays->H * rays->W > 0 && (!depth || !sem)) {
        set_last_error("sq_render_fwd_noalloc: depth/sem output is NULL");
        return SQ_ERR_INVALID_ARG;
    }
    if (prims->n > SQ_NOALLOC_MAX_PRIMS) {
        set_last_error("sq_render_fwd_noalloc: %d superquadrics exceed the built-in scratch limit of %d; "
                       "use sq_render_fwd with a caller-provided workspace",
                       prims->n, SQ_NOALLOC_MAX_PRIMS);
        return SQ_ERR_INVALID_ARG;
    }
    const size_t need = render_workspace_size(prims);
    if (need > kNoallocBytes) {
        set_last_error("sq_render_fwd_noalloc: needs %zu bytes of scratch, %zu built in", need, kNoallocBytes);
        return SQ_ERR_INVALID_ARG;
    }
    void* scratch = nullptr;
    if ((s = noalloc_scratch(&scratch)) != SQ_OK) return s;
    return render_fwd_impl(prims, index, grid, rays, depth, sem, t_final, nullptr, 0, scratch, kNoallocBytes,
                           (cudaStream_t)stream);
}
