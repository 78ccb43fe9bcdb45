// cr_noalloc.cu -- cr_persistence_noalloc: the persistence of one 1D/2D image
// for callers that cannot hand the library a device workspace.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's fixed device-memory pool (inference plugins, embedded hosts),
// where allocating would break the host's memory accounting or synchronise
// the device at a point the host forbids.  They still own their input and
// output buffers; this entry point gives them a workspace that needs no
// allocation call: a file-scope static device array, reserved when the
// module is loaded.  Every GPU that loads the library holds it until the
// process exits.
#include "cr_internal.cuh"
#include <mutex>

#define CR_NOALLOC_BYTES_ (64ull << 20)

// the shared scratch: one per device, reused by every call on that device
static __device__ __align__(256) unsigned char g_cr_noalloc_scratch[CR_NOALLOC_BYTES_];

namespace {
constexpr int kMaxDevices = 256;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Host code cannot use the symbol itself as a device address: it is a
// host-side stand-in.  Resolve the real address once per device, with that
// device current.
int scratch_for_current_device(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CR_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_cr_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return CR_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return CR_OK;
}
}  // namespace

extern "C" int cr_persistence_noalloc(const float *img, int ndim, const int64_t *shape, int maxdim,
                                      cr_pair *pairs_out, int64_t capacity, int64_t *n_pairs, cr_stream_t stream,
                                      uint32_t flags) {
    if (!img || !shape || !n_pairs || ndim < 1 || ndim > 3) return CR_ERR_INVALID_ARG;
    // volumes need the reduction scratch of the middle dimension: not served here
    for (int d = 0; d + 2 < ndim; d++)
        if (shape[d] > 1) return CR_ERR_INVALID_ARG;
    size_t need = 0;
    int rc = cr::workspace_size_serial(ndim, shape, maxdim, flags, &need);
    if (rc) return rc;
    if (need > CR_NOALLOC_BYTES_) return CR_ERR_TOO_LARGE;
    void *ws = nullptr;
    rc = scratch_for_current_device(&ws);
    if (rc) return rc;
    // every buffer the pipeline relies on being zero is cleared by the pipeline itself
    return cr::persistence_serial(img, ndim, shape, maxdim, pairs_out, capacity, n_pairs, ws,
                                  (size_t)CR_NOALLOC_BYTES_, (cudaStream_t)stream, flags);
}
