// cr_f64.cu -- float64 input (the precision of the paper's timing study,
// whose datasets were converted to double, Sec. 3).  The filtration depends
// on the input only through the order of its values (Sec. 2: cells enter by
// value, ties by the fixed index order), so a float64 image is replaced by the
// image of its dense value ranks, stored as positive normal float32 bit
// patterns (0x00800000 + rank, whose float order is the rank order), the
// float32 path runs on that image unchanged, and the pairs' values are mapped
// back through the table of distinct values.
//
//   k_f64_keys     order-preserving 64-bit keys of the values (-0.0 = +0.0, NaN flagged)
//   radix sort     (key, voxel) pairs by key (the library's LSD sort, 8 passes)
//   k_f64_starts   1 where a run of equal keys starts; an exclusive scan counts them
//   k_f64_scatter  rank image and the table of distinct values
//   k_f64_pairs    cr_pair (rank values) -> cr_pair64 (float64 values)
#include "cr_internal.cuh"

namespace cr {

constexpr uint32_t F64_RANK_BASE = 0x00800000u;  // smallest positive normal float32

__device__ __forceinline__ uint64_t ord64(double d) {
    uint64_t b = (uint64_t)__double_as_longlong(d);
    if (b == 0x8000000000000000ull) b = 0ull;  // -0.0 is +0.0
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_f64_keys(const double *__restrict__ img, int64_t n, uint64_t *__restrict__ key,
                           uint32_t *__restrict__ idx, int *status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = img[i];
        if (v != v) set_status(status, CR_ERR_NAN);
        key[i] = ord64(v);
        idx[i] = (uint32_t)i;
    }
}

__global__ void k_f64_starts(const uint64_t *__restrict__ skey, int64_t n, uint32_t *__restrict__ start) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        start[i] = (i == 0 || skey[i] != skey[i - 1]) ? 1u : 0u;
}

// before[i] = number of runs starting before sorted position i
__global__ void k_f64_scatter(const uint64_t *__restrict__ skey, const uint32_t *__restrict__ sidx,
                              const uint32_t *__restrict__ before, int64_t n, const double *__restrict__ img,
                              float *__restrict__ rank_img, double *__restrict__ uniq) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const bool first = i == 0 || skey[i] != skey[i - 1];
        const uint32_t r = before[i] + (first ? 1u : 0u) - 1u;
        const uint32_t v = sidx[i];
        rank_img[v] = __uint_as_float(F64_RANK_BASE + r);
        if (first) {
            const double x = img[v];
            uniq[r] = x == 0.0 ? 0.0 : x;
        }
    }
}

__device__ __forceinline__ double f64_value(float rv, const double *uniq, int64_t nv, int *status) {
    if (isinf(rv)) return (double)rv;  // the death of an essential class
    const uint32_t b = __float_as_uint(rv);
    const int64_t r = (int64_t)b - (int64_t)F64_RANK_BASE;
    if (r < 0 || r >= nv) {
        set_status(status, CR_ERR_INTERNAL);
        return 0.0;
    }
    return uniq[r];
}

__global__ void k_f64_pairs(const cr_pair *__restrict__ in, int64_t n, const double *__restrict__ uniq, int64_t nv,
                            cr_pair64 *__restrict__ out, int *status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const cr_pair p = in[i];
        cr_pair64 q;
        q.dim = p.dim;
        q.flags = p.flags;
        q.birth = f64_value(p.birth, uniq, nv, status);
        q.death = f64_value(p.death, uniq, nv, status);
        q.birth_cell = p.birth_cell;
        q.death_cell = p.death_cell;
        out[i] = q;
    }
}

// The float64 extras at the front of the workspace (everything 256-aligned);
// the float32 path's workspace follows.
struct F64Layout {
    size_t rank, uniq, key, key_tmp, idx, idx_tmp, start, scan, sort, pairs, status, total;
};

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

static F64Layout f64_layout(int64_t nv, int64_t capacity) {
    F64Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += up256(bytes);
        return at;
    };
    L.rank = take((size_t)nv * 4);
    L.uniq = take((size_t)nv * 8);
    L.key = take((size_t)nv * 8);
    L.key_tmp = take((size_t)nv * 8);
    L.idx = take((size_t)nv * 4);
    L.idx_tmp = take((size_t)nv * 4);
    L.start = take((size_t)nv * 4);
    L.scan = take(scan_temp_bytes(nv));
    L.sort = take(radix_temp_bytes(nv));
    L.pairs = take((size_t)(capacity > 0 ? capacity : 1) * sizeof(cr_pair));
    L.status = take(sizeof(int));
    L.total = o;
    return L;
}

static int f64_voxels(int ndim, const int64_t *shape, int64_t &nv) {
    if (!shape || ndim < 1 || ndim > 3) return CR_ERR_INVALID_ARG;
    nv = 1;
    for (int d = 0; d < ndim; d++) {
        if (shape[d] < 1) return CR_ERR_INVALID_ARG;
        if (shape[d] > ((int64_t)1 << 31) || nv > (((int64_t)1 << 31) / shape[d])) return CR_ERR_TOO_LARGE;
        nv *= shape[d];
    }
    // the float32 path's own limit (3 * voxels < 2^32) also keeps every rank pattern
    // 0x00800000 + rank a finite positive float
    if (3 * nv >= ((int64_t)1 << 32)) return CR_ERR_TOO_LARGE;
    return CR_OK;
}

}  // namespace cr

extern "C" {

int cr_workspace_size_f64(int ndim, const int64_t *shape, int maxdim, uint32_t flags, int64_t capacity,
                          int typical, size_t *bytes) {
    if (!bytes || capacity < 0) return CR_ERR_INVALID_ARG;
    int64_t nv = 0;
    int rc = cr::f64_voxels(ndim, shape, nv);
    if (rc) return rc;
    size_t b32 = 0;
    rc = typical ? cr_workspace_size_typical(ndim, shape, maxdim, flags, &b32)
                 : cr_workspace_size(ndim, shape, maxdim, flags, &b32);
    if (rc) return rc;
    *bytes = cr::f64_layout(nv, capacity).total + b32;
    return CR_OK;
}

int cr_persistence_f64(const double *img, int ndim, const int64_t *shape, int maxdim, cr_pair64 *pairs_out,
                       int64_t capacity, int64_t *n_pairs, void *ws, size_t ws_bytes, cr_stream_t stream,
                       uint32_t flags) {
    using namespace cr;
    if (!img || !pairs_out || !n_pairs || !ws || capacity < 0) return CR_ERR_INVALID_ARG;
    if (int e = injected_error_before_gpu()) return e;
    int64_t nv = 0;
    int rc = f64_voxels(ndim, shape, nv);
    if (rc) return rc;
    const F64Layout L = f64_layout(nv, capacity);
    if (((uintptr_t)ws & 255u) != 0 || ws_bytes <= L.total) {
        set_host_detail(SITE_FIXED);
        return CR_ERR_WORKSPACE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    char *base = (char *)ws;
    float *rank_img = (float *)(base + L.rank);
    double *uniq = (double *)(base + L.uniq);
    uint64_t *key = (uint64_t *)(base + L.key), *key_tmp = (uint64_t *)(base + L.key_tmp);
    uint32_t *idx = (uint32_t *)(base + L.idx), *idx_tmp = (uint32_t *)(base + L.idx_tmp);
    uint32_t *start = (uint32_t *)(base + L.start), *scan = (uint32_t *)(base + L.scan);
    cr_pair *p32 = (cr_pair *)(base + L.pairs);
    int *status = (int *)(base + L.status);
    const unsigned grid = (unsigned)((nv + 255) / 256 < 65535 ? (nv + 255) / 256 : 65535);
    // ranks
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return CR_ERR_CUDA;
    CR_NOTE_LAUNCH();
    k_f64_keys<<<grid, 256, 0, st>>>(img, nv, key, idx, status);
    if (radix_sort_u64(key, idx, key_tmp, idx_tmp, nv, 0, 64, base + L.sort, radix_temp_bytes(nv), st) !=
        cudaSuccess)
        return CR_ERR_CUDA;
    CR_NOTE_LAUNCH();
    k_f64_starts<<<grid, 256, 0, st>>>(key, nv, start);
    if (exclusive_scan_u32(start, nv, scan, st) != cudaSuccess) return CR_ERR_CUDA;
    CR_NOTE_LAUNCH();
    k_f64_scatter<<<grid, 256, 0, st>>>(key, idx, start, nv, img, rank_img, uniq);
    int hstatus = 0;
    cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return CR_ERR_CUDA;
    if (hstatus) return hstatus;
    // the float32 path on the rank image
    rc = cr_persistence(rank_img, ndim, shape, maxdim, p32, capacity, n_pairs, base + L.total, ws_bytes - L.total,
                        stream, flags);
    if (rc) return rc;
    const int64_t n = *n_pairs;
    if (n > 0) {
        const unsigned pg = (unsigned)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
        CR_NOTE_LAUNCH();
        k_f64_pairs<<<pg, 256, 0, st>>>(p32, n, uniq, nv, pairs_out, status);
        cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return CR_ERR_CUDA;
        if (hstatus) return hstatus;
    }
    return CR_OK;
}

}  // extern "C"
