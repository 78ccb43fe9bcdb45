// cr_sort.cu -- stable LSD radix sort of (u64 key, u32 value) pairs and a
// device-wide exclusive scan.  Used for the canonical order of the output
// pairs (dimension, birth), the cohomology order of the residual columns and
// the deterministic per-pixel sums of the backward pass.
//
// One pass sorts by an 8-bit digit: (1) per-block digit histograms of a
// 4096-key tile, (2) an exclusive scan of the digit-major histogram table,
// (3) a stable scatter in which each block ranks its keys in tile order with
// warp match masks and per-warp digit counts in shared memory.
#include "cr_internal.cuh"

namespace cr {

static constexpr int RS_THREADS = 256;
static constexpr int RS_ITEMS = 16;
static constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
static constexpr int RS_WARPS = RS_THREADS / 32;

static constexpr int SC_THREADS = 1024;
static constexpr int SC_ITEMS = 8;
static constexpr int SC_CHUNK = SC_THREADS * SC_ITEMS;

__global__ void k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, uint32_t dmask,
                          uint32_t *__restrict__ counts, int nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; r++) {
        int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & dmask], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
                             uint32_t dmask, const uint32_t *__restrict__ offsets, int nblocks) {
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_w[RS_WARPS][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    s_base[tid] = offsets[(int64_t)tid * nblocks + blockIdx.x];
    s_run[tid] = 0;
    const uint32_t lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; r++) {
        if (base + (int64_t)r * RS_THREADS >= n) break;  // uniform across the block
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) s_w[w][tid] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)r * RS_THREADS + tid;
        bool valid = i < n;
        uint64_t k = valid ? kin[i] : 0;
        uint32_t v = valid ? vin[i] : 0;
        uint32_t d = valid ? ((uint32_t)(k >> shift) & dmask) : 0x1000u;
        uint32_t same = __match_any_sync(0xFFFFFFFFu, d);
        uint32_t rank = __popc(same & lt);
        if (valid && rank == 0) s_w[warp][d] = __popc(same);
        __syncthreads();
        {
            uint32_t run = s_run[tid];
#pragma unroll
            for (int w = 0; w < RS_WARPS; w++) {
                uint32_t c = s_w[w][tid];
                s_w[w][tid] = run;
                run += c;
            }
            s_run[tid] = run;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = s_base[d] + s_w[warp][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
    }
}

// ---- exclusive scan of u32 (in place), three kernels ----
__device__ __forceinline__ uint32_t block_excl_scan_1024(uint32_t x, uint32_t *tot) {
    __shared__ uint32_t ws[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t s = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
        if (lane >= o) s += y;
    }
    if (lane == 31) ws[warp] = s;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < (int)(blockDim.x >> 5)) ? ws[lane] : 0;
        uint32_t t = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t - w;
        if (lane == 31) *tot = t;
    }
    __syncthreads();
    uint32_t r = ws[warp] + s - x;
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const uint32_t *__restrict__ a, int64_t n, uint32_t *__restrict__ part) {
    int64_t base = (int64_t)blockIdx.x * SC_CHUNK + (int64_t)threadIdx.x * SC_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; j++)
        if (base + j < n) s += a[base + j];
    __shared__ uint32_t tot;
    block_excl_scan_1024(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_scan_partials(uint32_t *part, int nb) {
    // one block of 1024 threads; each owns a contiguous run of partials
    int per = (nb + SC_THREADS - 1) / SC_THREADS;
    int b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int j = 0; j < per; j++)
        if (b0 + j < nb) s += part[b0 + j];
    __shared__ uint32_t tot;
    uint32_t off = block_excl_scan_1024(s, &tot);
    for (int j = 0; j < per; j++)
        if (b0 + j < nb) {
            uint32_t t = part[b0 + j];
            part[b0 + j] = off;
            off += t;
        }
}

__global__ void k_scan_apply(uint32_t *__restrict__ a, int64_t n, const uint32_t *__restrict__ part) {
    int64_t base = (int64_t)blockIdx.x * SC_CHUNK + (int64_t)threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; j++) {
        v[j] = (base + j < n) ? a[base + j] : 0;
        s += v[j];
    }
    __shared__ uint32_t tot;
    uint32_t off = block_excl_scan_1024(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SC_ITEMS; j++)
        if (base + j < n) {
            a[base + j] = off;
            off += v[j];
        }
}

static int64_t scan_partials(int64_t n) { return (n + SC_CHUNK - 1) / SC_CHUNK; }

size_t scan_temp_bytes(int64_t n) { return (size_t)(scan_partials(n) + 1) * sizeof(uint32_t); }

cudaError_t exclusive_scan_u32(uint32_t *a, int64_t n, uint32_t *part, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t nb = scan_partials(n);
    if (nb > (int64_t)SC_THREADS * 4096) return cudaErrorInvalidValue;
    CR_NOTE_LAUNCH();
    k_scan_reduce<<<(unsigned)nb, SC_THREADS, 0, st>>>(a, n, part);
    CR_NOTE_LAUNCH();
    k_scan_partials<<<1, SC_THREADS, 0, st>>>(part, (int)nb);
    CR_NOTE_LAUNCH();
    k_scan_apply<<<(unsigned)nb, SC_THREADS, 0, st>>>(a, n, part);
    return cudaGetLastError();
}

size_t radix_temp_bytes(int64_t n) {
    int64_t nblocks = (n + RS_TILE - 1) / RS_TILE;
    int64_t m = 256 * nblocks;
    return (size_t)m * sizeof(uint32_t) + 256 + scan_temp_bytes(m);
}

cudaError_t radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *keys_tmp, uint32_t *vals_tmp, int64_t n,
                           int lo, int hi, void *temp, size_t temp_bytes, cudaStream_t st) {
    if (n <= 1 || hi <= lo) return cudaSuccess;
    if (n > ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    if (temp_bytes < radix_temp_bytes(n)) return cudaErrorInvalidValue;
    int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
    int64_t m = 256 * (int64_t)nblocks;
    uint32_t *counts = (uint32_t *)temp;
    uint32_t *part = (uint32_t *)((char *)temp + (((size_t)m * sizeof(uint32_t) + 255) & ~(size_t)255));
    uint64_t *ka = keys, *kb = keys_tmp;
    uint32_t *va = vals, *vb = vals_tmp;
    int passes = 0;
    for (int sh = lo; sh < hi; sh += 8) {
        int nb = hi - sh < 8 ? hi - sh : 8;
        uint32_t dmask = (1u << nb) - 1u;
        CR_NOTE_LAUNCH();
        k_rs_hist<<<nblocks, RS_THREADS, 0, st>>>(ka, n, sh, dmask, counts, nblocks);
        cudaError_t e = exclusive_scan_u32(counts, m, part, st);
        if (e != cudaSuccess) return e;
        CR_NOTE_LAUNCH();
        k_rs_scatter<<<nblocks, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, sh, dmask, counts, nblocks);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
        passes++;
    }
    if (passes & 1) {
        cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(vals, va, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    }
    return cudaGetLastError();
}

}  // namespace cr
