// cr_internal.cuh -- internal declarations shared by the libcr translation units.
//
// Notation (Kaji, Sudo, Ahara, "Cubical Ripser", Sec. 2): a cube is
// (x, y, z, m, d); its value is the maximum over its vertices (V-construction);
// within one dimension cubes are totally ordered by the 64-bit key
//     key = ord32(value) << 32 | (0xFFFFFFFF - L),  L = ((m*Nz+z)*Ny+y)*Nx+x,
// where ord32 maps float bits to an unsigned integer with the same order
// (Herf's radix-sort trick: flip all bits of negatives, set the sign bit of
// non-negatives).  A smaller key enters the filtration earlier.  The tie part
// puts larger L first, which is the reverse of the paper's (-birth, m, z, y, x)
// order of Sec. 2.
#pragma once
#include <cstdint>
#include <utility>
#include <vector>
#include <cstddef>
#include <cstring>
#include <atomic>
#include <cuda.h>
#include <cuda_runtime.h>
#include "../../include/cr.h"

namespace cr {

// ---------------------------------------------------------------------------
// image segments (a single image is a batch of one)
// ---------------------------------------------------------------------------
struct Seg {
    int64_t voff;  // first vertex of this image in the packed vertex space
    int64_t loff;  // offset of this image's L-space (3 * voff) in L-indexed arrays
    int64_t coff;  // first dual node (top cube) of this image; its outer node is coff + ncell
    int64_t ncell; // number of top cubes of this image
    int32_t nx, ny, nz;
    int32_t edim;  // effective dimension (leading unit extents dropped), 0..3
    int64_t toff;  // first tile of this image in the tiled launches
    int32_t tiles_x, tiles_y, tiles_z;
    int32_t stoff; // first 32x32 super-tile of this image (2D batches), see k_stencil2d_batch
};

// super-tiles of the fused 2D batch stencil
constexpr int ST_X = 32, ST_Y = 32;

// tiles of the 2.5D stencil kernels: TILE_X x TILE_Y voxels marching TILE_Z planes
constexpr int TILE_X = 32, TILE_Y = 8, TILE_Z = 16;

// image of a tile (binary search over the segments' first tiles)
__device__ __forceinline__ int seg_of_tile(const Seg *segs, int n, int64_t t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (segs[mid].toff <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Block-aggregated append: every thread of the block calls it with the number
// of items it will write; one atomic per block reserves the space.  Returns
// this thread's first slot.
__device__ __forceinline__ int64_t block_append(int cnt, unsigned long long *counter) {
    __shared__ int s_w[32];
    __shared__ unsigned long long s_base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
        int v = lane < nw ? s_w[lane] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane < nw) s_w[lane] = inc - v;
        if (lane == 31) s_base = inc > 0 ? atomicAdd(counter, (unsigned long long)inc) : 0ull;
    }
    __syncthreads();
    int64_t base = (int64_t)s_base + s_w[w] + (incl - cnt);
    __syncthreads();
    return base;
}

constexpr int TMA_BX = TILE_X + 8, TMA_BY = TILE_Y + 2, TMA_BZ = TILE_Z + 2;
constexpr int TMA_BYTES = TMA_BX * TMA_BY * TMA_BZ * 4;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// wait on phase 0 of an mbarrier, at most `limit` polls; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, long long limit) {
    uint32_t a = smem_u32(bar);
    for (long long i = 0; i < limit; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a)
            : "memory");
        if (done) return true;
    }
    return false;
}


// origin of tile t of a single image
__device__ __forceinline__ void tile_origin(const Seg &S, uint32_t t, int &x0, int &y0, int &z0) {
    const uint32_t tix = t % (uint32_t)S.tiles_x;
    t /= (uint32_t)S.tiles_x;
    const uint32_t tiy = t % (uint32_t)S.tiles_y;
    const uint32_t tiz = t / (uint32_t)S.tiles_y;
    x0 = (int)tix * TILE_X;
    y0 = (int)tiy * TILE_Y;
    z0 = (int)tiz * TILE_Z;
}

// One thread: initialise the mbarrier, arm it for `bytes` and issue the 3D
// tensor copy of the box whose first element is (cx, cy, cz).  cx * 4 bytes
// must be a multiple of 16; outside the tensor the box is zero-filled.
__device__ __forceinline__ void tma_load_3d(const void *tmap, void *dst, uint64_t *bar, uint32_t bytes, int cx, int cy,
                                            int cz) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(tmap), "r"(cx), "r"(cy), "r"(cz), "r"(smem_u32(bar))
        : "memory");
}

// TMA copy of the box around a tile: x starts 4 voxels early (16-byte
// boundary), y and z one voxel early; issued by one thread, completion on bar
__device__ __forceinline__ void tma_load_box(const void *tmap, float *dst, uint64_t *bar, int x0, int y0, int z0) {
    tma_load_3d(tmap, dst, bar, TMA_BYTES, x0 - 4, y0 - 1, z0 - 1);
}

// box of the dual stencil: a cube and its neighbours across each facet reach
// two voxels past the tile in +y and +z
constexpr int DUAL_BX = TILE_X + 8, DUAL_BY = TILE_Y + 3, DUAL_BZ3 = TILE_Z + 3;

// Tile-grid launches (grid = tiles, block = TILE_X*TILE_Y threads): the
// block's image, looked up once, and this thread's column of the tile.
__device__ __forceinline__ int block_seg(const Seg *segs, int nseg) {
    __shared__ int s_si;
    if (threadIdx.x == 0) s_si = seg_of_tile(segs, nseg, blockIdx.x);
    __syncthreads();
    return s_si;
}
__device__ __forceinline__ void tile_column(const Seg &S, int &x, int &y, int &z0, int &z1) {
    uint32_t t = (uint32_t)(blockIdx.x - S.toff);
    uint32_t tix = t % (uint32_t)S.tiles_x;
    t /= (uint32_t)S.tiles_x;
    uint32_t tiy = t % (uint32_t)S.tiles_y;
    uint32_t tiz = t / (uint32_t)S.tiles_y;
    x = (int)tix * TILE_X + (int)(threadIdx.x & (TILE_X - 1));
    y = (int)tiy * TILE_Y + (int)(threadIdx.x / TILE_X);
    z0 = (int)tiz * TILE_Z;
    z1 = min(z0 + TILE_Z, S.nz);
}

// ---------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t ord32(float f) {
#ifdef __CUDA_ARCH__
    uint32_t b = __float_as_uint(f);
#else
    uint32_t b;
    memcpy(&b, &f, 4);
#endif
    if (b == 0x80000000u) b = 0u;  // -0.0 is +0.0
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__host__ __device__ __forceinline__ float unord32(uint32_t o) {
    uint32_t b = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, 4);
    return f;
#endif
}

__host__ __device__ __forceinline__ uint64_t make_key(uint32_t ordv, uint32_t L) {
    return ((uint64_t)ordv << 32) | (uint64_t)(0xFFFFFFFFu - L);
}
__host__ __device__ __forceinline__ uint32_t key_L(uint64_t k) { return 0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFu); }
__host__ __device__ __forceinline__ float key_value(uint64_t k) { return unord32((uint32_t)(k >> 32)); }

// L index of a cube of type m anchored at (x, y, z)
__host__ __device__ __forceinline__ uint32_t cube_L(const Seg &s, int m, int x, int y, int z) {
    return (uint32_t)((((int64_t)m * s.nz + z) * s.ny + y) * s.nx + x);
}

// ---------------------------------------------------------------------------
// status block (device): int word 0 = error code, int word 8 = failure site;
// the first error wins
// ---------------------------------------------------------------------------
enum Site {
    SITE_NONE = 0, SITE_GROUPS = 1, SITE_EDGES = 2, SITE_COLUMNS = 3, SITE_ARENA = 4, SITE_POOL = 5,
    SITE_UF_CARVE = 6, SITE_H1_CARVE = 7, SITE_OUT_CARVE = 8, SITE_FIXED = 9, SITE_INJECTED = 10
};
__device__ __forceinline__ void set_status(int *status, int code) { atomicCAS(status, 0, code); }
__device__ __forceinline__ void fail_ws(int *status, int site) {
    atomicCAS(status, 0, CR_ERR_WORKSPACE);
    atomicCAS(status + 8, 0, site);
}
void set_host_detail(int site);

// ---------------------------------------------------------------------------
// workspace carving
// ---------------------------------------------------------------------------
struct Carver {
    char *base;
    size_t cap, used;
    bool ok;
    Carver(void *b, size_t c) : base((char *)b), cap(c), used(0), ok(true) {}
    template <class T>
    T *take(size_t n) {
        size_t off = (used + 255) & ~(size_t)255;
        size_t bytes = n * sizeof(T);
        if (off + bytes > cap) { ok = false; used = off + bytes; return nullptr; }
        used = off + bytes;
        return base ? (T *)(base + off) : nullptr;
    }
};

// ---------------------------------------------------------------------------
// pair record used inside the pipeline (before the final sort)
// ---------------------------------------------------------------------------
struct PairBuf {
    cr_pair *pairs;     // capacity entries (the caller's output buffer)
    int64_t capacity;
    unsigned long long *count;  // device counter
};

// While the pipeline runs, bits 8..31 of cr_pair.flags hold the image index;
// the final gather clears them.
__device__ __forceinline__ void emit_pair(const PairBuf &pb, uint32_t seg, int dim, float birth, float death,
                                          int64_t bcell, int64_t dcell, uint32_t flags) {
    unsigned long long i = atomicAdd(pb.count, 1ull);
    if ((int64_t)i < pb.capacity) {
        cr_pair p;
        p.dim = dim;
        p.birth = birth;
        p.death = death;
        p.flags = (flags & 0xFFu) | (seg << 8);
        p.birth_cell = bcell;
        p.death_cell = dcell;
        pb.pairs[i] = p;
    }
}

// device counter block: status words and pair count in slots 0..7, the middle
// dimension's counters at 16.., each union-find run's UF_CNT counters at
// CNT_H0 / CNT_DUAL
constexpr int CR_CNT_SLOTS = 128, CNT_H1 = 16, CNT_H0 = 64, CNT_DUAL = 96, UF_CNT = 16;
// slots of a union-find run: 0 groups, 1-2 edges in the two edge buffers,
// 3 edges visited by the rounds, 4 barrier of the rounds, 5 barrier of the
// basin kernel, 6 rounds, 7 live edges (in-place list), 8-10 pointers changed
// per doubling pass, 11 doubling passes
enum UfSlot { UFC_GROUPS = 0, UFC_E0 = 1, UFC_E1 = 2, UFC_VISITED = 3, UFC_BAR_ROUNDS = 4, UFC_BAR_BASINS = 5,
              UFC_ROUNDS = 6, UFC_LIVE = 7, UFC_CHANGED = 8, UFC_PASSES = 11 };

// union-find buffers (cr_uf.cu)
struct UF {
    uint32_t *lab;   // node -> parent, then node -> group
    uint8_t *dd;     // node -> stencil hook code (0 = root)
    uint64_t *gkey;  // group -> age key of its root (smaller = older)
    uint32_t *groot, *gseg;
    uint8_t *gdead;
    uint64_t *minE, *minE2;  // min edge key at each group, for this round and the next
    uint64_t *dkey;          // key of the edge a group died at
    uint32_t *hook;
    uint64_t *ek[2];
    uint32_t *ea[2], *eb[2];
    int64_t max_edges, max_groups;
    unsigned long long *cnt;   // device counters [0] groups, [1] edges, [2] edges after a round
    unsigned long long *hcnt;  // host mirror
};
// single-image persistence with the two union-finds run one after the other
// (a workspace bound of one union-find; cr_api.cu)
int workspace_size_serial(int ndim, const int64_t *shape, int maxdim, uint32_t flags, size_t *bytes);
int persistence_serial(const float *img, int ndim, const int64_t *shape, int maxdim, cr_pair *pairs_out,
                       int64_t capacity, int64_t *n_pairs, void *ws, size_t ws_bytes, cudaStream_t stream,
                       uint32_t flags);

// union-find of H0 (u0, primal graph) and of the top dimension (u1, dual
// graph); either may be null
// nstiles > 0: every image is 2D and both stencils run fused over that many
// 32x32 super-tiles
int run_uf(const float *img, const Seg *segs, const Seg *hsegs, int nseg, int64_t vtot, int64_t ctot,
           int64_t ntiles, int64_t nstiles, UF *u0, UF *u1, const PairBuf &pb, uint32_t flags, uint32_t *extra_mask,
           int *status, cudaStream_t st);

// both union-finds of a batch of 2D images in one persistent launch, one image
// per block (cr_batch2d.cu); order: device, the images by size, largest
// first; CR_ERR_WORKSPACE if the region cannot hold one block's scratch
// (nothing launched).  threads_code: 1 = 256, 2 = 512, 3 = 1024 threads per
// block.
int run_batch2d(const float *img, const Seg *segs, const std::vector<Seg> &hsegs, const uint32_t *order,
                char *region, size_t region_cap, const PairBuf &pb, uint32_t flags, bool primal, bool dual,
                unsigned long long *queue, int *status, cudaStream_t st, int threads_code);

// middle-dimension buffers (cr_h1.cu)
struct H1Bufs {
    uint64_t *colkey, *colkey_tmp;
    uint32_t *colseg, *colseg_tmp;
    int64_t max_cols;
    void *sort_temp;
    size_t sort_temp_bytes;
    unsigned long long *P;  // face -> owner and version (cr_h1.cu, piv_make)
    int64_t P_len;
    unsigned long long *cur;
    uint64_t *arena;
    int64_t arena_cap;
    uint64_t *scratch;        // 2 * maxlen per warp
    int64_t nwarps;
    int maxlen;
    uint8_t *code;            // one code byte per voxel: apparent and residual edges (cr_h1.cu)
    uint64_t *pool;           // grown column buffers for columns longer than maxlen
    int64_t pool_cap;
    unsigned long long *cnt;  // [0] columns, [1] arena top, [2] work counter, [3] pool top
};
int h1_stats(int64_t *out, int n);
// tensor map over one image as an (nx, ny, nz) float32 tensor with the tile box; false if TMA cannot serve it;
// out-of-image elements of a box read as 0, or as NaN with nan_fill
bool make_image_map(CUtensorMap *m, const float *img, const Seg &S, int bx = TMA_BX, int by = TMA_BY,
                    int bz = TMA_BZ, bool nan_fill = false);
bool make_u8_map(CUtensorMap *m, const uint8_t *p, const Seg &S, int bx, int by, int bz);
int run_h1(const float *img, const uint8_t *dd, const uint32_t *extra, const Seg *segs, const Seg *hseg, int nseg,
           int64_t vtot, int64_t ntiles, H1Bufs &B, const PairBuf &pb, uint32_t flags, int *status,
           int64_t *ncols_out, cudaStream_t st);

// radix sort of (u64 key, u32 value) by bits [lo, hi) of the key, stable, LSD.
// tmp buffers must hold n entries each.  Returns cudaError.
size_t radix_temp_bytes(int64_t n);
cudaError_t radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *keys_tmp, uint32_t *vals_tmp, int64_t n,
                           int lo, int hi, void *temp, size_t temp_bytes, cudaStream_t st);
cudaError_t exclusive_scan_u32(uint32_t *a, int64_t n, uint32_t *part, cudaStream_t st);
size_t scan_temp_bytes(int64_t n);

// ---------------------------------------------------------------------------
// launch accounting / stage timing (cr_prof.cu)
// ---------------------------------------------------------------------------
enum Stage {
    STAGE_H0_STENCIL, STAGE_JUMP, STAGE_ROOTS, STAGE_RELABEL, STAGE_H0_CROSS, STAGE_UF_ROUND,
    STAGE_DUAL_STENCIL, STAGE_DUAL_CROSS, STAGE_H1_SCAN, STAGE_H1_SORT, STAGE_H1_REDUCE, STAGE_H1_EMIT,
    STAGE_OUT_SORT, STAGE_BW_CONTRIB, STAGE_BW_SORT, STAGE_BW_SUM, STAGE_IMAGES, STAGE_H1_COLUMNS, STAGE_COUNT
};
extern std::atomic<long long> g_launch_count;
void prof_begin(cudaStream_t st, int stage);
bool prof_active();
uint32_t prof_mask();
void prof_capture_begin();
void prof_capture_end(std::vector<std::pair<int, std::pair<void *, void *>>> &out, std::vector<double> &bytes);
void prof_replay(const std::vector<std::pair<int, std::pair<void *, void *>>> &recs, const std::vector<double> &bytes);
void prof_end(cudaStream_t st, int stage, double bytes);
void prof_flush();
void prof_add_bytes(int stage, double bytes);
#define CR_NOTE_LAUNCH() (::cr::g_launch_count.fetch_add(1, std::memory_order_relaxed))

// launch knobs (cr_tune_set); tune_epoch() changes whenever one does
int tune_value(int knob);
uint32_t tune_epoch();

// limits of the bounded device waits (cr_debug_limits): the defaults, or the
// lowered values the error-path tests set
struct DebugLimits {
    long long barrier_polls;    // polls of one grid-barrier wait
    long long reduce_iters;     // iterations of one column of the middle-dimension reduction
    unsigned int barrier_extra; // arrivals a barrier expects beyond the grid (1 = never satisfied)
};
DebugLimits debug_limits();
// the error a CR_FAULT injection makes a forward call return before any GPU work (CR_OK: none)
int injected_error_before_gpu();
constexpr long long DEFAULT_BARRIER_POLLS = 1ll << 24;
constexpr long long DEFAULT_REDUCE_ITERS = 1ll << 24;

}  // namespace cr
