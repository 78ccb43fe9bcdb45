// cr_uf.cu -- 0-dimensional persistence by union-find (Sec. 2: "computed
// efficiently by the union-find algorithm"; elder rule: the component with
// the larger birth is killed) and the top dimension by union-find on the dual
// graph in the reversed order (Sec. 2, Rem. 2.1, Alexander duality).
//
// Both are one algorithm on a graph whose nodes carry an age key (smaller =
// older) and whose edges carry a key (smaller = earlier); node and edge keys
// are unique.  The pairs are those of Kruskal's algorithm with the elder rule.
// Parallel form used here (Boruvka rounds over groups of nodes):
//   * every group G knows m(G), its minimum outgoing edge, and the group H at
//     its other end;
//   * if H's root is older than G's root, G's root dies at m(G), and G is
//     contracted into H (the "safe hook");  when m(G) = m(H) (mutual), the
//     younger root is the one that hooks, so mutual pairs are covered;
//   * otherwise G waits for a later round.
// Invariant that makes both rules exact: for every group and every edge e
// leaving it at member x, the tree path from x to the group root uses only
// edges smaller than e.  Hence, just before m(G), G's Kruskal component lies
// inside G and contains its root, and H's contains H's root.
//
// Round 0 runs on the image itself without materialising any edge: a node's
// minimum incident edge is found by a stencil, hooks become parent pointers,
// pointer jumping yields basins, and only edges between different basins are
// written out for the later rounds.
#include "cr_internal.cuh"
#include <cuda.h>
#include <cudaTypedefs.h>

namespace cr {

__device__ __forceinline__ int seg_of(const Seg *segs, int n, int64_t gv) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (segs[mid].voff <= gv) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int seg_of_node(const Seg *segs, int n, int64_t gc) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (segs[mid].coff <= gc) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// warp-aggregated append; every lane of the warp must call it
__device__ __forceinline__ int64_t warp_append(bool pred, unsigned long long *counter) {
    unsigned mask = __ballot_sync(0xFFFFFFFFu, pred);
    if (!mask) return -1;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (!pred) return -1;
    return (int64_t)(base + __popc(mask & ((1u << lane) - 1u)));
}

// ===========================================================================
// primal H0, round 0: each vertex's minimum incident edge
// direction codes: 1 -x, 2 +x, 3 -y, 4 +y, 5 -z, 6 +z, 0 = no hook
// ===========================================================================
// The stencil, tiled: a block owns TILE_X x TILE_Y voxels of one image
// and marches TILE_Z planes in z.  Each xy-plane is staged with a one-voxel
// halo in shared memory; the z neighbours come from registers.  All index
// arithmetic is 32-bit within the image.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(TILE_X *TILE_Y) k_h0_stencil_tiled(const float *__restrict__ img,
                                                                    const Seg *__restrict__ segs, int nseg,
                                                                    uint32_t *__restrict__ parent,
                                                                    uint8_t *__restrict__ dd, int *status, PairBuf pb,
                                                                    uint32_t flags) {
    __shared__ uint32_t pl[TILE_Y + 2][TILE_X + 2];
    __shared__ int s_si;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_si = seg_of_tile(segs, nseg, blockIdx.x);
    __syncthreads();
    const int si = s_si;
    const Seg S = segs[si];
    uint32_t t = (uint32_t)(blockIdx.x - S.toff);
    const uint32_t tix = t % (uint32_t)S.tiles_x;
    t /= (uint32_t)S.tiles_x;
    const uint32_t tiy = t % (uint32_t)S.tiles_y;
    const uint32_t tiz = t / (uint32_t)S.tiles_y;
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const uint32_t plane = (uint32_t)nx * (uint32_t)ny;
    const int x = (int)tix * TILE_X + threadIdx.x, y = (int)tiy * TILE_Y + threadIdx.y;
    const int z0 = (int)tiz * TILE_Z, z1 = min(z0 + TILE_Z, nz);
    const bool inxy = x < nx && y < ny;
    const float *im = img + S.voff;
    const int tid = threadIdx.y * TILE_X + threadIdx.x;
    // z neighbours of this thread's column
    uint32_t below = 0, cur = 0, above = 0;
    if (inxy) {
        uint32_t l = (uint32_t)y * nx + x;
        if (z0 > 0) below = ord32(im[(uint32_t)(z0 - 1) * plane + l]);
        cur = ord32(im[(uint32_t)z0 * plane + l]);
    }
    bool nan_seen = false;
    for (int z = z0; z < z1; z++) {
        const uint32_t zoff = (uint32_t)z * plane;
        // stage the plane with its halo
        for (int i = tid; i < (TILE_Y + 2) * (TILE_X + 2); i += TILE_X * TILE_Y) {
            int hy = i / (TILE_X + 2), hx = i % (TILE_X + 2);
            int gx = (int)tix * TILE_X + hx - 1, gy = (int)tiy * TILE_Y + hy - 1;
            uint32_t o = 0;
            if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
                float f = im[zoff + (uint32_t)gy * nx + gx];
                nan_seen |= isnan(f);
                o = ord32(f);
            }
            pl[hy][hx] = o;
        }
        if (inxy && z + 1 < nz) above = ord32(im[zoff + plane + (uint32_t)y * nx + x]);
        __syncthreads();
        if (inxy) {
            const uint32_t lv = zoff + (uint32_t)y * nx + x;
            const uint32_t ov = cur;
            // the first neighbour with ord <= ord(v) in descending edge-L
            // order (+z, -z, +y, -y, +x, -x) gives the minimum edge
            int dir = 0;
            uint32_t ou = 0;
#define CR_NB(OK, VAL, DIR)                 \
            {                               \
                const uint32_t o_ = (VAL);  \
                if ((OK) && o_ <= ov) {     \
                    dir = (DIR);            \
                    ou = o_;                \
                }                           \
            }
            CR_NB(x > 0, pl[threadIdx.y + 1][threadIdx.x], 1)
            CR_NB(x + 1 < nx, pl[threadIdx.y + 1][threadIdx.x + 2], 2)
            CR_NB(y > 0, pl[threadIdx.y][threadIdx.x + 1], 3)
            CR_NB(y + 1 < ny, pl[threadIdx.y + 2][threadIdx.x + 1], 4)
            CR_NB(z > 0, below, 5)
            CR_NB(z + 1 < nz, above, 6)
#undef CR_NB
            const int64_t gv = S.voff + lv;
            if (dir && (ou < ov || !(dir & 1))) {
                const uint32_t st = dir <= 2 ? 1u : (dir <= 4 ? (uint32_t)nx : plane);
                const uint32_t lu = (dir & 1) ? lv - st : lv + st;
                parent[gv] = (uint32_t)(S.voff + lu);
                dd[gv] = (uint8_t)dir;
                if (flags & CR_KEEP_ZERO) {
                    const uint32_t la = ((dir & 1) ? lu : lv) + (uint32_t)((dir - 1) >> 1) * plane * (uint32_t)nz;
                    emit_pair(pb, (uint32_t)si, 0, unord32(ov), unord32(ov), lv, la, 0);
                }
            } else {
                parent[gv] = (uint32_t)gv;
                dd[gv] = 0;
            }
        }
        below = cur;
        cur = above;
        __syncthreads();
    }
    if (nan_seen) set_status(status, CR_ERR_NAN);
}

// ---------------------------------------------------------------------------
// The same stencil fed by the tensor-memory accelerator: one
// cp.async.bulk.tensor copy brings the block's whole 32x8x16 tile with a
// halo (a 40x10x18 box, x starting 4 voxels early so the copy starts on a
// 16-byte boundary; outside the image the box is zero-filled and never used)
// into shared memory, completing on an mbarrier.  Single images whose rows
// are a multiple of 16 bytes; FLAT is the 2D case (one 40x10 plane).
// The hooks are then followed inside the tile, in shared memory, so that
// every voxel leaves with the first ancestor outside the tile or its in-tile
// root: the global pointer jumping starts from paths shortened by the tile.
// ---------------------------------------------------------------------------
template <bool FLAT>
__global__ void __launch_bounds__(TILE_X *TILE_Y) k_h0_stencil_tma(const __grid_constant__ CUtensorMap tmap,
                                                                  const Seg *__restrict__ segs,
                                                                  uint32_t *__restrict__ parent,
                                                                  uint8_t *__restrict__ dd, int *status, PairBuf pb,
                                                                  uint32_t flags) {
    constexpr int BZ = FLAT ? 1 : TMA_BZ, TZ = FLAT ? 1 : TILE_Z;
    constexpr uint32_t GLOBAL = 0x80000000u;  // lp entry: ancestor outside the tile (global index)
    __shared__ __align__(128) float box[BZ][TMA_BY][TMA_BX];
    __shared__ uint32_t lp[FLAT ? TILE_Y * TILE_X : 1];  // in-tile hooks (2D only)
    __shared__ __align__(8) uint64_t bar;
    const Seg S = segs[0];
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    int x0, y0, z0;
    tile_origin(S, blockIdx.x, x0, y0, z0);
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    if (leader)
        tma_load_3d(&tmap, &box[0][0][0], &bar, (uint32_t)(BZ * TMA_BY * TMA_BX * 4), x0 - 4, y0 - 1,
                    FLAT ? 0 : z0 - 1);
    __syncthreads();
    // the wait's outcome is made uniform so that no thread is left at a later barrier
    if (!__syncthreads_and(mbar_wait(&bar, 1ll << 24))) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            set_status(status, CR_ERR_TIMEOUT);
            mbar_wait(&bar, 1ll << 24);  // let a copy still in flight land before the block exits
        }
        return;
    }
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool inxy = x < nx && y < ny;
    const uint32_t plane = (uint32_t)nx * (uint32_t)ny;
    const int bx = threadIdx.x + 4, by = threadIdx.y + 1;
    bool nan_seen = false;
    const int zend = FLAT ? 1 : min(TILE_Z, nz - z0);
    const uint32_t P = plane * (uint32_t)nz;  // size of one type's L-range
    const int tl = threadIdx.y * TILE_X + threadIdx.x;  // local index in a plane of the tile
#pragma unroll 1
    for (int zz = 0; zz < TZ; zz++) {
        const int li = zz * TILE_X * TILE_Y + tl;
        if (zz >= zend || !inxy) {
            if (FLAT) lp[li] = (uint32_t)li;  // outside the image: never referenced
            continue;
        }
        const int z = z0 + zz, bz = FLAT ? 0 : zz + 1;
        const float fv = box[bz][by][bx];
        nan_seen |= isnan(fv);
        const uint32_t lv = (uint32_t)z * plane + (uint32_t)y * nx + x;
        // Every edge to a neighbour u with phi(u) <= phi(v) has value phi(v),
        // and any other edge is larger, so the minimum edge is the first such
        // neighbour in descending edge-L order (+z, -z, +y, -y, +x, -x).
        // Float comparisons order like ord32 here (-0 == +0; NaN is flagged).
        int dir = 0;
        float fu = 0.f;
#define CR_NB(OK, VAL, DIR)                  \
        {                                    \
            const float f_ = (VAL);          \
            if ((OK) && f_ <= fv) {          \
                dir = (DIR);                 \
                fu = f_;                     \
            }                                \
        }
        CR_NB(x > 0, box[bz][by][bx - 1], 1)
        CR_NB(x + 1 < nx, box[bz][by][bx + 1], 2)
        CR_NB(y > 0, box[bz][by - 1][bx], 3)
        CR_NB(y + 1 < ny, box[bz][by + 1][bx], 4)
        if (!FLAT) {
            CR_NB(z > 0, box[bz - 1][by][bx], 5)
            CR_NB(z + 1 < nz, box[bz + 1][by][bx], 6)
        }
#undef CR_NB
        // the neighbour is older iff its value is smaller, or equal with a
        // larger L (a neighbour in the + direction)
        if (dir && (fu < fv || !(dir & 1))) {
            const uint32_t st = dir <= 2 ? 1u : (dir <= 4 ? (uint32_t)nx : plane);
            const uint32_t lu = (dir & 1) ? lv - st : lv + st;
            // the same step inside the tile, when it stays there
            const int lstep = dir <= 2 ? 1 : (dir <= 4 ? TILE_X : TILE_X * TILE_Y);
            const bool inside = dir == 1 ? threadIdx.x > 0
                              : dir == 2 ? threadIdx.x + 1 < TILE_X
                              : dir == 3 ? threadIdx.y > 0
                              : dir == 4 ? threadIdx.y + 1 < TILE_Y
                              : dir == 5 ? zz > 0 : zz + 1 < TILE_Z;
            if (FLAT)
                lp[li] = inside ? (uint32_t)((dir & 1) ? li - lstep : li + lstep) : (GLOBAL | lu);
            else
                parent[lv] = lu;
            dd[lv] = (uint8_t)dir;
            if (flags & CR_KEEP_ZERO) {
                const uint32_t la = ((dir & 1) ? lu : lv) + (uint32_t)((dir - 1) >> 1) * P;
                const float cv = unord32(ord32(fv));
                emit_pair(pb, 0u, 0, cv, cv, lv, la, 0);
            }
        } else {
            if (FLAT)
                lp[li] = (uint32_t)li;
            else
                parent[lv] = lv;
            dd[lv] = 0;
        }
    }
    if (nan_seen) set_status(status, CR_ERR_NAN);
    if (!FLAT) return;
    __syncthreads();
    // pointer jumping inside the tile (every write stores an ancestor)
    for (int it = 0; it < 64; it++) {
        int ch = 0;
#pragma unroll 1
        for (int zz = 0; zz < TZ; zz++) {
            const int li = zz * TILE_X * TILE_Y + tl;
            const uint32_t p = lp[li];
            if (p & GLOBAL) continue;
            const uint32_t q = lp[p];
            if (q != p) {
                lp[li] = q;
                ch = 1;
            }
        }
        if (!__syncthreads_or(ch)) break;
    }
    if (!inxy) return;
#pragma unroll 1
    for (int zz = 0; zz < zend; zz++) {
        const int li = zz * TILE_X * TILE_Y + tl;
        const uint32_t p = lp[li];
        uint32_t g;
        if (p & GLOBAL) {
            g = p & ~GLOBAL;
        } else {
            const int pz = p / (TILE_X * TILE_Y), py = (p / TILE_X) % TILE_Y, px = p % TILE_X;
            g = (uint32_t)(z0 + pz) * plane + (uint32_t)(y0 + py) * nx + (uint32_t)(x0 + px);
        }
        parent[(uint32_t)(z0 + zz) * plane + (uint32_t)y * nx + x] = g;
    }
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// a tensor map over one image as an (nx, ny, nz) float32 tensor; false if TMA cannot serve it
bool make_image_map(CUtensorMap *m, const float *img, const Seg &S, int bx, int by, int bz, bool nan_fill) {
    if (((uintptr_t)img & 15) || (S.nx % 4) != 0) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)S.nx, (cuuint64_t)S.ny, (cuuint64_t)S.nz};
    cuuint64_t strides[2] = {(cuuint64_t)S.nx * 4, (cuuint64_t)S.nx * S.ny * 4};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)img, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     nan_fill ? CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA : CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// a tensor map over one image's 1-byte-per-voxel array (nx, ny, nz); rows must
// be 16-byte multiples
bool make_u8_map(CUtensorMap *m, const uint8_t *p, const Seg &S, int bx, int by, int bz) {
    if (((uintptr_t)p & 15) || (S.nx % 16) != 0) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)S.nx, (cuuint64_t)S.ny, (cuuint64_t)S.nz};
    cuuint64_t strides[2] = {(cuuint64_t)S.nx, (cuuint64_t)S.nx * S.ny};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void *)p, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}






// edges between different basins; an edge is a stencil (round-0) hook iff
// one of its endpoints points at the other through it
__global__ void k_h0_cross(const float *__restrict__ img, const Seg *__restrict__ segs, int nseg,
                           const uint32_t *__restrict__ lab, const uint8_t *__restrict__ dd,
                           uint64_t *__restrict__ ek, uint32_t *__restrict__ ea, uint32_t *__restrict__ eb,
                           unsigned long long *ne, int64_t max_edges, const unsigned long long *ngroups,
                           int *status) {
    const uint32_t ng = (uint32_t)*ngroups;
    const int si = block_seg(segs, nseg);
    const Seg S = segs[si];
    int x, y, z0, z1;
    tile_column(S, x, y, z0, z1);
    const bool inxy0 = x < S.nx && y < S.ny;
    const uint32_t nx = (uint32_t)S.nx, plane = (uint32_t)S.nx * (uint32_t)S.ny;
    // Edges along one axis met in consecutive planes often join the same two
    // basins; of parallel edges between two groups only the first in the
    // order can merge them, so a run of equal pairs is kept as one edge (the
    // smallest key).
    uint64_t pk[3];
    uint32_t pa[3], pb[3];
    bool pend[3] = {false, false, false};
    for (int z = z0; z <= z1; z++) {
        const bool inxy = inxy0 && z < z1;
        const uint32_t lv = (uint32_t)z * plane + (uint32_t)y * nx + (uint32_t)x;
        const int64_t gv = S.voff + lv;
        uint32_t ov = 0, la = 0;
        uint8_t dv = 0;
        if (inxy) {
            ov = ord32(img[gv]);
            la = lab[gv];
            dv = dd[gv];
        }
        uint64_t keys[3];
        uint32_t las[3], lbs[3];
        int cnt = 0;
        for (int ax = 0; ax < 3; ax++) {
            bool emit = false;
            uint64_t key = 0;
            uint32_t lb = 0;
            if (inxy) {
                const int ext = ax == 0 ? S.nx : (ax == 1 ? S.ny : S.nz);
                const int c = ax == 0 ? x : (ax == 1 ? y : z);
                if (c + 1 < ext) {
                    const uint32_t du = ax == 0 ? 1u : (ax == 1 ? nx : plane);
                    const int64_t u = gv + du;
                    const bool stencil = dv == (uint8_t)(2 * ax + 2) || dd[u] == (uint8_t)(2 * ax + 1);
                    lb = lab[u];
                    if (!stencil && lb != la) {
                        if (la >= ng || lb >= ng) {
                            set_status(status, CR_ERR_INTERNAL);
                        } else {
                            const uint32_t ou = ord32(img[u]);
                            key = make_key(ov > ou ? ov : ou, lv + (uint32_t)ax * plane * (uint32_t)S.nz);
                            emit = true;
                        }
                    }
                }
            }
            if (emit && pend[ax] && pa[ax] == la && pb[ax] == lb) {
                pk[ax] = key < pk[ax] ? key : pk[ax];  // the same two groups: one edge
                continue;
            }
            if (pend[ax] && (emit || z == z1)) {  // the run ends: its edge goes out
                keys[cnt] = pk[ax];
                las[cnt] = pa[ax];
                lbs[cnt] = pb[ax];
                cnt++;
                pend[ax] = false;
            }
            if (emit) {
                pk[ax] = key;
                pa[ax] = la;
                pb[ax] = lb;
                pend[ax] = true;
            }
        }
        int64_t i = block_append(cnt, ne);
        for (int k = 0; k < cnt; k++) {
            if (i + k < max_edges) {
                ek[i + k] = keys[k];
                ea[i + k] = las[k];
                eb[i + k] = lbs[k];
            } else {
                fail_ws(status, SITE_EDGES);
            }
        }
    }
}

// ===========================================================================
// dual graph (top cubes + one outer node per image), reversed order
// facet codes: 2D 1 -y, 2 +y, 3 -x, 4 +x;  3D 1 -z, 2 +z, 3 -y, 4 +y, 5 -x, 6 +x
// ===========================================================================
struct CellPos {
    int x, y, z;
};

__device__ __forceinline__ CellPos cell_pos(const Seg &S, int64_t c) {
    CellPos p;
    int cx = S.nx - 1, cy = S.ny - 1;
    p.x = (int)(c % cx);
    p.y = (int)((c / cx) % cy);
    p.z = S.edim == 3 ? (int)(c / ((int64_t)cx * cy)) : 0;
    return p;
}

__device__ __forceinline__ int64_t cell_index(const Seg &S, int x, int y, int z) {
    return ((int64_t)z * (S.ny - 1) + y) * (S.nx - 1) + x;
}

__device__ __forceinline__ uint32_t vmax_ord(const float *img, const Seg &S, int x, int y, int z, int sx, int sy,
                                             int sz) {
    uint32_t m = 0;
    for (int dz = 0; dz <= sz; dz++)
        for (int dy = 0; dy <= sy; dy++)
            for (int dx = 0; dx <= sx; dx++) {
                uint32_t o = ord32(img[S.voff + ((int64_t)(z + dz) * S.ny + (y + dy)) * S.nx + (x + dx)]);
                m = o > m ? o : m;
            }
    return m;
}

// key of a top cube
__device__ __forceinline__ uint64_t top_key(const float *img, const Seg &S, int x, int y, int z) {
    if (S.edim == 3) return make_key(vmax_ord(img, S, x, y, z, 1, 1, 1), cube_L(S, 0, x, y, z));
    return make_key(vmax_ord(img, S, x, y, 0, 1, 1, 0), cube_L(S, 0, x, y, 0));
}

// facet f (0-based code) of the top cube at (x,y,z): its key and the cube on the other side
__device__ __forceinline__ uint64_t facet_key(const float *img, const Seg &S, int x, int y, int z, int f, int &ox,
                                              int &oy, int &oz) {
    ox = x; oy = y; oz = z;
    if (S.edim == 2) {
        // 0: x-edge at (x,y) [-y], 1: x-edge at (x,y+1) [+y], 2: y-edge at (x,y) [-x], 3: y-edge at (x+1,y) [+x]
        if (f < 2) {
            int yy = y + f;
            oy = f ? y + 1 : y - 1;
            return make_key(vmax_ord(img, S, x, yy, 0, 1, 0, 0), cube_L(S, 0, x, yy, 0));
        }
        int xx = x + (f - 2);
        ox = (f - 2) ? x + 1 : x - 1;
        return make_key(vmax_ord(img, S, xx, y, 0, 0, 1, 0), cube_L(S, 1, xx, y, 0));
    }
    // 3D: 0/1 face {x,y} (m=0) at z / z+1; 2/3 face {x,z} (m=1) at y / y+1; 4/5 face {y,z} (m=2) at x / x+1
    int ax = 2 - (f >> 1);  // 0,1 -> z(2); 2,3 -> y(1); 4,5 -> x(0)
    int up = f & 1;
    int ax_x = x, ax_y = y, ax_z = z;
    if (ax == 2) { ax_z += up; oz = up ? z + 1 : z - 1; return make_key(vmax_ord(img, S, ax_x, ax_y, ax_z, 1, 1, 0), cube_L(S, 0, ax_x, ax_y, ax_z)); }
    if (ax == 1) { ax_y += up; oy = up ? y + 1 : y - 1; return make_key(vmax_ord(img, S, ax_x, ax_y, ax_z, 1, 0, 1), cube_L(S, 1, ax_x, ax_y, ax_z)); }
    ax_x += up; ox = up ? x + 1 : x - 1;
    return make_key(vmax_ord(img, S, ax_x, ax_y, ax_z, 0, 1, 1), cube_L(S, 2, ax_x, ax_y, ax_z));
}

__device__ __forceinline__ bool cell_in(const Seg &S, int x, int y, int z) {
    if (x < 0 || y < 0 || z < 0 || x >= S.nx - 1 || y >= S.ny - 1) return false;
    if (S.edim == 3) return z < S.nz - 1;
    return z == 0;
}

__global__ void k_dual_stencil(const float *__restrict__ img, const Seg *__restrict__ segs, int nseg,
                               uint32_t *__restrict__ parent, uint8_t *__restrict__ dd, PairBuf pb, uint32_t flags) {
    const int si = block_seg(segs, nseg);
    const Seg S = segs[si];
    if (blockIdx.x == S.toff && threadIdx.x == 0) {  // the outer node
        parent[S.coff + S.ncell] = (uint32_t)(S.coff + S.ncell);
        dd[S.coff + S.ncell] = 0;
    }
    if (S.ncell == 0) return;
    int x, y, z0, z1;
    tile_column(S, x, y, z0, z1);
    for (int z = z0; z < z1; z++) {
        if (!cell_in(S, x, y, z)) continue;
        const int64_t gc = S.coff + cell_index(S, x, y, z);
        uint64_t kc = top_key(img, S, x, y, z);
        int nf = S.edim == 3 ? 6 : 4;
        uint64_t best = 0;
        int bf = -1, bx = 0, by = 0, bz = 0;
        for (int f = 0; f < nf; f++) {
            int ox, oy, oz;
            uint64_t fk = facet_key(img, S, x, y, z, f, ox, oy, oz);
            if (bf < 0 || fk > best) { best = fk; bf = f; bx = ox; by = oy; bz = oz; }
        }
        bool hook;
        int64_t other;
        if (!cell_in(S, bx, by, bz)) {
            hook = true;  // the outer node is the oldest
            other = S.coff + S.ncell;
        } else {
            uint64_t ko = top_key(img, S, bx, by, bz);
            hook = ko > kc;  // larger key = older in the reversed order
            other = S.coff + cell_index(S, bx, by, bz);
        }
        if (hook) {
            parent[gc] = (uint32_t)other;
            dd[gc] = (uint8_t)(bf + 1);
            if (flags & CR_KEEP_ZERO)
                emit_pair(pb, (uint32_t)si, S.edim - 1, key_value(best), key_value(kc), key_L(best), key_L(kc), 0);
        } else {
            parent[gc] = (uint32_t)gc;
            dd[gc] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// The dual stencil fed by TMA (single 2D/3D images whose rows are 16-byte
// multiples).  The block's cubes, their vertices and the far vertices of every
// neighbour cube sit in one box (x from 4 voxels early, y and z from one
// voxel early, two past the tile in +y and +z).
// In the reversed order a cube's minimum dual edge is its facet with the
// largest key: the facets holding a vertex of the cube's value phi(c) all
// have value phi(c), the others less, and among those the smallest L wins,
// which is the first in the order -z, +z, -y, +y, -x, +x (2D: -y, +y, -x, +x).
// The neighbour across it shares that facet, so its value is max(phi(c), fo)
// with fo the largest of its other vertices: it is older if fo > phi(c), and
// otherwise (equal value) exactly when it lies on the - side (smaller L).
// ---------------------------------------------------------------------------
template <int EDIM>
__global__ void __launch_bounds__(TILE_X *TILE_Y) k_dual_stencil_tma(const __grid_constant__ CUtensorMap tmap,
                                                                    const Seg *__restrict__ segs,
                                                                    uint32_t *__restrict__ parent,
                                                                    uint8_t *__restrict__ dd, int *status,
                                                                    PairBuf pb, uint32_t flags) {
    constexpr int BZ = EDIM == 3 ? DUAL_BZ3 : 1;
    constexpr uint32_t BOX_BYTES = (uint32_t)BZ * DUAL_BY * DUAL_BX * 4;
    __shared__ __align__(128) float box[BZ][DUAL_BY][DUAL_BX];
    __shared__ uint32_t lp[EDIM == 2 ? TILE_Y * TILE_X : 1];  // in-tile hooks (2D only)
    __shared__ __align__(8) uint64_t bar;
    constexpr uint32_t GLOBAL = 0x80000000u;  // lp entry: ancestor outside the tile (global index)
    const Seg S = segs[0];
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    int x0, y0, z0;
    tile_origin(S, blockIdx.x, x0, y0, z0);
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    if (leader) {
        if (blockIdx.x == 0) {  // the outer node
            parent[S.coff + S.ncell] = (uint32_t)(S.coff + S.ncell);
            dd[S.coff + S.ncell] = 0;
        }
        tma_load_3d(&tmap, &box[0][0][0], &bar, BOX_BYTES, x0 - 4, y0 - 1, EDIM == 3 ? z0 - 1 : 0);
    }
    __syncthreads();
    // the wait's outcome is made uniform so that no thread is left at a later barrier
    if (!__syncthreads_and(mbar_wait(&bar, 1ll << 24))) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            set_status(status, CR_ERR_TIMEOUT);
            mbar_wait(&bar, 1ll << 24);  // let a copy still in flight land before the block exits
        }
        return;
    }
    const int cx = nx - 1, cy = ny - 1, cz = EDIM == 3 ? nz - 1 : 1;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const int tl = threadIdx.y * TILE_X + threadIdx.x;
    const bool incell = x < cx && y < cy;
    if (EDIM == 2 && !incell) lp[tl] = (uint32_t)tl;  // never referenced
    if (EDIM == 3 && !incell) return;
    const int bx = threadIdx.x + 4, by = threadIdx.y + 1;
    const int zend = EDIM == 3 ? min(TILE_Z, cz - z0) : 1;
    const uint32_t outer = (uint32_t)(S.coff + S.ncell);
    bool nan_seen = false;
    for (int zz = 0; zz < zend && incell; zz++) {
        const int z = z0 + zz, bz = EDIM == 3 ? zz + 1 : 0;
        const uint32_t c = ((uint32_t)z * (uint32_t)cy + (uint32_t)y) * (uint32_t)cx + (uint32_t)x;
        float fc;
        int f;
        if (EDIM == 3) {
            const float v000 = box[bz][by][bx], v001 = box[bz][by][bx + 1];
            const float v010 = box[bz][by + 1][bx], v011 = box[bz][by + 1][bx + 1];
            const float v100 = box[bz + 1][by][bx], v101 = box[bz + 1][by][bx + 1];
            const float v110 = box[bz + 1][by + 1][bx], v111 = box[bz + 1][by + 1][bx + 1];
            const float sum = ((v000 + v001) + (v010 + v011)) + ((v100 + v101) + (v110 + v111));
            if (sum != sum)  // a NaN, or infinities of both signs
                nan_seen |= v000 != v000 || v001 != v001 || v010 != v010 || v011 != v011 || v100 != v100 ||
                            v101 != v101 || v110 != v110 || v111 != v111;
            const float zlo = fmaxf(fmaxf(v000, v001), fmaxf(v010, v011));
            const float zhi = fmaxf(fmaxf(v100, v101), fmaxf(v110, v111));
            const float ylo = fmaxf(fmaxf(v000, v001), fmaxf(v100, v101));
            const float yhi = fmaxf(fmaxf(v010, v011), fmaxf(v110, v111));
            const float xlo = fmaxf(fmaxf(v000, v010), fmaxf(v100, v110));
            fc = fmaxf(zlo, zhi);
            f = zlo == fc ? 0 : zhi == fc ? 1 : ylo == fc ? 2 : yhi == fc ? 3 : xlo == fc ? 4 : 5;
        } else {
            const float v00 = box[0][by][bx], v01 = box[0][by][bx + 1];
            const float v10 = box[0][by + 1][bx], v11 = box[0][by + 1][bx + 1];
            const float sum = (v00 + v01) + (v10 + v11);
            if (sum != sum) nan_seen |= v00 != v00 || v01 != v01 || v10 != v10 || v11 != v11;
            const float ylo = fmaxf(v00, v01), yhi = fmaxf(v10, v11), xlo = fmaxf(v00, v10);
            fc = fmaxf(ylo, yhi);
            f = ylo == fc ? 0 : yhi == fc ? 1 : xlo == fc ? 2 : 3;
        }
        // the neighbour across facet f: outside the image (the outer node), or
        // the cube whose far vertices lie one step further
        const int axis = EDIM == 3 ? 2 - (f >> 1) : 1 - (f >> 1);  // 0 x, 1 y, 2 z
        const bool up = f & 1;
        const int coord = axis == 0 ? x : (axis == 1 ? y : z);
        const int ext = axis == 0 ? cx : (axis == 1 ? cy : cz);
        const bool outside = up ? coord + 1 >= ext : coord == 0;
        bool hook = true;
        uint32_t other = outer;
        if (!outside) {
            float fo;
            if (axis == 0) {
                const int xx = up ? bx + 2 : bx - 1;
                fo = fmaxf(box[bz][by][xx], box[bz][by + 1][xx]);
                if (EDIM == 3) fo = fmaxf(fo, fmaxf(box[bz + 1][by][xx], box[bz + 1][by + 1][xx]));
                other = up ? c + 1 : c - 1;
            } else if (axis == 1) {
                const int yy = up ? by + 2 : by - 1;
                fo = fmaxf(box[bz][yy][bx], box[bz][yy][bx + 1]);
                if (EDIM == 3) fo = fmaxf(fo, fmaxf(box[bz + 1][yy][bx], box[bz + 1][yy][bx + 1]));
                other = up ? c + (uint32_t)cx : c - (uint32_t)cx;
            } else {
                const int zb = up ? bz + 2 : bz - 1;
                fo = fmaxf(fmaxf(box[zb][by][bx], box[zb][by][bx + 1]),
                           fmaxf(box[zb][by + 1][bx], box[zb][by + 1][bx + 1]));
                const uint32_t pl = (uint32_t)cx * (uint32_t)cy;
                other = up ? c + pl : c - pl;
            }
            hook = fo > fc || !up;  // the neighbour's value is max(fo, phi(c))
            other += (uint32_t)S.coff;
        }
        const uint32_t gc = (uint32_t)S.coff + c;
        if (hook) {
            if (EDIM == 2) {
                // the same hook inside the tile, when it stays there
                const bool inside = !outside && (axis == 0 ? (up ? threadIdx.x + 1 < TILE_X : threadIdx.x > 0)
                                                           : (up ? threadIdx.y + 1 < TILE_Y : threadIdx.y > 0));
                const int lstep = axis == 0 ? 1 : TILE_X;
                lp[tl] = inside ? (uint32_t)(up ? tl + lstep : tl - lstep) : (GLOBAL | other);
            } else {
                parent[gc] = other;
            }
            dd[gc] = (uint8_t)(f + 1);
            if (flags & CR_KEEP_ZERO) {
                uint32_t fl;
                if (EDIM == 3) {
                    const int m = 2 - axis;  // face type: 0 normal z, 1 normal y, 2 normal x
                    fl = cube_L(S, m, x + (axis == 0 && up), y + (axis == 1 && up), z + (axis == 2 && up));
                } else {
                    const int m = 1 - axis;  // 0 x-edge (normal y), 1 y-edge (normal x)
                    fl = cube_L(S, m, x + (axis == 0 && up), y + (axis == 1 && up), 0);
                }
                const float cv = unord32(ord32(fc));
                emit_pair(pb, 0u, EDIM - 1, cv, cv, fl, cube_L(S, 0, x, y, z), 0);
            }
        } else {
            if (EDIM == 2)
                lp[tl] = (uint32_t)tl;
            else
                parent[gc] = gc;
            dd[gc] = 0;
        }
    }
    if (nan_seen) set_status(status, CR_ERR_NAN);
    if (EDIM == 3) return;
    // 2D: follow the hooks inside the tile (every write stores an ancestor)
    __syncthreads();
    for (int it = 0; it < 64; it++) {
        int ch = 0;
        const uint32_t p = lp[tl];
        if (!(p & GLOBAL)) {
            const uint32_t q = lp[p];
            if (q != p) {
                lp[tl] = q;
                ch = 1;
            }
        }
        if (!__syncthreads_or(ch)) break;
    }
    if (!incell) return;
    const uint32_t p = lp[tl];
    uint32_t g;
    if (p & GLOBAL) {
        g = p & ~GLOBAL;
    } else {
        const int py = (int)p / TILE_X, px = (int)p % TILE_X;
        g = (uint32_t)S.coff + (uint32_t)(y0 + py) * (uint32_t)cx + (uint32_t)(x0 + px);
    }
    parent[(uint32_t)S.coff + (uint32_t)y * (uint32_t)cx + (uint32_t)x] = g;
}


// dual edges = facets of the top cubes, iterated over the L-space of type m
__global__ void k_dual_cross(const float *__restrict__ img, const Seg *__restrict__ segs, int nseg,
                             const uint32_t *__restrict__ lab, const uint8_t *__restrict__ dd,
                             uint64_t *__restrict__ ek, uint32_t *__restrict__ ea, uint32_t *__restrict__ eb,
                             unsigned long long *ne, int64_t max_edges, const unsigned long long *ngroups,
                             int *status) {
    const uint32_t ng = (uint32_t)*ngroups;
    const int si = block_seg(segs, nseg);
    const Seg S = segs[si];
    int x, y, z0, z1;
    tile_column(S, x, y, z0, z1);
    const bool inxy = S.ncell > 0 && x < S.nx && y < S.ny;
    // Facets of one type met in consecutive planes often join the same two
    // groups (groups of the dual are runs along z).  Of parallel edges
    // between two groups only the first in the order can merge them, so a
    // run of equal group pairs is kept as one edge: its smallest key.
    uint64_t pk[3];
    uint32_t pa[3], pb[3];
    bool pend[3] = {false, false, false};
    for (int z = z0; z <= z1; z++) {
        const bool in = inxy && z < z1;
        uint64_t keys[3];
        uint32_t las[3], lbs[3];
        int cnt = 0;
        for (int m = 0; m < 3; m++) {
            bool emit = false;
            uint64_t key = 0;
            uint32_t la = 0, lb = 0;
            if (in && (S.edim == 3 || m < 2)) {
                // the two sides (a = "minus" side cube, b = "plus" side cube) and the facet code on each side
                int ax, ay, az, bx = x, by = y, bz = z, fa, fb;
                bool exists;
                uint64_t fk = 0;
                if (S.edim == 2) {
                    if (m == 0) {  // x-edge at (x,y)
                        exists = x + 1 < S.nx;
                        ax = x; ay = y - 1; az = 0; fa = 1; fb = 0;
                        if (exists) fk = make_key(vmax_ord(img, S, x, y, 0, 1, 0, 0), cube_L(S, 0, x, y, 0));
                    } else {  // y-edge at (x,y)
                        exists = y + 1 < S.ny;
                        ax = x - 1; ay = y; az = 0; fa = 3; fb = 2;
                        if (exists) fk = make_key(vmax_ord(img, S, x, y, 0, 0, 1, 0), cube_L(S, 1, x, y, 0));
                    }
                } else {
                    if (m == 0) {  // face {x,y}
                        exists = x + 1 < S.nx && y + 1 < S.ny;
                        ax = x; ay = y; az = z - 1; fa = 1; fb = 0;
                        if (exists) fk = make_key(vmax_ord(img, S, x, y, z, 1, 1, 0), cube_L(S, 0, x, y, z));
                    } else if (m == 1) {  // face {x,z}
                        exists = x + 1 < S.nx && z + 1 < S.nz;
                        ax = x; ay = y - 1; az = z; fa = 3; fb = 2;
                        if (exists) fk = make_key(vmax_ord(img, S, x, y, z, 1, 0, 1), cube_L(S, 1, x, y, z));
                    } else {  // face {y,z}
                        exists = y + 1 < S.ny && z + 1 < S.nz;
                        ax = x - 1; ay = y; az = z; fa = 5; fb = 4;
                        if (exists) fk = make_key(vmax_ord(img, S, x, y, z, 0, 1, 1), cube_L(S, 2, x, y, z));
                    }
                }
                if (exists) {
                    int64_t outer = S.coff + S.ncell;
                    bool ina = cell_in(S, ax, ay, az), inb = cell_in(S, bx, by, bz);
                    int64_t na = ina ? S.coff + cell_index(S, ax, ay, az) : outer;
                    int64_t nb = inb ? S.coff + cell_index(S, bx, by, bz) : outer;
                    bool stencil = (ina && dd[na] == (uint8_t)(fa + 1)) || (inb && dd[nb] == (uint8_t)(fb + 1));
                    if (!stencil) {
                        la = lab[na];
                        lb = lab[nb];
                        if (la != lb) {
                            emit = true;
                            key = ~fk;
                        }
                    }
                }
            }
            if (emit && (la >= ng || lb >= ng)) {
                set_status(status, CR_ERR_INTERNAL);
                emit = false;
            }
            if (emit && pend[m] && pa[m] == la && pb[m] == lb) {
                pk[m] = key < pk[m] ? key : pk[m];  // the same two groups: one edge
                continue;
            }
            if (pend[m] && (emit || z == z1)) {  // the run ends: its edge goes out
                keys[cnt] = pk[m];
                las[cnt] = pa[m];
                lbs[cnt] = pb[m];
                cnt++;
                pend[m] = false;
            }
            if (emit) {
                pk[m] = key;
                pa[m] = la;
                pb[m] = lb;
                pend[m] = true;
            }
        }
        int64_t i = block_append(cnt, ne);
        for (int k = 0; k < cnt; k++) {
            if (i + k < max_edges) {
                ek[i + k] = keys[k];
                ea[i + k] = las[k];
                eb[i + k] = lbs[k];
            } else {
                fail_ws(status, SITE_EDGES);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Batches of 2D images: both stencils in one kernel.  A block stages a 32x32
// super-tile of one image with a halo (x0-1 .. x0+33, y0-1 .. y0+33) in
// shared memory with plain coalesced loads; every pixel takes its primal hook
// (as in k_h0_stencil_tma) and every square its dual hook (as in
// k_dual_stencil_tma); both sets of hooks are then followed inside the
// super-tile, so that each node leaves with its in-tile root or its first
// ancestor outside the super-tile.
// ---------------------------------------------------------------------------
constexpr int SB_X = ST_X + 3, SB_Y = ST_Y + 3;
__global__ void __launch_bounds__(256) k_stencil2d_batch(const float *__restrict__ img, const Seg *__restrict__ segs,
                                                        int nseg, uint32_t *__restrict__ parent,
                                                        uint8_t *__restrict__ dd, uint32_t *__restrict__ parentc,
                                                        uint8_t *__restrict__ ddc, int *status, PairBuf pb,
                                                        uint32_t flags) {
    constexpr uint32_t GLOBAL = 0x80000000u;
    __shared__ float box[SB_Y][SB_X + 1];
    __shared__ uint32_t lp[ST_Y * ST_X], lq[ST_Y * ST_X];
    __shared__ int s_si;
    if (threadIdx.x == 0) {
        int lo = 0, hi = nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int64_t)segs[mid].stoff <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        s_si = lo;
    }
    __syncthreads();
    const int si = s_si;
    const Seg S = segs[si];
    const int nx = S.nx, ny = S.ny, cx = nx - 1, cy = ny - 1;
    const int sx = (nx + ST_X - 1) / ST_X;
    const int t = (int)blockIdx.x - S.stoff;
    const int x0 = (t % sx) * ST_X, y0 = (t / sx) * ST_Y;
    const float *im = img + S.voff;
    bool nan_seen = false;
    for (int i = threadIdx.x; i < SB_Y * SB_X; i += 256) {
        const int by = i / SB_X, bx = i % SB_X;
        const int gx = x0 - 1 + bx, gy = y0 - 1 + by;
        float v = 0.f;
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
            v = im[(int64_t)gy * nx + gx];
            nan_seen |= isnan(v);
        }
        box[by][bx] = v;
    }
    const bool do_p = parent != nullptr, do_d = parentc != nullptr && S.ncell > 0;
    if (do_d && t == 0 && threadIdx.x == 0) {  // the outer node
        parentc[S.coff + S.ncell] = (uint32_t)(S.coff + S.ncell);
        ddc[S.coff + S.ncell] = 0;
    }
    __syncthreads();
    const int tx = threadIdx.x & 31;
    const uint32_t P = (uint32_t)nx * (uint32_t)ny;  // one type's L-range (nz = 1)
#pragma unroll
    for (int k = 0; k < ST_Y / 8; k++) {
        const int ty = (threadIdx.x >> 5) + 8 * k;
        const int li = ty * ST_X + tx;
        const int x = x0 + tx, y = y0 + ty;
        const int bx = tx + 1, by = ty + 1;
        // ---- primal: the first neighbour with phi <= phi(v) in descending edge-L order (+y, -y, +x, -x)
        if (do_p) {
            if (x < nx && y < ny) {
                const float fv = box[by][bx];
                int dir = 0;
                float fu = 0.f;
                if (x > 0 && box[by][bx - 1] <= fv) { dir = 1; fu = box[by][bx - 1]; }
                if (x + 1 < nx && box[by][bx + 1] <= fv) { dir = 2; fu = box[by][bx + 1]; }
                if (y > 0 && box[by - 1][bx] <= fv) { dir = 3; fu = box[by - 1][bx]; }
                if (y + 1 < ny && box[by + 1][bx] <= fv) { dir = 4; fu = box[by + 1][bx]; }
                const uint32_t lv = (uint32_t)y * nx + x;
                if (dir && (fu < fv || !(dir & 1))) {
                    const uint32_t stp = dir <= 2 ? 1u : (uint32_t)nx;
                    const uint32_t lu = (dir & 1) ? lv - stp : lv + stp;
                    const bool inside = dir == 1 ? tx > 0 : dir == 2 ? tx + 1 < ST_X : dir == 3 ? ty > 0 : ty + 1 < ST_Y;
                    const int lstep = dir <= 2 ? 1 : ST_X;
                    lp[li] = inside ? (uint32_t)((dir & 1) ? li - lstep : li + lstep)
                                    : (GLOBAL | (uint32_t)(S.voff + lu));
                    dd[S.voff + lv] = (uint8_t)dir;
                    if (flags & CR_KEEP_ZERO) {
                        const uint32_t la = ((dir & 1) ? lu : lv) + (dir >= 3 ? P : 0u);
                        const float cv = unord32(ord32(fv));
                        emit_pair(pb, (uint32_t)si, 0, cv, cv, lv, la, 0);
                    }
                } else {
                    lp[li] = (uint32_t)li;
                    dd[S.voff + lv] = 0;
                }
            } else {
                lp[li] = (uint32_t)li;
            }
        }
        // ---- dual: the square's first facet (-y, +y, -x, +x) holding its value
        if (do_d) {
            if (x < cx && y < cy) {
                const float v00 = box[by][bx], v01 = box[by][bx + 1], v10 = box[by + 1][bx], v11 = box[by + 1][bx + 1];
                const float ylo = fmaxf(v00, v01), yhi = fmaxf(v10, v11), xlo = fmaxf(v00, v10);
                const float fc = fmaxf(ylo, yhi);
                const int f = ylo == fc ? 0 : yhi == fc ? 1 : xlo == fc ? 2 : 3;
                const int axis = 1 - (f >> 1);  // 0 x, 1 y
                const bool up = f & 1;
                const uint32_t c = (uint32_t)y * (uint32_t)cx + (uint32_t)x;
                const bool outside = axis == 0 ? (up ? x + 1 >= cx : x == 0) : (up ? y + 1 >= cy : y == 0);
                bool hook = true;
                uint32_t other = (uint32_t)(S.coff + S.ncell);
                bool inside = false;
                int lother = 0;
                if (!outside) {
                    float fo;
                    if (axis == 0) {
                        const int xx = up ? bx + 2 : bx - 1;
                        fo = fmaxf(box[by][xx], box[by + 1][xx]);
                        other = (uint32_t)S.coff + (up ? c + 1 : c - 1);
                        inside = up ? tx + 1 < ST_X : tx > 0;
                        lother = up ? li + 1 : li - 1;
                    } else {
                        const int yy = up ? by + 2 : by - 1;
                        fo = fmaxf(box[yy][bx], box[yy][bx + 1]);
                        other = (uint32_t)S.coff + (up ? c + (uint32_t)cx : c - (uint32_t)cx);
                        inside = up ? ty + 1 < ST_Y : ty > 0;
                        lother = up ? li + ST_X : li - ST_X;
                    }
                    hook = fo > fc || !up;  // the neighbour's value is max(fo, phi(c))
                }
                const uint32_t gc = (uint32_t)S.coff + c;
                if (hook) {
                    lq[li] = inside ? (uint32_t)lother : (GLOBAL | other);
                    ddc[gc] = (uint8_t)(f + 1);
                    if (flags & CR_KEEP_ZERO) {
                        const int m = 1 - axis;
                        const uint32_t fl = cube_L(S, m, x + (axis == 0 && up), y + (axis == 1 && up), 0);
                        const float cv = unord32(ord32(fc));
                        emit_pair(pb, (uint32_t)si, 1, cv, cv, fl, cube_L(S, 0, x, y, 0), 0);
                    }
                } else {
                    lq[li] = (uint32_t)li;
                    ddc[gc] = 0;
                }
            } else {
                lq[li] = (uint32_t)li;
            }
        }
    }
    if (nan_seen) set_status(status, CR_ERR_NAN);
    __syncthreads();
    // follow both sets of hooks inside the super-tile (every write stores an ancestor)
    for (int it = 0; it < 64; it++) {
        int ch = 0;
#pragma unroll
        for (int k = 0; k < ST_Y / 8; k++) {
            const int li = ((threadIdx.x >> 5) + 8 * k) * ST_X + tx;
            if (do_p) {
                const uint32_t p = lp[li];
                if (!(p & GLOBAL)) {
                    const uint32_t q = lp[p];
                    if (q != p) { lp[li] = q; ch = 1; }
                }
            }
            if (do_d) {
                const uint32_t p = lq[li];
                if (!(p & GLOBAL)) {
                    const uint32_t q = lq[p];
                    if (q != p) { lq[li] = q; ch = 1; }
                }
            }
        }
        if (!__syncthreads_or(ch)) break;
    }
#pragma unroll
    for (int k = 0; k < ST_Y / 8; k++) {
        const int ty = (threadIdx.x >> 5) + 8 * k;
        const int li = ty * ST_X + tx;
        const int x = x0 + tx, y = y0 + ty;
        if (do_p && x < nx && y < ny) {
            const uint32_t p = lp[li];
            parent[S.voff + (int64_t)y * nx + x] =
                (p & GLOBAL) ? (p & ~GLOBAL)
                             : (uint32_t)(S.voff + (int64_t)(y0 + (int)p / ST_X) * nx + x0 + (int)p % ST_X);
        }
        if (do_d && x < cx && y < cy) {
            const uint32_t p = lq[li];
            parentc[S.coff + (int64_t)y * cx + x] =
                (p & GLOBAL) ? (p & ~GLOBAL)
                             : (uint32_t)(S.coff + (int64_t)(y0 + (int)p / ST_X) * cx + x0 + (int)p % ST_X);
        }
    }
}

// ===========================================================================
// host drivers
// ===========================================================================


// ---------------------------------------------------------------------------
// All Boruvka rounds in one cooperative kernel: the counts stay on the
// device, phases are separated by a grid barrier with a bounded spin.  The
// primal graph (H0) and the dual graph (top dimension) are independent, so one
// launch runs both in lock step and they share every barrier.
// ---------------------------------------------------------------------------
constexpr int MAX_GRAPHS = 2;
struct RoundArgs {
    UF u[MAX_GRAPHS];
    int ngraph;
    int compact_mult;  // compact the edge list while it holds > compact_mult edges per thread
    int *status;
    long long polls;   // poll limit of each barrier wait
    unsigned int extra;  // arrivals the barriers expect beyond the grid (0; error-path tests only)
};

// Grid barrier on a monotonic arrival counter: thread 0 of every block adds 1
// with release semantics and polls with acquire loads until all blocks of
// barrier number n have arrived (counter >= n * blocks).  Returns false when
// another block reported an error or the wait gave up after `limit` polls
// (CR_ERR_TIMEOUT).
__device__ __forceinline__ bool grid_barrier(unsigned int *count, unsigned int &target, int *status,
                                             long long limit) {
    __shared__ int s_ok;
    target += gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
        for (long long polls = 1;; polls++) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if ((int)(v - target) >= 0) break;
            if ((polls & 63) == 0) {
                if (*(volatile int *)status) { ok = 0; break; }
                if (polls > limit) {
                    set_status(status, CR_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// Hooks of a volume's dual graph run along z only: a cube's minimum dual edge
// is one of its two z-facets (see k_dual_stencil_tma), so it hooks to the cube
// below, the cube above, the outer node or nothing.  A chain of hooks keeps
// its direction (a cube hooked to the one below is older than it, so that
// cube cannot hook back up).  One upward sweep of each (x, y) column of cubes
// therefore resolves the downward chains and one downward sweep the upward
// ones, leaving every cube pointing at its root; pointer jumping would take
// log2 of the longest chain (up to nz) passes over every cube to get there.
// ---------------------------------------------------------------------------
__global__ void k_dual_zsweep(uint32_t *__restrict__ parent, uint32_t coff, int cx, int cy, int cz) {
    const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= (int64_t)cx * cy) return;
    const int64_t pl = (int64_t)cx * cy;
    uint32_t *p = parent + coff + col;
    const uint32_t g0 = coff + (uint32_t)col;
    // targets are read eight planes at a time (a sweep writes only the cube
    // it is at, so the cubes ahead still hold their stencil hooks)
    constexpr int DEPTH = 8;
    uint32_t below = 0;  // the final target of the cube below
    for (int z0 = 0; z0 < cz; z0 += DEPTH) {
        uint32_t t[DEPTH];
#pragma unroll
        for (int k = 0; k < DEPTH; k++) t[k] = z0 + k < cz ? __ldcg(p + (z0 + k) * pl) : 0u;
#pragma unroll
        for (int k = 0; k < DEPTH; k++) {
            const int z = z0 + k;
            if (z >= cz) break;
            if (z > 0 && t[k] == g0 + (uint32_t)((z - 1) * pl)) {
                t[k] = below;
                p[z * pl] = below;
            }
            below = t[k];
        }
    }
    uint32_t above = 0;  // the final target of the cube above
    for (int z1 = cz - 1; z1 >= 0; z1 -= DEPTH) {
        uint32_t t[DEPTH];
#pragma unroll
        for (int k = 0; k < DEPTH; k++) t[k] = z1 - k >= 0 ? __ldcg(p + (z1 - k) * pl) : 0u;
#pragma unroll
        for (int k = 0; k < DEPTH; k++) {
            const int z = z1 - k;
            if (z < 0) break;
            if (z + 1 < cz && t[k] == g0 + (uint32_t)((z + 1) * pl)) {
                t[k] = above;
                p[z * pl] = above;
            }
            above = t[k];
        }
    }
}


// ---------------------------------------------------------------------------
// Basins in one cooperative launch (one 1024-thread block per SM), for one or
// both graphs at once:
//   passes of in-place pointer doubling until a pass changes nothing (every
//   write stores an ancestor, and a pass without writes saw every node
//   pointing at a root);
//   roots take group ids (primal: age key of the root vertex; dual: reversed
//   key of the root cube, the outer node oldest);
//   every node's label becomes its root's group id.
// ---------------------------------------------------------------------------
constexpr int BASIN_THREADS = 1024;
struct BasinArgs {
    const float *img;
    const Seg *segs;
    int nseg;
    int ngraph;
    int mode[MAX_GRAPHS];  // 0 primal vertices, 1 dual nodes (top cubes + outer nodes)
    int64_t n[MAX_GRAPHS];
    UF u[MAX_GRAPHS];
    int *status;
    long long polls;     // poll limit of each barrier wait
    unsigned int extra;  // arrivals the barriers expect beyond the grid (0; error-path tests only)
};

__device__ __forceinline__ int doubling_pass(uint32_t *lab, int64_t n, int64_t tid, int64_t nthr) {
    int ch = 0;
    int64_t i = tid;
    for (; i + 3 * nthr < n; i += 4 * nthr) {
        uint32_t a[4], b[4];
#pragma unroll
        for (int k = 0; k < 4; k++) a[k] = __ldcg(lab + i + k * nthr);
#pragma unroll
        for (int k = 0; k < 4; k++) b[k] = __ldcg(lab + a[k]);
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (b[k] != a[k]) {
                lab[i + k * nthr] = b[k];
                ch = 1;
            }
    }
    for (; i < n; i += nthr) {
        const uint32_t a = __ldcg(lab + i), b = __ldcg(lab + a);
        if (b != a) {
            lab[i] = b;
            ch = 1;
        }
    }
    return ch;
}

__global__ void __launch_bounds__(BASIN_THREADS, 1) k_basins(BasinArgs A) {
    if (*(volatile int *)A.status) return;
    unsigned int *bar = (unsigned int *)&A.u[0].cnt[UFC_BAR_BASINS];
    unsigned int target = A.extra;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    bool live[MAX_GRAPHS] = {A.ngraph > 0, A.ngraph > 1};
    for (int pass = 0; pass < 64; pass++) {
#pragma unroll
        for (int gi = 0; gi < MAX_GRAPHS; gi++) {
            if (!live[gi]) continue;
            unsigned long long *cnt = A.u[gi].cnt;
            if (tid == 0) {
                cnt[UFC_CHANGED + (pass + 1) % 3] = 0;  // last read two barriers ago
                cnt[UFC_PASSES] += 1ull;
            }
            const int ch = doubling_pass(A.u[gi].lab, A.n[gi], tid, nthr);
            if (__syncthreads_or(ch) && threadIdx.x == 0) atomicAdd(&cnt[UFC_CHANGED + pass % 3], 1ull);
        }
        if (!grid_barrier(bar, target, A.status, A.polls)) return;
        bool any = false;
#pragma unroll
        for (int gi = 0; gi < MAX_GRAPHS; gi++) {
            if (live[gi] && __ldcg(&A.u[gi].cnt[UFC_CHANGED + pass % 3]) == 0) live[gi] = false;
            any |= live[gi];
        }
        if (!any) break;
        if (pass == 63) {
            set_status(A.status, CR_ERR_INTERNAL);
            return;
        }
    }
    // roots
#pragma unroll
    for (int gi = 0; gi < MAX_GRAPHS; gi++) {
        if (gi >= A.ngraph) break;
        const UF &u = A.u[gi];
        uint32_t *lab = u.lab;
        const int64_t n = A.n[gi];
        for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += nthr) {
            const int64_t v = base + threadIdx.x;
            const bool isroot = v < n && __ldcg(lab + v) == (uint32_t)v;
            const int64_t g = warp_append(isroot, &u.cnt[UFC_GROUPS]);
            if (!isroot) continue;
            if (g >= u.max_groups) {
                fail_ws(A.status, SITE_GROUPS);
                lab[v] = 0x80000000u;
                continue;
            }
            uint64_t key;
            int si;
            if (A.mode[gi] == 0) {
                si = seg_of(A.segs, A.nseg, v);
                const int64_t lv = v - A.segs[si].voff;
                key = make_key(ord32(A.img[v]), (uint32_t)lv);
            } else {
                si = seg_of_node(A.segs, A.nseg, v);
                const Seg S = A.segs[si];
                const int64_t c = v - S.coff;
                key = 0;  // outer node: oldest
                if (c < S.ncell) {
                    const CellPos p = cell_pos(S, c);
                    key = ~top_key(A.img, S, p.x, p.y, p.z);
                }
            }
            u.gkey[g] = key;
            u.groot[g] = (uint32_t)v;
            u.gseg[g] = (uint32_t)si;
            lab[v] = 0x80000000u | (uint32_t)g;
        }
    }
    if (!grid_barrier(bar, target, A.status, A.polls)) return;
    // labels -> group ids (roots are marked; every other node points at a root)
#pragma unroll
    for (int gi = 0; gi < MAX_GRAPHS; gi++) {
        if (gi >= A.ngraph) break;
        uint32_t *lab = A.u[gi].lab;
        const int64_t n = A.n[gi];
        for (int64_t i = tid; i < n; i += nthr) {
            const uint32_t v = __ldcg(lab + i);
            lab[i] = (v & 0x80000000u) ? (v & 0x7FFFFFFFu) : (__ldcg(lab + v) & 0x7FFFFFFFu);
        }
    }
}

constexpr int UF_THREADS = 1024;

#ifdef CR_UF_TIMING
// diagnostics build: block 0 records the global timer at every phase end
__device__ unsigned long long g_uf_trace[1024];
__device__ int g_uf_trace_n;
#define UF_MARK(v)                                                              \
    do {                                                                        \
        if (blockIdx.x == 0 && threadIdx.x == 0) {                              \
            int m_ = g_uf_trace_n;                                              \
            if (m_ < 1024) {                                                    \
                unsigned long long t_;                                          \
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));          \
                g_uf_trace[m_] = (t_ << 20) | ((unsigned long long)(v) & 0xFFFFF); \
                g_uf_trace_n = m_ + 1;                                          \
            }                                                                   \
        }                                                                       \
    } while (0)
#else
#define UF_MARK(v) \
    do {           \
    } while (0)
#endif

// per-graph state of the rounds (identical in every thread)
struct RoundState {
    int cur;          // edge buffer in use
    bool inplace;     // list kept in place (dropped edges have a == b)
    bool compact;     // this round compacts into the other buffer
    bool done;
    unsigned long long live_seen;
    int64_t ne, live, ng;
};

// Borůvka rounds under the elder rule, three phases per round:
//   B  (edges)  the edge attaining minE[g] decides g's hook: g dies into the
//               other end if that end is older (death key kept in dkey[g]).
//               Groups clear the other min-edge buffer for the next round.
//   C  (groups) pointer jumping to the round's roots; every thread writes only
//               its own group's hook, always with an ancestor
//   D  (edges)  endpoints move to their roots and are offered to the next
//               round's min edge of both ends; edges inside a group drop out
// While there are more edges than threads, D compacts the survivors into the
// other edge buffer.  Once they fit, the list stays in place: an edge whose
// ends meet is marked by a == b and skipped, which saves the compaction's
// atomic and its count read on every round's critical path.
// The first round's min edges come from a prologue phase; the deaths are
// written out after the rounds by k_uf_emit.
__device__ __forceinline__ void phase_B(const UF &u, const RoundState &R, int round, int64_t tid, int64_t nthr) {
    const uint64_t *ek = R.cur ? u.ek[1] : u.ek[0];
    const uint32_t *ea = R.cur ? u.ea[1] : u.ea[0], *eb = R.cur ? u.eb[1] : u.eb[0];
    // the min-edge buffers alternate every round, the edge buffers only
    // when the list is compacted
    const uint64_t *mcur = (round & 1) ? u.minE2 : u.minE;
    uint64_t *mnext = (round & 1) ? u.minE : u.minE2;
    for (int64_t i = tid; i < R.ne; i += nthr) {
        const uint64_t k = ek[i];
        const uint32_t e0 = ea[i], e1 = eb[i];
        if (e0 == e1) continue;  // dropped edge (in-place list)
        const uint64_t m0 = __ldcg(mcur + e0), m1 = __ldcg(mcur + e1);
        const uint64_t k0 = u.gkey[e0], k1 = u.gkey[e1];
        // only the younger end can die, and only on its own min edge
        const bool young0 = k1 < k0;
        const uint32_t g = young0 ? e0 : e1, t = young0 ? e1 : e0;
        if ((young0 ? m0 : m1) != k) continue;
        u.hook[g] = t;
        u.gdead[g] = 1;
        u.dkey[g] = k;
    }
    for (int64_t g = tid; g < R.ng; g += nthr) mnext[g] = ~0ull;
}

__device__ __forceinline__ void phase_C(const UF &u, const RoundState &R, int64_t tid, int64_t nthr) {
    for (int64_t g = tid; g < R.ng; g += nthr) {
        uint32_t p = __ldcg(u.hook + g);
        if (p == (uint32_t)g) continue;
        for (int it = 0; it < (1 << 24); it++) {
            const uint32_t pp = __ldcg(u.hook + p);
            if (pp == p) break;
            p = pp;
            u.hook[g] = p;
        }
    }
}

__device__ __forceinline__ void phase_D(const UF &u, RoundState &R, int round, int64_t tid, int64_t nthr) {
    uint64_t *ek = R.cur ? u.ek[1] : u.ek[0];
    uint32_t *ea = R.cur ? u.ea[1] : u.ea[0], *eb = R.cur ? u.eb[1] : u.eb[0];
    uint64_t *mnext = (round & 1) ? u.minE : u.minE2;
    if (R.compact) {
        unsigned long long *nnext = R.cur ? &u.cnt[UFC_E0] : &u.cnt[UFC_E1];
        uint64_t *ok = R.cur ? u.ek[0] : u.ek[1];
        uint32_t *oa = R.cur ? u.ea[0] : u.ea[1], *ob = R.cur ? u.eb[0] : u.eb[1];
        for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < R.ne; base += nthr) {
            const int64_t i = base + threadIdx.x;
            bool keep = false;
            uint32_t a = 0, b = 0;
            uint64_t k = 0, ma = 0, mb = 0;
            if (i < R.ne) {
                a = __ldcg(u.hook + ea[i]);
                b = __ldcg(u.hook + eb[i]);
                k = ek[i];
                keep = a != b;
                if (keep) {
                    ma = __ldcg(mnext + a);
                    mb = __ldcg(mnext + b);
                }
            }
            const int64_t j = block_append(keep ? 1 : 0, nnext);
            if (keep) {
                ok[j] = k;
                oa[j] = a;
                ob[j] = b;
                if (ma > k) atomicMin((unsigned long long *)&mnext[a], k);
                if (mb > k) atomicMin((unsigned long long *)&mnext[b], k);
            }
        }
        R.cur ^= 1;
    } else {
        R.inplace = true;
        int nlive = 0;
        for (int64_t i = tid; i < R.ne; i += nthr) {
            const uint32_t e0 = ea[i], e1 = eb[i];
            const uint64_t k = ek[i];
            if (e0 == e1) continue;
            const uint32_t a = __ldcg(u.hook + e0), b = __ldcg(u.hook + e1);
            if (a == b) {
                ea[i] = a;
                eb[i] = a;
                continue;
            }
            const uint64_t ma = __ldcg(mnext + a), mb = __ldcg(mnext + b);
            if (a != e0) ea[i] = a;
            if (b != e1) eb[i] = b;
            if (ma > k) atomicMin((unsigned long long *)&mnext[a], k);
            if (mb > k) atomicMin((unsigned long long *)&mnext[b], k);
            nlive++;
        }
        nlive = __reduce_add_sync(0xFFFFFFFFu, nlive);
        if ((threadIdx.x & 31) == 0 && nlive) atomicAdd(&u.cnt[UFC_LIVE], (unsigned long long)nlive);
    }
}

__global__ void __launch_bounds__(UF_THREADS, 1) k_uf_rounds(RoundArgs A) {
    unsigned int *bar = (unsigned int *)&A.u[0].cnt[UFC_BAR_ROUNDS];
    unsigned int target = A.extra;
    if (*(volatile int *)A.status) return;
#ifdef CR_UF_TIMING
    if (blockIdx.x == 0 && threadIdx.x == 0) g_uf_trace_n = 0;
#endif
    UF_MARK(0);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    RoundState R[MAX_GRAPHS];
#pragma unroll
    for (int gi = 0; gi < MAX_GRAPHS; gi++) {
        R[gi] = RoundState{0, false, false, gi >= A.ngraph, 0ull, 0, 0, 0};
        if (R[gi].done) continue;
        const UF &u = A.u[gi];
        int64_t ng = (int64_t)__ldcg(&u.cnt[UFC_GROUPS]);
        R[gi].ng = ng > u.max_groups ? u.max_groups : ng;
        for (int64_t g = tid; g < R[gi].ng; g += nthr) {
            u.gdead[g] = 0;
            u.hook[g] = (uint32_t)g;
            u.minE[g] = ~0ull;
        }
    }
    if (!grid_barrier(bar, target, A.status, A.polls)) return;
    UF_MARK(1);
#pragma unroll
    for (int gi = 0; gi < MAX_GRAPHS; gi++) {
        if (R[gi].done) continue;
        const UF &u = A.u[gi];
        int64_t ne = (int64_t)__ldcg(&u.cnt[UFC_E0]);
        R[gi].ne = ne > u.max_edges ? u.max_edges : ne;
        R[gi].live = R[gi].ne;
        for (int64_t i = tid; i < R[gi].ne; i += nthr) {
            const unsigned long long k = u.ek[0][i];
            const uint32_t a = u.ea[0][i], b = u.eb[0][i];
            if (__ldcg(u.minE + a) > k) atomicMin((unsigned long long *)&u.minE[a], k);
            if (__ldcg(u.minE + b) > k) atomicMin((unsigned long long *)&u.minE[b], k);
        }
    }
    if (!grid_barrier(bar, target, A.status, A.polls)) return;
    UF_MARK(2);
    for (int round = 0; round < (1 << 20); round++) {
        bool any = false;
#pragma unroll
        for (int gi = 0; gi < MAX_GRAPHS; gi++) {
            RoundState &S = R[gi];
            if (S.done) continue;
            const UF &u = A.u[gi];
            if (round > 0) {
                if (S.inplace) {
                    const unsigned long long v = __ldcg(&u.cnt[UFC_LIVE]);
                    S.live = (int64_t)(v - S.live_seen);
                    S.live_seen = v;
                } else {
                    const int64_t ne = (int64_t)__ldcg(S.cur ? &u.cnt[UFC_E1] : &u.cnt[UFC_E0]);
                    S.ne = ne > u.max_edges ? u.max_edges : ne;
                    S.live = S.ne;
                }
            }
            if (S.live == 0) {
                S.done = true;
                continue;
            }
            any = true;
            S.compact = !S.inplace && S.ne > nthr * (int64_t)A.compact_mult;
            if (tid == 0) {
                if (S.compact) *(S.cur ? &u.cnt[UFC_E0] : &u.cnt[UFC_E1]) = 0;
                u.cnt[UFC_VISITED] += (unsigned long long)S.live;  // for the algorithmic byte count
                u.cnt[UFC_ROUNDS] += 1ull;
            }
        }
        if (!any) break;
#pragma unroll
        for (int gi = 0; gi < MAX_GRAPHS; gi++)
            if (!R[gi].done) phase_B(A.u[gi], R[gi], round, tid, nthr);
        if (!grid_barrier(bar, target, A.status, A.polls)) return;
        UF_MARK(R[0].live);
#pragma unroll
        for (int gi = 0; gi < MAX_GRAPHS; gi++)
            if (!R[gi].done) phase_C(A.u[gi], R[gi], tid, nthr);
        if (!grid_barrier(bar, target, A.status, A.polls)) return;
        UF_MARK(R[0].live);
#pragma unroll
        for (int gi = 0; gi < MAX_GRAPHS; gi++)
            if (!R[gi].done) phase_D(A.u[gi], R[gi], round, tid, nthr);
        if (!grid_barrier(bar, target, A.status, A.polls)) return;
        UF_MARK(R[0].live);
    }
}

// After the rounds: every group that died gives one pair (primal: born at the
// group's root, dying at its death edge, which is also marked as killed in
// dimension 0 for the middle dimension; dual: the reversed pair one dimension
// up).  The one surviving primal group of each image is its essential class.
__global__ void k_uf_emit(const unsigned long long *ngp, UF u, int mode, const Seg *__restrict__ segs, PairBuf pb,
                          uint32_t flags, uint32_t *extra_mask) {
    int64_t ng = (int64_t)*ngp;
    if (ng > u.max_groups) ng = u.max_groups;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < ng; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = base + threadIdx.x;
        int emit = 0;
        cr_pair p;
        if (g < ng) {
            const uint64_t kb = u.gkey[g];
            const uint32_t si = u.gseg[g];
            if (!u.gdead[g]) {
                if (mode == 0) {
                    p = cr_pair{0, key_value(kb), __int_as_float(0x7f800000), CR_PAIR_ESSENTIAL | (si << 8),
                                (int64_t)key_L(kb), -1};
                    emit = 1;
                }
            } else {
                const uint64_t k = u.dkey[g];
                if (mode == 0) {
                    const float bv = key_value(kb), dv = key_value(k);
                    if (extra_mask) {
                        const int64_t bit = segs[si].loff + key_L(k);
                        atomicOr(&extra_mask[bit >> 5], 1u << (bit & 31));
                    }
                    if ((flags & CR_KEEP_ZERO) || bv != dv) {
                        p = cr_pair{0, bv, dv, si << 8, (int64_t)key_L(kb), (int64_t)key_L(k)};
                        emit = 1;
                    }
                } else {
                    const uint64_t kf = ~k, kc = ~kb;
                    const float bv = key_value(kf), dv = key_value(kc);
                    if ((flags & CR_KEEP_ZERO) || bv != dv) {
                        p = cr_pair{segs[si].edim - 1, bv, dv, si << 8, (int64_t)key_L(kf), (int64_t)key_L(kc)};
                        emit = 1;
                    }
                }
            }
        }
        const int64_t j = block_append(emit, pb.count);
        if (emit && j < pb.capacity) pb.pairs[j] = p;
    }
}

static int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    }
    return sms;
}

// one 1024-thread block per SM at most (short barriers), fewer for small work
static int coop_blocks(int64_t work) {
    const int64_t maxb = sm_count();
    const int64_t want = work / ((int64_t)tune_value(CR_TUNE_UF_ITEMS) * UF_THREADS) + 1;
    const int blocks = (int)(want < maxb ? want : maxb);
    return blocks < 1 ? 1 : blocks;
}

// Union-find for H0 (u0, primal) and the top dimension (u1, dual); either may
// be null.  The stencils and cross-edge kernels run per graph; basins and
// rounds run both graphs in one cooperative launch each.
int run_uf(const float *img, const Seg *segs, const Seg *hsegs, int nseg, int64_t vtot, int64_t ctot,
           int64_t ntiles, int64_t nstiles, UF *u0, UF *u1, const PairBuf &pb, uint32_t flags, uint32_t *extra_mask,
           int *status, cudaStream_t st) {
    if (u0) cudaMemsetAsync(u0->cnt, 0, UF_CNT * sizeof(unsigned long long), st);
    if (u1) cudaMemsetAsync(u1->cnt, 0, UF_CNT * sizeof(unsigned long long), st);
    if (nstiles > 0) {
        prof_begin(st, STAGE_H0_STENCIL);
        CR_NOTE_LAUNCH();
        k_stencil2d_batch<<<(unsigned)nstiles, 256, 0, st>>>(img, segs, nseg, u0 ? u0->lab : nullptr,
                                                             u0 ? u0->dd : nullptr, u1 ? u1->lab : nullptr,
                                                             u1 ? u1->dd : nullptr, status, pb, flags);
        prof_end(st, STAGE_H0_STENCIL, 4.0 * vtot + (u0 ? 5.0 * vtot : 0.0) + (u1 ? 5.0 * ctot : 0.0));
    }
    if (u0 && nstiles == 0) {
        prof_begin(st, STAGE_H0_STENCIL);
        CR_NOTE_LAUNCH();
        CUtensorMap tmap;
        const bool flat = hsegs[0].nz == 1;
        if (nseg == 1 && make_image_map(&tmap, img, hsegs[0], TMA_BX, TMA_BY, flat ? 1 : TMA_BZ)) {
            if (flat)
                k_h0_stencil_tma<true><<<(unsigned)ntiles, dim3(TILE_X, TILE_Y), 0, st>>>(tmap, segs, u0->lab,
                                                                                        u0->dd, status, pb, flags);
            else
                k_h0_stencil_tma<false><<<(unsigned)ntiles, dim3(TILE_X, TILE_Y), 0, st>>>(tmap, segs, u0->lab,
                                                                                         u0->dd, status, pb, flags);
        } else {
            k_h0_stencil_tiled<<<(unsigned)ntiles, dim3(TILE_X, TILE_Y), 0, st>>>(img, segs, nseg, u0->lab, u0->dd,
                                                                                  status, pb, flags);
        }
        prof_end(st, STAGE_H0_STENCIL, 9.0 * vtot);
    }
    bool dual_z_only = false;  // the dual's hooks all run along z (a single volume's stencil)
    if (u1 && nstiles == 0) {
        prof_begin(st, STAGE_DUAL_STENCIL);
        CR_NOTE_LAUNCH();
        CUtensorMap tmap;
        const int edim = hsegs[0].edim;
        if (nseg == 1 && (edim == 2 || edim == 3) &&
            make_image_map(&tmap, img, hsegs[0], DUAL_BX, DUAL_BY, edim == 3 ? DUAL_BZ3 : 1)) {
            if (edim == 3) {
                k_dual_stencil_tma<3><<<(unsigned)ntiles, dim3(TILE_X, TILE_Y), 0, st>>>(tmap, segs, u1->lab,
                                                                                       u1->dd, status, pb, flags);
                dual_z_only = true;
            }
            else
                k_dual_stencil_tma<2><<<(unsigned)ntiles, dim3(TILE_X, TILE_Y), 0, st>>>(tmap, segs, u1->lab,
                                                                                       u1->dd, status, pb, flags);
        } else {
            k_dual_stencil<<<(unsigned)ntiles, TILE_X * TILE_Y, 0, st>>>(img, segs, nseg, u1->lab, u1->dd, pb,
                                                                         flags);
        }
        prof_end(st, STAGE_DUAL_STENCIL, 4.0 * vtot + 5.0 * ctot);
    }
    // basins of both graphs
    {
        BasinArgs A{};
        A.img = img;
        A.segs = segs;
        A.nseg = nseg;
        A.status = status;
        A.polls = debug_limits().barrier_polls;
        A.extra = debug_limits().barrier_extra;
        int64_t work = 0;
        for (UF *u : {u0, u1}) {
            if (!u) continue;
            const int k = A.ngraph++;
            A.u[k] = *u;
            A.mode[k] = u == u0 ? 0 : 1;
            A.n[k] = u == u0 ? vtot : ctot;
            work = A.n[k] > work ? A.n[k] : work;
        }
        void *args[] = {&A};
        prof_begin(st, STAGE_JUMP);
        if (dual_z_only) {
            const Seg &H = hsegs[0];
            const int cx = H.nx - 1, cy = H.ny - 1, cz = H.nz - 1;
            const int64_t cols = (int64_t)cx * cy;
            if (cols > 0 && cz > 0) {
                CR_NOTE_LAUNCH();
                k_dual_zsweep<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(u1->lab, (uint32_t)H.coff, cx, cy, cz);
            }
        }
        CR_NOTE_LAUNCH();
        cudaError_t e = cudaLaunchCooperativeKernel((void *)k_basins, dim3(coop_blocks(work)), dim3(BASIN_THREADS),
                                                    args, 0, st);
        prof_end(st, STAGE_JUMP, 8.0 * (double)((u0 ? vtot : 0) + (u1 ? ctot : 0)));
        if (e != cudaSuccess) return CR_ERR_CUDA;
    }
    if (u0) {
        prof_begin(st, STAGE_H0_CROSS);
        CR_NOTE_LAUNCH();
        k_h0_cross<<<(unsigned)ntiles, TILE_X * TILE_Y, 0, st>>>(img, segs, nseg, u0->lab, u0->dd, u0->ek[0],
                                                                 u0->ea[0], u0->eb[0], &u0->cnt[UFC_E0],
                                                                 u0->max_edges, &u0->cnt[UFC_GROUPS], status);
        prof_end(st, STAGE_H0_CROSS, 9.0 * vtot);
    }
    if (u1) {
        prof_begin(st, STAGE_DUAL_CROSS);
        CR_NOTE_LAUNCH();
        k_dual_cross<<<(unsigned)ntiles, TILE_X * TILE_Y, 0, st>>>(img, segs, nseg, u1->lab, u1->dd, u1->ek[0],
                                                                   u1->ea[0], u1->eb[0], &u1->cnt[UFC_E0],
                                                                   u1->max_edges, &u1->cnt[UFC_GROUPS], status);
        prof_end(st, STAGE_DUAL_CROSS, 4.0 * vtot + 5.0 * ctot);
    }
    // rounds of both graphs
    {
        RoundArgs A{};
        A.status = status;
        A.polls = debug_limits().barrier_polls;
        A.extra = debug_limits().barrier_extra;
        A.compact_mult = tune_value(CR_TUNE_UF_COMPACT);
        for (UF *u : {u0, u1})
            if (u) A.u[A.ngraph++] = *u;
        void *args[] = {&A};
        prof_begin(st, STAGE_UF_ROUND);
        CR_NOTE_LAUNCH();
        cudaError_t e = cudaLaunchCooperativeKernel((void *)k_uf_rounds, dim3(coop_blocks(vtot)), dim3(UF_THREADS),
                                                    args, 0, st);
        prof_end(st, STAGE_UF_ROUND, 0.0);
        if (e != cudaSuccess) return CR_ERR_CUDA;
    }
    if (u0) {
        CR_NOTE_LAUNCH();
        k_uf_emit<<<2 * sm_count(), 256, 0, st>>>(&u0->cnt[UFC_GROUPS], *u0, 0, segs, pb, flags, extra_mask);
    }
    if (u1) {
        CR_NOTE_LAUNCH();
        k_uf_emit<<<2 * sm_count(), 256, 0, st>>>(&u1->cnt[UFC_GROUPS], *u1, 1, segs, pb, flags, nullptr);
    }
    return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

}  // namespace cr

#ifdef CR_UF_TIMING
extern "C" int cr_debug_uf_trace(unsigned long long *out, int cap) {
    int n = 0;
    cudaMemcpyFromSymbol(&n, cr::g_uf_trace_n, sizeof(int));
    if (n > cap) n = cap;
    cudaMemcpyFromSymbol(out, cr::g_uf_trace, n * sizeof(unsigned long long));
    return n;
}
#endif
