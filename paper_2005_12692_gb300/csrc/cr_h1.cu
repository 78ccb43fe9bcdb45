// cr_h1.cu -- the middle dimension of a volume (1-dimensional pairs of a 3D
// image) by reduction of the coboundary matrix (Sec. 2: cohomology, implicit
// coboundary columns generated on the fly, clearing by D^2 = 0).
//
// Columns are the edges that are not killed in dimension 0 (clearing: their
// reduced columns are zero).  Rows are faces; a column's pivot is its
// earliest face in the filtration (the lowest row of the reversed order).
//
// 1. Scan: for every column edge s, t = its earliest cofacet; if s is the
//    latest facet of t, (s, t) is an apparent pair -- a persistence pair
//    that needs no reduction (the pairs Ripser calls apparent, inherited by
//    the paper's adaptation of Ripser, Sec. 1).  The scan writes one code
//    byte per voxel (below); a compaction lists the other columns.
// 2. Reduction of the kept columns in the lock-free form of Morozov and
//    Nigmetov: one warp per column, a pivot table face -> owning column,
//    immutable published column versions in an arena.  When the pivot of
//    column j is owned by an earlier column (later edge in the filtration),
//    j adds that column; when it is owned by a later column, j takes the
//    pivot over and continues with the displaced column.  A pivot owned by an
//    apparent pair is recognised from the image alone and its (at most four
//    entry) column is generated on the fly.  Every sequence of such
//    additions reaches the same pivots, so the pairs equal those of the
//    sequential reduction.
#include "cr_internal.cuh"

namespace cr {

// Code byte of voxel v, for the three edges anchored at v (v to v+x, v+y, v+z):
//   bits 0-2  the x-edge is apparent with the face on its side: 1 +z, 2 -z,
//             3 +y, 4 -y ({x,z} faces have type 1, {x,y} faces type 0);
//   bits 3-4  the y-edge is apparent with its face ({y,z}, type 2): 1 +z, 2 -z;
//   bits 5-7  the x-, y-, z-edge is a residual column (not killed in
//             dimension 0, not apparent).
// z-edges are never apparent, and y-edges only through their {y,z} faces: in
// any other face an edge of equal value and smaller L is the latest facet.
// A face is the pivot of at most one apparent pair, so whether it is one, and
// with which edge, is read from the codes of the two edges that could pair it.
constexpr uint8_t CODE_RX = 1u << 5, CODE_RY = 1u << 6, CODE_RZ = 1u << 7;

struct Img3 {
    const float *img;
    const uint8_t *dd;       // primal stencil hooks
    const uint32_t *extra;   // edges that died in later union-find rounds (L-space bits)
    uint8_t *code;           // one code byte per voxel (above)
};

__device__ __forceinline__ uint32_t vord(const Img3 &I, const Seg &S, const int *c) {
    return ord32(I.img[S.voff + ((int64_t)c[2] * S.ny + c[1]) * S.nx + c[0]]);
}

__device__ __forceinline__ int ext_of(const Seg &S, int a) { return a == 0 ? S.nx : (a == 1 ? S.ny : S.nz); }

__device__ __forceinline__ uint64_t edge_key(const Img3 &I, const Seg &S, int a, const int *c) {
    int d[3] = {c[0], c[1], c[2]};
    d[a] += 1;
    uint32_t u = vord(I, S, c), v = vord(I, S, d);
    return make_key(u > v ? u : v, cube_L(S, a, c[0], c[1], c[2]));
}

// face spanning axes a < b, type a + b - 1
__device__ __forceinline__ uint64_t face_key(const Img3 &I, const Seg &S, int a, int b, const int *c) {
    uint32_t m = 0;
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
            int d[3] = {c[0], c[1], c[2]};
            d[a] += i;
            d[b] += j;
            uint32_t o = vord(I, S, d);
            m = o > m ? o : m;
        }
    return make_key(m, cube_L(S, a + b - 1, c[0], c[1], c[2]));
}

__device__ __forceinline__ bool h0_negative(const Img3 &I, const Seg &S, int a, const int *c) {
    int64_t va = S.voff + ((int64_t)c[2] * S.ny + c[1]) * S.nx + c[0];
    int64_t du = a == 0 ? 1 : (a == 1 ? (int64_t)S.nx : (int64_t)S.nx * S.ny);
    if (I.dd[va] == (uint8_t)(2 * a + 2) || I.dd[va + du] == (uint8_t)(2 * a + 1)) return true;
    int64_t bit = S.loff + cube_L(S, a, c[0], c[1], c[2]);
    return (I.extra[bit >> 5] >> (bit & 31)) & 1u;
}

__device__ __forceinline__ void decode_L(const Seg &S, uint32_t L, int &m, int *c) {
    c[0] = (int)(L % (uint32_t)S.nx);
    uint32_t r = L / (uint32_t)S.nx;
    c[1] = (int)(r % (uint32_t)S.ny);
    r /= (uint32_t)S.ny;
    c[2] = (int)(r % (uint32_t)S.nz);
    m = (int)(r / (uint32_t)S.nz);
}

// cofacets of the edge along axis a at c: keys in out[], returns count (<= 4)
__device__ __forceinline__ int edge_cofacets(const Img3 &I, const Seg &S, int a, const int *c, uint64_t *out) {
    int n = 0;
    for (int b = 0; b < 3; b++) {
        if (b == a) continue;
        int lo = a < b ? a : b, hi = a < b ? b : a;
        if (c[b] + 1 < ext_of(S, b)) out[n++] = face_key(I, S, lo, hi, c);
        if (c[b] >= 1) {
            int d[3] = {c[0], c[1], c[2]};
            d[b] -= 1;
            out[n++] = face_key(I, S, lo, hi, d);
        }
    }
    return n;
}

// The cofacets of the edge along axis a at c in ascending order, in four
// registers (absent ones are ~0 and sort last); returns how many exist.  A
// face's value is the larger of the edge's and its parallel edge's, so the
// ten vertex values are independent loads issued together.
__device__ __forceinline__ void cswap(uint64_t &x, uint64_t &y) {
    const uint64_t lo = x < y ? x : y, hi = x < y ? y : x;
    x = lo;
    y = hi;
}
__device__ __forceinline__ int edge_cofacets_sorted(const Img3 &I, const Seg &S, int a, const int *c, uint64_t &k0,
                                                    uint64_t &k1, uint64_t &k2, uint64_t &k3) {
    // axis quantities by selection (no dynamically indexed local arrays)
    const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;  // the other two axes, b1 < b2
    const int x = c[0], y = c[1], z = c[2];
    const int64_t sxy = (int64_t)S.nx * S.ny;
    const int64_t sa = a == 0 ? 1 : (a == 1 ? (int64_t)S.nx : sxy);
    const int64_t s1 = b1 == 0 ? 1 : (int64_t)S.nx;
    const int64_t s2 = b2 == 1 ? (int64_t)S.nx : sxy;
    const int c1 = b1 == 0 ? x : y, c2 = b2 == 1 ? y : z;
    const int n1 = b1 == 0 ? S.nx : S.ny, n2 = b2 == 1 ? S.ny : S.nz;
    const float *f = I.img + S.voff + ((int64_t)z * S.ny + y) * S.nx + x;
    const bool p1 = c1 + 1 < n1, m1 = c1 >= 1;
    const bool p2 = c2 + 1 < n2, m2 = c2 >= 1;
    const uint32_t e0 = ord32(f[0]), e1 = ord32(f[sa]);
    const uint32_t u0 = p1 ? ord32(f[s1]) : 0u, u1 = p1 ? ord32(f[s1 + sa]) : 0u;
    const uint32_t v0 = m1 ? ord32(f[-s1]) : 0u, v1 = m1 ? ord32(f[sa - s1]) : 0u;
    const uint32_t w0 = p2 ? ord32(f[s2]) : 0u, w1 = p2 ? ord32(f[s2 + sa]) : 0u;
    const uint32_t x0 = m2 ? ord32(f[-s2]) : 0u, x1 = m2 ? ord32(f[sa - s2]) : 0u;
    const uint32_t ve = max(e0, e1);
    const int t1 = min(a, b1) + max(a, b1) - 1, t2 = min(a, b2) + max(a, b2) - 1;  // face types
    // the - faces are anchored one step back along b1 (x or y) or b2 (y or z)
    k0 = p1 ? make_key(max(ve, max(u0, u1)), cube_L(S, t1, x, y, z)) : ~0ull;
    k1 = m1 ? make_key(max(ve, max(v0, v1)), cube_L(S, t1, x - (b1 == 0), y - (b1 == 1), z)) : ~0ull;
    k2 = p2 ? make_key(max(ve, max(w0, w1)), cube_L(S, t2, x, y, z)) : ~0ull;
    k3 = m2 ? make_key(max(ve, max(x0, x1)), cube_L(S, t2, x, y - (b2 == 1), z - (b2 == 2))) : ~0ull;
    cswap(k0, k1);
    cswap(k2, k3);
    cswap(k0, k2);
    cswap(k1, k3);
    cswap(k1, k2);
    return (int)p1 + (int)m1 + (int)p2 + (int)m2;
}

// latest facet (max key) of the face of type fm at c; its axis and anchor returned
__device__ __forceinline__ uint64_t face_max_facet(const Img3 &I, const Seg &S, int fm, const int *c, int &ea,
                                                   int *ec) {
    int a = fm == 2 ? 1 : 0, b = fm == 0 ? 1 : 2;
    uint64_t best = 0;
    for (int k = 0; k < 4; k++) {
        int ax = k < 2 ? a : b, other = k < 2 ? b : a;
        int d[3] = {c[0], c[1], c[2]};
        d[other] += (k & 1);
        uint64_t key = edge_key(I, S, ax, d);
        if (k == 0 || key > best) {
            best = key;
            ea = ax;
            ec[0] = d[0]; ec[1] = d[1]; ec[2] = d[2];
        }
    }
    return best;
}

// ---------------------------------------------------------------------------
// 1. scan
// ---------------------------------------------------------------------------
__device__ __forceinline__ int seg_of_v(const Seg *segs, int n, int64_t gv) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (segs[mid].voff <= gv) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// the side code of the apparent face t of the edge along axis a at c (see Img3)
__device__ __forceinline__ int apparent_side(const Seg &S, int a, const int *c, uint64_t t) {
    int fm, fc[3];
    decode_L(S, key_L(t), fm, fc);
    if (a == 0 && fm == 1) return fc[2] == c[2] ? 1 : 2;  // {x,z}: +z or -z
    if (a == 0 && fm == 0) return fc[1] == c[1] ? 3 : 4;  // {x,y}: +y or -y
    if (a == 1 && fm == 2) return fc[2] == c[2] ? 1 : 2;  // {y,z}: +z or -z
    return 0;
}

__global__ void k_h1_scan(Img3 I, const Seg *__restrict__ segs, int nseg, PairBuf pb, uint32_t flags, int *status) {
    const int si = block_seg(segs, nseg);
    const Seg S = segs[si];
    int tx, ty, z0, z1;
    tile_column(S, tx, ty, z0, z1);
    if (tx >= S.nx || ty >= S.ny) return;
    for (int zz = z0; zz < z1; zz++) {
        int c[3] = {tx, ty, zz};
        uint8_t code = 0;  // images of a batch that are not volumes have no middle dimension: code 0
        for (int a = 0; a < 3 && S.edim == 3; a++) {
            if (c[a] + 1 >= ext_of(S, a) || h0_negative(I, S, a, c)) continue;
            const uint64_t sk = edge_key(I, S, a, c);
            uint64_t cf[4];
            const int n = edge_cofacets(I, S, a, c, cf);
            if (n == 0) {
                set_status(status, CR_ERR_INTERNAL);
                continue;
            }
            uint64_t t = cf[0];
            for (int i = 1; i < n; i++) t = cf[i] < t ? cf[i] : t;
            int fm, fc[3];
            decode_L(S, key_L(t), fm, fc);
            int ea, ec[3];
            const uint64_t top = face_max_facet(I, S, fm, fc, ea, ec);
            if (top == sk) {
                const int side = apparent_side(S, a, c, t);
                if (side == 0 || a == 2) {
                    set_status(status, CR_ERR_INTERNAL);  // excluded by the face order
                    continue;
                }
                code |= (uint8_t)(a == 0 ? side : side << 3);
                if (flags & CR_KEEP_ZERO)
                    emit_pair(pb, (uint32_t)si, 1, key_value(sk), key_value(t), key_L(sk), key_L(t), 0);
            } else {
                code |= (uint8_t)(CODE_RX << a);
            }
        }
        I.code[S.voff + ((int64_t)zz * S.ny + ty) * S.nx + tx] = code;
    }
}

// ---------------------------------------------------------------------------
// The scan fed by TMA (single volumes whose rows are 16-byte multiples).  A
// block owns a 32x8x16 tile.  One mbarrier covers two tensor copies: the
// tile's values with a halo (float box) and, when rows are 16-byte multiples
// of bytes, the tile's stencil hook codes up to one voxel past the tile in +x,
// +y, +z (byte box; otherwise the threads stage them).  Meanwhile the threads
// stage the words of the dimension-0 death mask covering the tile's edges.
// Each thread then walks its column of 16 voxels in z and writes each
// voxel's code byte; a warp writes 32 consecutive bytes.
// ---------------------------------------------------------------------------
constexpr int SC_DX = 48, SC_DY = TILE_Y + 1, SC_DZ = TILE_Z + 1;  // hook-code box (x0..x0+47)
constexpr int SC_DD_BYTES = SC_DX * SC_DY * SC_DZ;
constexpr int SCAN_DYN_SMEM = TMA_BYTES + SC_DD_BYTES + 128;
static_assert(TMA_BYTES % 128 == 0, "hook-code box must start on a 128-byte boundary");

constexpr int SCAN_THREADS = TILE_X * TILE_Y;
__global__ void __launch_bounds__(SCAN_THREADS) k_h1_scan_tma(const __grid_constant__ CUtensorMap tmap,
                                                               const __grid_constant__ CUtensorMap tmap_dd,
                                                               int dd_by_tma, Img3 I, const Seg *__restrict__ segs,
                                                               PairBuf pb, uint32_t flags, int *status) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    unsigned char *dyn = dyn_smem + ((128u - (smem_u32(dyn_smem) & 127u)) & 127u);
    float(*box)[TMA_BY][TMA_BX] = reinterpret_cast<float(*)[TMA_BY][TMA_BX]>(dyn);
    uint8_t(*dds)[SC_DY][SC_DX] = reinterpret_cast<uint8_t(*)[SC_DY][SC_DX]>(dyn + TMA_BYTES);
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t ext[3][TILE_Z][TILE_Y];  // death-mask bits of each edge row, bit tx = x0 + tx
    const Seg S = segs[0];
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    int x0, y0, z0;
    tile_origin(S, blockIdx.x, x0, y0, z0);
    const uint32_t plane = (uint32_t)nx * (uint32_t)ny, P = plane * (uint32_t)nz;
    if (threadIdx.x == 0) {
        const uint32_t b = smem_u32(&bar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const uint32_t bytes = (uint32_t)TMA_BYTES + (dd_by_tma ? (uint32_t)SC_DD_BYTES : 0u);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
            ::"r"(smem_u32(dyn)), "l"(&tmap), "r"(x0 - 4), "r"(y0 - 1), "r"(z0 - 1), "r"(b)
            : "memory");
        if (dd_by_tma)
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                ::"r"(smem_u32(dyn + TMA_BYTES)), "l"(&tmap_dd), "r"(x0), "r"(y0), "r"(z0), "r"(b)
                : "memory");
    }
    if (!dd_by_tma) {
        for (int i = threadIdx.x; i < SC_DZ * SC_DY * (TILE_X + 1); i += TILE_X * TILE_Y) {
            const int dx = i % (TILE_X + 1), r = i / (TILE_X + 1);
            const int dy = r % SC_DY, dz = r / SC_DY;
            const int gx = x0 + dx, gy = y0 + dy, gz = z0 + dz;
            uint8_t c = 0;
            if (gx < nx && gy < ny && gz < nz) c = I.dd[S.voff + (int64_t)gz * plane + (int64_t)gy * nx + gx];
            dds[dz][dy][dx] = c;
        }
    }
    for (int i = threadIdx.x; i < 3 * TILE_Z * TILE_Y; i += TILE_X * TILE_Y) {
        const int dy = i % TILE_Y, r = i / TILE_Y;
        const int dz = r % TILE_Z, ax = r / TILE_Z;
        const int gy = y0 + dy, gz = z0 + dz;
        uint32_t w0 = 0, w1 = 0, sh = 0;
        if (gy < ny && gz < nz) {
            const int64_t bit = S.loff + (int64_t)ax * P + (int64_t)gz * plane + (int64_t)gy * nx + x0;
            const int64_t last = (S.loff + (int64_t)3 * P + 31) >> 5;  // words of the mask
            w0 = __ldg(I.extra + (bit >> 5));
            if ((bit >> 5) + 1 < last) w1 = __ldg(I.extra + (bit >> 5) + 1);
            sh = (uint32_t)(bit & 31);
        }
        ext[ax][dz][dy] = __funnelshift_r(w0, w1, sh);  // 32 bits starting at x0's
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
    const int tx = threadIdx.x & (TILE_X - 1), ty = threadIdx.x / TILE_X;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= nx || y >= ny) return;
    const int bx = tx + 4, by = ty + 1;
    const int zend = min(TILE_Z, nz - z0);
    const bool keep_zero = (flags & CR_KEEP_ZERO) != 0;
    const bool hx = x + 1 < nx, hy = y + 1 < ny;
    uint8_t *code = I.code + S.voff + (uint32_t)y * nx + (uint32_t)x;
    // Values of this thread's column roll through registers: f(x,y,z), f(x+1,y,z),
    // f(x,y+1,z) and the x- and y-edge values of planes z-1, z (and z+1 once read).
    // Out-of-image entries of the box are NaN (the tensor map's fill), and so is
    // the value of an edge outside the image (fmaxf of two NaNs): every
    // comparison with it is false, so a face beyond the image never qualifies
    // and needs no test of its own.  The edge itself is tested (hx, hy, hz):
    // an edge with one vertex outside would take the other vertex's value.
    float fa = box[1][by][bx], fb = box[1][by][bx + 1], fc = box[1][by + 1][bx];
    float exc = fmaxf(fa, fb), eyc = fmaxf(fa, fc);
    float exp_ = fmaxf(box[0][by][bx], box[0][by][bx + 1]), eyp = fmaxf(box[0][by][bx], box[0][by + 1][bx]);
#pragma unroll 4  // a full unroll stalls on instruction fetch
    for (int zz = 0; zz < TILE_Z; zz++) {
        if (zz >= zend) break;
        const int z = z0 + zz, bz = zz + 1;
        const uint32_t rowL = (uint32_t)z * plane + (uint32_t)y * nx + (uint32_t)x0;  // L of (x0, y, z)
        const uint32_t lv = rowL + (uint32_t)tx;
        const bool hz = z + 1 < nz;
        const float fa1 = box[bz + 1][by][bx], fb1 = box[bz + 1][by][bx + 1], fc1 = box[bz + 1][by + 1][bx];
        const float exn = fmaxf(fa1, fb1), eyn = fmaxf(fa1, fc1);
        const uint8_t dv = dds[zz][ty][tx];
        uint32_t cd = 0;
        // an edge killed in dimension 0 (a stencil hook or a later round's
        // death) is not a column (and is never apparent, being paired with a vertex)
#define KILLED(AX, DU)                                                         \
        (dv == (uint8_t)(2 * (AX) + 2) || (DU) == (uint8_t)(2 * (AX) + 1) || \
         ((ext[AX][zz][ty] >> tx) & 1u))
        // Candidates for the earliest cofacet of an edge sigma come in
        // descending face-L order; the first whose parallel edge sigma' has
        // value <= value(sigma) gives a face of value value(sigma), the least
        // possible.  sigma is that face's latest facet unless an edge of the
        // face with equal value has a smaller L: sigma' on the - side with
        // equal value, or one of the two edges along the other axis b when
        // b < a (one of them always has value(sigma)).  With no such
        // candidate the earliest cofacet is larger than sigma and sigma is not
        // its latest facet.  So z-edges (b < a always) are never apparent,
        // y-edges only through their +-z faces, x-edges through any.
        // -- x-edge (v, v+x): faces +z, -z ({x,z}, type 1), +y, -y ({x,y}, type 0)
        if (hx) {
            const float fs = exc;
            const float cpy = fmaxf(fc, box[bz][by + 1][bx + 1]);
            const float cmy = fmaxf(box[bz][by - 1][bx], box[bz][by - 1][bx + 1]);
            uint32_t side = 0;  // 1 +z, 2 -z, 3 +y, 4 -y; the first qualifying wins
            float fp = 0.f;
            if (cmy <= fs) { side = 4; fp = cmy; }
            if (cpy <= fs) { side = 3; fp = cpy; }
            if (exp_ <= fs) { side = 2; fp = exp_; }
            if (exn <= fs) { side = 1; fp = exn; }
            if (side != 0 && ((side & 1) || fp < fs)) {
                cd = side;
                if (keep_zero) {
                    const int m = side <= 2 ? 1 : 0;
                    const int dyf = side == 4 ? -1 : 0, dzf = side == 2 ? -1 : 0;
                    const uint32_t fr = (uint32_t)m * P + rowL + (uint32_t)(dzf * (int)plane + dyf * nx);
                    const float cv = unord32(ord32(fs));
                    emit_pair(pb, 0u, 1, cv, cv, lv, fr + (uint32_t)tx, 0);
                }
            } else if (!KILLED(0, dds[zz][ty][tx + 1])) {
                cd = CODE_RX;
            }
        }
        // -- y-edge (v, v+y): only the {y,z} faces (+z, -z, type 2) can make it apparent
        if (hy) {
            const float fs = eyc;
            const bool pz = eyn <= fs;
            const bool qz = !pz && eyp < fs;
            if (pz || qz) {
                cd |= (pz ? 1u : 2u) << 3;
                if (keep_zero) {
                    const uint32_t fr = 2u * P + rowL - (qz ? plane : 0u);
                    const float cv = unord32(ord32(fs));
                    emit_pair(pb, 0u, 1, cv, cv, lv + P, fr + (uint32_t)tx, 0);
                }
            } else if (!KILLED(1, dds[zz][ty + 1][tx])) {
                cd |= CODE_RY;
            }
        }
        // -- z-edge (v, v+z): a column whenever it survives dimension 0
        if (hz && !KILLED(2, dds[zz + 1][ty][tx])) cd |= CODE_RZ;
#undef KILLED
        code[(size_t)z * plane] = (uint8_t)cd;
        fa = fa1;
        fb = fb1;
        fc = fc1;
        exp_ = exc;
        exc = exn;
        eyp = eyc;
        eyc = eyn;
    }
}

// The residual columns listed from the code bytes: each with its edge's key
// (stored complemented, so that the ascending sort gives cohomology order)
// and its image.  A thread reads 4 code bytes at once (the code array starts
// on a 256-byte boundary); one reservation per warp.
__global__ void k_h1_columns(const float *__restrict__ img, const uint8_t *__restrict__ code,
                             const Seg *__restrict__ segs, int nseg, int64_t vtot, uint64_t *__restrict__ colkey,
                             uint32_t *__restrict__ colseg, unsigned long long *ncol, int64_t max_cols, int *status) {
    const int lane = threadIdx.x & 31;
    const int64_t nchunk = (vtot + 3) / 4;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nchunk; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ch = base + threadIdx.x;
        uint32_t w = 0u;
        if (ch < nchunk) {
            if (ch * 4 + 4 <= vtot) {
                w = __ldg(reinterpret_cast<const uint32_t *>(code) + ch);
            } else {
                for (int64_t v = ch * 4; v < vtot; v++) w |= (uint32_t)code[v] << (8 * (v & 3));
            }
        }
        w &= 0xE0E0E0E0u;  // the residual bits
        const int cnt = __popc(w);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (!total) continue;  // the whole warp has none
        unsigned long long wbase = 0;
        if (lane == 31) wbase = atomicAdd(ncol, (unsigned long long)total);
        wbase = __shfl_sync(0xFFFFFFFFu, wbase, 31);
        if (!cnt) continue;
        int64_t i = (int64_t)wbase + (incl - cnt);
        const int si = seg_of_v(segs, nseg, ch * 4);  // a chunk of four voxels can straddle two images
        // every value the four voxels' columns need is loaded before any is used
        int sj[4];
        float f0[4], fu[4][3];
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const uint32_t cd = (w >> (8 * b)) & 0xE0u;
            const int64_t gv = ch * 4 + b;
            sj[b] = (cd && si + 1 < nseg && gv >= segs[si + 1].voff) ? seg_of_v(segs, nseg, gv) : si;
            const int64_t nx = segs[sj[b]].nx, plane = nx * segs[sj[b]].ny;
            f0[b] = cd ? img[gv] : 0.f;
            fu[b][0] = (cd & CODE_RX) ? img[gv + 1] : 0.f;
            fu[b][1] = (cd & CODE_RY) ? img[gv + nx] : 0.f;
            fu[b][2] = (cd & CODE_RZ) ? img[gv + plane] : 0.f;
        }
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const uint32_t cd = (w >> (8 * b)) & 0xE0u;
            if (!cd) continue;
            const int64_t gv = ch * 4 + b;
            const Seg S = segs[sj[b]];
            const uint32_t lv = (uint32_t)(gv - S.voff);
            const uint32_t P = (uint32_t)S.nx * (uint32_t)S.ny * (uint32_t)S.nz;
            const uint32_t ov = ord32(f0[b]);
#pragma unroll
            for (int a = 0; a < 3; a++) {
                if (!((cd >> (5 + a)) & 1u)) continue;
                const uint32_t ou = ord32(fu[b][a]);
                if (i < max_cols) {
                    colkey[i] = ~make_key(ov > ou ? ov : ou, lv + (uint32_t)a * P);
                    colseg[i] = (uint32_t)sj[b];
                } else {
                    fail_ws(status, SITE_COLUMNS);
                }
                i++;
            }
        }
    }
}

// 2. lock-free reduction
// ---------------------------------------------------------------------------
struct RedParams {
    Img3 I;
    const Seg *segs;
    const uint64_t *colkey;   // edge key of column j, columns in cohomology order
    const uint32_t *colseg;
    int64_t ncols;
    unsigned long long *P;    // face (global L-space index) -> owner << 33 | arena offset of the owner's version
                              // whose head is that face (PIV_FREE: none), see piv_make
    unsigned long long *cur;  // published version of column j: offset << 24 | length (0 = none)
    uint64_t *arena;
    unsigned long long *arena_top;
    int64_t arena_cap;
    uint64_t *scratch;        // 2 * maxlen per warp
    int maxlen;
    uint64_t *pool;           // buffers for columns that outgrow the per-warp scratch
    unsigned long long *pool_top;
    int64_t pool_cap;
    unsigned long long *next; // work counter
    unsigned long long *stats;
    int *status;
    int64_t cap;              // iterations one column may take in one pass before CR_ERR_TIMEOUT
    int64_t budget;           // > 0: iterations after which a column is set aside for the next pass
    int resume;               // take the columns set aside by the previous pass
    unsigned long long *dlist;   // columns set aside: owner << 33 | arena offset of the version
    unsigned long long *dcount;  // entries appended (may exceed dcap: the rest were kept)
    unsigned long long *dnext;   // work counter of the resuming pass
    int64_t dcap;
};

__device__ __forceinline__ uint64_t ld_cg(const uint64_t *p) { return __ldcg((const unsigned long long *)p); }

// A pivot-table entry names the owning column and the arena offset of the
// owner's version that was published with that face as its pivot.  Published
// versions never change, so one load gives an owner together with a column to
// add: no second lookup of the owner's current version.  A version in the
// arena is a header word (its length n) followed by its n entries, the first
// of which is the pivot.
constexpr unsigned long long PIV_FREE = ~0ull;
constexpr int PIV_OFF_BITS = 33;
constexpr unsigned long long PIV_OFF_MASK = (1ull << PIV_OFF_BITS) - 1;
__device__ __forceinline__ unsigned long long piv_make(int64_t owner, unsigned long long off) {
    return ((unsigned long long)owner << PIV_OFF_BITS) | off;
}
__device__ __forceinline__ int piv_owner(unsigned long long e) {
    return e == PIV_FREE ? -1 : (int)(e >> PIV_OFF_BITS);
}
__device__ __forceinline__ unsigned long long piv_off(unsigned long long e) { return e & PIV_OFF_MASK; }
// versions are read speculatively past their end (a header and four entries,
// or a header and 31 entries): the arena keeps this much slack
constexpr int ARENA_SLACK = 32;

// Sizes of a warp's working column and its residency (compile-time; the
// defaults were chosen by measurement, see the design notes).  The reduction
// is compiled twice (cr_h1_reduce.cuh): a wide instance, 16 warps per SM with
// a small inbox, takes every column first and sets aside the few that run
// past an iteration budget; a deep instance, 8 warps per SM with a large
// inbox and merge tiles, then finishes those (the budget is a launch knob,
// CR_TUNE_RED_BUDGET).
#ifndef CR_RED_DMAX
#define CR_RED_DMAX 256
#endif
#ifndef CR_RED_ICAP
#define CR_RED_ICAP 1024
#endif
#ifndef CR_RED_TT
#define CR_RED_TT 256
#endif
#ifndef CR_RED_BLOCKS_PER_SM
#define CR_RED_BLOCKS_PER_SM 2
#endif
#ifndef CR_RED_WIDE_ICAP
#define CR_RED_WIDE_ICAP 256
#endif
#ifndef CR_RED_WIDE_TT
#define CR_RED_WIDE_TT 128
#endif
#ifndef CR_RED_WIDE_BLOCKS_PER_SM
#define CR_RED_WIDE_BLOCKS_PER_SM 4
#endif
constexpr int DMAX = CR_RED_DMAX;  // entries of a published column staged in shared memory
constexpr int FCAP = 256;          // capacity of the front
constexpr int RED_WARPS = 4;
// a long version's entries up to tau (at most a front's worth) are staged in
// the column buffer before they are merged into the front
static_assert(DMAX >= FCAP, "the staged-column buffer must hold a full front");

// Lookahead cache: one entry per lane, filled for the next 32 entries of the
// front in one parallel step, so that a pivot needs no dependent global
// lookup.  kind 0 = neither apparent nor owned at the time of the fill,
// kind 1 = apparent pivot (column tail c1..c3), kind 2 = owned by column
// `own`, `ver` the pivot-table entry read (owner and the arena offset of a
// version with this pivot); when that version has at most four entries,
// k > 0 and c1..c3 hold its tail.
struct Look {
    uint64_t key, c1, c2, c3, ver;
    int kind, k, own;
};

// ---------------------------------------------------------------------------
// Working column of one warp.  An added column shares the pivot and has only
// larger entries, so the pivots of one column's reduction increase and the
// column is kept in four parts whose symmetric difference it is:
//   front   f[fb][fh..fn)  sorted, in shared memory: every entry <= tau;
//   inbox   in[0..ni)      unsorted, in shared memory: entries > tau;
//   middle  mg[mown][mstart..nm)  sorted, global (long columns only);
//   base    g[bown][start..nb)    sorted, global.
// Every entry of inbox, middle and base is larger than tau, so the pivot is
// the front's first entry.  An addition toggles entries up to tau in the
// front (a short merge) and appends the rest to the inbox; entries inserted
// far behind the pivot -- the common case in long reductions -- cost one
// shared-memory store.  When the front runs empty it is refilled with the
// entries of the other three parts up to a new cut.
// ---------------------------------------------------------------------------
#ifndef CR_RED_MIDMAX
#define CR_RED_MIDMAX 8192
#endif
constexpr int MIDMAX = CR_RED_MIDMAX;  // the middle level is merged into the base past this many entries
constexpr int MID_ON = 8192;          // base entries from which a column keeps a middle level
constexpr int MIDCAP = 2 * MIDMAX + DMAX;

struct Work {
    uint64_t *g[2];  // this warp's global buffers (base lives in g[bown])
    int cap;
    int bown;
    int nb, start;
    uint64_t *mg[2]; // middle level buffers (null until first needed)
    int mown, nm, mstart;
    bool mid_on;
    int fb, fh, fn;  // the front
    int ni;          // entries in the inbox
    uint64_t tau;    // ~0: nothing lies beyond the front
};

// diagnostic counters (cnt[8..15]): iterations, apparent additions, column
// additions, merged entries, takeovers, stale or lost races, base rebuilds,
// max iterations spent on one column
constexpr int NT = 10;
struct RedStats {
    unsigned long long it = 0, app = 0, add = 0, merged = 0, take = 0, retry = 0, flush = 0, maxit = 0;
    // cycles per phase (diagnostic builds): refill, lookup, apparent, cached, staged, inbox
    // flushes, misses, long iterations, whole iterations, pivot-table reads
    unsigned long long t[NT] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool lng = false;
};
#ifdef CR_H1_TIMING
// only iterations of long column runs (beyond 16384) are timed: the critical path
__device__ bool g_long_iter_dummy;
#define TMARK(v) long long v = clock64()
#define TADD(st, i, v) ((st).lng ? (void)((st).t[i] += (unsigned long long)(clock64() - (v))) : (void)0)
// cycles of a whole iteration of a long column, on every way out of it
struct IterTimer {
    RedStats &s;
    long long t0;
    __device__ explicit IterTimer(RedStats &st) : s(st), t0(0) {
#ifdef __CUDA_ARCH__
        t0 = clock64();
#endif
    }
    __device__ ~IterTimer() {
#ifdef __CUDA_ARCH__
        if (s.lng) s.t[8] += (unsigned long long)(clock64() - t0);
#endif
    }
};
#define TITER(st) IterTimer iter_timer_(st)
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// timestamps (ns): warps' start, start and end of columns longer than 16384
// iterations, last column end; minima are kept as maxima of complements
#define TSTAMP_KERNEL(R) \
    if ((threadIdx.x & 31) == 0) atomicMax(&(R).stats[18], ~gtimer())
#define TSTAMP_COLSTART(v) const unsigned long long v = gtimer()
#define TSTAMP_COLEND(R, it, v)                                 \
    if ((threadIdx.x & 31) == 0) {                              \
        const unsigned long long e_ = gtimer();                 \
        atomicMax(&(R).stats[21], e_);                          \
        if ((it) > 16384) {                                     \
            atomicMax(&(R).stats[19], ~(v));                    \
            atomicMax(&(R).stats[20], e_);                      \
            atomicAdd(&(R).stats[22], 1ull);                    \
        }                                                       \
    }
#else
#define TMARK(v)
#define TADD(st, i, v)
#define TITER(st)
#define TSTAMP_KERNEL(R)
#define TSTAMP_COLSTART(v)
#define TSTAMP_COLEND(R, it, v)
#endif
__device__ void flush_stats(const RedParams &R, const RedStats &s) {
    if ((threadIdx.x & 31) != 0) return;
    unsigned long long *c = R.stats;
    atomicAdd(&c[0], s.it);
    atomicAdd(&c[1], s.app);
    atomicAdd(&c[2], s.add);
    atomicAdd(&c[3], s.merged);
    atomicAdd(&c[4], s.take);
    atomicAdd(&c[5], s.retry);
    atomicAdd(&c[6], s.flush);
    atomicMax(&c[7], s.maxit);
    for (int i = 0; i < NT; i++) atomicAdd(&c[8 + i], s.t[i]);
}

// new buffer pair of at least `need` entries from the shared pool (the old
// buffers stay readable); false when the pool is exhausted
__device__ bool grow_to(const RedParams &R, Work &W, int64_t need) {
    const int lane = threadIdx.x & 31;
    int64_t nc = W.cap;
    while (nc < need) nc *= 2;
    if (nc > (1 << 28)) return false;
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(R.pool_top, (unsigned long long)(2 * nc));
    off = __shfl_sync(0xFFFFFFFFu, off, 0);
    if ((int64_t)(off + 2 * nc) > R.pool_cap) return false;
    W.g[0] = R.pool + off;
    W.g[1] = R.pool + off + nc;
    W.cap = (int)nc;
    W.bown = 1;  // the next write goes to g[0]; the old base is in the old buffers
    return true;
}


// The two instances of the reduction (see the sizes above)
namespace deep {
constexpr int ICAP = CR_RED_ICAP;  // capacity of the inbox
constexpr int TT = CR_RED_TT;      // merged positions per tile of a merge of sorted runs
constexpr int RED_BLOCKS = CR_RED_BLOCKS_PER_SM;
#include "cr_h1_reduce.cuh"
}  // namespace deep
namespace wide {
constexpr int ICAP = CR_RED_WIDE_ICAP;
constexpr int TT = CR_RED_WIDE_TT;
constexpr int RED_BLOCKS = CR_RED_WIDE_BLOCKS_PER_SM;
#include "cr_h1_reduce.cuh"
}  // namespace wide

__global__ void k_h1_emit(const uint64_t *__restrict__ colkey, const uint32_t *__restrict__ colseg, int64_t ncols,
                          const Seg *__restrict__ segs, const unsigned long long *__restrict__ P,
                          const unsigned long long *__restrict__ cur, const uint64_t *__restrict__ arena, PairBuf pb,
                          uint32_t flags, int *status) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncols) return;
    unsigned long long v = cur[j];
    int len = (int)(v & 0xFFFFFFull);
    if (len == 0) { set_status(status, CR_ERR_INTERNAL); return; }
    uint64_t p = arena[(v >> 24) + 1];  // the entry after the version's header
    const Seg S = segs[colseg[j]];
    const unsigned long long e = P[S.loff + key_L(p)];
    if (e == PIV_FREE || (int64_t)(e >> PIV_OFF_BITS) != j) { set_status(status, CR_ERR_INTERNAL); return; }
    uint64_t sk = colkey[j];
    float b = key_value(sk), d = key_value(p);
    if ((flags & CR_KEEP_ZERO) || b != d) emit_pair(pb, colseg[j], 1, b, d, key_L(sk), key_L(p), 0);
}

__global__ void k_not_keys(uint64_t *k, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) k[i] = ~k[i];
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------

static inline unsigned nb1(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

static unsigned long long g_h1_stats[24];
static int64_t g_h1_stats_cols = 0;
int h1_stats(int64_t *out, int n) {
    out[0] = g_h1_stats_cols;
    for (int i = 0; i < 24 && i + 1 < n; i++) out[i + 1] = (int64_t)g_h1_stats[i];
    return CR_OK;
}

int run_h1(const float *img, const uint8_t *dd, const uint32_t *extra, const Seg *segs, const Seg *hseg, int nseg,
           int64_t vtot, int64_t ntiles, H1Bufs &B, const PairBuf &pb, uint32_t flags, int *status,
           int64_t *ncols_out, cudaStream_t st) {
    Img3 I{img, dd, extra, B.code};
    cudaMemsetAsync(B.cnt, 0, 32 * sizeof(unsigned long long), st);  // counters and statistics (CNT_H1 .. CNT_H1 + 32)
    prof_begin(st, STAGE_H1_SCAN);
    CR_NOTE_LAUNCH();
    CUtensorMap tmap, tmap_dd;
    if (nseg == 1 && hseg && hseg->edim == 3 && make_image_map(&tmap, img, *hseg, TMA_BX, TMA_BY, TMA_BZ, true)) {
        static int attr_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (attr_dev != dev) {
            cudaFuncSetAttribute(k_h1_scan_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, SCAN_DYN_SMEM);
            attr_dev = dev;
        }
        const int dd_tma = make_u8_map(&tmap_dd, dd, *hseg, SC_DX, SC_DY, SC_DZ) ? 1 : 0;
        if (!dd_tma) memset(&tmap_dd, 0, sizeof(tmap_dd));
        k_h1_scan_tma<<<(unsigned)ntiles, SCAN_THREADS, SCAN_DYN_SMEM, st>>>(tmap, tmap_dd, dd_tma, I, segs,
                                                                               pb, flags, status);
    } else {
        k_h1_scan<<<(unsigned)ntiles, TILE_X * TILE_Y, 0, st>>>(I, segs, nseg, pb, flags, status);
    }
    // algorithmic bytes: value and hook code read (5 B), death-mask bits read
    // (3/8 B) and the code byte written (1 B) per voxel
    prof_end(st, STAGE_H1_SCAN, 6.375 * vtot);
    // the residual columns from the codes (1 B read per voxel; 12 B written per
    // column and its two values read, added below once the count is known)
    prof_begin(st, STAGE_H1_COLUMNS);
    CR_NOTE_LAUNCH();
    {
        int sms = 0, dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
        const int64_t want = ((vtot + 3) / 4 + 255) / 256, cap = (int64_t)sms * 64;
        k_h1_columns<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(img, B.code, segs, nseg, vtot, B.colkey,
                                                                           B.colseg, &B.cnt[0], B.max_cols, status);
    }
    prof_end(st, STAGE_H1_COLUMNS, 1.0 * vtot);
    unsigned long long hc = 0;
    int hstatus = 0;
    cudaMemcpyAsync(&hc, &B.cnt[0], sizeof(hc), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return CR_ERR_CUDA;
    // an earlier stage failed (its status is returned by the caller): no reduction on its output
    if (hstatus) return CR_OK;
    int64_t ncols = (int64_t)hc;
    prof_add_bytes(STAGE_H1_COLUMNS, 20.0 * (double)(ncols < B.max_cols ? ncols : B.max_cols));
    *ncols_out = ncols;
    if (ncols > B.max_cols) { set_host_detail(SITE_COLUMNS); return CR_ERR_WORKSPACE; }
    if (ncols == 0) return CR_OK;
    if (ncols >= ((int64_t)1 << 31) - 1) return CR_ERR_TOO_LARGE;  // owner field of a pivot-table entry
    // cohomology order: decreasing edge key (keys were stored complemented)
    prof_begin(st, STAGE_H1_SORT);
    if (radix_sort_u64(B.colkey, B.colseg, B.colkey_tmp, B.colseg_tmp, ncols, 0, 64, B.sort_temp, B.sort_temp_bytes,
                       st) != cudaSuccess)
        return CR_ERR_CUDA;
    prof_end(st, STAGE_H1_SORT, 8.0 * 24.0 * ncols);
    CR_NOTE_LAUNCH();
    k_not_keys<<<nb1(ncols), 256, 0, st>>>(B.colkey, ncols);
    cudaMemsetAsync(B.P, 0xFF, (size_t)B.P_len * sizeof(unsigned long long), st);
    cudaMemsetAsync(B.cur, 0, (size_t)ncols * sizeof(unsigned long long), st);
    RedParams R;
    R.I = I;
    R.segs = segs;
    R.colkey = B.colkey;
    R.colseg = B.colseg;
    R.ncols = ncols;
    R.P = B.P;
    R.cur = B.cur;
    R.arena = B.arena;
    R.arena_top = &B.cnt[1];
    // ARENA_SLACK words of slack: a version is read speculatively past its end
    R.arena_cap = B.arena_cap - ARENA_SLACK;
    if (R.arena_cap > (int64_t)PIV_OFF_MASK) R.arena_cap = (int64_t)PIV_OFF_MASK;
    R.scratch = B.scratch;
    R.maxlen = B.maxlen;
    R.pool = B.pool;
    R.pool_top = &B.cnt[3];
    R.pool_cap = B.pool_cap;
    R.next = &B.cnt[2];
    R.stats = &B.cnt[8];
    R.status = status;
    R.cap = debug_limits().reduce_iters;
    // columns set aside by the wide pass: the sort's spare key buffer, free once the columns are sorted
    R.dlist = reinterpret_cast<unsigned long long *>(B.colkey_tmp);
    R.dcap = B.max_cols;
    R.dcount = &B.cnt[4];
    R.dnext = &B.cnt[5];
    int sms = 0;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
        static int red_attr_dev = -1;
        if (red_attr_dev != dev) {
            cudaFuncSetAttribute(deep::k_h1_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)deep::RED_SMEM);
            cudaFuncSetAttribute(wide::k_h1_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wide::RED_SMEM);
            red_attr_dev = dev;
        }
    }
    prof_begin(st, STAGE_H1_REDUCE);
    const int budget = tune_value(CR_TUNE_RED_BUDGET);  // steps a column may take in the wide pass
    if (budget > 0) {
        // the wide pass: every column, those past the budget set aside
        int64_t w = (int64_t)sms * RED_WARPS * wide::RED_BLOCKS;
        if (w > B.nwarps) w = B.nwarps;  // the scratch holds B.nwarps warps
        if (w > ncols) w = ncols;
        R.budget = budget;
        R.resume = 0;
        CR_NOTE_LAUNCH();
        wide::k_h1_reduce<<<(unsigned)((w + RED_WARPS - 1) / RED_WARPS), RED_WARPS * 32, wide::RED_SMEM, st>>>(R);
        R.resume = 1;
    } else {
        R.resume = 0;
    }
    // the deep pass: the columns set aside (or, without a budget, every column).
    // B.nwarps = 16 warps per SM (the scratch is sized for them); the knob may launch fewer
    R.budget = 0;
    int64_t warps = B.nwarps / 16 * tune_value(CR_TUNE_RED_WARPS);
    if (warps > B.nwarps) warps = B.nwarps;
    if (warps > ncols) warps = ncols;
    if (warps < 1) warps = 1;
    unsigned blocks = (unsigned)((warps + RED_WARPS - 1) / RED_WARPS);
    CR_NOTE_LAUNCH();
    deep::k_h1_reduce<<<blocks, RED_WARPS * 32, deep::RED_SMEM, st>>>(R);
    prof_end(st, STAGE_H1_REDUCE, 12.0 * ncols);
    CR_NOTE_LAUNCH();
    k_h1_emit<<<nb1(ncols), 256, 0, st>>>(B.colkey, B.colseg, ncols, segs, B.P, B.cur, B.arena, pb, flags, status);
    cudaMemcpyAsync(g_h1_stats, &B.cnt[8], 24 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    g_h1_stats_cols = ncols;
    return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

}  // namespace cr
