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
//    the paper's adaptation of Ripser, Sec. 1).  Other columns are kept.
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

struct Img3 {
    const float *img;
    const uint8_t *dd;       // primal stencil hooks
    const uint32_t *extra;   // edges that died in later union-find rounds (L-space bits)
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

__device__ __forceinline__ void sort4(uint64_t *v, int n) {
    for (int i = 1; i < n; i++) {
        uint64_t x = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; j--; }
        v[j + 1] = x;
    }
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

// If the face with key fk is the pivot of an apparent pair, the key of its
// edge; 0 otherwise.
__device__ uint64_t apparent_edge(const Img3 &I, const Seg &S, uint64_t fk) {
    int fm, c[3];
    decode_L(S, key_L(fk), fm, c);
    int ea, ec[3];
    uint64_t sk = face_max_facet(I, S, fm, c, ea, ec);
    if (h0_negative(I, S, ea, ec)) return 0;
    uint64_t cf[4];
    int n = edge_cofacets(I, S, ea, ec, cf);
    uint64_t mn = ~0ull;
    for (int i = 0; i < n; i++) mn = cf[i] < mn ? cf[i] : mn;
    return mn == fk ? sk : 0;
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

__global__ void k_h1_scan(Img3 I, const Seg *__restrict__ segs, int nseg, int64_t vtot, uint64_t *__restrict__ colkey,
                          uint32_t *__restrict__ colseg, unsigned long long *ncol, int64_t max_cols, PairBuf pb,
                          uint32_t flags, int *status) {
    int64_t gv = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool in = gv < vtot;
    Seg S;
    int si = 0;
    int c[3] = {0, 0, 0};
    if (in) {
        si = seg_of_v(segs, nseg, gv);
        S = segs[si];
        if (S.edim != 3) in = false;
        int64_t lv = gv - S.voff;
        c[0] = (int)(lv % S.nx);
        c[1] = (int)((lv / S.nx) % S.ny);
        c[2] = (int)(lv / ((int64_t)S.nx * S.ny));
    }
    for (int a = 0; a < 3; a++) {
        bool keep = false;
        uint64_t sk = 0;
        if (in && c[a] + 1 < ext_of(S, a) && !h0_negative(I, S, a, c)) {
            sk = edge_key(I, S, a, c);
            uint64_t cf[4];
            int n = edge_cofacets(I, S, a, c, cf);
            if (n == 0) {
                set_status(status, CR_ERR_INTERNAL);
            } else {
                uint64_t t = cf[0];
                for (int i = 1; i < n; i++) t = cf[i] < t ? cf[i] : t;
                int fm, fc[3];
                decode_L(S, key_L(t), fm, fc);
                int ea, ec[3];
                uint64_t top = face_max_facet(I, S, fm, fc, ea, ec);
                if (top == sk) {
                    if (flags & CR_KEEP_ZERO)
                        emit_pair(pb, (uint32_t)si, 1, key_value(sk), key_value(t), key_L(sk), key_L(t), 0);
                } else {
                    keep = true;
                }
            }
        }
        unsigned mask = __ballot_sync(0xFFFFFFFFu, keep);
        if (mask) {
            int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(ncol, (unsigned long long)__popc(mask));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (keep) {
                int64_t i = (int64_t)base + __popc(mask & ((1u << lane) - 1u));
                if (i < max_cols) {
                    colkey[i] = ~sk;  // sorted ascending below = cohomology order
                    colseg[i] = (uint32_t)si;
                } else {
                    set_status(status, CR_ERR_WORKSPACE);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 2. lock-free reduction
// ---------------------------------------------------------------------------
struct RedParams {
    Img3 I;
    const Seg *segs;
    const uint64_t *colkey;   // edge key of column j, columns in cohomology order
    const uint32_t *colseg;
    int64_t ncols;
    int *P;                   // face (global L-space index) -> owning column, -1 none
    unsigned long long *cur;  // published version of column j: offset << 24 | length (0 = none)
    uint64_t *arena;
    unsigned long long *arena_top;
    int64_t arena_cap;
    uint64_t *scratch;        // 2 * maxlen per warp
    int maxlen;
    unsigned long long *next; // work counter
    int *status;
};

__device__ __forceinline__ uint64_t ld_cg(const uint64_t *p) { return __ldcg((const unsigned long long *)p); }

// out = A xor B (sorted, distinct), warp-cooperative; returns length or -1 if it exceeds cap
__device__ int warp_xor(const uint64_t *A, int na, const uint64_t *B, int nb, uint64_t *out, int cap, bool bcg) {
    const int lane = threadIdx.x & 31;
    const int T = na + nb;
    if (T <= 32) {
        uint64_t v = ~0ull;
        bool valid = lane < T;
        if (lane < na) v = A[lane];
        else if (valid) v = bcg ? ld_cg(B + lane - na) : B[lane - na];
        unsigned same = __match_any_sync(0xFFFFFFFFu, v);
        bool keep = valid && __popc(same) == 1;
        int rank = 0;
        for (int k = 0; k < 32; k++) {
            uint64_t w = __shfl_sync(0xFFFFFFFFu, v, k);
            int kk = __shfl_sync(0xFFFFFFFFu, (int)keep, k);
            rank += (kk && w < v) ? 1 : 0;
        }
        unsigned km = __ballot_sync(0xFFFFFFFFu, keep);
        int n = __popc(km);
        if (n > cap) return -1;
        if (keep) out[rank] = v;
        __syncwarp();
        return n;
    }
    // merge path: lane takes merged positions [s, e)
    const int per = (T + 31) / 32;
    const int s = min(lane * per, T), e = min(s + per, T);
    int lo = max(0, s - nb), hi = min(s, na);
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        uint64_t am = A[mid], bm = bcg ? ld_cg(B + s - 1 - mid) : B[s - 1 - mid];
        if (am <= bm) lo = mid + 1; else hi = mid;
    }
    const int i0 = lo, j0 = s - lo;
    // predecessor of position s in the merged order
    uint64_t prev = 0;
    bool hasprev = false;
    if (s > 0) {
        uint64_t pa = i0 > 0 ? A[i0 - 1] : 0, pb = j0 > 0 ? (bcg ? ld_cg(B + j0 - 1) : B[j0 - 1]) : 0;
        prev = pa > pb ? pa : pb;
        hasprev = true;
    }
    int kept = 0;
    for (int pass = 0; pass < 2; pass++) {
        int i = i0, j = j0;
        uint64_t pv = prev;
        bool hp = hasprev;
        int wpos = 0;
        if (pass == 1) {
            int incl = kept;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            wpos = incl - kept;
            int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            if (total > cap) return -1;
        }
        // current element
        uint64_t curv = 0;
        bool have = false;
        auto take = [&](uint64_t &x) -> bool {
            if (i + j >= T) return false;
            uint64_t av = i < na ? A[i] : ~0ull;
            uint64_t bv = j < nb ? (bcg ? ld_cg(B + j) : B[j]) : ~0ull;
            if (j >= nb || (i < na && av <= bv)) { x = av; i++; }
            else { x = bv; j++; }
            return true;
        };
        int q = s;
        if (q < e) have = take(curv);
        while (q < e && have) {
            uint64_t nxt = 0;
            bool hn = take(nxt);  // may read one element past e: that is the successor
            bool dup = (hp && pv == curv) || (hn && nxt == curv);
            if (!dup) {
                if (pass == 0) kept++;
                else out[wpos++] = curv;
            }
            pv = curv;
            hp = true;
            curv = nxt;
            have = hn;
            q++;
        }
        if (pass == 1) {
            int incl = kept;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            __syncwarp();
            return __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
    }
    return -1;  // unreachable
}

// publish column j's current state; returns false on arena overflow
__device__ bool publish(const RedParams &R, int64_t j, const uint64_t *buf, int n) {
    const int lane = threadIdx.x & 31;
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(R.arena_top, (unsigned long long)n);
    off = __shfl_sync(0xFFFFFFFFu, off, 0);
    if ((int64_t)(off + n) > R.arena_cap) return false;
    for (int k = lane; k < n; k += 32) __stcg((unsigned long long *)&R.arena[off + k], buf[k]);
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicExch(&R.cur[j], (off << 24) | (unsigned long long)n);
    __threadfence();
    __syncwarp();
    return true;
}

__device__ __forceinline__ void load_version(const RedParams &R, int64_t o, unsigned long long &off, int &len) {
    unsigned long long v = 0;
    if ((threadIdx.x & 31) == 0) v = atomicAdd(&R.cur[o], 0ull);
    v = __shfl_sync(0xFFFFFFFFu, v, 0);
    __threadfence();
    off = v >> 24;
    len = (int)(v & 0xFFFFFFull);
}

__global__ void __launch_bounds__(256) k_h1_reduce(RedParams R) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t *bufA = R.scratch + wid * 2 * (int64_t)R.maxlen;
    uint64_t *bufB = bufA + R.maxlen;
    const int64_t CAP = (int64_t)1 << 24;
    for (;;) {
        unsigned long long jj = 0;
        if (lane == 0) jj = atomicAdd(R.next, 1ull);
        jj = __shfl_sync(0xFFFFFFFFu, jj, 0);
        if ((int64_t)jj >= R.ncols) return;
        int64_t j = (int64_t)jj;
        uint64_t jkey = R.colkey[j];
        const Seg S = R.segs[R.colseg[j]];
        // the coboundary of edge j
        int n;
        {
            int a, c[3];
            decode_L(S, key_L(jkey), a, c);
            uint64_t cf[4];
            int k = edge_cofacets(R.I, S, a, c, cf);
            sort4(cf, k);
            if (lane < k) bufA[lane] = cf[lane];
            n = k;
            __syncwarp();
        }
        int64_t it = 0;
        for (;;) {
            if (++it > CAP) { if (lane == 0) set_status(R.status, CR_ERR_TIMEOUT); return; }
            if (n <= 0) { if (lane == 0) set_status(R.status, CR_ERR_INTERNAL); break; }
            uint64_t p = bufA[0];
            int64_t gidx = S.loff + key_L(p);
            uint64_t ak = 0;
            if (lane == 0) ak = apparent_edge(R.I, S, p);
            ak = __shfl_sync(0xFFFFFFFFu, ak, 0);
            if (ak) {
                int a, c[3];
                decode_L(S, key_L(ak), a, c);
                uint64_t cf[4];
                int k = edge_cofacets(R.I, S, a, c, cf);
                sort4(cf, k);
                int m = warp_xor(bufA, n, cf, k, bufB, R.maxlen, false);
                if (m < 0) { if (lane == 0) set_status(R.status, CR_ERR_WORKSPACE); return; }
                uint64_t *t = bufA; bufA = bufB; bufB = t;
                n = m;
                continue;
            }
            int o = 0;
            if (lane == 0) o = atomicAdd(&R.P[gidx], 0);
            o = __shfl_sync(0xFFFFFFFFu, o, 0);
            __threadfence();
            if (o < 0) {
                if (!publish(R, j, bufA, n)) { if (lane == 0) set_status(R.status, CR_ERR_WORKSPACE); return; }
                int prev = 0;
                if (lane == 0) prev = atomicCAS(&R.P[gidx], -1, (int)j);
                prev = __shfl_sync(0xFFFFFFFFu, prev, 0);
                if (prev == -1) break;  // j settled
                continue;
            }
            if ((int64_t)o == j) break;
            uint64_t okey = R.colkey[o];
            if (okey > jkey) {
                // o is an earlier column (a later edge): add it
                unsigned long long off;
                int len;
                load_version(R, o, off, len);
                if (len == 0) continue;
                if (ld_cg(&R.arena[off]) != p) continue;  // stale snapshot: re-read the table
                int m = warp_xor(bufA, n, R.arena + off, len, bufB, R.maxlen, true);
                if (m < 0) { if (lane == 0) set_status(R.status, CR_ERR_WORKSPACE); return; }
                uint64_t *t = bufA; bufA = bufB; bufB = t;
                n = m;
                continue;
            }
            // o is a later column: take its pivot, then continue with o
            if (!publish(R, j, bufA, n)) { if (lane == 0) set_status(R.status, CR_ERR_WORKSPACE); return; }
            int prev = 0;
            if (lane == 0) prev = atomicCAS(&R.P[gidx], o, (int)j);
            prev = __shfl_sync(0xFFFFFFFFu, prev, 0);
            if (prev != o) continue;
            unsigned long long off;
            int len;
            load_version(R, o, off, len);
            int m = warp_xor(bufA, n, R.arena + off, len, bufB, R.maxlen, true);
            if (m < 0) { if (lane == 0) set_status(R.status, CR_ERR_WORKSPACE); return; }
            uint64_t *t = bufA; bufA = bufB; bufB = t;
            n = m;
            j = o;
            jkey = okey;
        }
    }
}

__global__ void k_h1_emit(const uint64_t *__restrict__ colkey, const uint32_t *__restrict__ colseg, int64_t ncols,
                          const Seg *__restrict__ segs, const int *__restrict__ P,
                          const unsigned long long *__restrict__ cur, const uint64_t *__restrict__ arena, PairBuf pb,
                          uint32_t flags, int *status) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncols) return;
    unsigned long long v = cur[j];
    int len = (int)(v & 0xFFFFFFull);
    if (len == 0) { set_status(status, CR_ERR_INTERNAL); return; }
    uint64_t p = arena[v >> 24];
    const Seg S = segs[colseg[j]];
    if (P[S.loff + key_L(p)] != (int)j) { set_status(status, CR_ERR_INTERNAL); return; }
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

int run_h1(const float *img, const uint8_t *dd, const uint32_t *extra, const Seg *segs, int nseg, int64_t vtot,
           H1Bufs &B, const PairBuf &pb, uint32_t flags, int *status, int64_t *ncols_out, cudaStream_t st) {
    Img3 I{img, dd, extra};
    cudaMemsetAsync(B.cnt, 0, 3 * sizeof(unsigned long long), st);
    prof_begin(st, STAGE_H1_SCAN);
    CR_NOTE_LAUNCH();
    k_h1_scan<<<nb1(vtot), 256, 0, st>>>(I, segs, nseg, vtot, B.colkey, B.colseg, &B.cnt[0], B.max_cols, pb, flags,
                                         status);
    prof_end(st, STAGE_H1_SCAN, 5.0 * vtot);
    unsigned long long hc = 0;
    cudaMemcpyAsync(&hc, &B.cnt[0], sizeof(hc), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return CR_ERR_CUDA;
    int64_t ncols = (int64_t)hc;
    *ncols_out = ncols;
    if (ncols > B.max_cols) return CR_ERR_WORKSPACE;
    if (ncols == 0) return CR_OK;
    if (ncols >= ((int64_t)1 << 31)) return CR_ERR_TOO_LARGE;
    // cohomology order: decreasing edge key (keys were stored complemented)
    prof_begin(st, STAGE_H1_SORT);
    if (radix_sort_u64(B.colkey, B.colseg, B.colkey_tmp, B.colseg_tmp, ncols, 0, 64, B.sort_temp, B.sort_temp_bytes,
                       st) != cudaSuccess)
        return CR_ERR_CUDA;
    prof_end(st, STAGE_H1_SORT, 8.0 * 24.0 * ncols);
    CR_NOTE_LAUNCH();
    k_not_keys<<<nb1(ncols), 256, 0, st>>>(B.colkey, ncols);
    cudaMemsetAsync(B.P, 0xFF, (size_t)B.P_len * sizeof(int), st);
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
    R.arena_cap = B.arena_cap;
    R.scratch = B.scratch;
    R.maxlen = B.maxlen;
    R.next = &B.cnt[2];
    R.status = status;
    int64_t warps = B.nwarps < ncols ? B.nwarps : ncols;
    unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    prof_begin(st, STAGE_H1_REDUCE);
    CR_NOTE_LAUNCH();
    k_h1_reduce<<<blocks, 256, 0, st>>>(R);
    prof_end(st, STAGE_H1_REDUCE, 12.0 * ncols);
    CR_NOTE_LAUNCH();
    k_h1_emit<<<nb1(ncols), 256, 0, st>>>(B.colkey, B.colseg, ncols, segs, B.P, B.cur, B.arena, pb, flags, status);
    return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

}  // namespace cr
