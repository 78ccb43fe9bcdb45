// cr_batch2d.cu -- batches of 2D images in one persistent launch.
//
// The union-finds of a batch of 2D images (H0 on the pixel graph, the top
// dimension on the dual graph of squares plus an outer node, Sec. 2 and
// Rem. 2.1) are independent per image.  Here every block pulls images from a
// work queue ordered by size, largest first, and computes both union-finds of
// an image on its own, with block barriers only:
//   stencil (each node's first hook, as in the tile kernels), pointer jumping
//   to the roots, group numbering, the edges between groups, Borůvka rounds
//   under the elder rule, and the pairs of the dead groups.
// The rules are those of the grid-wide kernels in cr_uf.cu, applied to one
// image: a node hooks along its minimum edge when the other end is older; a
// group's minimum outgoing edge kills it when the other end is older; the
// younger end of a mutual pair hooks.  Group numbering and the order in which
// pairs are written do not matter: the output is sorted afterwards.
#include "cr_internal.cuh"
#include <vector>

namespace cr {

namespace {

constexpr uint32_t MARK = 0x80000000u;

// per-block scratch in global memory, sized for the largest image of the batch
struct B2Work {
    uint32_t *par;   // node -> parent, then node -> group
    uint8_t *dd;     // node -> hook code (0 = root)
    uint64_t *gkey;  // group -> age key of its root (smaller = older)
    uint64_t *mA, *mB, *dkey;
    uint32_t *hook;
    uint8_t *dead;
    uint64_t *ek[2];
    uint32_t *ea[2], *eb[2];  // two edge buffers: the rounds compact the live edges into the other
};

__host__ __device__ __forceinline__ size_t b2_al(size_t x) { return (x + 255) & ~(size_t)255; }

__host__ __device__ __forceinline__ size_t b2_stride(int64_t nmax, int64_t emax) {
    return b2_al(nmax * 4) + b2_al(nmax) + 4 * b2_al(nmax * 8) + b2_al(nmax * 4) + b2_al(nmax) +
           2 * (b2_al(emax * 8) + 2 * b2_al(emax * 4));
}

struct B2Args {
    const float *img;
    const Seg *segs;
    const uint32_t *order;  // images by size, largest first
    int nimg;
    unsigned long long *queue;
    char *scratch;
    size_t stride;
    int64_t nmax, emax;
    PairBuf pb;
    uint32_t flags;
    int *status;
    long long round_cap;
    bool primal, dual;  // which union-finds the call wants
};

__device__ __forceinline__ B2Work b2_work(const B2Args &A) {
    char *b = A.scratch + (size_t)blockIdx.x * A.stride;
    B2Work W;
    size_t o = 0;
    W.par = (uint32_t *)(b + o); o += b2_al(A.nmax * 4);
    W.dd = (uint8_t *)(b + o); o += b2_al(A.nmax);
    W.gkey = (uint64_t *)(b + o); o += b2_al(A.nmax * 8);
    W.mA = (uint64_t *)(b + o); o += b2_al(A.nmax * 8);
    W.mB = (uint64_t *)(b + o); o += b2_al(A.nmax * 8);
    W.dkey = (uint64_t *)(b + o); o += b2_al(A.nmax * 8);
    W.hook = (uint32_t *)(b + o); o += b2_al(A.nmax * 4);
    W.dead = (uint8_t *)(b + o); o += b2_al(A.nmax);
    for (int k = 0; k < 2; k++) {
        W.ek[k] = (uint64_t *)(b + o); o += b2_al(A.emax * 8);
        W.ea[k] = (uint32_t *)(b + o); o += b2_al(A.emax * 4);
        W.eb[k] = (uint32_t *)(b + o); o += b2_al(A.emax * 4);
    }
    return W;
}

// warp-aggregated increment of a shared counter; every lane calls it
__device__ __forceinline__ int b2_take(bool pred, int *counter) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, pred);
    if (!m) return -1;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    return pred ? base + __popc(m & ((1u << lane) - 1u)) : -1;
}

// block-aggregated increment of a shared counter by cnt; every thread of the
// block calls it (warp-aggregated atomics; no block barrier)
__device__ __forceinline__ int b2_take_block(int cnt, int *counter) {
    const int lane = threadIdx.x & 31;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    int base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, total);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    return base + incl - cnt;
}

// One graph of one image.  mode 0: the pixels (H0); mode 1: the squares and
// the outer node (dimension 1 by duality, reversed keys).  Returns false when
// the call must stop (an error was recorded in the status word).
template <int T>
__device__ bool b2_graph(const B2Args &A, const B2Work &W, const Seg &S, int si, int mode, int *s_cnt,
                         int *s_ne, int *s_flag) {
    const int tid = threadIdx.x;
    const int nx = S.nx, ny = S.ny, cx = nx - 1, cy = ny - 1;
    const int64_t N = mode == 0 ? (int64_t)nx * ny : (int64_t)cx * cy + 1;  // the outer node is the last
    const int64_t outer = N - 1;
    const float *im = A.img + S.voff;
    const uint32_t P = (uint32_t)nx * (uint32_t)ny;  // one type's L-range
    const bool keep_zero = (A.flags & CR_KEEP_ZERO) != 0;
    if (N > A.nmax) { if (tid == 0) fail_ws(A.status, SITE_GROUPS); return false; }

    // 1. each node's first hook (the tile kernels' stencils, one image)
    bool nan_seen = false;
    for (int64_t i = tid; i < N; i += T) {
        if (mode == 0) {
            const int x = (int)(i % nx), y = (int)(i / nx);
            const float fv = im[i];
            nan_seen |= isnan(fv);
            // the first neighbour with phi <= phi(v) in descending edge-L order (+y, -y, +x, -x)
            int dir = 0;
            float fu = 0.f;
            if (x > 0 && im[i - 1] <= fv) { dir = 1; fu = im[i - 1]; }
            if (x + 1 < nx && im[i + 1] <= fv) { dir = 2; fu = im[i + 1]; }
            if (y > 0 && im[i - nx] <= fv) { dir = 3; fu = im[i - nx]; }
            if (y + 1 < ny && im[i + nx] <= fv) { dir = 4; fu = im[i + nx]; }
            if (dir && (fu < fv || !(dir & 1))) {  // the neighbour is older
                const uint32_t stp = dir <= 2 ? 1u : (uint32_t)nx;
                const uint32_t lu = (dir & 1) ? (uint32_t)i - stp : (uint32_t)i + stp;
                W.par[i] = lu;
                W.dd[i] = (uint8_t)dir;
                if (keep_zero) {
                    const uint32_t la = ((dir & 1) ? lu : (uint32_t)i) + (dir >= 3 ? P : 0u);
                    const float cv = unord32(ord32(fv));
                    emit_pair(A.pb, (uint32_t)si, 0, cv, cv, (int64_t)i, la, 0);
                }
            } else {
                W.par[i] = (uint32_t)i;
                W.dd[i] = 0;
            }
        } else {
            if (i == outer) {
                W.par[i] = (uint32_t)i;
                W.dd[i] = 0;
                continue;
            }
            const int x = (int)(i % cx), y = (int)(i / cx);
            const int64_t v = (int64_t)y * nx + x;
            const float v00 = im[v], v01 = im[v + 1], v10 = im[v + nx], v11 = im[v + nx + 1];
            // the square's first facet (-y, +y, -x, +x) holding its value
            const float ylo = fmaxf(v00, v01), yhi = fmaxf(v10, v11), xlo = fmaxf(v00, v10);
            const float fc = fmaxf(ylo, yhi);
            const int f = ylo == fc ? 0 : yhi == fc ? 1 : xlo == fc ? 2 : 3;
            const int axis = 1 - (f >> 1);  // 0 x, 1 y
            const bool up = f & 1;
            const bool outside = axis == 0 ? (up ? x + 1 >= cx : x == 0) : (up ? y + 1 >= cy : y == 0);
            bool hook = true;  // the outer node is the oldest
            int64_t other = outer;
            if (!outside) {
                float fo;
                if (axis == 0) {
                    const int64_t xx = up ? v + 2 : v - 1;
                    fo = fmaxf(im[xx], im[xx + nx]);
                    other = up ? i + 1 : i - 1;
                } else {
                    const int64_t yy = up ? v + 2 * (int64_t)nx : v - nx;
                    fo = fmaxf(im[yy], im[yy + 1]);
                    other = up ? i + cx : i - cx;
                }
                hook = fo > fc || !up;  // the neighbour's value is max(fo, phi(c)); equal values: the - side is older
            }
            if (hook) {
                W.par[i] = (uint32_t)other;
                W.dd[i] = (uint8_t)(f + 1);
                if (keep_zero) {
                    const int m = 1 - axis;
                    const uint32_t fl = cube_L(S, m, x + (axis == 0 && up), y + (axis == 1 && up), 0);
                    const float cv = unord32(ord32(fc));
                    emit_pair(A.pb, (uint32_t)si, 1, cv, cv, fl, cube_L(S, 0, x, y, 0), 0);
                }
            } else {
                W.par[i] = (uint32_t)i;
                W.dd[i] = 0;
            }
        }
    }
    if (nan_seen) set_status(A.status, CR_ERR_NAN);
    __syncthreads();

    // 2. pointer jumping to the roots (every write stores an ancestor)
    for (int pass = 0;; pass++) {
        int ch = 0;
        for (int64_t i = tid; i < N; i += T) {
            const uint32_t a = W.par[i], b = W.par[a];
            if (b != a) {
                W.par[i] = b;
                ch = 1;
            }
        }
        if (!__syncthreads_or(ch)) break;
        if (pass >= 64) {
            if (tid == 0) set_status(A.status, CR_ERR_INTERNAL);
            return false;
        }
    }

    // 3. the roots become groups (age key of the root: primal its vertex key,
    // dual the complemented key of its square; the outer node is the oldest)
    if (tid == 0) *s_cnt = 0;
    __syncthreads();
    for (int64_t base = 0; base < N; base += T) {
        const int64_t i = base + tid;
        const bool root = i < N && W.par[i] == (uint32_t)i;
        const int g = b2_take(root, s_cnt);
        if (!root) continue;
        uint64_t key;
        if (mode == 0) {
            key = make_key(ord32(im[i]), (uint32_t)i);
        } else if (i == outer) {
            key = 0;
        } else {
            const int x = (int)(i % cx), y = (int)(i / cx);
            const int64_t v = (int64_t)y * nx + x;
            const uint32_t o = max(max(ord32(im[v]), ord32(im[v + 1])), max(ord32(im[v + nx]), ord32(im[v + nx + 1])));
            key = ~make_key(o, cube_L(S, 0, x, y, 0));
        }
        W.gkey[g] = key;
        W.hook[g] = (uint32_t)g;
        W.dead[g] = 0;
        W.mA[g] = ~0ull;
        W.par[i] = MARK | (uint32_t)g;
    }
    __syncthreads();
    const int G = *s_cnt;
    for (int64_t i = tid; i < N; i += T) {
        const uint32_t v = W.par[i];
        W.par[i] = (v & MARK) ? (v & ~MARK) : (W.par[v] & ~MARK);
    }
    if (tid == 0) *s_ne = 0;
    __syncthreads();

    // 4. the edges between groups, and the first round's minimum edges
    const int64_t NE = mode == 0 ? (int64_t)nx * ny : (int64_t)nx * ny;  // positions: two edges each
    for (int64_t base = 0; base < NE; base += T) {
        const int64_t p = base + tid;
        uint64_t keys[2];
        uint32_t las[2], lbs[2];
        int cnt = 0;
        if (p < NE) {
            const int x = (int)(p % nx), y = (int)(p / nx);
            for (int a = 0; a < 2; a++) {
                if (mode == 0) {
                    const bool exists = a == 0 ? x + 1 < nx : y + 1 < ny;
                    if (!exists) continue;
                    const int64_t u = a == 0 ? p + 1 : p + nx;
                    if (W.dd[p] == (uint8_t)(2 * a + 2) || W.dd[u] == (uint8_t)(2 * a + 1)) continue;  // a hook
                    const uint32_t la = W.par[p], lb = W.par[u];
                    if (la == lb) continue;
                    const uint32_t ov = ord32(im[p]), ou = ord32(im[u]);
                    keys[cnt] = make_key(ov > ou ? ov : ou, (uint32_t)p + (uint32_t)a * P);
                    las[cnt] = la;
                    lbs[cnt] = lb;
                    cnt++;
                } else {
                    // a = 0: the x-edge at (x, y) between the squares (x, y-1) and (x, y);
                    // a = 1: the y-edge at (x, y) between the squares (x-1, y) and (x, y)
                    const bool exists = a == 0 ? x + 1 < nx : y + 1 < ny;
                    if (!exists) continue;
                    const int ax = a == 0 ? x : x - 1, ay = a == 0 ? y - 1 : y;
                    const bool ina = ax >= 0 && ay >= 0 && ax < cx && ay < cy;
                    const bool inb = x < cx && y < cy;
                    const int64_t na = ina ? (int64_t)ay * cx + ax : outer, nb = inb ? (int64_t)y * cx + x : outer;
                    const uint8_t fa = a == 0 ? 2 : 4, fb = a == 0 ? 1 : 3;  // hook codes across this facet
                    if ((ina && W.dd[na] == fa) || (inb && W.dd[nb] == fb)) continue;
                    const uint32_t la = W.par[na], lb = W.par[nb];
                    if (la == lb) continue;
                    const int64_t u = a == 0 ? p + 1 : p + nx;
                    const uint32_t ov = ord32(im[p]), ou = ord32(im[u]);
                    keys[cnt] = ~make_key(ov > ou ? ov : ou, (uint32_t)p + (uint32_t)a * P);
                    las[cnt] = la;
                    lbs[cnt] = lb;
                    cnt++;
                }
            }
        }
        for (int k = 0; k < 2; k++) {
            const int e = b2_take(k < cnt, s_ne);
            if (k >= cnt) continue;
            if (e >= A.emax) {
                fail_ws(A.status, SITE_EDGES);
                continue;
            }
            W.ek[0][e] = keys[k];
            W.ea[0][e] = las[k];
            W.eb[0][e] = lbs[k];
            atomicMin((unsigned long long *)&W.mA[las[k]], keys[k]);
            atomicMin((unsigned long long *)&W.mA[lbs[k]], keys[k]);
        }
    }
    if (tid == 0) *s_flag = *(volatile int *)A.status;  // one reading for the whole block
    __syncthreads();
    const int64_t ne = *s_ne < A.emax ? *s_ne : A.emax;
    if (*s_flag) return false;

    // 5. Borůvka rounds under the elder rule.  The edge loops take four edges
    // per thread at a time (their loads are independent), and the edges that
    // stay live are compacted into the other buffer.
    constexpr int U = 4;
    uint64_t *mcur = W.mA, *mnext = W.mB;
    int64_t nlive = ne;
    int cb = 0;  // edge buffer in use
    for (long long round = 0;; round++) {
        if (round >= A.round_cap) {
            if (tid == 0) set_status(A.status, CR_ERR_TIMEOUT);
            return false;
        }
        const uint64_t *ek = W.ek[cb];
        const uint32_t *ea = W.ea[cb], *eb = W.eb[cb];
        // B: the edge attaining the younger end's minimum edge kills it
        for (int64_t i0 = tid; i0 < nlive; i0 += (int64_t)U * T) {
            uint32_t e0[U], e1[U];
            uint64_t k[U], k0[U], k1[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t i = i0 + (int64_t)u * T;
                e0[u] = i < nlive ? ea[i] : 0u;
                e1[u] = i < nlive ? eb[i] : 0u;
                k[u] = i < nlive ? ek[i] : 0ull;
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                k0[u] = W.gkey[e0[u]];
                k1[u] = W.gkey[e1[u]];
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (e0[u] == e1[u]) continue;  // past the end (0, 0)
                const bool young0 = k1[u] < k0[u];
                const uint32_t g = young0 ? e0[u] : e1[u], t = young0 ? e1[u] : e0[u];
                if (mcur[g] != k[u]) continue;
                W.hook[g] = t;
                W.dead[g] = 1;
                W.dkey[g] = k[u];
            }
        }
        for (int g = tid; g < G; g += T) mnext[g] = ~0ull;
        __syncthreads();
        // C: pointer jumping to this round's roots (and the live-edge counter
        // reset: every thread read it before the barrier above)
        if (tid == 0) *s_ne = 0;
        for (int g = tid; g < G; g += T) {
            uint32_t p = W.hook[g];
            if (p == (uint32_t)g) continue;
            for (int it = 0; it < (1 << 24); it++) {
                const uint32_t pp = W.hook[p];
                if (pp == p) break;
                p = pp;
                W.hook[g] = p;
            }
        }
        __syncthreads();
        // D: edges move to their roots; those between two groups go to the
        // other buffer and are offered to the next minimum edges
        uint64_t *ok = W.ek[cb ^ 1];
        uint32_t *oa = W.ea[cb ^ 1], *ob = W.eb[cb ^ 1];
        for (int64_t base = 0; base < nlive; base += (int64_t)U * T) {
            uint32_t a[U], b[U];
            uint64_t k[U];
            bool keep[U];
            int cnt = 0;
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t i = base + tid + (int64_t)u * T;
                const bool in = i < nlive;
                const uint32_t e0 = in ? ea[i] : 0u, e1 = in ? eb[i] : 0u;
                k[u] = in ? ek[i] : 0ull;
                a[u] = W.hook[e0];
                b[u] = W.hook[e1];
                keep[u] = in && a[u] != b[u];
                cnt += keep[u];
            }
            int64_t j = b2_take_block(cnt, s_ne);
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (!keep[u]) continue;
                ok[j] = k[u];
                oa[j] = a[u];
                ob[j] = b[u];
                j++;
                atomicMin((unsigned long long *)&mnext[a[u]], k[u]);
                atomicMin((unsigned long long *)&mnext[b[u]], k[u]);
            }
        }
        __syncthreads();
        nlive = *s_ne;
        cb ^= 1;
        uint64_t *t = mcur;
        mcur = mnext;
        mnext = t;
        if (nlive == 0) break;
    }

    // 6. the pairs: a dead group dies at its death edge; the surviving primal
    // group is the essential class
    for (int64_t base = 0; base < G; base += T) {
        const int g = (int)(base + tid);
        int emit = 0;
        cr_pair pr;
        if (g < G) {
            const uint64_t kb = W.gkey[g];
            if (!W.dead[g]) {
                if (mode == 0) {
                    pr = cr_pair{0, key_value(kb), __int_as_float(0x7f800000), CR_PAIR_ESSENTIAL | ((uint32_t)si << 8),
                                 (int64_t)key_L(kb), -1};
                    emit = 1;
                }
            } else {
                const uint64_t k = W.dkey[g];
                if (mode == 0) {
                    const float bv = key_value(kb), dv = key_value(k);
                    if (keep_zero || bv != dv) {
                        pr = cr_pair{0, bv, dv, (uint32_t)si << 8, (int64_t)key_L(kb), (int64_t)key_L(k)};
                        emit = 1;
                    }
                } else {
                    const uint64_t kf = ~k, kc = ~kb;
                    const float bv = key_value(kf), dv = key_value(kc);
                    if (keep_zero || bv != dv) {
                        pr = cr_pair{1, bv, dv, (uint32_t)si << 8, (int64_t)key_L(kf), (int64_t)key_L(kc)};
                        emit = 1;
                    }
                }
            }
        }
        const int64_t j = block_append(emit, A.pb.count);
        if (emit && j < A.pb.capacity) A.pb.pairs[j] = pr;
    }
    __syncthreads();  // the scratch is reused by the next graph
    return true;
}

template <int T>
__global__ void __launch_bounds__(T) k_batch2d(B2Args A) {
    __shared__ int s_img, s_cnt, s_ne, s_flag;
    const B2Work W = b2_work(A);
    for (int it = 0; it <= A.nimg; it++) {
        if (threadIdx.x == 0) {
            const unsigned long long q = atomicAdd(A.queue, 1ull);
            s_img = (q < (unsigned long long)A.nimg && !*(volatile int *)A.status) ? (int)A.order[q] : -1;
        }
        __syncthreads();
        const int si = s_img;
        __syncthreads();
        if (si < 0) return;
        const Seg S = A.segs[si];
        if (A.primal && !b2_graph<T>(A, W, S, si, 0, &s_cnt, &s_ne, &s_flag)) return;
        if (A.dual && !b2_graph<T>(A, W, S, si, 1, &s_cnt, &s_ne, &s_flag)) return;
    }
}

}  // namespace

// Both union-finds of a batch of 2D images (every image with nx, ny >= 2), one
// image per block.  `region` holds the work order and the blocks' scratch.
// Returns CR_ERR_WORKSPACE (nothing launched) when the region is too small
// for one block; the caller then runs the grid-wide path.
int run_batch2d(const float *img, const Seg *segs, const std::vector<Seg> &hsegs, const uint32_t *order,
                char *region, size_t region_cap, const PairBuf &pb, uint32_t flags, bool primal, bool dual,
                unsigned long long *queue, int *status, cudaStream_t st, int threads_code) {
    const int n = (int)hsegs.size();
    int64_t nmax = 1;
    for (const Seg &S : hsegs) {
        const int64_t v = (int64_t)S.nx * S.ny;
        nmax = v > nmax ? v : nmax;
    }
    const int64_t emax = 2 * nmax + 8;
    const size_t stride = b2_stride(nmax, emax);
    if (region_cap < stride) return CR_ERR_WORKSPACE;
    int threads = threads_code == 1 ? 256 : (threads_code == 3 ? 1024 : 512);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    int64_t blocks = (int64_t)sms * (2048 / threads);
    if (blocks > n) blocks = n;
    const int64_t fit = (int64_t)(region_cap / stride);
    if (blocks > fit) blocks = fit;
    cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st);
    B2Args A;
    A.img = img;
    A.segs = segs;
    A.order = order;
    A.nimg = n;
    A.queue = queue;
    A.scratch = region;
    A.stride = stride;
    A.nmax = nmax;
    A.emax = emax;
    A.pb = pb;
    A.flags = flags;
    A.status = status;
    A.round_cap = 1ll << 20;
    A.primal = primal;
    A.dual = dual;
    prof_begin(st, STAGE_UF_ROUND);
    CR_NOTE_LAUNCH();
    if (threads == 256)
        k_batch2d<256><<<(unsigned)blocks, 256, 0, st>>>(A);
    else if (threads == 1024)
        k_batch2d<1024><<<(unsigned)blocks, 1024, 0, st>>>(A);
    else
        k_batch2d<512><<<(unsigned)blocks, 512, 0, st>>>(A);
    prof_end(st, STAGE_UF_ROUND, 0.0);
    return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

}  // namespace cr
