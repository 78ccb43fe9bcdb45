// cr_api.cu -- the C ABI of libcr (declared in include/cr.h): validation,
// workspace layout, the order of the stages, the canonical output order and
// the backward scatter.
//
// Stages of one call (all images of a batch at once):
//   H0      union-find with the elder rule on the pixel graph (Sec. 2);
//   H1 (3D) apparent pairs + lock-free coboundary reduction (Sec. 2);
//   top     union-find on the dual graph in the reversed order (Sec. 2,
//           Rem. 2.1): dimension 1 of a 2D image, dimension 2 of a volume;
//   output  pairs sorted by (image, dim, birth, birth cell).
#include "cr_internal.cuh"
#include <algorithm>
#include <mutex>
#include <vector>
#include <cmath>
#include <cstdlib>

namespace cr {

// ---------------------------------------------------------------------------
// Launch knobs (host-side, per process): see cr_tune_set in include/cr.h.
// ---------------------------------------------------------------------------
static std::atomic<int> g_tune[CR_TUNE_COUNT] = {{8}, {16}, {1}, {2}, {1024}};
static std::atomic<uint32_t> g_tune_epoch{0};
static const int g_tune_lo[CR_TUNE_COUNT] = {1, 1, 1, 0, 0}, g_tune_hi[CR_TUNE_COUNT] = {64, 16, 64, 3, 1 << 24};
int tune_value(int knob) { return g_tune[knob].load(std::memory_order_relaxed); }
uint32_t tune_epoch() { return g_tune_epoch.load(std::memory_order_relaxed); }

static thread_local int g_detail = 0;
void set_host_detail(int site) { g_detail = site; }

// limits of the bounded device waits (cr_debug_limits)
static std::atomic<long long> g_dbg_polls{DEFAULT_BARRIER_POLLS}, g_dbg_iters{DEFAULT_REDUCE_ITERS};
static std::atomic<unsigned int> g_dbg_extra{0};
DebugLimits debug_limits() {
    return DebugLimits{g_dbg_polls.load(std::memory_order_relaxed), g_dbg_iters.load(std::memory_order_relaxed),
                       g_dbg_extra.load(std::memory_order_relaxed)};
}

// Host-side fault injection (CR_FAULT=<site> in the environment, read at each
// call): the forward entry points fail as the named fault would, before any
// GPU work ("shape", "nan", "workspace") or, for "capacity", by running with
// no room for pairs, so that every error return can be exercised without a
// faulty input or a GPU fault.
enum Fault { FAULT_NONE = 0, FAULT_SHAPE, FAULT_NAN, FAULT_WORKSPACE, FAULT_CAPACITY };
static int injected_fault() {
    const char *e = getenv("CR_FAULT");
    if (!e || !*e) return FAULT_NONE;
    if (!strcmp(e, "shape")) return FAULT_SHAPE;
    if (!strcmp(e, "nan")) return FAULT_NAN;
    if (!strcmp(e, "workspace")) return FAULT_WORKSPACE;
    if (!strcmp(e, "capacity")) return FAULT_CAPACITY;
    return FAULT_NONE;
}
int injected_error_before_gpu() {
    switch (injected_fault()) {
    case FAULT_SHAPE: return CR_ERR_INVALID_ARG;
    case FAULT_NAN: return CR_ERR_NAN;
    case FAULT_WORKSPACE: g_detail = SITE_INJECTED; return CR_ERR_WORKSPACE;
    default: return CR_OK;
    }
}



// ---------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------
struct HostPlan {
    std::vector<Seg> segs;
    int64_t vtot = 0, ctot = 0, cells = 0, ntiles = 0;
    int64_t nstiles = 0;  // 32x32 super-tiles over all images (used when every image is 2D)
    bool all_2d = true;
    int64_t max_face_per_image = 0;
    bool any_h0 = false, any_dual = false, any_mid = false;
    bool serial_uf = false;  // run the two union-finds one after the other (half the region)
    bool graphs = true;      // single 1D/2D images may replay their launches as a CUDA graph
    int nseg_bits = 0;
};

static int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    }
    return sms;
}

static int64_t cube_count(int64_t nz, int64_t ny, int64_t nx) {
    // all cubes of the full grid: prod over axes of (n + (n-1)) = prod (2n - 1)
    return (2 * nz - 1) * (2 * ny - 1) * (2 * nx - 1);
}

static int plan_images(const int64_t *const *shapes_rows, int n, int ndim, int maxdim, uint32_t flags, HostPlan &P) {
    if (n < 1 || ndim < 1 || ndim > 3 || maxdim < 0) return CR_ERR_INVALID_ARG;
    if (flags & ~(CR_KEEP_ZERO | CR_TOPDIM_ONLY | CR_LOC_DEATH)) return CR_ERR_INVALID_ARG;
    P.segs.resize(n);
    int64_t voff = 0, coff = 0;
    for (int i = 0; i < n; i++) {
        const int64_t *sh = shapes_rows[i];
        int64_t nz = 1, ny = 1, nx = 1;
        if (ndim == 1) nx = sh[0];
        else if (ndim == 2) { ny = sh[0]; nx = sh[1]; }
        else { nz = sh[0]; ny = sh[1]; nx = sh[2]; }
        if (nz < 1 || ny < 1 || nx < 1) return CR_ERR_INVALID_ARG;
        int64_t v = nz * ny * nx;
        if (nz > 65535 * 32 || ny > 65535 * 32 || nx > 65535 * 32 || 3 * v >= ((int64_t)1 << 32))
            return CR_ERR_TOO_LARGE;
        Seg &S = P.segs[i];
        S.voff = voff;
        S.loff = 3 * voff;
        S.nx = (int32_t)nx;
        S.ny = (int32_t)ny;
        S.nz = (int32_t)nz;
        S.edim = nz > 1 ? 3 : (ny > 1 ? 2 : (nx > 1 ? 1 : 0));
        int top = S.edim >= 1 ? S.edim - 1 : 0;
        bool topdim = (flags & CR_TOPDIM_ONLY) != 0;
        bool want_h0 = maxdim >= 0 && (!topdim || top == 0);
        bool want_dual = S.edim >= 2 && (topdim || maxdim >= S.edim - 1);
        bool want_mid = S.edim == 3 && !topdim && maxdim >= 1;
        int64_t ncell = 0;
        if (want_dual) ncell = S.edim == 3 ? (nx - 1) * (ny - 1) * (nz - 1) : (nx - 1) * (ny - 1);
        S.coff = coff;
        S.ncell = ncell;
        S.tiles_x = (int32_t)((nx + TILE_X - 1) / TILE_X);
        S.tiles_y = (int32_t)((ny + TILE_Y - 1) / TILE_Y);
        S.tiles_z = (int32_t)((nz + TILE_Z - 1) / TILE_Z);
        S.stoff = (int32_t)P.nstiles;
        P.nstiles += ((nx + ST_X - 1) / ST_X) * ((ny + ST_Y - 1) / ST_Y);
        P.all_2d &= S.edim == 2 && nz == 1;
        S.toff = P.ntiles;
        P.ntiles += (int64_t)S.tiles_x * S.tiles_y * S.tiles_z;
        P.any_h0 |= want_h0 || want_mid;
        P.any_dual |= ncell > 0;
        P.any_mid |= want_mid;
        int64_t faces = 3 * v;
        if (faces > P.max_face_per_image) P.max_face_per_image = faces;
        voff += v;
        coff += ncell + 1;
        P.cells += cube_count(nz, ny, nx);
    }
    P.vtot = voff;
    P.ctot = coff;
    if (P.nstiles >= ((int64_t)1 << 31)) P.all_2d = false;
    if (P.vtot >= ((int64_t)1 << 31) - 2 || P.ctot >= ((int64_t)1 << 31) - 2 || 3 * P.vtot >= ((int64_t)1 << 40))
        return CR_ERR_TOO_LARGE;
    int b = 0;
    while (((int64_t)1 << b) < n) b++;
    P.nseg_bits = b;
    return CR_OK;
}

// scratch geometry of the reduction
static void red_geometry(const HostPlan &P, int64_t &nwarps, int &maxlen) {
    nwarps = (int64_t)num_sms() * 16;
    int64_t ml = P.max_face_per_image + 32;
    if (ml > 4096) ml = 4096;  // longer columns move to buffers grown from the pool
    maxlen = (int)((ml + 31) & ~31);
}

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// pairs of a single image sorted by rank on the device (see k_out_rank)
constexpr int SMALL_SORT = 16384;

// fixed part of the workspace
static size_t fixed_bytes(const HostPlan &P) {
    size_t b = 0;
    b += al(P.segs.size() * sizeof(Seg));
    b += al(P.segs.size() * sizeof(uint32_t));          // work order of a batch (largest image first)
    b += al(CR_CNT_SLOTS * sizeof(unsigned long long));  // status + counters
    b += al((size_t)P.vtot * sizeof(uint32_t));  // primal labels
    b += al((size_t)P.ctot * sizeof(uint32_t));  // dual labels
    b += al((size_t)P.vtot);                    // primal hooks
    b += al((size_t)P.ctot);                    // dual hooks
    b += al((size_t)((3 * P.vtot + 31) / 32) * sizeof(uint32_t));  // extra H0 edge mask
    return b;
}

// region shared by the stages; `worst` gives a bound that the union-find and
// sorting stages never exceed
static size_t region_bytes(const HostPlan &P, uint32_t flags, bool worst) {
    int64_t nodes = P.vtot > P.ctot ? P.vtot : P.ctot;
    size_t uf, h1 = 0, out;
    if (worst) {
        uf = al((size_t)nodes * 45) + al((size_t)(3 * P.vtot) * 32) + (1 << 20);
    } else {
        // the dual graph of a volume keeps most of its 3 faces per voxel as
        // cross edges (its first groups are small: the cubes around one
        // maximal vertex), so volumes get room for ~2.5 edges per voxel
        int edim = 1;
        for (const Seg &S : P.segs) edim = S.edim > edim ? S.edim : edim;
        uf = al((size_t)nodes * 16) + al((size_t)P.vtot * (edim == 3 && P.any_dual ? 96 : 48)) + (8 << 20);
    }
    if (P.any_h0 && P.any_dual && !P.serial_uf) uf *= 2;  // both union-finds are live at once
    if (P.any_mid) {
        int64_t nw;
        int ml;
        red_geometry(P, nw, ml);
        int64_t cols = worst ? 3 * P.vtot : (3 * P.vtot) / 8 + 4096;
        int64_t arena = worst ? 12 * P.vtot : 2 * P.vtot + (1 << 20);
        int64_t pool = worst ? 8 * P.vtot : 2 * P.vtot + (1 << 22);
        h1 = al((size_t)cols * 32) + al(radix_temp_bytes(cols)) + al((size_t)(3 * P.vtot) * 8) +
             al((size_t)P.vtot) +
             al((size_t)arena * 8) + al((size_t)pool * 8) + al((size_t)nw * 2 * ml * 8) + (1 << 20);
    }
    int64_t maxpairs = (flags & CR_KEEP_ZERO) ? P.cells / 2 + (int64_t)P.segs.size() + 16
                                              : (worst ? P.cells / 2 + (int64_t)P.segs.size() + 16
                                                       : P.vtot / 4 + 4096);
    out = al((size_t)maxpairs * (24 + 32)) + al(radix_temp_bytes(maxpairs)) + al((size_t)P.segs.size() * 4 + 64) +
          al(scan_temp_bytes((int64_t)P.segs.size() + 1)) + (1 << 20);
    if (P.segs.size() == 1) {  // the rank sort's buffers
        const size_t rk = al((size_t)SMALL_SORT * 4) + al((size_t)SMALL_SORT * sizeof(cr_pair)) + 1024;
        out = out > rk ? out : rk;
    }
    size_t r = uf;
    if (h1 > r) r = h1;
    if (out > r) r = out;
    return r;
}

static size_t total_bytes(const HostPlan &P, uint32_t flags, bool worst) {
    size_t w = fixed_bytes(P) + region_bytes(P, flags, true) + 1024;
    if (worst) return w;
    size_t t = fixed_bytes(P) + region_bytes(P, flags, false) + 1024;
    return t < w ? t : w;
}

// ---------------------------------------------------------------------------
// output: sort by (image, dim, birth, birth cell), write pair offsets
// ---------------------------------------------------------------------------
__global__ void k_out_keys(cr_pair *pairs, int64_t np, uint64_t *keys, uint32_t *vals, uint32_t *segc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    cr_pair p = pairs[i];
    keys[i] = ((uint64_t)ord32(p.birth) << 32) | (uint64_t)(uint32_t)p.birth_cell;
    vals[i] = (uint32_t)i;
    if (segc) atomicAdd(&segc[p.flags >> 8], 1u);
}
__global__ void k_out_rekey(const cr_pair *pairs, int64_t np, const uint32_t *vals, uint64_t *keys, int what) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const cr_pair &p = pairs[vals[i]];
    keys[i] = what == 0 ? (uint64_t)p.dim : (uint64_t)(p.flags >> 8);
}
// the final copy clears the image index (bits 8..31) and sets `setbits`
// (CR_PAIR_LOC_DEATH when the caller asked for death locations)
__global__ void k_out_gather(const cr_pair *src, int64_t np, const uint32_t *vals, cr_pair *dst, uint32_t setbits) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    cr_pair p = src[vals[i]];
    p.flags = (p.flags & 0xFFu) | setbits;
    dst[i] = p;
}
__global__ void k_out_offsets(const uint32_t *scanned, int n, int64_t np, int64_t *offs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) offs[i] = (int64_t)scanned[i];
    if (i == n) offs[n] = np;
}
static inline unsigned nbk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Up to SMALL_SORT pairs of a single image are ordered by rank: the packed
// key dim:2 | ord32(birth):32 | birth_cell:30 is unique (a cell gives birth
// to at most one class of its dimension), so the destination of pair i is the
// number of smaller keys.  Blocks own RK_T*RK_R pairs and one slice of the
// keys to compare against, so a few thousand pairs still spread over the GPU.
constexpr int RK_T = 128, RK_R = 4, RK_TILE = 1024;

__device__ __forceinline__ uint64_t pair_sort_key(const cr_pair *p) {
    return ((uint64_t)(p->dim & 3) << 62) | ((uint64_t)ord32(p->birth) << 30) | (uint64_t)(p->birth_cell & 0x3FFFFFFF);
}

// rank[i] += #{j in this block's slice : key_j < key_i}; slice 0 also copies
// the pairs to tmp.  The pair count is read on the device (at most `cap`);
// counts above SMALL_SORT are left to the radix path (the kernels do nothing).
__global__ void __launch_bounds__(RK_T) k_out_rank(const cr_pair *__restrict__ pairs,
                                                   const unsigned long long *__restrict__ npp, int64_t cap,
                                                   uint32_t *__restrict__ rank, cr_pair *__restrict__ tmp) {
    __shared__ uint64_t tile[RK_TILE];
    const int64_t npl = (int64_t)*npp < cap ? (int64_t)*npp : cap;
    if (npl > SMALL_SORT) return;
    const int np = (int)npl;
    const int base = blockIdx.x * RK_T * RK_R;
    if (base >= np) return;
    const int chunk = (np + gridDim.y - 1) / gridDim.y;
    uint64_t mine[RK_R];
    uint32_t cnt[RK_R];
#pragma unroll
    for (int r = 0; r < RK_R; r++) {
        const int i = base + r * RK_T + threadIdx.x;
        mine[r] = i < np ? pair_sort_key(pairs + i) : 0ull;
        cnt[r] = 0;
        if (blockIdx.y == 0 && i < np) tmp[i] = pairs[i];
    }
    const int j0 = blockIdx.y * chunk, j1 = min(np, j0 + chunk);
    for (int t0 = j0; t0 < j1; t0 += RK_TILE) {
        const int n = min(RK_TILE, j1 - t0);
        for (int q = threadIdx.x; q < n; q += RK_T) tile[q] = pair_sort_key(pairs + t0 + q);
        __syncthreads();
        int q = 0;
        for (; q + 4 <= n; q += 4) {
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const uint64_t kj = tile[q + u];
#pragma unroll
                for (int r = 0; r < RK_R; r++) cnt[r] += kj < mine[r] ? 1u : 0u;
            }
        }
        for (; q < n; q++) {
            const uint64_t kj = tile[q];
#pragma unroll
            for (int r = 0; r < RK_R; r++) cnt[r] += kj < mine[r] ? 1u : 0u;
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < RK_R; r++) {
        const int i = base + r * RK_T + threadIdx.x;
        if (i < np && cnt[r]) atomicAdd(&rank[i], cnt[r]);
    }
}

__global__ void k_out_place(const cr_pair *__restrict__ tmp, const unsigned long long *__restrict__ npp, int64_t cap,
                            const uint32_t *__restrict__ rank, cr_pair *__restrict__ pairs, uint32_t setbits) {
    const int64_t npl = (int64_t)*npp < cap ? (int64_t)*npp : cap;
    if (npl > SMALL_SORT) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int)npl) return;
    cr_pair p = tmp[i];
    p.flags = (p.flags & 0xFFu) | setbits;
    const uint32_t d = rank[i];
    if (d < (uint32_t)npl) pairs[d] = p;
}

// Group and edge arrays of one union-find in [base, base + cap): the number of
// roots is not known yet, so the groups get a share proportional to the node
// count (at most a third) and the edges the rest, two buffers of at most
// 3 edges per voxel.
static int carve_uf(char *base, size_t cap, int64_t nodes, int64_t vtot, UF &u) {
    Carver R(base, cap);
    int64_t max_groups = nodes;
    size_t gbytes = (size_t)max_groups * 45 + 8 * 256;
    if (gbytes > cap / 3) max_groups = (int64_t)((cap / 3) / 45) - 64;
    if (max_groups < 1) { g_detail = SITE_UF_CARVE; return CR_ERR_WORKSPACE; }
    u.gkey = R.take<uint64_t>(max_groups);
    u.minE = R.take<uint64_t>(max_groups);
    u.groot = R.take<uint32_t>(max_groups);
    u.gseg = R.take<uint32_t>(max_groups);
    u.minE2 = R.take<uint64_t>(max_groups);
    u.dkey = R.take<uint64_t>(max_groups);
    u.hook = R.take<uint32_t>(max_groups);
    u.gdead = R.take<uint8_t>(max_groups);
    u.max_groups = max_groups;
    size_t left = R.cap > R.used ? R.cap - R.used : 0;
    int64_t max_edges = (int64_t)(left / 32) - 64;
    if (max_edges > 3 * vtot + 1) max_edges = 3 * vtot + 1;
    if (max_edges < 1 || !R.ok) { g_detail = SITE_UF_CARVE; return CR_ERR_WORKSPACE; }
    for (int b = 0; b < 2; b++) {
        u.ek[b] = R.take<uint64_t>(max_edges);
        u.ea[b] = R.take<uint32_t>(max_edges);
        u.eb[b] = R.take<uint32_t>(max_edges);
    }
    u.max_edges = max_edges;
    if (!R.ok) { g_detail = SITE_UF_CARVE; return CR_ERR_WORKSPACE; }
    return CR_OK;
}

// ---------------------------------------------------------------------------
// CUDA graphs of the launch sequence of single 1D/2D images and of batches
// of them, forward and backward.  The sequence depends only on the arguments
// below, so the second call with the same arguments captures it and later
// calls replay it with one launch; the first call runs directly (it also sets
// kernel attributes, which are not stream operations).  Host data the
// sequence reads (image table, work order) is copied before the captured part.
// Capture failures fall back to direct launches.
// ---------------------------------------------------------------------------
// Everything a launch sequence depends on, as words: the entry point, the
// pointers and sizes of the call, the images' shapes (hashed), the stream and
// device, the stage-timing state and the launch-knob epoch (launch shapes
// were fixed at capture).
struct GraphKey {
    static constexpr int NW = 20;
    uint64_t w[NW] = {0};
    int n = 0;
    void add(uint64_t v) {
        if (n < NW) w[n++] = v;
    }
    void addp(const void *p) { add((uint64_t)(uintptr_t)p); }
    bool operator==(const GraphKey &o) const {
        if (n != o.n) return false;
        for (int i = 0; i < n; i++)
            if (w[i] != o.w[i]) return false;
        return true;
    }
};
static uint64_t shapes_hash(const std::vector<Seg> &segs) {
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the extents
    for (const Seg &S : segs)
        for (int32_t e : {S.nx, S.ny, S.nz}) {
            h ^= (uint64_t)(uint32_t)e;
            h *= 1099511628211ull;
        }
    return h ^ (uint64_t)segs.size();
}
struct GraphEntry {
    GraphKey key;
    int state;  // 0 seen once, 1 capturing, 2 replayable, -1 not capturable
    cudaGraphExec_t exec;
    long long launches;
    std::vector<std::pair<int, std::pair<void *, void *>>> prof_recs;
    std::vector<double> prof_bytes;
    uint64_t last_use;
};
static std::mutex g_graph_mu;
static std::vector<GraphEntry> g_graphs;
static uint64_t g_graph_tick = 0;
constexpr size_t MAX_GRAPHS_CACHED = 32;

static int current_device();
static cudaStream_t capture_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {nullptr};
    const int d = current_device();
    if (d < 0 || d >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!streams[d] && cudaStreamCreateWithFlags(&streams[d], cudaStreamNonBlocking) != cudaSuccess)
        streams[d] = nullptr;
    return streams[d];
}

static int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

template <class Fn>
static int run_graphed(const GraphKey &key, Fn &&launch_all, cudaStream_t st) {
    GraphEntry *E = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        for (auto &e : g_graphs)
            if (e.key == key) E = &e;
        if (!E) {
            if (g_graphs.size() >= MAX_GRAPHS_CACHED) {  // drop the least recently used
                size_t victim = 0;
                for (size_t i = 1; i < g_graphs.size(); i++)
                    if (g_graphs[i].last_use < g_graphs[victim].last_use) victim = i;
                if (g_graphs[victim].state == 1) return launch_all(st);  // busy: do not disturb
                if (g_graphs[victim].exec) cudaGraphExecDestroy(g_graphs[victim].exec);
                g_graphs.erase(g_graphs.begin() + (long)victim);
            }
            g_graphs.push_back(GraphEntry{key, 0, nullptr, 0, {}, {}, ++g_graph_tick});
            E = nullptr;  // first sighting: run directly
        } else {
            E->last_use = ++g_graph_tick;
            if (E->state == 2) {
                if (cudaGraphLaunch(E->exec, st) != cudaSuccess) return CR_ERR_CUDA;
                g_launch_count.fetch_add(E->launches, std::memory_order_relaxed);
                prof_replay(E->prof_recs, E->prof_bytes);
                return CR_OK;
            }
            if (E->state != 0) return launch_all(st);
            E->state = 1;
        }
    }
    if (!E) return launch_all(st);
    // capture this call's launches
    const long long l0 = g_launch_count.load();
    std::vector<std::pair<int, std::pair<void *, void *>>> recs;
    std::vector<double> bytes;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    // captured on a stream of our own (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the caller's
    cudaStream_t cs = capture_stream();
    bool ok = cs && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int rc = CR_OK;
    if (ok) {
        prof_capture_begin();
        rc = launch_all(cs);
        prof_capture_end(recs, bytes);
        ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && g && rc == CR_OK;
        if (ok) ok = cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
    }
    std::lock_guard<std::mutex> lk(g_graph_mu);
    GraphEntry *G = nullptr;
    for (auto &e : g_graphs)
        if (e.key == key) G = &e;
    if (!ok) {
        cudaGetLastError();  // clear a capture error
        g_launch_count.store(l0);
        if (G) G->state = -1;
        return launch_all(st);
    }
    if (!G) {  // evicted meanwhile: keep it anyway
        g_graphs.push_back(GraphEntry{key, 2, x, 0, {}, {}, ++g_graph_tick});
        G = &g_graphs.back();
    }
    G->state = 2;
    G->exec = x;
    G->launches = g_launch_count.load() - l0;
    G->prof_recs = recs;
    G->prof_bytes = bytes;
    if (cudaGraphLaunch(x, st) != cudaSuccess) return CR_ERR_CUDA;
    prof_replay(G->prof_recs, G->prof_bytes);
    return CR_OK;
}

// ---------------------------------------------------------------------------
// the pipeline
// ---------------------------------------------------------------------------
static int pipeline(const float *imgs, HostPlan &P, int maxdim, uint32_t flags, cr_pair *pairs_out, int64_t capacity,
                    int64_t *pair_offsets, int64_t *n_pairs, void *ws, size_t ws_bytes, cudaStream_t st) {
    (void)maxdim;
    const int n = (int)P.segs.size();
    g_detail = 0;
    if (int e = injected_error_before_gpu()) return e;
    if (injected_fault() == FAULT_CAPACITY) capacity = 0;
    size_t need_min = fixed_bytes(P) + 1024;
    if (!ws || ws_bytes < need_min) { g_detail = SITE_FIXED; return CR_ERR_WORKSPACE; }
    Carver C(ws, ws_bytes);
    Seg *segs = C.take<Seg>(n);
    uint32_t *order = C.take<uint32_t>(n);
    unsigned long long *cnt = C.take<unsigned long long>(CR_CNT_SLOTS);
    uint32_t *lab = C.take<uint32_t>(P.vtot);
    uint32_t *labc = C.take<uint32_t>(P.ctot);
    uint8_t *dd = C.take<uint8_t>(P.vtot);
    uint8_t *ddc = C.take<uint8_t>(P.ctot);
    int64_t mask_words = (3 * P.vtot + 31) / 32;
    uint32_t *extra = C.take<uint32_t>(mask_words);
    if (!C.ok) { g_detail = SITE_FIXED; return CR_ERR_WORKSPACE; }
    char *region = (char *)ws + ((C.used + 255) & ~(size_t)255);
    size_t region_cap = ws_bytes - ((C.used + 255) & ~(size_t)255);
    int *status = (int *)&cnt[0];
    unsigned long long *pair_count = &cnt[1];

    cudaMemcpyAsync(segs, P.segs.data(), n * sizeof(Seg), cudaMemcpyHostToDevice, st);
    const bool batch2d = n > 1 && P.all_2d && !P.any_mid && (P.any_h0 || P.any_dual) &&
                         tune_value(CR_TUNE_BATCH_THREADS) > 0;
    std::vector<uint32_t> horder;
    if (batch2d) {  // the work queue of the persistent launch: images by size, largest first
        horder.resize(n);
        for (int i = 0; i < n; i++) horder[i] = (uint32_t)i;
        std::stable_sort(horder.begin(), horder.end(), [&](uint32_t a, uint32_t b) {
            return (int64_t)P.segs[a].nx * P.segs[a].ny > (int64_t)P.segs[b].nx * P.segs[b].ny;
        });
        cudaMemcpyAsync(order, horder.data(), (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    }

    PairBuf pb;
    pb.pairs = pairs_out;
    pb.capacity = capacity;
    pb.count = pair_count;

    unsigned long long hc[4];
    int rc = CR_OK;
    const bool rank_sort = n == 1 && 3 * P.vtot < ((int64_t)1 << 30);
    const uint32_t locbits = (flags & CR_LOC_DEATH) ? CR_PAIR_LOC_DEATH : 0u;

    // everything up to the count readback; a fixed sequence of launches for a
    // given image, so 1D/2D single images replay it as a CUDA graph
    auto phase1 = [&](cudaStream_t st) -> int {
    int rc = CR_OK;
    cudaMemsetAsync(cnt, 0, CR_CNT_SLOTS * sizeof(unsigned long long), st);
    if (P.any_mid) cudaMemsetAsync(extra, 0, (size_t)mask_words * 4, st);

    // ---- batches of 2D images: both union-finds in one persistent launch,
    // one image per block from a queue ordered by size (unless the launch knob
    // selects the grid-wide kernels, or the region cannot hold a block) ----
    bool batched_done = false;
    if (batch2d) {
        rc = run_batch2d(imgs, segs, P.segs, order, region, region_cap, pb, flags, P.any_h0, P.any_dual, &cnt[9],
                         status, st, tune_value(CR_TUNE_BATCH_THREADS));
        if (rc != CR_OK && rc != CR_ERR_WORKSPACE) return rc;
        batched_done = rc == CR_OK;
        rc = CR_OK;
    }
    // ---- H0 and the top dimension by duality: two independent union-finds,
    // run side by side in halves of the region ----
    if (!batched_done && (P.any_h0 || P.any_dual)) {
        const bool both = P.any_h0 && P.any_dual && !P.serial_uf;
        const size_t half = both ? (region_cap / 2) & ~(size_t)255 : region_cap;
        // several 2D images: both stencils in one kernel over 32x32 super-tiles
        const int64_t fused2d = (n > 1 && P.all_2d) ? P.nstiles : 0;
        UF uh, ud;
        if (P.any_h0) {
            rc = carve_uf(region, half, P.vtot, P.vtot, uh);
            if (rc) return rc;
            uh.lab = lab;
            uh.dd = dd;
            uh.cnt = &cnt[CNT_H0];
            uh.hcnt = hc;
        }
        if (P.any_h0 && !both) {
            rc = run_uf(imgs, segs, P.segs.data(), n, P.vtot, P.ctot, P.ntiles, fused2d, &uh, nullptr, pb, flags,
                        P.any_mid ? extra : nullptr, status, st);
            if (rc) return rc;
        }
        if (P.any_dual) {
            rc = carve_uf(region + (both ? half : 0), both ? region_cap - half : region_cap, P.ctot, P.vtot, ud);
            if (rc) return rc;
            ud.lab = labc;
            ud.dd = ddc;
            ud.cnt = &cnt[CNT_DUAL];
            ud.hcnt = hc;
        }
        if (both || P.any_dual) {
            rc = run_uf(imgs, segs, P.segs.data(), n, P.vtot, P.ctot, P.ntiles, fused2d, both ? &uh : nullptr, &ud,
                        pb, flags, both && P.any_mid ? extra : nullptr, status, st);
            if (rc) return rc;
        }
    }

    // ---- middle dimension of volumes ----
    if (P.any_mid) {
        Carver R(region, region_cap);
        H1Bufs B;
        int64_t nw;
        int ml;
        red_geometry(P, nw, ml);
        B.nwarps = nw;
        B.maxlen = ml;
        B.P_len = 3 * P.vtot;
        B.P = R.take<unsigned long long>(B.P_len);
        B.code = R.take<uint8_t>(P.vtot);
        B.scratch = R.take<uint64_t>((size_t)nw * 2 * ml);
        B.cnt = &cnt[CNT_H1];
        if (!R.ok) { g_detail = SITE_H1_CARVE; return CR_ERR_WORKSPACE; }
        size_t left = R.cap - R.used;
        // columns (32 B each + sort temp) get up to half of what is left, the arena the rest
        int64_t max_cols = (int64_t)((left / 2) / 40) - 1024;
        if (max_cols > 3 * P.vtot + 1) max_cols = 3 * P.vtot + 1;
        if (max_cols < 1) { g_detail = SITE_H1_CARVE; return CR_ERR_WORKSPACE; }
        B.colkey = R.take<uint64_t>(max_cols);
        B.colkey_tmp = R.take<uint64_t>(max_cols);
        B.colseg = R.take<uint32_t>(max_cols);
        B.colseg_tmp = R.take<uint32_t>(max_cols);
        B.cur = R.take<unsigned long long>(max_cols);
        B.sort_temp_bytes = radix_temp_bytes(max_cols);
        B.sort_temp = R.take<char>(B.sort_temp_bytes);
        B.max_cols = max_cols;
        if (!R.ok) { g_detail = SITE_H1_CARVE; return CR_ERR_WORKSPACE; }
        left = R.cap - R.used;
        // the rest: 60% arena of published columns, 40% pool for long columns
        B.arena_cap = (int64_t)((left / 8) * 3 / 5) - 64;
        if (B.arena_cap < 64) { set_host_detail(SITE_H1_CARVE); return CR_ERR_WORKSPACE; }
        B.arena = R.take<uint64_t>(B.arena_cap);
        left = R.cap > R.used ? R.cap - R.used : 0;
        B.pool_cap = (int64_t)(left / 8) - 64;
        if (B.pool_cap < 64) { set_host_detail(SITE_H1_CARVE); return CR_ERR_WORKSPACE; }
        B.pool = R.take<uint64_t>(B.pool_cap);
        int64_t ncols = 0;
        rc = run_h1(imgs, dd, extra, segs, P.segs.data(), n, P.vtot, P.ntiles, B, pb, flags, status, &ncols, st);
        if (rc) return rc;
    }

    // ---- canonical order of a single image's pairs, without reading the count:
    // the rank sort reads it on the device and stands aside above SMALL_SORT ----
    if (rank_sort) {
        Carver R(region, region_cap);
        uint32_t *rank = R.take<uint32_t>(SMALL_SORT);
        cr_pair *tmp = R.take<cr_pair>(SMALL_SORT);
        if (!R.ok) { g_detail = SITE_OUT_CARVE; return CR_ERR_WORKSPACE; }
        // blocks over pairs x slices of the keys: about two blocks per SM for ~8 k pairs
        const unsigned slices = (unsigned)((2 * num_sms() + 15) / 16);
        prof_begin(st, STAGE_OUT_SORT);
        cudaMemsetAsync(rank, 0, SMALL_SORT * sizeof(uint32_t), st);
        CR_NOTE_LAUNCH();
        k_out_rank<<<dim3(SMALL_SORT / (RK_T * RK_R), slices), RK_T, 0, st>>>(pairs_out, pair_count, capacity, rank,
                                                                            tmp);
        CR_NOTE_LAUNCH();
        k_out_place<<<SMALL_SORT / 256, 256, 0, st>>>(tmp, pair_count, capacity, rank, pairs_out, locbits);
        prof_end(st, STAGE_OUT_SORT, 64.0 * SMALL_SORT);
    }
    return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
    };
    if (!P.any_mid && P.graphs) {
        GraphKey key;
        key.add(0);  // forward
        key.addp(imgs);
        key.add((uint64_t)P.vtot);
        key.add(shapes_hash(P.segs));
        key.add((uint64_t)maxdim);
        key.add(flags);
        key.addp(pairs_out);
        key.add((uint64_t)capacity);
        key.addp(pair_offsets);
        key.addp(ws);
        key.add((uint64_t)ws_bytes);
        key.addp(st);
        key.add((uint64_t)current_device());
        key.add(prof_active());
        key.add(prof_mask());
        key.add(P.serial_uf);
        key.add(tune_epoch());
        rc = run_graphed(key, phase1, st);
    } else {
        rc = phase1(st);
    }
    if (rc) return rc;

    // ---- count, status ----
    int hstatus[16] = {0};
    unsigned long long ufc[CR_CNT_SLOTS];
    cudaMemcpyAsync(ufc, cnt, CR_CNT_SLOTS * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hc, pair_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hstatus, status, 16 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return CR_ERR_CUDA;
    if (hstatus[0]) {
        g_detail = hstatus[8];
        return hstatus[0];
    }
    // algorithmic bytes of the union-find rounds, per round and live edge
    // 104 B (phase B: the edge, both ends' min edge and age key; phase D: the
    // edge, both ends' root, the kept edge and both min-edge updates), per
    // group and round 12 B (min-edge reset, hook read); counters of both runs
    for (int base : {CNT_H0, CNT_DUAL}) {
        double e = (double)ufc[base + 3], r = (double)ufc[base + 6], g = (double)ufc[base + 0];
        prof_add_bytes(STAGE_UF_ROUND, 104.0 * e + 12.0 * g * r);
    }
    int64_t np = (int64_t)hc[0];
    *n_pairs = np;
    if (np > capacity) return CR_ERR_CAPACITY;

    // ---- canonical order ----
    {
        Carver R(region, region_cap);
        uint64_t *k0 = R.take<uint64_t>(np + 1), *k1 = R.take<uint64_t>(np + 1);
        uint32_t *v0 = R.take<uint32_t>(np + 1), *v1 = R.take<uint32_t>(np + 1);
        cr_pair *tmp = R.take<cr_pair>(np + 1);
        size_t rt = radix_temp_bytes(np + 1);
        void *rtemp = R.take<char>(rt);
        uint32_t *segc = R.take<uint32_t>(n + 1);
        uint32_t *part = R.take<uint32_t>(scan_temp_bytes(n + 1) / 4 + 1);
        if (!R.ok) { g_detail = SITE_OUT_CARVE; return CR_ERR_WORKSPACE; }
        const bool small = rank_sort && np <= SMALL_SORT;  // already sorted on the device
        if (small) {
        } else if (np > 0) {
            prof_begin(st, STAGE_OUT_SORT);
            if (pair_offsets) cudaMemsetAsync(segc, 0, (n + 1) * sizeof(uint32_t), st);
            CR_NOTE_LAUNCH();
            k_out_keys<<<nbk(np), 256, 0, st>>>(pairs_out, np, k0, v0, pair_offsets ? segc : nullptr);
            if (radix_sort_u64(k0, v0, k1, v1, np, 0, 64, rtemp, rt, st) != cudaSuccess) return CR_ERR_CUDA;
            CR_NOTE_LAUNCH();
            k_out_rekey<<<nbk(np), 256, 0, st>>>(pairs_out, np, v0, k0, 0);
            if (radix_sort_u64(k0, v0, k1, v1, np, 0, 2, rtemp, rt, st) != cudaSuccess) return CR_ERR_CUDA;
            if (n > 1) {
                CR_NOTE_LAUNCH();
                k_out_rekey<<<nbk(np), 256, 0, st>>>(pairs_out, np, v0, k0, 1);
                if (radix_sort_u64(k0, v0, k1, v1, np, 0, P.nseg_bits, rtemp, rt, st) != cudaSuccess)
                    return CR_ERR_CUDA;
            }
            cudaMemcpyAsync(tmp, pairs_out, (size_t)np * sizeof(cr_pair), cudaMemcpyDeviceToDevice, st);
            CR_NOTE_LAUNCH();
            k_out_gather<<<nbk(np), 256, 0, st>>>(tmp, np, v0, pairs_out, locbits);
            prof_end(st, STAGE_OUT_SORT, 3.0 * 24.0 * np + 64.0 * np);
        }
        if (pair_offsets) {
            if (np == 0) cudaMemsetAsync(segc, 0, (n + 1) * sizeof(uint32_t), st);
            if (exclusive_scan_u32(segc, n, part, st) != cudaSuccess) return CR_ERR_CUDA;
            CR_NOTE_LAUNCH();
            k_out_offsets<<<nbk(n + 1), 256, 0, st>>>(segc, n, np, pair_offsets);
        }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return CR_ERR_CUDA;
    prof_flush();
    return CR_OK;
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t argmax_vertex(const float *img, const Seg &S, int dim, uint32_t L) {
    int c[3];
    c[0] = (int)(L % (uint32_t)S.nx);
    uint32_t r = L / (uint32_t)S.nx;
    c[1] = (int)(r % (uint32_t)S.ny);
    r /= (uint32_t)S.ny;
    c[2] = (int)(r % (uint32_t)S.nz);
    int m = (int)(r / (uint32_t)S.nz);
    int span = 0;  // bits x=1, y=2, z=4
    if (dim == 1) span = 1 << m;
    else if (dim == 2) span = m == 0 ? 3 : (m == 1 ? 5 : 6);
    else if (dim == 3) span = 7;
    uint64_t best = 0;
    int64_t bv = -1;
    for (int dz = 0; dz <= ((span >> 2) & 1); dz++)
        for (int dy = 0; dy <= ((span >> 1) & 1); dy++)
            for (int dx = 0; dx <= (span & 1); dx++) {
                int64_t lv = ((int64_t)(c[2] + dz) * S.ny + (c[1] + dy)) * S.nx + (c[0] + dx);
                uint64_t k = make_key(ord32(img[S.voff + lv]), (uint32_t)lv);
                if (bv < 0 || k > best) { best = k; bv = S.voff + lv; }
            }
    return bv;
}

__global__ void k_bw_contrib(const float *img, const Seg *segs, int nseg, const cr_pair *pairs, int64_t np,
                             const int64_t *pair_offsets, const float *gb, const float *gd, uint64_t *keys,
                             uint32_t *vals) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    int si = 0;
    if (pair_offsets && nseg > 1) {
        int lo = 0, hi = nseg - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (pair_offsets[mid] <= k) lo = mid; else hi = mid - 1;
        }
        si = lo;
    }
    const Seg S = segs[si];
    cr_pair p = pairs[k];
    int64_t vb = argmax_vertex(img, S, p.dim, (uint32_t)p.birth_cell);
    keys[2 * k] = ((uint64_t)vb << 32) | (uint64_t)(2 * k);
    vals[2 * k] = __float_as_uint(gb[k]);
    if (p.death_cell >= 0) {
        int64_t vd = argmax_vertex(img, S, p.dim + 1, (uint32_t)p.death_cell);
        keys[2 * k + 1] = ((uint64_t)vd << 32) | (uint64_t)(2 * k + 1);
        vals[2 * k + 1] = __float_as_uint(gd[k]);
    } else {
        keys[2 * k + 1] = ~0ull;
        vals[2 * k + 1] = 0;
    }
}

__global__ void k_bw_sum(const uint64_t *keys, const uint32_t *vals, int64_t nc, float *grad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    uint64_t k = keys[i];
    if (k == ~0ull) return;
    uint32_t pix = (uint32_t)(k >> 32);
    if (i > 0 && (uint32_t)(keys[i - 1] >> 32) == pix && keys[i - 1] != ~0ull) return;
    double s = 0.0;
    for (int64_t j = i; j < nc; j++) {
        uint64_t kj = keys[j];
        if (kj == ~0ull || (uint32_t)(kj >> 32) != pix) break;
        s += (double)__uint_as_float(vals[j]);
    }
    grad[pix] = (float)s;
}

static size_t backward_bytes(int64_t np, int n) {
    int64_t nc = 2 * np + 1;
    return al((size_t)n * sizeof(Seg)) + 2 * al((size_t)nc * 8) + 2 * al((size_t)nc * 4) + al(radix_temp_bytes(nc)) +
           1024;
}

static int backward_impl(const float *imgs, HostPlan &P, const cr_pair *pairs, const int64_t *pair_offsets,
                         int64_t np, const float *gb, const float *gd, float *grad, void *ws, size_t ws_bytes,
                         cudaStream_t st) {
    const int n = (int)P.segs.size();
    if (np < 0 || (np > 0 && (!pairs || !gb || !gd)) || !grad) return CR_ERR_INVALID_ARG;
    if (np >= ((int64_t)1 << 30)) return CR_ERR_TOO_LARGE;
    if (!ws || ws_bytes < backward_bytes(np, n)) { g_detail = SITE_FIXED; return CR_ERR_WORKSPACE; }
    Carver C(ws, ws_bytes);
    Seg *segs = C.take<Seg>(n);
    int64_t nc = 2 * np;
    uint64_t *k0 = C.take<uint64_t>(nc + 1), *k1 = C.take<uint64_t>(nc + 1);
    uint32_t *v0 = C.take<uint32_t>(nc + 1), *v1 = C.take<uint32_t>(nc + 1);
    size_t rt = radix_temp_bytes(nc + 1);
    void *rtemp = C.take<char>(rt);
    if (!C.ok) { g_detail = SITE_FIXED; return CR_ERR_WORKSPACE; }
    cudaMemcpyAsync(segs, P.segs.data(), n * sizeof(Seg), cudaMemcpyHostToDevice, st);
    // a fixed launch sequence for these arguments: replayed as a CUDA graph
    auto launch_all = [&](cudaStream_t s) -> int {
        cudaMemsetAsync(grad, 0, (size_t)P.vtot * sizeof(float), s);
        if (np > 0) {
            prof_begin(s, STAGE_BW_CONTRIB);
            CR_NOTE_LAUNCH();
            k_bw_contrib<<<nbk(np), 256, 0, s>>>(imgs, segs, n, pairs, np, pair_offsets, gb, gd, k0, v0);
            int bits = 1;
            while (((int64_t)1 << bits) <= P.vtot) bits++;
            // the pixel sits in the high word; a stable sort on it keeps pair order inside a pixel
            if (radix_sort_u64(k0, v0, k1, v1, nc, 32, 32 + (bits > 32 ? 32 : bits + 1), rtemp, rt, s) !=
                cudaSuccess)
                return CR_ERR_CUDA;
            CR_NOTE_LAUNCH();
            k_bw_sum<<<nbk(nc), 256, 0, s>>>(k0, v0, nc, grad);
            prof_end(s, STAGE_BW_CONTRIB, 4.0 * P.vtot + 32.0 * np + 12.0 * nc);
        }
        return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
    };
    GraphKey key;
    key.add(1);  // backward
    key.addp(imgs);
    key.add((uint64_t)P.vtot);
    key.add(shapes_hash(P.segs));
    key.addp(pairs);
    key.addp(pair_offsets);
    key.add((uint64_t)np);
    key.addp(gb);
    key.addp(gd);
    key.addp(grad);
    key.addp(ws);
    key.add((uint64_t)ws_bytes);
    key.addp(st);
    key.add((uint64_t)current_device());
    key.add(prof_active());
    key.add(prof_mask());
    key.add(tune_epoch());
    const int rc = run_graphed(key, launch_all, st);
    if (rc) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CR_ERR_CUDA;
    prof_flush();
    return CR_OK;
}

}  // namespace cr

// ===========================================================================
// C ABI
// ===========================================================================
using namespace cr;

static int plan_single(int ndim, const int64_t *shape, int maxdim, uint32_t flags, HostPlan &P) {
    if (!shape || ndim < 1 || ndim > 3) return CR_ERR_INVALID_ARG;
    const int64_t *rows[1] = {shape};
    return plan_images(rows, 1, ndim, maxdim, flags, P);
}

static int plan_batched(const int32_t *shapes, int n_images, int ndim, int maxdim, uint32_t flags, HostPlan &P) {
    if (!shapes || n_images < 1 || ndim < 1 || ndim > 3) return CR_ERR_INVALID_ARG;
    if (n_images > (1 << 24) - 1) return CR_ERR_TOO_LARGE;
    std::vector<int64_t> buf((size_t)n_images * ndim);
    std::vector<const int64_t *> rows(n_images);
    for (int i = 0; i < n_images; i++) {
        for (int d = 0; d < ndim; d++) buf[(size_t)i * ndim + d] = shapes[(size_t)i * ndim + d];
        rows[i] = &buf[(size_t)i * ndim];
    }
    return plan_images(rows.data(), n_images, ndim, maxdim, flags, P);
}

namespace cr {
// single image with the two union-finds run one after the other, so that the
// workspace bound is that of one of them (used by the no-alloc entry point)
int workspace_size_serial(int ndim, const int64_t *shape, int maxdim, uint32_t flags, size_t *bytes) {
    if (!bytes) return CR_ERR_INVALID_ARG;
    HostPlan P;
    int rc = plan_single(ndim, shape, maxdim, flags, P);
    if (rc) return rc;
    P.serial_uf = true;
    *bytes = total_bytes(P, flags, true);
    return CR_OK;
}
int persistence_serial(const float *img, int ndim, const int64_t *shape, int maxdim, cr_pair *pairs_out,
                       int64_t capacity, int64_t *n_pairs, void *ws, size_t ws_bytes, cudaStream_t stream,
                       uint32_t flags) {
    if (!img || !n_pairs || capacity < 0 || (capacity > 0 && !pairs_out)) return CR_ERR_INVALID_ARG;
    HostPlan P;
    int rc = plan_single(ndim, shape, maxdim, flags, P);
    if (rc) return rc;
    P.serial_uf = true;
    // no graph capture here: instantiating a graph (and creating the capture
    // stream) may allocate, which the no-alloc entry point must not do
    P.graphs = false;
    return pipeline(img, P, maxdim, flags, pairs_out, capacity, nullptr, n_pairs, ws, ws_bytes, stream);
}
}  // namespace cr

extern "C" {

int cr_tune_set(int knob, int value) {
    if (knob < 0 || knob >= CR_TUNE_COUNT) return CR_ERR_INVALID_ARG;
    if (value < cr::g_tune_lo[knob] || value > cr::g_tune_hi[knob]) return CR_ERR_INVALID_ARG;
    if (cr::g_tune[knob].exchange(value) != value) cr::g_tune_epoch.fetch_add(1);
    return CR_OK;
}

int cr_debug_limits(int64_t barrier_polls, int64_t reduce_iters, int barrier_unsatisfiable) {
    if (barrier_polls < 0 || reduce_iters < 0 || barrier_unsatisfiable < 0 || barrier_unsatisfiable > 1)
        return CR_ERR_INVALID_ARG;
    cr::g_dbg_polls.store(barrier_polls ? (long long)barrier_polls : cr::DEFAULT_BARRIER_POLLS);
    cr::g_dbg_iters.store(reduce_iters ? (long long)reduce_iters : cr::DEFAULT_REDUCE_ITERS);
    cr::g_dbg_extra.store((unsigned int)barrier_unsatisfiable);
    cr::g_tune_epoch.fetch_add(1);  // launch sequences cached as graphs hold the old limits
    return CR_OK;
}

int cr_tune_get(int knob, int *value) {
    if (knob < 0 || knob >= CR_TUNE_COUNT || !value) return CR_ERR_INVALID_ARG;
    *value = cr::tune_value(knob);
    return CR_OK;
}


int cr_workspace_size(int ndim, const int64_t *shape, int maxdim, uint32_t flags, size_t *bytes) {
    if (!bytes) return CR_ERR_INVALID_ARG;
    HostPlan P;
    int rc = plan_single(ndim, shape, maxdim, flags, P);
    if (rc) return rc;
    *bytes = total_bytes(P, flags, true);
    return CR_OK;
}

int cr_workspace_size_typical(int ndim, const int64_t *shape, int maxdim, uint32_t flags, size_t *bytes) {
    if (!bytes) return CR_ERR_INVALID_ARG;
    HostPlan P;
    int rc = plan_single(ndim, shape, maxdim, flags, P);
    if (rc) return rc;
    *bytes = total_bytes(P, flags, false);
    return CR_OK;
}

int cr_workspace_size_batched(const int32_t *shapes, int n_images, int ndim, int maxdim, uint32_t flags,
                              size_t *bytes) {
    if (!bytes) return CR_ERR_INVALID_ARG;
    HostPlan P;
    int rc = plan_batched(shapes, n_images, ndim, maxdim, flags, P);
    if (rc) return rc;
    *bytes = total_bytes(P, flags, true);
    return CR_OK;
}

int cr_workspace_size_batched_typical(const int32_t *shapes, int n_images, int ndim, int maxdim, uint32_t flags,
                                      size_t *bytes) {
    if (!bytes) return CR_ERR_INVALID_ARG;
    HostPlan P;
    int rc = plan_batched(shapes, n_images, ndim, maxdim, flags, P);
    if (rc) return rc;
    *bytes = total_bytes(P, flags, false);
    return CR_OK;
}

int cr_persistence(const float *img, int ndim, const int64_t *shape, int maxdim, cr_pair *pairs_out,
                   int64_t capacity, int64_t *n_pairs, void *ws, size_t ws_bytes, cr_stream_t stream,
                   uint32_t flags) {
    if (!img || !n_pairs || capacity < 0 || (capacity > 0 && !pairs_out)) return CR_ERR_INVALID_ARG;
    HostPlan P;
    int rc = plan_single(ndim, shape, maxdim, flags, P);
    if (rc) return rc;
    rc = pipeline(img, P, maxdim, flags, pairs_out, capacity, nullptr, n_pairs, ws, ws_bytes, (cudaStream_t)stream);
    if (rc == CR_ERR_CUDA) return rc;
    return rc;
}

int cr_persistence_batched(const float *imgs, const int64_t *img_offsets, const int32_t *shapes, int n_images,
                           int ndim, int maxdim, cr_pair *pairs_out, int64_t capacity, int64_t *pair_offsets,
                           int64_t *n_pairs, void *ws, size_t ws_bytes, cr_stream_t stream, uint32_t flags) {
    if (!imgs || !img_offsets || !n_pairs || !pair_offsets || capacity < 0 || (capacity > 0 && !pairs_out))
        return CR_ERR_INVALID_ARG;
    HostPlan P;
    int rc = plan_batched(shapes, n_images, ndim, maxdim, flags, P);
    if (rc) return rc;
    for (int i = 0; i < n_images; i++)
        if (img_offsets[i] != P.segs[i].voff) return CR_ERR_INVALID_ARG;
    if (img_offsets[n_images] != P.vtot) return CR_ERR_INVALID_ARG;
    return pipeline(imgs, P, maxdim, flags, pairs_out, capacity, pair_offsets, n_pairs, ws, ws_bytes,
                    (cudaStream_t)stream);
}

int cr_backward_workspace_size(int64_t n_pairs, int n_images, size_t *bytes) {
    if (!bytes || n_pairs < 0 || n_images < 1) return CR_ERR_INVALID_ARG;
    *bytes = backward_bytes(n_pairs, n_images);
    return CR_OK;
}

int cr_backward(const float *img, int ndim, const int64_t *shape, const cr_pair *pairs, int64_t n_pairs,
                const float *grad_birth, const float *grad_death, float *grad_img, void *ws, size_t ws_bytes,
                cr_stream_t stream) {
    if (!img) return CR_ERR_INVALID_ARG;
    HostPlan P;
    int rc = plan_single(ndim, shape, 0, 0, P);
    if (rc) return rc;
    return backward_impl(img, P, pairs, nullptr, n_pairs, grad_birth, grad_death, grad_img, ws, ws_bytes,
                         (cudaStream_t)stream);
}

int cr_backward_batched(const float *imgs, const int64_t *img_offsets, const int32_t *shapes, int n_images,
                        int ndim, const cr_pair *pairs, const int64_t *pair_offsets, int64_t n_pairs,
                        const float *grad_birth, const float *grad_death, float *grad_imgs, void *ws,
                        size_t ws_bytes, cr_stream_t stream) {
    if (!imgs || !img_offsets || !pair_offsets) return CR_ERR_INVALID_ARG;
    HostPlan P;
    int rc = plan_batched(shapes, n_images, ndim, 0, 0, P);
    if (rc) return rc;
    for (int i = 0; i < n_images; i++)
        if (img_offsets[i] != P.segs[i].voff) return CR_ERR_INVALID_ARG;
    if (img_offsets[n_images] != P.vtot) return CR_ERR_INVALID_ARG;
    return backward_impl(imgs, P, pairs, pair_offsets, n_pairs, grad_birth, grad_death, grad_imgs, ws, ws_bytes,
                         (cudaStream_t)stream);
}

int cr_cell_location(int64_t L, int dim, int ndim, const int64_t *shape, int *m, int64_t *x, int64_t *y,
                     int64_t *z) {
    if (!shape || !m || !x || !y || !z || ndim < 1 || ndim > 3 || dim < 0 || dim > 3 || L < 0)
        return CR_ERR_INVALID_ARG;
    int64_t nz = 1, ny = 1, nx = 1;
    if (ndim == 1) nx = shape[0];
    else if (ndim == 2) { ny = shape[0]; nx = shape[1]; }
    else { nz = shape[0]; ny = shape[1]; nx = shape[2]; }
    if (nx < 1 || ny < 1 || nz < 1) return CR_ERR_INVALID_ARG;
    *x = L % nx;
    int64_t r = L / nx;
    *y = r % ny;
    r /= ny;
    *z = r % nz;
    *m = (int)(r / nz);
    int maxm = (dim == 1 || dim == 2) ? 2 : 0;
    if (*m > maxm) return CR_ERR_INVALID_ARG;
    return CR_OK;
}

int cr_h1_last_stats(int64_t *out, int n) {
    if (!out || n < 1) return CR_ERR_INVALID_ARG;
    return cr::h1_stats(out, n);
}

const char *cr_last_error_detail(void) {
    switch (cr::g_detail) {
    case cr::SITE_NONE: return "";
    case cr::SITE_GROUPS: return "union-find groups";
    case cr::SITE_EDGES: return "cross-basin edge list";
    case cr::SITE_COLUMNS: return "residual column list";
    case cr::SITE_ARENA: return "column arena";
    case cr::SITE_POOL: return "long-column pool";
    case cr::SITE_UF_CARVE: return "union-find region";
    case cr::SITE_H1_CARVE: return "reduction region";
    case cr::SITE_OUT_CARVE: return "output sort region";
    case cr::SITE_FIXED: return "fixed part of the workspace";
    case cr::SITE_INJECTED: return "injected by CR_FAULT=workspace";
    default: return "unknown";
    }
}

const char *cr_error_string(int code) {
    switch (code) {
    case CR_OK: return "success";
    case CR_ERR_INVALID_ARG: return "invalid argument";
    case CR_ERR_NAN: return "NaN in input";
    case CR_ERR_TOO_LARGE: return "input too large for 32-bit cell indices";
    case CR_ERR_CAPACITY: return "pairs_out capacity too small (n_pairs holds the count needed)";
    case CR_ERR_WORKSPACE: return "workspace too small";
    case CR_ERR_CUDA: return "CUDA runtime error";
    case CR_ERR_TIMEOUT: return "a bounded device-side wait or iteration limit expired";
    case CR_ERR_INTERNAL: return "internal consistency check failed";
    default: return "unknown error code";
    }
}

}  // extern "C"
