/*
 * cr.h -- C ABI of libcr.so: persistent homology of cubical images on one GPU.
 *
 * The library computes Z/2 persistent homology of the sublevel filtration of a
 * 1D, 2D or 3D float32 array under the V-construction (Kaji, Sudo, Ahara,
 * "Cubical Ripser", Sec. 2): every pixel/voxel is a 0-cube with its value, and
 * every higher cube takes the maximum of the values of its vertices.  Pairs
 * are the persistence pairs of one fixed total order on the cubes:
 *
 *   ascending value, then ascending dimension, then descending
 *   L = ((m*Nz + z)*Ny + y)*Nx + x,
 *
 * which is the reverse of the paper's (-birth, m, z, y, x) cohomology order
 * (Sec. 2).  Cube types m: 1-cubes m=0,1,2 step in x, y, z; 2-cubes m=0,1,2
 * span {x,y}, {x,z}, {y,z}; 0- and 3-cubes have m=0.  Arrays are C-order with
 * x the fastest index (Sec. 2, Fig. 1: the cell "to the right" is x+1); a 2D
 * array is (Ny, Nx), a 1D array (Nx).
 *
 * Conventions shared by every entry point:
 *   - All pointers named *_dev, and img/imgs/pairs_out/grad_* are DEVICE
 *     pointers owned by the caller; shape arrays and n_pairs are HOST memory.
 *   - ws/ws_bytes: caller-owned device workspace; size it with the matching
 *     *_workspace_size call.  The library allocates no device memory.
 *   - Work is enqueued on `stream`; the call returns after the stream reaches
 *     the point where the host must read a count (it synchronises `stream`).
 *   - Return value: CR_OK or a negative CR_ERR_* code; the library never
 *     aborts the process.  After CR_ERR_CUDA the CUDA error is also returned
 *     by cudaGetLastError on the calling thread.
 *   - -0.0 is treated as +0.0; +inf is an ordinary (largest) value; NaN
 *     anywhere is rejected with CR_ERR_NAN.
 */
#ifndef CR_H_
#define CR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cr_stream_t; /* same object as cudaStream_t */

/* ---- error codes ---- */
#define CR_OK 0
#define CR_ERR_INVALID_ARG (-1) /* bad ndim/shape/pointer/flag */
#define CR_ERR_NAN (-2)         /* NaN in the input */
#define CR_ERR_TOO_LARGE (-3)   /* 3 * voxels of one image >= 2^32, or all images >= 2^31 voxels */
#define CR_ERR_CAPACITY (-4)    /* pairs_out too small; *n_pairs = pairs needed */
#define CR_ERR_WORKSPACE (-5)   /* ws_bytes too small, or a data-dependent buffer overflowed */
#define CR_ERR_CUDA (-6)        /* a CUDA runtime call failed */
#define CR_ERR_TIMEOUT (-7)     /* a bounded device-side wait or iteration cap expired */
#define CR_ERR_INTERNAL (-8)    /* an internal consistency check failed */

/* ---- flags ---- */
#define CR_KEEP_ZERO 1u   /* also emit pairs with death == birth */
#define CR_TOPDIM_ONLY 2u /* only the (ndim-1)-dimensional pairs, by duality (Sec. 2, Rem. 2.1) */
/* Report the death cell as each pair's location instead of the birth cell
 * (the location option of Sec. 4, Ex. 4.1 / Ex. 4.6; the paper notes the
 * representative is one choice among several).  Pairs keep both cells; the
 * flag sets CR_PAIR_LOC_DEATH in every pair's flags, and the location-based
 * calls (cr_pair_table, the localised images) called with
 * location = CR_LOC_FROM_PAIRS follow it.  An essential pair has no death
 * cell: its location stays its birth cell. */
#define CR_LOC_DEATH 4u

/* A persistence pair [birth, death) of dimension `dim` (Sec. 1: a d-cycle
 * born at `birth`, killed at `death`).  birth_cell is the L index of the
 * dim-cube that creates the class, death_cell the L index of the
 * (dim+1)-cube that kills it (its location is the paper's "location of the
 * cell giving birth", Sec. 4, Ex. 4.6).  Essential classes: death = +inf,
 * death_cell = -1.  32 bytes. */
typedef struct {
    int32_t dim;
    float birth;
    float death;
    uint32_t flags; /* bit 0: essential */
    int64_t birth_cell;
    int64_t death_cell;
} cr_pair;

#define CR_PAIR_ESSENTIAL 1u
#define CR_PAIR_LOC_DEATH 2u /* set by the CR_LOC_DEATH flag: the pair is located at its death cell */

/* `location` argument of the location-based calls: the birth cell (0), the
 * death cell (1), or what each pair records (CR_PAIR_LOC_DEATH). */
#define CR_LOC_BIRTH_CELL 0
#define CR_LOC_DEATH_CELL 1
#define CR_LOC_FROM_PAIRS (-1)

/* Device workspace (bytes) for cr_persistence on one image of this shape,
 * maxdim and flags.  Host-only; no GPU work.
 *   cr_workspace_size          a bound that the union-find stages, the
 *                              residual-column lists and the output sort
 *                              cannot exceed for any input of this shape;
 *   cr_workspace_size_typical  a smaller size that suffices for smooth or
 *                              noisy fields; an input that needs more makes
 *                              the call return CR_ERR_WORKSPACE (nothing else
 *                              is wrong; retry with the bound).
 * The column arena of the 3D reduction is data-dependent: it takes what is
 * left of the workspace and reports CR_ERR_WORKSPACE if that is exceeded. */
int cr_workspace_size(int ndim, const int64_t *shape, int maxdim, uint32_t flags, size_t *bytes);
int cr_workspace_size_typical(int ndim, const int64_t *shape, int maxdim, uint32_t flags, size_t *bytes);

/*
 * Persistent homology of one image (Sec. 2; Sec. 4, Ex. 4.1 `computePH`).
 *   img       device float32[prod(shape)], C-order.
 *   ndim      1, 2 or 3; shape[ndim] host array of extents >= 1.
 *   maxdim    pairs of dimension 0..maxdim are computed (Ex. 4.1 `maxdim`);
 *             maxdim >= ndim-1 includes the top dimension via duality.
 *   pairs_out device cr_pair[capacity]; on success sorted by
 *             (dim, birth, birth_cell).
 *   n_pairs   host; number of pairs written (or needed, on CR_ERR_CAPACITY).
 *   flags     CR_KEEP_ZERO | CR_TOPDIM_ONLY | CR_LOC_DEATH.
 */
int cr_persistence(const float *img, int ndim, const int64_t *shape, int maxdim, cr_pair *pairs_out,
                   int64_t capacity, int64_t *n_pairs, void *ws, size_t ws_bytes, cr_stream_t stream,
                   uint32_t flags);

/* Pairs of a float64 image: as cr_pair, with double birth and death.
 * 40 bytes. */
typedef struct {
    int32_t dim;
    uint32_t flags; /* bit 0: essential */
    double birth;
    double death;
    int64_t birth_cell;
    int64_t death_cell;
} cr_pair64;

/* Workspace for cr_persistence_f64: the float64 extras (about 48 bytes per
 * voxel, plus 32 bytes per pair of capacity) and the float32 path's
 * workspace (the bound if typical == 0, the typical size otherwise).
 * Host-only. */
int cr_workspace_size_f64(int ndim, const int64_t *shape, int maxdim, uint32_t flags, int64_t capacity,
                          int typical, size_t *bytes);

/*
 * Persistent homology of one float64 image, the precision of the paper's
 * timing study (its datasets were converted to double, Sec. 3).  The
 * filtration depends on the values only through their order (cells enter by
 * value, ties by the fixed index order, Sec. 2), so the call ranks the
 * distinct values on the device (-0.0 = +0.0; one 64-bit radix sort), runs the
 * float32 path on the image of ranks and maps each pair's values back: the
 * result equals the persistence of the float64 image.
 *   img       device float64[prod(shape)], C-order; fewer than 2^31 voxels.
 *   pairs_out device cr_pair64[capacity], sorted by (dim, birth, birth_cell).
 *   ws        device, 256-byte aligned, cr_workspace_size_f64 bytes for this
 *             capacity.
 * Other arguments, flags and errors as cr_persistence; a NaN gives
 * CR_ERR_NAN before the float32 path runs.
 */
int cr_persistence_f64(const double *img, int ndim, const int64_t *shape, int maxdim, cr_pair64 *pairs_out,
                       int64_t capacity, int64_t *n_pairs, void *ws, size_t ws_bytes, cr_stream_t stream,
                       uint32_t flags);

/* Workspace for cr_persistence_batched over these images (shapes: host
 * int32[n_images * ndim], each row the extents of one image). */
int cr_workspace_size_batched(const int32_t *shapes, int n_images, int ndim, int maxdim, uint32_t flags,
                              size_t *bytes);
int cr_workspace_size_batched_typical(const int32_t *shapes, int n_images, int ndim, int maxdim, uint32_t flags,
                                      size_t *bytes);

/*
 * Many images of possibly different shapes in one pass: the persistence of
 * each image, independently, with every stage run once over all images.
 *   imgs         device float32, images packed back to back.
 *   img_offsets  host int64[n_images+1]; image i is imgs[img_offsets[i] ..
 *                img_offsets[i+1]); must equal the running product of shapes.
 *   shapes       host int32[n_images * ndim].
 *   pairs_out    device cr_pair[capacity], grouped by image, each group
 *                sorted as in cr_persistence.
 *   pair_offsets device int64[n_images+1]; pairs of image i are
 *                pairs_out[pair_offsets[i] .. pair_offsets[i+1]).
 *   n_pairs      host; total pairs.
 */
int cr_persistence_batched(const float *imgs, const int64_t *img_offsets, const int32_t *shapes, int n_images,
                           int ndim, int maxdim, cr_pair *pairs_out, int64_t capacity, int64_t *pair_offsets,
                           int64_t *n_pairs, void *ws, size_t ws_bytes, cr_stream_t stream, uint32_t flags);

/* Workspace for cr_backward (n_images = 1) / cr_backward_batched with
 * n_pairs pairs.  Host-only. */
int cr_backward_workspace_size(int64_t n_pairs, int n_images, size_t *bytes);

/*
 * Gradient of a loss L(diagram) with respect to the image.  A pair's birth
 * (death) is the value of its birth (death) cube, which is the value of the
 * cube's latest vertex in the filtration order (largest value; among equal
 * values the smallest linear index).  dL/dbirth and dL/ddeath are therefore
 * added to the image gradient at that vertex (V-construction, Sec. 2).
 * Essential deaths contribute nothing.  Contributions to one pixel are summed
 * in double precision in a fixed order (by pair index), then rounded once to
 * float32, so the result is deterministic.
 *   pairs       device cr_pair[n_pairs] as returned by cr_persistence.
 *   grad_birth  device float32[n_pairs]; grad_death device float32[n_pairs].
 *   grad_img    device float32[prod(shape)], overwritten (zeroed by callee).
 */
int cr_backward(const float *img, int ndim, const int64_t *shape, const cr_pair *pairs, int64_t n_pairs,
                const float *grad_birth, const float *grad_death, float *grad_img, void *ws, size_t ws_bytes,
                cr_stream_t stream);

/* Batched gradient: pairs/pair_offsets as returned by
 * cr_persistence_batched (pair_offsets is a device array), img_offsets and
 * shapes as passed to it; grad_imgs is packed like imgs. */
int cr_backward_batched(const float *imgs, const int64_t *img_offsets, const int32_t *shapes, int n_images,
                        int ndim, const cr_pair *pairs, const int64_t *pair_offsets, int64_t n_pairs,
                        const float *grad_birth, const float *grad_death, float *grad_imgs, void *ws,
                        size_t ws_bytes, cr_stream_t stream);

/* Localised-feature images (Sec. 4, the example on localised features).
 * The location of a pair is the anchor voxel (x, y, z) of its birth cell
 * (location = CR_LOC_BIRTH_CELL), of its death cell (CR_LOC_DEATH_CELL), or
 * of the cell the pair records (CR_LOC_FROM_PAIRS: the death cell where
 * CR_PAIR_LOC_DEATH is set), i.e. the cell's L-index with the type dropped.
 * Essential pairs (infinite death) are left out.
 *
 * cr_lifetime_image: out[d * V + v], d < ndim, V = prod(shape), is the
 *   largest lifetime death - birth (float32 subtraction) of the pairs of
 *   dimension d located at voxel v, 0 where there is none: the lifetime
 *   channels of the paper's lifetime enhanced image (stacked with the image
 *   itself by the caller).
 * cr_persistent_histogram_image: out[((d * nb + i) * nl + j) * V + v] counts
 *   the pairs of dimension d located at v whose birth falls in bin
 *   i = floor((birth - b_lo) / (b_hi - b_lo) * nb) and whose lifetime falls in
 *   bin j = floor((death - birth) / l_hi * nl), both computed in double; pairs
 *   with i outside [0, nb) or j outside [0, nl) are not counted.
 *
 *   pairs   device cr_pair[n_pairs] of one image (as from cr_persistence)
 *   shape   host int64[ndim], the image's shape (C order)
 *   out     device float32, ndim * V (lifetime) or ndim * nb * nl * V
 *           (histogram) values; zero-filled by the call
 * Asynchronous on `stream`.  Errors: CR_ERR_INVALID_ARG (ndim not 1-3, an
 * extent < 1, location not 0/1, nb or nl < 1, b_hi <= b_lo, l_hi <= 0, a null
 * buffer that is needed), CR_ERR_CUDA. */
int cr_lifetime_image(const cr_pair *pairs, int64_t n_pairs, int ndim, const int64_t *shape, int location,
                      float *out, cr_stream_t stream);
int cr_persistent_histogram_image(const cr_pair *pairs, int64_t n_pairs, int ndim, const int64_t *shape,
                                  int location, int nb, double b_lo, double b_hi, int nl, double l_hi, float *out,
                                  cr_stream_t stream);

/* The pairs as the paper's table (Sec. 4, Ex. 4.1: computePH returns one
 * row (dim, birth, death, x, y, z) per pair, located at the birth cell or,
 * with the location option, the death cell).
 *   pairs     device cr_pair[n_pairs] of one image
 *   shape     host int64[ndim], the image's shape; (x, y, z) is the anchor of
 *             the located cube as cr_cell_location gives it (x the fastest
 *             array index; y = 0 in 1D, z = 0 in 1D/2D)
 *   location  CR_LOC_BIRTH_CELL, CR_LOC_DEATH_CELL or CR_LOC_FROM_PAIRS; an
 *             essential pair is always located at its birth cell
 *   out       device double[n_pairs * 6], row-major; essential deaths +inf
 * Asynchronous on `stream`.  Errors: CR_ERR_INVALID_ARG (ndim not 1-3, an
 * extent < 1, a bad location, a null buffer that is needed), CR_ERR_CUDA. */
int cr_pair_table(const cr_pair *pairs, int64_t n_pairs, int ndim, const int64_t *shape, int location,
                  double *out, cr_stream_t stream);

/* Anchor (x, y, z) and type m of the cube (dim, L) of an image of this shape
 * (the paper's cell tuple (x, y, z, m, d), Sec. 2).  Host-only. */
int cr_cell_location(int64_t L, int dim, int ndim, const int64_t *shape, int *m, int64_t *x, int64_t *y,
                     int64_t *z);

/*
 * cr_persistence_noalloc -- cr_persistence for callers that cannot allocate
 * device memory.  (The paper has no counterpart; this is a deployment
 * convenience.)  Some callers cannot call cudaMalloc: code running inside a
 * host framework's fixed device-memory pool (inference plugins, embedded
 * hosts) where an allocation would break the host's memory accounting or
 * synchronise the device at a forbidden point.  They still pass their input
 * and output buffers; the workspace is a file-scope static device array of
 * CR_NOALLOC_SCRATCH_BYTES, reserved when the library is loaded and held by
 * every GPU that loads it until the process exits.  The call itself makes no
 * cudaMalloc, cudaFree or other allocating call.
 *   - Serves 1D and 2D images (a 3D array is accepted only with a leading
 *     extent of 1) whose cr_workspace_size bound fits the array (about
 *     490,000 pixels, e.g. 512x512 with maxdim 1); larger inputs return
 *     CR_ERR_TOO_LARGE, volumes CR_ERR_INVALID_ARG, before any GPU work.
 *   - The first call on a device resolves the array's device address with
 *     cudaGetSymbolAddress while that device is current; make that first call
 *     before any stream capture.
 *   - All calls on a device share the one array, which keeps the contents of
 *     the last call; the call clears everything it relies on being zero.
 *     Calls that overlap on the GPU (other streams, other host threads) race
 *     on the array: serialise them.
 * Arguments and results are those of cr_persistence without ws/ws_bytes.
 */
#define CR_NOALLOC_SCRATCH_BYTES (64ull << 20)
int cr_persistence_noalloc(const float *img, int ndim, const int64_t *shape, int maxdim, cr_pair *pairs_out,
                           int64_t capacity, int64_t *n_pairs, cr_stream_t stream, uint32_t flags);

/* Diagnostics for benchmarks.  With profiling on, every stage of a call is
 * bracketed by CUDA events recorded on the caller's stream; totals per stage
 * are read with cr_profile_read (stage 0..17; name, total milliseconds,
 * number of timed launches, algorithmic bytes the stage must move).  Returns
 * CR_ERR_INVALID_ARG past the last stage.  cr_profile_select restricts the
 * events to the stages whose bit is set in stage_mask (bit s = stage s;
 * default all), so that one kernel can be timed inside an otherwise
 * unobserved run.  cr_launch_count is the number of kernels the library has
 * launched since it was loaded.  Host-only. */
int cr_profile_enable(int on);
int cr_profile_select(uint32_t stage_mask);
void cr_profile_reset(void);
int cr_profile_read(int stage, const char **name, double *total_ms, int64_t *count, double *bytes);
int64_t cr_launch_count(void);
/* Counters of the last 3D reduction on this process (out[0..n), n <= 25):
 * residual columns, loop iterations, apparent-column additions, column
 * additions, merged entries, pivot takeovers, lost races and stale reads,
 * long-column buffer growths, most iterations spent on one column in one
 * pass (the counts add up both passes of the reduction); then
 * (builds with CR_H1_TIMING only, zero otherwise) cycles spent in the
 * iterations of long column runs per phase: front refills, lookups, apparent
 * additions, cached additions, staged additions, inbox flushes, then lookahead
 * misses, iterations timed, whole-iteration cycles and pivot-table reads,
 * then timestamps.  Host-only. */
int cr_h1_last_stats(int64_t *out, int n);

/* Launch knobs, set by the autotuner (host-side, per process).  They change
 * how many blocks or warps a kernel is launched with, never what it computes:
 *   CR_TUNE_UF_ITEMS   work items per thread that the cooperative union-find
 *                      grids aim for: blocks = min(SMs, work / (items * 1024) + 1);
 *                      1..64, default 8.  A smaller value launches more blocks
 *                      for mid-size inputs: more parallel work, more blocks
 *                      arriving at every grid barrier.
 *   CR_TUNE_RED_WARPS  warps per SM launched for the deep pass of the
 *                      middle-dimension reduction of 3D images; 1..16,
 *                      default 16 (the workspace is sized for 16).
 *   CR_TUNE_RED_BUDGET steps a residual column may take in the wide pass of
 *                      that reduction (16 warps per SM, small buffers) before
 *                      it is published and set aside for the deep pass;
 *                      0..2^24, default 1024; 0 runs the deep pass alone.
 *                      Any budget gives the same pairs: the reduction reaches
 *                      the same pivots whatever the order of its additions.
 *   CR_TUNE_UF_COMPACT the union-find rounds compact their edge list while it
 *                      holds more than this many edges per launched thread,
 *                      then mark dead edges in place; 1..64, default 1.
 *   CR_TUNE_BATCH_THREADS  batches of 2D images (every extent >= 2): the
 *                      union-finds run in one persistent launch, each block
 *                      taking whole images from a queue ordered by size,
 *                      largest first, with 256 (1), 512 (2, default) or 1024
 *                      (3) threads per block; 0 runs them as grid-wide
 *                      kernels over all images at once instead.
 * cr_tune_set returns CR_ERR_INVALID_ARG for an unknown knob or a value out of
 * range (the knob keeps its value); cr_tune_get writes the current value to
 * *value.  A launch sequence cached as a CUDA graph is captured afresh after a
 * knob changes.  Host-only. */
#define CR_TUNE_UF_ITEMS 0
#define CR_TUNE_RED_WARPS 1
#define CR_TUNE_UF_COMPACT 2
#define CR_TUNE_BATCH_THREADS 3
#define CR_TUNE_RED_BUDGET 4
#define CR_TUNE_COUNT 5
int cr_tune_set(int knob, int value);
int cr_tune_get(int knob, int *value);

/* Limits of the bounded device-side waits, for tests of the error paths.
 * Every wait in the library gives up after a limit and makes the call return
 * CR_ERR_TIMEOUT (the status is read by the host; no kernel traps, and the
 * CUDA context stays usable).  This call lowers the limits so that a test can
 * make a wait run out:
 *   barrier_polls          polls of one grid-barrier wait of the union-find
 *                          kernels (0 = the default, 2^24);
 *   reduce_iters           iterations one column of the 3D middle-dimension
 *                          reduction may take in one pass (0 = the default,
 *                          2^24);
 *   barrier_unsatisfiable  1: the grid barriers wait for one block more than
 *                          the grid has (a flag that nothing sets), so every
 *                          barrier wait runs out after barrier_polls polls;
 *                          0: normal barriers.
 * Host-side and per process; launch sequences cached as CUDA graphs are
 * captured afresh.  Returns CR_ERR_INVALID_ARG for a negative limit or a flag
 * other than 0/1.
 *
 * Host-side fault injection: with CR_FAULT=<site> in the environment (read at
 * each call), cr_persistence, cr_persistence_batched, cr_persistence_f64 and
 * cr_persistence_noalloc fail as that fault would, leaving no GPU state
 * behind: "shape" -> CR_ERR_INVALID_ARG and "nan" -> CR_ERR_NAN before any
 * GPU work, "workspace" -> CR_ERR_WORKSPACE (cr_last_error_detail names the
 * injection) before any GPU work, "capacity" -> the call runs with no room
 * for pairs and returns CR_ERR_CAPACITY with *n_pairs = the pairs needed.
 * Any other value is ignored. */
int cr_debug_limits(int64_t barrier_polls, int64_t reduce_iters, int barrier_unsatisfiable);

/* Static description of an error code. */
const char *cr_error_string(int code);

/* After CR_ERR_WORKSPACE on this host thread: the name of the buffer that
 * was too small ("" if none).  Host-only. */
const char *cr_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* CR_H_ */
