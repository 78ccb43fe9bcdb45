// cr_images.cu -- the localised-feature images of the paper's Sec. 4: per
// voxel, the largest lifetime (or a (birth, lifetime) histogram) of the pairs
// located there.  One thread per pair scatters into a zero-filled output.
#include "cr_internal.cuh"
#include <cfloat>

namespace cr {

struct ImgGeom {
    int64_t nx, ny, nz, V;
    int nd;
};

// L-index of the cell a pair is located at: its birth cell, its death cell,
// or (location < 0) the one its CR_PAIR_LOC_DEATH bit names; an essential
// pair has no death cell and stays at its birth cell
__device__ __forceinline__ int64_t located_cell(const cr_pair &p, int location) {
    const bool death = location < 0 ? (p.flags & CR_PAIR_LOC_DEATH) != 0 : location == 1;
    return death && p.death_cell >= 0 ? p.death_cell : p.birth_cell;
}

// anchor voxel of the located cell, -1 for a pair without a finite lifetime
__device__ __forceinline__ int64_t located_voxel(const cr_pair &p, const ImgGeom &G, int location) {
    if (!(p.death <= FLT_MAX)) return -1;  // infinite (or NaN) death: no finite lifetime
    if (p.dim < 0 || p.dim >= G.nd) return -1;
    const int64_t L = located_cell(p, location);
    if (L < 0) return -1;
    const int64_t x = L % G.nx, y = (L / G.nx) % G.ny, z = (L / (G.nx * G.ny)) % G.nz;
    return (z * G.ny + y) * G.nx + x;
}

// one row (dim, birth, death, x, y, z) per pair
__global__ void k_pair_table(const cr_pair *__restrict__ pairs, int64_t n, ImgGeom G, int location,
                             double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const cr_pair p = pairs[i];
    const int64_t L = located_cell(p, location);
    double *r = out + 6 * i;
    r[0] = (double)p.dim;
    r[1] = (double)p.birth;
    r[2] = (double)p.death;
    r[3] = (double)(L % G.nx);
    r[4] = (double)((L / G.nx) % G.ny);
    r[5] = (double)((L / (G.nx * G.ny)) % G.nz);
}

__global__ void k_lifetime_image(const cr_pair *__restrict__ pairs, int64_t n, ImgGeom G, int location,
                                 float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const cr_pair p = pairs[i];
    const int64_t v = located_voxel(p, G, location);
    if (v < 0) return;
    const float life = p.death - p.birth;
    // non-negative floats order like their bit patterns; the output starts at +0
    if (life > 0.f) atomicMax((int *)&out[(int64_t)p.dim * G.V + v], __float_as_int(life));
}

__global__ void k_histogram_image(const cr_pair *__restrict__ pairs, int64_t n, ImgGeom G, int location, int nb,
                                  double b_lo, double b_hi, int nl, double l_hi, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const cr_pair p = pairs[i];
    const int64_t v = located_voxel(p, G, location);
    if (v < 0) return;
    const double b = (double)p.birth, d = (double)p.death;
    const double fi = floor((b - b_lo) / (b_hi - b_lo) * (double)nb);
    const double fj = floor((d - b) / l_hi * (double)nl);
    if (!(fi >= 0.0 && fi < (double)nb && fj >= 0.0 && fj < (double)nl)) return;
    const int64_t ch = ((int64_t)p.dim * nb + (int64_t)fi) * nl + (int64_t)fj;
    atomicAdd(&out[ch * G.V + v], 1.0f);
}

static int image_geom(int ndim, const int64_t *shape, ImgGeom &G) {
    if (ndim < 1 || ndim > 3 || !shape) return CR_ERR_INVALID_ARG;
    int64_t e[3] = {1, 1, 1};
    for (int d = 0; d < ndim; d++) {
        if (shape[d] < 1) return CR_ERR_INVALID_ARG;
        e[3 - ndim + d] = shape[d];
    }
    G.nz = e[0];
    G.ny = e[1];
    G.nx = e[2];
    G.V = e[0] * e[1] * e[2];
    G.nd = ndim;
    return CR_OK;
}

}  // namespace cr

extern "C" {

int cr_lifetime_image(const cr_pair *pairs, int64_t n_pairs, int ndim, const int64_t *shape, int location,
                      float *out, cr_stream_t stream) {
    cr::ImgGeom G;
    int rc = cr::image_geom(ndim, shape, G);
    if (rc) return rc;
    if (n_pairs < 0 || (n_pairs > 0 && !pairs) || !out || location < -1 || location > 1) return CR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cr::prof_begin(st, cr::STAGE_IMAGES);
    cudaMemsetAsync(out, 0, (size_t)G.nd * (size_t)G.V * sizeof(float), st);
    if (n_pairs > 0) {
        CR_NOTE_LAUNCH();
        cr::k_lifetime_image<<<(unsigned)((n_pairs + 255) / 256), 256, 0, st>>>(pairs, n_pairs, G, location, out);
    }
    cr::prof_end(st, cr::STAGE_IMAGES, 4.0 * G.nd * G.V + 32.0 * n_pairs);
    return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

int cr_persistent_histogram_image(const cr_pair *pairs, int64_t n_pairs, int ndim, const int64_t *shape,
                                  int location, int nb, double b_lo, double b_hi, int nl, double l_hi, float *out,
                                  cr_stream_t stream) {
    cr::ImgGeom G;
    int rc = cr::image_geom(ndim, shape, G);
    if (rc) return rc;
    if (n_pairs < 0 || (n_pairs > 0 && !pairs) || !out || location < -1 || location > 1 || nb < 1 || nl < 1 ||
        !(b_hi > b_lo) || !(l_hi > 0.0))
        return CR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cr::prof_begin(st, cr::STAGE_IMAGES);
    cudaMemsetAsync(out, 0, (size_t)G.nd * nb * nl * (size_t)G.V * sizeof(float), st);
    if (n_pairs > 0) {
        CR_NOTE_LAUNCH();
        cr::k_histogram_image<<<(unsigned)((n_pairs + 255) / 256), 256, 0, st>>>(pairs, n_pairs, G, location, nb,
                                                                                 b_lo, b_hi, nl, l_hi, out);
    }
    cr::prof_end(st, cr::STAGE_IMAGES, 4.0 * G.nd * nb * nl * G.V + 32.0 * n_pairs);
    return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

int cr_pair_table(const cr_pair *pairs, int64_t n_pairs, int ndim, const int64_t *shape, int location,
                  double *out, cr_stream_t stream) {
    cr::ImgGeom G;
    int rc = cr::image_geom(ndim, shape, G);
    if (rc) return rc;
    if (n_pairs < 0 || (n_pairs > 0 && (!pairs || !out)) || location < -1 || location > 1) return CR_ERR_INVALID_ARG;
    if (n_pairs == 0) return CR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    CR_NOTE_LAUNCH();
    cr::k_pair_table<<<(unsigned)((n_pairs + 255) / 256), 256, 0, st>>>(pairs, n_pairs, G, location, out);
    return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

}  // extern "C"
