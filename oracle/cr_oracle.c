/*
 * cr_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU computation of the persistent homology
 * (coefficients Z/2) of the weighted cubical complex of a 1D/2D/3D float32
 * or float64 array under the V-construction (values are held in double; a
 * float32 input is promoted exactly).  It exists so that the CUDA path can be
 * checked against something obviously correct; only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header or table with the CUDA library.
 *
 * What it computes, and where the paper fixes it (Kaji, Sudo, Ahara,
 * "Cubical Ripser", Sec. 2):
 *   - a cell is (x, y, z, m, d): location, type, dimension (Sec. 2, cell
 *     encoding).  1-cells of type m = 0, 1, 2 extend the anchor by one step
 *     in x, y, z.  2-cells of type 0, 1, 2 span {x,y}, {x,z}, {y,z}.  The
 *     paper's text for the type-2 1-cell names a diagonal; it is read here as
 *     the z-edge, the only reading consistent with 6-neighbour connectivity.
 *   - the value (birth-time) of a cell is the maximum of the values of the
 *     0-cells it contains (V-construction, Sec. 2).
 *   - cells of one dimension are ordered by (-value, m, z, y, x) in the
 *     paper's cohomology order; the filtration used here is its reverse:
 *     ascending value, then descending L = ((m*Nz + z)*Ny + y)*Nx + x.
 *     Across dimensions, ties in value put the lower dimension first, so
 *     every face precedes its cofaces.
 *   - persistence pairs are read off a reduced boundary matrix (Sec. 2,
 *     pivots of the reduced matrix give the pairs; the paper reduces the
 *     coboundary matrix, which yields the same pairs).
 *
 * Algorithm, in the textbook's order:
 *   1. validate (no NaN), map -0.0 to +0.0;
 *   2. enumerate every cube of every dimension with its value and L;
 *   3. sort all cubes by (value, dim, -L) with qsort;
 *   4. boundary column of a d-cube = positions of its 2d facets;
 *   5. standard left-to-right column reduction over Z/2 (optionally with the
 *      twist/clearing of Chen and Kerber: dimensions reduced from the top
 *      down, and the column of a cell that became a pivot is zeroed);
 *   6. every non-zero reduced column j with lowest entry i gives the pair
 *      (i, j); a cell that is neither paired nor a pivot is essential.
 *
 * Build: gcc -O2 -shared -fPIC cr_oracle.c -o libcr_oracle.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define CRO_OK 0
#define CRO_ERR_INVALID_ARG (-1)
#define CRO_ERR_NAN (-2)
#define CRO_ERR_CAPACITY (-3)
#define CRO_ERR_NOMEM (-4)

typedef struct {
    double value;    /* birth-time of the cube (float32 inputs are promoted exactly) */
    int32_t dim;     /* 0..3 */
    int32_t m;       /* type */
    int64_t x, y, z; /* anchor (minimum corner) */
    int64_t L;       /* ((m*Nz + z)*Ny + y)*Nx + x */
} cro_cell;

/* spanned directions of a (dim, type) cube, as a bit set over {x=1, y=2, z=4} */
static int span_of(int dim, int m) {
    if (dim == 0) return 0;
    if (dim == 1) return m == 0 ? 1 : (m == 1 ? 2 : 4);
    if (dim == 2) return m == 0 ? 3 : (m == 1 ? 5 : 6);
    return 7;
}

/* inverse of span_of for the facets */
static int type_of_span(int span) {
    switch (span) {
    case 0: return 0;
    case 1: return 0;
    case 2: return 1;
    case 4: return 2;
    case 3: return 0;
    case 5: return 1;
    case 6: return 2;
    default: return 0;
    }
}

static int popcount3(int s) { return (s & 1) + ((s >> 1) & 1) + ((s >> 2) & 1); }

static int ntypes(int dim) { return (dim == 0 || dim == 3) ? 1 : 3; }

static void canonical_shape(int ndim, const int64_t *shape, int64_t *nz, int64_t *ny, int64_t *nx) {
    if (ndim == 1) { *nz = 1; *ny = 1; *nx = shape[0]; }
    else if (ndim == 2) { *nz = 1; *ny = shape[0]; *nx = shape[1]; }
    else { *nz = shape[0]; *ny = shape[1]; *nx = shape[2]; }
}

static int cube_exists(int span, int64_t x, int64_t y, int64_t z, int64_t nz, int64_t ny, int64_t nx) {
    if ((span & 1) && x + 1 >= nx) return 0;
    if ((span & 2) && y + 1 >= ny) return 0;
    if ((span & 4) && z + 1 >= nz) return 0;
    return 1;
}

/* value of a cube: maximum over its vertices */
static double cube_value(const double *img, int span, int64_t x, int64_t y, int64_t z, int64_t ny, int64_t nx) {
    double v = -INFINITY;
    int first = 1;
    for (int dz = 0; dz <= ((span >> 2) & 1); dz++)
        for (int dy = 0; dy <= ((span >> 1) & 1); dy++)
            for (int dx = 0; dx <= (span & 1); dx++) {
                double w = img[((z + dz) * ny + (y + dy)) * nx + (x + dx)];
                if (first || w > v) { v = w; first = 0; }
            }
    return v;
}

static int cmp_cells(const void *pa, const void *pb) {
    const cro_cell *a = (const cro_cell *)pa, *b = (const cro_cell *)pb;
    if (a->value < b->value) return -1;
    if (a->value > b->value) return 1;
    if (a->dim != b->dim) return a->dim < b->dim ? -1 : 1;
    if (a->L != b->L) return a->L > b->L ? -1 : 1; /* larger L enters first */
    return 0;
}

/* number of cubes of every dimension in the full grid */
int64_t cro_num_cells(int ndim, const int64_t *shape) {
    if (ndim < 1 || ndim > 3) return -1;
    int64_t nz, ny, nx;
    canonical_shape(ndim, shape, &nz, &ny, &nx);
    if (nz < 1 || ny < 1 || nx < 1) return -1;
    int64_t tot = 0;
    for (int d = 0; d <= 3; d++)
        for (int m = 0; m < ntypes(d); m++) {
            int s = span_of(d, m);
            int64_t cx = (s & 1) ? nx - 1 : nx, cy = (s & 2) ? ny - 1 : ny, cz = (s & 4) ? nz - 1 : nz;
            tot += cx * cy * cz;
        }
    return tot;
}

/* ---- growable sorted columns of filtration positions ---- */
typedef struct { int64_t *v; int64_t n, cap; } col_t;

static int col_reserve(col_t *c, int64_t n) {
    if (c->cap >= n) return 0;
    int64_t nc = c->cap ? c->cap : 8;
    while (nc < n) nc *= 2;
    int64_t *p = (int64_t *)realloc(c->v, (size_t)nc * sizeof(int64_t));
    if (!p) return -1;
    c->v = p; c->cap = nc;
    return 0;
}

/* out = a XOR b (symmetric difference of sorted lists) */
static int col_xor(const col_t *a, const col_t *b, col_t *out) {
    if (col_reserve(out, a->n + b->n)) return -1;
    int64_t i = 0, j = 0, k = 0;
    while (i < a->n && j < b->n) {
        if (a->v[i] < b->v[j]) out->v[k++] = a->v[i++];
        else if (a->v[i] > b->v[j]) out->v[k++] = b->v[j++];
        else { i++; j++; }
    }
    while (i < a->n) out->v[k++] = a->v[i++];
    while (j < b->n) out->v[k++] = b->v[j++];
    out->n = k;
    return 0;
}

static int cmp_i64(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/*
 * Full persistence of the V-construction complex.
 *   img      : dense C-order array (x fastest), float64 here; the float32
 *              entry point below promotes its input exactly
 *   ndim     : 1, 2 or 3; shape[ndim] extents, each >= 1
 *   twist    : 1 = reduce dimensions top-down with clearing, 0 = plain
 *              left-to-right reduction over all columns
 *   capacity : length of the five output arrays
 * Output: every pair, zero-length ones included, in the order the reduction
 * finds them; essential classes have death = +inf and death_L = -1.
 */
static int persistence_core(const double *img, int ndim, const int64_t *shape, int twist, int64_t capacity,
                            int32_t *out_dim, double *out_birth, double *out_death, int64_t *out_birth_L,
                            int64_t *out_death_L, int64_t *n_out) {
    if (!img || !shape || !n_out || ndim < 1 || ndim > 3) return CRO_ERR_INVALID_ARG;
    int64_t nz, ny, nx;
    canonical_shape(ndim, shape, &nz, &ny, &nx);
    if (nz < 1 || ny < 1 || nx < 1) return CRO_ERR_INVALID_ARG;
    int64_t nv = nz * ny * nx;

    /* step 1: validate and canonicalise */
    double *f = (double *)malloc((size_t)nv * sizeof(double));
    if (!f) return CRO_ERR_NOMEM;
    for (int64_t i = 0; i < nv; i++) {
        double w = img[i];
        if (isnan(w)) { free(f); return CRO_ERR_NAN; }
        f[i] = (w == 0.0) ? 0.0 : w;
    }

    /* step 2: enumerate all cubes */
    int64_t ncell = cro_num_cells(ndim, shape);
    cro_cell *cells = (cro_cell *)malloc((size_t)ncell * sizeof(cro_cell));
    if (!cells) { free(f); return CRO_ERR_NOMEM; }
    int64_t k = 0;
    for (int d = 0; d <= 3; d++)
        for (int m = 0; m < ntypes(d); m++) {
            int s = span_of(d, m);
            for (int64_t z = 0; z < nz; z++)
                for (int64_t y = 0; y < ny; y++)
                    for (int64_t x = 0; x < nx; x++) {
                        if (!cube_exists(s, x, y, z, nz, ny, nx)) continue;
                        cro_cell *c = &cells[k++];
                        c->value = cube_value(f, s, x, y, z, ny, nx);
                        c->dim = d; c->m = m; c->x = x; c->y = y; c->z = z;
                        c->L = ((m * nz + z) * ny + y) * nx + x;
                    }
        }

    /* step 3: the filtration order */
    qsort(cells, (size_t)ncell, sizeof(cro_cell), cmp_cells);

    /* position of (dim, L) in the filtration; L < 3*nv for every dimension */
    int64_t lspace = 3 * nv;
    int64_t *pos = (int64_t *)malloc((size_t)(4 * lspace) * sizeof(int64_t));
    int64_t *low_owner = (int64_t *)malloc((size_t)ncell * sizeof(int64_t)); /* pivot row -> column */
    int64_t *partner = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));   /* paired cell or -1 */
    unsigned char *cleared = (unsigned char *)calloc((size_t)ncell, 1);
    col_t *reduced = (col_t *)calloc((size_t)ncell, sizeof(col_t));
    if (!pos || !low_owner || !partner || !cleared || !reduced) {
        free(f); free(cells); free(pos); free(low_owner); free(partner); free(cleared); free(reduced);
        return CRO_ERR_NOMEM;
    }
    for (int64_t i = 0; i < 4 * lspace; i++) pos[i] = -1;
    for (int64_t i = 0; i < ncell; i++) {
        pos[cells[i].dim * lspace + cells[i].L] = i;
        low_owner[i] = -1;
        partner[i] = -1;
    }

    col_t cur = {0}, tmp = {0};
    int rc = CRO_OK;

    /* the order in which columns are visited */
    int64_t *order = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    if (!order) { rc = CRO_ERR_NOMEM; goto done; }
    int64_t no = 0;
    if (twist) {
        for (int d = 3; d >= 1; d--)
            for (int64_t j = 0; j < ncell; j++)
                if (cells[j].dim == d) order[no++] = j;
    } else {
        for (int64_t j = 0; j < ncell; j++)
            if (cells[j].dim >= 1) order[no++] = j;
    }

    /* steps 4-5: reduce */
    for (int64_t t = 0; t < no; t++) {
        int64_t j = order[t];
        if (cleared[j]) continue;
        const cro_cell *c = &cells[j];
        int s = span_of(c->dim, c->m);
        /* boundary: two facets per spanned direction */
        if (col_reserve(&cur, 6)) { rc = CRO_ERR_NOMEM; goto done; }
        cur.n = 0;
        for (int b = 0; b < 3; b++) {
            if (!(s & (1 << b))) continue;
            int fs = s & ~(1 << b);
            int fm = type_of_span(fs);
            int fd = popcount3(fs);
            for (int off = 0; off <= 1; off++) {
                int64_t fx = c->x + (b == 0 ? off : 0);
                int64_t fy = c->y + (b == 1 ? off : 0);
                int64_t fz = c->z + (b == 2 ? off : 0);
                int64_t fL = ((fm * nz + fz) * ny + fy) * nx + fx;
                cur.v[cur.n++] = pos[fd * lspace + fL];
            }
        }
        qsort(cur.v, (size_t)cur.n, sizeof(int64_t), cmp_i64);
        while (cur.n > 0) {
            int64_t low = cur.v[cur.n - 1];
            int64_t o = low_owner[low];
            if (o < 0) break;
            if (col_xor(&cur, &reduced[o], &tmp)) { rc = CRO_ERR_NOMEM; goto done; }
            col_t sw = cur; cur = tmp; tmp = sw;
        }
        if (cur.n > 0) {
            int64_t low = cur.v[cur.n - 1];
            low_owner[low] = j;
            partner[low] = j;
            partner[j] = low;
            if (twist) cleared[low] = 1;
            if (col_reserve(&reduced[j], cur.n)) { rc = CRO_ERR_NOMEM; goto done; }
            memcpy(reduced[j].v, cur.v, (size_t)cur.n * sizeof(int64_t));
            reduced[j].n = cur.n;
        }
    }

    /* step 6: read off the pairs */
    {
        int64_t np = 0;
        for (int64_t i = 0; i < ncell; i++) {
            int64_t j = partner[i];
            if (j >= 0 && j < i) continue;      /* reported at its birth cell */
            if (j >= 0 && cells[j].dim != cells[i].dim + 1) continue;
            if (np < capacity) {
                out_dim[np] = cells[i].dim;
                out_birth[np] = cells[i].value;
                out_birth_L[np] = cells[i].L;
                if (j >= 0) { out_death[np] = cells[j].value; out_death_L[np] = cells[j].L; }
                else { out_death[np] = INFINITY; out_death_L[np] = -1; }
            }
            np++;
        }
        *n_out = np;
        if (np > capacity) rc = CRO_ERR_CAPACITY;
    }

done:
    for (int64_t i = 0; i < ncell; i++) free(reduced[i].v);
    free(reduced); free(cur.v); free(tmp.v); free(order);
    free(f); free(cells); free(pos); free(low_owner); free(partner); free(cleared);
    return rc;
}

/* float64 input: the values of the paper's timing study (its datasets were
 * converted to double, Sec. 3) */
int cro_persistence_f64(const double *img, int ndim, const int64_t *shape, int twist, int64_t capacity,
                        int32_t *out_dim, double *out_birth, double *out_death, int64_t *out_birth_L,
                        int64_t *out_death_L, int64_t *n_out) {
    return persistence_core(img, ndim, shape, twist, capacity, out_dim, out_birth, out_death, out_birth_L,
                            out_death_L, n_out);
}

/* float32 input: promoted to double exactly, values reported back in float32
 * (every reported value is an input value, so the conversion back is exact) */
int cro_persistence(const float *img, int ndim, const int64_t *shape, int twist, int64_t capacity,
                    int32_t *out_dim, float *out_birth, float *out_death, int64_t *out_birth_L,
                    int64_t *out_death_L, int64_t *n_out) {
    if (!img || !shape || !n_out || ndim < 1 || ndim > 3) return CRO_ERR_INVALID_ARG;
    int64_t nz, ny, nx;
    canonical_shape(ndim, shape, &nz, &ny, &nx);
    if (nz < 1 || ny < 1 || nx < 1) return CRO_ERR_INVALID_ARG;
    int64_t nv = nz * ny * nx;
    int64_t cap = capacity > 0 ? capacity : 0;
    double *d = (double *)malloc((size_t)nv * sizeof(double));
    double *b = (double *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(double));
    double *e = (double *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(double));
    if (!d || !b || !e) { free(d); free(b); free(e); return CRO_ERR_NOMEM; }
    for (int64_t i = 0; i < nv; i++) d[i] = (double)img[i];
    int rc = persistence_core(d, ndim, shape, twist, capacity, out_dim, b, e, out_birth_L, out_death_L, n_out);
    if (rc == CRO_OK || rc == CRO_ERR_CAPACITY) {
        int64_t k = *n_out < cap ? *n_out : cap;
        for (int64_t i = 0; i < k; i++) {
            out_birth[i] = (float)b[i];
            out_death[i] = (float)e[i];
        }
    }
    free(d); free(b); free(e);
    return rc;
}
