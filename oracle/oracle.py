"""TEST INFRASTRUCTURE ONLY -- the CPU oracle and its brute-force checkers.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  Nothing here is shared with the CUDA
path: the oracle has its own C source (``cr_oracle.c``), its own cell
enumeration and its own gradient rule.

Contents, each following the paper (Kaji, Sudo, Ahara, "Cubical Ripser"):

* ``persistence``      -- textbook boundary-matrix reduction of the full
                          V-construction complex (Sec. 2), via ``cr_oracle.c``.
* ``filtration``       -- Python enumeration of the cubes with their values and
                          the total order (ascending value, then dimension, then
                          descending L; the reverse of the (-birth, m, z, y, x)
                          order of Sec. 2).
* ``brute_force_pairs``-- the persistence pairing of that cell-by-cell
                          filtration from the rank function alone
                          (mu(a, b) = r(a+1, b) - r(a, b) - r(a+1, b+1) + r(a, b+1),
                          r(i, j) = rank H_p(K_i) -> H_p(K_j), ranks over Z/2).
                          No matrix reduction; tiny inputs only.
* ``brute_force_rank_diagram`` -- the same at value thresholds (diagram values).
* ``h0_1d_brute_force``-- 0-dim diagram of a sequence by counting sublevel
                          intervals (Sec. 2, connected components, Fig. 2).
* ``euler_characteristic`` -- cell counts of a sublevel set.
* ``gradient``         -- FP64 gradient of a loss given per-pair dL/dbirth and
                          dL/ddeath: each is routed to the vertex that attains
                          the cell's value (maximum vertex in the filtration
                          order), summed in double.
* ``pair_table``       -- the pairs as rows (dim, birth, death, x, y, z), located
                          at the birth or the death cell (Sec. 4, Ex. 4.1).
* ``lifetime_image``, ``persistent_histogram_image`` -- the localised-feature
                          images of Sec. 4 (largest lifetime, or a (birth,
                          lifetime) histogram, of the pairs located at each voxel).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cr_oracle.c")
_LIB = os.path.join(_HERE, "libcr_oracle.so")

PAIR_DTYPE = np.dtype([("dim", np.int32), ("birth", np.float32), ("death", np.float32),
                       ("birth_L", np.int64), ("death_L", np.int64)])
PAIR64_DTYPE = np.dtype([("dim", np.int32), ("birth", np.float64), ("death", np.float64),
                         ("birth_L", np.int64), ("death_L", np.int64)])


def build(force: bool = False) -> str:
    """Compile the C oracle in place (gcc, no GPU needed)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


@lru_cache(maxsize=1)
def _lib():
    lib = ctypes.CDLL(build())
    lib.cro_num_cells.restype = ctypes.c_int64
    lib.cro_num_cells.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
    lib.cro_persistence.restype = ctypes.c_int
    lib.cro_persistence.argtypes = [
        ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int64,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.POINTER(ctypes.c_int64)]
    lib.cro_persistence_f64.restype = ctypes.c_int
    lib.cro_persistence_f64.argtypes = lib.cro_persistence.argtypes
    return lib


def _canon(shape):
    shape = tuple(int(s) for s in shape)
    if len(shape) == 1:
        return 1, 1, shape[0]
    if len(shape) == 2:
        return 1, shape[0], shape[1]
    return shape


def num_cells(shape) -> int:
    arr = (ctypes.c_int64 * len(shape))(*[int(s) for s in shape])
    return int(_lib().cro_num_cells(len(shape), arr))


def persistence(img: np.ndarray, maxdim: int | None = None, twist: bool = True) -> np.ndarray:
    """All persistence pairs of the V-construction complex of ``img``.

    Returns a structured array (dim, birth, death, birth_L, death_L),
    zero-length pairs included; essential classes have death=+inf and
    death_L=-1.  ``maxdim`` keeps dimensions <= maxdim.  Raises ValueError for
    NaN input (the oracle's validation, Sec. 2 domain)."""
    img = np.ascontiguousarray(img, dtype=np.float32)
    if img.ndim < 1 or img.ndim > 3:
        raise ValueError("ndim must be 1, 2 or 3")
    shape = (ctypes.c_int64 * img.ndim)(*img.shape)
    cap = max(1, num_cells(img.shape))
    out = np.zeros(cap, dtype=PAIR_DTYPE)
    dim = np.zeros(cap, np.int32)
    birth = np.zeros(cap, np.float32)
    death = np.zeros(cap, np.float32)
    bl = np.zeros(cap, np.int64)
    dl = np.zeros(cap, np.int64)
    n = ctypes.c_int64(0)
    rc = _lib().cro_persistence(img.ctypes.data, img.ndim, shape, int(bool(twist)), cap,
                                dim.ctypes.data, birth.ctypes.data, death.ctypes.data,
                                bl.ctypes.data, dl.ctypes.data, ctypes.byref(n))
    if rc == -2:
        raise ValueError("NaN in input")
    if rc != 0:
        raise RuntimeError("oracle failed with code %d" % rc)
    k = n.value
    out = out[:k]
    out["dim"], out["birth"], out["death"] = dim[:k], birth[:k], death[:k]
    out["birth_L"], out["death_L"] = bl[:k], dl[:k]
    if maxdim is not None:
        out = out[out["dim"] <= maxdim]
    return out


def persistence_f64(img: np.ndarray, maxdim: int | None = None, twist: bool = True) -> np.ndarray:
    """``persistence`` for a float64 image, computed in double (the precision
    of the paper's timing study, whose datasets were converted to double,
    Sec. 3); births and deaths are float64."""
    img = np.ascontiguousarray(img, dtype=np.float64)
    if img.ndim < 1 or img.ndim > 3:
        raise ValueError("ndim must be 1, 2 or 3")
    shape = (ctypes.c_int64 * img.ndim)(*img.shape)
    cap = max(1, num_cells(img.shape))
    out = np.zeros(cap, dtype=PAIR64_DTYPE)
    dim = np.zeros(cap, np.int32)
    birth = np.zeros(cap, np.float64)
    death = np.zeros(cap, np.float64)
    bl = np.zeros(cap, np.int64)
    dl = np.zeros(cap, np.int64)
    n = ctypes.c_int64(0)
    rc = _lib().cro_persistence_f64(img.ctypes.data, img.ndim, shape, int(bool(twist)), cap,
                                    dim.ctypes.data, birth.ctypes.data, death.ctypes.data,
                                    bl.ctypes.data, dl.ctypes.data, ctypes.byref(n))
    if rc == -2:
        raise ValueError("NaN in input")
    if rc != 0:
        raise RuntimeError("oracle failed with code %d" % rc)
    k = n.value
    out = out[:k]
    out["dim"], out["birth"], out["death"] = dim[:k], birth[:k], death[:k]
    out["birth_L"], out["death_L"] = bl[:k], dl[:k]
    if maxdim is not None:
        out = out[out["dim"] <= maxdim]
    return out


# ---------------------------------------------------------------------------
# Python cell enumeration (independent of the C code above)
# ---------------------------------------------------------------------------
_SPAN = {(0, 0): (), (1, 0): (0,), (1, 1): (1,), (1, 2): (2,),
         (2, 0): (0, 1), (2, 1): (0, 2), (2, 2): (1, 2), (3, 0): (0, 1, 2)}
_TYPE = {v: k for k, v in _SPAN.items()}


def _decode(L, shape):
    nz, ny, nx = _canon(shape)
    x = L % nx
    y = (L // nx) % ny
    z = (L // (nx * ny)) % nz
    m = L // (nx * ny * nz)
    return int(m), int(z), int(y), int(x)


def cell_vertices(dim: int, L: int, shape):
    """Linear vertex indices of the cube (dim, L); axes 0,1,2 = x,y,z."""
    nz, ny, nx = _canon(shape)
    m, z, y, x = _decode(L, shape)
    span = _SPAN[(dim, m)]
    out = []
    for dz in range(2 if 2 in span else 1):
        for dy in range(2 if 1 in span else 1):
            for dx in range(2 if 0 in span else 1):
                out.append(((z + dz) * ny + (y + dy)) * nx + (x + dx))
    return out


def _canon_values(img, dtype=np.float32):
    f = np.ascontiguousarray(img, dtype=dtype).reshape(-1).copy()
    f[f == 0] = 0.0  # -0.0 -> +0.0
    return f


def _vertex_values(img, vs):
    """Canonical float32 values of the listed vertices (only those are read)."""
    return _canon_values(np.asarray(img).reshape(-1)[np.asarray(vs, dtype=np.int64)])


def cell_value(img, dim: int, L: int) -> float:
    vs = cell_vertices(dim, L, img.shape)
    return float(max(_vertex_values(img, vs)))


def argmax_vertex(img, dim: int, L: int) -> int:
    """The vertex that attains the cube's value: the latest vertex of the cube
    in the filtration (largest value; among equal values the smallest linear
    index, since larger indices enter first)."""
    vs = cell_vertices(dim, L, img.shape)
    f = _vertex_values(img, vs)
    best = max(range(len(vs)), key=lambda i: (float(f[i]), -vs[i]))
    return vs[best]


def gradient(img, pairs, grad_birth, grad_death) -> np.ndarray:
    """FP64 gradient of a loss w.r.t. the image given dL/dbirth, dL/ddeath per
    pair: each is added at the argmax vertex of the birth / death cube;
    essential deaths (death_L < 0) contribute nothing."""
    g = np.zeros(int(np.prod(img.shape)), dtype=np.float64)
    for k in range(len(pairs)):
        d = int(pairs["dim"][k])
        g[argmax_vertex(img, d, int(pairs["birth_L"][k]))] += float(grad_birth[k])
        if int(pairs["death_L"][k]) >= 0:
            g[argmax_vertex(img, d + 1, int(pairs["death_L"][k]))] += float(grad_death[k])
    return g.reshape(img.shape)


def filtration(img, dtype=np.float32):
    """All cubes as (value, dim, L, facets) sorted by (value, dim, -L); facets
    are the (dim-1, L) of the 2*dim facets.  Values are taken in ``dtype``."""
    nz, ny, nx = _canon(img.shape)
    f = _canon_values(img, dtype)
    cells = []
    ext = (nx, ny, nz)
    for (dim, m), span in _SPAN.items():
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    a = (x, y, z)
                    if any(a[k] + 1 >= ext[k] for k in span):
                        continue
                    L = ((m * nz + z) * ny + y) * nx + x
                    verts = cell_vertices(dim, L, img.shape)
                    val = float(max(f[v] for v in verts))
                    facets = []
                    for k in span:
                        rest = tuple(s for s in span if s != k)
                        fm = _TYPE[rest][1]
                        for off in (0, 1):
                            b = list(a)
                            b[k] += off
                            fL = ((fm * nz + b[2]) * ny + b[1]) * nx + b[0]
                            facets.append((dim - 1, fL))
                    cells.append((val, dim, L, facets))
    cells.sort(key=lambda c: (c[0], c[1], -c[2]))
    return cells


def _xor_rank_insert(basis: dict, v: int) -> bool:
    """Insert v into a GF(2) basis keyed by leading bit; True if independent."""
    while v:
        h = v.bit_length() - 1
        if h in basis:
            v ^= basis[h]
        else:
            basis[h] = v
            return True
    return False


def brute_force_pairs(img, dtype=np.float32):
    """Cell pairs from the rank function of the cell-by-cell filtration.

    Returns a set of (dim, birth_L, death_L) with death_L = -1 for essential
    classes, zero-length pairs included.  Cost grows like n^3 in the number of
    cubes n: inputs of at most ~120 cubes.  Values are taken in ``dtype``."""
    cells = filtration(img, dtype)
    n = len(cells)
    posmap = {(c[1], c[2]): i for i, c in enumerate(cells)}
    bnd = []
    for (val, dim, L, facets) in cells:
        v = 0
        for fc in facets:
            v |= 1 << posmap[fc]
        bnd.append(v)
    top = max(c[1] for c in cells)
    result = set()
    for p in range(0, top + 1):
        # Z_p(K_i) for every prefix i: kernel vectors of boundary restricted to p-cells
        Z = [[] for _ in range(n + 1)]
        piv = {}  # leading bit -> (reduced boundary, combination)
        kern = []
        for i in range(n):
            if cells[i][1] == p:
                b, e = bnd[i], 1 << i
                while b:
                    h = b.bit_length() - 1
                    if h in piv:
                        b ^= piv[h][0]
                        e ^= piv[h][1]
                    else:
                        piv[h] = (b, e)
                        break
                if b == 0:
                    kern.append(e)
            Z[i + 1] = list(kern)
        # r(i, j) = dim(Z_i + B_j) - dim(B_j), for all i <= j
        R = np.zeros((n + 1, n + 1), dtype=np.int64)
        for i in range(n + 1):
            zb = {}
            for z in Z[i]:
                _xor_rank_insert(zb, z)
            bb = {}
            rz = len(zb)
            rb = 0
            for j in range(n + 1):
                if j > 0 and cells[j - 1][1] == p + 1:
                    if _xor_rank_insert(bb, bnd[j - 1]):
                        rb += 1
                    if _xor_rank_insert(zb, bnd[j - 1]):
                        rz += 1
                if j >= i:
                    R[i, j] = rz - rb
        for a in range(n):
            if cells[a][1] != p:
                continue
            ess = R[a + 1, n] - R[a, n]
            if ess == 1:
                result.add((p, cells[a][2], -1))
            for b in range(a + 1, n):
                if cells[b][1] != p + 1:
                    continue
                mu = R[a + 1, b] - R[a, b] - R[a + 1, b + 1] + R[a, b + 1]
                if mu:
                    result.add((p, cells[a][2], cells[b][2]))
    return result


def brute_force_rank_diagram(img, dtype=np.float32):
    """Diagram values (dim, birth, death) with multiplicity, from ranks of the
    maps between sublevel complexes at the distinct values; zero-length bars
    do not appear.  Returns a sorted list of (dim, birth, death).  Values are
    taken in ``dtype``."""
    cells = filtration(img, dtype)
    vals = sorted(set(c[0] for c in cells))
    T = len(vals)
    n = len(cells)
    posmap = {(c[1], c[2]): i for i, c in enumerate(cells)}
    bnd = []
    for (val, dim, L, facets) in cells:
        v = 0
        for fc in facets:
            v |= 1 << posmap[fc]
        bnd.append(v)
    # prefix length at each threshold
    cut = [sum(1 for c in cells if c[0] <= t) for t in vals]
    top = max(c[1] for c in cells)
    out = []
    for p in range(0, top + 1):
        def zbasis(k):
            piv, kern = {}, []
            for i in range(k):
                if cells[i][1] != p:
                    continue
                b, e = bnd[i], 1 << i
                while b:
                    h = b.bit_length() - 1
                    if h in piv:
                        b ^= piv[h][0]
                        e ^= piv[h][1]
                    else:
                        piv[h] = (b, e)
                        break
                if b == 0:
                    kern.append(e)
            return kern

        def rank(i, j):  # rank H_p(K_vals[i]) -> H_p(K_vals[j]); i = -1 means empty
            if i < 0:
                return 0
            zb, bb = {}, {}
            for z in zbasis(cut[i]):
                _xor_rank_insert(zb, z)
            rb = 0
            for q in range(cut[j]):
                if cells[q][1] == p + 1:
                    if _xor_rank_insert(bb, bnd[q]):
                        rb += 1
                    _xor_rank_insert(zb, bnd[q])
            return len(zb) - rb

        Rm = {}
        for i in range(-1, T):
            for j in range(max(i, 0), T):
                Rm[(i, j)] = rank(i, j)
        for a in range(T):
            for b in range(a + 1, T):
                mu = Rm[(a, b - 1)] - Rm[(a - 1, b - 1)] - Rm[(a, b)] + Rm[(a - 1, b)]
                out += [(p, vals[a], vals[b])] * int(mu)
            ess = Rm[(a, T - 1)] - Rm[(a - 1, T - 1)]
            out += [(p, vals[a], float("inf"))] * int(ess)
    return sorted(out)


def h0_1d_brute_force(seq):
    """Non-zero 0-dim bars of a 1D sequence from sublevel interval counts.

    rank H_0(K_s) -> H_0(K_t) = number of maximal runs of {f <= t} that meet
    {f <= s}.  Returns a sorted list of (birth, death)."""
    f = _canon_values(np.asarray(seq, np.float32))
    vals = sorted(set(float(v) for v in f))
    T = len(vals)

    def runs(t):
        out, cur = [], None
        for i, v in enumerate(f):
            if v <= t:
                cur = [i, i] if cur is None else [cur[0], i]
            elif cur is not None:
                out.append(tuple(cur))
                cur = None
        if cur is not None:
            out.append(tuple(cur))
        return out

    def r(i, j):
        if i < 0:
            return 0
        s, t = vals[i], vals[j]
        return sum(1 for (a, b) in runs(t) if any(f[k] <= s for k in range(a, b + 1)))

    out = []
    for a in range(T):
        for b in range(a + 1, T):
            mu = r(a, b - 1) - r(a - 1, b - 1) - r(a, b) + r(a - 1, b)
            out += [(vals[a], vals[b])] * mu
        ess = r(a, T - 1) - r(a - 1, T - 1)
        out += [(vals[a], float("inf"))] * ess
    return sorted(out)


def euler_characteristic(img, t: float) -> int:
    """Alternating count of the cubes whose value is <= t."""
    chi = 0
    for (val, dim, L, facets) in filtration(img):
        if val <= t:
            chi += (-1) ** dim
    return chi


# ---------------------------------------------------------------------------
# Localised features (Sec. 4, the example on localised features): images
# built from the pairs and the locations of their cells
# ---------------------------------------------------------------------------
def _location_pixel(L: int, shape) -> int:
    """Linear index of the voxel at which the cell with L-index ``L`` is
    anchored (its (x, y, z) location; the cell type m is dropped)."""
    nz, ny, nx = _canon(shape)
    _, z, y, x = _decode(L, shape)
    return (z * ny + y) * nx + x


def pair_table(shape, pairs, location: str = "birth") -> np.ndarray:
    """One row (dim, birth, death, x, y, z) per pair, the layout of the table
    the paper's ``computePH`` returns (Sec. 4, Ex. 4.1): (x, y, z) is the anchor
    of the birth cell, or of the death cell with ``location="death"``; an
    essential pair has no death cell and is located at its birth cell.  x is
    the fastest array index; unused axes are 0."""
    out = np.zeros((len(pairs), 6), dtype=np.float64)
    for k in range(len(pairs)):
        L = int(pairs["birth_L"][k])
        if location == "death" and int(pairs["death_L"][k]) >= 0:
            L = int(pairs["death_L"][k])
        _, z, y, x = _decode(L, shape)
        out[k] = (int(pairs["dim"][k]), float(pairs["birth"][k]), float(pairs["death"][k]), x, y, z)
    return out


def lifetime_image(shape, pairs, location: str = "birth") -> np.ndarray:
    """Lifetime channels of the lifetime enhanced image: channel d (d < ndim)
    holds at each voxel the largest lifetime death - birth (float32
    subtraction) of the finite pairs of dimension d located there, 0 where
    there is none.  The location of a pair is the anchor voxel of its birth
    cell (or of its death cell, ``location="death"``).  Essential pairs have no
    finite lifetime and are left out."""
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    out = np.zeros((nd, int(np.prod(shape))), dtype=np.float32)
    for k in range(len(pairs)):
        death = np.float32(pairs["death"][k])
        if not np.isfinite(death):
            continue
        d = int(pairs["dim"][k])
        L = int(pairs["birth_L"][k] if location == "birth" else pairs["death_L"][k])
        v = _location_pixel(L, shape)
        life = np.float32(death - np.float32(pairs["birth"][k]))
        if life > out[d, v]:
            out[d, v] = life
    return out.reshape((nd,) + shape)


def persistent_histogram_image(shape, pairs, nb: int, b_lo: float, b_hi: float, nl: int, l_hi: float,
                               location: str = "birth") -> np.ndarray:
    """Persistent histogram image: for each voxel, per dimension d, the 2D
    histogram of (birth, lifetime) of the finite pairs located at the voxel,
    flattened into channels ((d * nb + i) * nl + j).  Bin i of birth covers
    [b_lo + i w, b_lo + (i+1) w), w = (b_hi - b_lo) / nb, computed as
    floor((birth - b_lo) / (b_hi - b_lo) * nb) in double; lifetime bin j is
    floor(lifetime / l_hi * nl) with lifetime = death - birth in double.
    Pairs outside [b_lo, b_hi) x [0, l_hi) are not counted."""
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    out = np.zeros((nd * nb * nl, int(np.prod(shape))), dtype=np.float32)
    for k in range(len(pairs)):
        death = float(pairs["death"][k])
        if not np.isfinite(death):
            continue
        birth = float(pairs["birth"][k])
        i = int(np.floor((birth - float(b_lo)) / (float(b_hi) - float(b_lo)) * nb))
        j = int(np.floor((death - birth) / float(l_hi) * nl))
        if i < 0 or i >= nb or j < 0 or j >= nl:
            continue
        d = int(pairs["dim"][k])
        L = int(pairs["birth_L"][k] if location == "birth" else pairs["death_L"][k])
        out[(d * nb + i) * nl + j, _location_pixel(L, shape)] += 1.0
    return out.reshape((nd * nb * nl,) + shape)
