"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(no GPU).  Each test checks the oracle against something other than itself:
the paper's worked examples, a brute-force rank computation, 1D interval
counting, Euler characteristics, cell counts, symmetries and finite
differences."""
import itertools

import numpy as np
import pytest

from tests.golden.golden_io import read_image_and_bars, read_pairs


def nonzero(p):
    keep = p["birth"] != p["death"]
    return sorted((int(d), float(b), float(e)) for d, b, e in zip(p["dim"][keep], p["birth"][keep], p["death"][keep]))


def cellset(p):
    return set((int(d), int(b), int(e)) for d, b, e in zip(p["dim"], p["birth_L"], p["death_L"]))


def test_ttk_example(oracle_mod):
    # Rem. 3.2: the 3x3 image with 9 in the centre has the 1-cycle [0, 9)
    img, bars = read_image_and_bars("ttk_3x3.txt")
    p = oracle_mod.persistence(img)
    assert nonzero(p) == sorted((int(b[0]), b[1], b[2]) for b in bars)
    # hand count including zero-length pairs: 7 (0,0) + 1 (9,9) in H0, 3 (9,9) in H1
    z = p[p["birth"] == p["death"]]
    assert sorted((int(a), float(b)) for a, b in zip(z["dim"], z["birth"])) == \
        [(0, 0.0)] * 7 + [(0, 9.0)] + [(1, 9.0)] * 3


def test_fig2_h0(oracle_mod):
    img, bars = read_image_and_bars("fig2_h0.txt")
    p = oracle_mod.persistence(img)
    assert [b for b in nonzero(p) if b[0] == 0] == sorted((0, b[0], b[1]) for b in bars)


def _random_images(rng, count, shapes, levels=(1, 2, 3, 5)):
    out = []
    for _ in range(count):
        sh = shapes[rng.integers(len(shapes))]
        lev = levels[rng.integers(len(levels))]
        if rng.random() < 0.25:
            out.append(rng.random(sh).astype(np.float32))
        else:
            out.append(rng.integers(0, lev, sh).astype(np.float32))
    return out


@pytest.mark.parametrize("kind", ["1d", "2d", "3d"])
def test_cell_pairs_equal_rank_function(oracle_mod, kind):
    # the pairing of a cell-by-cell filtration is fixed by its rank function
    rng = np.random.default_rng({"1d": 11, "2d": 12, "3d": 13}[kind])
    shapes = {"1d": [(1,), (2,), (5,), (9,)],
              "2d": [(1, 1), (1, 4), (4, 1), (2, 2), (3, 3), (2, 4), (3, 4)],
              "3d": [(2, 2, 2), (1, 2, 3), (2, 1, 3), (2, 3, 2), (2, 2, 3)]}[kind]
    for img in _random_images(rng, {"1d": 40, "2d": 40, "3d": 12}[kind], shapes):
        assert cellset(oracle_mod.persistence(img)) == oracle_mod.brute_force_pairs(img), img.tolist()


def test_diagram_equals_rank_diagram_3x3(oracle_mod):
    # a deterministic sample of the 3^9 three-level 3x3 images
    rng = np.random.default_rng(3)
    codes = rng.choice(3 ** 9, size=300, replace=False)
    for c in codes:
        vals = [(int(c) // 3 ** k) % 3 for k in range(9)]
        img = np.array(vals, np.float32).reshape(3, 3)
        assert nonzero(oracle_mod.persistence(img)) == oracle_mod.brute_force_rank_diagram(img)


def test_h0_1d_interval_counting(oracle_mod):
    rng = np.random.default_rng(4)
    for n in [1, 2, 3, 7, 20, 41]:
        for lev in [2, 4, 100]:
            seq = rng.integers(0, lev, n).astype(np.float32)
            got = [(b, e) for d, b, e in nonzero(oracle_mod.persistence(seq)) if d == 0]
            assert got == oracle_mod.h0_1d_brute_force(seq)


def test_sine_example_golden(oracle_mod):
    # Sec. 4, Ex. 4.4 input; golden written by tests/golden/make_golden.py
    x = np.linspace(0, 4 * np.pi, 100)
    seq = (np.sin(x) + 0.1 * x).astype(np.float32)
    got = nonzero(oracle_mod.persistence(seq))
    exp = sorted((d, b, e) for d, b, e, _, _ in read_pairs("sine100_pairs.txt"))
    assert [(d, np.float32(b), np.float32(e)) for d, b, e in got] == \
        [(d, np.float32(b), np.float32(e)) for d, b, e in exp]
    # and it agrees with interval counting
    assert [(b, e) for d, b, e in got] == oracle_mod.h0_1d_brute_force(seq)


@pytest.mark.parametrize("shape", [(7,), (5, 6), (3, 4, 5)])
def test_euler_characteristic_every_threshold(oracle_mod, shape):
    rng = np.random.default_rng(5)
    for lev in [3, 50]:
        img = rng.integers(0, lev, shape).astype(np.float32)
        p = oracle_mod.persistence(img)
        for t in sorted(set(img.reshape(-1).tolist())) + [1e9]:
            alive = (p["birth"] <= t) & (t < p["death"])
            chi_bars = int(sum((-1) ** int(d) for d in p["dim"][alive]))
            assert chi_bars == oracle_mod.euler_characteristic(img, t)


@pytest.mark.parametrize("shape", [(13,), (6, 9), (4, 5, 6), (1, 5, 6), (3, 1, 4)])
def test_totals(oracle_mod, shape):
    rng = np.random.default_rng(6)
    img = rng.integers(0, 4, shape).astype(np.float32)
    p = oracle_mod.persistence(img)
    nz, ny, nx = (1, 1) + shape if len(shape) == 1 else ((1,) + shape if len(shape) == 2 else shape)
    V = nx * ny * nz
    E = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    F = (nx - 1) * (ny - 1) * nz + (nx - 1) * ny * (nz - 1) + nx * (ny - 1) * (nz - 1)
    C = (nx - 1) * (ny - 1) * (nz - 1)
    cnt = [int((p["dim"] == d).sum()) for d in range(3)]
    ess = p[~np.isfinite(p["death"])]
    assert len(ess) == 1 and ess["dim"][0] == 0  # beta_0 = 1, higher Betti numbers 0
    assert cnt[0] == V  # V - 1 finite + 1 essential
    assert cnt[1] == E - V + 1
    assert cnt[2] == C
    assert E - V + 1 == F - C  # chi = 1


def test_twist_does_not_change_pairs(oracle_mod):
    rng = np.random.default_rng(7)
    for sh in [(6, 7), (3, 4, 5), (30,)]:
        img = rng.integers(0, 3, sh).astype(np.float32)
        assert cellset(oracle_mod.persistence(img, twist=True)) == cellset(oracle_mod.persistence(img, twist=False))


def test_embedding_and_symmetries(oracle_mod):
    rng = np.random.default_rng(8)
    img2 = rng.integers(0, 5, (6, 7)).astype(np.float32)
    # (1, Ny, Nx) volume = the 2D image, cell for cell (Sec. 2: 2D is the slice k = 0)
    assert cellset(oracle_mod.persistence(img2[None])) == cellset(oracle_mod.persistence(img2))
    seq = img2[0]
    assert cellset(oracle_mod.persistence(seq[None, None])) == cellset(oracle_mod.persistence(seq))
    assert cellset(oracle_mod.persistence(seq[None])) == cellset(oracle_mod.persistence(seq))
    base = nonzero(oracle_mod.persistence(img2))
    for t in [img2[::-1], img2[:, ::-1], img2.T, img2[::-1, ::-1].T]:
        assert nonzero(oracle_mod.persistence(np.ascontiguousarray(t))) == base
    vol = rng.integers(0, 4, (3, 4, 5)).astype(np.float32)
    vb = nonzero(oracle_mod.persistence(vol))
    for t in [vol[::-1], np.transpose(vol, (2, 0, 1)), np.transpose(vol, (1, 2, 0))[:, ::-1]]:
        assert nonzero(oracle_mod.persistence(np.ascontiguousarray(t))) == vb
    # scaling by 2 scales every bar exactly
    sc = nonzero(oracle_mod.persistence(img2 * 2))
    assert sc == [(d, 2 * b, 2 * e) for d, b, e in base]


def test_nan_and_negative_zero(oracle_mod):
    img = np.zeros((3, 3), np.float32)
    img[1, 1] = np.nan
    with pytest.raises(ValueError):
        oracle_mod.persistence(img)
    a = np.array([[0.0, 1.0], [2.0, 0.0]], np.float32)
    b = a.copy()
    b[0, 0] = -0.0
    assert cellset(oracle_mod.persistence(a)) == cellset(oracle_mod.persistence(b))


def test_plus_infinity_is_an_ordinary_value(oracle_mod):
    # Sec. 2: outside a non-rectangular domain the image is extended by a huge value
    img = np.array([[0, 1, np.inf], [2, np.inf, 0.5], [np.inf, 3, 0]], np.float32)
    p = oracle_mod.persistence(img)
    assert cellset(p) == oracle_mod.brute_force_pairs(img)


def _loss(oracle_mod, img):
    p = oracle_mod.persistence(img)
    fin = np.isfinite(p["death"])
    d = p["death"][fin].astype(np.float64) - p["birth"][fin].astype(np.float64)
    return float((d * d).sum())


@pytest.mark.parametrize("shape", [(12,), (5, 6), (3, 3, 4)])
def test_gradient_rule_matches_finite_differences(oracle_mod, shape):
    # L = sum (d - b)^2; on a tie-free image every bar end is one pixel's value
    rng = np.random.default_rng(9)
    img = rng.permutation(np.prod(shape)).reshape(shape).astype(np.float32)
    p = oracle_mod.persistence(img)
    fin = np.isfinite(p["death"])
    life = np.where(fin, p["death"].astype(np.float64) - p["birth"].astype(np.float64), 0.0)
    g = oracle_mod.gradient(img, p, -2 * life, 2 * life)
    h = 0.25  # values are integers: +-0.25 keeps the order
    for idx in itertools.islice(np.ndindex(*shape), 0, None, 3):
        up, dn = img.copy(), img.copy()
        up[idx] += h
        dn[idx] -= h
        fd = (_loss(oracle_mod, up) - _loss(oracle_mod, dn)) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-9 * max(1.0, abs(fd)), (idx, fd, g[idx])


def test_uniform64_golden(oracle_mod):
    from paper_2005_12692_gb300 import synth
    p = oracle_mod.persistence(synth.uniform64())
    got = sorted((int(a), float(b), float(c), int(d), int(e)) for a, b, c, d, e in
                 zip(p["dim"], p["birth"], p["death"], p["birth_L"], p["death_L"]) if b != c)
    exp = sorted((d, float(np.float32(b)), float(np.float32(e)), bl, dl) for d, b, e, bl, dl in
                 read_pairs("uniform64_pairs.txt"))
    assert got == exp


# ---------------------------------------------------------------------------
# localised-feature images (Sec. 4, the example on localised features)
# ---------------------------------------------------------------------------
def test_lifetime_image_hand_1d(oracle_mod):
    # f = [0, 2, 1, 3]: the component born at 1 (vertex 2) dies at value 2 when
    # the edge (0,1) enters; the equal-valued edge (1,2) enters first (larger L)
    # and kills the younger vertex 1 at zero length.
    f = np.array([0, 2, 1, 3], np.float32)
    p = oracle_mod.persistence(f)
    assert np.array_equal(oracle_mod.lifetime_image(f.shape, p), [[0, 0, 1, 0]])
    assert np.array_equal(oracle_mod.lifetime_image(f.shape, p, "death"), [[1, 0, 0, 0]])


def test_lifetime_and_histogram_images_hand_2d(oracle_mod):
    # a 3x4 plateau of 5 with two wells: 0 at (y=1, x=1) lives forever, 1 at
    # (y=1, x=3) dies at 5 -> lifetime 4 located at row 1, column 3; every other
    # class is born and killed at 5.
    img = np.array([[5, 5, 5, 5], [5, 0, 5, 1], [5, 5, 5, 5]], np.float32)
    p = oracle_mod.persistence(img)
    p = p[p["death"] > p["birth"]]
    li = oracle_mod.lifetime_image(img.shape, p)
    exp = np.zeros((2, 3, 4), np.float32)
    exp[0, 1, 3] = 4.0
    assert np.array_equal(li, exp)
    # birth bins of width 2 on [0, 8), lifetime bins of width 2 on [0, 8): the
    # pair (1, 5) falls in birth bin 0 and lifetime bin 2 -> channel 2
    h = oracle_mod.persistent_histogram_image(img.shape, p, 4, 0.0, 8.0, 4, 8.0)
    assert h.shape == (2 * 4 * 4, 3, 4)
    assert np.argwhere(h).tolist() == [[2, 1, 3]] and h[2, 1, 3] == 1.0


def test_localised_images_invariants(oracle_mod):
    # on random tie-heavy 2D/3D inputs: channel d's maximum is the largest finite
    # lifetime of dimension d; a histogram spanning every pair counts each finite
    # pair once, at the voxel of its birth cell
    rng = np.random.default_rng(31)
    for shape in [(7, 9), (4, 5, 6)]:
        img = rng.integers(0, 6, size=shape).astype(np.float32)
        p = oracle_mod.persistence(img)
        for loc, key in (("birth", "birth_L"), ("death", "death_L")):
            li = oracle_mod.lifetime_image(shape, p, loc)
            for d in range(len(shape)):
                sel = (p["dim"] == d) & np.isfinite(p["death"])
                m = float((p["death"][sel] - p["birth"][sel]).max()) if sel.any() else 0.0
                assert float(li[d].max()) == m
        h = oracle_mod.persistent_histogram_image(shape, p, 3, -1.0, 7.0, 2, 8.0)
        fin = np.isfinite(p["death"])
        assert h.sum() == fin.sum()
        for d in range(len(shape)):
            per_voxel = h[d * 6:(d + 1) * 6].sum(axis=0).reshape(-1)
            sel = fin & (p["dim"] == d)
            cnt = np.zeros(per_voxel.size)
            for L in p["birth_L"][sel]:
                m, z, y, x = oracle_mod.oracle._decode(int(L), shape)
                nz, ny, nx = oracle_mod.oracle._canon(shape)
                cnt[(z * ny + y) * nx + x] += 1
            assert np.array_equal(per_voxel, cnt)


def _near_tied_f64(rng, shape):
    """float64 images whose values differ below float32 resolution: small
    integer levels plus multiples of 2^-40, so that casting to float32 ties
    values the float64 filtration orders."""
    base = rng.integers(0, 3, shape).astype(np.float64)
    return base + rng.integers(0, 4, shape) * 2.0 ** -40


@pytest.mark.parametrize("kind", ["1d", "2d", "3d"])
def test_f64_cell_pairs_equal_rank_function(oracle_mod, kind):
    # the float64 oracle against the rank function of the float64 cell-by-cell filtration
    rng = np.random.default_rng({"1d": 21, "2d": 22, "3d": 23}[kind])
    shapes = {"1d": [(3,), (6,), (9,)], "2d": [(2, 3), (3, 3), (3, 4)], "3d": [(2, 2, 2), (2, 2, 3)]}[kind]
    differs = 0
    for _ in range({"1d": 25, "2d": 25, "3d": 8}[kind]):
        img = _near_tied_f64(rng, shapes[rng.integers(len(shapes))])
        p = oracle_mod.persistence_f64(img)
        assert p["birth"].dtype == np.float64
        assert cellset(p) == oracle_mod.brute_force_pairs(img, np.float64), img.tolist()
        differs += cellset(p) != cellset(oracle_mod.persistence(img))  # the float32 cast ties values
    assert differs > 0


def test_f64_diagram_equals_rank_diagram(oracle_mod):
    rng = np.random.default_rng(24)
    for _ in range(40):
        img = _near_tied_f64(rng, (3, 3))
        got = nonzero(oracle_mod.persistence_f64(img))
        assert got == oracle_mod.brute_force_rank_diagram(img, np.float64)
        # values are the image's own float64 values, not float32 roundings
        assert all(b in set(img.ravel().tolist()) for _, b, _ in got)


def test_f64_promotes_float32_inputs_exactly(oracle_mod):
    from paper_2005_12692_gb300 import synth
    for img in [synth.grf((17, 23), 2.0, 25), synth.quantised(synth.grf((5, 6, 7), 2.0, 26), 4)]:
        a = oracle_mod.persistence(img)
        b = oracle_mod.persistence_f64(img.astype(np.float64))
        assert cellset(a) == cellset(b)
        assert np.array_equal(a["birth"].astype(np.float64), b["birth"])
        assert np.array_equal(a["death"].astype(np.float64), b["death"])
    with pytest.raises(ValueError):
        oracle_mod.persistence_f64(np.array([0.0, np.nan]))


def _uf_find(par, x):
    while par[x] != x:
        par[x] = par[par[x]]
        x = par[x]
    return x


def _h0_by_union_find(cells):
    """H0 cell pairs by the elder rule (Sec. 2, union-find on vertices): edges in
    filtration order; a merge kills the component whose oldest vertex entered
    later."""
    pos = {(c[1], c[2]): i for i, c in enumerate(cells)}
    par = {}
    pairs = set()
    for i, (val, dim, L, facets) in enumerate(cells):
        if dim == 0:
            par[L] = L
        elif dim == 1:
            a, b = (_uf_find(par, fL) for _, fL in facets)
            if a == b:
                continue
            young, old = (a, b) if pos[(0, a)] > pos[(0, b)] else (b, a)
            par[young] = old  # the root is the oldest vertex of its component
            pairs.add((0, young, L))
    roots = {_uf_find(par, v) for v in list(par)}
    assert len(roots) == 1
    pairs.add((0, roots.pop(), -1))
    return pairs


def _top_by_dual_union_find(cells, shape):
    """Top-dimensional cell pairs by duality (Rem. 2.1): the top cubes plus one
    outer node are the vertices of the dual graph, the (top-1)-cubes its edges
    (a boundary cube joins its one top cube to the outer node).  Edges are taken
    in reverse filtration order; a merge kills the component whose oldest
    member in that order (its latest top cube in the filtration) comes later in
    it, and pairs the edge with that cube."""
    D = len(shape)  # dimension of the top cubes (every extent > 1)
    pos = {(c[1], c[2]): i for i, c in enumerate(cells)}
    cof = {}
    for val, dim, L, facets in cells:
        if dim == D:
            for f in facets:
                cof.setdefault(f, []).append(L)
    OUT = -1
    par = {OUT: OUT}
    age = {OUT: float("inf")}  # the outer node is older than everything
    pairs = set()
    for val, dim, L, facets in reversed(cells):
        if dim == D:
            par[L] = L
            age[L] = pos[(D, L)]
        elif dim == D - 1:
            ends = cof.get((dim, L), [])
            assert 1 <= len(ends) <= 2
            ends = ends + [OUT] * (2 - len(ends))
            a, b = (_uf_find(par, e) for e in ends)
            if a == b:
                continue
            young, old = (a, b) if age[a] < age[b] else (b, a)
            par[young] = old
            pairs.add((D - 1, L, young))
    return pairs


@pytest.mark.parametrize("kind", ["2d", "3d"])
def test_h0_and_top_dimension_by_union_find_and_duality(oracle_mod, kind):
    # the reduction's pairs in dimension 0 equal the elder-rule union-find, and in
    # the top dimension the union-find on the dual graph in reverse order
    rng = np.random.default_rng({"2d": 41, "3d": 42}[kind])
    shapes = {"2d": [(2, 2), (3, 5), (6, 4), (9, 11), (14, 13)],
              "3d": [(2, 2, 2), (2, 3, 4), (4, 4, 3), (5, 6, 5)]}[kind]
    for _ in range({"2d": 40, "3d": 20}[kind]):
        sh = shapes[rng.integers(len(shapes))]
        img = (rng.integers(0, 4, sh) if rng.random() < 0.7 else rng.random(sh)).astype(np.float32)
        cells = oracle_mod.filtration(img)
        p = oracle_mod.persistence(img)
        got = cellset(p)
        assert {c for c in got if c[0] == 0} == _h0_by_union_find(cells), img.tolist()
        top = len(sh) - 1
        assert {c for c in got if c[0] == top} == _top_by_dual_union_find(cells, sh), img.tolist()


def test_tie_order_by_hand(oracle_mod):
    # Sec. 2 orders cells by (-value, type, z, y, x) in cohomology; the filtration is
    # its reverse, so among equal values larger L enters first, vertices before edges.
    # [0, 0, 0]: vertices enter as v2, v1, v0; then edges e1 = (v1, v2), e0 = (v0, v1).
    # e1 joins {v2} and {v1}: v1 entered later and dies, pair (v1, e1); e0 joins
    # {v2, v1} and {v0}: v0 dies, pair (v0, e0); v2 is essential.
    p = oracle_mod.persistence(np.zeros(3, np.float32))
    assert cellset(p) == {(0, 1, 1), (0, 0, 0), (0, 2, -1)}
    # 2x2 all equal: vertices L 3, 2, 1, 0; x-edges (type 0) L 2, 0 and y-edges (type 1)
    # L 4 + 1, 4 + 0 (L = (m*Ny + y)*Nx + x); edges enter by descending L: y-edge at x=1
    # (L 5, joins v1 and v3), y-edge at x=0 (L 4, joins v0 and v2), x-edge at y=1
    # (L 2, joins v2 and v3), x-edge at y=0 (L 0, joins v0 and v1, closing the loop);
    # the square (L 0) kills that loop.
    p = oracle_mod.persistence(np.zeros((2, 2), np.float32))
    assert cellset(p) == {(0, 1, 5), (0, 0, 4), (0, 2, 2), (0, 3, -1), (1, 0, 0)}


def test_argmax_vertex_on_ties_by_hand(oracle_mod):
    # A cube's value is the value of its vertex that enters the filtration last
    # (V-construction, Sec. 2).  Among equal values larger L enters first (the
    # reverse of the (-value, m, z, y, x) order), so among tied vertices the one
    # with the smallest linear index enters last and carries the value.
    av = oracle_mod.argmax_vertex
    one = np.array([1.0, 1.0], np.float32)
    assert av(one, 1, 0) == 0  # edge {0, 1}: vertex 1 enters before vertex 0
    assert av(one, 0, 1) == 1  # a vertex is its own argmax
    # 2x2 image (index y*2 + x): [[1, 1], [0, 1]]
    img = np.array([[1.0, 1.0], [0.0, 1.0]], np.float32)
    assert av(img, 2, 0) == 0  # square: vertices 0, 1, 3 tie at 1, vertex 0 is last
    assert av(img, 1, 0) == 0  # x-edge at y=0 (L 0): vertices 0, 1 tie
    assert av(img, 1, 2) == 3  # x-edge at y=1 (L 2): vertex 3 (value 1) over vertex 2 (value 0)
    assert av(img, 1, 5) == 1  # y-edge at x=1 (L (1*2+0)*2+1): vertices 1, 3 tie
    assert av(img, 1, 4) == 0  # y-edge at x=0 (L 4): vertex 0 (value 1) over vertex 2 (value 0)
    # 2x2x2 cube of equal values: the cube's value is carried by vertex 0
    assert av(np.ones((2, 2, 2), np.float32), 3, 0) == 0
    # -0.0 and +0.0 are one value, so they tie as well
    assert av(np.array([0.0, -0.0], np.float32), 1, 0) == 0


def test_gradient_on_ties_by_hand(oracle_mod):
    # [1, 1]: vertices enter as v1, v0 (both value 1), then edge e0 joins them;
    # v0 entered later and dies: pair (v0, e0) of length 0; v1 is essential.
    img = np.array([1.0, 1.0], np.float32)
    p = oracle_mod.persistence(img)
    assert cellset(p) == {(0, 0, 0), (0, 1, -1)}
    rows = {(int(d), int(b), int(e)): k for k, (d, b, e) in enumerate(zip(p["dim"], p["birth_L"], p["death_L"]))}
    gb = np.zeros(len(p), np.float32)
    gd = np.zeros(len(p), np.float32)
    gb[rows[(0, 0, 0)]], gd[rows[(0, 0, 0)]] = 3.0, 5.0
    gb[rows[(0, 1, -1)]], gd[rows[(0, 1, -1)]] = 7.0, 11.0  # an essential death contributes nothing
    # dL/dbirth of (v0, e0) goes to v0; dL/ddeath to the edge's last vertex, v0 again
    assert oracle_mod.gradient(img, p, gb, gd).tolist() == [8.0, 7.0]
    # 2x2 all equal: pairs (v1, e5), (v0, e4), (v2, e2), v3 essential and (e0, square 0)
    # (hand-derived in test_tie_order_by_hand).  Every edge and the square is carried
    # by its smallest vertex: e5 = {1, 3} -> 1, e4 = {0, 2} -> 0, e2 = {2, 3} -> 2,
    # e0 = {0, 1} -> 0, the square -> 0.
    img = np.zeros((2, 2), np.float32)
    p = oracle_mod.persistence(img)
    gb = np.zeros(len(p), np.float32)
    gd = np.zeros(len(p), np.float32)
    want = np.zeros(4)
    births = {(0, 1): 1, (0, 0): 0, (0, 2): 2, (0, 3): 3, (1, 0): 0}
    deaths = {(0, 5): 1, (0, 4): 0, (0, 2): 2, (1, 0): 0}
    for k in range(len(p)):
        d, bl, dl = int(p["dim"][k]), int(p["birth_L"][k]), int(p["death_L"][k])
        gb[k], gd[k] = 2.0 ** k, 2.0 ** (k + 8)
        want[births[(d, bl)]] += gb[k]
        if dl >= 0:
            want[deaths[(d, dl)]] += gd[k]
    assert oracle_mod.gradient(img, p, gb, gd).reshape(-1).tolist() == want.tolist()


def test_pair_table_by_hand(oracle_mod):
    # 1D [0, 2, 1, 3]: the component born at vertex 2 (value 1) dies at the edge
    # (0, 1) of value 2 (the equal-valued edge (1, 2) enters first and kills the
    # younger vertex 1 at zero length); vertex 0 is essential.
    p = oracle_mod.persistence(np.array([0, 2, 1, 3], np.float32))
    p = p[p["birth"] != p["death"]]
    rows = sorted(map(tuple, oracle_mod.pair_table((4,), p).tolist()))
    assert rows == [(0.0, 0.0, float("inf"), 0.0, 0.0, 0.0), (0.0, 1.0, 2.0, 2.0, 0.0, 0.0)]
    rows = sorted(map(tuple, oracle_mod.pair_table((4,), p, "death").tolist()))
    assert rows == [(0.0, 0.0, float("inf"), 0.0, 0.0, 0.0), (0.0, 1.0, 2.0, 0.0, 0.0, 0.0)]
    # 2D [[0, 5, 1], [5, 5, 5]] (rows y, columns x).  At value 5 the vertices
    # enter (L 5, 4, 3, 1), then the edges by descending L: y-edges 8, 7, 6 and
    # x-edges 4, 3, 1, 0 (L = (m*Ny + y)*Nx + x).  Edge 3, the x-edge anchored
    # at (x 0, y 1), joins the component of vertex 0 (born 0) with the one of
    # vertex 2 (born 1): [1, 5) is born at (x 2, y 0) and dies at (x 0, y 1).
    img = np.array([[0, 5, 1], [5, 5, 5]], np.float32)
    p = oracle_mod.persistence(img)
    assert (0, 2, 3) in cellset(p)
    p = p[p["birth"] != p["death"]]
    rows = sorted(map(tuple, oracle_mod.pair_table(img.shape, p).tolist()))
    assert rows == [(0.0, 0.0, float("inf"), 0.0, 0.0, 0.0), (0.0, 1.0, 5.0, 2.0, 0.0, 0.0)]
    rows = sorted(map(tuple, oracle_mod.pair_table(img.shape, p, "death").tolist()))
    assert rows == [(0.0, 0.0, float("inf"), 0.0, 0.0, 0.0), (0.0, 1.0, 5.0, 0.0, 1.0, 0.0)]
