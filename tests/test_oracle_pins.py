"""Pins for the CPU oracle: each test checks it against something other than itself --
values the paper prints, closed forms, textbook facts of discrete Morse theory, brute
force on tiny inputs, or hand-built fields whose expected edit follows from the paper's
case descriptions (Sec. 4.3 / 4.4)."""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2409_17346_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------------------
# helpers written from the definitions, independent of the oracle's C code
# --------------------------------------------------------------------------------------

def _coords(v, nx, ny):
    return v % nx, (v // nx) % ny, v // (nx * ny)


def _adj(u, v, nx, ny):
    a = np.array(_coords(u, nx, ny))
    b = np.array(_coords(v, nx, ny))
    d = b - a
    return u != v and (np.all((d >= 0) & (d <= 1)) or np.all((d <= 0) & (d >= -1)))


def _rows_to_sets(rows):
    return {tuple(int(x) for x in r if x >= 0) for r in rows}


def _pairs_dict(field):
    """cell (tuple of ids) -> partner (tuple), from the oracle's pair list"""
    d = {}
    for r in oracle.gradient_pairs(field):
        L = tuple(int(x) for x in r[:4] if x >= 0)
        U = tuple(int(x) for x in r[4:] if x >= 0)
        d[L] = U
        d[U] = L
    return d


def _crit_counts(field, dim):
    _, d = oracle.critical_cells(field)
    return np.bincount(d, minlength=dim + 1)


# --------------------------------------------------------------------------------------
# worked example (Sec. 3.1, Fig. 3)
# --------------------------------------------------------------------------------------

def _read_golden(name):
    vals, pairs, crit = {}, [], []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "pair_f":
                pairs.append((tok[1], tok[2]))
            elif tok[0] == "critical_fhat":
                crit.append(tok[1])
            else:
                vals[tok[0]] = (float(tok[1]), float(tok[2]))
    return vals, pairs, crit


def test_worked_example_sec3_1():
    vals, pairs, crit = _read_golden("worked_example_sec3_1.txt")
    # embed triangle ijk as triangle {0,1,3} of a 2x2 grid; vertex 2 is far above
    ids = {"k": 0, "j": 1, "i": 3}
    f = np.full(4, 10.0, np.float32)
    fh = np.full(4, 10.0, np.float32)
    for name, v in ids.items():
        f[v], fh[v] = vals[name]
    f = f.reshape(2, 2)
    fh = fh.reshape(2, 2)
    P = _pairs_dict(f)
    for vname, ename in pairs:
        edge = tuple(sorted(ids[c] for c in ename))
        assert P[(ids[vname],)] == edge
    cells, dims = oracle.critical_cells(fh)
    crit_vertices = {int(c[0]) for c, d in zip(cells, dims) if d == 0}
    for name in crit:
        assert ids[name] in crit_vertices
    # the FPmin j of the example is fixed by lowering the extra vertex of j's f-partner (k)
    cases, _ = oracle.targets(f, fh, pass_=0)
    rows = {tuple(int(x) for x in r[1:] if x >= 0): int(r[0]) for r in cases}
    assert rows[(ids["j"],)] == ids["k"]


# --------------------------------------------------------------------------------------
# the complex (Sec. 4.8.1: N1 ~ 7 N0, N2 ~ 12 N0, N3 ~ 6 N0 in 3D)
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(2, 2, 1), (3, 2, 1), (5, 4, 1), (2, 2, 2), (3, 4, 2), (4, 3, 5)])
def test_cell_counts_closed_form(dims):
    nx, ny, nz = dims
    rows = oracle.cells(nx, ny, nz)
    nv = (rows >= 0).sum(axis=1)
    counts = np.bincount(nv - 1, minlength=4)
    if nz == 1:
        e = (nx - 1) * ny + nx * (ny - 1) + (nx - 1) * (ny - 1)
        t = 2 * (nx - 1) * (ny - 1)
        assert list(counts[:3]) == [nx * ny, e, t] and counts[3] == 0
    else:
        a, b, c = nx - 1, ny - 1, nz - 1
        e = a * ny * nz + nx * b * nz + nx * ny * c + a * b * nz + a * ny * c + nx * b * c + a * b * c
        tets = 6 * a * b * c
        tris = 1 - nx * ny * nz + e + tets      # Euler characteristic of a box is 1
        assert list(counts) == [nx * ny * nz, e, tris, tets]


@pytest.mark.parametrize("dims", [(3, 3, 1), (2, 3, 2), (3, 3, 3)])
def test_cells_are_exactly_the_cliques(dims):
    """The Kuhn cells are the cliques of the neighbour graph (the complex is a flag complex)."""
    nx, ny, nz = dims
    n = nx * ny * nz
    adj = {v: {w for w in range(n) if _adj(v, w, nx, ny)} for v in range(n)}
    cliques = set()
    for v in range(n):
        cliques.add((v,))
        for k in (2, 3, 4):
            for comb in itertools.combinations(sorted(adj[v] | {v}), k):
                if v != comb[0]:
                    continue
                if all(b in adj[a] for a, b in itertools.combinations(comb, 2)):
                    cliques.add(comb)
    assert _rows_to_sets(oracle.cells(nx, ny, nz)) == cliques


# --------------------------------------------------------------------------------------
# pairing: closed-form rules (Sec. 4.2) == brute-force Eq. 1 + lowest cofacet (Sec. 3.1)
# --------------------------------------------------------------------------------------

_SHAPES = [(2, 2), (3, 3), (4, 3), (3, 5), (5, 5), (2, 2, 2), (3, 3, 2), (2, 3, 4), (3, 3, 3), (4, 4, 3)]


@pytest.mark.parametrize("shape", _SHAPES)
@pytest.mark.parametrize("kind", ["normal", "equal", "binary", "signed_zero", "few_levels"])
def test_rules_equal_brute_force(shape, kind):
    rng = np.random.default_rng(hash((shape, kind)) % 2**32)
    shp = shape[::-1]
    for rep in range(3):
        if kind == "normal":
            a = rng.standard_normal(shp)
        elif kind == "equal":
            a = np.zeros(shp)
        elif kind == "binary":
            a = rng.integers(0, 2, shp).astype(float)
        elif kind == "signed_zero":
            a = np.where(rng.random(shp) < 0.5, -0.0, 0.0) + (rng.random(shp) < 0.2)
        else:
            a = rng.integers(0, 4, shp).astype(float) * 0.25
        a = a.astype(np.float32)
        assert np.array_equal(oracle.gradient_pairs(a), oracle.gradient_pairs(a, brute=True))


def test_pairs_are_a_matching_of_facet_pairs():
    rng = np.random.default_rng(7)
    for shp in [(6, 7), (4, 5, 3)]:
        a = rng.standard_normal(shp).astype(np.float32)
        seen = set()
        for r in oracle.gradient_pairs(a):
            L = tuple(x for x in r[:4] if x >= 0)
            U = tuple(x for x in r[4:] if x >= 0)
            assert len(U) == len(L) + 1 and set(L) < set(U)
            assert L not in seen and U not in seen
            seen.add(L)
            seen.add(U)


def test_gradient_is_acyclic():
    """V-paths never close: the Hasse diagram with gradient pairs reversed is a DAG."""
    rng = np.random.default_rng(11)
    for shp in [(5, 6), (3, 4, 4)]:
        a = rng.integers(0, 3, shp).astype(np.float32)
        P = _pairs_dict(a)
        cells = _rows_to_sets(oracle.cells(*shp[::-1], *([1] if len(shp) == 2 else [])))
        edges = {c: [] for c in cells}
        for U in cells:
            for i in range(len(U)):
                L = U[:i] + U[i + 1:]
                if not L:
                    continue
                if P.get(L) == U:
                    edges[L].append(U)        # paired: point upward
                else:
                    edges[U].append(L)        # unpaired facet: point downward
        state = {}

        def dfs(c):
            state[c] = 1
            for d in edges[c]:
                if state.get(d) == 1:
                    return False
                if d not in state and not dfs(d):
                    return False
            state[c] = 2
            return True

        import sys
        sys.setrecursionlimit(100000)
        assert all(dfs(c) for c in cells if c not in state)


# --------------------------------------------------------------------------------------
# critical cells: Euler characteristic, SoS special cases, fields with known counts
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(8, 9), (13, 4), (4, 5, 6), (7, 3, 3)])
def test_euler_characteristic(shape):
    rng = np.random.default_rng(5)
    for kind in range(3):
        a = [rng.standard_normal(shape), rng.integers(0, 2, shape) * 1.0, np.zeros(shape)][kind]
        c = _crit_counts(a.astype(np.float32), len(shape))
        assert sum((-1) ** d * c[d] for d in range(len(c))) == 1


@pytest.mark.parametrize("shape", [(4, 6), (5, 3, 4)])
def test_constant_field_is_the_index_ramp(shape):
    """With all values equal SoS orders vertices by index: one minimum at vertex 0, no
    other critical cell, and exactly the pairs of the field f_v = v."""
    const = np.zeros(shape, np.float32)
    ramp = np.arange(const.size, dtype=np.float32).reshape(shape)
    cells, dims = oracle.critical_cells(const)
    assert len(cells) == 1 and dims[0] == 0 and cells[0][0] == 0
    assert np.array_equal(oracle.gradient_pairs(const), oracle.gradient_pairs(ramp))


def test_pairing_depends_on_order_only():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((6, 5, 4)).astype(np.float32)
    ranks = np.argsort(np.argsort(a.reshape(-1), kind="stable"), kind="stable").reshape(a.shape)
    assert np.array_equal(oracle.gradient_pairs(a), oracle.gradient_pairs(ranks.astype(np.float32)))
    assert np.array_equal(oracle.gradient_pairs(a), oracle.gradient_pairs((a * 3 + 1).astype(np.float32)))


def test_single_peak_and_bowl_counts():
    """Fields whose critical cells follow from the geometry.  Q(d) = dx^2 + dy^2 - dx dy is
    the quadratic form under which all six neighbours of a vertex of the 2D triangulation
    are at distance 1, so a Q-radial peak has a lower link on which the field is linear:
    one interior maximum, the four box corners as minima, and by the Euler characteristic
    four saddles.  A bowl (2D or 3D) flows to one interior minimum and out through the
    boundary: one minimum and nothing else."""
    for n in (9, 12):
        y, x = np.mgrid[0:n, 0:n].astype(float)
        dx, dy = x - n / 2 + 0.137, y - n / 2 + 0.291
        Q = dx * dx + dy * dy - dx * dy
        assert list(_crit_counts((-Q).astype(np.float32), 2)) == [4, 4, 1]
        assert list(_crit_counts(Q.astype(np.float32), 2)) == [1, 0, 0]
    for n in (6, 7):
        z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(float)
        r2 = (x - n / 2 + 0.137) ** 2 + (y - n / 2 + 0.291) ** 2 + (z - n / 2 + 0.173) ** 2
        assert list(_crit_counts(r2.astype(np.float32), 3)) == [1, 0, 0, 0]


# --------------------------------------------------------------------------------------
# separatrices: brute-force V-path enumeration from the pair list
# --------------------------------------------------------------------------------------

def _brute_paths(field, nx, ny, nz):
    P = _pairs_dict(field)
    cells = _rows_to_sets(oracle.cells(nx, ny, nz))
    dim = 3 if nz > 1 else 2
    crit = {c for c in cells if c not in P}
    cof = {c: [] for c in cells}
    for U in cells:
        for i in range(len(U)):
            L = U[:i] + U[i + 1:]
            if L:
                cof[L].append(U)
    desc, asc = [], []
    for s in sorted(crit):
        if len(s) == 2:
            for start in s:
                seq, u = [], (start,)
                while u not in crit:           # alternate vertex -> paired edge -> vertex
                    e = P[u]
                    seq.append((u, e))
                    u = tuple(x for x in e if x not in u)
                desc.append((s, (start,), len(seq), u))
        if len(s) == dim:
            for beta in sorted(cof[s]):
                seq, b = [], beta
                while True:                    # alternate top cell -> paired facet -> cofacet
                    if b in crit:
                        term = b
                        break
                    a = P[b]
                    seq.append((a, b))
                    nxt = [c for c in cof[a] if c != b]
                    if not nxt:
                        term = a
                        break
                    b = nxt[0]
                asc.append((s, beta, len(seq), term))
    return desc, asc


@pytest.mark.parametrize("shape", [(7, 8), (6, 5, 4)])
def test_separatrices_match_brute_force(shape):
    rng = np.random.default_rng(17)
    a = rng.standard_normal(shape).astype(np.float32)
    dims = shape[::-1] + ((1,) if len(shape) == 2 else ())
    desc, asc = _brute_paths(a, *dims)

    def rows(kind):
        out = set()
        for r in oracle.separatrices(a, kind):
            t = lambda q: tuple(int(x) for x in q if x >= 0)
            out.add((t(r[0:4]), t(r[4:8]), int(r[8]), t(r[9:13])))
        return out

    assert rows(0) == set(desc)
    assert rows(1) == set(asc)
    assert len(desc) > 0 and len(asc) > 0


# --------------------------------------------------------------------------------------
# edit arithmetic (Eq. 2, Sec. 4.7)
# --------------------------------------------------------------------------------------

def test_edit_values_exact_case():
    """f = 1, f_hat = 1.125, xi = 0.25, q_max = 2: step 1/16; every value exact."""
    lb, ub, fc, qv = oracle.edit_values(np.float32([1.0]), np.float32([1.125]), 0.25, 2)
    assert lb[0] == 0.75 and ub[0] == 1.25 and fc[0] == 1.125
    assert list(qv[0]) == [1.125, 1.0625, 1.0]


def test_edit_values_clamp_and_signed_zero():
    f = np.float32([0.5, 0.5, -0.25, 0.25])
    fh = np.float32([2.0, -2.0, 0.0, 0.0])
    lb, ub, fc, _ = oracle.edit_values(f, fh, 0.25, 3)
    assert fc[0] == ub[0] == 0.75 and fc[1] == lb[1] == 0.25
    # exact zero bounds: f - xi rounds toward +inf (+0), f + xi toward -inf (-0)
    assert ub[2] == 0.0 and np.signbit(ub[2])
    assert lb[3] == 0.0 and not np.signbit(lb[3])


def test_edit_bounds_are_tight_and_safe():
    """lb is the smallest float >= f - xi and ub the largest float <= f + xi, exactly."""
    rng = np.random.default_rng(23)
    f = np.concatenate([rng.standard_normal(2000), rng.uniform(-1e-38, 1e-38, 200),
                        [1.0, -1.0, 2.0 ** -126, -(2.0 ** -149), 0.0, -0.0, 3.0e-39]]).astype(np.float32)
    for xi in (1e-3, 2.0 ** -20, 3.3e-7, 1e-39):
        xi = float(np.float32(xi))
        lb, ub, _, _ = oracle.edit_values(f, f, xi, 6)
        for i in range(len(f)):
            lo = Fraction(float(f[i])) - Fraction(xi)
            hi = Fraction(float(f[i])) + Fraction(xi)
            assert Fraction(float(lb[i])) >= lo
            assert Fraction(float(np.nextafter(lb[i], np.float32(-np.inf)))) < lo
            assert Fraction(float(ub[i])) <= hi
            assert Fraction(float(np.nextafter(ub[i], np.float32(np.inf)))) > hi


def test_quantised_values_are_rounded_steps():
    """value_q is the float nearest to fc - fl(q * step), monotone in q, within one rounding."""
    rng = np.random.default_rng(29)
    f = rng.uniform(-3, 3, 500).astype(np.float32)
    fh = (f + rng.uniform(-1e-3, 1e-3, 500)).astype(np.float32)
    xi = float(np.float32(1e-3))
    _, _, fc, qv = oracle.edit_values(f, fh, xi, 6)
    step = Fraction(xi) / 64
    for i in range(len(f)):
        assert all(qv[i, q + 1] <= qv[i, q] for q in range(6))
        for q in range(7):
            exact = Fraction(float(fc[i])) - q * step
            ulp = Fraction(float(np.spacing(np.float32(abs(float(exact)) + 1e-30))))
            assert abs(Fraction(float(qv[i, q])) - exact) <= ulp


# --------------------------------------------------------------------------------------
# false-case rules on hand-built fields (Sec. 4.3)
# --------------------------------------------------------------------------------------

def _case_target(f, g, cell, pass_=0, tier=4):
    cases, _ = oracle.targets(np.float32(f), np.float32(g), pass_=pass_, tier=tier)
    found = [int(r[0]) for r in cases if tuple(int(x) for x in r[1:] if x >= 0) == cell]
    assert len(found) == 1, (cell, cases)
    return found[0]


RAMP = np.arange(9, dtype=np.float32).reshape(3, 3)     # 3x3 grid, vertex id = x + 3 y


def test_fp_min_lowers_partner():
    """FPmin: vertex 4 pairs with edge {0,4} in f; in g it is a minimum -> lower 0."""
    g = RAMP.copy(); g[1, 1] = -1
    assert _case_target(RAMP, g, (4,)) == 0


def test_fn_min_lowers_itself():
    """FNmin: vertex 0 is a minimum in f but paired in g -> lower vertex 0."""
    g = RAMP.copy(); g[0, 0] = 4.5
    assert _case_target(RAMP, g, (0,)) == 0


def test_fp_1saddle_vertex_type():
    """Edge {0,4} is paired with vertex 4 in f; in g vertex 4 pairs with {4,8} and no
    triangle takes the edge, so it is critical -> lower 0 (the vertex of the edge that is
    not the f-partner vertex)."""
    g = RAMP.copy(); g[2, 2] = -0.5
    assert _case_target(RAMP, g, (0, 4)) == 0


def test_fp_1saddle_triangle_type():
    """Edge {1,4} is paired with triangle {0,1,4} in f; in g it is critical -> lower 0,
    the extra vertex of the f-partner triangle."""
    g = np.float32([1.5, 1, 2, 0.5, 4, 5, 6, 7, 8]).reshape(3, 3)
    assert _case_target(RAMP, g, (1, 4)) == 0


F_SADDLE = np.float32([0, 5, 1, 6, 7, 8]).reshape(2, 3)    # minima 0 and 2, saddle {1,2}


def test_fn_1saddle_vertex_type_paper_choice():
    """Saddle {1,2} (f: 2 below 1) is paired in g with vertex 2, now above 1 ->
    lower vertex 2 so that g_2 < g_1 again (the paper's FN1saddle fix)."""
    g = np.float32([0, 0.5, 1, 6, 7, 8]).reshape(2, 3)
    assert _case_target(F_SADDLE, g, (1, 2)) == 2


def test_fn_1saddle_vertex_type_repairs_facet():
    """Saddle {1,2} is paired in g with its higher vertex 1 while the order of 1 and 2 is
    still f's: lowering 1 cannot help within the bound, so the f-pairing of vertex 1
    (edge {0,1}) is repaired by lowering 0."""
    g = np.float32([1.5, 5, 1, 6, 7, 8]).reshape(2, 3)
    assert _case_target(F_SADDLE, g, (1, 2)) == 0


def test_fn_1saddle_triangle_type():
    """Saddle {1,2} is paired in g with triangle {1,2,5} -> lower the edge's f-lowest
    vertex (2)."""
    g = np.float32([0, 5, 1, 6, 7, -1]).reshape(2, 3)
    assert _case_target(F_SADDLE, g, (1, 2)) == 2


F_MAX = np.float32([0, 1, 2, 3, 8, 4, 5, 6, 7]).reshape(3, 3)  # max triangle {4,7,8}


def test_fp_max_2d():
    """Triangle {0,1,4} is paired with edge {1,4} in the ramp; in g it is a maximum ->
    lower 0, its extra vertex."""
    g = np.float32([10, 11, 2, 3, 12, 5, 6, 7, 8]).reshape(3, 3)
    assert _case_target(RAMP, g, (0, 1, 4)) == 0


def test_fn_max_2d_paper_choice():
    """Max {4,7,8} is paired in g with edge {4,7}; its f-lowest vertex 7 is lowered (one
    of the paper's choices i or k)."""
    g = np.float32([0, 1, 2, 6.5, 8, 4, 5, 6, 5.5]).reshape(3, 3)
    assert oracle.critical_cells(F_MAX)[1].tolist().count(2) == 1
    assert _case_target(F_MAX, g, (4, 7, 8)) == 7


def test_fn_max_2d_repairs_facet():
    """Max {4,7,8} is paired in g with its f-highest edge {4,8}; the edge's f-partner
    {4,5,8} is restored by lowering 5."""
    g = np.float32([0, 1, 2, 3, 8, 7.5, 5, 6, 7]).reshape(3, 3)
    assert _case_target(F_MAX, g, (4, 7, 8)) == 5


# 3D cases on a 3 x 2 x 2 grid (nx = 3, ny = 2, nz = 2), vertex id = x + 3 y + 6 z:
#   0 (0,0,0)  1 (1,0,0)  2 (2,0,0)  3 (0,1,0)  4 (1,1,0)  5 (2,1,0)
#   6 (0,0,1)  7 (1,0,1)  8 (2,0,1)  9 (0,1,1) 10 (1,1,1) 11 (2,1,1)
# Each field below is f with one (or two) vertices moved; the docstrings derive the pairs
# involved from the rules of Sec. 4.2 by hand, and the expected vertex from Sec. 4.3/4.4.

def _g3(f, moves):
    g = np.float32(f).copy()
    for v, val in moves.items():
        g[v] = val
    return g.reshape(2, 2, 3)


def _crit_set(field):
    rows, _ = oracle.critical_cells(field)
    return {tuple(int(x) for x in r if x >= 0) for r in rows}


def test_fp_2saddle_edge_type_and_fp_1saddle_triangle_type_3d():
    """f: edge {0,4} (values 4, 5) is not paired down (V(0) = {0,7}, V(4) = {4,5}) and its
    only cofacet whose extra vertex lies below both ends is {0,1,4} (vertex 1, value 3), so
    triangle {0,1,4} is paired with edge {0,4}.  Raising vertex 1 to 4.5 breaks the
    condition f_1 < f_0, f_4: the edge becomes an FP1saddle (triangle type, Sec. 4.3: lower
    the triangle's vertex l = 1) and the triangle an FP2saddle of the edge type (lower
    the vertex k = 1 that the pairing requires below the edge)."""
    f = np.float32([4, 3, 10, 9, 5, 1, 6, 0, 2, 8, 11, 7])
    g = _g3(f, {1: 4.5})
    f = f.reshape(2, 2, 3)
    P = _pairs_dict(f)
    assert P[(0, 4)] == (0, 1, 4) and (0, 4) in _crit_set(g) and (0, 1, 4) in _crit_set(g)
    assert _case_target(f, g, (0, 1, 4)) == 1
    assert _case_target(f, g, (0, 4)) == 1


def test_fp_2saddle_tet_type_and_fp_max_3d():
    """f: triangle {7,10,11} (values 5, 10, 7) is claimed by none of its edges ({7,10}
    pairs with {6,7,10}, {7,11} with {7,8,11}, {10,11} with {4,10,11}) and its one tet
    {1,7,10,11} has extra vertex 1 (value 4) below all three, so it pairs with that tet.
    Raising vertex 1 to 5.5 (above vertex 7) breaks the pair: the triangle is an
    FP2saddle of the tetrahedron type and the tet an FPmax (3D); Sec. 4.3 lowers l = 1
    for both."""
    f = np.float32([11, 4, 3, 9, 1, 8, 2, 5, 0, 6, 10, 7])
    g = _g3(f, {1: 5.5})
    f = f.reshape(2, 2, 3)
    assert _pairs_dict(f)[(7, 10, 11)] == (1, 7, 10, 11)
    assert {(7, 10, 11), (1, 7, 10, 11)} <= _crit_set(g)
    assert _case_target(f, g, (7, 10, 11)) == 1
    assert _case_target(f, g, (1, 7, 10, 11)) == 1


def test_fn_2saddle_tet_type_and_fn_max_3d():
    """f: triangle {4,10,11} (values 4, 10, 6) and tet {1,4,10,11} are critical (a
    2-saddle and a maximum).  Raising vertex 4 to 5.5 puts the tet's vertex 1 (value 5)
    below all of the triangle, so g pairs them.  FN2saddle paired with a tetrahedron: edit
    i, j or k (Sec. 4.3), here the triangle's lowest vertex in f, 4.  FNmax (3D) paired with
    triangle ijk: edit i, j or k, again the f-lowest, 4."""
    f = np.float32([1, 5, 7, 9, 4, 0, 2, 3, 8, 11, 10, 6])
    g = _g3(f, {4: 5.5})
    f = f.reshape(2, 2, 3)
    assert {(4, 10, 11), (1, 4, 10, 11)} <= _crit_set(f)
    assert _pairs_dict(g)[(4, 10, 11)] == (1, 4, 10, 11)
    assert _case_target(f, g, (4, 10, 11)) == 4
    assert _case_target(f, g, (1, 4, 10, 11)) == 4


def test_fn_2saddle_edge_type_and_fn_1saddle_triangle_type_3d():
    """f: edge {0,4} and triangle {0,1,4} are critical (vertex 1, value 3, is not below
    vertex 0, value 2).  Raising vertex 0 to 3.5 makes g pair the edge with the triangle.
    FN2saddle paired with edge ij: edit i or j; FN1saddle paired with triangle ijl: edit i
    or j (Sec. 4.3).  Both cases take vertex 0, the lowest of the edge in f."""
    f = np.float32([2, 3, 11, 8, 7, 1, 4, 0, 5, 9, 10, 6])
    g = _g3(f, {0: 3.5})
    f = f.reshape(2, 2, 3)
    assert {(0, 4), (0, 1, 4)} <= _crit_set(f)
    assert _pairs_dict(g)[(0, 4)] == (0, 1, 4)
    assert _case_target(f, g, (0, 1, 4)) == 0
    assert _case_target(f, g, (0, 4)) == 0


def test_fn_2saddle_edge_type_repairs_facet_3d():
    """f: edge {7,10} (values 10, 8) pairs with triangle {7,10,11}: of its cofacets'
    extra vertices below both ends (11: 5, 6: 6, 1: 7) vertex 11 is the lowest.  Triangle
    {6,7,10} is then a 2-saddle.  Raising vertex 11 to 6.5 lets vertex 6 win: g pairs
    {7,10} with {6,7,10} (an FN2saddle of the edge type) and {7,10,11} becomes critical
    (an FP2saddle, lower k = 11).  For the FN case the paper allows i or j (7 or 10), but
    vertex 6, the triangle's lowest in f, is already below both in g, so the reading
    repairs the facet's f-pair ({7,10}, {7,10,11}) instead: it lowers 11 as well."""
    f = np.float32([11, 7, 4, 9, 2, 3, 6, 10, 1, 0, 8, 5])
    g = _g3(f, {11: 6.5})
    f = f.reshape(2, 2, 3)
    assert _pairs_dict(f)[(7, 10)] == (7, 10, 11) and (6, 7, 10) in _crit_set(f)
    assert _pairs_dict(g)[(7, 10)] == (6, 7, 10)
    assert _case_target(f, g, (6, 7, 10)) == 11
    assert _case_target(f, g, (7, 10, 11)) == 11


def test_one_dim_troublemaker_2d():
    """1-dimensional troublemaker (Sec. 4.4) on a 4 x 4 grid (id = x + 4 y).  In f, edge
    {2,6} (values 10, 8) is not paired down and pairs with triangle {1,2,6}: vertex 1
    (value 6) is below both ends, vertex 7 of the other cofacet {2,6,7} (value 9) is not.
    The pair lies on an ascending separatrix.  In g vertex 1 rises to 9.5 and vertex 7
    falls to 2.5, so the edge pairs with {2,6,7} (the paper's ijl) while every critical
    cell stays: the S-pass lowers k = 1, and that is its only troublemaker."""
    f = np.float32([2, 6, 10, 11, 13, 4, 8, 9, 7, 3, 5, 0, 1, 15, 14, 12]).reshape(4, 4)
    g = f.copy().reshape(-1)
    g[1], g[7] = 9.5, 2.5
    g = g.reshape(4, 4)
    assert _pairs_dict(f)[(2, 6)] == (1, 2, 6) and _pairs_dict(g)[(2, 6)] == (2, 6, 7)
    assert len(oracle.targets(f, g, pass_=0)[0]) == 0
    cases, _ = oracle.targets(f, g, pass_=1, tier=4)
    assert [int(c[0]) for c in cases] == [1]
    assert _case_target(f, g, (1, 2, 6), pass_=1) == 1


def test_two_dim_troublemaker_3d():
    """2-dimensional troublemaker (Sec. 4.4).  In f, triangle {0,3,10} (values 8, 9, 11)
    pairs with tet {0,3,9,10}: vertex 9 (value 7) lies below all three, vertex 4 of the
    other tet {0,3,4,10} (value 10) does not.  The pair lies on an ascending separatrix.
    In g vertex 9 rises to 9.5 and vertex 4 falls to 6.5, so the triangle pairs with
    {0,3,4,10} (the paper's ijkq) and no critical cell changes: the S-pass lowers l = 9,
    its only troublemaker."""
    f = np.float32([8, 0, 6, 9, 10, 3, 4, 5, 2, 7, 11, 1])
    g = _g3(f, {4: 6.5, 9: 9.5})
    f = f.reshape(2, 2, 3)
    assert _pairs_dict(f)[(0, 3, 10)] == (0, 3, 9, 10) and _pairs_dict(g)[(0, 3, 10)] == (0, 3, 4, 10)
    assert len(oracle.targets(f, g, pass_=0)[0]) == 0
    cases, _ = oracle.targets(f, g, pass_=1, tier=4)
    assert [int(c[0]) for c in cases] == [9]
    assert _case_target(f, g, (0, 3, 9, 10), pass_=1) == 9


def test_one_dim_troublemaker_on_saddle_connector_3d():
    """1-dimensional troublemaker on a saddle-saddle connector (Sec. 4.4) on a 3 x 3 x 3
    grid (id = x + 3 y + 9 z).  In f, edge {15,16} (values 22, 24) pairs with triangle
    {15,16,25}: its extra vertex 25 (value 12) is the lowest below both ends, ahead of
    vertex 12 (value 13, triangle {12,15,16}); the walk from a 2-saddle crosses this pair.
    Lowering vertex 12 to 11.5 makes g pair the edge with {12,15,16}: the troublemaker is
    the edge, and the S-pass lowers k = 25.  (Triangle {12,15,16}, paired in f with tet
    {12,15,16,25} on an ascending path, is re-paired with the edge in g; that 2-dim
    troublemaker names vertex 25 too.)"""
    f = np.float32([11, 0, 9, 23, 26, 5, 17, 25, 19, 20, 18, 7, 13, 8, 14, 22, 24, 10, 3, 21, 16, 4, 6, 15,
                    1, 12, 2])
    g = f.copy()
    g[12] = 11.5
    f, g = f.reshape(3, 3, 3), g.reshape(3, 3, 3)
    assert _pairs_dict(f)[(15, 16)] == (15, 16, 25) and _pairs_dict(g)[(15, 16)] == (12, 15, 16)
    crossed = {(tuple(int(x) for x in r[5:9] if x >= 0), tuple(int(x) for x in r[9:13] if x >= 0))
               for r in oracle.saddle_connectors(f) if r[4] == 1}
    assert ((15, 16), (15, 16, 25)) in crossed
    assert len(oracle.targets(f, g, pass_=0)[0]) == 0
    cases, _ = oracle.targets(f, g, pass_=1, tier=4)
    assert {int(c[0]) for c in cases} == {25}
    assert _case_target(f, g, (15, 16, 25), pass_=1) == 25
    assert _case_target(f, g, (12, 15, 16, 25), pass_=1) == 25


@pytest.mark.parametrize("shape", [(6, 7), (4, 4, 4), (3, 5, 4)])
def test_case_rules_on_random_fields(shape):
    """For every false case of every dimension: an FP case lowers the extra vertex of the
    cell's f-partner; an FN case lowers one of the vertices of the g-pair's lower cell,
    the lowest in f (or, when the order of the cell is unchanged, repairs a facet)."""
    rng = np.random.default_rng(31)
    f = rng.standard_normal(shape).astype(np.float32)
    g = (f + rng.uniform(-0.4, 0.4, shape)).astype(np.float32)
    Pf, Pg = _pairs_dict(f), _pairs_dict(g)
    cases, _ = oracle.targets(f, g, pass_=0)
    assert len(cases) > 5
    fl = f.reshape(-1)
    gl = g.reshape(-1)
    key_f = lambda v: (fl[v], v)
    key_g = lambda v: (gl[v], v)
    for r in cases:
        t = int(r[0])
        cell = tuple(int(x) for x in r[1:] if x >= 0)
        if cell in Pf and cell not in Pg:
            U, L = (Pf[cell], cell) if len(Pf[cell]) > len(cell) else (cell, Pf[cell])
            assert t == (set(U) - set(L)).pop()
        else:
            assert cell not in Pf and cell in Pg
            P = Pg[cell]
            L = cell if len(P) > len(cell) else P
            if len(P) > len(cell) or min(cell, key=key_g) != min(cell, key=key_f):
                assert t == min(cell, key=key_f) and t in L
            else:
                Q = Pf.get(L)
                if Q is None:
                    assert t == min(L, key=key_f)
                else:
                    big, small = (Q, L) if len(Q) > len(L) else (L, Q)
                    assert t == (set(big) - set(small)).pop()


# --------------------------------------------------------------------------------------
# S-pass troublemakers (Sec. 4.4)
# --------------------------------------------------------------------------------------

def test_zero_dim_troublemaker():
    """Hand-built 0-dim troublemaker (Sec. 4.4).  In f (ids x + 4 y) vertex 6 (value 6)
    pairs with edge {6,7} (7 is its lowest lower neighbour, value 2) and lies on the
    descending separatrix of saddle {5,6}.  Swapping the values of vertices 2 and 7 leaves
    every critical cell in place but makes vertex 6 pair with {2,6}: the S-pass must lower
    j = 7 so that 6 pairs with {6,7} again, and it is the only troublemaker."""
    f = np.float32([[9, 10, 4, 1], [7, 8, 6, 2], [0, 3, 11, 5]])
    g = np.float32([[9, 10, 2, 1], [7, 8, 6, 4], [0, 3, 11, 5]])
    assert len(oracle.targets(f, g, pass_=0)[0]) == 0
    cases, _ = oracle.targets(f, g, pass_=1, tier=4)
    assert [int(c[0]) for c in cases] == [7]
    assert _case_target(f, g, (6, 7), pass_=1) == 7


def test_troublemakers_random_descending():
    """Perturb one vertex on a descending separatrix of a random field so that it pairs
    with a different lower neighbour while the critical cells stay the same; the S-pass
    must then lower the original partner of the first disagreeing vertex."""
    rng = np.random.default_rng(41)
    hits = 0
    for trial in range(200):
        f = rng.standard_normal((7, 7)).astype(np.float32)
        Pf = _pairs_dict(f)
        rows = oracle.separatrices(f, 0)
        rows = [r for r in rows if r[8] >= 2]
        if not rows:
            continue
        r = rows[int(rng.integers(0, len(rows)))]
        # walk the f-path: u0 -> ... ; pick the first vertex of the path
        u = int(r[4])
        w = (set(Pf[(u,)]) - {u}).pop()
        fl = f.reshape(-1)
        lower = [v for v in range(f.size) if _adj(u, v, 7, 7) and (fl[v], v) < (fl[u], u) and v != w]
        if not lower:
            continue
        v2 = lower[0]
        g = f.copy().reshape(-1)
        g[v2] = np.nextafter(fl[w], np.float32(-np.inf))
        g = g.reshape(f.shape)
        if len(oracle.targets(f, g, pass_=0)[0]):
            continue
        Pg = _pairs_dict(g)
        if Pg.get((u,)) == Pf[(u,)]:
            continue
        cases, _ = oracle.targets(f, g, pass_=1, tier=4)
        assert w in {int(c[0]) for c in cases}
        hits += 1
    assert hits >= 3


# --------------------------------------------------------------------------------------
# the whole loop: invariants and final MSC equality (Sec. 4.1, 4.5)
# --------------------------------------------------------------------------------------

def _exact_bound_ok(f, g, xi):
    fl, gl = f.reshape(-1).astype(np.float64), g.reshape(-1).astype(np.float64)
    # differences of floats within a few binades are exact in double
    d = np.abs(gl - fl)
    return bool(np.all(d <= xi))


def _cases():
    yield synth.config_case("gauss2d")
    yield synth.config_case("gauss2d", seed=9, size=(23, 41), rel=1e-2)
    yield synth.config_case("multiscale2d", size=(40, 56), rel=1e-2)
    yield synth.config_case("grf3d", size=9, rel=1e-2)
    yield synth.config_case("kolmogorov3d", size=10, rel=3e-3)


@pytest.mark.parametrize("idx", range(5))
@pytest.mark.parametrize("tier", [1, 2, 3, 4])
def test_loop_converges_and_preserves_msc(idx, tier):
    f, fh, xi, _ = list(_cases())[idx]
    r = oracle.fix(f, fh, xi, tier=tier)
    assert r["status"] == 0
    g = r["g"]
    assert _exact_bound_ok(f, g, xi)
    rep = oracle.verify(f, g)
    dim = f.ndim
    ext = [rep["fp0"], rep["fn0"], rep["fp%d" % dim], rep["fn%d" % dim]]
    assert sum(ext) == 0
    if tier >= 2:
        assert all(rep[k] == 0 for k in ("fp0", "fp1", "fp2", "fp3", "fn0", "fn1", "fn2", "fn3"))
    if tier == 3:
        assert rep["term_desc"] == 0 and rep["term_asc"] == 0
    if tier == 4:
        assert rep["sep_desc"] == 0 and rep["sep_asc"] == 0 and rep["sep_saddle"] == 0
    c = _crit_counts(g, dim)
    assert sum((-1) ** d * c[d] for d in range(len(c))) == 1
    # the critical cells of g are exactly those of f
    if tier >= 2:
        cf, df = oracle.critical_cells(f)
        cg, dg = oracle.critical_cells(g)
        assert np.array_equal(cf, cg) and np.array_equal(df, dg)
    # stored edits rebuild g bit-exactly on the decompression side
    qm, li, lv = oracle.edits_from_state(f, fh, xi, r["state"], g)
    g2 = oracle.apply_edits(fh, xi, 6, qm, li, lv)
    assert np.array_equal(g2.view(np.uint32), g.view(np.uint32))


def test_edits_are_monotone_per_iteration():
    """g^(k+1) <= g^(k) at every vertex (Sec. 3.2) except exact-fallback restores, and
    g >= f - xi throughout, checked on every prefix of the loop."""
    f, fh, xi, tier = synth.config_case("gauss2d", seed=3, size=(20, 24), rel=2e-2)
    full = oracle.fix(f, fh, xi, tier=4)
    n = full["n_c"] + full["n_s"]
    assert n > 3
    prev = None
    for k in range(1, n + 1):
        r = oracle.fix(f, fh, xi, tier=4, max_iters=k)
        assert r["status"] in (0, 4)
        g = r["g"]
        assert _exact_bound_ok(f, g, xi)
        if prev is not None:
            ok = (g <= prev[0]) | (r["state"] == oracle.ST_EXACT)
            assert ok.all()
        prev = (g, r["state"])
    assert np.array_equal(prev[0], full["g"])


def test_stall_fallback_on_floor_ties():
    """f - xi can round two different f values to the same float; SoS then orders the
    floors by index, against f.  Vertex 1 (below vertex 0 in f) and vertex 0 tie at the
    floor: the loop must restore them to f exactly (exact fallback) or report a stall."""
    a = np.float32(-1.0 + 2.0 ** -24)        # f of vertex 1 (lower)
    b = np.float32(-1.0 + 2.0 ** -23)        # f of vertex 0 (higher)
    xi = float(np.float32(2.0 ** -23))
    lb, _, _, _ = oracle.edit_values(np.float32([a, b]), np.float32([a, b]), xi, 6)
    assert lb[0] == lb[1] == -1.0
    f = np.float32([[b, a], [10, 11]])
    fh = np.float32([[b - 0.0, a + 2 ** -24], [10, 11]])
    fh[0, 0] = lb[1]                          # vertex 0 already at its floor
    fh = fh.astype(np.float32)
    r = oracle.fix(f, fh, xi, tier=4)
    assert r["status"] == 0 and r["n_exact_iters"] >= 1
    assert oracle.verify(f, r["g"])["fp0"] == 0
    r2 = oracle.fix(f, fh, xi, tier=4, exact_fallback=0)
    assert r2["status"] == 6


def test_invalid_inputs_rejected():
    f = np.zeros((4, 4), np.float32)
    bad = f.copy(); bad[1, 1] = np.nan
    assert oracle.fix(f, bad, 0.1)["status"] == 1
    assert oracle.fix(f, f, 0.0)["status"] == 1
    assert oracle.fix(f, f, 0.1, q_max=8)["status"] == 1


# --------------------------------------------------------------------------------------
# packed edit record (Sec. 4.7: the quantised counts as a fixed-bit bitstream)
# --------------------------------------------------------------------------------------

def test_packed_record_hand_built():
    """q_max = 6 needs 3 bits (values 0..6 and the lossless escape 7).  Nine vertices with
    counts 0,1,2,3,4,5,6, lossless, 1 and one lossless value 1.5 give: the header, group 0 as
    the 24-bit integer 0 | 1<<3 | 2<<6 | 3<<9 | 4<<12 | 5<<15 | 6<<18 | 7<<21 = 0xFAC688 in three
    little-endian bytes, group 1 = 1, then 1.5f = 0x3FC00000."""
    qm = np.array([0, 1, 2, 3, 4, 5, 6, 0xFF, 1], np.uint8)
    out = oracle.pack_edits(qm, 6, np.float32([1.5]))
    head = b"MSCE" + bytes([1, 6, 3, 0]) + (9).to_bytes(8, "little") + (1).to_bytes(8, "little") + bytes(8)
    body = bytes([0x88, 0xC6, 0xFA, 0x01, 0x00, 0x00]) + bytes([0x00, 0x00, 0xC0, 0x3F])
    assert out.tobytes() == head + body
    assert oracle.packed_bytes(9, 1, 6) == len(head + body)


@pytest.mark.parametrize("q_max", [1, 2, 3, 6, 7])
def test_packed_record_round_trip(q_max):
    rng = np.random.default_rng(40 + q_max)
    n = 1000 + q_max
    qm = rng.integers(0, q_max + 1, n).astype(np.uint8)
    qm[rng.random(n) < 0.1] = 0xFF
    lv = rng.standard_normal(int((qm == 0xFF).sum())).astype(np.float32)
    buf = oracle.pack_edits(qm, q_max, lv)
    bits = {1: 2, 2: 2, 3: 3, 6: 3, 7: 4}[q_max]
    assert buf.size == 32 + ((n + 7) // 8) * bits + 4 * lv.size
    qm2, li2, lv2, q2 = oracle.unpack_edits(buf)
    assert q2 == q_max and np.array_equal(qm2, qm)
    assert np.array_equal(li2, np.nonzero(qm == 0xFF)[0]) and np.array_equal(lv2.view(np.uint32), lv.view(np.uint32))


def test_packed_record_rejects_bad_input():
    with pytest.raises(RuntimeError):
        oracle.pack_edits(np.array([0, 9], np.uint8), 6, np.zeros(0, np.float32))   # count above q_max
    with pytest.raises(RuntimeError):
        oracle.pack_edits(np.array([0xFF], np.uint8), 6, np.zeros(0, np.float32))   # missing value
    buf = oracle.pack_edits(np.array([1, 2], np.uint8), 6, np.zeros(0, np.float32))
    with pytest.raises(RuntimeError):
        oracle.unpack_edits(buf[:-1])


def test_packed_record_rebuilds_the_fix():
    f, fh, xi, _ = synth.config_case("gauss2d", seed=3)
    r = oracle.fix(f, fh, xi, tier=3)
    qm, li, lv = oracle.edits_from_state(f, fh, xi, r["state"], r["g"])
    qm2, li2, lv2, q = oracle.unpack_edits(oracle.pack_edits(qm, 6, lv))
    g = oracle.apply_edits(fh, xi, q, qm2, li2, lv2)
    assert np.array_equal(g.view(np.uint32), r["g"].view(np.uint32))


def _nb_and_ring_offsets(ndim):
    """Neighbour offsets of the Freudenthal grid and the offsets within two edges."""
    if ndim == 2:
        nb = [(1, 0, 0), (0, 1, 0), (1, 1, 0)]
    else:
        nb = [(A & 1, (A >> 1) & 1, (A >> 2) & 1) for A in range(1, 8)]
    nb = nb + [tuple(-c for c in o) for o in nb]
    ring = set(nb) | {tuple(a[i] + b[i] for i in range(3)) for a in nb for b in nb}
    ring.discard((0, 0, 0))
    return set(nb), ring


def test_gradient_depends_only_on_orders_within_two_edges():
    """Every comparison the pairing rules make (Sec. 4.2) is between two vertices within two
    edges of each other: two neighbours of a vertex, two cofacet candidates of an edge or a
    triangle, two vertices of a cell.  So moving one vertex's value without crossing any
    vertex within two edges (in SoS order) leaves the gradient unchanged, checked here both
    with the closed-form rules and by brute force on Eq. 1.  Crossing a single vertex two
    edges away that is not a neighbour does change it on some fields, so the neighbours
    alone would not do.  (The GPU loop skips the refresh of edits that cross nothing.)"""
    rng = np.random.default_rng(23)
    kept = changed = tried = 0
    for trial in range(240):
        ndim = 2 if trial % 2 else 3
        shape = tuple(int(s) for s in (rng.integers(4, 7, 2) if ndim == 2 else rng.integers(3, 6, 3)))
        a = rng.standard_normal(shape).astype(np.float32)
        flat = a.reshape(-1)
        nx, ny = shape[-1], shape[-2]
        nz = 1 if ndim == 2 else shape[0]
        nbs, ring = _nb_and_ring_offsets(ndim)
        v = int(rng.integers(0, flat.size))
        x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
        parts = []
        for o in ring:
            X, Y, Z = x + o[0], y + o[1], z + o[2]
            if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz:
                parts.append((X + nx * (Y + ny * Z), o in nbs))
        key = lambda u: (float(flat[u]), u)
        brute = trial % 4 == 0
        # a new value strictly between the nearest partners below and above: no order changes
        lo = max([float(flat[u]) for u, _ in parts if key(u) < key(v)] + [float(flat[v]) - 4])
        hi = min([float(flat[u]) for u, _ in parts if key(u) > key(v)] + [float(flat[v]) + 4])
        w = np.float32(rng.uniform(lo, hi)) if lo < hi else None
        if w is not None and lo < w < hi:
            g = flat.copy()
            g[v] = w
            assert np.array_equal(oracle.gradient_pairs(g.reshape(shape), brute=brute),
                                  oracle.gradient_pairs(a, brute=brute)), trial
            kept += 1
        # just past the nearest non-neighbour partner above, with no neighbour in between
        far = sorted([u for u, isnb in parts if not isnb and key(u) > key(v)], key=key)
        if far and not [p for p, isnb in parts if isnb and key(v) < key(p) <= key(far[0])]:
            u = far[0]
            hi2 = min([float(flat[p]) for p, _ in parts if key(p) > key(u)] + [float(flat[u]) + 1])
            w = np.float32((float(flat[u]) + hi2) / 2)
            if float(flat[u]) < w < hi2:
                g = flat.copy()
                g[v] = w
                tried += 1
                changed += not np.array_equal(oracle.gradient_pairs(g.reshape(shape)), oracle.gradient_pairs(a))
    assert kept > 200 and tried > 100 and changed > 0


# --------------------------------------------------------------------------------------
# saddle-saddle connectors (Sec. 3.1 V-paths, Sec. 4.4): brute-force enumeration of every
# alternating triangle -> facet edge -> paired triangle sequence from each 2-saddle
# --------------------------------------------------------------------------------------

def _facets(cell):
    return [cell[:i] + cell[i + 1:] for i in range(len(cell))]


def _brute_connector_paths(P, crit, saddle, limit=200000):
    """Every V-path of a gradient (pair dict P) from 2-saddle triangle `saddle`, by plain
    recursion without a visited set (V is acyclic, so every path ends).  A path is a list
    of items: ("cross", e, t') for a facet edge e paired up with another triangle t',
    ("dead", e, v) for a facet edge paired down with vertex v (the path ends there), and
    ("saddle", e, None) for a critical facet edge (a 1-saddle: the path ends there)."""
    paths = []

    def rec(t, prefix):
        if len(paths) > limit:
            raise RuntimeError("too many V-paths")
        for e in _facets(t):
            if e in crit:
                paths.append(prefix + [("saddle", e, None)])
                continue
            p = P[e]
            if len(p) == 1:
                paths.append(prefix + [("dead", e, p)])
                continue
            if p == t:           # e is the pair that brought the path into t
                continue
            rec(p, prefix + [("cross", e, p)])

    rec(saddle, [])
    return paths


def _connector_fields():
    rng = np.random.default_rng(61)
    out = []
    for shape in [(3, 3, 3), (4, 3, 4), (4, 4, 4), (5, 4, 3), (5, 5, 5)]:
        out.append(("normal", rng.standard_normal(shape).astype(np.float32)))
        out.append(("binary", rng.integers(0, 2, shape).astype(np.float32)))
        out.append(("few_levels", rng.integers(0, 4, shape).astype(np.float32)))
    return out


@pytest.mark.parametrize("idx", range(15))
def test_saddle_connectors_match_brute_force(idx):
    """From every 2-saddle, the oracle's walk reaches exactly the 1-saddles, crosses
    exactly the (edge, triangle) pairs and stops at exactly the dead-end edges that the
    enumeration of every V-path of V_f from that 2-saddle does (per 2-saddle, so a walk
    that shared visited marks between 2-saddles, crossed a pair backwards or skipped a
    dead end would differ)."""
    kind, f = _connector_fields()[idx]
    nz, ny, nx = f.shape
    P = _pairs_dict(f)
    cells = _rows_to_sets(oracle.cells(nx, ny, nz))
    crit = {c for c in cells if c not in P}
    t = lambda q: tuple(int(x) for x in q if x >= 0)
    got = {}
    for r in oracle.saddle_connectors(f):
        got.setdefault(t(r[0:4]), set()).add((int(r[4]), t(r[5:9]), t(r[9:13])))
    want = {}
    code = {"saddle": 0, "cross": 1, "dead": 2}
    for s in sorted(c for c in crit if len(c) == 3):
        items = set()
        for path in _brute_connector_paths(P, crit, s):
            for what, e, other in path:
                items.add((code[what], e, other if other is not None else ()))
        want[s] = items
    assert set(got) == set(want)
    for s in want:
        assert got[s] == want[s], s
    if kind == "normal" and f.size >= 64:
        assert any(any(k == 1 for k, _, _ in v) for v in want.values())


def _brute_s_cases(f, g):
    """The S-pass at tier 4 restated from exhaustive path enumeration on the pair lists of
    f and g (Sec. 4.4): along every separatrix of f, the first pair (L, U) that g's
    gradient does not have is a troublemaker, and the vertex U \\ L is lowered.  On a
    saddle-saddle path a dead-end edge e paired down with v in f is kept as long as g also
    pairs e down; otherwise its f-pair (v, e) is the troublemaker.  Returns the set of
    (target vertex, case cell)."""
    nz, ny, nx = f.shape if f.ndim == 3 else (1,) + f.shape
    dims = (nx, ny, nz)
    Pf, Pg = _pairs_dict(f), _pairs_dict(g)
    cells = _rows_to_sets(oracle.cells(*dims))
    crit = {c for c in cells if c not in Pf}
    top = 3 if nz > 1 else 2
    cof = {c: [] for c in cells}
    for U in cells:
        for L in _facets(U):
            if L:
                cof[L].append(U)
    extra = lambda U, L: (set(U) - set(L)).pop()
    cases = set()

    def first_bad(pairs):
        for L, U in pairs:
            if Pg.get(L) != U:
                cases.add((extra(U, L), U))
                return

    for s in sorted(crit):
        if len(s) == 2:                                  # descending, one per endpoint
            for start in s:
                pairs, u = [], (start,)
                while u not in crit:
                    e = Pf[u]
                    pairs.append((u, e))
                    u = (extra(e, u),)
                first_bad(pairs)
        if len(s) == top:                                # ascending, one per top cofacet
            for beta in cof[s]:
                pairs, b = [], beta
                while b not in crit:
                    a = Pf[b]
                    pairs.append((a, b))
                    nxt = [c for c in cof[a] if c != b]
                    if not nxt:
                        break
                    b = nxt[0]
                first_bad(pairs)
        if top == 3 and len(s) == 3:                     # saddle-saddle, every V-path
            for path in _brute_connector_paths(Pf, crit, s):
                for what, e, other in path:
                    if what == "cross" and Pg.get(e) != other:
                        cases.add((extra(other, e), other))
                        break
                    if what == "dead" and len(Pg.get(e, ())) != 1:
                        cases.add((extra(e, other), e))
                        break
    return cases


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 4, 3), (3, 5, 5), (7, 9)])
def test_s_pass_targets_match_path_enumeration(shape):
    """On perturbed copies of random fields whose critical cells are unchanged, the
    oracle's S-pass (tier 4) names exactly the troublemakers that exhaustive path
    enumeration finds: the first disagreeing pair on every descending, ascending and
    saddle-saddle path of f."""
    rng = np.random.default_rng(67 + len(shape))
    checked = saddle_hits = 0
    for trial in range(6000):
        if checked >= 12 and (saddle_hits >= 3 or len(shape) == 2):
            break
        if trial % 2 == 0:       # ties: a small move re-orders only equal values
            f = rng.integers(0, 4, shape).astype(np.float32)
            scale = 0.4
        else:
            f = rng.standard_normal(shape).astype(np.float32)
            scale = 1.0
        g = f.copy().reshape(-1)
        for v in rng.choice(f.size, size=int(rng.integers(1, 3)), replace=False):
            g[v] = g[v] + np.float32(rng.uniform(-scale, scale))
        g = g.reshape(shape)
        if len(oracle.targets(f, g, pass_=0)[0]):
            continue                                     # the S-pass runs only after the C-loop
        cases, _ = oracle.targets(f, g, pass_=1, tier=4)
        got = {(int(r[0]), tuple(int(x) for x in r[1:] if x >= 0)) for r in cases}
        want = _brute_s_cases(f, g)
        assert got == want, (trial, got ^ want)
        checked += bool(want)
        saddle_hits += any(len(c) == 3 for _, c in want)
    assert checked >= 12
    if len(shape) == 3:
        assert saddle_hits >= 3


# --------------------------------------------------------------------------------------
# the oracle's parallel loops: results independent of the number of threads
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("name,kw", [("kolmogorov3d", dict(size=14, rel=1e-3)),
                                     ("multiscale2d", dict(size=(40, 72), rel=3e-3))])
def test_results_do_not_depend_on_threads(name, kw):
    f, fh, xi, _ = synth.config_case(name, **kw)
    n0 = oracle.threads()
    try:
        oracle.set_threads(1)
        one = oracle.fix(f, fh, xi, tier=4)
        vone = oracle.verify(f, np.clip(fh, f - xi, f + xi).astype(np.float32))
        oracle.set_threads(max(4, n0))
        many = oracle.fix(f, fh, xi, tier=4)
        vmany = oracle.verify(f, np.clip(fh, f - xi, f + xi).astype(np.float32))
    finally:
        oracle.set_threads(n0)
    assert one["status"] == many["status"] == 0
    assert np.array_equal(one["g"].view(np.uint32), many["g"].view(np.uint32))
    assert np.array_equal(one["state"], many["state"])
    assert np.array_equal(one["trace"], many["trace"])
    assert vone == vmany


# --------------------------------------------------------------------------------------
# floating edits (Sec. 4.7: every edit stored as a float, so no cap on the step count)
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("name,kw,tier", [("gauss2d", dict(seed=3, size=(40, 52), rel=1e-2), 3),
                                          ("kolmogorov3d", dict(size=12, rel=1e-2), 4)])
def test_floating_edits_loop(name, kw, tier):
    """The floating-edit loop converges with |f - g| <= xi and the MSC of f; every vertex that
    did not reach its floor holds exactly the value after its count of steps (Eq. 2 without
    the q_max cap), some counts exceed q_max, and the stored (index, value) pairs rebuild g."""
    f, fh, xi, _ = synth.config_case(name, **kw)
    q_max = 2
    r = oracle.fix(f, fh, xi, tier=tier, q_max=q_max, edit_mode=1)
    assert r["status"] == 0
    g, st = r["g"], r["state"].reshape(-1)
    assert _exact_bound_ok(f, g, xi)
    v = oracle.verify(f, g)
    keys = [k for k in oracle.REPORT_KEYS if k.startswith(("fp", "fn", "term"))]
    if tier == 4:
        keys = list(oracle.REPORT_KEYS)
    assert all(v[k] == 0 for k in keys), v
    lb, ub, fc, qv = oracle.edit_values(f, fh, xi, q_max, n_steps=0xEF + 1)
    quant = st <= 0xEF
    assert np.array_equal(g.reshape(-1)[quant].view(np.uint32),
                          qv[np.nonzero(quant)[0], st[quant]].view(np.uint32))
    assert np.any(quant & (st > q_max))
    q_map, idx, val = oracle.edits_from_state(f, fh, xi, r["state"], g, edit_mode=1)
    assert set(np.unique(q_map)) <= {0, 0xFF}
    assert np.array_equal(idx, np.nonzero((st > 0) | (fc.view(np.uint32) != fh.reshape(-1).view(np.uint32)))[0])
    g2 = oracle.apply_edits(fh, xi, q_max, q_map, idx, val)
    assert np.array_equal(g2.view(np.uint32), g.view(np.uint32))
    # the same loop with quantised edits snaps vertices to the floor after q_max steps
    rq = oracle.fix(f, fh, xi, tier=tier, q_max=q_max)
    assert rq["status"] == 0 and np.all((rq["state"] <= q_max) | (rq["state"] >= 0xF0))
