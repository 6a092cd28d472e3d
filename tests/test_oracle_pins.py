"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, closed forms, invariants, or a textbook special case, chosen so
that a dropped term, a wrong sign, index or vertex order fails one of them.
"""
import itertools
import math
import os
from collections import Counter

import numpy as np
import pytest

from oracle import hhg_oracle as O
from paper_1709_06793_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "stencil_level2.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, di, dj, dk, val = line.split()
        out.setdefault(name, {})[(int(di), int(dj), int(dk))] = val
    return out


def _row_at(lm, A, t, ijk):
    row = A[lm.local[t][ijk]].toarray().ravel()
    return row


@pytest.mark.parametrize("name,mesh", [("unit", I.unit_tet), ("regular", I.regular_tet)])
def test_printed_reference_stencils(name, mesh):
    """Fig. "stencilsign": the level-2 inner-node stencil, to the printed digits."""
    V, T = mesh()
    lm = O.LevelMesh(O.MacroMesh(V, T), 2)
    A = lm.assemble(np.ones(lm.n), "scaled")
    row = _row_at(lm, A, 0, (1, 1, 1))
    golden = _golden()[name]
    assert len(golden) == 15
    nnz = np.count_nonzero(np.abs(row) > 1e-13)
    assert nnz == 15
    for (di, dj, dk), txt in golden.items():
        printed = float(txt)
        mant, exp = txt.split("e")
        half_ulp = 0.5 * 10.0 ** (int(exp) - (len(mant.split(".")[1])))
        got = row[lm.local[0][1 + di, 1 + dj, 1 + dk]]
        assert abs(got - printed) <= half_ulp + 1e-15, ((di, dj, dk), got, printed)


def test_unit_tet_stencil_exact_fractions():
    """The unit-tet values of Fig. "stencilsign" are 5/3, -1/3, -1/6, -1/12 and
    +1/12 (a hand computation with the Kuhn-type micro tetrahedra)."""
    V, T = I.unit_tet()
    lm = O.LevelMesh(O.MacroMesh(V, T), 2)
    A = lm.assemble(np.ones(lm.n), "laplace")
    row = _row_at(lm, A, 0, (1, 1, 1))
    want = {(0, 0, 0): 5 / 3, (1, 0, 0): -1 / 3, (0, 0, 1): -1 / 3, (0, 1, 0): -1 / 6,
            (1, -1, 0): -1 / 12, (0, 1, -1): -1 / 12, (1, 0, -1): 1 / 12, (1, -1, 1): 1 / 12}
    for d, v in want.items():
        for s in ((1,) if d == (0, 0, 0) else (1, -1)):
            p = tuple(1 + s * x for x in d)
            assert abs(row[lm.local[0][p]] - v) < 1e-14


def test_stencil_scales_with_h():
    """In 3D int grad phi_i . grad phi_j scales like h: the inner stencil at
    level 3 is half the one at level 2 (same macro tetrahedron)."""
    V, T = I.regular_tet()
    mm = O.MacroMesh(V, T)
    l2, l3 = O.LevelMesh(mm, 2), O.LevelMesh(mm, 3)
    A2, A3 = l2.assemble(None, "laplace"), l3.assemble(None, "laplace")
    r2 = _row_at(l2, A2, 0, (1, 1, 1))
    r3 = _row_at(l3, A3, 0, (2, 2, 2))
    for d in itertools.product((-1, 0, 1), repeat=3):
        a = r2[l2.local[0][tuple(1 + np.array(d))]]
        b = r3[l3.local[0][tuple(2 + np.array(d))]]
        assert abs(b - 0.5 * a) < 1e-14


def test_bey_refinement_is_freudenthal_in_kuhn_coordinates():
    """Bey's rule with the vertex order preserved gives, in the coordinates
    (a,b,c) = (i+j+k, j+k, k), the Freudenthal-Kuhn triangulation: every unit
    cube split into the 6 simplices along its main diagonal, kept where they lie
    in N >= a >= b >= c >= 0 (the three congruence classes of Sec. 4.3)."""
    for level in (1, 2, 3):
        N = 1 << level
        mt = O.micro_tets(level)
        kuhn = np.stack([mt.sum(axis=2), mt[:, :, 1] + mt[:, :, 2], mt[:, :, 2]], axis=2)
        got = {tuple(sorted(map(tuple, t))) for t in kuhn.tolist()}
        want = set()
        for base in itertools.product(range(N), repeat=3):
            for perm in itertools.permutations(range(3)):
                p = list(base)
                verts = [tuple(p)]
                for ax in perm:
                    p[ax] += 1
                    verts.append(tuple(p))
                if all(N >= v[0] >= v[1] >= v[2] >= 0 for v in verts):
                    want.add(tuple(sorted(verts)))
        assert len(got) == 8 ** level
        assert got == want


def _cube_grid_lookup(lm):
    N = lm.N
    key = np.rint(lm.coords * N).astype(np.int64)
    table = -np.ones((N + 1,) * 3, dtype=np.int64)
    table[key[:, 0], key[:, 1], key[:, 2]] = np.arange(lm.n)
    return key, table


def test_kuhn_cube_equals_seven_point():
    """On the path-ordered 6-tet Kuhn cube the scaled operator is the 7-point
    finite-difference operator h * sum_axis (k_i+k_j)/2 (u_i-u_j) (textbook:
    P1 on the Freudenthal triangulation of a cubic grid)."""
    V, T = I.kuhn_cube()
    lm = O.LevelMesh(O.MacroMesh(V, T), 3)
    rng = np.random.default_rng(0)
    k = I.k_cube(lm.coords) + 0.3 * rng.random(lm.n)
    u = rng.uniform(-1, 1, lm.n)
    u[lm.dirichlet] = 0.0
    y = lm.apply(u, k, "scaled")
    key, table = _cube_grid_lookup(lm)
    h = 1.0 / lm.N
    for n in lm.unknowns:
        s = 0.0
        for ax in range(3):
            for sg in (-1, 1):
                q = key[n].copy()
                q[ax] += sg
                m = table[tuple(q)]
                s += h * 0.5 * (k[n] + k[m]) * (u[n] - u[m])
        assert abs(y[n] - s) < 1e-13 * max(1.0, abs(s)), n


@pytest.mark.parametrize("mesh,level", [(I.unit_tet, 3), (I.cube24, 2), (I.regular_tet, 3)])
def test_zero_row_sums_and_symmetry(mesh, level):
    """Eq. "zerosum": every row of the (Dirichlet-free) scaled matrix sums to 0;
    K_t o A_t is symmetric (proof of Lemma "equal")."""
    V, T = mesh()
    lm = O.LevelMesh(O.MacroMesh(V, T), level)
    rng = np.random.default_rng(1)
    k = 0.5 + rng.random(lm.n)
    A = lm.assemble(k, "scaled")
    assert np.max(np.abs(A @ np.ones(lm.n))) < 1e-13
    assert abs(A - A.T).max() < 1e-14


def _on_macro_boundary(lm):
    """Nodes on any macro face (not in a volume primitive)."""
    return np.any(lm.ident[:, 1::2] == 0, axis=1) | (np.count_nonzero(lm.ident[:, 1::2], axis=1) < 4)


def test_affine_k_scaled_equals_nodal_on_volume_rows():
    """Proof of Lemma "repro": for affine k the scaled entries k_ij (s^T)_j equal
    the nodal-integration ones at volume nodes, so both operators agree on
    volume rows for any u; they differ on macro-boundary rows."""
    V, T = I.cube12()
    lm = O.LevelMesh(O.MacroMesh(V, T), 3)
    x = lm.coords
    k = 2 * x[:, 0] + 3 * x[:, 1] + 5 * x[:, 2] + 1  # the affine k of Sec. 5's example
    rng = np.random.default_rng(2)
    u = rng.uniform(-1, 1, lm.n)
    ys = lm.apply(u, k, "scaled")
    yn = lm.apply(u, k, "nodal")
    vol = ~_on_macro_boundary(lm)
    assert vol.sum() > 100
    assert np.max(np.abs(ys[vol] - yn[vol])) < 1e-12
    bnd = _on_macro_boundary(lm) & ~lm.dirichlet
    assert np.max(np.abs(ys[bnd] - yn[bnd])) > 1e-6


def test_constant_k_both_forms_are_k_times_laplacian():
    """For k constant on T, a_h = a (Sec. 2.1): scaled = nodal = k * Laplacian."""
    V, T = I.cube24()
    lm = O.LevelMesh(O.MacroMesh(V, T), 2)
    rng = np.random.default_rng(3)
    u = rng.uniform(-1, 1, lm.n)
    c = 2.75
    k = np.full(lm.n, c)
    yl = lm.apply(u, None, "laplace")
    assert np.max(np.abs(lm.apply(u, k, "scaled") - c * yl)) < 1e-13
    assert np.max(np.abs(lm.apply(u, k, "nodal") - c * yl)) < 1e-13


def test_quadratic_k_nodal_is_vertex_quadrature():
    """Eq. "standardfe": the nodal form equals |t|/4 sum_i k(x_i) grad u . grad v
    on every micro tetrahedron; check on one element against that sum."""
    rng = np.random.default_rng(4)
    X = rng.random((1, 4, 3))
    kv = rng.random((1, 4)) + 0.5
    M = O.nodal_element(O.p1_stiffness(X), kv)
    G, vol = O.p1_gradients(X)
    uu, vv = rng.random(4), rng.random(4)
    gu, gv = uu @ G[0], vv @ G[0]
    want = vol[0] / 4 * np.sum(kv[0]) * float(gu @ gv)
    assert abs(vv @ M[0] @ uu - want) < 1e-14


def test_p1_gradients_reproduce_linear_functions():
    rng = np.random.default_rng(5)
    X = rng.random((3, 4, 3))
    G, vol = O.p1_gradients(X)
    c = rng.random(3)
    vals = X @ c
    assert np.allclose(np.einsum("na,nai->ni", vals, G), c[None, :], atol=1e-12)
    assert np.allclose(G.sum(axis=1), 0.0, atol=1e-12)
    d = np.abs(np.linalg.det(X[:, 1:] - X[:, :1])) / 6
    assert np.allclose(vol, d)


def test_mass_matrix_moments():
    V, T = I.cube24()
    lm = O.LevelMesh(O.MacroMesh(V, T), 2)
    M = lm.assemble_mass()
    one = np.ones(lm.n)
    assert abs(one @ M @ one - 1.0) < 1e-13
    assert abs(one @ M @ lm.coords[:, 0] - 0.5) < 1e-13
    # exact for quadratics: int x^2 over the unit cube = 1/3
    assert abs(lm.coords[:, 0] @ M @ lm.coords[:, 0] - 1 / 3) < 1e-13


def test_row_apply_matches_element_loop():
    """The one-row evaluator (for sampled checks at large sizes) agrees with
    the full element loop, on interface, edge and vertex nodes too."""
    V, T = I.cube12()
    mm = O.MacroMesh(V, T)
    lm = O.LevelMesh(mm, 2)
    kf = I.k_cube
    uf = lambda g, w, x: np.sin(3 * x[:, 0]) + x[:, 1] * x[:, 2]
    kfun = lambda g, w, x: kf(x)
    u = uf(None, None, lm.coords)
    k = kf(lm.coords)
    for kind in ("scaled", "nodal"):
        y = lm.apply(u, k, kind)
        for n in range(0, lm.n, 7):
            sup = lm.ident[n, 0::2][lm.ident[n, 1::2] > 0]
            w = lm.ident[n, 1::2][lm.ident[n, 1::2] > 0]
            got = O.row_apply(mm, 2, sup, w, uf, kfun, kind)
            assert abs(got - y[n]) < 1e-12, (kind, n)


def test_prolongation_exact_for_affine_functions():
    V, T = I.cube24()
    mm = O.MacroMesh(V, T)
    c, f = O.LevelMesh(mm, 1), O.LevelMesh(mm, 2)
    P = O.prolongation(c, f)
    a = np.array([0.3, -1.2, 2.0])
    assert np.max(np.abs(P @ (c.coords @ a + 0.7) - (f.coords @ a + 0.7))) < 1e-13
    assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0)


def _small_hierarchy(smoother="jacobi", finest=3):
    V, T = I.kuhn_cube()
    return O.Hierarchy(V, T, finest, 1, k_func=I.k_cube, smoother=smoother)


def test_jacobi_error_propagation():
    H = _small_hierarchy()
    l = H.finest
    A, D = H.A[l].toarray(), H.D[l]
    rng = np.random.default_rng(6)
    e = rng.standard_normal(A.shape[0])
    E = np.eye(len(D)) - H.omega * (A / D[:, None])
    got = H.jacobi(l, np.zeros_like(e), e, 3)
    assert np.allclose(got, np.linalg.matrix_power(E, 3) @ e, atol=1e-12)


def test_chebyshev_error_propagation_is_chebyshev_polynomial():
    """Applied to an eigenvector of D^-1 A with eigenvalue lam (f = 0), the
    degree-m smoother multiplies it by T_m((theta-lam)/delta) / T_m(theta/delta)."""
    H = _small_hierarchy("chebyshev")
    l = H.finest
    A, D = H.A[l].toarray(), H.D[l]
    Dh = np.sqrt(D)
    lam, W = np.linalg.eigh(A / np.outer(Dh, Dh))
    a, b = H.cheb_lo * H.lam[l], H.cheb_hi * H.lam[l]
    theta, delta = (a + b) / 2, (b - a) / 2
    for m in (1, 2, 3):
        for idx in (0, len(lam) // 2, len(lam) - 1):
            v = W[:, idx] / Dh
            got = H.chebyshev(l, np.zeros_like(v), v.copy(), degree=m)
            Tm = lambda x: np.cosh(m * np.arccosh(x)) if abs(x) >= 1 else np.cos(m * np.arccos(x))
            fac = Tm((theta - lam[idx]) / delta) / Tm(theta / delta)
            assert np.allclose(got, fac * v, atol=1e-10 * np.max(np.abs(v)))


def test_power_iteration_bounds_largest_eigenvalue():
    H = _small_hierarchy()
    for l in H.levels:
        A, D = H.A[l].toarray(), H.D[l]
        Dh = np.sqrt(D)
        lmax = np.linalg.eigvalsh(A / np.outer(Dh, Dh))[-1]
        assert H.lam[l] <= lmax * (1 + 1e-12)
        assert H.lam[l] >= 0.8 * lmax


def test_coarse_cholesky_solves_coarse_system():
    H = _small_hierarchy()
    Ac = H.A[H.coarsest].toarray()
    f = np.arange(Ac.shape[0], dtype=float) + 1
    assert np.allclose(Ac @ H.coarse_solve(f), f, atol=1e-12)


def test_vcycle_is_symmetric_preconditioner():
    """V(2,2) with the same symmetric smoother before and after the coarse
    correction, R = P^T and an exact coarse solve, is a symmetric operator."""
    for sm in ("jacobi", "chebyshev"):
        H = _small_hierarchy(sm, finest=2)
        n = H.A[2].shape[0]
        B = np.stack([H.vcycle(2, np.eye(n)[i], np.zeros(n)) for i in range(n)], axis=1)
        assert np.max(np.abs(B - B.T)) < 1e-12 * np.max(np.abs(B))
        assert np.min(np.linalg.eigvalsh(0.5 * (B + B.T))) > 0


@pytest.mark.slow
def test_pcg_converges_level_independent():
    its = []
    for finest in (3, 4):
        V, T = I.kuhn_cube()
        H = O.Hierarchy(V, T, finest, 2, k_func=I.k_cube)
        lm = H.mesh[finest]
        f = lm.assemble_mass()[lm.unknowns][:, lm.unknowns] @ I.f_cube_sine(lm.coords[lm.unknowns])
        x, it, hist = H.pcg(f, tol=1e-10)
        xs = H.direct_solve(f)
        assert np.max(np.abs(x - xs)) <= 1e-8 * np.max(np.abs(xs))
        its.append(it)
    assert max(its) <= 16 and abs(its[0] - its[1]) <= 3


def _solve_manufactured(level):
    V, T = I.kuhn_cube()
    mm = O.MacroMesh(V, T)
    lm = O.LevelMesh(mm, level)
    k = I.k_cube(lm.coords)
    A = lm.system(k, "scaled")
    M = lm.assemble_mass()
    f = (M @ I.f_cube_sine(lm.coords))[lm.unknowns]
    import scipy.sparse.linalg as spla
    uh = np.zeros(lm.n)
    uh[lm.unknowns] = spla.spsolve(A.tocsc(), f)
    e = uh - I.u_sine(lm.coords)
    return O.discrete_l2(lm, e), O.h1_seminorm_error(lm, uh, I.grad_u_sine)


@pytest.mark.slow
def test_convergence_orders_manufactured_solution():
    """Lemma "optimalorder": O(h^2) in L2 and O(h) in H1 for the scaled form."""
    errs = [_solve_manufactured(l) for l in (2, 3, 4)]
    l2 = [e[0] for e in errs]
    h1 = [e[1] for e in errs]
    eoc_l2 = [math.log2(l2[i] / l2[i + 1]) for i in range(2)]
    eoc_h1 = [math.log2(h1[i] / h1[i + 1]) for i in range(2)]
    assert 1.8 < eoc_l2[-1] < 2.3, eoc_l2
    assert 0.9 < eoc_h1[-1] < 1.15, eoc_h1


def test_manufactured_rhs_is_minus_div_k_grad_u():
    """The hand-derived f = -div(k grad u) against central differences."""
    rng = np.random.default_rng(7)
    x = rng.uniform(0.1, 0.9, (20, 3))
    h = 1e-4
    flux = lambda p: I.k_cube(p)[:, None] * I.grad_u_sine(p)
    div = np.zeros(len(x))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        div += (flux(x + e)[:, a] - flux(x - e)[:, a]) / (2 * h)
    assert np.allclose(I.f_cube_sine(x), -div, rtol=1e-6, atol=1e-6)


def test_cube48_is_a_conforming_partition_of_the_unit_cube():
    """The 48-tetrahedron mesh: volumes sum to 1, every tet is non-degenerate,
    inner faces are shared by exactly two tets and the 48 boundary faces lie
    on the cube's faces (so the domain is the unit cube)."""
    V, T = I.cube48()
    vol = [abs(np.linalg.det(np.stack([V[t[1]] - V[t[0]], V[t[2]] - V[t[0]], V[t[3]] - V[t[0]]]))) / 6 for t in T]
    assert abs(sum(vol) - 1.0) < 1e-12 and min(vol) > 0.01
    faces = Counter(tuple(sorted(f)) for t in T for f in itertools.combinations(t, 3))
    assert sorted(Counter(faces.values()).items()) == [(1, 48), (2, 72)]
    for f, c in faces.items():
        if c == 1:
            P = V[list(f)]
            assert any(np.all(np.abs(P[:, a] - P[0, a]) < 1e-15) and P[0, a] in (0.0, 1.0) for a in range(3))
