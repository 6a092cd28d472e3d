"""Pins of the pre-asymptotic modification of Sec. 4 (eq. "defKmin") in the
oracle, against facts that do not use its formulas:

* with a constant k, k_min = k and the modified operator is the scaled one;
* on the Kuhn cube the reference stencil is the 7-point one (no positive
  off-centre entry), so nothing is modified, whatever k is;
* k_min of a node is the minimum of k over the node and the in-tetrahedron
  neighbours at the 14 stencil offsets (brute force over index space);
* the reference stencil has zero row sum, and a flat tetrahedron with an
  obtuse dihedral angle has positive ("gray") entries;
* where the scaled operator is indefinite (an obtuse tetrahedron, rough
  high-contrast k, a coarse level) the modified one is positive definite
  (Lemma of Sec. 4.2: the modification makes the form uniformly coercive).
"""
import numpy as np
import pytest

from oracle import hhg_oracle as O
from paper_1709_06793_gb300 import inputs as I

# a flat tetrahedron: vertex 3 close to the midpoint of edge 0-1
OBTUSE = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.3, 0.8, 0.1], [0.52, 0.05, 0.12]])


def _one_tet(P, level):
    return O.LevelMesh(O.MacroMesh(P, np.array([[0, 1, 2, 3]])), level)


def _rough_k(lm, seed, contrast):
    return np.exp(np.random.default_rng(seed).uniform(0.0, np.log(contrast), lm.n))


@pytest.mark.parametrize("mesh,level", [(I.kuhn_cube, 2), (I.cube12, 2), (I.unit_tet, 3)])
def test_constant_k_leaves_the_operator_unchanged(mesh, level):
    V, T = mesh()
    lm = O.LevelMesh(O.MacroMesh(V, T), level)
    k = np.full(lm.n, 2.5)
    a = lm.assemble(k, "scaled").toarray()
    b = lm.assemble(k, "kmin").toarray()
    assert np.abs(a - b).max() <= 1e-15 * np.abs(a).max()


def test_kuhn_cube_has_no_gray_edges_so_nothing_changes():
    V, T = I.kuhn_cube()
    for t in range(len(T)):
        s = O.reference_volume_stencil(V, T[t])
        neg = s < -1e-14
        assert neg.sum() == 6 and np.allclose(s[neg], s[neg][0]) and np.all(np.abs(s[~neg]) <= 1e-14)
    lm = O.LevelMesh(O.MacroMesh(V, T), 3)
    k = _rough_k(lm, 3, 1e3)
    a = lm.assemble(k, "scaled").toarray()
    b = lm.assemble(k, "kmin").toarray()
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()


def test_kmin_is_the_minimum_over_the_in_tet_stencil_neighbourhood():
    lm = _one_tet(OBTUSE, 3)
    N = lm.N
    k = _rough_k(lm, 5, 1e2)
    km = O.tet_kmin(lm, k, 0)
    L = lm.local[0]
    for i in range(N + 1):
        for j in range(N + 1 - i):
            for kk in range(N + 1 - i - j):
                vals = [k[L[i, j, kk]]]
                for (a, b, c) in O.STENCIL_DIRS:
                    p, q, r = i + a, j + b, kk + c
                    if min(p, q, r) >= 0 and p + q + r <= N:
                        vals.append(k[L[p, q, r]])
                assert km[L[i, j, kk]] == min(vals)


def test_reference_stencil_sums_to_zero_and_the_flat_tet_has_gray_entries():
    for P in (OBTUSE, np.array([[0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])):
        lm = _one_tet(P, 2)
        A = lm.assemble(None, "laplace").toarray()
        x = lm.local[0][1, 1, 1]
        s = O.reference_volume_stencil(P, [0, 1, 2, 3])
        assert abs(A[x, x] + s.sum()) <= 1e-13 * abs(A[x, x])
    assert O.gray_directions(OBTUSE, [0, 1, 2, 3]).any()


def test_modification_restores_positive_definiteness():
    lm = _one_tet(OBTUSE, 3)
    k = _rough_k(lm, 11, 1e4)
    lam_plain = np.linalg.eigvalsh(lm.system(k, "scaled").toarray())[0]
    lam_kmin = np.linalg.eigvalsh(lm.system(k, "kmin").toarray())[0]
    assert lam_plain < 0.0 < lam_kmin, (lam_plain, lam_kmin)


def test_configured_random_tets_and_grf_cube_are_coercive_without_the_modification():
    """The positivity check of the configured workloads (eigenvalues of the
    scaled operator on the unknowns): the 48 random tetrahedra (all have
    gray directions) with their tanh-Fourier k at level 4, and the 6-tet cube
    with the contrast-1e2 Gaussian random field at level 3, are positive
    definite, so they run unmodified."""
    V, T = I.random_tets(48, seed=1)
    kf = I.k_batched(1)
    worst = np.inf
    for t in range(len(T)):
        assert O.gray_directions(V, T[t]).any()
        lm = O.LevelMesh(O.MacroMesh(V[T[t]], np.array([[0, 1, 2, 3]])), 4)
        ev = np.linalg.eigvalsh(lm.system(kf(lm.coords), "scaled").toarray())
        worst = min(worst, ev[0] / ev[-1])
    assert worst > 1e-3, worst
    V, T = I.kuhn_cube()
    lm = O.LevelMesh(O.MacroMesh(V, T), 3)
    ev = np.linalg.eigvalsh(lm.system(I.k_learned()(lm.coords), "scaled").toarray())
    assert ev[0] / ev[-1] > 1e-3, ev[0] / ev[-1]
