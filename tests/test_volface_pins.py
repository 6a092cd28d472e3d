"""Pins of the "scale Vol+Face" operator of the oracle (eq. "modst" with
I = W_V u W_E): Lemma "repro" (affine k and affine u are reproduced exactly,
which plain scaling does not do on a mesh with interior macro edges), the
O(h^2) decay of its asymmetry (remark after eq. "modst"), and the row split
between the nodal and the scaled forms."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import hhg_oracle as O
from paper_1709_06793_gb300 import inputs as I


def _affine_solve(lm, A):
    """Solve with Dirichlet data u on the boundary and the load vector of
    f = -div(k grad u) (constant), for k = 1 + 0.3x + 0.2y - 0.1z and
    u = 0.5 + x - 2y + 0.7z; returns max |u_h - u| on the unknowns."""
    x = lm.coords
    u = 0.5 + x[:, 0] - 2 * x[:, 1] + 0.7 * x[:, 2]
    f = -(0.3 * 1.0 + 0.2 * (-2.0) + (-0.1) * 0.7)
    b = f * (lm.assemble_mass() @ np.ones(lm.n))  # (f, phi_i) exactly: f constant
    Iu, B = lm.unknowns, np.nonzero(lm.dirichlet)[0]
    A = A.tocsr()
    uh = spla.spsolve(A[Iu][:, Iu].tocsc(), b[Iu] - A[Iu][:, B] @ u[B])
    return float(np.max(np.abs(uh - u[Iu])))


def _affine_k(lm):
    x = lm.coords
    return 1 + 0.3 * x[:, 0] + 0.2 * x[:, 1] - 0.1 * x[:, 2]


@pytest.mark.parametrize("level", [2, 3])
def test_volface_reproduces_affine_solutions(level):
    V, T = I.cube12()  # body centre + face triangles: interior macro edges and vertices
    lm = O.LevelMesh(O.MacroMesh(V, T), level)
    k = _affine_k(lm)
    assert _affine_solve(lm, O.volface_matrix(lm, k)) <= 1e-12
    assert _affine_solve(lm, lm.assemble(k, "nodal")) <= 1e-12
    # plain scaling misses it through the macro-edge/vertex rows
    assert _affine_solve(lm, lm.assemble(k, "scaled")) >= 1e-4


def test_volface_asymmetry_decays_like_h_squared():
    V, T = I.cube12()
    mm = O.MacroMesh(V, T)
    asym = []
    for level in (2, 3, 4):
        lm = O.LevelMesh(mm, level)
        A = O.volface_matrix(lm, I.k_cube(lm.coords))
        Iu = lm.unknowns
        A = A[Iu][:, Iu]
        asym.append(spla.norm(A - A.T) / spla.norm(A))
    assert asym[0] > 0
    assert asym[0] / asym[1] >= 3.5 and asym[1] / asym[2] >= 3.5


def test_volface_rows_split_by_primitive():
    """Vertex/edge rows equal the nodal matrix, face/volume rows the scaled
    one; the classification counts the non-zero barycentric weights."""
    V, T = I.cube12()
    lm = O.LevelMesh(O.MacroMesh(V, T), 2)
    dim = O.primitive_dim(lm)
    # macro vertices: 8 cube corners + body centre + 6 face centres
    assert int(np.sum(dim == 0)) == len(V)
    k = I.k_cube(lm.coords)
    A = O.volface_matrix(lm, k).toarray()
    An = lm.assemble(k, "nodal").toarray()
    As = lm.assemble(k, "scaled").toarray()
    ve = dim <= 1
    np.testing.assert_array_equal(A[ve], An[ve])
    np.testing.assert_array_equal(A[~ve], As[~ve])
    assert np.max(np.abs(An[ve] - As[ve])) > 1e-6
    u = np.where(lm.dirichlet, 0.0, np.sin(lm.coords[:, 0] + 2 * lm.coords[:, 1]))
    y = O.volface_apply(lm, u, k)
    yr = A @ np.where(lm.dirichlet, 0.0, u)
    np.testing.assert_allclose(y[~lm.dirichlet], yr[~lm.dirichlet], rtol=0, atol=1e-13)


@pytest.mark.parametrize("kind", ["nodal", "volface", "scaled"])
def test_mg_solver_converges_at_a_level_independent_rate(kind):
    """Multigrid as the solver (V(3,3), i* = 10, rho of Sec. 7) on the paper's
    scalar 3D test coefficient k = cos(3 pi x y z) + 2 on the 6-tet cube: the
    rate stays bounded across levels and the discrete L2 error of the
    manufactured u = sin(pi x) sin(pi y) sin(pi z) drops by ~4 per level."""
    V, T = I.kuhn_cube()
    rho, err = [], []
    for level in (3, 4):
        H = O.Hierarchy(V, T, level, 2, k_func=I.k_cosine(3), kind=kind)
        lm = H.mesh[level]
        f = (lm.assemble_mass() @ I.f_sine_cosine_k(3)(lm.coords))[lm.unknowns]
        x, hist = H.mg_solve(f, 10)
        assert all(b < a for a, b in zip(hist, hist[1:]))
        rho.append(O.mg_rate(hist))
        e = np.zeros(lm.n)
        e[lm.unknowns] = x - I.u_sine(lm.coords)[lm.unknowns]
        err.append(O.discrete_l2(lm, e))
    assert max(rho) <= 0.4 and rho[1] <= 1.5 * rho[0]
    assert 3.0 <= err[0] / err[1] <= 5.0
