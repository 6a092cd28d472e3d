"""GPU parity of the pre-asymptotic modification (Sec. 4, eq. "defKmin"):
with the mesh option kappa = 1 the scaled operator scales gray directions
with k_min; every mode goes through it.  Compared with the oracle's "kmin"
operator on the same seeded inputs: a flat tetrahedron with an obtuse
dihedral angle and rough high-contrast k (where the plain operator is
indefinite), four disjoint random tetrahedra, and the 12-tet cube (shared
faces: interface copies carry their own tetrahedron's k_min).  FP64 to
1e-12 relative max-norm, FP32 and BF16-k to 1e-6 on the rounded inputs."""
import math

import numpy as np
import pytest

from oracle import hhg_oracle as O
from paper_1709_06793_gb300 import inputs as I
from tests import hhg_testutil as U

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

OBTUSE = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.3, 0.8, 0.1], [0.52, 0.05, 0.12]])


def _bf16(x):
    x = np.asarray(x, dtype=np.float64)
    q = np.exp2(np.floor(np.log2(x)) - 7)
    return np.round(x / q) * q


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06793_gb300 import build
    build.build()
    from paper_1709_06793_gb300 import hhg
    return hhg


def _rough_k(keys):
    """log-uniform in [1, 1e4] from the nodes' generator keys (one value per
    node, so every stored copy gets it)"""
    return np.exp(np.log(1e4) * (0.5 + 0.5 * I.uniform_from_keys(keys, 3)))


CASES = {
    "obtuse_l4": (lambda: (OBTUSE, np.array([[0, 1, 2, 3]])), 4, 2),
    "random4_l3": (lambda: I.random_tets(4, seed=1), 3, 1),
    "cube12_l3": (I.cube12, 3, 1),
}


class Case:
    def __init__(self, H, V, T, level, coarsest):
        self.m = H.Mesh(V, T, level, coarsest)
        self.off, self.lev, self.n = self.m.layout(0)
        self.lm = O.LevelMesh(O.MacroMesh(V, T), level)
        self.idx = U.oracle_map(self.lm, U.stored_nodes(self.off, self.lev))
        self.k_or = _rough_k(U.oracle_keys(self.lm))
        H.hhg_set_coefficient(self.m.h, torch.tensor(self.k_or[self.idx], device="cuda"))
        self.u = np.where(self.lm.dirichlet, 0.0, I.uniform_from_keys(U.oracle_keys(self.lm), 7))

    def back(self, t):
        a = t.double().cpu().numpy()
        out = np.zeros(self.lm.n)
        out[self.idx] = a
        assert np.array_equal(a, out[self.idx]), "interface copies disagree"
        return out


@pytest.fixture(scope="module", params=list(CASES))
def case(request, H):
    mesh, level, coarsest = CASES[request.param]
    V, T = mesh()
    c = Case(H, V, T, level, coarsest)
    H.hhg_set_option(c.m.h, "kappa", 1)
    yield c
    c.m.close()


def test_the_cases_have_gray_directions():
    for name, (mesh, level, coarsest) in CASES.items():
        V, T = mesh()
        assert any(O.gray_directions(V, T[t]).any() for t in range(len(T))), name


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_kappa_apply_parity(H, case, dtype):
    uin = case.u if dtype == 0 else _f32(case.u)
    kk = case.k_or if dtype == 0 else (_f32(case.k_or) if dtype == 1 else _bf16(case.k_or))
    want = case.lm.apply(uin, kk, "kmin")
    ud = torch.tensor(uin[case.idx], device="cuda", dtype=torch.float64 if dtype == 0 else torch.float32)
    y = torch.empty_like(ud)
    H.hhg_apply_scaled(case.m.h, 0, ud, y, dtype)
    got = case.back(y)
    tol = 1e-12 if dtype == 0 else 1e-6
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err <= tol, err
    assert np.all(got[case.lm.dirichlet] == 0)


def test_kappa_residual_and_jacobi_parity(H, case):
    f = np.where(case.lm.dirichlet, 0.0, I.uniform_from_keys(U.oracle_keys(case.lm), 9))
    fd = torch.tensor(f[case.idx], device="cuda")
    ud = torch.tensor(case.u[case.idx], device="cuda")
    r = torch.empty_like(ud)
    H.hhg_residual(case.m.h, 0, fd, ud, r, 0)
    A = case.lm.assemble(case.k_or, "kmin")
    want = np.where(case.lm.dirichlet, 0.0, f - A @ np.where(case.lm.dirichlet, 0.0, case.u))
    got = case.back(r)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= 1e-12
    # one damped Jacobi sweep u + omega D^-1 (f - A u), D the modified diagonal
    H.hhg_smooth(case.m.h, 0, H.HHG_SMOOTH_JACOBI, 1, 0.6, fd, ud, 0)
    D = A.diagonal()
    wj = np.where(case.lm.dirichlet, 0.0, case.u + 0.6 * want / np.where(D == 0, 1.0, D))
    gj = case.back(ud)
    assert np.max(np.abs(gj - wj)) / np.max(np.abs(wj)) <= 1e-12


def test_kappa_solve_reaches_the_modified_discrete_solution(H):
    """Where the plain operator is indefinite, GMG-CG with the modification
    converges to the oracle's solution of the modified system."""
    V, T = CASES["obtuse_l4"][0]()
    c = Case(H, V, T, 4, 2)
    lm = c.lm
    A_plain = lm.system(c.k_or, "scaled").toarray()
    assert np.linalg.eigvalsh(A_plain)[0] < 0  # the unmodified operator is indefinite here
    H.hhg_set_option(c.m.h, "kappa", 1)
    f = np.where(lm.dirichlet, 0.0, lm.assemble_mass() @ np.ones(lm.n))
    import scipy.sparse.linalg as spla
    A = lm.system(c.k_or, "kmin")
    xs = np.zeros(lm.n)
    xs[lm.unknowns] = spla.spsolve(A.tocsc(), f[lm.unknowns])
    x = torch.zeros(c.n, device="cuda", dtype=torch.float64)
    st = H.hhg_solve(c.m.h, torch.tensor(f[c.idx], device="cuda"), x, tol=1e-11, mode=H.HHG_SOLVE_FP64, maxit=400)
    assert st["rel_residual"] <= 1e-11, st
    e = (c.back(x) - xs)[lm.unknowns]
    xa = xs[lm.unknowns]
    assert math.sqrt(abs(e @ (A @ e))) / math.sqrt(xa @ (A @ xa)) <= 1e-8
    c.m.close()


def test_kuhn_cube_is_unchanged_and_bad_values_are_rejected(H):
    V, T = I.kuhn_cube()
    m = H.Mesh(V, T, 4, 2)
    off, lev, n = m.layout(0)
    lm = O.LevelMesh(O.MacroMesh(V, T), 4)
    idx = U.oracle_map(lm, U.stored_nodes(off, lev))
    H.hhg_set_coefficient(m.h, torch.tensor(_rough_k(U.oracle_keys(lm))[idx], device="cuda"))
    u = torch.rand(n, device="cuda", dtype=torch.float64)
    mask = torch.empty_like(u)
    H.hhg_residual(m.h, 0, torch.ones_like(u), torch.zeros_like(u), mask, 0)
    u *= mask
    y0, y1 = torch.empty_like(u), torch.empty_like(u)
    H.hhg_apply_scaled(m.h, 0, u, y0, 0)
    H.hhg_set_option(m.h, "kappa", 1)
    assert H.hhg_get_option(m.h, "kappa") == 1
    H.hhg_apply_scaled(m.h, 0, u, y1, 0)
    assert float((y0 - y1).abs().max() / y0.abs().max()) <= 1e-13
    with pytest.raises(H.HHGError):
        H.hhg_set_option(m.h, "kappa", 2)
    m.close()
