"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Tolerances: FP64 rel. max-norm 1e-12 (operators; the
smoothers and V-cycles accumulate rounding over many steps, see each test),
FP32 rel. max-norm 1e-6 on inputs rounded to the kernel's precision."""
import math

import numpy as np
import pytest

from oracle import hhg_oracle as O
from paper_1709_06793_gb300 import inputs as I
from tests import hhg_testutil as U

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06793_gb300 import build
    build.build()
    from paper_1709_06793_gb300 import hhg
    return hhg


def _bf16(x):
    """Round to bfloat16 (8 significant bits), nearest-even, directly from
    double (as the library's conversion does); positive inputs."""
    x = np.asarray(x, dtype=np.float64)
    q = np.exp2(np.floor(np.log2(x)) - 7)
    return np.round(x / q) * q


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


class Case:
    """A mesh on the GPU plus the oracle's view of the same nodes."""

    def __init__(self, H, V, T, level, coarsest, kfun, seed=0):
        self.H = H
        self.V, self.T, self.level = V, T, level
        self.m = H.Mesh(V, T, level, coarsest)
        self.off, self.lev, self.n = self.m.layout(0)
        self.nodes = U.stored_nodes(self.off, self.lev)
        self.lm = O.LevelMesh(O.MacroMesh(V, T), level)
        self.idx = U.oracle_map(self.lm, self.nodes)
        self.xyz = self.m.coords(0)
        self.k_st = kfun(self.xyz)
        self.k_or = kfun(self.lm.coords)
        H.hhg_set_coefficient(self.m.h, torch.tensor(self.k_st, device="cuda"))
        keys = U.oracle_keys(self.lm)
        self.dir = self.lm.dirichlet
        self.rand_or = np.where(self.dir, 0.0, I.uniform_from_keys(keys, seed))

    def to_stored(self, v_or):
        return v_or[self.idx]

    def dev(self, v_or, dtype):
        t = torch.float64 if dtype == self.H.HHG_F64 else torch.float32
        return torch.tensor(self.to_stored(v_or), device="cuda", dtype=t)

    def back(self, t):
        """Stored GPU vector -> oracle indexing; checks all copies agree."""
        a = t.double().cpu().numpy()
        out = np.zeros(self.lm.n)
        out[self.idx] = a
        assert np.array_equal(a, out[self.idx]), "interface copies disagree"
        return out

    def kprec(self, dtype):
        if dtype == self.H.HHG_F64:
            return self.k_or
        if dtype == self.H.HHG_F32:
            return _f32(self.k_or)
        return _bf16(self.k_or)


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


MESHES = {
    "unit_tet_l5": (I.unit_tet, 5, 3, I.k_unit_tet),
    "kuhn_cube_l4": (I.kuhn_cube, 4, 2, I.k_cube),
    "cube24_l3": (I.cube24, 3, 1, I.k_large),
    "cube12_l3": (I.cube12, 3, 1, I.k_cube),
    "cube48_l3": (I.cube48, 3, 1, I.k_batched(1)),  # 48 tets sharing faces (a batch with interfaces)
}


@pytest.fixture(scope="module", params=list(MESHES))
def case(request, H):
    mesh, level, coarsest, kf = MESHES[request.param]
    V, T = mesh()
    return Case(H, V, T, level, coarsest, kf)


@pytest.mark.parametrize("kind", ["scaled", "nodal"])
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_apply_parity(H, case, kind, dtype):
    u = case.rand_or
    tol = 1e-12 if dtype == H.HHG_F64 else 1e-6
    uin = u if dtype == H.HHG_F64 else _f32(u)
    ud = case.dev(uin, dtype)
    y = torch.empty_like(ud)
    f = H.hhg_apply_scaled if kind == "scaled" else H.hhg_apply_nodal
    f(case.m.h, 0, ud, y, dtype)
    torch.cuda.synchronize()
    got = case.back(y)
    want = case.lm.apply(uin, case.kprec(dtype), kind)
    assert _rel(got, want) <= tol, _rel(got, want)
    assert np.all(got[case.dir] == 0)


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_volface_apply_parity(H, case, dtype):
    """"Scale Vol+Face" (eq. "modst", I = W_V u W_E) against the oracle's
    row split of its nodal and scaled element loops."""
    u = case.rand_or
    tol = 1e-12 if dtype == H.HHG_F64 else 1e-6
    uin = u if dtype == H.HHG_F64 else _f32(u)
    ud = case.dev(uin, dtype)
    y = torch.empty_like(ud)
    H.hhg_apply_volface(case.m.h, 0, ud, y, dtype)
    torch.cuda.synchronize()
    got = case.back(y)
    want = O.volface_apply(case.lm, uin, case.kprec(dtype))
    assert _rel(got, want) <= tol, _rel(got, want)
    assert np.all(got[case.dir] == 0)
    # it differs from plain scaling exactly on macro-vertex/edge rows
    ys = torch.empty_like(ud)
    H.hhg_apply_scaled(case.m.h, 0, ud, ys, dtype)
    diff = np.abs(got - case.back(ys)) > 0
    ve = O.volface_rows(case.lm) & ~case.dir
    assert not np.any(diff & ~ve)
    if ve.any() and dtype == H.HHG_F64:
        assert np.any(diff & ve)


def test_scaled_and_nodal_differ_for_nonaffine_k(H, case):
    ud = case.dev(case.rand_or, H.HHG_F64)
    ys, yn = torch.empty_like(ud), torch.empty_like(ud)
    H.hhg_apply_scaled(case.m.h, 0, ud, ys, H.HHG_F64)
    H.hhg_apply_nodal(case.m.h, 0, ud, yn, H.HHG_F64)
    assert torch.max(torch.abs(ys - yn)).item() > 1e-8


def test_residual_parity(H, case):
    f_or = np.where(case.dir, 0.0, np.sin(7 * case.lm.coords[:, 0]) + case.lm.coords[:, 2])
    u = case.rand_or
    r = torch.empty(case.n, device="cuda", dtype=torch.float64)
    H.hhg_residual(case.m.h, 0, case.dev(f_or, 0), case.dev(u, 0), r, H.HHG_F64)
    want = np.where(case.dir, 0.0, f_or - case.lm.apply(u, case.k_or, "scaled"))
    assert _rel(case.back(r), want) <= 1e-12


def test_unit_tet_fifty_jacobi_sweeps(H):
    """The small configuration: unit tetrahedron, level 5, k = 1 + 0.5 sin sin sin,
    u ~ U[-1,1], 50 damped Jacobi sweeps (omega = 2/3), FP64, against the oracle."""
    V, T = I.unit_tet()
    c = Case(H, V, T, 5, 3, I.k_unit_tet)
    A = c.lm.system(c.k_or, "scaled")
    Dg = A.diagonal()
    keys = U.oracle_keys(c.lm)
    f_or = np.where(c.dir, 0.0, I.uniform_from_keys(keys, 11))
    u = c.rand_or.copy()
    ud = c.dev(u, 0)
    H.hhg_smooth(c.m.h, 0, H.HHG_SMOOTH_JACOBI, 50, 2.0 / 3.0, c.dev(f_or, 0), ud, H.HHG_F64)
    uu = u[c.lm.unknowns]
    fu = f_or[c.lm.unknowns]
    for _ in range(50):
        uu = uu + (2.0 / 3.0) * (fu - A @ uu) / Dg
    want = np.zeros(c.lm.n)
    want[c.lm.unknowns] = uu
    assert _rel(c.back(ud), want) <= 1e-11


def test_fp32_jacobi_sweeps(H):
    V, T = I.kuhn_cube()
    c = Case(H, V, T, 4, 2, I.k_cube)
    A = c.lm.system(_f32(c.k_or), "scaled")
    Dg = A.diagonal()
    f_or = np.where(c.dir, 0.0, 1.0)
    u = _f32(c.rand_or)
    ud = c.dev(u, 1)
    H.hhg_smooth(c.m.h, 0, H.HHG_SMOOTH_JACOBI, 5, 2.0 / 3.0, c.dev(f_or, 1), ud, H.HHG_F32)
    uu, fu = u[c.lm.unknowns], f_or[c.lm.unknowns]
    for _ in range(5):
        uu = uu + (2.0 / 3.0) * (fu - A @ uu) / Dg
    want = np.zeros(c.lm.n)
    want[c.lm.unknowns] = uu
    assert _rel(c.back(ud), want) <= 1e-5


def test_batched_mixed_levels_apply(H):
    """Independent random tetrahedra with levels 3..6 in one launch: each tet
    agrees with its own single-tet oracle."""
    V, T = I.random_tets(6, seed=1)
    levels = [3, 6, 4, 5, 6, 3]
    m = H.Mesh(V, T, levels, 2)
    off, lev, n = m.layout(0)
    xyz = m.coords(0)
    kf = I.k_batched(1)
    H.hhg_set_coefficient(m.h, torch.tensor(kf(xyz), device="cuda"))
    nodes = U.stored_nodes(off, lev)
    u = np.zeros(n)
    refs = []
    for t in range(len(T)):
        lm = O.LevelMesh(O.MacroMesh(V[4 * t:4 * t + 4], np.array([[0, 1, 2, 3]])), levels[t])
        sel = nodes[:, 0] == t
        loc = lm.local[0][nodes[sel, 1], nodes[sel, 2], nodes[sel, 3]]
        ut = np.where(lm.dirichlet, 0.0, np.cos(5 * lm.coords[:, 0]) * lm.coords[:, 1] + 0.3)
        u[sel] = ut[loc]
        refs.append((sel, loc, lm, ut))
    for dtype, tol in ((0, 1e-12), (1, 1e-6)):
        tdt = torch.float64 if dtype == 0 else torch.float32
        ud = torch.tensor(u, device="cuda", dtype=tdt)
        y = torch.empty_like(ud)
        H.hhg_apply_scaled(m.h, 0, ud, y, dtype)
        got = y.double().cpu().numpy()
        for t, (sel, loc, lm, ut) in enumerate(refs):
            kk = kf(lm.coords)
            if dtype == 1:
                want = lm.apply(_f32(ut), _f32(kk), "scaled")
            else:
                want = lm.apply(ut, kk, "scaled")
            assert _rel(got[sel], want[loc]) <= tol, (t, dtype)
    m.close()


def test_tiny_levels(H):
    """Levels whose tets have no volume node (N <= 2) or exactly one (N = 4)."""
    for level in (1, 2):
        V, T = I.cube24()
        c = Case(H, V, T, level, 1, I.k_cube)
        ud = c.dev(c.rand_or, 0)
        y = torch.empty_like(ud)
        H.hhg_apply_scaled(c.m.h, 0, ud, y, 0)
        assert _rel(c.back(y), c.lm.apply(c.rand_or, c.k_or, "scaled")) <= 1e-12


def test_dot_counts_each_unknown_once(H, case):
    a, b = case.rand_or, np.cos(case.lm.coords[:, 0] * 3.0)
    b = np.where(case.dir, 0.0, b)
    got = H.hhg_dot(case.m.h, 0, case.dev(a, 0), case.dev(b, 0), 0)
    assert abs(got - float(a @ b)) <= 1e-12 * max(1.0, abs(float(a @ b)))


def test_fp32_dot_counts_each_unknown_once(H, case):
    """FP32 vectors: groups of four products are summed in FP32 (2^-22
    relative each), the groups in FP64."""
    a, b = _f32(case.rand_or), _f32(np.where(case.dir, 0.0, np.cos(case.lm.coords[:, 0] * 3.0)))
    got = H.hhg_dot(case.m.h, 0, case.dev(a, 1), case.dev(b, 1), 1)
    want = float(a @ b)
    assert abs(got - want) <= 1e-6 * float(np.abs(a) @ np.abs(b))


def _hier(V, T, level, coarsest, kf, smoother="jacobi"):
    return O.Hierarchy(V, T, level, coarsest, k_func=kf, smoother=smoother)


def _depth_case(H, c, depth):
    off, lev, n = c.m.layout(depth)
    nodes = U.stored_nodes(off, lev)
    lm = O.LevelMesh(O.MacroMesh(c.V, c.T), c.level - depth)
    return n, lm, U.oracle_map(lm, nodes)


def test_restrict_and_prolongate_parity(H):
    V, T = I.cube24()
    c = Case(H, V, T, 3, 1, I.k_large)
    nc, lmc, idxc = _depth_case(H, c, 1)
    P = O.prolongation(lmc, c.lm)
    rf = c.rand_or
    rc = torch.zeros(nc, device="cuda", dtype=torch.float64)
    H.hhg_restrict(c.m.h, 0, c.dev(rf, 0), rc, 0)
    want = np.where(lmc.dirichlet, 0.0, P.T @ rf)
    got = np.zeros(lmc.n)
    got[idxc] = rc.cpu().numpy()
    assert _rel(got, want) <= 1e-13
    ec = np.where(lmc.dirichlet, 0.0, np.sin(3 * lmc.coords[:, 1]))
    uf = c.dev(c.rand_or, 0)
    H.hhg_prolongate_add(c.m.h, 0, torch.tensor(ec[idxc], device="cuda"), uf, 0)
    assert _rel(c.back(uf), c.rand_or + P @ ec) <= 1e-13


@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
def test_vcycle_parity_fp64(H, smoother):
    V, T = I.kuhn_cube()
    c = Case(H, V, T, 4, 2, I.k_cube)
    Hh = _hier(V, T, 4, 2, I.k_cube, smoother)
    f = np.where(c.dir, 0.0, I.f_cube_sine(c.lm.coords))
    u0 = 0.1 * c.rand_or
    ud = c.dev(u0, 0)
    sm = H.HHG_SMOOTH_JACOBI if smoother == "jacobi" else H.HHG_SMOOTH_CHEBYSHEV
    H.hhg_vcycle(c.m.h, 2, 2, sm, c.dev(f, 0), ud, 0)
    un = Hh.vcycle(4, f[c.lm.unknowns], u0[c.lm.unknowns])
    want = np.zeros(c.lm.n)
    want[c.lm.unknowns] = un
    assert _rel(c.back(ud), want) <= 1e-10


def test_lambda_max_parity(H):
    V, T = I.kuhn_cube()
    c = Case(H, V, T, 4, 2, I.k_cube)
    Hh = _hier(V, T, 4, 2, I.k_cube)
    for depth in (0, 1):
        lam = H.hhg_lambda_max(c.m.h, depth, 15)
        assert abs(lam - Hh.lam[4 - depth]) <= 1e-10 * Hh.lam[4 - depth]


@pytest.mark.parametrize("mode", [0, 1, 2, 4])
def test_solve_matches_oracle_discrete_solution(H, mode):
    """Modes 0, 1 and 4 (BF16 k in the inner solve only) reach the discrete
    solution of the FP64 k; mode 2 (BF16 k throughout) that of k rounded to
    bfloat16."""
    V, T = I.kuhn_cube()
    level = 5
    c = Case(H, V, T, level, 2, I.k_cube)
    lm = c.lm
    M = lm.assemble_mass()
    f_or = np.where(c.dir, 0.0, M @ I.f_cube_sine(lm.coords))
    kk = c.k_or if mode != 2 else _bf16(c.k_or)
    import scipy.sparse.linalg as spla
    A = lm.system(kk, "scaled")
    xs = np.zeros(lm.n)
    xs[lm.unknowns] = spla.spsolve(A.tocsc(), f_or[lm.unknowns])
    ud = torch.zeros(c.n, device="cuda", dtype=torch.float64)
    st = H.hhg_solve(c.m.h, c.dev(f_or, 0), ud, tol=1e-10, mode=mode)
    assert st["rel_residual"] <= 1e-10
    got = c.back(ud)
    err = got - xs
    e_A = math.sqrt(abs(err[lm.unknowns] @ (A @ err[lm.unknowns])))
    x_A = math.sqrt(xs[lm.unknowns] @ (A @ xs[lm.unknowns]))
    assert e_A / x_A <= 1e-8
    assert _rel(got, xs) <= 1e-7


@pytest.mark.parametrize("dtype,tol", [(0, 1e-13), (1, 1e-6)])
def test_mass_apply_parity(H, case, dtype, tol):
    """f_h = M I_h f (Sec. 7.2): every input entry is used, Dirichlet rows are 0."""
    x = case.lm.coords
    v = np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2] + 1.0  # nonzero on the boundary too
    vin = v if dtype == 0 else _f32(v)
    y = torch.empty(case.n, device="cuda", dtype=torch.float64 if dtype == 0 else torch.float32)
    H.hhg_apply_mass(case.m.h, 0, case.dev(vin, dtype), y, dtype)
    want = np.where(case.dir, 0.0, case.lm.assemble_mass() @ vin)
    assert _rel(case.back(y), want) <= tol


def test_autotune_keeps_results_identical(H, tmp_path):
    V, T = I.kuhn_cube()
    c = Case(H, V, T, 5, 2, I.k_cube)
    ud = c.dev(c.rand_or, 1)
    y0 = torch.empty_like(ud)
    H.hhg_apply_scaled(c.m.h, 0, ud, y0, 1)
    cache = str(tmp_path / "tune.txt")
    r1 = H.hhg_autotune(c.m.h, 1, cache)
    assert r1["kseg"] in (16, 32, 64) and r1["korder"] in (0, 1) and r1["best_ms"] > 0
    r2 = H.hhg_autotune(c.m.h, 1, cache)  # cache hit
    assert (r2["kseg"], r2["korder"], r2["vkernel"]) == (r1["kseg"], r1["korder"], r1["vkernel"])
    y1 = torch.empty_like(ud)
    H.hhg_apply_scaled(c.m.h, 0, ud, y1, 1)
    # the column marches (one or two column sets per lane) round every node
    # alike whatever the work split; the tile march sums in another order
    if r1["vkernel"] in (1, 2):
        assert torch.equal(y0, y1)
    else:
        assert _rel(y1.double().cpu().numpy(), y0.double().cpu().numpy()) <= 1e-6
    H.hhg_set_option(c.m.h, "vkernel", 1)
    H.hhg_apply_scaled(c.m.h, 0, ud, y1, 1)
    assert torch.equal(y0, y1)


def _batch(H, levels, seed=4, coarsest=2):
    V, T = I.random_tets(len(levels), seed=seed)
    m = H.Mesh(V, T, levels, coarsest)
    off, lev, n = m.layout(0)
    kf = I.k_batched(seed)
    H.hhg_set_coefficient(m.h, torch.tensor(kf(m.coords(0)), device="cuda"))
    nodes = U.stored_nodes(off, lev)
    parts = []
    for t in range(len(T)):
        Vt, Tt = V[4 * t:4 * t + 4], np.array([[0, 1, 2, 3]])
        sel = nodes[:, 0] == t
        lm = O.LevelMesh(O.MacroMesh(Vt, Tt), levels[t])
        loc = lm.local[0][nodes[sel, 1], nodes[sel, 2], nodes[sel, 3]]
        parts.append((sel, loc, lm, Vt, Tt))
    return m, n, kf, parts


def test_batched_mixed_levels_vcycle_and_solve(H):
    """Independent tets of levels 3..5 in one hierarchy (depth-aligned V-cycle,
    one persistent launch per stage): the V-cycle equals each tet's own oracle
    V-cycle, and the solve reaches every tet's discrete solution."""
    levels = [5, 3, 4, 5]
    m, n, kf, parts = _batch(H, levels)
    f = np.zeros(n)
    hs = []
    for sel, loc, lm, Vt, Tt in parts:
        ft = np.where(lm.dirichlet, 0.0, np.cos(3 * lm.coords[:, 0]) + lm.coords[:, 1])
        f[sel] = ft[loc]
        hs.append(O.Hierarchy(Vt, Tt, lm.level, 2, k_func=kf))
    u = torch.zeros(n, device="cuda", dtype=torch.float64)
    H.hhg_vcycle(m.h, 2, 2, H.HHG_SMOOTH_JACOBI, torch.tensor(f, device="cuda"), u, H.HHG_F64)
    got = u.cpu().numpy()
    for (sel, loc, lm, Vt, Tt), Hh in zip(parts, hs):
        ft = np.zeros(lm.n)
        ft[loc] = f[sel]
        un = Hh.vcycle(lm.level, ft[lm.unknowns], np.zeros(len(lm.unknowns)))
        want = np.zeros(lm.n)
        want[lm.unknowns] = un
        assert _rel(got[sel], want[loc]) <= 1e-10
    x = torch.zeros(n, device="cuda", dtype=torch.float64)
    st = H.hhg_solve(m.h, torch.tensor(f, device="cuda"), x, tol=1e-10, mode=H.HHG_SOLVE_MIXED)
    assert st["rel_residual"] <= 1e-10
    got = x.cpu().numpy()
    for (sel, loc, lm, Vt, Tt), Hh in zip(parts, hs):
        ft = np.zeros(lm.n)
        ft[loc] = f[sel]
        xs = np.zeros(lm.n)
        xs[lm.unknowns] = Hh.direct_solve(ft[lm.unknowns])
        assert _rel(got[sel], xs[loc]) <= 1e-7
    m.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_chebyshev_solve(H, mode):
    V, T = I.cube24()
    c = Case(H, V, T, 3, 1, I.k_large)
    f_or = np.where(c.dir, 0.0, c.lm.assemble_mass() @ np.ones(c.lm.n))
    ud = torch.zeros(c.n, device="cuda", dtype=torch.float64)
    st = H.hhg_solve(c.m.h, c.dev(f_or, 0), ud, tol=1e-9, mode=mode, smoother=H.HHG_SMOOTH_CHEBYSHEV)
    assert st["rel_residual"] <= 1e-9
    import scipy.sparse.linalg as spla
    A = c.lm.system(c.k_or, "scaled")
    xs = np.zeros(c.lm.n)
    xs[c.lm.unknowns] = spla.spsolve(A.tocsc(), f_or[c.lm.unknowns])
    assert _rel(c.back(ud), xs) <= 1e-7


def test_device_status_clean(H, case):
    H.hhg_device_status(case.m.h)  # raises on a recorded timeout


@pytest.mark.parametrize("kind,op", [("scaled", 0), ("volface", 1), ("nodal", 2)])
@pytest.mark.parametrize("name", ["kuhn_cube_l4", "cube12_l3"])
def test_mg_solver_parity(H, name, kind, op):
    """HHG_SOLVE_MG (FP64 V(3,3) cycles as the solver) with each operator
    against the oracle hierarchy of the same operator: the iterate after 3
    cycles (1e-10) and the rate rho over 10 cycles."""
    mesh, level, coarsest, kf = MESHES[name]
    V, T = mesh()
    c = Case(H, V, T, level, coarsest, kf)
    Ho = O.Hierarchy(V, T, level, coarsest, k_func=kf, kind=kind)
    f_or = c.rand_or
    fu = f_or[c.lm.unknowns]
    for its in (3, 10):
        u = torch.zeros(c.n, device="cuda", dtype=torch.float64)
        st = H.hhg_solve(c.m.h, c.dev(f_or, 0), u, tol=1e-30, maxit=its, mode=H.HHG_SOLVE_MG, nu1=3, nu2=3,
                         op=op, raise_on_fail=False)
        assert st["iterations"] == its
        x, hist = Ho.mg_solve(fu, its)
        got = c.back(u)[c.lm.unknowns]
        assert _rel(got, x) <= 1e-10, _rel(got, x)
        if its == 10:
            assert abs(st["rho"] - O.mg_rate(hist)) <= 1e-6 * O.mg_rate(hist)
            assert 0 < st["rho"] < 0.5
    c.m.close()


def test_mg_solver_rejects_operator_outside_mg_mode(H):
    mesh, level, coarsest, kf = MESHES["kuhn_cube_l4"]
    V, T = mesh()
    c = Case(H, V, T, level, coarsest, kf)
    u = torch.zeros(c.n, device="cuda", dtype=torch.float64)
    with pytest.raises(H.HHGError, match="HHG_SOLVE_MG"):
        H.hhg_solve(c.m.h, c.dev(c.rand_or, 0), u, mode=H.HHG_SOLVE_FP64, op=H.HHG_OP_VOLFACE)
    c.m.close()


# the tensor operator's column march: several column tiles (30 wide) and row
# tiles (16 high) per macro-tet with ragged last tiles at levels 5 and 6
TENSOR_MESHES = {**MESHES, "cube12_l5": (I.cube12, 5, 2, I.k_cube), "kuhn_cube_l6": (I.kuhn_cube, 6, 2, I.k_cube)}


def _tensor_case(H, name):
    mesh, level, coarsest, kf = TENSOR_MESHES[name]
    V, T = mesh()
    c = Case(H, V, T, level, coarsest, kf)
    K6 = np.ascontiguousarray(I.K_tensor(c.xyz).T)  # (6, n_stored)
    H.hhg_set_tensor_coefficient(c.m.h, torch.tensor(K6, device="cuda"))
    return c, (V, T, level, coarsest)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("name", ["kuhn_cube_l4", "cube12_l3", "cube12_l5", "kuhn_cube_l6"])
def test_tensor_apply_parity(H, name, dtype):
    """Scaled operator of the tensor coefficient (M = 6) against the oracle's
    element loop over the six terms; FP32 on FP32-rounded inputs."""
    c, _ = _tensor_case(H, name)
    km = O.tensor_split(I.K_tensor(c.lm.coords))
    u = c.rand_or
    if dtype == H.HHG_F32:
        km, u = _f32(km), _f32(u)
    ud = c.dev(u, dtype)
    y = torch.empty_like(ud)
    H.hhg_apply_tensor(c.m.h, 0, ud, y, dtype)
    torch.cuda.synchronize()
    got = c.back(y)
    want = O.tensor_apply(c.lm, u, km, "scaled")
    tol = 1e-12 if dtype == H.HHG_F64 else 1e-6
    assert _rel(got, want) <= tol, _rel(got, want)
    assert np.all(got[c.dir] == 0)
    c.m.close()


@pytest.mark.parametrize("name", ["kuhn_cube_l4", "cube12_l3", "cube12_l5"])
def test_tensor_mg_solver_parity(H, name):
    c, (V, T, level, coarsest) = _tensor_case(H, name)
    Ho = O.Hierarchy(V, T, level, coarsest, K_func=I.K_tensor)
    fu = c.rand_or[c.lm.unknowns]
    for its in (3, 10):
        u = torch.zeros(c.n, device="cuda", dtype=torch.float64)
        st = H.hhg_solve(c.m.h, c.dev(c.rand_or, 0), u, tol=1e-30, maxit=its, mode=H.HHG_SOLVE_MG, nu1=3, nu2=3,
                         op=H.HHG_OP_TENSOR, raise_on_fail=False)
        x, hist = Ho.mg_solve(fu, its)
        assert _rel(c.back(u)[c.lm.unknowns], x) <= 1e-10
        if its == 10:
            assert abs(st["rho"] - O.mg_rate(hist)) <= 1e-6 * O.mg_rate(hist)
    c.m.close()


def test_tensor_operator_needs_its_coefficient(H):
    mesh, level, coarsest, kf = MESHES["kuhn_cube_l4"]
    V, T = mesh()
    c = Case(H, V, T, level, coarsest, kf)
    ud = c.dev(c.rand_or, 0)
    with pytest.raises(H.HHGError, match="tensor"):
        H.hhg_apply_tensor(c.m.h, 0, ud, torch.empty_like(ud), H.HHG_F64)
    c.m.close()


def test_tensor_mg_solve_needs_no_scalar_coefficient(H):
    V, T = I.kuhn_cube()
    m = H.Mesh(V, T, 4, 2)
    off, lev, n = m.layout(0)
    xyz = m.coords(0)
    H.hhg_set_tensor_coefficient(m.h, torch.tensor(np.ascontiguousarray(I.K_tensor(xyz).T), device="cuda"))
    f = torch.tensor(np.where(np.any((xyz <= 0) | (xyz >= 1), axis=1), 0.0, 1.0), device="cuda")
    u = torch.zeros(n, device="cuda", dtype=torch.float64)
    st = H.hhg_solve(m.h, f, u, tol=1e-9, maxit=60, mode=H.HHG_SOLVE_MG, nu1=3, nu2=3, op=H.HHG_OP_TENSOR)
    assert st["rel_residual"] <= 1e-9 and 0 < st["rho"] < 0.5
    m.close()


def test_zero_sweeps_and_single_depth_mesh(H):
    """Degenerate calls: zero smoothing sweeps leave u unchanged; a mesh whose
    finest level is the coarsest one has one depth, and the solver is then
    the dense coarse solve (exact to rounding)."""
    mesh, level, coarsest, kf = MESHES["kuhn_cube_l4"]
    V, T = mesh()
    c = Case(H, V, T, level, coarsest, kf)
    f = c.dev(c.rand_or, 0)
    u = f.flip(0).contiguous()
    u0 = u.clone()
    H.hhg_smooth(c.m.h, 0, H.HHG_SMOOTH_JACOBI, 0, 0.6, f, u, H.HHG_F64)
    H.hhg_smooth(c.m.h, 0, H.HHG_SMOOTH_CHEBYSHEV, 0, 0.6, f, u, H.HHG_F64)
    torch.cuda.synchronize()
    assert torch.equal(u, u0)
    c.m.close()
    c2 = Case(H, V, T, 2, 2, kf)
    assert c2.m.ndepth == 1
    f = c2.rand_or
    u = torch.zeros(c2.n, device="cuda", dtype=torch.float64)
    st = H.hhg_solve(c2.m.h, c2.dev(f, 0), u, tol=1e-12, mode=H.HHG_SOLVE_FP64)
    A = c2.lm.system(c2.k_or, "scaled")
    x = np.linalg.solve(A.toarray(), f[c2.lm.unknowns])
    assert _rel(c2.back(u)[c2.lm.unknowns], x) <= 1e-10 and st["iterations"] <= 2
    c2.m.close()


# The three volume kernels of the scaled operator: the tile march (vkernel
# 0), the column march (1) and the column march with two column sets per
# lane in packed FP32x2 arithmetic (2; FP64 runs as 1).  Meshes with several
# 30- and 60-column tiles per tet and ragged last tiles.
VK_MESHES = {"kuhn_cube_l6": (I.kuhn_cube, 6, 2, I.k_cube), "cube24_l5": (I.cube24, 5, 2, I.k_large),
             "cube48_l5": (I.cube48, 5, 2, I.k_batched(1))}


@pytest.fixture(scope="module", params=list(VK_MESHES))
def vk_case(request, H):
    mesh, level, coarsest, kf = VK_MESHES[request.param]
    V, T = mesh()
    c = Case(H, V, T, level, coarsest, kf)
    c.f_or = np.where(c.dir, 0.0, np.sin(7 * c.lm.coords[:, 0]) + c.lm.coords[:, 2])
    return c


@pytest.mark.parametrize("vkernel", [0, 1, 2])
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_volume_kernels_apply_residual_jacobi(H, vk_case, vkernel, dtype):
    c = vk_case
    H.hhg_set_option(c.m.h, "vkernel", vkernel)
    try:
        tol = 1e-12 if dtype == H.HHG_F64 else 1e-6
        rnd = (lambda x: x) if dtype == H.HHG_F64 else _f32
        u, f = rnd(c.rand_or), rnd(c.f_or)
        kp = c.kprec(dtype)
        ud, fd = c.dev(u, dtype), c.dev(f, dtype)
        y = torch.empty_like(ud)
        H.hhg_apply_scaled(c.m.h, 0, ud, y, dtype)
        Au = c.lm.apply(u, kp, "scaled")
        assert _rel(c.back(y), Au) <= tol, _rel(c.back(y), Au)
        H.hhg_residual(c.m.h, 0, fd, ud, y, dtype)
        want = np.where(c.dir, 0.0, f - Au)
        assert _rel(c.back(y), want) <= tol, _rel(c.back(y), want)
        # one damped Jacobi sweep: u + omega (f - A u) / diag(A)
        Dg = np.ones(c.lm.n)
        Dg[c.lm.unknowns] = c.lm.system(kp, "scaled").diagonal()
        H.hhg_smooth(c.m.h, 0, H.HHG_SMOOTH_JACOBI, 1, 0.6, fd, ud, dtype)
        want = np.where(c.dir, 0.0, u + 0.6 * (f - Au) / Dg)
        assert _rel(c.back(ud), want) <= (1e-12 if dtype == H.HHG_F64 else 1e-5)
    finally:
        H.hhg_set_option(c.m.h, "vkernel", 1)


@pytest.mark.parametrize("dtype", [1, 2])
def test_two_column_sets_chebyshev_sweeps_match_the_column_march(H, vk_case, dtype):
    """Three Chebyshev sweeps (the smoother's recurrence carries d between
    sweeps) with vkernel 2 against vkernel 1 (itself checked against the
    oracle through the V-cycle tests)."""
    c = vk_case
    f = c.dev(_f32(c.f_or), dtype)
    outs = []
    for vk in (1, 2):
        H.hhg_set_option(c.m.h, "vkernel", vk)
        ud = c.dev(_f32(c.rand_or), dtype)
        H.hhg_smooth(c.m.h, 0, H.HHG_SMOOTH_CHEBYSHEV, 3, 0.6, f, ud, dtype)
        outs.append(c.back(ud))
    H.hhg_set_option(c.m.h, "vkernel", 1)
    assert _rel(outs[1], outs[0]) <= 1e-5, _rel(outs[1], outs[0])


@pytest.mark.parametrize("dtype", [1, 2])
def test_one_and_two_column_sets_round_alike(H, vk_case, dtype):
    """The packed FP32x2 march rounds each component as the scalar march
    does (same operations in the same order, no contraction): apply and
    residual bitwise equal."""
    c = vk_case
    ud, fd = c.dev(_f32(c.rand_or), dtype), c.dev(_f32(c.f_or), dtype)
    outs = []
    for vk in (1, 2):
        H.hhg_set_option(c.m.h, "vkernel", vk)
        y, r = torch.empty_like(ud), torch.empty_like(ud)
        H.hhg_apply_scaled(c.m.h, 0, ud, y, dtype)
        H.hhg_residual(c.m.h, 0, fd, ud, r, dtype)
        outs.append((y, r))
    H.hhg_set_option(c.m.h, "vkernel", 1)
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1])
