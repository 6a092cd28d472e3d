"""Parity at the full size of the large configuration: the unit cube split
into 24 macro tetrahedra, every one at level 9 (513 nodes per edge,
543,184,920 stored nodes), FP32 u with the coefficient in BF16,
k = 1 + 0.5 sin(4 pi x) cos(4 pi y) sin(4 pi z).

The coefficient handed to the library is k rounded to bfloat16, so the BF16
copy the kernels read equals it exactly and every precision solves the same
discrete problem.  u is a rough field (a hash of the node's coordinates on
the 1/1024 lattice, the same value on every copy), 0 on Dirichlet nodes as
the ABI requires.

- Apply: sampled rows of the FP32 / BF16-k operator (autotuned work lists,
  the launch configuration of the other full-size applies), volume rows and
  rows on macro faces, edges and vertices, against the oracle's one-row
  evaluator (row_apply, pinned against the element loop) with the same
  inputs.  Tolerance 1e-6 of the largest sampled row value (sums of 14 FP32
  products, as for the other FP32 applies).
- Solve: mixed-precision GMG-CG with the BF16 coefficient, rhs M 1; the FP64
  residual the test computes with the FP64 operator (whose k holds the same
  bfloat16 values) is within the requested 1e-8 (a property at any size).
"""
import numpy as np
import pytest

from oracle import hhg_oracle as O
from paper_1709_06793_gb300 import inputs as I
from tests import hhg_testutil as U

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LEVEL = 9


def _bf16(x):
    """Round positive values to bfloat16 (8 significant bits), nearest-even."""
    x = np.asarray(x, dtype=np.float64)
    q = np.exp2(np.floor(np.log2(x)) - 7)
    return np.round(x / q) * q


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def _u_field(X):
    """Rough field in [-1, 1) from the node's coordinates (every level-9 node
    of this mesh lies on the 1/1024 lattice, and both sides form the
    coordinates exactly)."""
    return U.lattice_field(X, 1024)


def _k_field(X):
    return _bf16(I.k_large(X))


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06793_gb300 import build
    build.build()
    from paper_1709_06793_gb300 import hhg as H
    V, T = I.cube24()
    m = H.Mesh(V, T, LEVEL, 2)
    off, lev, n = m.layout(0)
    X = m.coords(0)
    k = np.empty(n)
    u = np.empty(n, dtype=np.float32)
    step = 1 << 25
    for a in range(0, n, step):
        b = min(n, a + step)
        k[a:b] = _k_field(X[a:b])
        u[a:b] = _u_field(X[a:b])
    del X
    H.hhg_set_coefficient(m.h, torch.from_numpy(k).cuda())
    del k
    yield H, m, V, T, off, lev, n, u
    m.close()


def test_layout_index_helper_matches_enumeration():
    """The node-index helper the sampling below uses agrees with the stored
    enumeration (small level; bookkeeping only)."""
    off = np.array([0, 35, 70])
    lev = np.array([2, 2])
    nodes = U.stored_nodes(off, lev)
    t, i, j, k = nodes.T
    np.testing.assert_array_equal(U.node_index(off, t, i, j, k, 4), np.arange(len(nodes)))


def _sample_nodes(rng, nt, N, n_vol, n_face):
    t = rng.integers(0, nt, n_vol + n_face)
    ijk = []
    while len(ijk) < n_vol:  # strictly inside the tet
        c = rng.integers(1, N - 1, 3)
        if c.sum() <= N - 1:
            ijk.append(c)
    for _ in range(n_face):  # on a face (edges and vertices included)
        while True:
            a, b = rng.integers(0, N + 1, 2)
            if a + b <= N:
                break
        f = rng.integers(0, 4)
        ijk.append([(0, a, b), (a, 0, b), (a, b, 0), (a, b, N - a - b)][f])
    # the four macro vertices of tet 0 as well
    extra = [(0, 0, 0), (N, 0, 0), (0, N, 0), (0, 0, N)]
    t = np.concatenate([t, np.zeros(len(extra), dtype=t.dtype)])
    ijk = np.array(list(ijk) + extra, dtype=np.int64)
    return t, ijk[:, 0], ijk[:, 1], ijk[:, 2]


def test_large_bf16k_apply_sampled(big):
    H, m, V, T, off, lev, n, u = big
    N = 1 << LEVEL
    ud = torch.from_numpy(u).cuda()
    mask = torch.empty_like(ud)
    H.hhg_residual(m.h, 0, torch.ones_like(ud), torch.zeros_like(ud), mask, H.HHG_F32_KBF16)
    ud *= mask
    H.hhg_autotune(m.h, H.HHG_F32_KBF16)
    y = torch.empty_like(ud)
    H.hhg_apply_scaled(m.h, 0, ud, y, H.HHG_F32_KBF16)
    torch.cuda.synchronize()
    rng = np.random.default_rng(21)
    t, i, j, k = _sample_nodes(rng, len(T), N, 1200, 600)
    idx = U.node_index(off, t, i, j, k, N)
    got = y[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    mm = O.MacroMesh(V, T)
    Tn = np.asarray(T)

    def field_u(gv, W, X):
        return _f32(_u_field(X))

    def field_k(gv, W, X):
        return _k_field(X)

    want = np.empty(len(t))
    for q in range(len(t)):
        Wt = np.array([N - i[q] - j[q] - k[q], i[q], j[q], k[q]])
        sup, w = Tn[t[q]][Wt > 0], Wt[Wt > 0]
        want[q] = O.row_apply(mm, LEVEL, sup, w, field_u, field_k, "scaled")
    scale = np.max(np.abs(want))
    assert scale > 0
    err = np.max(np.abs(got - want)) / scale
    assert err <= 1e-6, err


def test_large_bf16k_mixed_solve_residual(big):
    """BF16-k mixed solve at full size: the oracle's FP64 residual of the
    returned solution at sampled volume and interface rows (the coefficient
    is the bfloat16-rounded k the library was given) is within the requested
    1e-8 of ||f||_2 (bounded above here by the 2-norm over all stored copies),
    and the library's FP64 residual agrees with it at those rows."""
    H, m, V, T, off, lev, n, u = big
    ones = torch.ones(n, device="cuda", dtype=torch.float64)
    f = torch.empty_like(ones)
    H.hhg_apply_mass(m.h, 0, ones, f, H.HHG_F64)
    del ones
    x = torch.zeros_like(f)
    st = H.hhg_solve(m.h, f, x, tol=1e-8, mode=H.HHG_SOLVE_MIXED_KBF16)
    assert st["rel_residual"] <= 1e-8, st
    nf_upper = float(torch.sqrt(torch.sum(f * f)))
    sample, r_or = U.sampled_residuals(O, H, m, V, T, LEVEL, x, f, _k_field, 200, 100, seed=31)
    assert np.max(np.abs(r_or)) <= 1e-8 * nf_upper, (np.max(np.abs(r_or)), nf_upper)
    r = torch.empty_like(x)
    H.hhg_residual(m.h, 0, f, x, r, H.HHG_F64)
    r_lib = r[torch.as_tensor(sample, device="cuda")].cpu().numpy()
    # both are FP64 sums of a row's terms, whose size is bounded by
    # 2 kmax sum_d |c_d| max|x| (the volume stencil; f itself is far smaller)
    c = np.abs(m.stencils(0, 0)[0]).sum()
    scale = 2 * 1.5 * c * float(torch.max(torch.abs(x)))
    assert np.max(np.abs(r_lib - r_or)) <= 1e-13 * scale, (np.max(np.abs(r_lib - r_or)), scale)
