"""The stated precision errors of the solves.

Rounding k to bfloat16 (relative error at most delta = 2^-8 per node, RN)
moves the discrete solution.  Where the stiffness matrix is a sum over
micro edges of k_edge times positive semi-definite edge matrices (every
off-diagonal reference weight <= 0, as on the Kuhn cube, whose reference
stencil is the 7-point one), (1 - delta) A(k) <= A(k_bf16) <= (1 + delta) A(k)
in the Loewner order, so the energy-norm shift is at most delta / (1 - delta):
the oracle's shift is checked against that bound (and to be non-zero).  On
the GPU the shift between the BF16-k solve (mode 2) and the FP64 solve
equals the oracle's, and the solve with BF16 k in the inner solve only
(mode 4) reaches the FP64-k solution.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import hhg_oracle as O
from paper_1709_06793_gb300 import inputs as I

DELTA = 2.0 ** -8  # unit roundoff of bfloat16 (8 significant bits)
LEVEL = 5


def _bf16(x):
    """Round positive values to bfloat16 (8 significant bits), nearest-even."""
    x = np.asarray(x, dtype=np.float64)
    q = np.exp2(np.floor(np.log2(x)) - 7)
    return np.round(x / q) * q


def _problem():
    V, T = I.kuhn_cube()
    lm = O.LevelMesh(O.MacroMesh(V, T), LEVEL)
    k = I.k_cube(lm.coords)
    f = np.where(lm.dirichlet, 0.0, lm.assemble_mass() @ I.f_cube_sine(lm.coords))
    return V, T, lm, k, f


def _solve(lm, k, f):
    A = lm.system(k, "scaled")
    x = np.zeros(lm.n)
    x[lm.unknowns] = spla.spsolve(A.tocsc(), f[lm.unknowns])
    return x


def _energy(lm, A, e):
    e = e[lm.unknowns]
    return math.sqrt(abs(float(e @ (A @ e))))


def oracle_shift():
    V, T, lm, k, f = _problem()
    x = _solve(lm, k, f)
    xq = _solve(lm, _bf16(k), f)
    A = lm.system(k, "scaled")
    return V, T, lm, k, f, x, xq, _energy(lm, A, xq - x) / _energy(lm, A, x)


def test_bf16_rounding_is_within_half_an_ulp():
    k = I.k_cube(np.random.default_rng(0).uniform(0, 1, (10000, 3)))
    rel = np.abs(_bf16(k) - k) / k
    assert rel.max() <= DELTA and rel.max() > 0.5 * DELTA


def test_oracle_bf16_solution_shift_is_within_the_loewner_bound():
    V, T, lm, k, f, x, xq, shift = oracle_shift()
    # the hypothesis of the bound: the reference stencil's off-diagonal weights
    # (every primitive of the Kuhn cube) are <= 0
    A1 = lm.system(np.ones(lm.n), "scaled").tocoo()
    off = A1.row != A1.col
    assert np.all(A1.data[off] <= 1e-14)
    assert 0.0 < shift <= DELTA / (1.0 - DELTA)


@pytest.mark.gpu
def test_gpu_bf16_solution_shift_matches_the_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06793_gb300 import build
    build.build()
    from paper_1709_06793_gb300 import hhg as H
    from tests import hhg_testutil as U

    V, T, lm, k, f, x, xq, shift = oracle_shift()
    m = H.Mesh(V, T, LEVEL, 2)
    off, lev, n = m.layout(0)
    idx = U.oracle_map(lm, U.stored_nodes(off, lev))
    H.hhg_set_coefficient(m.h, torch.tensor(I.k_cube(m.coords(0)), device="cuda"))
    fd = torch.tensor(f[idx], device="cuda")
    sols = {}
    for mode in (H.HHG_SOLVE_FP64, H.HHG_SOLVE_MIXED_KBF16, H.HHG_SOLVE_MIXED_KBF16_INNER):
        u = torch.zeros(n, device="cuda", dtype=torch.float64)
        st = H.hhg_solve(m.h, fd, u, tol=1e-11, mode=mode, max_outer=40)
        assert st["rel_residual"] <= 1e-11
        sols[mode] = u
    y = torch.empty_like(fd)

    def energy(e):
        H.hhg_apply_scaled(m.h, 0, e, y, H.HHG_F64)
        return math.sqrt(abs(H.hhg_dot(m.h, 0, e, y, H.HHG_F64)))

    x64 = sols[H.HHG_SOLVE_FP64]
    nx = energy(x64)
    gpu_shift = energy(sols[H.HHG_SOLVE_MIXED_KBF16] - x64) / nx
    assert abs(gpu_shift - shift) <= 1e-4 * shift, (gpu_shift, shift)
    assert energy(sols[H.HHG_SOLVE_MIXED_KBF16_INNER] - x64) / nx <= 1e-8
    m.close()
