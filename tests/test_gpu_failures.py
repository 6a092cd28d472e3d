"""Failure paths that need no GPU fault: a solver stopped by its iteration
limits, a coefficient the library must refuse, a learned smoother the plain
V-cycle rejects, and a learned inner solve that fails and is replaced by the
plain V-cycle.  Every failure is made on the host side (arguments, weights)."""
import math

import numpy as np
import pytest

from oracle import learned_oracle as LO
from paper_1709_06793_gb300 import inputs as I

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


def _cube(H, level=5):
    V, T = I.kuhn_cube()
    m = H.Mesh(V, T, level, 2)
    off, lev, n = m.layout(0)
    xyz = m.coords(0)
    H.hhg_set_coefficient(m.h, torch.tensor(I.k_cube(xyz), device="cuda"))
    fi = torch.tensor(I.f_cube_sine(xyz), device="cuda")
    f = torch.empty_like(fi)
    H.hhg_apply_mass(m.h, 0, fi, f, H.HHG_F64)
    return m, n, xyz, f


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_iteration_limit_returns_not_converged_with_stats(H, mode):
    m, n, xyz, f = _cube(H)
    u = torch.zeros(n, device="cuda", dtype=torch.float64)
    if mode == "fp64":
        st = H.hhg_solve(m.h, f, u, tol=1e-8, maxit=2, mode=H.HHG_SOLVE_FP64, raise_on_fail=False)
        assert st["iterations"] == 2
    else:
        st = H.hhg_solve(m.h, f, u, tol=1e-8, maxit=3, mode=H.HHG_SOLVE_MIXED, max_outer=1, raise_on_fail=False)
        assert 1 <= st["iterations"] <= 3 and st["outer"] == 1
    assert st["status"] == "HHG_ERR_NOT_CONVERGED"
    assert math.isfinite(st["rel_residual"]) and 1e-8 < st["rel_residual"] < 1.0
    with pytest.raises(H.HHGError) as e:
        H.hhg_solve(m.h, f, torch.zeros_like(u), tol=1e-8, maxit=2, mode=H.HHG_SOLVE_FP64)
    assert e.value.code == -4
    m.close()


@pytest.mark.parametrize("bad", ["nan", "zero", "negative", "inf"])
def test_set_coefficient_rejects_bad_values(H, bad):
    m, n, xyz, f = _cube(H, 4)
    k = torch.tensor(I.k_cube(xyz), device="cuda")
    bk = k.clone()
    bk[n // 3] = {"nan": float("nan"), "zero": 0.0, "negative": -0.5, "inf": float("inf")}[bad]
    with pytest.raises(H.HHGError) as e:
        H.hhg_set_coefficient(m.h, bk)
    assert e.value.code == -1 and "finite and positive" in str(e.value)
    # the mesh keeps the previous coefficient and still solves
    u = torch.zeros(n, device="cuda", dtype=torch.float64)
    st = H.hhg_solve(m.h, f, u, tol=1e-8, mode=H.HHG_SOLVE_MIXED)
    assert st["rel_residual"] <= 1e-8
    m.close()


def test_rejected_network_leaves_the_plain_vcycle(H):
    """A network of large random weights (one training step at a negligible
    learning rate) converges worse than the plain V-cycle; the judge rejects
    it and hhg_solve runs the plain V-cycle (stats.smoother_used)."""
    m, n, xyz, f = _cube(H)
    st = H.hhg_learned_train(m.h, steps=1, pairs=1, lr=1e-12, init_noise=3.0, seed=11, weights_bf16=1)
    assert st["accepted"] == 0, st
    assert st["rho_learned"] >= st["rho_plain"]
    u = torch.zeros(n, device="cuda", dtype=torch.float64)
    s = H.hhg_solve(m.h, f, u, tol=1e-8, mode=H.HHG_SOLVE_MIXED, smoother=H.HHG_SMOOTH_LEARNED)
    assert s["smoother_used"] == H.HHG_SMOOTH_JACOBI and s["rel_residual"] <= 1e-8
    m.close()


def test_failed_learned_inner_solve_falls_back(H):
    """A network with NaN weights, installed directly (no judge), makes the
    first learned inner solve fail; the solve discards it, continues with the
    plain V-cycle and still reaches the tolerance."""
    m, n, xyz, f = _cube(H)
    w = np.full(LO.N_W, np.nan, dtype=np.float32)
    H.hhg_learned_set_weights(m.h, w, weights_bf16=0)
    u = torch.zeros(n, device="cuda", dtype=torch.float64)
    s = H.hhg_solve(m.h, f, u, tol=1e-8, mode=H.HHG_SOLVE_MIXED, smoother=H.HHG_SMOOTH_LEARNED)
    assert s["smoother_used"] == H.HHG_SMOOTH_JACOBI
    assert s["rel_residual"] <= 1e-8 and torch.isfinite(u).all()
    m.close()
