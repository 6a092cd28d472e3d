"""GPU parity of the learned smoother against the FP64 oracle
(oracle/learned_oracle.py), and what training gains.

Tolerances (max-norm error relative to the largest oracle value):
* FP32 weights: the kernels form sums of at most 54 (layer 1) and 432
  (layer 2) FP32 products per value, so a few hundred units of 2^-24 bound the
  error: 1e-5.  Weight gradients sum FP32 products over 8^3-node tiles and the
  tiles in FP64: the same bound, 1e-5.
* BF16 weights against the oracle given the same BF16-rounded weights: only
  the accumulation differs, 1e-5.  Against the unrounded FP32 weights the
  rounding of each weight (2^-9 relative) dominates: 1e-2 for the output;
  the gradient, a product of both layers' weights, moves by up to 2e-2, and
  by no more than the oracle's own gradient moves under the same rounding.
"""
import numpy as np
import pytest

from oracle import hhg_oracle as O
from oracle import learned_oracle as LO
from paper_1709_06793_gb300 import inputs as I
from tests.hhg_testutil import oracle_map, stored_nodes

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


def bf16_round(w):
    return torch.tensor(np.asarray(w, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


class Case:
    """Kuhn cube at `level` (coarsest 2), k = k_cube; oracle hierarchy alongside."""

    def __init__(self, H, level=4, kf=I.k_cube, mesh=I.kuhn_cube):
        V, T = mesh()
        self.H = H
        self.m = H.Mesh(V, T, level, 2)
        self.level = level
        self.Ho = O.Hierarchy(V, T, level, 2, k_func=kf)
        off, lev, n = self.m.layout(0)
        H.hhg_set_coefficient(self.m.h, torch.tensor(kf(self.m.coords(0)), device="cuda"))
        self.maps = {}

    def depth(self, d):
        if d not in self.maps:
            off, lev, n = self.m.layout(d)
            lm = self.Ho.mesh[self.level - d]
            self.maps[d] = (lm, oracle_map(lm, stored_nodes(off, lev)), n)
        return self.maps[d]

    def pair(self, d, seed):
        """(r, e) on the oracle's unique nodes with r = A e (FP64), rounded to
        FP32 values."""
        lm, mp, n = self.depth(d)
        l = self.level - d
        rng = np.random.default_rng(seed)
        e = np.zeros(lm.n)
        e[lm.unknowns] = rng.uniform(-1, 1, len(lm.unknowns))
        e = e.astype(np.float32).astype(np.float64)
        r = np.zeros(lm.n)
        r[lm.unknowns] = self.Ho.A[l] @ e[lm.unknowns]
        r = r.astype(np.float32).astype(np.float64)
        return r, e

    def diag_k(self, d):
        lm, mp, n = self.depth(d)
        l = self.level - d
        diag = np.ones(lm.n)
        diag[lm.unknowns] = self.Ho.D[l]
        return diag, self.Ho.k[l]

    def dev(self, d, x_unique):
        lm, mp, n = self.depth(d)
        return torch.tensor(np.asarray(x_unique)[mp], device="cuda", dtype=torch.float32)

    def close(self):
        self.m.close()


def rel_err(gpu, ref):
    return float(np.max(np.abs(gpu - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("bf16", [0, 1])
@pytest.mark.parametrize("d", [0, 1])
def test_forward_matches_oracle(H, bf16, d):
    c = Case(H)
    rng = np.random.default_rng(10 + d)
    w = rng.normal(0, 0.3, LO.N_W).astype(np.float32)
    H.hhg_learned_set_weights(c.m.h, w, weights_bf16=bf16)
    r, e = c.pair(d, 20 + d)
    lm, mp, n = c.depth(d)
    diag, k = c.diag_k(d)
    cg = torch.zeros(n, device="cuda", dtype=torch.float32)
    H.hhg_learned_forward(c.m.h, d, c.dev(d, r), cg)
    cg = cg.cpu().numpy().astype(np.float64)
    a0, a1 = LO.features(lm, r, diag, k)
    w_used = bf16_round(w) if bf16 else w.astype(np.float64)
    ref = LO.forward(lm, w_used, a0, a1)[0][mp]
    assert rel_err(cg, ref) <= 1e-5
    if bf16:
        ref32 = LO.forward(lm, w.astype(np.float64), a0, a1)[0][mp]
        assert rel_err(cg, ref32) <= 1e-2
    c.close()


@pytest.mark.parametrize("bf16", [0, 1])
@pytest.mark.parametrize("d", [0, 1])
def test_loss_and_gradient_match_oracle(H, bf16, d):
    c = Case(H)
    rng = np.random.default_rng(30 + d)
    w = rng.normal(0, 0.3, LO.N_W).astype(np.float32)
    H.hhg_learned_set_weights(c.m.h, w, weights_bf16=bf16)
    r, e = c.pair(d, 40 + d)
    lm, mp, n = c.depth(d)
    diag, k = c.diag_k(d)
    loss, g = H.hhg_learned_loss_grad(c.m.h, d, c.dev(d, r), c.dev(d, e))
    l = c.level - d
    w_used = bf16_round(w) if bf16 else w.astype(np.float64)
    loss_o, g_o, _ = LO.loss_and_grad(lm, c.Ho.A[l], w_used, r, e, diag, k)
    assert abs(loss - loss_o) <= 1e-5 * abs(loss_o)
    assert rel_err(g, g_o) <= 1e-5
    if bf16:
        # rounding the weights moves the gradient itself: the GPU's distance to
        # the FP32-weight gradient is the oracle's own (plus accumulation)
        g32 = LO.loss_and_grad(lm, c.Ho.A[l], w.astype(np.float64), r, e, diag, k)[1]
        assert rel_err(g, g32) <= rel_err(g_o, g32) + 1e-5
        assert rel_err(g, g32) <= 2e-2
    c.close()


@pytest.mark.parametrize("d", [0, 1])
def test_tensor_core_forward_matches_oracle(H, d):
    """BF16 forward on the tensor cores (mma.sync, BF16 inputs, hidden
    activations and per-tap partial products, FP32 accumulation).  Rounding
    the two input channels, the 16 hidden channels and the 27 per-tap
    partials to BF16 (2^-9 relative each) before FP32 sums of 54, 16 and 27
    terms bounds the error by a few 2^-9 of the largest value: 1e-2."""
    c = Case(H)
    rng = np.random.default_rng(80 + d)
    w = rng.normal(0, 0.3, LO.N_W).astype(np.float32)
    H.hhg_learned_set_weights(c.m.h, w, weights_bf16=1)
    H.hhg_set_option(c.m.h, "learned_tc_all", 1)
    assert H.hhg_get_option(c.m.h, "learned_tc_all") == 1
    r, e = c.pair(d, 90 + d)
    lm, mp, n = c.depth(d)
    diag, k = c.diag_k(d)
    cg = torch.zeros(n, device="cuda", dtype=torch.float32)
    H.hhg_learned_forward(c.m.h, d, c.dev(d, r), cg)
    H.hhg_set_option(c.m.h, "learned_tc_all", 0)
    cf = torch.zeros(n, device="cuda", dtype=torch.float32)
    H.hhg_learned_forward(c.m.h, d, c.dev(d, r), cf)
    cg = cg.cpu().numpy().astype(np.float64)
    ref = LO.forward(lm, bf16_round(w), *LO.features(lm, r, diag, k))[0][mp]
    assert rel_err(cg, ref) <= 1e-2
    assert rel_err(cg, cf.cpu().numpy().astype(np.float64)) <= 1e-2
    assert rel_err(cg, ref) > 0  # the two paths are distinct kernels
    c.close()


def test_jacobi_network_is_a_jacobi_sweep(H):
    """Weights equal to damped Jacobi (omega = 1/2, exact in BF16): the
    learned correction is one Jacobi sweep from zero."""
    c = Case(H)
    H.hhg_learned_set_weights(c.m.h, LO.jacobi_weights(0.5).astype(np.float32), weights_bf16=1)
    r, e = c.pair(0, 50)
    lm, mp, n = c.depth(0)
    rd = c.dev(0, r)
    cg = torch.zeros(n, device="cuda", dtype=torch.float32)
    H.hhg_learned_forward(c.m.h, 0, rd, cg)
    u = torch.zeros(n, device="cuda", dtype=torch.float32)
    H.hhg_smooth(c.m.h, 0, H.HHG_SMOOTH_JACOBI, 1, 0.5, rd, u, H.HHG_F32)
    torch.cuda.synchronize()
    assert rel_err(cg.cpu().numpy(), u.cpu().numpy()) <= 1e-6
    c.close()


def test_learned_smoothing_matches_oracle_composition(H):
    """hhg_smooth(LEARNED, 3 sweeps) = Jacobi, learned step, Jacobi (oracle)."""
    c = Case(H)
    rng = np.random.default_rng(60)
    w = LO.jacobi_weights(2.0 / 3.0, noise=rng.normal(0, 0.05, LO.N_W))
    H.hhg_learned_set_weights(c.m.h, w.astype(np.float32), weights_bf16=0)
    w = w.astype(np.float32).astype(np.float64)
    lm, mp, n = c.depth(0)
    l = c.level
    A = c.Ho.A[l]
    diag, k = c.diag_k(0)
    x = lm.coords
    f = np.where(lm.dirichlet, 0.0, np.sin(3 * x[:, 0] + x[:, 1]) * np.cos(2 * x[:, 2]))
    u0 = np.where(lm.dirichlet, 0.0, np.cos(2 * x[:, 0] - x[:, 1] + 3 * x[:, 2]))
    f = f.astype(np.float32).astype(np.float64)
    u0 = u0.astype(np.float32).astype(np.float64)
    ud = c.dev(0, u0)
    H.hhg_smooth(c.m.h, 0, H.HHG_SMOOTH_LEARNED, 3, 2.0 / 3.0, c.dev(0, f), ud, H.HHG_F32)
    I_ = lm.unknowns
    u = u0.copy()
    u[I_] = c.Ho.jacobi(l, f[I_], u[I_], 1)
    res = np.zeros(lm.n)
    res[I_] = f[I_] - A @ u[I_]
    u = u + LO.forward(lm, w, *LO.features(lm, res, diag, k))[0]
    u[I_] = c.Ho.jacobi(l, f[I_], u[I_], 1)
    assert rel_err(ud.cpu().numpy().astype(np.float64), u[mp]) <= 1e-5
    c.close()


def test_tensor_core_smoothing_matches_oracle_composition(H):
    """hhg_smooth(LEARNED, 2 sweeps) with BF16 weights on the tensor cores =
    Jacobi then learned step (oracle, BF16-rounded weights), within the BF16
    activation bound of the correction (1e-2 of the correction's size)."""
    c = Case(H)
    rng = np.random.default_rng(61)
    w = LO.jacobi_weights(2.0 / 3.0, noise=rng.normal(0, 0.05, LO.N_W)).astype(np.float32)
    H.hhg_learned_set_weights(c.m.h, w, weights_bf16=1)
    lm, mp, n = c.depth(0)
    l = c.level
    A = c.Ho.A[l]
    diag, k = c.diag_k(0)
    x = lm.coords
    f = np.where(lm.dirichlet, 0.0, np.sin(3 * x[:, 0] + x[:, 1]) * np.cos(2 * x[:, 2])).astype(np.float32)
    u0 = np.where(lm.dirichlet, 0.0, np.cos(2 * x[:, 0] - x[:, 1] + 3 * x[:, 2])).astype(np.float32)
    f, u0 = f.astype(np.float64), u0.astype(np.float64)
    ud = c.dev(0, u0)
    H.hhg_smooth(c.m.h, 0, H.HHG_SMOOTH_LEARNED, 2, 2.0 / 3.0, c.dev(0, f), ud, H.HHG_F32)
    I_ = lm.unknowns
    u = u0.copy()
    u[I_] = c.Ho.jacobi(l, f[I_], u[I_], 1)
    res = np.zeros(lm.n)
    res[I_] = f[I_] - A @ u[I_]
    corr = LO.forward(lm, bf16_round(w), *LO.features(lm, res, diag, k))[0]
    got = ud.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - (u + corr)[mp])) <= 1e-2 * np.max(np.abs(corr))
    c.close()


def test_features_follow_the_coefficient(H):
    c = Case(H)
    rng = np.random.default_rng(70)
    w = rng.normal(0, 0.3, LO.N_W).astype(np.float32)
    H.hhg_learned_set_weights(c.m.h, w, weights_bf16=0)
    r, e = c.pair(0, 71)
    lm, mp, n = c.depth(0)
    cg = torch.zeros(n, device="cuda", dtype=torch.float32)
    H.hhg_learned_forward(c.m.h, 0, c.dev(0, r), cg)
    # new coefficient 2 k: D doubles, log k shifts by log 2
    H.hhg_set_coefficient(c.m.h, torch.tensor(2 * I.k_cube(c.m.coords(0)), device="cuda"))
    cg2 = torch.zeros(n, device="cuda", dtype=torch.float32)
    H.hhg_learned_forward(c.m.h, 0, c.dev(0, r), cg2)
    diag, k = c.diag_k(0)
    ref = LO.forward(lm, w.astype(np.float64), *LO.features(lm, r, 2 * diag, 2 * k))[0][mp]
    assert rel_err(cg2.cpu().numpy().astype(np.float64), ref) <= 1e-5
    assert rel_err(cg.cpu().numpy().astype(np.float64), ref) > 1e-3
    c.close()


def test_training_gains_over_plain_vcycle(H, capsys):
    """Train on the GPU (high-contrast Gaussian-random-field coefficient,
    Kuhn cube) and compare FP32-inner GMG-CG to 1e-8 with and without the
    trained network."""
    V, T = I.kuhn_cube()
    level = 6
    m = H.Mesh(V, T, level, 2)
    k = I.k_learned()(m.coords(0))
    H.hhg_set_coefficient(m.h, torch.tensor(k, device="cuda"))
    st = H.hhg_learned_train(m.h, steps=120, pairs=4, lr=3e-3, max_depth=1, vcycle_pairs=2, init_noise=0.02,
                             seed=3, weights_bf16=1)
    off, lev, n = m.layout(0)
    f = torch.tensor(I.f_cube_sine(m.coords(0)), device="cuda", dtype=torch.float64)
    res = {}
    for name, sm in (("plain", H.HHG_SMOOTH_JACOBI), ("learned", H.HHG_SMOOTH_LEARNED)):
        u = torch.zeros(n, device="cuda", dtype=torch.float64)
        res[name] = H.hhg_solve(m.h, f, u, tol=1e-8, maxit=300, mode=H.HHG_SOLVE_MIXED, smoother=sm)
    with capsys.disabled():
        print(f"\n[learned] train {st}\n[learned] plain {res['plain']}\n[learned] learned {res['learned']}")
    assert st["loss_final"] < st["loss_init"]
    assert st["loss_final"] < st["loss_jacobi"]
    assert res["plain"]["rel_residual"] <= 1e-8 and res["learned"]["rel_residual"] <= 1e-8
    assert st["accepted"] == 1
    assert res["learned"]["smoother_used"] == H.HHG_SMOOTH_LEARNED
    assert res["learned"]["iterations"] < res["plain"]["iterations"]
    m.close()
