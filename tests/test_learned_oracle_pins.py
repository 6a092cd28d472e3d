"""Pins of the learned-smoother oracle (oracle/learned_oracle.py) against
things it must agree with but does not share code with: scipy's 3-D
correlation, central finite differences of its own loss, the damped Jacobi
step of the multigrid oracle, and positive homogeneity."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import hhg_oracle as O
from oracle import learned_oracle as LO
from paper_1709_06793_gb300 import inputs as I


def _setup(mesh, level, seed):
    V, T = mesh()
    H = O.Hierarchy(V, T, level, level, k_func=I.k_cube)
    lm = H.mesh[level]
    rng = np.random.default_rng(seed)
    A_sys = H.A[level]
    diag = np.ones(lm.n)
    diag[lm.unknowns] = H.D[level]
    e = np.zeros(lm.n)
    e[lm.unknowns] = rng.uniform(-1, 1, len(lm.unknowns))
    r = np.zeros(lm.n)
    r[lm.unknowns] = A_sys @ e[lm.unknowns]
    return H, lm, A_sys, diag, H.k[level], r, e, rng


def _forward_by_correlate(lm, w, a0, a1):
    """The same network with scipy.ndimage.correlate (zero padding) on each
    macro tetrahedron's (N+1)^3 box."""
    W1, W2 = LO.unpack(w)
    csum = np.zeros(lm.n)
    cnt = np.zeros(lm.n)
    for t in range(len(lm.macro.T)):
        L = lm.local[t]
        mask = L >= 0
        ids = L[mask]
        boxes = []
        for a in (a0, a1):
            b = np.zeros(L.shape)
            b[mask] = a[ids]
            boxes.append(b)
        h = []
        for c in range(LO.N_HID):
            z = np.zeros(L.shape)
            for a in range(LO.N_IN):
                # tap number 9 (dk+1) + 3 (dj+1) + (di+1) -> kernel[di+1, dj+1, dk+1]
                ker = W1[:, a, c].reshape(3, 3, 3).transpose(2, 1, 0)
                z += ndimage.correlate(boxes[a], ker, mode="constant", cval=0.0)
            h.append(np.where(mask, np.maximum(z, 0.0), 0.0))
        ch = np.zeros(L.shape)
        for c in range(LO.N_HID):
            ch += ndimage.correlate(h[c], W2[:, c].reshape(3, 3, 3).transpose(2, 1, 0), mode="constant", cval=0.0)
        csum += np.bincount(ids, weights=ch[mask], minlength=lm.n)
        cnt += np.bincount(ids, minlength=lm.n)
    c = csum / cnt
    c[lm.dirichlet] = 0.0
    return c


@pytest.mark.parametrize("mesh,level", [(I.kuhn_cube, 2), (I.unit_tet, 3), (I.cube12, 1)])
def test_forward_matches_scipy_correlate(mesh, level):
    H, lm, A_sys, diag, k, r, e, rng = _setup(mesh, level, 3)
    w = rng.normal(0, 0.3, LO.N_W)
    a0, a1 = LO.features(lm, r, diag, k)
    c, _ = LO.forward(lm, w, a0, a1)
    c_ref = _forward_by_correlate(lm, w, a0, a1)
    assert np.max(np.abs(c)) > 1e-3
    np.testing.assert_allclose(c, c_ref, rtol=0, atol=1e-12 * np.max(np.abs(c_ref)))


@pytest.mark.parametrize("mesh,level", [(I.kuhn_cube, 2), (I.unit_tet, 3)])
def test_gradient_matches_central_differences(mesh, level):
    H, lm, A_sys, diag, k, r, e, rng = _setup(mesh, level, 4)
    w = rng.normal(0, 0.3, LO.N_W)
    loss, g, _ = LO.loss_and_grad(lm, A_sys, w, r, e, diag, k)
    idx = np.concatenate([rng.choice(LO.N_W1, 16, replace=False), LO.N_W1 + rng.choice(LO.N_W2, 12, replace=False),
                          [LO.CENTRE * 32, LO.N_W1 + LO.CENTRE * 16]])
    gmax = np.max(np.abs(g))
    assert gmax > 1e-3
    for i in idx:
        hstep = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[i] += hstep
        wm[i] -= hstep
        lp = LO.loss_and_grad(lm, A_sys, wp, r, e, diag, k)[0]
        lm_ = LO.loss_and_grad(lm, A_sys, wm, r, e, diag, k)[0]
        fd = (lp - lm_) / (2 * hstep)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, gmax), (i, fd, g[i])


@pytest.mark.parametrize("mesh,level", [(I.kuhn_cube, 3), (I.regular_tet, 3)])
def test_jacobi_weights_are_one_damped_jacobi_step(mesh, level):
    H, lm, A_sys, diag, k, r, e, rng = _setup(mesh, level, 5)
    omega = 2.0 / 3.0
    w = LO.jacobi_weights(omega)
    a0, a1 = LO.features(lm, r, diag, k)
    c, _ = LO.forward(lm, w, a0, a1)
    u1 = H.jacobi(level, r[lm.unknowns], np.zeros(len(lm.unknowns)), 1)
    np.testing.assert_allclose(c[lm.unknowns], u1, rtol=1e-14, atol=1e-15)
    assert np.all(c[lm.dirichlet] == 0)
    # the loss of that network is the energy error left by the Jacobi step
    loss = LO.loss_and_grad(lm, A_sys, w, r, e, diag, k)[0]
    eu = e[lm.unknowns]
    d = eu - u1
    assert abs(loss - (d @ (A_sys @ d)) / (eu @ (A_sys @ eu))) <= 1e-13
    # damped Jacobi reduces the energy error of a random vector
    assert 0.0 < loss < 1.0


def test_network_is_positively_homogeneous():
    H, lm, A_sys, diag, k, r, e, rng = _setup(I.kuhn_cube, 2, 6)
    w = rng.normal(0, 0.3, LO.N_W)
    c1, _ = LO.forward(lm, w, *LO.features(lm, r, diag, k))
    c2, _ = LO.forward(lm, w, *LO.features(lm, 2.5 * r, diag, k))
    np.testing.assert_allclose(c2, 2.5 * c1, rtol=1e-13, atol=1e-14)
    cm, _ = LO.forward(lm, w, *LO.features(lm, -r, diag, k))
    assert np.max(np.abs(cm + c1)) > 1e-6  # not odd: the ReLU makes it nonlinear


def test_interface_value_is_mean_of_copies():
    """A node on a macro face gets the mean of the values its tetrahedra
    compute; checked with a network whose output depends on the local index
    set (an off-centre tap sees zero padding in one tetrahedron only)."""
    H, lm, A_sys, diag, k, r, e, rng = _setup(I.kuhn_cube, 2, 7)
    w = LO.jacobi_weights(1.0)
    W1, W2 = LO.unpack(w)
    W2[LO.CENTRE] = 0.0
    W2[LO.CENTRE + 1, 0], W2[LO.CENTRE + 1, 1] = 1.0, -1.0  # ch(p) = a0(p + e1)
    a0, a1 = LO.features(lm, r, diag, k)
    c, _ = LO.forward(lm, w, a0, a1)
    for x in lm.unknowns[:200]:
        vals = []
        for t in range(len(lm.macro.T)):
            p = np.argwhere(lm.local[t] == x)
            if len(p):
                i, j, kk = p[0]
                N = lm.N
                vals.append(a0[lm.local[t][i + 1, j, kk]] if i + 1 + j + kk <= N else 0.0)
        assert abs(c[x] - np.mean(vals)) <= 1e-14 * max(1.0, abs(c[x]))
