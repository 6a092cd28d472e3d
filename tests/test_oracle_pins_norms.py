"""Pins of the oracle's convergence rate, discrete L2 norm and coefficient
injection against quantities fixed without the oracle's own formulas:

* the rate of Sec. 7, rho = (r^(i*) / r^(5))^(1/(i* - 5)), of a residual
  history that decays geometrically from step 5 on is that decay factor, and
  the steps before 5 do not enter;
* the lumped P1 mass weight of a node is the integral of its hat function,
  1/4 of the volume of every micro tetrahedron at the node (determinants
  computed here), so the weights of all nodes add up to the domain's volume;
* injecting a fine nodal coefficient into a coarse level equals sampling the
  coefficient at the coarse nodes (they are fine nodes).
"""
import math

import numpy as np
import pytest

from oracle import hhg_oracle as O
from paper_1709_06793_gb300 import inputs as I


@pytest.mark.parametrize("q,i_star", [(0.37, 10), (0.081, 10), (0.6, 14)])
def test_mg_rate_of_geometric_history(q, i_star):
    rng = np.random.default_rng(3)
    hist = [float(rng.uniform(1, 50)) for _ in range(5)]  # arbitrary transient
    c = 7.3
    hist += [c * q ** i for i in range(5, i_star + 3)]
    rho = O.mg_rate(hist, i_star=i_star)
    assert abs(rho - q) <= 1e-13 * q
    # a history one step longer or shorter in the window gives another value
    assert abs(O.mg_rate(hist, i_star=i_star, i0=5) - (hist[i_star - 1] / hist[5]) ** (1 / (i_star - 5))) > 1e-3 * q


def _micro_volume_weights(lm):
    """Sum over micro tets of |t| / 4 onto each vertex, |t| from the determinant."""
    w = np.zeros(lm.n)
    for t in range(len(lm.macro.T)):
        ids = lm.micro[t]
        X = lm.coords[ids]
        d = np.abs(np.linalg.det(X[:, 1:] - X[:, :1])) / 6.0
        for a in range(4):
            np.add.at(w, ids[:, a], d / 4.0)
    return w


@pytest.mark.parametrize("mesh,level,volume", [(I.unit_tet, 2, 1.0 / 6.0), (I.kuhn_cube, 2, 1.0), (I.cube12, 1, 1.0)])
def test_discrete_l2_weights_are_node_volumes(mesh, level, volume):
    V, T = mesh()
    lm = O.LevelMesh(O.MacroMesh(V, T), level)
    assert abs(O.discrete_l2(lm, np.ones(lm.n)) ** 2 - volume) <= 1e-14
    w = _micro_volume_weights(lm)
    assert abs(w.sum() - volume) <= 1e-14
    for i in range(lm.n):
        e = np.zeros(lm.n)
        e[i] = 1.0
        assert abs(O.discrete_l2(lm, e) ** 2 - w[i]) <= 1e-15
    # and for a general vector the norm is the weighted sum of squares
    e = np.random.default_rng(1).normal(size=lm.n)
    assert abs(O.discrete_l2(lm, e) - math.sqrt(float(np.sum(w * e * e)))) <= 1e-13


def test_inject_equals_sampling_at_coarse_nodes():
    V, T = I.kuhn_cube()
    kf = I.k_cube
    h_func = O.Hierarchy(V, T, 3, 1, k_func=kf)
    fine = h_func.mesh[3]
    h_inj = O.Hierarchy(V, T, 3, 1, k_fine=kf(fine.coords))
    for l in (1, 2, 3):
        assert np.array_equal(h_inj.k[l], h_func.k[l])
        assert abs(h_inj.A[l] - h_func.A[l]).max() == 0.0
