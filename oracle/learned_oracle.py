"""FP64 CPU oracle of the learned convolutional smoother.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU
baseline may import this module; the product path never does.

The paper has no learned component.  This module writes out, in the plainest
form, the definition that the library's learned smoother implements, so that
its forward pass, loss and gradients can be checked:

* Taps.  tau = (di, dj, dk) in {-1, 0, 1}^3, numbered
  t = 9 (dk + 1) + 3 (dj + 1) + (di + 1) (TAPS[t]).
* Weights.  One vector of 1296 numbers: W1[t, a, c] (27 x 2 x 16, first 864)
  then W2[t, c] (27 x 16).  No biases, so the network is positively
  homogeneous: N(alpha r) = alpha N(r) for alpha > 0, and it needs no input
  normalisation.
* Inputs at every node of a level: the residual r, the diagonal D of the
  scaled operator and the coefficient k.  Input channels
  a0 = r / D (0 on Dirichlet nodes) and a1 = a0 * log k.
* Per macro tetrahedron, on its index set S = {(i,j,k) >= 0, i+j+k <= N}
  (Sec. 2.1: the structured refinement of one macro tetrahedron), with every
  value outside S taken as zero:
      z_c(p)  = sum_t sum_a W1[t, a, c] a_a(p + tau_t)
      h_c(p)  = max(z_c(p), 0)
      ch(p)   = sum_t sum_c W2[t, c] h_c(p + tau_t)
  Each macro tetrahedron sees only its own index set, so a node on a macro
  face, edge or vertex gets one value ch per containing tetrahedron.
* Correction c(x) = mean over the tetrahedra containing node x of ch, and
  c = 0 on Dirichlet nodes.  A smoothing step is u <- u + c.
* Training loss for a residual/error pair (r, e) with r = A e on the unknowns:
      L = (e - c)^T A (e - c) / (e^T r),
  the squared energy norm of the error left after the step, relative to the
  error before it.

Vectors here are indexed by unique node of a LevelMesh (hhg_oracle), never by
the CUDA path's stored layout.  Nothing here shares code with the CUDA path.
"""
from __future__ import annotations

import numpy as np

TAPS = np.array([(di, dj, dk) for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)], dtype=np.int64)
N_TAPS = 27
N_IN = 2
N_HID = 16
N_W1 = N_TAPS * N_IN * N_HID
N_W2 = N_TAPS * N_HID
N_W = N_W1 + N_W2
CENTRE = 13


def unpack(w):
    """(W1 [27,2,16], W2 [27,16]) views of a weight vector."""
    w = np.asarray(w, dtype=np.float64)
    assert w.shape == (N_W,)
    return w[:N_W1].reshape(N_TAPS, N_IN, N_HID), w[N_W1:].reshape(N_TAPS, N_HID)


def jacobi_weights(omega, noise=None):
    """Weights for which the network equals one damped Jacobi step.

    h_0 = max(a0, 0) and h_1 = max(-a0, 0) through the centre tap, and
    ch = omega (h_0 - h_1) = omega a0 = omega r / D.  `noise` (1296 values or
    None) is added to every other entry."""
    w = np.zeros(N_W) if noise is None else np.array(noise, dtype=np.float64)
    W1, W2 = w[:N_W1].reshape(N_TAPS, N_IN, N_HID), w[N_W1:].reshape(N_TAPS, N_HID)
    W1[CENTRE, 0, 0], W1[CENTRE, 0, 1] = 1.0, -1.0
    W2[CENTRE, 0], W2[CENTRE, 1] = omega, -omega
    return w


def _shift(box, tau):
    """out[p] = box[p + tau] over the leading three axes, zero where p + tau
    leaves the box."""
    out = np.zeros_like(box)
    n = box.shape[0]
    src, dst = [], []
    for d in tau:
        d = int(d)
        if d >= 0:
            src.append(slice(d, n))
            dst.append(slice(0, n - d))
        else:
            src.append(slice(0, n + d))
            dst.append(slice(-d, n))
    out[tuple(dst)] = box[tuple(src)]
    return out


def features(lm, r_full, diag_full, k_full):
    """Input channels (a0, a1) on the unique nodes of a level."""
    a0 = np.where(lm.dirichlet, 0.0, np.asarray(r_full, dtype=np.float64) / np.asarray(diag_full, dtype=np.float64))
    return a0, a0 * np.log(np.asarray(k_full, dtype=np.float64))


def forward(lm, w, a0, a1):
    """Correction c on unique nodes, and the per-tetrahedron intermediates
    needed by backward()."""
    W1, W2 = unpack(w)
    csum = np.zeros(lm.n)
    cnt = np.zeros(lm.n)
    cache = []
    for t in range(len(lm.macro.T)):
        L = lm.local[t]
        mask = L >= 0
        ids = L[mask]
        A = np.zeros(L.shape + (N_IN,))
        A[mask, 0] = a0[ids]
        A[mask, 1] = a1[ids]
        z = np.zeros(L.shape + (N_HID,))
        for ti in range(N_TAPS):
            z += _shift(A, TAPS[ti]) @ W1[ti]
        z[~mask] = 0.0
        h = np.maximum(z, 0.0)
        ch = np.zeros(L.shape)
        for ti in range(N_TAPS):
            ch += _shift(h, TAPS[ti]) @ W2[ti]
        ch[~mask] = 0.0
        csum += np.bincount(ids, weights=ch[mask], minlength=lm.n)
        cnt += np.bincount(ids, minlength=lm.n)
        cache.append((mask, ids, A, z, h))
    c = csum / cnt
    c[lm.dirichlet] = 0.0
    return c, (cache, cnt)


def backward(lm, w, saved, g_c):
    """Gradient of a scalar with respect to the weights, given its gradient
    g_c with respect to the correction c (unique nodes)."""
    W1, W2 = unpack(w)
    cache, cnt = saved
    g_c = np.where(lm.dirichlet, 0.0, np.asarray(g_c, dtype=np.float64))
    gW1 = np.zeros_like(W1)
    gW2 = np.zeros_like(W2)
    for (mask, ids, A, z, h) in cache:
        # c(x) is the mean of the copies' ch: each copy receives g_c / copies
        gch = np.zeros(mask.shape)
        gch[mask] = g_c[ids] / cnt[ids]
        gh = np.zeros(h.shape)
        for ti in range(N_TAPS):
            # ch(p) = sum W2[t, c] h_c(p + tau_t)
            gW2[ti] += np.einsum("ijk,ijkc->c", gch, _shift(h, TAPS[ti]))
            gh += _shift(gch, -TAPS[ti])[..., None] * W2[ti][None, None, None, :]
        gh[~mask] = 0.0
        gz = gh * (z > 0.0)
        for ti in range(N_TAPS):
            # z_c(p) = sum W1[t, a, c] a_a(p + tau_t)
            gW1[ti] += np.einsum("ijka,ijkc->ac", _shift(A, TAPS[ti]), gz)
    return np.concatenate([gW1.reshape(-1), gW2.reshape(-1)])


def loss_and_grad(lm, A_sys, w, r_full, e_full, diag_full, k_full):
    """L = (e - c)^T A (e - c) / (e^T r) over the unknowns and dL/dw.

    A_sys is the scaled operator on the unknowns (LevelMesh.system), r_full
    and e_full are on all unique nodes (Dirichlet entries ignored)."""
    a0, a1 = features(lm, r_full, diag_full, k_full)
    c, saved = forward(lm, w, a0, a1)
    I = lm.unknowns
    d = np.asarray(e_full, dtype=np.float64)[I] - c[I]
    q = A_sys @ d
    den = float(np.dot(np.asarray(e_full, dtype=np.float64)[I], np.asarray(r_full, dtype=np.float64)[I]))
    loss = float(np.dot(d, q)) / den
    g_c = np.zeros(lm.n)
    g_c[I] = -2.0 * q / den
    return loss, backward(lm, w, saved, g_c), c
