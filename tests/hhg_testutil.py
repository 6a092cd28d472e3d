"""Test helpers: enumerate the library's stored layout (documented in
include/hhg.h) and map stored nodes to the oracle's unique nodes.  Only
bookkeeping lives here; no operator arithmetic."""
import numpy as np

from oracle import hhg_oracle as O
from paper_1709_06793_gb300 import inputs as I


def stored_nodes(offsets, tet_levels):
    """(tet, i, j, k) of every stored node at one depth, in stored order."""
    nt = len(tet_levels)
    order = sorted([t for t in range(nt) if tet_levels[t] >= 0], key=lambda t: offsets[t])
    out = []
    for t in order:
        N = 1 << int(tet_levels[t])
        ii, jj, kk = [], [], []
        for k in range(N + 1):
            for j in range(N - k + 1):
                n = N - j - k + 1
                ii.append(np.arange(n))
                jj.append(np.full(n, j))
                kk.append(np.full(n, k))
        i = np.concatenate(ii)
        assert offsets[t] + len(i) <= offsets[-1] or len(i) == 0
        out.append(np.stack([np.full(len(i), t), i, np.concatenate(jj), np.concatenate(kk)], axis=1))
    return np.concatenate(out) if out else np.zeros((0, 4), dtype=np.int64)


def stored_keys(T, nodes, tet_levels):
    """Key hashes (inputs.node_keys) of stored nodes."""
    t, i, j, k = nodes.T
    N = np.array([1 << int(tet_levels[x]) for x in t])
    W = np.stack([N - i - j - k, i, j, k], axis=1)
    keys = np.empty(len(t), dtype=np.uint64)
    for n in np.unique(N):
        sel = N == n
        keys[sel] = I.node_keys(np.asarray(T)[t[sel]], W[sel], int(n))
    return keys


def oracle_map(lm, nodes):
    """Oracle unique-node index of each stored node (single-level meshes)."""
    t, i, j, k = nodes.T
    out = np.empty(len(t), dtype=np.int64)
    for tt in np.unique(t):
        sel = t == tt
        out[sel] = lm.local[tt][i[sel], j[sel], k[sel]]
    assert np.all(out >= 0)
    return out


def oracle_keys(lm):
    return I.node_keys(lm.node_gverts, lm.node_weights, lm.N)


def node_index(offsets, t, i, j, k, N):
    """Stored index of node (i, j, k) of tet t (all at refinement N): the
    tet's offset plus planes 0..k-1, rows 0..j-1 of plane k, then i."""
    t, i, j, k = (np.asarray(a, dtype=np.int64) for a in (t, i, j, k))

    def tetnum(x):
        return x * (x + 1) * (x + 2) // 6

    M = N - k
    return (np.asarray(offsets, dtype=np.int64)[t] + tetnum(N + 1) - tetnum(N + 1 - k)
            + j * (M + 1) - j * (j - 1) // 2 + i)


def lattice_field(X, scale):
    """Rough reproducible input field in [-1, 1) from node coordinates that lie
    on the lattice (1/scale) Z^3: an integer hash of the lattice point, so
    every stored copy of a node gets the same value."""
    q = np.rint(np.asarray(X, dtype=np.float64) * float(scale)).astype(np.int64)
    h = (q[:, 0] * np.int64(73856093)) ^ (q[:, 1] * np.int64(19349663)) ^ (q[:, 2] * np.int64(83492791))
    h = h * np.int64(-7046029254386353131)
    h = h ^ ((h >> 29) & np.int64((1 << 35) - 1))
    h = h * np.int64(-4658895280553007687)
    v = ((h >> 20) & np.int64((1 << 40) - 1)).astype(np.float64) / float(1 << 40)
    return 2.0 * v - 1.0


def sampled_residuals(O, H, m, V, T, level, x_dev, f_dev, kfun, n_vol, n_face, seed):
    """FP64 residuals f_i - (A x)_i at sampled stored rows of a single-level
    mesh, each row evaluated by the oracle's one-row evaluator (row_apply)
    from the solution's values at the row's neighbours (gathered from the
    device vector) and the exact coefficient kfun(X).  Returns (sampled stored
    indices, oracle residuals).  Dirichlet rows are not sampled."""
    import torch

    off, lev, n = m.layout(0)
    nodes = stored_nodes(off, lev)
    N = 1 << level
    t_, i_, j_, k_ = nodes.T
    face = (i_ == 0) | (j_ == 0) | (k_ == 0) | (i_ + j_ + k_ == N)
    mm = O.MacroMesh(V, T)
    Tn = np.asarray(T)
    tet_of = {tuple(int(v) for v in Tn[t]): t for t in range(len(Tn))}
    rng = np.random.default_rng(seed)
    cand_v = np.nonzero(~face)[0]
    cand_f = np.nonzero(face)[0]
    pick_f = []
    for q in rng.permutation(cand_f):  # face rows that are not Dirichlet
        t, i, j, kk = nodes[q]
        Wt = np.array([N - i - j - kk, i, j, kk])
        if not mm.on_boundary(Tn[t][Wt > 0]):
            pick_f.append(q)
        if len(pick_f) == n_face:
            break
    sample = np.concatenate([rng.choice(cand_v, n_vol, replace=False), np.array(pick_f, dtype=np.int64)])

    def field_u(gv, W, X):
        t = tet_of[tuple(int(v) for v in gv[0])]
        idx = node_index(off, np.full(len(W), t), W[:, 1], W[:, 2], W[:, 3], N)
        return x_dev[torch.as_tensor(idx, device=x_dev.device)].double().cpu().numpy()

    def field_k(gv, W, X):
        return kfun(X)

    fs = f_dev[torch.as_tensor(sample, device=f_dev.device)].double().cpu().numpy()
    r = np.empty(len(sample))
    for q, (t, i, j, kk) in enumerate(nodes[sample]):
        Wt = np.array([N - i - j - kk, i, j, kk])
        r[q] = fs[q] - O.row_apply(mm, level, Tn[t][Wt > 0], Wt[Wt > 0], field_u, field_k, "scaled")
    return sample, r
