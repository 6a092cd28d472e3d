"""FP64 CPU oracle for the stencil-scaled P1 operator on hierarchical hybrid grids.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU
baseline may import this module; the product path never does.

It computes, from the paper's definitions and nothing else,

* the uniform refinement of every macro tetrahedron by Bey's rule (Sec. 2.1,
  "uniform mesh refinement ... see [Bey95]"; the interior diagonal joins the
  midpoints of x1x3 and x2x4 in the paper's 1-based numbering, Fig.
  "stencilsign" caption);
* the P1 element stiffness matrix A_t with entries int_t grad(phi_i).grad(phi_j)
  (Sec. 3.2, matrix \\hat A_t);
* the scaled operator of eq. "discrete" in its element-wise algebraic form of
  Lemma "equal" / eq. "equal": K_t o A_t with off-diagonal (k_i+k_j)/2 and the
  diagonal fixed by the zero row sum of eq. "zerosum";
* the nodal-integration operator of eq. "standardfe": mean vertex k times A_t;
* the "scale Vol+Face" operator of eq. "modst" (nodal rows on macro vertices
  and edges, scaled rows elsewhere);
* the pre-asymptotic modification of Sec. 4 (eq. "defKmin"): on the edges of
  "gray type" (positive reference stencil entry) of a macro tetrahedron the
  scaling (k_i+k_j)/2 becomes (k_min(x_i)+k_min(x_j))/2, k_min the minimum
  of k over a node and its edge neighbours inside that macro tetrahedron;
* the consistent P1 mass matrix (right-hand side f_h = M I_h f, Sec. 7.2);
* global assembly over unique nodes (nodes on macro faces/edges/vertices are
  shared by all macro tetrahedra that contain them, Sec. 2.1), homogeneous
  Dirichlet rows removed (Sec. 2);
* geometric multigrid (the paper fixes only the V(3,3) cycle, Sec. 7.2; these
  are readings where it is silent): linear interpolation P (exact for nested
  P1 spaces), R = P^T, coarse operators re-discretised with the same scaled
  rule and k sampled at the coarse nodes, damped Jacobi (omega = 2/3) and
  degree-2 Chebyshev smoothers, dense Cholesky on the coarsest level, a
  symmetric V-cycle and CG preconditioned by one V-cycle from a zero guess.

Nothing here shares code with the CUDA path.  Vectors are indexed by unique
node (see LevelMesh), never by the CUDA path's stored layout.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ----------------------------------------------------------------------------
# Uniform refinement (Bey's rule)
# ----------------------------------------------------------------------------


def bey_children(tets):
    """Children of tetrahedra by Bey's rule.

    tets: (n,4,3) integer coordinates with even entries (so midpoints stay
    integral).  Returns (8n,4,3), the children of tetrahedron m at rows
    8m..8m+7, each with Bey's vertex order: the four corner tetrahedra
    (x0,x01,x02,x03), (x01,x1,x12,x13), (x02,x12,x2,x23), (x03,x13,x23,x3) and
    the octahedron cut along x02-x13 into (x01,x02,x03,x13), (x01,x02,x12,x13),
    (x02,x03,x13,x23), (x02,x12,x13,x23).
    """
    t = np.asarray(tets, dtype=np.int64)
    x0, x1, x2, x3 = t[:, 0], t[:, 1], t[:, 2], t[:, 3]

    def mid(a, b):
        s = a + b
        assert not np.any(s % 2), "midpoint not on the lattice"
        return s // 2

    x01, x02, x03 = mid(x0, x1), mid(x0, x2), mid(x0, x3)
    x12, x13, x23 = mid(x1, x2), mid(x1, x3), mid(x2, x3)
    kids = [
        (x0, x01, x02, x03),
        (x01, x1, x12, x13),
        (x02, x12, x2, x23),
        (x03, x13, x23, x3),
        (x01, x02, x03, x13),
        (x01, x02, x12, x13),
        (x02, x03, x13, x23),
        (x02, x12, x13, x23),
    ]
    out = np.stack([np.stack(k, axis=1) for k in kids], axis=1)  # (n,8,4,3)
    return out.reshape(-1, 4, 3)


def macro_index_tet(level):
    """The macro tetrahedron in index coordinates at refinement level `level`:
    vertex a sits at N e_a (e_0 = 0), N = 2^level, so node (i,j,k) has
    barycentric weights (N-i-j-k, i, j, k)/N."""
    N = 1 << level
    return np.array([[[0, 0, 0], [N, 0, 0], [0, N, 0], [0, 0, N]]], dtype=np.int64)


def micro_tets(level):
    """All 8^level micro tetrahedra of one refined macro tetrahedron, in index
    coordinates, by refining `level` times with Bey's rule."""
    cur = macro_index_tet(level)
    for _ in range(level):
        cur = bey_children(cur)
    return cur


def _det3(a, b, c):
    return (a[..., 0] * (b[..., 1] * c[..., 2] - b[..., 2] * c[..., 1])
            - a[..., 1] * (b[..., 0] * c[..., 2] - b[..., 2] * c[..., 0])
            + a[..., 2] * (b[..., 0] * c[..., 1] - b[..., 1] * c[..., 0]))


def _contains(tets, p):
    """Closed tetrahedra (integer coords) containing integer point p."""
    a, b, c, d = tets[:, 0], tets[:, 1], tets[:, 2], tets[:, 3]
    vol = _det3(b - a, c - a, d - a)
    l1 = _det3(p - a, c - a, d - a)
    l2 = _det3(b - a, p - a, d - a)
    l3 = _det3(b - a, c - a, p - a)
    l0 = vol - l1 - l2 - l3
    s = np.sign(vol)
    return (l0 * s >= 0) & (l1 * s >= 0) & (l2 * s >= 0) & (l3 * s >= 0)


def micro_tets_at(level, p):
    """Micro tetrahedra that have index point p as a vertex: Bey refinement of
    the macro tetrahedron, keeping at each step only the children that contain
    p (a lattice point inside a micro tetrahedron is one of its vertices)."""
    p = np.asarray(p, dtype=np.int64)
    cur = macro_index_tet(level)
    for _ in range(level):
        ch = bey_children(cur)
        cur = ch[_contains(ch, p)]
    keep = np.all(cur == p[None, None, :], axis=2).any(axis=1)
    return cur[keep]


# ----------------------------------------------------------------------------
# P1 element matrices (Sec. 3.2 and eq. "standardfe")
# ----------------------------------------------------------------------------


def p1_gradients(X):
    """Gradients of the 4 barycentric basis functions and the volume.

    X: (n,4,3) vertex coordinates.  Returns G (n,4,3) with G[:,a] = grad phi_a,
    and vol (n,).  phi_a(x) = c_a + g_a.x solves phi_a(x_b) = delta_ab."""
    X = np.asarray(X, dtype=np.float64)
    B = np.concatenate([np.ones(X.shape[:2] + (1,)), X], axis=2)  # rows (1, x_b)
    C = np.linalg.inv(B)  # column a: coefficients of phi_a
    G = np.transpose(C[:, 1:, :], (0, 2, 1))
    vol = np.abs(np.linalg.det(B)) / 6.0
    return G, vol


def p1_stiffness(X):
    """(\\hat A_t)_ab = int_t grad phi_a . grad phi_b = vol * g_a . g_b."""
    G, vol = p1_gradients(X)
    return vol[:, None, None] * np.einsum("nai,nbi->nab", G, G)


def p1_mass(X):
    """Consistent P1 mass matrix: vol/20 * (1 + delta_ab)."""
    _, vol = p1_gradients(X)
    return (vol / 20.0)[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None]


def scaled_element(A, kv):
    """K_t o \\hat A_t of Lemma "equal": off-diagonal (k_a + k_b)/2 * A_ab; the
    diagonal by eq. "zerosum" makes every row sum vanish."""
    A = np.asarray(A, dtype=np.float64)
    kv = np.asarray(kv, dtype=np.float64)
    K = 0.5 * (kv[:, :, None] + kv[:, None, :])
    M = K * A
    idx = np.arange(4)
    M[:, idx, idx] = 0.0
    M[:, idx, idx] = -M.sum(axis=2)
    return M


def nodal_element(A, kv):
    """Nodal-integration element matrix of eq. "standardfe": mean(k_a) * A_t."""
    return np.mean(np.asarray(kv, dtype=np.float64), axis=1)[:, None, None] * np.asarray(A, dtype=np.float64)


def element_matrices(X, kv, kind):
    A = p1_stiffness(X)
    if kind == "scaled":
        return scaled_element(A, kv)
    if kind == "nodal":
        return nodal_element(A, kv)
    if kind == "laplace":
        return A
    raise ValueError(kind)


# ----------------------------------------------------------------------------
# Pre-asymptotic modification (Sec. 4, eq. "defKmin")
# ----------------------------------------------------------------------------

# the 14 stencil directions (di, dj, dk): e1, e2, e3, e1-e2, e1-e3, e2-e3,
# e1-e2+e3 and their negatives (the edge directions of the refined mesh)
STENCIL_DIRS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, -1, 0), (1, 0, -1), (0, 1, -1), (1, -1, 1)]
STENCIL_DIRS = STENCIL_DIRS + [(-a, -b, -c) for (a, b, c) in STENCIL_DIRS]


def reference_volume_stencil(V, tet):
    """Laplacian stencil (14 off-centre entries, STENCIL_DIRS order) of a node
    inside the macro tetrahedron with vertices V[tet] in refinement order:
    the row of node (1,1,1) of the level-2 refinement of that tetrahedron
    alone (the volume stencil does not depend on the level or the node)."""
    lm = LevelMesh(MacroMesh(np.asarray(V, dtype=np.float64)[list(tet)], np.array([[0, 1, 2, 3]])), 2)
    A = lm.assemble(None, "laplace").tocsr()
    x = lm.local[0][1, 1, 1]
    return np.array([A[x, lm.local[0][1 + a, 1 + b, 1 + c]] for (a, b, c) in STENCIL_DIRS])


def gray_directions(V, tet, tol=1e-14):
    """Directions of gray type (Sec. 4.2: edges with a positive reference
    stencil entry), as a boolean mask over STENCIL_DIRS."""
    return reference_volume_stencil(V, tet) > tol


def tet_kmin(lm, k, t):
    """k_min(x) of eq. "defKmin" for the nodes of macro tetrahedron t: the
    minimum of k over x and every node joined to x by an edge that belongs to
    the macro tetrahedron (the edges of its micro tetrahedra).  Full-size
    array; entries of nodes outside t are k itself."""
    k = np.asarray(k, dtype=np.float64)
    km = k.copy()
    ids = lm.micro[t]
    np.minimum.at(km, ids.reshape(-1), np.repeat(k[ids].min(axis=1), 4))
    return km


def kmin_element(A, kv, kmv, gray_pair):
    """Scaled element matrix with the modification: entry (a, b) scaled by
    (k_a + k_b)/2, or by (kmin_a + kmin_b)/2 where gray_pair[:, a, b]; the
    diagonal by the zero row sum."""
    A = np.asarray(A, dtype=np.float64)
    K = 0.5 * (kv[:, :, None] + kv[:, None, :])
    Km = 0.5 * (kmv[:, :, None] + kmv[:, None, :])
    M = np.where(gray_pair, Km, K) * A
    idx = np.arange(4)
    M[:, idx, idx] = 0.0
    M[:, idx, idx] = -M.sum(axis=2)
    return M


# ----------------------------------------------------------------------------
# Macro mesh topology
# ----------------------------------------------------------------------------


class MacroMesh:
    """Macro tetrahedra T (nt,4) over vertices V (nv,3); the vertex order of
    each tetrahedron is its refinement order.  Faces that belong to exactly one
    macro tetrahedron form the domain boundary (homogeneous Dirichlet)."""

    def __init__(self, V, T):
        self.V = np.asarray(V, dtype=np.float64)
        self.T = np.asarray(T, dtype=np.int64)
        count = {}
        for t in self.T:
            for opp in range(4):
                f = tuple(sorted(int(t[a]) for a in range(4) if a != opp))
                count[f] = count.get(f, 0) + 1
        self.boundary_faces = {f for f, c in count.items() if c == 1}

    def tets_containing(self, support):
        s = set(int(g) for g in support)
        return [t for t in range(len(self.T)) if s <= set(int(g) for g in self.T[t])]

    def on_boundary(self, support):
        """A point whose barycentric support is `support` lies on the domain
        boundary iff some boundary face contains all its support vertices."""
        s = set(int(g) for g in support)
        return any(s <= set(f) for f in self.boundary_faces)


def _identity_rows(gv, w):
    """Rows (n,8) = sorted (vertex id, weight) pairs with zero weights dropped
    (padded with (-1,0)): the exact identity of a node in the macro mesh."""
    g = np.asarray(gv, dtype=np.int64).copy()
    w = np.asarray(w, dtype=np.int64).copy()
    g[w == 0] = np.iinfo(np.int64).max
    order = np.argsort(g, axis=1, kind="stable")
    g = np.take_along_axis(g, order, axis=1)
    w = np.take_along_axis(w, order, axis=1)
    g[w == 0] = -1
    out = np.empty((g.shape[0], 8), dtype=np.int64)
    out[:, 0::2] = g
    out[:, 1::2] = w
    return out


class LevelMesh:
    """All nodes and micro tetrahedra of a macro mesh refined `level` times.

    Unique nodes are identified exactly by their barycentric support in the
    macro mesh (vertex ids with non-zero integer weights out of N).
    Attributes:
      N, n (number of unique nodes), ident (n,8), coords (n,3),
      dirichlet (n,) bool, node_tet/node_weights (one containing macro tet and
      its weights, for key generation), local[t] (N+1)^3 -> unique id or -1,
      micro[t] (8^level,4) unique ids of each micro tetrahedron's vertices.
    """

    def __init__(self, macro: MacroMesh, level: int, build_micro: bool = True):
        self.macro = macro
        self.level = level
        N = self.N = 1 << level
        ii, jj, kk = np.meshgrid(np.arange(N + 1), np.arange(N + 1), np.arange(N + 1), indexing="ij")
        m = (ii + jj + kk) <= N
        ijk = np.stack([ii[m], jj[m], kk[m]], axis=1)
        W = np.stack([N - ijk.sum(axis=1), ijk[:, 0], ijk[:, 1], ijk[:, 2]], axis=1)
        rows = []
        for t in range(len(macro.T)):
            rows.append(_identity_rows(np.broadcast_to(macro.T[t], W.shape), W))
        allrows = np.concatenate(rows)
        uniq, inv = np.unique(allrows, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        self.ident = uniq
        self.n = len(uniq)
        npt = len(ijk)
        self.local = []
        for t in range(len(macro.T)):
            L = -np.ones((N + 1, N + 1, N + 1), dtype=np.int64)
            L[ijk[:, 0], ijk[:, 1], ijk[:, 2]] = inv[t * npt:(t + 1) * npt]
            self.local.append(L)
        # coordinates: weighted vertex sum in increasing vertex-id order
        g = uniq[:, 0::2]
        w = uniq[:, 1::2].astype(np.float64)
        x = np.zeros((self.n, 3))
        for a in range(4):
            ga = np.where(g[:, a] >= 0, g[:, a], 0)
            x += (w[:, a] / N)[:, None] * macro.V[ga]
        self.coords = x
        # one containing tet per node (for generator keys)
        self.node_tet = np.empty(self.n, dtype=np.int64)
        self.node_weights = np.empty((self.n, 4), dtype=np.int64)
        for t in range(len(macro.T) - 1, -1, -1):
            sel = inv[t * npt:(t + 1) * npt]
            self.node_tet[sel] = t
            self.node_weights[sel] = W
        self.node_gverts = macro.T[self.node_tet]
        # Dirichlet: node lies on a boundary face (w = 0 for the opposite vertex)
        dirichlet = np.zeros(self.n, dtype=bool)
        for t in range(len(macro.T)):
            for opp in range(4):
                f = tuple(sorted(int(macro.T[t][a]) for a in range(4) if a != opp))
                if f in macro.boundary_faces:
                    on = W[:, opp] == 0
                    dirichlet[inv[t * npt:(t + 1) * npt][on]] = True
        self.dirichlet = dirichlet
        self.unknowns = np.nonzero(~dirichlet)[0]
        self.micro = None
        if build_micro:
            mt = micro_tets(level)
            self.micro_index = mt
            self.micro = [self.local[t][mt[:, :, 0], mt[:, :, 1], mt[:, :, 2]] for t in range(len(macro.T))]

    # -- element loops -------------------------------------------------------

    def _elements(self, t, k, kind):
        ids = self.micro[t]
        X = self.coords[ids]
        kv = None if k is None else np.asarray(k, dtype=np.float64)[ids]
        if kind == "kmin":
            return ids, kmin_element(p1_stiffness(X), kv, tet_kmin(self, k, t)[ids], self._gray_pairs(t))
        return ids, element_matrices(X, kv, kind)

    def _gray_pairs(self, t):
        """(ne, 4, 4) mask: the micro edge (a, b) of each micro tetrahedron of
        macro tetrahedron t runs along a gray direction of t."""
        gray = gray_directions(self.macro.V, self.macro.T[t])
        mt = self.micro_index  # (ne, 4, 3) index coordinates of the vertices
        out = np.zeros((len(mt), 4, 4), dtype=bool)
        lut = {d: g for d, g in zip(STENCIL_DIRS, gray)}
        for a in range(4):
            for b in range(4):
                if a != b:
                    dv = mt[:, b, :] - mt[:, a, :]
                    out[:, a, b] = [lut[tuple(v)] for v in dv]
        return out

    def assemble(self, k, kind="scaled"):
        """Full n x n matrix (Dirichlet rows and columns kept)."""
        R, C, D = [], [], []
        for t in range(len(self.macro.T)):
            ids, M = self._elements(t, k, kind)
            R.append(np.repeat(ids, 4, axis=1).reshape(-1))
            C.append(np.tile(ids, (1, 4)).reshape(-1))
            D.append(M.reshape(-1))
        return sp.csr_matrix((np.concatenate(D), (np.concatenate(R), np.concatenate(C))), shape=(self.n, self.n))

    def assemble_mass(self):
        R, C, D = [], [], []
        for t in range(len(self.macro.T)):
            ids = self.micro[t]
            M = p1_mass(self.coords[ids])
            R.append(np.repeat(ids, 4, axis=1).reshape(-1))
            C.append(np.tile(ids, (1, 4)).reshape(-1))
            D.append(M.reshape(-1))
        return sp.csr_matrix((np.concatenate(D), (np.concatenate(R), np.concatenate(C))), shape=(self.n, self.n))

    def apply(self, u, k, kind="scaled"):
        """Matrix-free element loop y = sum_t P_t^T M_t P_t u on the unknowns:
        Dirichlet entries of u are taken as 0 and those of y are set to 0."""
        u = np.where(self.dirichlet, 0.0, np.asarray(u, dtype=np.float64))
        y = np.zeros(self.n)
        for t in range(len(self.macro.T)):
            ids, M = self._elements(t, k, kind)
            contrib = np.einsum("nab,nb->na", M, u[ids])
            y += np.bincount(ids.reshape(-1), weights=contrib.reshape(-1), minlength=self.n)
        y[self.dirichlet] = 0.0
        return y

    def system(self, k, kind="scaled"):
        """A_II: the operator restricted to unknown (non-Dirichlet) nodes
        (kind "scaled", "nodal" or "volface")."""
        A = volface_matrix(self, k) if kind == "volface" else self.assemble(k, kind)
        I = self.unknowns
        return A[I][:, I].tocsr()


# ----------------------------------------------------------------------------
# "Scale Vol+Face" (Sec. 5, eq. "modst" with I = W_V u W_E): rows of nodes on
# macro vertices and edges come from the nodal-integration form of
# eq. "standardfe", all other rows (macro faces, volumes) from stencil scaling.
# ----------------------------------------------------------------------------


def primitive_dim(lm):
    """Dimension of the macro primitive holding each unique node: 0 vertex,
    1 edge, 2 face, 3 volume (number of non-zero barycentric weights - 1)."""
    return np.count_nonzero(lm.ident[:, 1::2], axis=1) - 1


def volface_rows(lm):
    """Rows taken from the nodal-integration form: nodes on macro vertices and
    edges (the index set I = W_V u W_E of eq. "modst")."""
    return primitive_dim(lm) <= 1


def volface_matrix(lm, k):
    """Full n x n matrix of a_{h;I} (Dirichlet rows and columns kept)."""
    sel = volface_rows(lm).astype(np.float64)
    An = lm.assemble(k, "nodal")
    As = lm.assemble(k, "scaled")
    return (sp.diags(sel) @ An + sp.diags(1.0 - sel) @ As).tocsr()


def volface_apply(lm, u, k):
    """y = a_{h;I}(u, .) on the unknowns (Dirichlet entries of u taken as 0,
    those of y set to 0), from the two element loops."""
    return np.where(volface_rows(lm), lm.apply(u, k, "nodal"), lm.apply(u, k, "scaled"))


# ----------------------------------------------------------------------------
# Tensor coefficient, M = 6 (eq. "integral" / eq. "meshdep" with M > 1;
# Sec. 7.3): a(v, w) = sum_m int k_m (d_m . grad v)(d_m . grad w) with the
# directions d = e1, e2, e3, e1-e2, e1-e3, e2-e3 and, for a symmetric K,
# k_i = K_ii + sum_{j != i} K_ij and k_ij = -K_ij (non-negative when the
# off-diagonal entries of K are <= 0, as in Sec. 7.3), so that
# sum_m k_m d_m d_m^T = K.  Each a_m is scaled or nodally integrated like the
# scalar form.
# ----------------------------------------------------------------------------

TENSOR_DIRS = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, -1, 0], [1, 0, -1], [0, 1, -1]], dtype=np.float64)


def tensor_split(K6):
    """K6 (n,6) = (K11, K22, K33, K12, K13, K23) -> the six k_m (n,6)."""
    K6 = np.asarray(K6, dtype=np.float64)
    K11, K22, K33, K12, K13, K23 = K6.T
    return np.stack([K11 + K12 + K13, K22 + K12 + K23, K33 + K13 + K23, -K12, -K13, -K23], axis=1)


def tensor_from_split(km):
    """Inverse map: sum_m k_m d_m d_m^T as (n,3,3)."""
    return np.einsum("nm,mi,mj->nij", np.asarray(km, dtype=np.float64), TENSOR_DIRS, TENSOR_DIRS)


def p1_directional_stiffness(X, d):
    """int_t (d . grad phi_a)(d . grad phi_b) = vol * (g_a . d)(g_b . d)."""
    G, vol = p1_gradients(X)
    gd = G @ np.asarray(d, dtype=np.float64)
    return vol[:, None, None] * gd[:, :, None] * gd[:, None, :]


def tensor_matrix(lm, km, kind="scaled"):
    """Full n x n matrix of sum_m a_m^h (kind "scaled", eq. "discrete" per m)
    or of the nodal-integration form (kind "nodal", mean k_m per micro tet);
    km: (n,6) nodal values of the k_m."""
    km = np.asarray(km, dtype=np.float64)
    R, C, D = [], [], []
    for t in range(len(lm.macro.T)):
        ids = lm.micro[t]
        X = lm.coords[ids]
        M = np.zeros((len(ids), 4, 4))
        for m in range(6):
            A = p1_directional_stiffness(X, TENSOR_DIRS[m])
            kv = km[ids, m]
            M += scaled_element(A, kv) if kind == "scaled" else nodal_element(A, kv)
        R.append(np.repeat(ids, 4, axis=1).reshape(-1))
        C.append(np.tile(ids, (1, 4)).reshape(-1))
        D.append(M.reshape(-1))
    return sp.csr_matrix((np.concatenate(D), (np.concatenate(R), np.concatenate(C))), shape=(lm.n, lm.n))


def tensor_apply(lm, u, km, kind="scaled"):
    """y = A u on the unknowns (Dirichlet entries of u taken as 0, those of y 0)."""
    u = np.where(lm.dirichlet, 0.0, np.asarray(u, dtype=np.float64))
    y = tensor_matrix(lm, km, kind) @ u
    y[lm.dirichlet] = 0.0
    return y


# ----------------------------------------------------------------------------
# One row at a time (for sampled checks at sizes too large to enumerate)
# ----------------------------------------------------------------------------


def row_apply(macro: MacroMesh, level, support, weights, field_u, field_k, kind="scaled"):
    """(A u)_x for the single node x with barycentric support `support` (vertex
    ids) and integer weights `weights` (sum N): the sum, over every macro
    tetrahedron containing x and every micro tetrahedron at x, of the element
    matrix row of x applied to u.  field_u / field_k(gverts (m,4), W (m,4),
    X (m,3)) give nodal values; u is taken as 0 on Dirichlet nodes.  Returns 0
    for a Dirichlet node."""
    N = 1 << level
    if macro.on_boundary(support):
        return 0.0
    total = 0.0
    wmap = dict(zip([int(s) for s in support], [int(w) for w in weights]))
    for t in macro.tets_containing(support):
        gv = macro.T[t]
        wl = np.array([wmap.get(int(g), 0) for g in gv], dtype=np.int64)
        p = wl[1:]
        mts = micro_tets_at(level, p)  # (m,4,3)
        m = len(mts)
        Wm = np.concatenate([(N - mts.sum(axis=2))[..., None], mts], axis=2).reshape(-1, 4)
        gvm = np.broadcast_to(gv, (m * 4, 4))
        X = (Wm.astype(np.float64) / N) @ macro.V[gv]
        X = X.reshape(m, 4, 3)
        ident = _identity_rows(gvm, Wm)
        bd = np.array([macro.on_boundary(ident[q, 0::2][ident[q, 1::2] > 0]) for q in range(4 * m)])
        uv = np.where(bd, 0.0, field_u(gvm, Wm, X.reshape(-1, 3))).reshape(m, 4)
        kv = field_k(gvm, Wm, X.reshape(-1, 3)).reshape(m, 4)
        M = element_matrices(X, kv, kind)
        a_x = np.argmax(np.all(mts == p[None, None, :], axis=2), axis=1)
        total += float(np.einsum("nb,nb->", M[np.arange(m), a_x], uv))
    return total


# ----------------------------------------------------------------------------
# Geometric multigrid (readings: P linear interpolation, R = P^T, coarse
# operators re-discretised with k sampled at the coarse nodes, damped Jacobi
# or Chebyshev smoothing, Cholesky on the coarsest level)
# ----------------------------------------------------------------------------


def prolongation(coarse: LevelMesh, fine: LevelMesh):
    """Linear interpolation from coarse to fine unique nodes (full matrices,
    Dirichlet included).  A fine node at a coarse node takes its value; a fine
    node at the midpoint of a coarse micro-tetrahedron edge takes the mean of
    the edge's two end values (nested P1 spaces)."""
    rows, cols, vals = [], [], []
    for t in range(len(coarse.macro.T)):
        Lf, Lc = fine.local[t], coarse.local[t]
        mt = coarse.micro_index  # coarse index coords (m,4,3)
        # coincident nodes
        ids_c = coarse.micro[t]
        rows.append(Lf[2 * mt[:, :, 0], 2 * mt[:, :, 1], 2 * mt[:, :, 2]].reshape(-1))
        cols.append(ids_c.reshape(-1))
        vals.append(np.ones(ids_c.size))
        for a, b in itertools.combinations(range(4), 2):
            mid = mt[:, a] + mt[:, b]  # fine index of the edge midpoint
            f = Lf[mid[:, 0], mid[:, 1], mid[:, 2]]
            for e in (a, b):
                rows.append(f)
                cols.append(ids_c[:, e])
                vals.append(np.full(len(f), 0.5))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    key = r * coarse.n + c
    _, first = np.unique(key, return_index=True)
    return sp.csr_matrix((v[first], (r[first], c[first])), shape=(fine.n, coarse.n))


def power_start(lm: LevelMesh):
    """Deterministic start vector for the largest-eigenvalue estimate:
    cos(pi N (x+y+z)) + 1/4 at the unknowns."""
    x = lm.coords
    return np.cos(np.pi * lm.N * (x[:, 0] + x[:, 1] + x[:, 2]))[lm.unknowns] + 0.25


class Hierarchy:
    """Multigrid hierarchy on levels coarsest..finest of one macro mesh.

    k_func(x) gives the coefficient at node coordinates (sampling it at the
    coarse nodes equals injecting the fine nodal values).  All matrices act on
    unknowns only."""

    def __init__(self, V, T, finest, coarsest, k_func=None, k_fine=None, kind="scaled", K_func=None,
                 smoother="jacobi", omega=2.0 / 3.0, cheb_degree=2, cheb_lo=0.3, cheb_hi=1.1,
                 power_its=15):
        self.macro = MacroMesh(V, T)
        self.finest, self.coarsest = finest, coarsest
        self.levels = list(range(coarsest, finest + 1))
        self.mesh = {l: LevelMesh(self.macro, l) for l in self.levels}
        self.A, self.D, self.P, self.k = {}, {}, {}, {}
        for l in self.levels:
            lm = self.mesh[l]
            if K_func is not None:  # tensor coefficient (M = 6), scaled form
                kl = tensor_split(K_func(lm.coords))
                self.k[l] = kl
                self.A[l] = tensor_matrix(lm, kl, "scaled")[lm.unknowns][:, lm.unknowns].tocsr()
                self.D[l] = self.A[l].diagonal()
                continue
            if k_fine is not None:
                kl = self._inject(k_fine, l)
            else:
                kl = k_func(lm.coords)
            self.k[l] = kl
            self.A[l] = lm.system(kl, kind)
            self.D[l] = self.A[l].diagonal()
        for l in self.levels[1:]:
            Pf = prolongation(self.mesh[l - 1], self.mesh[l])
            self.P[l] = Pf[self.mesh[l].unknowns][:, self.mesh[l - 1].unknowns].tocsr()
        Ac = self.A[coarsest].toarray()
        self.kind = kind
        if kind == "volface":  # not symmetric: LU on the coarsest level
            self.lu = sla.lu_factor(Ac)
        else:
            self.chol = np.linalg.cholesky(Ac)
        self.smoother, self.omega = smoother, omega
        self.cheb_degree, self.cheb_lo, self.cheb_hi = cheb_degree, cheb_lo, cheb_hi
        self.lam = {l: self.lambda_max(l, power_its) for l in self.levels}

    def _inject(self, k_fine, l):
        fine = self.mesh[self.finest]
        lm = self.mesh[l]
        s = 1 << (self.finest - l)
        out = np.empty(lm.n)
        for t in range(len(self.macro.T)):
            L = lm.local[t]
            sel = L >= 0
            ii, jj, kk = np.nonzero(sel)
            out[L[sel]] = k_fine[fine.local[t][s * ii, s * jj, s * kk]]
        return out

    def lambda_max(self, l, its):
        """Power iteration on D^-1 A; returns the Rayleigh quotient
        (x.Ax)/(x.Dx) of the last iterate."""
        A, D = self.A[l], self.D[l]
        x = power_start(self.mesh[l])
        lam = 0.0
        for _ in range(its):
            y = (A @ x) / D
            x = y / math.sqrt(float(np.dot(y, y)))
        Ax = A @ x
        lam = float(np.dot(x, Ax)) / float(np.dot(x, D * x))
        return lam

    def coarse_solve(self, f):
        if self.kind == "volface":
            return sla.lu_solve(self.lu, f)
        y = sla.solve_triangular(self.chol, f, lower=True)
        return sla.solve_triangular(self.chol.T, y, lower=False)

    def jacobi(self, l, f, u, sweeps):
        A, D = self.A[l], self.D[l]
        for _ in range(sweeps):
            u = u + self.omega * (f - A @ u) / D
        return u

    def chebyshev(self, l, f, u, degree=None):
        """Chebyshev iteration of the given degree for D^-1 A on
        [lo * lam, hi * lam] (three-term recurrence, Saad, Iterative Methods
        for Sparse Linear Systems, Alg. 12.1)."""
        m = degree or self.cheb_degree
        A, D = self.A[l], self.D[l]
        a, b = self.cheb_lo * self.lam[l], self.cheb_hi * self.lam[l]
        theta, delta = 0.5 * (b + a), 0.5 * (b - a)
        sigma = theta / delta
        rho = 1.0 / sigma
        d = (f - A @ u) / D / theta
        u = u + d
        for _ in range(1, m):
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * ((f - A @ u) / D)
            u = u + d
            rho = rho_new
        return u

    def smooth(self, l, f, u, sweeps):
        if self.smoother == "jacobi":
            return self.jacobi(l, f, u, sweeps)
        for _ in range(sweeps):
            u = self.chebyshev(l, f, u)
        return u

    def vcycle(self, l, f, u, nu1=2, nu2=2):
        """Symmetric V(nu1,nu2): smooth, restrict the residual with P^T,
        recurse from a zero guess, prolongate the correction, smooth."""
        if l == self.coarsest:
            return self.coarse_solve(f)
        u = self.smooth(l, f, u, nu1)
        r = f - self.A[l] @ u
        rc = self.P[l].T @ r
        ec = self.vcycle(l - 1, rc, np.zeros_like(rc), nu1, nu2)
        u = u + self.P[l] @ ec
        return self.smooth(l, f, u, nu2)

    def pcg(self, f, tol=1e-8, maxit=100, nu1=2, nu2=2, x0=None):
        """CG preconditioned by one V-cycle from a zero guess; stops when
        ||r||_2 / ||f||_2 <= tol.  Returns (x, iterations, residual history)."""
        l = self.finest
        A = self.A[l]
        x = np.zeros_like(f) if x0 is None else x0.copy()
        r = f - A @ x
        nf = math.sqrt(float(np.dot(f, f)))
        hist = [math.sqrt(float(np.dot(r, r))) / nf]
        z = self.vcycle(l, r, np.zeros_like(r), nu1, nu2)
        p = z.copy()
        rz = float(np.dot(r, z))
        it = 0
        for it in range(1, maxit + 1):
            q = A @ p
            alpha = rz / float(np.dot(p, q))
            x = x + alpha * p
            r = r - alpha * q
            hist.append(math.sqrt(float(np.dot(r, r))) / nf)
            if hist[-1] <= tol:
                break
            z = self.vcycle(l, r, np.zeros_like(r), nu1, nu2)
            rz_new = float(np.dot(r, z))
            p = z + (rz_new / rz) * p
            rz = rz_new
        return x, it, hist

    def mg_solve(self, f, its, nu1=3, nu2=3, x0=None):
        """Multigrid as the solver (Sec. 7.2: V(3,3) cycles, i* = 10): x <-
        V-cycle(f, x) from x0 = 0; returns x and the residual 2-norms r^(i),
        i = 0..its."""
        l = self.finest
        A = self.A[l]
        x = np.zeros_like(f) if x0 is None else x0.copy()
        hist = [float(np.linalg.norm(f - A @ x))]
        for _ in range(its):
            x = self.vcycle(l, f, x, nu1, nu2)
            hist.append(float(np.linalg.norm(f - A @ x)))
        return x, hist

    def direct_solve(self, f):
        return spla.spsolve(self.A[self.finest].tocsc(), f)


# ----------------------------------------------------------------------------
# Error norms (Sec. 7.2 asks for an appropriately scaled nodal L2 error without
# fixing it: read as sqrt(e^T M_L e) with the lumped P1 mass; H1 by quadrature)
# ----------------------------------------------------------------------------


def mg_rate(hist, i_star=10, i0=5):
    """Asymptotic convergence rate of Sec. 7 (start of the numerical section):
    rho = (r^(i*) / r^(5))^(1 / (i* - 5))."""
    return (hist[i_star] / hist[i0]) ** (1.0 / (i_star - i0))


def discrete_l2(lm: LevelMesh, e):
    """sqrt(e^T M_L e) with lumped (row-sum) P1 mass weights."""
    M = lm.assemble_mass()
    mL = np.asarray(M.sum(axis=1)).reshape(-1)
    return math.sqrt(float(np.sum(mL * e * e)))


def _tet_rule(q=4):
    """Collapsed (Duffy) Gauss-Legendre rule on the reference tetrahedron:
    returns barycentric points (m,4) and weights summing to 1/6."""
    g, w = np.polynomial.legendre.leggauss(q)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    pts, wts = [], []
    for a, wa in zip(g, w):
        for b, wb in zip(g, w):
            for c, wc in zip(g, w):
                xi = a
                eta = (1 - a) * b
                zeta = (1 - a) * (1 - b) * c
                pts.append([1 - xi - eta - zeta, xi, eta, zeta])
                wts.append(wa * wb * wc * (1 - a) ** 2 * (1 - b))
    return np.array(pts), np.array(wts)


def h1_seminorm_error(lm: LevelMesh, uh, grad_u, q=4):
    """sqrt(sum_t int_t |grad u - grad u_h|^2) by a Duffy rule per micro tet."""
    lam, wq = _tet_rule(q)
    tot = 0.0
    for t in range(len(lm.macro.T)):
        ids = lm.micro[t]
        X = lm.coords[ids]
        G, vol = p1_gradients(X)
        guh = np.einsum("na,nai->ni", uh[ids], G)
        for lq, w in zip(lam, wq):
            xq = np.einsum("a,nai->ni", lq, X)
            d = grad_u(xq) - guh
            tot += float(np.sum(6.0 * vol * w * np.sum(d * d, axis=1)))
    return math.sqrt(tot)
