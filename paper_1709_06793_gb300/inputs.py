"""Seeded synthetic inputs shared by the tests, the bench and the smoke run.

This module holds macro meshes (vertex coordinates + tetrahedra with their
refinement vertex order), coefficient fields, manufactured solutions and a
keyed counter-based random generator.  It contains none of the method's
arithmetic (no stencils, element matrices, refinement or solver steps), so both
the CUDA path and the CPU oracle can take their inputs from here.

It must stay importable without the CUDA library: it imports only numpy.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

# ----------------------------------------------------------------------------
# Macro meshes.  A mesh is (V, T): V float64 (nv, 3); T int32 (nt, 4).  The
# order of a tetrahedron's vertices is its refinement order (it fixes the
# interior diagonal of the uniform refinement, Sec. 2.1 / Bey's rule).
# ----------------------------------------------------------------------------


def unit_tet():
    """Unit reference tetrahedron of Fig. "stencilsign" (A)."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    return V, np.array([[0, 1, 2, 3]], dtype=np.int32)


def regular_tet():
    """Regular tetrahedron of Fig. "stencilsign" (B) (edge length 2)."""
    s = 1.0 / math.sqrt(2.0)
    V = np.array([[1, 0, -s], [-1, 0, -s], [0, 1, s], [0, -1, s]], dtype=np.float64)
    return V, np.array([[0, 1, 2, 3]], dtype=np.int32)


def kuhn_cube():
    """Unit cube split into the 6 Kuhn (path) tetrahedra.

    Each tetrahedron is ordered along its monotone path 0 -> e_a -> e_a+e_b ->
    (1,1,1); all six share the main diagonal.  The paper only states "six
    tetrahedra" for the 3D scalar test (Sec. 7.2); this is the reading used.
    """
    V = np.array(list(itertools.product([0, 1], repeat=3)), dtype=np.float64)  # index = 4x+2y+z

    def vid(p):
        return 4 * p[0] + 2 * p[1] + p[2]

    T = []
    for perm in itertools.permutations(range(3)):
        p = [0, 0, 0]
        path = [vid(p)]
        for a in perm:
            p = list(p)
            p[a] = 1
            path.append(vid(p))
        T.append(path)
    return V, np.array(T, dtype=np.int32)


def cube48(seed=3, jitter=0.08):
    """Unit cube as a conforming mesh of 48 tetrahedra with shared faces: the
    2 x 2 x 2 grid of half cubes, each split into the 6 Kuhn tetrahedra of
    kuhn_cube (the same path orientation everywhere, so neighbouring half
    cubes meet face to face), then the grid's vertices moved at random
    (seeded): the centre in all three directions, face centres within their
    face, edge midpoints along their edge, by up to `jitter` (the half-cube
    edge is 0.5); the corners and the cube's boundary stay.  A batched mesh
    whose tetrahedra share faces, edges and vertices."""
    rng = np.random.default_rng(seed)
    grid = list(itertools.product(range(3), repeat=3))  # index = 9x+3y+z
    V = np.array(grid, dtype=np.float64) * 0.5
    for n, g in enumerate(grid):
        for a in range(3):
            if g[a] == 1:  # interior coordinate of this vertex's face / edge / the centre
                V[n, a] += rng.uniform(-jitter, jitter)

    def vid(p):
        return 9 * p[0] + 3 * p[1] + p[2]

    T = []
    for base in itertools.product(range(2), repeat=3):
        for perm in itertools.permutations(range(3)):
            p = list(base)
            path = [vid(p)]
            for a in perm:
                p = list(p)
                p[a] += 1
                path.append(vid(p))
            T.append(path)
    return V, np.array(T, dtype=np.int32)


def cube12():
    """Unit cube: body centre + 2 triangles per face, coned to the centre (12 tets)."""
    corners = np.array(list(itertools.product([0, 1], repeat=3)), dtype=np.float64)
    V = np.vstack([corners, [[0.5, 0.5, 0.5]]])
    c = 8
    T = []
    for axis in range(3):
        for side in (0, 1):
            face = [i for i in range(8) if corners[i, axis] == side]
            # order the 4 face corners around the face
            others = [a for a in range(3) if a != axis]
            face.sort(key=lambda i: (corners[i, others[0]], corners[i, others[1]]))
            q = [face[0], face[1], face[3], face[2]]  # cyclic
            T.append([c, q[0], q[1], q[2]])
            T.append([c, q[0], q[2], q[3]])
    return V, np.array(T, dtype=np.int32)


def cube24():
    """Unit cube: body centre + 6 face centres; each face cut into 4 triangles
    (face centre + one face edge), each triangle coned to the body centre:
    24 macro tetrahedra (the large-run configuration's cube split)."""
    corners = np.array(list(itertools.product([0, 1], repeat=3)), dtype=np.float64)
    V = [tuple(x) for x in corners]
    V.append((0.5, 0.5, 0.5))
    body = 8
    T = []
    for axis in range(3):
        for side in (0, 1):
            face = [i for i in range(8) if corners[i, axis] == side]
            others = [a for a in range(3) if a != axis]
            face.sort(key=lambda i: (corners[i, others[0]], corners[i, others[1]]))
            q = [face[0], face[1], face[3], face[2]]
            fc = [0.5, 0.5, 0.5]
            fc[axis] = float(side)
            V.append(tuple(fc))
            fid = len(V) - 1
            for e in range(4):
                T.append([body, fid, q[e], q[(e + 1) % 4]])
    return np.array(V, dtype=np.float64), np.array(T, dtype=np.int32)


def _angles_ok(P, min_deg):
    """All 12 face angles and 6 dihedral angles of tetrahedron P (4,3) >= min_deg."""
    lim = math.radians(min_deg)
    for f in itertools.combinations(range(4), 3):
        for a in range(3):
            p = P[f[a]]
            u = P[f[(a + 1) % 3]] - p
            v = P[f[(a + 2) % 3]] - p
            c = np.dot(u, v) / (np.linalg.norm(u) * np.linalg.norm(v))
            if math.acos(max(-1.0, min(1.0, c))) < lim:
                return False
    normals = []
    for opp in range(4):
        f = [a for a in range(4) if a != opp]
        n = np.cross(P[f[1]] - P[f[0]], P[f[2]] - P[f[0]])
        if np.dot(n, P[opp] - P[f[0]]) > 0:
            n = -n  # outward
        normals.append(n / np.linalg.norm(n))
    for a, b in itertools.combinations(range(4), 2):
        dih = math.pi - math.acos(max(-1.0, min(1.0, float(np.dot(normals[a], normals[b])))))
        if dih < lim:
            return False
    return True


def random_tets(n, seed=1, min_deg=20.0):
    """n independent shape-regular tetrahedra from seeded random affine maps.

    Each is an affine image of the regular tetrahedron, rejection-sampled until
    every face angle and dihedral angle is >= min_deg.  The tetrahedra share no
    vertex: they form n independent problems (a batch)."""
    rng = np.random.default_rng(seed)
    base, _ = regular_tet()
    Vs, Ts = [], []
    for t in range(n):
        while True:
            A = np.eye(3) + 0.35 * rng.standard_normal((3, 3))
            P = base @ A.T
            if np.linalg.det(A) <= 0.1:
                continue
            if _angles_ok(P, min_deg):
                break
        P = P / np.max(np.abs(P)) * 0.5 + rng.uniform(-2, 2, 3)
        Vs.append(P)
        Ts.append([4 * t, 4 * t + 1, 4 * t + 2, 4 * t + 3])
    return np.vstack(Vs), np.array(Ts, dtype=np.int32)


# ----------------------------------------------------------------------------
# Coefficient fields k(x) and right-hand sides (vectorised over x: (n,3)).
# ----------------------------------------------------------------------------


def k_unit_tet(x):
    """1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z)."""
    x = np.asarray(x, dtype=np.float64)
    return 1.0 + 0.5 * np.sin(2 * np.pi * x[:, 0]) * np.sin(2 * np.pi * x[:, 1]) * np.sin(2 * np.pi * x[:, 2])


def k_cube(x):
    """exp(sin(pi x) cos(pi y) z)."""
    x = np.asarray(x, dtype=np.float64)
    return np.exp(np.sin(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1]) * x[:, 2])


def grad_k_cube(x):
    x = np.asarray(x, dtype=np.float64)
    sx, cx = np.sin(np.pi * x[:, 0]), np.cos(np.pi * x[:, 0])
    sy, cy = np.sin(np.pi * x[:, 1]), np.cos(np.pi * x[:, 1])
    z = x[:, 2]
    k = np.exp(sx * cy * z)
    return np.stack([k * np.pi * cx * cy * z, -k * np.pi * sx * sy * z, k * sx * cy], axis=1)


def u_sine(x):
    """Manufactured solution sin(pi x) sin(pi y) sin(pi z)."""
    x = np.asarray(x, dtype=np.float64)
    return np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.sin(np.pi * x[:, 2])


def grad_u_sine(x):
    x = np.asarray(x, dtype=np.float64)
    s = np.sin(np.pi * x)
    c = np.cos(np.pi * x)
    return np.pi * np.stack([c[:, 0] * s[:, 1] * s[:, 2], s[:, 0] * c[:, 1] * s[:, 2], s[:, 0] * s[:, 1] * c[:, 2]], axis=1)


def f_cube_sine(x):
    """f = -div(k grad u) for k = k_cube, u = u_sine (Laplacian of u is -3 pi^2 u)."""
    gk = grad_k_cube(x)
    gu = grad_u_sine(x)
    return -(np.sum(gk * gu, axis=1) + k_cube(x) * (-3.0 * np.pi ** 2) * u_sine(x))


def k_cosine(m):
    """k = cos(m pi x y z) + 2 (the parameter-dependent coefficient of the
    paper's 3D scalar test, Sec. 7.2, m = 3 and 8)."""

    def k(x):
        x = np.asarray(x, dtype=np.float64)
        return np.cos(m * np.pi * x[:, 0] * x[:, 1] * x[:, 2]) + 2.0

    return k


def f_sine_cosine_k(m):
    """f = -div(k grad u) for k = k_cosine(m) and u = u_sine (zero on the
    cube's boundary)."""

    def f(x):
        x = np.asarray(x, dtype=np.float64)
        p = x[:, 0] * x[:, 1] * x[:, 2]
        s = -m * np.pi * np.sin(m * np.pi * p)
        gk = np.stack([s * x[:, 1] * x[:, 2], s * x[:, 0] * x[:, 2], s * x[:, 0] * x[:, 1]], axis=1)
        k = np.cos(m * np.pi * p) + 2.0
        return -(np.sum(gk * grad_u_sine(x), axis=1) + k * (-3.0 * np.pi ** 2) * u_sine(x))

    return f


def K_tensor(x):
    """The permeability tensor of the paper's 3D tensor test (Sec. 7.3), as
    (n,6) = (K11, K22, K33, K12, K13, K23); its off-diagonal entries are <= 0."""
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[:, 0] ** 2, x[:, 1] ** 2, x[:, 2] ** 2
    return np.stack([X + 2 * Y + 3 * Z + 1, 2 * X + 3 * Y + Z + 1, 3 * X + Y + 2 * Z + 1, -Y, -Z, -X], axis=1)


def f_sine_tensor(x):
    """f = -div(K grad u) for K = K_tensor and u = u_sine."""
    x = np.asarray(x, dtype=np.float64)
    p = np.pi
    sx, sy, sz = np.sin(p * x[:, 0]), np.sin(p * x[:, 1]), np.sin(p * x[:, 2])
    cx, cy, cz = np.cos(p * x[:, 0]), np.cos(p * x[:, 1]), np.cos(p * x[:, 2])
    g = np.stack([p * cx * sy * sz, p * sx * cy * sz, p * sx * sy * cz], axis=1)  # grad u
    H = np.empty((len(x), 3, 3))  # Hessian of u
    H[:, 0, 0] = H[:, 1, 1] = H[:, 2, 2] = -p * p * sx * sy * sz
    H[:, 0, 1] = H[:, 1, 0] = p * p * cx * cy * sz
    H[:, 0, 2] = H[:, 2, 0] = p * p * cx * sy * cz
    H[:, 1, 2] = H[:, 2, 1] = p * p * sx * cy * cz
    K6 = K_tensor(x)
    K = np.empty((len(x), 3, 3))
    K[:, 0, 0], K[:, 1, 1], K[:, 2, 2] = K6[:, 0], K6[:, 1], K6[:, 2]
    K[:, 0, 1] = K[:, 1, 0] = K6[:, 3]
    K[:, 0, 2] = K[:, 2, 0] = K6[:, 4]
    K[:, 1, 2] = K[:, 2, 1] = K6[:, 5]
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    # div of K's columns: d/dx_j K_ij summed over j, for each row i
    divK = np.empty((len(x), 3))
    dK11 = (2 * X, 4 * Y, 6 * Z)
    dK22 = (4 * X, 6 * Y, 2 * Z)
    dK33 = (6 * X, 2 * Y, 4 * Z)
    dK12 = (0 * X, -2 * Y, 0 * Z)
    dK13 = (0 * X, 0 * Y, -2 * Z)
    dK23 = (-2 * X, 0 * Y, 0 * Z)
    # (div K)_j = sum_i d/dx_i K_ij
    divK[:, 0] = dK11[0] + dK12[1] + dK13[2]
    divK[:, 1] = dK12[0] + dK22[1] + dK23[2]
    divK[:, 2] = dK13[0] + dK23[1] + dK33[2]
    return -(np.einsum("nj,nj->n", divK, g) + np.einsum("nij,nij->n", K, H))


def k_large(x):
    """1 + 0.5 sin(4 pi x) cos(4 pi y) sin(4 pi z).  x: (n, 3) float64, a numpy
    array or a torch tensor (then evaluated on the tensor's device)."""
    if hasattr(x, "sin"):  # torch tensor
        a = 4 * np.pi * x
        return 1.0 + 0.5 * a[:, 0].sin() * a[:, 1].cos() * a[:, 2].sin()
    x = np.asarray(x, dtype=np.float64)
    return 1.0 + 0.5 * np.sin(4 * np.pi * x[:, 0]) * np.cos(4 * np.pi * x[:, 1]) * np.sin(4 * np.pi * x[:, 2])


def u_wave(x):
    """sin(9 x) cos(7 y): a smooth non-polynomial operand for apply timings
    (numpy array or torch tensor, as k_large)."""
    if hasattr(x, "sin"):
        return (9 * x[:, 0]).sin() * (7 * x[:, 1]).cos()
    x = np.asarray(x, dtype=np.float64)
    return np.sin(9 * x[:, 0]) * np.cos(7 * x[:, 1])


def fourier_field(seed, n_modes=8):
    """Smooth random field: sum of n_modes cosines with integer wave vectors in
    {-3..3}^3 \\ {0}, amplitudes N(0,1)/sqrt(n_modes), normalised to max|.| = 1
    on a 16^3 probe grid of the unit cube.  Returns a callable x -> values."""
    rng = np.random.default_rng(seed)
    W = []
    while len(W) < n_modes:
        w = rng.integers(-3, 4, 3)
        if np.any(w != 0):
            W.append(w)
    W = np.array(W, dtype=np.float64)
    amp = rng.standard_normal(n_modes) / math.sqrt(n_modes)
    phase = rng.uniform(0, 2 * np.pi, n_modes)

    def raw(x):
        x = np.asarray(x, dtype=np.float64)
        return np.cos(2 * np.pi * x @ W.T + phase) @ amp

    g = np.linspace(0, 1, 16)
    probe = np.array(list(itertools.product(g, g, g)))
    scale = 1.0 / np.max(np.abs(raw(probe)))
    return lambda x: raw(x) * scale


def k_batched(seed=1):
    """1 + 0.9 tanh(smooth random Fourier field of 8 modes)."""
    g = fourier_field(seed)
    return lambda x: 1.0 + 0.9 * np.tanh(g(x))


def gaussian_random_field(seed=2, corr_len=0.2, n_features=256):
    """Smooth Gaussian random field with squared-exponential covariance
    (correlation length corr_len, unit variance) by random Fourier features."""
    rng = np.random.default_rng(seed)
    Wf = rng.standard_normal((n_features, 3)) / corr_len
    b = rng.uniform(0, 2 * np.pi, n_features)
    a = rng.standard_normal(n_features)

    def g(x):
        x = np.asarray(x, dtype=np.float64)
        return math.sqrt(2.0 / n_features) * (np.cos(x @ Wf.T + b) @ a) / math.sqrt(np.mean(a ** 2))

    return g


def k_learned(seed=2, contrast=100.0):
    """exp(2 g), g a GRF, rescaled so that max k / min k <= contrast on a probe grid."""
    g = gaussian_random_field(seed)
    pts = np.array(list(itertools.product(np.linspace(0, 1, 17), repeat=3)))
    vals = 2.0 * g(pts)
    span = float(vals.max() - vals.min())
    s = min(1.0, math.log(contrast) / span) if span > 0 else 1.0
    return lambda x: np.exp(2.0 * s * g(x))


# ----------------------------------------------------------------------------
# Keyed counter-based uniform generator (SplitMix64 finaliser, Steele et al.
# 2014).  A node is identified by its canonical key: the macro-mesh vertex ids
# carrying a non-zero barycentric weight, those integer weights, and the
# level's N = 2^level.  Copies of one node in several macro tetrahedra share
# the key, so they get the same value on every side.
# ----------------------------------------------------------------------------

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(z):
    z = (z + np.uint64(0x9E3779B97F4A7C15)) & _M64
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
    return z ^ (z >> np.uint64(31))


def node_keys(gverts, weights, N):
    """Canonical key hash per node.

    gverts: (n,4) int global vertex ids of the containing macro tetrahedron;
    weights: (n,4) int barycentric weights (sum N).  Returns uint64 (n,)."""
    g = np.asarray(gverts, dtype=np.int64).copy()
    w = np.asarray(weights, dtype=np.int64)
    g[w == 0] = np.iinfo(np.int64).max
    order = np.argsort(g, axis=1, kind="stable")
    g = np.take_along_axis(g, order, axis=1)
    w = np.take_along_axis(w, order, axis=1)
    g[w == 0] = -1
    with np.errstate(over="ignore"):
        h = _splitmix64(np.full(g.shape[0], N, dtype=np.uint64))
        for a in range(4):
            packed = (g[:, a].astype(np.uint64) << np.uint64(24)) ^ w[:, a].astype(np.uint64)
            h = _splitmix64(h ^ packed)
    return h


def uniform_from_keys(keys, seed, lo=-1.0, hi=1.0):
    """Uniform values in [lo, hi) from key hashes and a seed."""
    with np.errstate(over="ignore"):
        z = _splitmix64(np.asarray(keys, dtype=np.uint64) ^ _splitmix64(np.full(1, seed, dtype=np.uint64)))
    u01 = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u01
