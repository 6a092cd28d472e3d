"""CPU-side checks of the C-ABI library: it loads, exports every symbol the
header declares, and its host-only setup (layout, coordinates, the 15
reference stencils per primitive) agrees with the oracle.  No GPU compute."""
import os
import re

import numpy as np
import pytest

from oracle import hhg_oracle as O
from paper_1709_06793_gb300 import inputs as I
from tests import hhg_testutil as U

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_1709_06793_gb300 import build
    build.build()
    from paper_1709_06793_gb300 import hhg
    return hhg


def test_library_exports_every_declared_symbol(H):
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            names |= set(re.findall(r"^(?:int|const char\*)\s+(hhg_\w+)\s*\(", text, re.M))
    assert len(names) >= 18
    for n in sorted(names):
        assert hasattr(H.lib(), n), n


def _dirs():
    out = []
    for d in range(14):
        b = d % 7
        s = 1 if d < 7 else -1
        v = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, -1, 0), (1, 0, -1), (0, 1, -1), (1, -1, 1)][b]
        out.append(tuple(s * x for x in v))
    return out


@pytest.mark.parametrize("mesh", [I.unit_tet, I.regular_tet, lambda: I.random_tets(1, seed=5)])
@pytest.mark.parametrize("level", [2, 3])
def test_primitive_stencils_match_oracle_rows(H, mesh, level):
    """Every one of the 15 primitive stencils equals the oracle's assembled
    (Laplace) row at a node of that primitive, times 1/2 (Sec. 6.1)."""
    V, T = mesh()
    m = H.Mesh(V, T, level, 1, host_only=True)
    st = m.stencils(0, 0)
    lm = O.LevelMesh(O.MacroMesh(V, T), level)
    A = lm.assemble(None, "laplace").tocsr()
    N = 1 << level
    seen = set()
    for i in range(N + 1):
        for j in range(N + 1 - i):
            for k in range(N + 1 - i - j):
                mask = (i + j + k == N) | ((i == 0) << 1) | ((j == 0) << 2) | ((k == 0) << 3)
                if mask in seen:
                    continue
                seen.add(mask)
                x = lm.local[0][i, j, k]
                row = A[x].toarray().ravel()
                for d, (di, dj, dk) in enumerate(_dirs()):
                    a, b, c = i + di, j + dj, k + dk
                    if min(a, b, c) < 0 or a + b + c > N:
                        assert st[mask, d] == 0.0
                        continue
                    assert abs(2 * st[mask, d] - row[lm.local[0][a, b, c]]) < 1e-13
    want = 15 if level >= 2 else 10
    assert len(seen) == want
    m.close()


@pytest.mark.parametrize("mesh,level", [(I.kuhn_cube, 2), (I.cube24, 1), (I.cube12, 2)])
def test_layout_and_coordinates_match_oracle(H, mesh, level):
    V, T = mesh()
    m = H.Mesh(V, T, level, 1, host_only=True)
    off, lev, n = m.layout(0)
    assert off[-1] == n
    nodes = U.stored_nodes(off, lev)
    assert len(nodes) == n
    lm = O.LevelMesh(O.MacroMesh(V, T), level)
    idx = U.oracle_map(lm, nodes)
    assert set(idx.tolist()) == set(range(lm.n))  # every unique node stored at least once
    xyz = m.coords(0)
    assert np.max(np.abs(xyz - lm.coords[idx])) < 1e-15
    # copies of one node share bitwise identical coordinates
    for u in np.unique(idx)[:200]:
        c = xyz[idx == u]
        assert np.all(c == c[0])
    # keys from the stored side agree with the oracle's
    assert np.all(U.stored_keys(T, nodes, lev) == U.oracle_keys(lm)[idx])
    m.close()


def test_mixed_levels_and_depths(H):
    V, T = I.random_tets(5, seed=3)
    levels = [3, 5, 4, 3, 6]
    m = H.Mesh(V, T, levels, 2, host_only=True)
    assert m.ndepth == 5
    for d in range(m.ndepth):
        off, lev, n = m.layout(d)
        for t in range(5):
            want = levels[t] - d
            assert lev[t] == (want if want >= 2 else -1)
        # tets above the coarsest level come first
        act = [t for t in range(5) if lev[t] >= 0]
        nc = [t for t in act if lev[t] > 2]
        first = sorted(act, key=lambda t: off[t])
        assert first[:len(nc)] == sorted(nc, key=lambda t: off[t])
    m.close()


def test_bad_arguments_are_reported(H):
    V, T = I.kuhn_cube()
    with pytest.raises(H.HHGError, match="same level"):
        H.Mesh(V, T, [3, 3, 3, 3, 3, 4], 2, host_only=True)
    with pytest.raises(H.HHGError, match="vertex id"):
        H.Mesh(V, np.array([[0, 1, 2, 99]]), 3, 2, host_only=True)
    Vd = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 0, 1.0]])
    with pytest.raises(H.HHGError, match="degenerate"):
        H.Mesh(Vd, np.array([[0, 1, 2, 3]]), 3, 2, host_only=True)
    m = H.Mesh(V, T, 3, 2, host_only=True)
    with pytest.raises(H.HHGError, match="host-only"):
        H.hhg_apply_scaled(m.h, 0, 1, 2, H.HHG_F32)
    m.close()
    # the peak probe checks its arguments before it launches anything
    for kind, blocks, iters, out in ((3, 1, 1, 16), (0, 0, 1, 16), (1, 1, 0, 16), (2, 1, 1, None)):
        with pytest.raises(H.HHGError, match="hhg_alu_probe"):
            H.hhg_alu_probe(kind, blocks, iters, out)


def test_size_limits_and_empty_meshes_are_reported(H):
    """Maximum level 10 (N = 1024: i, j, k fit the work lists' 11-bit
    fields), coarsest level in [1, level], at least one tetrahedron."""
    V, T = I.unit_tet()
    m = H.Mesh(V, T, 10, 3, host_only=True)
    assert m.layout(0)[2] == 1025 * 1026 * 1027 // 6 and m.ndepth == 8
    m.close()
    with pytest.raises(H.HHGError, match="level must be in"):
        H.Mesh(V, T, 11, 3, host_only=True)
    with pytest.raises(H.HHGError, match="level must be in"):
        H.Mesh(V, T, 2, 3, host_only=True)
    with pytest.raises(H.HHGError, match="coarsest_level"):
        H.Mesh(V, T, 3, 0, host_only=True)
    with pytest.raises(H.HHGError, match="at least"):
        H.Mesh(V, np.zeros((0, 4), dtype=np.int32), 3, 2, host_only=True)
