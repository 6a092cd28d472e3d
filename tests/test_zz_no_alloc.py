"""The allocation-free Jacobi entry point, hhg_smooth_noalloc.

It serves callers that must not cause a device allocation during a call
(hhg_smooth allocates its ping-pong vector the first time a depth is used).
This file runs last so that a failure here leaves every other test already
run; it also passes alone in a fresh process.  It checks, through the C ABI,
that two calls in a row give the same result as hhg_smooth (same kernel, so
the tolerance is the FP64/FP32 parity tolerance of the other GPU tests), and
that a depth too large for the fixed scratch array is refused.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("dtype,tol", [(0, 1e-12), (1, 1e-6), (2, 1e-6)])
def test_noalloc_matches_smooth_on_two_calls(H, dtype, tol):
    V, T = I.kuhn_cube()
    m = H.Mesh(V, T, 5, 2)
    off, lev, n = m.layout(0)
    xyz = m.coords(0)
    H.hhg_set_coefficient(m.h, torch.tensor(I.k_cube(xyz), device="cuda"))
    tdt = torch.float64 if dtype == 0 else torch.float32  # dtype 2: FP32 vectors, bfloat16 k
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]  # smooth fields: equal on every copy of a node
    f = torch.tensor(np.sin(2 * x + y) * np.cos(z), device="cuda", dtype=tdt)
    u0 = torch.tensor(np.cos(3 * x - 2 * y + z), device="cuda", dtype=tdt)
    ua, ub = u0.clone(), u0.clone()
    for sweeps in (3, 2):  # odd then even: the result ends in the scratch array, then in u
        H.hhg_smooth(m.h, 0, H.HHG_SMOOTH_JACOBI, sweeps, 2.0 / 3.0, f, ua, dtype)
        H.hhg_smooth_noalloc(m.h, 0, sweeps, 2.0 / 3.0, f, ub, dtype)
        torch.cuda.synchronize()
        err = (torch.max(torch.abs(ua - ub)) / torch.max(torch.abs(ua))).item()
        assert err <= tol, (sweeps, err)
    assert torch.max(torch.abs(ua - u0)).item() > 1e-3  # the sweeps did change u
    m.close()


def test_noalloc_rejects_depth_beyond_scratch(H):
    V, T = I.kuhn_cube()
    m = H.Mesh(V, T, 8, 2)  # 17.2 M stored nodes: 69 MB in FP32 > 16 MiB
    off, lev, n = m.layout(0)
    H.hhg_set_coefficient(m.h, torch.ones(n, device="cuda", dtype=torch.float64))
    f = torch.zeros(n, device="cuda", dtype=torch.float32)
    u = torch.zeros(n, device="cuda", dtype=torch.float32)
    with pytest.raises(H.HHGError, match="scratch"):
        H.hhg_smooth_noalloc(m.h, 0, 1, 2.0 / 3.0, f, u, H.HHG_F32)
    # a coarser depth of the same mesh fits
    off3, lev3, n3 = m.layout(3)
    f3 = torch.zeros(n3, device="cuda", dtype=torch.float32)
    u3 = torch.zeros(n3, device="cuda", dtype=torch.float32)
    H.hhg_smooth_noalloc(m.h, 3, 2, 2.0 / 3.0, f3, u3, H.HHG_F32)
    torch.cuda.synchronize()
    m.close()
