"""Thin ctypes binding of the hhg C ABI (include/hhg.h).

Every function here has the name of the C entry point it calls and only
marshals arguments: torch tensors become device pointers, streams become
cudaStream_t handles, status codes become exceptions.  All arithmetic runs in
the CUDA library; if libhhg.so is missing the import fails loudly (there is no
fallback path).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhhg.so")

HHG_F64, HHG_F32, HHG_F32_KBF16 = 0, 1, 2
HHG_SMOOTH_JACOBI, HHG_SMOOTH_CHEBYSHEV, HHG_SMOOTH_LEARNED = 0, 1, 2
HHG_SOLVE_FP64, HHG_SOLVE_MIXED, HHG_SOLVE_MIXED_KBF16, HHG_SOLVE_MG, HHG_SOLVE_MIXED_KBF16_INNER = 0, 1, 2, 3, 4
HHG_OP_SCALED, HHG_OP_VOLFACE, HHG_OP_NODAL, HHG_OP_TENSOR = 0, 1, 2, 3
STATUS = {0: "HHG_OK", -1: "HHG_ERR_ARG", -2: "HHG_ERR_CUDA", -3: "HHG_ERR_NOMEM",
          -4: "HHG_ERR_NOT_CONVERGED", -5: "HHG_ERR_TIMEOUT", -6: "HHG_ERR_STATE"}


class HHGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class SolveParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("mode", C.c_int), ("smoother", C.c_int),
                ("nu1", C.c_int), ("nu2", C.c_int), ("omega", C.c_double), ("inner_rtol", C.c_double),
                ("max_outer", C.c_int), ("use_graph", C.c_int), ("op", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer", C.c_int), ("rel_residual", C.c_double),
                ("time_ms", C.c_double), ("smoother_used", C.c_int), ("rho", C.c_double)]


class LearnParams(C.Structure):
    _fields_ = [("steps", C.c_int), ("pairs", C.c_int), ("lr", C.c_double), ("omega", C.c_double),
                ("max_depth", C.c_int), ("vcycle_pairs", C.c_int), ("init_noise", C.c_double),
                ("seed", C.c_ulonglong), ("weights_bf16", C.c_int), ("validate_its", C.c_int), ("resume", C.c_int)]


class LearnStats(C.Structure):
    _fields_ = [("loss_jacobi", C.c_double), ("loss_init", C.c_double), ("loss_final", C.c_double),
                ("rho_plain", C.c_double), ("rho_learned", C.c_double), ("accepted", C.c_int), ("steps", C.c_int),
                ("time_ms", C.c_double)]


N_LEARNED_WEIGHTS = 1296


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1709_06793_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P, I, D, L = C.c_void_p, C.c_int, C.c_double, C.c_int64
    sig = {
        "hhg_create_macromesh": [P, I, P, I, P, I, C.POINTER(P)],
        "hhg_create_macromesh_host": [P, I, P, I, P, I, C.POINTER(P)],
        "hhg_destroy_macromesh": [P],
        "hhg_num_depths": [P, C.POINTER(I)],
        "hhg_layout": [P, I, P, P, C.POINTER(L)],
        "hhg_node_coords": [P, I, P],
        "hhg_get_stencils": [P, I, I, P],
        "hhg_set_coefficient": [P, P, P],
        "hhg_apply_scaled": [P, I, P, P, I, P],
        "hhg_apply_nodal": [P, I, P, P, I, P],
        "hhg_apply_volface": [P, I, P, P, I, P],
        "hhg_set_tensor_coefficient": [P, P, P],
        "hhg_apply_tensor": [P, I, P, P, I, P],
        "hhg_residual": [P, I, P, P, P, I, P],
        "hhg_apply_mass": [P, I, P, P, I, P],
        "hhg_autotune": [P, I, C.c_char_p, C.POINTER(I), C.POINTER(I), C.POINTER(D), P],
        "hhg_smooth": [P, I, I, I, D, P, P, I, P],
        "hhg_smooth_noalloc": [P, I, I, D, P, P, I, P],
        "hhg_restrict": [P, I, P, P, I, P],
        "hhg_prolongate_add": [P, I, P, P, I, P],
        "hhg_vcycle": [P, I, I, I, P, P, I, P],
        "hhg_lambda_max": [P, I, I, I, C.POINTER(D), P],
        "hhg_dot": [P, I, P, P, I, C.POINTER(D), P],
        "hhg_solve": [P, C.POINTER(SolveParams), P, P, C.POINTER(SolveStats), P],
        "hhg_set_option": [P, C.c_char_p, D],
        "hhg_device_status": [P],
        "hhg_get_option": [P, C.c_char_p, C.POINTER(D)],
        "hhg_learned_train": [P, C.POINTER(LearnParams), C.POINTER(LearnStats), P],
        "hhg_learned_set_weights": [P, P, I],
        "hhg_learned_get_weights": [P, P],
        "hhg_learned_forward": [P, I, P, P, P],
        "hhg_learned_loss_grad": [P, I, P, P, C.POINTER(D), P, P],
        "hhg_alu_probe": [I, I, I, P, C.POINTER(D), P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.hhg_last_error.argtypes = []
    lib.hhg_last_error.restype = C.c_char_p
    return lib


_lib = _load()


def lib():
    return _lib


def _check(code):
    if code != 0:
        raise HHGError(code, _lib.hhg_last_error().decode())
    return code


def _ptr(x):
    """Device pointer of a torch tensor (or an int address); None -> NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return C.c_void_p(x)
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return C.c_void_p(s)
    return C.c_void_p(s.cuda_stream)


def _host_arrays(verts, tets, levels):
    V = np.ascontiguousarray(verts, dtype=np.float64)
    T = np.ascontiguousarray(tets, dtype=np.int32)
    if np.isscalar(levels) or np.ndim(levels) == 0:
        levels = np.full(len(T), int(levels), dtype=np.int32)
    Lv = np.ascontiguousarray(levels, dtype=np.int32)
    return V, T, Lv


def hhg_create_macromesh(verts, tets, levels, coarsest_level, host_only=False):
    V, T, Lv = _host_arrays(verts, tets, levels)
    out = C.c_void_p()
    f = _lib.hhg_create_macromesh_host if host_only else _lib.hhg_create_macromesh
    _check(f(V.ctypes.data, len(V), T.ctypes.data, len(T), Lv.ctypes.data, int(coarsest_level), C.byref(out)))
    return out


def hhg_create_macromesh_host(verts, tets, levels, coarsest_level):
    return hhg_create_macromesh(verts, tets, levels, coarsest_level, host_only=True)


def hhg_destroy_macromesh(mesh):
    _check(_lib.hhg_destroy_macromesh(mesh))


def hhg_num_depths(mesh):
    n = C.c_int()
    _check(_lib.hhg_num_depths(mesh, C.byref(n)))
    return n.value


def hhg_layout(mesh, depth, nt):
    off = np.zeros(nt + 1, dtype=np.int64)
    lev = np.zeros(nt, dtype=np.int32)
    n = C.c_int64()
    _check(_lib.hhg_layout(mesh, depth, off.ctypes.data, lev.ctypes.data, C.byref(n)))
    return off, lev, n.value


def hhg_node_coords(mesh, depth, n_stored):
    xyz = np.zeros((n_stored, 3), dtype=np.float64)
    _check(_lib.hhg_node_coords(mesh, depth, xyz.ctypes.data))
    return xyz


def hhg_get_stencils(mesh, tet, depth):
    out = np.zeros((16, 14), dtype=np.float64)
    _check(_lib.hhg_get_stencils(mesh, tet, depth, out.ctypes.data))
    return out


def hhg_set_coefficient(mesh, k, stream=None):
    _check(_lib.hhg_set_coefficient(mesh, _ptr(k), _stream(stream)))


def hhg_apply_scaled(mesh, depth, u, y, dtype, stream=None):
    _check(_lib.hhg_apply_scaled(mesh, depth, _ptr(u), _ptr(y), dtype, _stream(stream)))


def hhg_apply_nodal(mesh, depth, u, y, dtype, stream=None):
    _check(_lib.hhg_apply_nodal(mesh, depth, _ptr(u), _ptr(y), dtype, _stream(stream)))


def hhg_apply_volface(mesh, depth, u, y, dtype, stream=None):
    _check(_lib.hhg_apply_volface(mesh, depth, _ptr(u), _ptr(y), dtype, _stream(stream)))


def hhg_set_tensor_coefficient(mesh, K6, stream=None):
    """K6: FP64 device tensor of shape (6, n_stored) = (K11, K22, K33, K12, K13, K23)."""
    _check(_lib.hhg_set_tensor_coefficient(mesh, _ptr(K6), _stream(stream)))


def hhg_apply_tensor(mesh, depth, u, y, dtype, stream=None):
    _check(_lib.hhg_apply_tensor(mesh, depth, _ptr(u), _ptr(y), dtype, _stream(stream)))


def hhg_apply_mass(mesh, depth, u, y, dtype, stream=None):
    _check(_lib.hhg_apply_mass(mesh, depth, _ptr(u), _ptr(y), dtype, _stream(stream)))


def hhg_autotune(mesh, dtype, cache_path=None, stream=None):
    ks, ko, ms = C.c_int(), C.c_int(), C.c_double()
    _check(_lib.hhg_autotune(mesh, dtype, cache_path.encode() if cache_path else None, C.byref(ks), C.byref(ko),
                             C.byref(ms), _stream(stream)))
    return {"kseg": ks.value, "korder": ko.value, "vkernel": int(hhg_get_option(mesh, "vkernel")), "best_ms": ms.value}


def hhg_residual(mesh, depth, f, u, r, dtype, stream=None):
    _check(_lib.hhg_residual(mesh, depth, _ptr(f), _ptr(u), _ptr(r), dtype, _stream(stream)))


def hhg_smooth(mesh, depth, kind, sweeps, omega, f, u, dtype, stream=None):
    _check(_lib.hhg_smooth(mesh, depth, kind, sweeps, float(omega), _ptr(f), _ptr(u), dtype, _stream(stream)))


def hhg_smooth_noalloc(mesh, depth, sweeps, omega, f, u, dtype, stream=None):
    _check(_lib.hhg_smooth_noalloc(mesh, depth, sweeps, float(omega), _ptr(f), _ptr(u), dtype, _stream(stream)))


def hhg_restrict(mesh, depth, rf, rc, dtype, stream=None):
    _check(_lib.hhg_restrict(mesh, depth, _ptr(rf), _ptr(rc), dtype, _stream(stream)))


def hhg_prolongate_add(mesh, depth, ec, uf, dtype, stream=None):
    _check(_lib.hhg_prolongate_add(mesh, depth, _ptr(ec), _ptr(uf), dtype, _stream(stream)))


def hhg_vcycle(mesh, nu1, nu2, smoother, f, u, dtype, stream=None):
    _check(_lib.hhg_vcycle(mesh, nu1, nu2, smoother, _ptr(f), _ptr(u), dtype, _stream(stream)))


def hhg_lambda_max(mesh, depth, its, dtype=HHG_F64, stream=None):
    out = C.c_double()
    _check(_lib.hhg_lambda_max(mesh, depth, its, dtype, C.byref(out), _stream(stream)))
    return out.value


def hhg_dot(mesh, depth, x, y, dtype, stream=None):
    out = C.c_double()
    _check(_lib.hhg_dot(mesh, depth, _ptr(x), _ptr(y), dtype, C.byref(out), _stream(stream)))
    return out.value


def hhg_solve(mesh, f, u, tol=1e-8, maxit=200, mode=HHG_SOLVE_FP64, smoother=HHG_SMOOTH_JACOBI, nu1=2, nu2=2,
              omega=2.0 / 3.0, inner_rtol=3e-5, max_outer=20, use_graph=1, stream=None, raise_on_fail=True,
              op=HHG_OP_SCALED):
    p = SolveParams(tol, maxit, mode, smoother, nu1, nu2, omega, inner_rtol, max_outer, use_graph, op)
    st = SolveStats()
    code = _lib.hhg_solve(mesh, C.byref(p), _ptr(f), _ptr(u), C.byref(st), _stream(stream))
    if code != 0 and (raise_on_fail or code != -4):
        _check(code)
    return {"iterations": st.iterations, "outer": st.outer, "rel_residual": st.rel_residual,
            "time_ms": st.time_ms, "smoother_used": st.smoother_used, "rho": st.rho,
            "status": STATUS.get(code, code)}


def hhg_learned_train(mesh, steps=150, pairs=4, lr=3e-3, omega=2.0 / 3.0, max_depth=0, vcycle_pairs=0,
                      init_noise=0.0, seed=0, weights_bf16=1, validate_its=8, resume=0, stream=None):
    p = LearnParams(steps, pairs, lr, omega, max_depth, vcycle_pairs, init_noise, seed, weights_bf16, validate_its,
                    resume)
    st = LearnStats()
    _check(_lib.hhg_learned_train(mesh, C.byref(p), C.byref(st), _stream(stream)))
    return {f: getattr(st, f) for f, _ in LearnStats._fields_}


def hhg_learned_set_weights(mesh, w, weights_bf16=1):
    w = np.ascontiguousarray(w, dtype=np.float32)
    assert w.shape == (N_LEARNED_WEIGHTS,)
    _check(_lib.hhg_learned_set_weights(mesh, w.ctypes.data, int(weights_bf16)))


def hhg_learned_get_weights(mesh):
    w = np.zeros(N_LEARNED_WEIGHTS, dtype=np.float32)
    _check(_lib.hhg_learned_get_weights(mesh, w.ctypes.data))
    return w


def hhg_learned_forward(mesh, depth, r, c, stream=None):
    _check(_lib.hhg_learned_forward(mesh, depth, _ptr(r), _ptr(c), _stream(stream)))


def hhg_learned_loss_grad(mesh, depth, r, e, stream=None):
    loss = C.c_double()
    g = np.zeros(N_LEARNED_WEIGHTS, dtype=np.float64)
    _check(_lib.hhg_learned_loss_grad(mesh, depth, _ptr(r), _ptr(e), C.byref(loss), g.ctypes.data, _stream(stream)))
    return loss.value, g


def hhg_alu_probe(kind, blocks, iters, out, stream=None):
    """Launch the multiply-add peak probe; returns the launch's flop count."""
    flops = C.c_double()
    _check(_lib.hhg_alu_probe(kind, blocks, iters, _ptr(out), C.byref(flops), _stream(stream)))
    return flops.value


def hhg_device_status(mesh):
    _check(_lib.hhg_device_status(mesh))


def hhg_set_option(mesh, key, value):
    _check(_lib.hhg_set_option(mesh, key.encode(), float(value)))


def hhg_get_option(mesh, key):
    out = C.c_double()
    _check(_lib.hhg_get_option(mesh, key.encode(), C.byref(out)))
    return out.value


class Mesh:
    """Owning handle around hhg_create_macromesh / hhg_destroy_macromesh."""

    def __init__(self, verts, tets, levels, coarsest_level, host_only=False):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int32)
        self.nt = len(self.tets)
        self.h = hhg_create_macromesh(verts, tets, levels, coarsest_level, host_only=host_only)
        self.ndepth = hhg_num_depths(self.h)

    def layout(self, depth=0):
        return hhg_layout(self.h, depth, self.nt)

    def n_stored(self, depth=0):
        return self.layout(depth)[2]

    def coords(self, depth=0):
        return hhg_node_coords(self.h, depth, self.n_stored(depth))

    def stencils(self, tet, depth=0):
        return hhg_get_stencils(self.h, tet, depth)

    def close(self):
        if self.h is not None:
            hhg_destroy_macromesh(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
