// Scaled operator with the pre-asymptotic modification of Sec. 4 (eq.
// "defKmin"): on the directions of gray type of a macro tetrahedron (positive
// entries of its reference volume stencil, Sec. 4.2) the scaling
// (k_x + k_y)/2 of an edge becomes (k_min(x) + k_min(y))/2, where k_min(x)
// is the minimum of k over x and the nodes joined to x by an edge inside the
// same macro tetrahedron.  k_min depends on the tetrahedron, so each stored
// copy of an interface node carries the value of its own tetrahedron, and
// the partial row of each copy (its tetrahedron's micro-elements) uses it.
// Every other direction keeps k: where no stencil entry is positive the
// operator is the unmodified one.
//
// The modified operator runs when the mesh's "kappa" option is on, in every
// mode of the scaled operator (apply, residual, Jacobi, Chebyshev,
// diagonal), so the multigrid, its coarse solve and the CG all use it.  The
// kernels are plain row evaluators (one thread per node of a stored row, one
// thread per unique interface node); this operator is a guard for
// pre-asymptotic meshes, not the throughput path.
#include <algorithm>

#include "hhg_internal.h"

namespace hhg {

namespace {

int grid_for(long long n, int block, int max_blocks) {
  const long long b = (n + block - 1) / block;
  return (int)std::max<long long>(1, std::min<long long>(b, max_blocks));
}

__device__ __forceinline__ int row_start(int N, int q, int j) {
  const int M = N - q;
  const int pl = (N + 1) * (N + 2) * (N + 3) / 6 - (M + 1) * (M + 2) * (M + 3) / 6;
  return pl + j * (M + 1) - j * (j - 1) / 2;
}

template <class T, class E>
__device__ __forceinline__ T as_t(E v) {
  if constexpr (sizeof(E) == 2)
    return (T)__bfloat162float(v);
  else
    return (T)v;
}

// k_min of every stored node of the depth (a warp per stored row, lanes
// along the row), from the FP64 coefficient of the same depth
__global__ void kmin_kernel(DepthDev D, const double* __restrict__ k, double* __restrict__ km, int n_rows) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int w = blockIdx.x * wpb + (threadIdx.x >> 5); w < n_rows; w += gridDim.x * wpb) {
    const int4 r = D.rows[w];
    const TetDev td = D.tets[r.x];
    const int N = td.N, j = r.y, q = r.z;
    const long long rs = td.base + row_start(N, q, j);
    for (int i = lane; i <= N - q - j; i += 32) {
      double mn = k[rs + i];
#pragma unroll
      for (int d = 0; d < kNDir; ++d) {
        int di, dj, dk;
        dir_of(d, di, dj, dk);
        const int a = i + di, b = j + dj, c = q + dk;
        if (a < 0 || b < 0 || c < 0 || a + b + c > N) continue;
        mn = fmin(mn, k[td.base + row_start(N, c, b) + a]);
      }
      km[rs + i] = mn;
    }
  }
}

// FP32, bfloat16 (RN) and bfloat16-in-double copies (rounding is monotone,
// so these are the minima of the rounded coefficients)
__global__ void kmin_convert_kernel(const double* __restrict__ km, long long n, float* __restrict__ k32,
                                    __nv_bfloat16* __restrict__ k16, double* __restrict__ k16d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = km[i];
    k32[i] = (float)v;
    const __nv_bfloat16 b = __double2bfloat16(v);
    k16[i] = b;
    k16d[i] = (double)__bfloat162float(b);
  }
}

// Partial row of node (i, j, q) with stencil `mask` in tet `slot`: the
// off-centre terms of the tet's micro-elements, diagonal accumulated in *dg
template <class T, class KT>
__device__ __forceinline__ T kappa_partial(const DepthDev& D, const T* __restrict__ sten, int slot, int i, int j,
                                           int q, int mask, const T* __restrict__ u, const KT* __restrict__ k,
                                           const KT* __restrict__ km, T* dg) {
  const TetDev td = D.tets[slot];
  const int N = td.N;
  const unsigned gray = D.gray[slot];
  const T* st = sten + (slot * 16 + mask) * kNDir;
  const long long x = td.base + row_start(N, q, j) + i;
  const T ux = u[x], kx = as_t<T>(k[x]), kmx = as_t<T>(km[x]);
  T y = 0, d = 0;
#pragma unroll
  for (int dd = 0; dd < kNDir; ++dd) {
    int di, dj, dk;
    dir_of(dd, di, dj, dk);
    const int a = i + di, b = j + dj, c = q + dk;
    if (a < 0 || b < 0 || c < 0 || a + b + c > N) continue;
    const long long n = td.base + row_start(N, c, b) + a;
    const T kk = (gray >> dd) & 1u ? kmx + as_t<T>(km[n]) : kx + as_t<T>(k[n]);
    const T s = st[dd] * kk;
    y = fma(s, u[n] - ux, y);
    d -= s;
  }
  *dg += d;
  return y;
}

struct KPtrs {
  const void* u;
  const void* k;
  const void* km;
  const void* f;
  void* out;
  const void* d_in;
  void* d_out;
  double omega, ca, cb;
};

template <class T, int MODE>
__device__ __forceinline__ void kappa_finish(const KPtrs& p, long long idx, T y, T diag, T ux, T& val, T& dval) {
  if (MODE == OP_APPLY) {
    val = y;
  } else if (MODE == OP_RESID) {
    val = __ldg(static_cast<const T*>(p.f) + idx) - y;
  } else if (MODE == OP_JACOBI) {
    val = ux + (T)p.omega * (__ldg(static_cast<const T*>(p.f) + idx) - y) / diag;
  } else if (MODE == OP_CHEB) {
    const T prev = p.ca != 0.0 ? (T)p.ca * __ldg(static_cast<const T*>(p.d_in) + idx) : (T)0;
    dval = prev + (T)p.cb * (__ldg(static_cast<const T*>(p.f) + idx) - y) / diag;
    val = ux + dval;
  } else {
    val = diag;
  }
}

// volume rows: a warp per stored row, the row's interior nodes along the lanes
template <class T, class KT, int MODE>
__global__ void kappa_volume_kernel(DepthDev D, const T* __restrict__ sten, KPtrs p, int n_rows) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const T* u = static_cast<const T*>(p.u);
  const KT* k = static_cast<const KT*>(p.k);
  const KT* km = static_cast<const KT*>(p.km);
  for (int w = blockIdx.x * wpb + (threadIdx.x >> 5); w < n_rows; w += gridDim.x * wpb) {
    const int4 r = D.rows[w];
    const TetDev td = D.tets[r.x];
    const int N = td.N, j = r.y, q = r.z;
    if (j < 1 || q < 1) continue;
    const long long rs = td.base + row_start(N, q, j);
    for (int i = 1 + lane; i + j + q <= N - 1; i += 32) {
      T dg = 0;
      const T y = kappa_partial<T, KT>(D, sten, r.x, i, j, q, 0, u, k, km, &dg);
      T val = 0, dval = 0;
      kappa_finish<T, MODE>(p, rs + i, y, dg, u[rs + i], val, dval);
      static_cast<T*>(p.out)[rs + i] = val;
      if (MODE == OP_CHEB) static_cast<T*>(p.d_out)[rs + i] = dval;
    }
  }
}

// interface rows: one thread per unique node, the partial rows of its copies
// summed; Dirichlet nodes get 0 (1 for the diagonal)
template <class T, class KT, int MODE>
__global__ void kappa_boundary_kernel(DepthDev D, const T* __restrict__ sten, KPtrs p, int n_b) {
  const T* u = static_cast<const T*>(p.u);
  const KT* k = static_cast<const KT*>(p.k);
  const KT* km = static_cast<const KT*>(p.km);
  T* out = static_cast<T*>(p.out);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_b; b += gridDim.x * blockDim.x) {
    const int lo = D.bstart[b], hi = D.bstart[b + 1];
    if (D.bdir[b]) {
      for (int c = lo; c < hi; ++c) {
        out[D.bcopies[c].idx] = MODE == OP_DIAG ? (T)1 : (T)0;
        if (MODE == OP_CHEB) static_cast<T*>(p.d_out)[D.bcopies[c].idx] = 0;
      }
      continue;
    }
    T y = 0, dg = 0;
    for (int c = lo; c < hi; ++c) {
      const BCopy cp = D.bcopies[c];
      y += kappa_partial<T, KT>(D, sten, cp.slot, cp.i, cp.j, cp.k, cp.mask, u, k, km, &dg);
    }
    const long long i0 = D.bcopies[lo].idx;
    T val = 0, dval = 0;
    kappa_finish<T, MODE>(p, i0, y, dg, u[i0], val, dval);
    for (int c = lo; c < hi; ++c) {
      out[D.bcopies[c].idx] = val;
      if (MODE == OP_CHEB) static_cast<T*>(p.d_out)[D.bcopies[c].idx] = dval;
    }
  }
}

template <class T, class KT, int MODE>
void launch_t(const Mesh& m, int depth, const OpArgs& a, const void* k, const void* km, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  const DepthDev& D = Dh.dev;
  const int n_rows = a.nc_only ? D.n_rows_nc : D.n_rows;
  const int n_b = a.nc_only ? D.n_bnodes_nc : D.n_bnodes;
  const T* sten = sizeof(T) == 8 ? reinterpret_cast<const T*>(D.sten64) : reinterpret_cast<const T*>(D.sten32);
  KPtrs p{a.u, k, km, a.f, a.out, a.d_in, a.d_out, a.omega, a.ca, a.cb};
  if (n_rows > 0) {
    kappa_volume_kernel<T, KT, MODE><<<grid_for((long long)n_rows * 32, 256, 16 * m.num_sms), 256, 0, s>>>(D, sten, p,
                                                                                                           n_rows);
    HHG_CUDA(cudaGetLastError());
  }
  if (n_b > 0) {
    kappa_boundary_kernel<T, KT, MODE><<<(n_b + 127) / 128, 128, 0, s>>>(D, sten, p, n_b);
    HHG_CUDA(cudaGetLastError());
  }
}

template <int MODE>
void launch_mode(const Mesh& m, int depth, int dtype, const OpArgs& a, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  HHG_REQUIRE(Dh.kmin64, "the kappa option needs the coefficient (hhg_set_coefficient)");
  if (dtype == HHG_F64)
    launch_t<double, double, MODE>(m, depth, a, Dh.k64, Dh.kmin64, s);
  else if (dtype == kF64KBF16)
    launch_t<double, double, MODE>(m, depth, a, Dh.k16d, Dh.kmin16d, s);
  else if (dtype == HHG_F32)
    launch_t<float, float, MODE>(m, depth, a, Dh.k32, Dh.kmin32, s);
  else
    launch_t<float, __nv_bfloat16, MODE>(m, depth, a, Dh.k16, Dh.kmin16, s);
}

}  // namespace

void compute_kmin(Mesh& m, cudaStream_t s) {
  for (int d = 0; d < m.ndepth; ++d) {
    Depth& D = m.depth[d];
    const long long n = std::max<long long>(D.n_stored, 1);
    if (!D.kmin64) {
      D.kmin64 = static_cast<double*>(dalloc(D, n * 8 + kCoefPad));
      D.kmin16d = static_cast<double*>(dalloc(D, n * 8 + kCoefPad));
      D.kmin32 = static_cast<float*>(dalloc(D, n * 4 + kCoefPad));
      D.kmin16 = static_cast<__nv_bfloat16*>(dalloc(D, n * 2 + kCoefPad));
      HHG_CUDA(cudaMemsetAsync(D.kmin64, 0, n * 8 + kCoefPad, s));
      HHG_CUDA(cudaMemsetAsync(D.kmin16d, 0, n * 8 + kCoefPad, s));
      HHG_CUDA(cudaMemsetAsync(D.kmin32, 0, n * 4 + kCoefPad, s));
      HHG_CUDA(cudaMemsetAsync(D.kmin16, 0, n * 2 + kCoefPad, s));
    }
    if (D.dev.n_rows > 0) {
      kmin_kernel<<<grid_for((long long)D.dev.n_rows * 32, 256, 16 * m.num_sms), 256, 0, s>>>(D.dev, D.k64, D.kmin64,
                                                                                             D.dev.n_rows);
      HHG_CUDA(cudaGetLastError());
      kmin_convert_kernel<<<grid_for(D.n_stored, 256, 16 * m.num_sms), 256, 0, s>>>(D.kmin64, D.n_stored, D.kmin32, D.kmin16,
                                                                                   D.kmin16d);
      HHG_CUDA(cudaGetLastError());
    }
  }
}

void launch_kappa_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, cudaStream_t s) {
  switch (mode) {
    case OP_APPLY: launch_mode<OP_APPLY>(m, depth, dtype, a, s); break;
    case OP_RESID: launch_mode<OP_RESID>(m, depth, dtype, a, s); break;
    case OP_JACOBI: launch_mode<OP_JACOBI>(m, depth, dtype, a, s); break;
    case OP_CHEB: launch_mode<OP_CHEB>(m, depth, dtype, a, s); break;
    case OP_DIAG: launch_mode<OP_DIAG>(m, depth, dtype, a, s); break;
  }
}

}  // namespace hhg
