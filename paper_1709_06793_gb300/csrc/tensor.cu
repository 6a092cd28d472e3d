// Operator of a tensor coefficient (M = 6; eq. "integral", eq. "meshdep"
// with M > 1, Sec. 7.3) in the modes of the scaled kernel.
#include <algorithm>

#include "hhg_internal.h"

namespace hhg {

// pointers and scalars of one tensor-operator launch
struct TensorPtrs {
  const void* u;
  const void* f;
  void* out;
  double omega;
};

// ---------------------------------------------------------------------------
// Tensor coefficient, M = 6 (eq. "meshdep" with M > 1, Sec. 7.3): row of x
//     sum_d sum_m c^m_d (k_m(x) + k_m(x+w_d)) (u_{x+w_d} - u_x)
// with c^m = (1/2) reference stencil of the m-th term (d_m . grad)(d_m . grad)
// of x's primitive.  Volume rows: one warp per stored row with the
// per-direction node weights below; rows of nodes on macro faces, edges and
// vertices: one thread per unique node sums its copies' partial rows.
// ---------------------------------------------------------------------------
template <class T, int MODE>
__device__ __forceinline__ T tensor_finish(T y, T dg, T ux, long long idx, const TensorPtrs& p) {
  if (MODE == OP_RESID) return static_cast<const T*>(p.f)[idx] - y;
  if (MODE == OP_JACOBI) return ux + (T)p.omega * (static_cast<const T*>(p.f)[idx] - y) / dg;
  if (MODE == OP_DIAG) return dg;
  return y;
}

// the six k_m of a node (node-major, 8- or 16-byte aligned: three vector loads)
__device__ __forceinline__ void load6(const float* p, float (&v)[6]) {
  const float2* q = reinterpret_cast<const float2*>(p);
  const float2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}
__device__ __forceinline__ void load6(const double* p, double (&v)[6]) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}

// Per-direction node weights.  Every term's volume stencil is point
// symmetric (c^m_{-d} = c^m_d), so the weight of a volume row's edge
// (x, x+w_d) is
//     sum_m c^m_d (k_m(x) + k_m(x+w_d)) = B_d(x) + B_d(x+w_d),
//     B_d(z) = sum_m c^m_d k_m(z)   (d = the 7 positive directions),
// with c^m the volume stencil of the tet (also where x+w_d lies on a face).
// One warp per stored row, lanes along i; direction major (B_d of all
// nodes, then B_{d+1}), so a warp's loads of one direction are coalesced.
__global__ void tensor_weights_kernel(DepthDev D, const double* __restrict__ tsten, const double* __restrict__ km,
                                      long long n, double* __restrict__ tb64, float* __restrict__ tb32) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < D.n_rows; r += nwarps) {
    const int4 row = D.rows[r];
    const TetDev td = D.tets[row.x];
    const int N = td.N, j = row.y, k = row.z;
    const double* st = tsten + (size_t)row.x * 6 * 16 * kNDir;  // mask 0 = volume rows
    for (int i = lane; i + j + k <= N; i += 32) {
      const long long x = td.base + node_offset(N, i, j, k);
      double kx[6];
      load6(km + 6 * x, kx);
      for (int d = 0; d < 7; ++d) {
        double b = 0;
#pragma unroll
        for (int m = 0; m < 6; ++m) b = fma(st[m * 16 * kNDir + d], kx[m], b);
        tb64[d * n + x] = b;
        tb32[d * n + x] = (float)b;
      }
    }
  }
}

void compute_tensor_weights(Mesh& m, cudaStream_t s) {
  for (int d = 0; d < m.ndepth; ++d) {
    Depth& D = m.depth[d];
    if (D.n_rows == 0) continue;
    if (!D.tb64) {
      const size_t n = std::max<long long>(D.n_stored, 1);
      D.tb64 = static_cast<double*>(dalloc(D, 7 * n * 8));
      D.tb32 = static_cast<float*>(dalloc(D, 7 * n * 4));
    }
    const int g = std::max(1, std::min((D.n_rows + 7) / 8, 16 * m.num_sms));
    tensor_weights_kernel<<<g, 256, 0, s>>>(D.dev, D.tsten64, D.km64, D.n_stored, D.tb64, D.tb32);
    HHG_CUDA(cudaGetLastError());
  }
}

// Volume rows: one warp per stored row with volume nodes (j, k >= 1, j + k <=
// N - 2), lanes along i = 1 .. N-j-k-1; every neighbour is in the tet.
template <class T, int MODE>
__global__ void __launch_bounds__(256) tensor_volume_kernel(DepthDev D, const T* __restrict__ tb, long long nst,
                                                            TensorPtrs p, int n_rows) {
  const T* u = static_cast<const T*>(p.u);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < n_rows; r += nwarps) {
    const int4 row = D.rows[r];
    const TetDev td = D.tets[row.x];
    const int N = td.N, j = row.y, k = row.z;
    if (j < 1 || k < 1 || j + k > N - 2) continue;
    for (int i = 1 + lane; i + j + k <= N - 1; i += 32) {
      const long long x = td.base + node_offset(N, i, j, k);
      const T ux = u[x];
      T bx[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) bx[q] = __ldg(tb + q * nst + x);
      T y = 0, dg = 0;
#pragma unroll
      for (int d = 0; d < kNDir; ++d) {
        int di, dj, dk;
        dir_of(d, di, dj, dk);
        const int dp = d < 7 ? d : d - 7;
        const long long yx = td.base + node_offset(N, i + di, j + dj, k + dk);
        const T s = bx[dp] + __ldg(tb + dp * nst + yx);
        y = fma(s, u[yx] - ux, y);
        dg -= s;
      }
      static_cast<T*>(p.out)[x] = tensor_finish<T, MODE>(y, dg, ux, x, p);
    }
  }
}

// Partial row (and partial diagonal) of one copy of a node on a macro
// face/edge/vertex, from the six k_m and the stencils of its primitive.
template <class T>
__device__ __forceinline__ void tensor_partial(const DepthDev& D, const T* __restrict__ tsten,
                                               const T* __restrict__ km, const T* __restrict__ u, const BCopy& cp,
                                               T& y, T& dg) {
  const TetDev td = D.tets[cp.slot];
  const int N = td.N, i = cp.i, j = cp.j, k = cp.k, mask = cp.mask;
  const T* st = tsten + (size_t)cp.slot * 6 * 16 * kNDir;
  const long long x = cp.idx;
  const T ux = u[x];
  T kx[6];
  load6(km + 6 * x, kx);
#pragma unroll
  for (int d = 0; d < kNDir; ++d) {
    int di, dj, dk;
    dir_of(d, di, dj, dk);
    const int a = i + di, b = j + dj, c = k + dk;
    if (a < 0 || b < 0 || c < 0 || a + b + c > N) continue;
    const long long yx = td.base + node_offset(N, a, b, c);
    T ky[6];
    load6(km + 6 * yx, ky);
    T s = 0;
#pragma unroll
    for (int m = 0; m < 6; ++m) s = fma(st[(m * 16 + mask) * kNDir + d], kx[m] + ky[m], s);
    y = fma(s, u[yx] - ux, y);
    dg -= s;
  }
}

// Interface rows: one thread per unique boundary node sums its copies'
// partial rows, applies the epilogue and writes every copy (Dirichlet: 0).
template <class T, int MODE>
__global__ void tensor_bnodes_kernel(DepthDev D, const T* __restrict__ tsten, const T* __restrict__ km,
                                     TensorPtrs p, int n_b) {
  const T* u = static_cast<const T*>(p.u);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_b; b += gridDim.x * blockDim.x) {
    const int lo = D.bstart[b], hi = D.bstart[b + 1];
    T val;
    if (D.bdir[b]) {
      val = MODE == OP_DIAG ? (T)1 : (T)0;
    } else {
      T y = 0, dg = 0;
      for (int q = lo; q < hi; ++q) tensor_partial<T>(D, tsten, km, u, D.bcopies[q], y, dg);
      const long long i0 = D.bcopies[lo].idx;
      val = tensor_finish<T, MODE>(y, dg, u[i0], i0, p);
    }
    for (int q = lo; q < hi; ++q) static_cast<T*>(p.out)[D.bcopies[q].idx] = val;
  }
}

template <class T, int MODE>
static void tensor_typed(const Mesh& m, int depth, const OpArgs& a, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  const DepthDev& D = Dh.dev;
  const int n_rows = a.nc_only ? D.n_rows_nc : D.n_rows;
  const int n_b = a.nc_only ? D.n_bnodes_nc : D.n_bnodes;
  const T* tsten;
  const T* km;
  const T* tb;
  if constexpr (sizeof(T) == 8) {
    tsten = Dh.tsten64;
    km = Dh.km64;
    tb = Dh.tb64;
  } else {
    tsten = Dh.tsten32;
    km = Dh.km32;
    tb = Dh.tb32;
  }
  TensorPtrs p{a.u, a.f, a.out, a.omega};
  if (n_rows > 0) {
    const int g = std::max(1, std::min((n_rows + 7) / 8, 16 * m.num_sms));
    tensor_volume_kernel<T, MODE><<<g, 256, 0, s>>>(D, tb, D.n_stored, p, n_rows);
    HHG_CUDA(cudaGetLastError());
  }
  if (n_b > 0) {
    tensor_bnodes_kernel<T, MODE><<<std::min((n_b + 127) / 128, 16 * m.num_sms), 128, 0, s>>>(D, tsten, km, p, n_b);
    HHG_CUDA(cudaGetLastError());
  }
}

template <class T>
static void tensor_dispatch(const Mesh& m, int depth, OpMode mode, const OpArgs& a,
                            cudaStream_t s) {
  switch (mode) {
    case OP_APPLY: tensor_typed<T, OP_APPLY>(m, depth, a, s); break;
    case OP_RESID: tensor_typed<T, OP_RESID>(m, depth, a, s); break;
    case OP_JACOBI: tensor_typed<T, OP_JACOBI>(m, depth, a, s); break;
    case OP_DIAG: tensor_typed<T, OP_DIAG>(m, depth, a, s); break;
    default: throw Error{HHG_ERR_ARG, "the tensor operator has no Chebyshev mode"};
  }
}

void launch_tensor_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a,
                      cudaStream_t s) {
  HHG_REQUIRE(m.tensor_set, "hhg_set_tensor_coefficient must be called first");
  HHG_REQUIRE(dtype == HHG_F64 || dtype == HHG_F32, "the tensor operator runs in HHG_F64 or HHG_F32");
  if (dtype == HHG_F64)
    tensor_dispatch<double>(m, depth, mode, a, s);
  else
    tensor_dispatch<float>(m, depth, mode, a, s);
}

}  // namespace hhg
