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
// of x's primitive.  Pass 1: one warp per stored row, lanes along i; volume
// rows are final, rows of copies on macro faces/edges/vertices go to the
// scratch vectors (partial row, partial diagonal).  Pass 2: one thread per
// interface node sums its copies' partials and writes every copy.
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

template <class T, int MODE>
__global__ void __launch_bounds__(256) tensor_rows_kernel(DepthDev D, const T* __restrict__ tsten,
                                                          const T* __restrict__ km, long long nst, TensorPtrs p,
                                                          int n_rows, T* __restrict__ py, T* __restrict__ pd) {
  const T* u = static_cast<const T*>(p.u);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < n_rows; r += nwarps) {
    const int4 row = D.rows[r];
    const TetDev td = D.tets[row.x];
    const int N = td.N, j = row.y, k = row.z;
    const T* st = tsten + (size_t)row.x * 6 * 16 * kNDir;
    for (int i = lane; i + j + k <= N; i += 32) {
      const int mask = face_mask(N, i, j, k);
      const long long x = td.base + node_offset(N, i, j, k);
      const T ux = u[x];
      T kx[6];
      load6(km + 6 * x, kx);
      T y = 0, dg = 0;
#pragma unroll
      for (int d = 0; d < kNDir; ++d) {
        int di, dj, dk;
        dir_of(d, di, dj, dk);
        const int a = i + di, b = j + dj, c = k + dk;
        if (a < 0 || b < 0 || c < 0 || a + b + c > N) continue;
        const long long yx = td.base + node_offset(N, a, b, c);
        const T du = u[yx] - ux;
        T ky[6];
        load6(km + 6 * yx, ky);
        T s = 0;
#pragma unroll
        for (int m = 0; m < 6; ++m) s = fma(st[(m * 16 + mask) * kNDir + d], kx[m] + ky[m], s);
        y = fma(s, du, y);
        dg -= s;
      }
      if (mask == 0) {
        static_cast<T*>(p.out)[x] = tensor_finish<T, MODE>(y, dg, ux, x, p);
      } else {
        py[x] = y;
        pd[x] = dg;
      }
    }
  }
}

template <class T, int MODE>
__global__ void tensor_bnodes_kernel(DepthDev D, TensorPtrs p, const T* __restrict__ py, const T* __restrict__ pd,
                                     int n_b) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_b; b += gridDim.x * blockDim.x) {
    const int lo = D.bstart[b], hi = D.bstart[b + 1];
    T val;
    if (D.bdir[b]) {
      val = MODE == OP_DIAG ? (T)1 : (T)0;
    } else {
      T y = 0, dg = 0;
      for (int q = lo; q < hi; ++q) {
        const long long idx = D.bcopies[q].idx;
        y += py[idx];
        dg += pd[idx];
      }
      const long long i0 = D.bcopies[lo].idx;
      val = tensor_finish<T, MODE>(y, dg, static_cast<const T*>(p.u)[i0], i0, p);
    }
    for (int q = lo; q < hi; ++q) static_cast<T*>(p.out)[D.bcopies[q].idx] = val;
  }
}

template <class T, int MODE>
static void tensor_typed(const Mesh& m, int depth, const OpArgs& a, void* py, void* pd, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  const DepthDev& D = Dh.dev;
  const int n_rows = a.nc_only ? D.n_rows_nc : D.n_rows;
  const int n_b = a.nc_only ? D.n_bnodes_nc : D.n_bnodes;
  const T* tsten;
  const T* km;
  if constexpr (sizeof(T) == 8) {
    tsten = Dh.tsten64;
    km = Dh.km64;
  } else {
    tsten = Dh.tsten32;
    km = Dh.km32;
  }
  TensorPtrs p{a.u, a.f, a.out, a.omega};
  if (n_rows > 0) {
    const int g = std::max(1, std::min((n_rows + 7) / 8, 16 * m.num_sms));
    tensor_rows_kernel<T, MODE><<<g, 256, 0, s>>>(D, tsten, km, D.n_stored, p, n_rows, static_cast<T*>(py),
                                                 static_cast<T*>(pd));
    HHG_CUDA(cudaGetLastError());
  }
  if (n_b > 0) {
    tensor_bnodes_kernel<T, MODE><<<std::min((n_b + 127) / 128, 16 * m.num_sms), 128, 0, s>>>(
        D, p, static_cast<const T*>(py), static_cast<const T*>(pd), n_b);
    HHG_CUDA(cudaGetLastError());
  }
}

template <class T>
static void tensor_dispatch(const Mesh& m, int depth, OpMode mode, const OpArgs& a, void* py, void* pd,
                            cudaStream_t s) {
  switch (mode) {
    case OP_APPLY: tensor_typed<T, OP_APPLY>(m, depth, a, py, pd, s); break;
    case OP_RESID: tensor_typed<T, OP_RESID>(m, depth, a, py, pd, s); break;
    case OP_JACOBI: tensor_typed<T, OP_JACOBI>(m, depth, a, py, pd, s); break;
    case OP_DIAG: tensor_typed<T, OP_DIAG>(m, depth, a, py, pd, s); break;
    default: throw Error{HHG_ERR_ARG, "the tensor operator has no Chebyshev mode"};
  }
}

void launch_tensor_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, void* py, void* pd,
                      cudaStream_t s) {
  HHG_REQUIRE(m.tensor_set, "hhg_set_tensor_coefficient must be called first");
  HHG_REQUIRE(dtype == HHG_F64 || dtype == HHG_F32, "the tensor operator runs in HHG_F64 or HHG_F32");
  if (dtype == HHG_F64)
    tensor_dispatch<double>(m, depth, mode, a, py, pd, s);
  else
    tensor_dispatch<float>(m, depth, mode, a, py, pd, s);
}

}  // namespace hhg
