// Multigrid and Krylov components around the scaled operator: coefficient
// injection, restriction / prolongation (linear interpolation between nested
// P1 spaces), the coarsest-level direct solve, deterministic FP64 dot
// products, smoothers, the V-cycle, preconditioned CG and FP64 iterative
// refinement around an FP32 inner solve.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "hhg_internal.h"

namespace hhg {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
static inline int grid_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)std::min<long long>(b, cap);
}

size_t elem_size(int dtype) { return dtype == HHG_F64 || dtype == kF64KBF16 ? 8 : 4; }
static int prec_of(int dtype) { return elem_size(dtype) == 8 ? 0 : 1; }

// Workspace vector `w` of a depth for a precision (zero-initialised on first use).
void* workspace(Mesh& m, int depth, int prec, int w) {
  Depth& D = m.depth[depth];
  if (!D.ws[prec][w]) {
    const size_t bytes = (size_t)std::max<long long>(D.n_stored, 1) * (prec == 0 ? 8 : 4);
    D.ws[prec][w] = dalloc(D, bytes);
    HHG_CUDA(cudaMemset(D.ws[prec][w], 0, bytes));
  }
  return D.ws[prec][w];
}

// ---------------------------------------------------------------------------
// coefficient: copies in FP64 / FP32 / BF16 and injection to coarser depths
// ---------------------------------------------------------------------------
__global__ void convert_k_kernel(const double* __restrict__ k, long long n, double* k64, float* k32,
                                 __nv_bfloat16* k16, double* k16d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = k[i];
    k64[i] = v;
    k32[i] = (float)v;
    const __nv_bfloat16 b = __double2bfloat16(v);
    k16[i] = b;
    k16d[i] = (double)__bfloat162float(b);
  }
}

// coarse node (i,j,k) of tet slot s at depth d+1 takes the fine value at (2i,2j,2k)
template <class V>
__global__ void inject_kernel(DepthDev C, DepthDev F, const V* __restrict__ fine, V* __restrict__ coarse) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < C.n_rows; r += nwarps) {
    const int4 row = C.rows[r];
    const TetDev tc = C.tets[row.x];
    const TetDev tf = F.tets[C.fslot[row.x]];
    const int j = row.y, k = row.z;
    const long long cb = tc.base + node_offset(tc.N, 0, j, k);
    const long long fb = tf.base + node_offset(tf.N, 0, 2 * j, 2 * k);
    for (int i = lane; i + j + k <= tc.N; i += 32) coarse[cb + i] = fine[fb + 2 * i];
  }
}

// the six k_m of one node, moved as one value by the injection kernel
struct K6d {
  double v[6];
};
struct K6f {
  float v[6];
};

// k_m of the six-term split of a symmetric tensor (directions e1, e2, e3,
// e1-e2, e1-e3, e2-e3): k_i = K_ii + sum_{j != i} K_ij, k_ij = -K_ij
__global__ void tensor_split_kernel(const double* __restrict__ K6, long long n, double* __restrict__ km64,
                                    float* __restrict__ km32) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double K11 = K6[i], K22 = K6[n + i], K33 = K6[2 * n + i];
    const double K12 = K6[3 * n + i], K13 = K6[4 * n + i], K23 = K6[5 * n + i];
    const double v[6] = {K11 + K12 + K13, K22 + K12 + K23, K33 + K13 + K23, -K12, -K13, -K23};
    for (int m = 0; m < 6; ++m) {  // node major: the six values of a node are contiguous
      km64[6 * i + m] = v[m];
      km32[6 * i + m] = (float)v[m];
    }
  }
}

void set_tensor_coefficient(Mesh& m, const double* K6, cudaStream_t s) {
  drop_graphs(m);
  ensure_tensor_stencils(m);
  for (int d = 0; d < m.ndepth; ++d) {
    Depth& D = m.depth[d];
    const size_t n = std::max<long long>(D.n_stored, 1);
    if (!D.km64) {
      D.km64 = static_cast<double*>(dalloc(D, 6 * n * 8));
      D.km32 = static_cast<float*>(dalloc(D, 6 * n * 4));
    }
  }
  Depth& D0 = m.depth[0];
  tensor_split_kernel<<<grid_for(D0.n_stored, 256, 4096), 256, 0, s>>>(K6, D0.n_stored, D0.km64, D0.km32);
  HHG_CUDA(cudaGetLastError());
  for (int d = 1; d < m.ndepth; ++d) {
    Depth& C = m.depth[d];
    Depth& F = m.depth[d - 1];
    const int g = grid_for((long long)C.n_rows * 32, 256, 4096);
    inject_kernel<K6d><<<g, 256, 0, s>>>(C.dev, F.dev, reinterpret_cast<const K6d*>(F.km64),
                                         reinterpret_cast<K6d*>(C.km64));
    inject_kernel<K6f><<<g, 256, 0, s>>>(C.dev, F.dev, reinterpret_cast<const K6f*>(F.km32),
                                         reinterpret_cast<K6f*>(C.km32));
    HHG_CUDA(cudaGetLastError());
  }
  init_tensor_configs();
  compute_tensor_weights(m, s);
  m.tensor_set = true;
  for (int t = 0; t < 4; ++t) m.cinv_ready[3][t] = false;
}

// Flags a coefficient that is not finite and positive at some stored node
// (the scaled rule of eq. "discrete" needs k > 0 for a positive operator).
__global__ void check_k_kernel(const double* __restrict__ k, long long n, unsigned* bad) {
  unsigned b = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = k[i];
    if (!(v > 0.0) || !isfinite(v)) b = 1;  // NaN fails v > 0
  }
  if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

void set_coefficient(Mesh& m, const double* k, cudaStream_t s) {
  {
    unsigned* bad = m.d_counter + 48;
    HHG_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned), s));
    const long long n = m.depth[0].n_stored;
    if (n > 0) {
      check_k_kernel<<<grid_for(n, 256, 8 * std::max(m.num_sms, 1)), 256, 0, s>>>(k, n, bad);
      HHG_CUDA(cudaGetLastError());
    }
    unsigned hb = 0;
    HHG_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    HHG_CUDA(cudaStreamSynchronize(s));
    HHG_REQUIRE(hb == 0, "hhg_set_coefficient: k must be finite and positive at every stored node");
  }
  drop_graphs(m);
  learned_invalidate(m);
  for (int d = 0; d < m.ndepth; ++d) {
    Depth& D = m.depth[d];
    const size_t n = std::max<long long>(D.n_stored, 1);
    if (!D.k64) {
      // kCoefPad zero bytes past the end: the volume kernel's bulk copies
      // move whole 16-byte chunks and may reach past the last node
      D.k64 = static_cast<double*>(dalloc(D, n * 8 + kCoefPad));
      D.k16d = static_cast<double*>(dalloc(D, n * 8 + kCoefPad));
      D.k32 = static_cast<float*>(dalloc(D, n * 4 + kCoefPad));
      D.k16 = static_cast<__nv_bfloat16*>(dalloc(D, n * 2 + kCoefPad));
      HHG_CUDA(cudaMemsetAsync(D.k64, 0, n * 8 + kCoefPad, s));
      HHG_CUDA(cudaMemsetAsync(D.k16d, 0, n * 8 + kCoefPad, s));
      HHG_CUDA(cudaMemsetAsync(D.k32, 0, n * 4 + kCoefPad, s));
      HHG_CUDA(cudaMemsetAsync(D.k16, 0, n * 2 + kCoefPad, s));
    }
  }
  Depth& D0 = m.depth[0];
  convert_k_kernel<<<grid_for(D0.n_stored, 256, 4096), 256, 0, s>>>(k, D0.n_stored, D0.k64, D0.k32, D0.k16,
                                                                     D0.k16d);
  HHG_CUDA(cudaGetLastError());
  for (int d = 1; d < m.ndepth; ++d) {
    Depth& C = m.depth[d];
    Depth& F = m.depth[d - 1];
    const int g = grid_for((long long)C.n_rows * 32, 256, 4096);
    inject_kernel<double><<<g, 256, 0, s>>>(C.dev, F.dev, F.k64, C.k64);
    inject_kernel<double><<<g, 256, 0, s>>>(C.dev, F.dev, F.k16d, C.k16d);
    inject_kernel<float><<<g, 256, 0, s>>>(C.dev, F.dev, F.k32, C.k32);
    inject_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(C.dev, F.dev, F.k16, C.k16);
    HHG_CUDA(cudaGetLastError());
  }
  m.coef_set = true;
  if (m.kappa) compute_kmin(m, s);
  for (int o = 0; o < 4; ++o)
    for (int t = 0; t < 4; ++t) m.cinv_ready[o][t] = false;
  for (Depth& D : m.depth)
    for (int t = 0; t < 4; ++t)
      if (D.ndinv[t]) {
        D.ndinv[t] = nullptr;  // recomputed on next use (the memory stays with the depth)
      }
  for (int d = 0; d < m.ndepth; ++d) m.depth[d].lam = 0.0;
}

// ---------------------------------------------------------------------------
// restriction r_c = P^T r_f and prolongation u_f += P e_c
// ---------------------------------------------------------------------------
// Fine node 2c+w_d is the midpoint of the coarse edge (c, c+w_d): P has 1 at
// the coincident node and 1/2 at the 14 edge midpoints around c.
template <class T>
__device__ __forceinline__ T restrict_partial(const DepthDev& F, int fslot, int ci, int cj, int ck,
                                              const T* __restrict__ rf, bool weighted) {
  const TetDev tf = F.tets[fslot];
  const int N = tf.N;
  const int fi = 2 * ci, fj = 2 * cj, fk = 2 * ck;
  T w0 = 1;
  if (weighted) w0 = (T)1 / (T)F.mult[fslot * 16 + face_mask(N, fi, fj, fk)];
  T acc = w0 * rf[tf.base + node_offset(N, fi, fj, fk)];
#pragma unroll
  for (int d = 0; d < kNDir; ++d) {
    int di, dj, dk;
    dir_of(d, di, dj, dk);
    const int a = fi + di, b = fj + dj, c = fk + dk;
    if (a < 0 || b < 0 || c < 0 || a + b + c > N) continue;
    T w = (T)0.5;
    if (weighted) w = w / (T)F.mult[fslot * 16 + face_mask(N, a, b, c)];
    acc = fma(w, rf[tf.base + node_offset(N, a, b, c)], acc);
  }
  return acc;
}

template <class T>
__global__ void restrict_volume_kernel(DepthDev C, DepthDev F, const T* __restrict__ rf, T* __restrict__ rc) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < C.n_rows; r += nwarps) {
    const int4 row = C.rows[r];
    const TetDev tc = C.tets[row.x];
    const int j = row.y, k = row.z, N = tc.N;
    if (j == 0 || k == 0 || j + k >= N - 1) continue;
    const int fs = C.fslot[row.x];
    for (int i = 1 + lane; i + j + k <= N - 1; i += 32)
      rc[tc.base + node_offset(N, i, j, k)] = restrict_partial<T>(F, fs, i, j, k, rf, false);
  }
}

template <class T>
__global__ void restrict_boundary_kernel(DepthDev C, DepthDev F, const T* __restrict__ rf, T* __restrict__ rc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= C.n_bnodes) return;
  const int lo = C.bstart[b], hi = C.bstart[b + 1];
  T v = 0;
  if (!C.bdir[b])
    for (int q = lo; q < hi; ++q) {
      const BCopy cp = C.bcopies[q];
      v += restrict_partial<T>(F, C.fslot[cp.slot], cp.i, cp.j, cp.k, rf, true);
    }
  for (int q = lo; q < hi; ++q) rc[C.bcopies[q].idx] = v;
}

// u_f += P e_c on every stored node of the tets above the coarsest level.
template <class T>
__global__ void prolong_add_kernel(DepthDev F, DepthDev C, const int* __restrict__ cslot_of_fslot,
                                   const T* __restrict__ ec, T* __restrict__ uf) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < F.n_rows_nc; r += nwarps) {
    const int4 row = F.rows[r];
    const TetDev tf = F.tets[row.x];
    const TetDev tc = C.tets[cslot_of_fslot[row.x]];
    const int j = row.y, k = row.z, N = tf.N, Nc = tc.N;
    const long long fb = tf.base + node_offset(N, 0, j, k);
    for (int i = lane; i + j + k <= N; i += 32) {
      const int pi = i & 1, pj = j & 1, pk = k & 1;
      T e;
      if (!(pi | pj | pk)) {
        e = ec[tc.base + node_offset(Nc, i >> 1, j >> 1, k >> 1)];
      } else {
        // the edge direction w with w = (i,j,k) mod 2 (one of the 7 edge directions)
        int wi = pi, wj = pj, wk = pk;
        if (pi && pj && !pk) wj = -1;                 // e1-e2
        else if (pi && !pj && pk) wk = -1;            // e1-e3
        else if (!pi && pj && pk) wk = -1;            // e2-e3
        else if (pi && pj && pk) wj = -1;             // e1-e2+e3
        const int ai = (i - wi) >> 1, aj = (j - wj) >> 1, ak = (k - wk) >> 1;
        const int bi = (i + wi) >> 1, bj = (j + wj) >> 1, bk = (k + wk) >> 1;
        e = (T)0.5 * (ec[tc.base + node_offset(Nc, ai, aj, ak)] + ec[tc.base + node_offset(Nc, bi, bj, bk)]);
      }
      uf[fb + i] += e;
    }
  }
}

void restrict_residual(Mesh& m, int depth, int dtype, const void* rf, void* rc, cudaStream_t s) {
  HHG_REQUIRE(depth + 1 < m.ndepth, "no coarser depth");
  const Depth& C = m.depth[depth + 1];
  const Depth& F = m.depth[depth];
  const int g = grid_for((long long)C.n_rows * 32, 256, 8192);
  if (elem_size(dtype) == 8) {
    restrict_volume_kernel<double><<<g, 256, 0, s>>>(C.dev, F.dev, (const double*)rf, (double*)rc);
    if (C.n_bnodes)
      restrict_boundary_kernel<double><<<(C.n_bnodes + 127) / 128, 128, 0, s>>>(C.dev, F.dev, (const double*)rf,
                                                                                (double*)rc);
  } else {
    restrict_volume_kernel<float><<<g, 256, 0, s>>>(C.dev, F.dev, (const float*)rf, (float*)rc);
    if (C.n_bnodes)
      restrict_boundary_kernel<float><<<(C.n_bnodes + 127) / 128, 128, 0, s>>>(C.dev, F.dev, (const float*)rf,
                                                                               (float*)rc);
  }
  HHG_CUDA(cudaGetLastError());
}

// slot at depth+1 of each slot at depth (for prolongation); built on demand
const int* coarse_slot_map(Mesh& m, int depth) {
  Depth& F = m.depth[depth];
  if (!F.cslot_map) {
    std::vector<int> map(std::max<size_t>(F.slot_tet.size(), 1), -1);
    const Depth& C = m.depth[depth + 1];
    for (size_t s = 0; s < F.slot_tet.size(); ++s) map[s] = C.tet_slot[F.slot_tet[s]];
    F.cslot_map = static_cast<int*>(dalloc(F, map.size() * sizeof(int)));
    HHG_CUDA(cudaMemcpy(F.cslot_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  return F.cslot_map;
}

void prolongate_add(Mesh& m, int depth, int dtype, const void* ec, void* uf, cudaStream_t s) {
  HHG_REQUIRE(depth + 1 < m.ndepth, "no coarser depth");
  const Depth& F = m.depth[depth];
  const Depth& C = m.depth[depth + 1];
  const int* map = coarse_slot_map(m, depth);
  const int g = grid_for((long long)std::max(F.n_rows_nc, 1) * 32, 256, 8192);
  if (F.n_rows_nc == 0) return;
  if (elem_size(dtype) == 8)
    prolong_add_kernel<double><<<g, 256, 0, s>>>(F.dev, C.dev, map, (const double*)ec, (double*)uf);
  else
    prolong_add_kernel<float><<<g, 256, 0, s>>>(F.dev, C.dev, map, (const float*)ec, (float*)uf);
  HHG_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// deterministic FP64 reductions: fixed grid, per-block partials, the last
// block sums the partials in block order.
// ---------------------------------------------------------------------------
constexpr int kRedBlocks = 592;  // fixed (4 x 148): the summation order never changes
constexpr int kRedThreads = 256;

enum RedPost { RED_STORE = 0, RED_ALPHA = 1, RED_BETA = 2, RED_FBETA = 3 };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// finishes the reduction; slot = where the result goes in S[], post op on scalars
__device__ void block_finish(double v, double* partials, unsigned* counter, double* S, int slot, int post) {
  __shared__ double sh[kRedThreads / 32];
  __shared__ bool last;
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0;
    for (int w = 0; w < kRedThreads / 32; ++w) b += sh[w];
    partials[blockIdx.x] = b;
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double tot = 0;
    for (unsigned b = 0; b < gridDim.x; ++b) tot += ((volatile double*)partials)[b];
    S[slot] = tot;
    if (post == RED_ALPHA) {  // S[2] = alpha = rz / pq
      S[2] = S[0] / tot;
    } else if (post == RED_BETA) {  // beta = rz_new / rz; rz = rz_new
      S[5] = tot / S[0];
      S[0] = tot;
    } else if (post == RED_FBETA) {  // flexible CG: beta = (rz_new - alpha z.q) / rz, z.q in S[8]
      S[5] = (tot - S[2] * S[8]) / S[0];
      S[0] = tot;
    }
    *counter = 0;
  }
}

// sum_i x_i y_i over [0, n) minus the non-owner copies (each unique unknown once)
template <class T>
__global__ void __launch_bounds__(kRedThreads) dot_kernel(const T* __restrict__ x, const T* __restrict__ y,
                                                          long long n, const long long* __restrict__ extra,
                                                          int n_extra, double* partials, unsigned* counter,
                                                          double* S, int slot, int post) {
  double v = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
    v += (double)x[i] * (double)y[i];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_extra; e += stride) {
    const long long i = extra[e];
    v -= (double)x[i] * (double)y[i];
  }
  block_finish(v, partials, counter, S, slot, post);
}

// FP32 vectors: 16-byte loads, each group of four products summed in FP32
// (relative rounding <= 2^-22 of the group), the groups accumulated in FP64;
// x and y must be 16-byte aligned (as every vector of the library).
__global__ void __launch_bounds__(kRedThreads) dot_f32_kernel(const float* __restrict__ x, const float* __restrict__ y,
                                                              long long n, const long long* __restrict__ extra,
                                                              int n_extra, double* partials, unsigned* counter,
                                                              double* S, int slot, int post) {
  double v = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n4 = n / 4;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const float4* y4 = reinterpret_cast<const float4*>(y);
  for (long long i = tid; i < n4; i += stride) {
    const float4 a = __ldg(x4 + i), b = __ldg(y4 + i);
    v += (double)fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
  }
  for (long long i = 4 * n4 + tid; i < n; i += stride) v += (double)x[i] * (double)y[i];
  for (long long e = tid; e < n_extra; e += stride) {
    const long long i = extra[e];
    v -= (double)x[i] * (double)y[i];
  }
  block_finish(v, partials, counter, S, slot, post);
}

void dot(Mesh& m, int depth, int dtype, const void* x, const void* y, int slot, int post, bool nc_only,
         cudaStream_t s) {
  const Depth& D = m.depth[depth];
  const long long n = nc_only ? D.n_stored_nc : D.n_stored;
  const int ne = nc_only ? D.n_extra_nc : D.n_extra;
  if (elem_size(dtype) == 8)
    dot_kernel<double><<<kRedBlocks, kRedThreads, 0, s>>>((const double*)x, (const double*)y, n, D.dev.extra, ne,
                                                          m.d_red, m.d_counter, m.d_scalars, slot, post);
  else
    dot_f32_kernel<<<kRedBlocks, kRedThreads, 0, s>>>((const float*)x, (const float*)y, n, D.dev.extra, ne, m.d_red,
                                                      m.d_counter, m.d_scalars, slot, post);
  HHG_CUDA(cudaGetLastError());
}

// CG update x += alpha p, r -= alpha q (alpha = S[2] on the device)
template <class T>
__global__ void cg_update_kernel(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                 const T* __restrict__ q, long long n, const double* S) {
  const T alpha = (T)S[2];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
  }
}

// p = z + beta p
template <class T>
__global__ void xpay_kernel(T* __restrict__ p, const T* __restrict__ z, long long n, const double* S) {
  const T beta = (T)S[5];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

template <class A, class B>
__global__ void convert_kernel(const A* __restrict__ a, B* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (B)a[i];
}

// x64 += (double) d32
__global__ void add_f32_to_f64_kernel(double* __restrict__ x, const float* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

// elementwise z = a * b (FP64 accumulate in the target type)
template <class T>
__global__ void mul_kernel(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ z, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = a[i] * b[i];
}

__global__ void div_kernel(double* __restrict__ y, const double* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] /= d[i];
}

template <class T>
__global__ void scale_kernel(T* __restrict__ x, long long n, const double* S, int slot, int mode) {
  // mode 0: x *= 1/sqrt(S[slot])
  const T f = (T)(1.0 / sqrt(S[slot]));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] *= f;
}

// ---------------------------------------------------------------------------
// coarsest level: dense inverse of the re-discretised operator (host
// Cholesky, FP64), applied on the device per component.
// ---------------------------------------------------------------------------
struct DepthPtrs {
  void* f[kMaxLevel + 2];
  void* u[kMaxLevel + 2];
};

template <class T>
__global__ void coarse_apply_kernel(const double* __restrict__ cinv, const long long* __restrict__ cinv_off,
                                    const int* __restrict__ cn, const int* __restrict__ cdepth,
                                    const int* __restrict__ crep, const int* __restrict__ crep_off,
                                    const int* __restrict__ ccstart, const long long* __restrict__ ccopies,
                                    const int* __restrict__ ccopies_off, DepthPtrs P) {
  extern __shared__ double sb[];
  const int c = blockIdx.x;
  const int n = cn[c];
  const T* f = static_cast<const T*>(P.f[cdepth[c]]);
  T* u = static_cast<T*>(P.u[cdepth[c]]);
  const int* rep = crep + crep_off[c];
  for (int i = threadIdx.x; i < n; i += blockDim.x) sb[i] = (double)f[rep[i]];
  __syncthreads();
  const double* Ainv = cinv + cinv_off[c];
  const int* cs = ccstart + crep_off[c] + c;  // n+1 entries per component
  const long long* cp = ccopies + ccopies_off[c];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = 0;
    for (int j = 0; j < n; ++j) acc += Ainv[(long long)i * n + j] * sb[j];
    for (int q = cs[i]; q < cs[i + 1]; ++q) u[cp[q]] = (T)acc;
  }
}

static void host_cholesky_inverse(std::vector<double>& A, int n) {
  // A (n x n, row-major, SPD) -> A^-1 via L L^T
  std::vector<double> L(A);
  for (int j = 0; j < n; ++j) {
    double d = L[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > 0)) throw Error{HHG_ERR_ARG, "coarse operator is not positive definite"};
    d = std::sqrt(d);
    L[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = L[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = v / d;
    }
  }
  std::vector<double> X((size_t)n * n, 0.0);
  std::vector<double> y(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= L[(size_t)i * n + k] * y[k];
      y[i] = v / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double v = y[i];
      for (int k = i + 1; k < n; ++k) v -= L[(size_t)k * n + i] * X[(size_t)k * n + c];
      X[(size_t)i * n + c] = v / L[(size_t)i * n + i];
    }
  }
  A.swap(X);
}

static void coarse_by_columns(Mesh& m, std::vector<double>& all, std::vector<long long>& off, cudaStream_t s);

void ensure_coarse(Mesh& m, int dtype, cudaStream_t s) {
  if (m.cinv_ready[m.opk][dtype]) return;
  HHG_CUDA(cudaStreamSynchronize(s));
  Depth& D0 = m.depth[0];
  // index arrays (once)
  if (!m.d_cn) {
    std::vector<int> cn, cdepth, crep, crep_off, ccstart, ccopies_off;
    std::vector<long long> ccopies;
    for (auto& C : m.coarse) {
      cn.push_back(C.n);
      cdepth.push_back(C.depth);
      crep_off.push_back((int)crep.size());
      crep.insert(crep.end(), C.h_rep.begin(), C.h_rep.end());
      ccstart.insert(ccstart.end(), C.h_cstart.begin(), C.h_cstart.end());
      ccopies_off.push_back((int)ccopies.size());
      ccopies.insert(ccopies.end(), C.h_copies.begin(), C.h_copies.end());
    }
    auto up = [&](auto& v) {
      using E = typename std::decay_t<decltype(v)>::value_type;
      E* p = static_cast<E*>(dalloc(D0, std::max<size_t>(v.size(), 1) * sizeof(E)));
      if (!v.empty()) HHG_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice));
      return p;
    };
    m.d_cn = up(cn);
    m.d_cdepth = up(cdepth);
    m.d_crep = up(crep);
    m.d_crep_off = up(crep_off);
    m.d_ccstart = up(ccstart);
    m.d_ccopies = up(ccopies);
    m.d_ccopies_off = up(ccopies_off);
  }
  // assemble each component's coarse matrix with the coefficient of this dtype
  std::vector<double> all;
  std::vector<long long> off;
  if (m.opk != 0) coarse_by_columns(m, all, off, s);
  for (int c = 0; c < m.ncomp && m.opk == 0; ++c) {
    const CoarseComp& C = m.coarse[c];
    const Depth& D = m.depth[C.depth];
    std::vector<double> k(D.n_stored);
    if (dtype == HHG_F64) {
      HHG_CUDA(cudaMemcpy(k.data(), D.k64, D.n_stored * 8, cudaMemcpyDeviceToHost));
    } else if (dtype == HHG_F32) {
      std::vector<float> kf(D.n_stored);
      HHG_CUDA(cudaMemcpy(kf.data(), D.k32, D.n_stored * 4, cudaMemcpyDeviceToHost));
      for (long long i = 0; i < D.n_stored; ++i) k[i] = kf[i];
    } else {
      HHG_CUDA(cudaMemcpy(k.data(), D.k16d, D.n_stored * 8, cudaMemcpyDeviceToHost));
    }
    std::vector<int> uid(D.n_stored, -1);
    for (int u = 0; u < C.n; ++u)
      for (int q = C.h_cstart[u]; q < C.h_cstart[u + 1]; ++q) uid[C.h_copies[q]] = u;
    const int n = C.n;
    std::vector<double> A((size_t)n * n, 0.0);
    for (size_t sl = 0; sl < D.slot_tet.size(); ++sl) {
      const int t = D.slot_tet[sl];
      if (m.comp[t] != c) continue;
      const int N = D.h_tets[sl].N;
      const long long base = D.h_tets[sl].base;
      const double* st = &D.h_sten[sl * 16 * kNDir];
      for (int kk = 0; kk <= N; ++kk)
        for (int j = 0; j <= N - kk; ++j)
          for (int i = 0; i <= N - j - kk; ++i) {
            const long long x = base + node_offset(N, i, j, kk);
            const int ux = uid[x];
            if (ux < 0) continue;
            const int mask = face_mask(N, i, j, kk);
            for (int d = 0; d < kNDir; ++d) {
              int di, dj, dk;
              dir_of(d, di, dj, dk);
              const int a = i + di, b = j + dj, cc = kk + dk;
              if (a < 0 || b < 0 || cc < 0 || a + b + cc > N) continue;
              const long long y = base + node_offset(N, a, b, cc);
              double sv;
              if (dtype == HHG_F32) {  // the FP32 kernels' arithmetic on FP32 data
                sv = (double)((float)st[mask * kNDir + d] * ((float)k[x] + (float)k[y]));
              } else {
                sv = st[mask * kNDir + d] * (k[x] + k[y]);
              }
              const int uy = uid[y];
              if (uy >= 0) A[(size_t)ux * n + uy] += sv;
              A[(size_t)ux * n + ux] -= sv;
            }
          }
    }
    // the scaled operator is symmetric; symmetrise rounding noise before Cholesky
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) {
        const double v = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
        A[(size_t)i * n + j] = A[(size_t)j * n + i] = v;
      }
    host_cholesky_inverse(A, n);
    off.push_back((long long)all.size());
    all.insert(all.end(), A.begin(), A.end());
  }
  double*& cinv = m.d_cinv[m.opk][dtype];
  if (!cinv) cinv = static_cast<double*>(dalloc(D0, std::max<size_t>(all.size(), 1) * 8));
  HHG_CUDA(cudaMemcpy(cinv, all.data(), all.size() * 8, cudaMemcpyHostToDevice));
  if (!m.d_cinv_off) m.d_cinv_off = static_cast<long long*>(dalloc(D0, std::max<size_t>(off.size(), 1) * 8));
  HHG_CUDA(cudaMemcpy(m.d_cinv_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice));
  m.cinv_ready[m.opk][dtype] = true;
}

// u = A_c^-1 f for every component at its coarse depth; f, u given per depth.
// ensure_coarse() must have run (it synchronises); this only enqueues work.
void coarse_solve(Mesh& m, int dtype, void* const* fdepth, void* const* udepth, cudaStream_t s) {
  const int kd = dtype == kF64KBF16 ? (int)HHG_F32_KBF16 : dtype;
  HHG_REQUIRE(m.cinv_ready[m.opk][kd], "internal: coarse inverse not prepared");
  DepthPtrs P{};
  for (int d = 0; d < m.ndepth; ++d) {
    P.f[d] = fdepth[d];
    P.u[d] = udepth[d];
  }
  int maxn = 1;
  for (auto& C : m.coarse) maxn = std::max(maxn, C.n);
  const size_t shm = (size_t)maxn * 8;
  if (elem_size(dtype) == 8) {
    if (shm > 48 * 1024)
      HHG_CUDA(cudaFuncSetAttribute(coarse_apply_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    coarse_apply_kernel<double><<<m.ncomp, 256, shm, s>>>(m.d_cinv[m.opk][kd], m.d_cinv_off, m.d_cn, m.d_cdepth, m.d_crep,
                                                         m.d_crep_off, m.d_ccstart, m.d_ccopies, m.d_ccopies_off, P);
  } else {
    if (shm > 48 * 1024)
      HHG_CUDA(cudaFuncSetAttribute(coarse_apply_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    coarse_apply_kernel<float><<<m.ncomp, 256, shm, s>>>(m.d_cinv[m.opk][kd], m.d_cinv_off, m.d_cn, m.d_cdepth, m.d_crep,
                                                        m.d_crep_off, m.d_ccstart, m.d_ccopies, m.d_ccopies_off, P);
  }
  HHG_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// operator helpers
// ---------------------------------------------------------------------------
// 1/diag of the nodal operator at a depth (computed once per coefficient)
const void* nodal_dinv(Mesh& m, int depth, int dtype, cudaStream_t s) {
  Depth& D = m.depth[depth];
  if (!D.ndinv[dtype]) {
    void* p = workspace(m, depth, prec_of(dtype), 11);
    for (int t = 0; t < 4; ++t)  // dtypes of one precision share the buffer
      if (prec_of(t) == prec_of(dtype)) D.ndinv[t] = nullptr;
    launch_nodal_dinv(m, depth, dtype, p, s);
    D.ndinv[dtype] = p;
  }
  return D.ndinv[dtype];
}

// one operator launch in the given mode, with the operator of m.opk
static void op(Mesh& m, int depth, int dtype, OpMode mode, const void* u, const void* f, void* out, const void* din,
               void* dout, double omega, double ca, double cb, bool nc_only, cudaStream_t s) {
  OpArgs a{u, f, out, din, dout, omega, ca, cb, nc_only ? 1 : 0};
  if (m.opk == 3)
    launch_tensor_op(m, depth, dtype, mode, a, s);
  else if (m.opk == 1)
    launch_volface_op(m, depth, dtype, mode, a, s);
  else if (m.opk == 2)
    launch_nodal_op(m, depth, dtype, mode, a, nodal_dinv(m, depth, dtype, s), workspace(m, depth, prec_of(dtype), 10),
                    s);
  else
    launch_scaled_op(m, depth, dtype, mode, a, s);
}

// Coarse matrices of a non-scaled operator, column by column: the operator
// applied (FP64, on the GPU) to the unit vector of each coarse unknown, then
// inverted by Gauss-Jordan elimination with partial pivoting (the Vol+Face
// operator is not symmetric).
static void coarse_by_columns(Mesh& m, std::vector<double>& all, std::vector<long long>& off, cudaStream_t s) {
  for (int c = 0; c < m.ncomp; ++c) {
    const CoarseComp& C = m.coarse[c];
    const int d = C.depth;
    const long long ns = m.depth[d].n_stored;
    const int n = C.n;
    double* e = static_cast<double*>(workspace(m, d, 0, 9));
    double* y = static_cast<double*>(workspace(m, d, 0, 10));
    std::vector<double> A((size_t)n * n, 0.0), eh(ns, 0.0), yh(ns);
    for (int u = 0; u < n; ++u) {
      for (int q = C.h_cstart[u]; q < C.h_cstart[u + 1]; ++q) eh[C.h_copies[q]] = 1.0;
      HHG_CUDA(cudaMemcpyAsync(e, eh.data(), ns * 8, cudaMemcpyHostToDevice, s));
      op(m, d, HHG_F64, OP_APPLY, e, nullptr, y, nullptr, nullptr, 0, 0, 0, false, s);
      HHG_CUDA(cudaMemcpyAsync(yh.data(), y, ns * 8, cudaMemcpyDeviceToHost, s));
      HHG_CUDA(cudaStreamSynchronize(s));
      for (int v = 0; v < n; ++v) A[(size_t)v * n + u] = yh[C.h_rep[v]];
      for (int q = C.h_cstart[u]; q < C.h_cstart[u + 1]; ++q) eh[C.h_copies[q]] = 0.0;
    }
    // Gauss-Jordan with partial pivoting: A <- A^-1
    std::vector<double> I((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
    for (int col = 0; col < n; ++col) {
      int piv = col;
      for (int r = col + 1; r < n; ++r)
        if (std::fabs(A[(size_t)r * n + col]) > std::fabs(A[(size_t)piv * n + col])) piv = r;
      HHG_REQUIRE(A[(size_t)piv * n + col] != 0.0, "singular coarse matrix");
      if (piv != col)
        for (int j = 0; j < n; ++j) {
          std::swap(A[(size_t)piv * n + j], A[(size_t)col * n + j]);
          std::swap(I[(size_t)piv * n + j], I[(size_t)col * n + j]);
        }
      const double inv = 1.0 / A[(size_t)col * n + col];
      for (int j = 0; j < n; ++j) {
        A[(size_t)col * n + j] *= inv;
        I[(size_t)col * n + j] *= inv;
      }
      for (int r = 0; r < n; ++r) {
        if (r == col) continue;
        const double fct = A[(size_t)r * n + col];
        if (fct == 0.0) continue;
        for (int j = 0; j < n; ++j) {
          A[(size_t)r * n + j] -= fct * A[(size_t)col * n + j];
          I[(size_t)r * n + j] -= fct * I[(size_t)col * n + j];
        }
      }
    }
    off.push_back((long long)all.size());
    all.insert(all.end(), I.begin(), I.end());
  }
}

void apply_scaled(Mesh& m, int depth, int dtype, const void* u, void* y, cudaStream_t s) {
  op(m, depth, dtype, OP_APPLY, u, nullptr, y, nullptr, nullptr, 0, 0, 0, false, s);
}

void residual(Mesh& m, int depth, int dtype, const void* f, const void* u, void* r, bool nc_only, cudaStream_t s) {
  op(m, depth, dtype, OP_RESID, u, f, r, nullptr, nullptr, 0, 0, 0, nc_only, s);
}

static void copy_vec(Mesh& m, int depth, int dtype, const void* src, void* dst, bool nc_only, cudaStream_t s) {
  const Depth& D = m.depth[depth];
  const long long n = nc_only ? D.n_stored_nc : D.n_stored;
  if (n > 0 && src != dst) HHG_CUDA(cudaMemcpyAsync(dst, src, n * elem_size(dtype), cudaMemcpyDeviceToDevice, s));
}

double lambda_max(Mesh& m, int depth, int its, cudaStream_t s);

// Smoothing in place on u (workspace slots 4, 5 and 6 of the depth).
// post = false: sweeps run Jacobi, learned, Jacobi, ...; post = true: learned,
// Jacobi, ... (HHG_SMOOTH_LEARNED only)
void smooth(Mesh& m, int depth, int dtype, int kind, int sweeps, double omega, const void* f, void* u, bool nc_only,
            cudaStream_t s, bool post) {
  const int pr = prec_of(dtype);
  void* w = workspace(m, depth, pr, 4);
  if (kind == HHG_SMOOTH_LEARNED) {
    void* a = u;
    void* b = w;
    for (int it = 0; it < sweeps; ++it) {
      if ((it % 2 == 0) == post)
        learned_step(m, depth, dtype, f, a, b, nc_only, s);
      else
        op(m, depth, dtype, OP_JACOBI, a, f, b, nullptr, nullptr, omega, 0, 0, nc_only, s);
      std::swap(a, b);
    }
    if (a != u) copy_vec(m, depth, dtype, a, u, nc_only, s);
    return;
  }
  if (kind == HHG_SMOOTH_JACOBI) {
    void* a = u;
    void* b = w;
    for (int it = 0; it < sweeps; ++it) {
      op(m, depth, dtype, OP_JACOBI, a, f, b, nullptr, nullptr, omega, 0, 0, nc_only, s);
      std::swap(a, b);
    }
    if (a != u) copy_vec(m, depth, dtype, a, u, nc_only, s);
    return;
  }
  HHG_REQUIRE(kind == HHG_SMOOTH_CHEBYSHEV, "unknown smoother");
  const double lam = lambda_max(m, depth, m.power_its, s);
  const double lo = m.cheb_lo * lam, hi = m.cheb_hi * lam;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  void* d0 = workspace(m, depth, pr, 5);
  void* d1 = workspace(m, depth, pr, 6);
  void* a = u;
  void* b = w;
  for (int sw = 0; sw < sweeps; ++sw) {
    double rho = 1.0 / sigma;
    // first step: d = D^-1 r / theta
    op(m, depth, dtype, OP_CHEB, a, f, b, d1, d0, 0, 0.0, 1.0 / theta, nc_only, s);
    std::swap(a, b);
    void* dc = d0;
    void* dn = d1;
    for (int q = 1; q < m.cheb_degree; ++q) {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      op(m, depth, dtype, OP_CHEB, a, f, b, dc, dn, 0, rho_new * rho, 2.0 * rho_new / delta, nc_only, s);
      std::swap(a, b);
      std::swap(dc, dn);
      rho = rho_new;
    }
  }
  if (a != u) copy_vec(m, depth, dtype, a, u, nc_only, s);
}

// start vector of the power iteration: cos(pi N (x+y+z)) + 1/4 at unknowns
__global__ void power_start_kernel(DepthDev D, const double* __restrict__ V, const int* __restrict__ T, double* x) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < D.n_rows; r += nwarps) {
    const int4 row = D.rows[r];
    const TetDev td = D.tets[row.x];
    const int* g = T + 4 * td.tet;
    const int N = td.N, j = row.y, k = row.z;
    for (int i = lane; i + j + k <= N; i += 32) {
      // coordinates from the macro vertices in increasing id order
      int gs[4] = {g[0], g[1], g[2], g[3]};
      int ws[4] = {N - i - j - k, i, j, k};
      for (int a = 1; a < 4; ++a)
        for (int b = a; b > 0 && (gs[b] < gs[b - 1]); --b) {
          int t = gs[b]; gs[b] = gs[b - 1]; gs[b - 1] = t;
          t = ws[b]; ws[b] = ws[b - 1]; ws[b - 1] = t;
        }
      double sxyz = 0;
      for (int c = 0; c < 3; ++c) {
        double xc = 0;
        for (int a = 0; a < 4; ++a)
          if (ws[a]) xc += ((double)ws[a] / N) * V[3 * gs[a] + c];
        sxyz += xc;
      }
      x[td.base + node_offset(N, i, j, k)] = cos(3.14159265358979323846 * N * sxyz) + 0.25;
    }
  }
}

__global__ void zero_dirichlet_kernel(DepthDev D, double* x) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= D.n_bnodes || !D.bdir[b]) return;
  for (int q = D.bstart[b]; q < D.bstart[b + 1]; ++q) x[D.bcopies[q].idx] = 0.0;
}

// Power iteration on D^-1 A (FP64): x <- y / |y|, y = D^-1 A x; the estimate is
// the Rayleigh quotient (x.Ax)/(x.Dx) of the last iterate.
double lambda_max(Mesh& m, int depth, int its, cudaStream_t s) {
  Depth& D = m.depth[depth];
  if (D.lam > 0) return D.lam;
  double* x = static_cast<double*>(workspace(m, depth, 0, 0));
  double* y = static_cast<double*>(workspace(m, depth, 0, 1));
  double* t = static_cast<double*>(workspace(m, depth, 0, 2));
  double* dg = static_cast<double*>(workspace(m, depth, 0, 3));
  // macro geometry on the device (small)
  Depth& D0 = m.depth[0];
  if (!m.d_geom) {
    m.d_geom = static_cast<double*>(dalloc(D0, m.V.size() * 8 + m.T.size() * 4 + 64));
    HHG_CUDA(cudaMemcpy(m.d_geom, m.V.data(), m.V.size() * 8, cudaMemcpyHostToDevice));
    HHG_CUDA(cudaMemcpy(reinterpret_cast<char*>(m.d_geom) + m.V.size() * 8, m.T.data(), m.T.size() * 4,
                        cudaMemcpyHostToDevice));
  }
  const double* dV = m.d_geom;
  const int* dT = reinterpret_cast<const int*>(reinterpret_cast<const char*>(m.d_geom) + m.V.size() * 8);
  const int g = grid_for((long long)D.n_rows * 32, 256, 8192);
  power_start_kernel<<<g, 256, 0, s>>>(D.dev, dV, dT, x);
  if (D.n_bnodes) zero_dirichlet_kernel<<<(D.n_bnodes + 127) / 128, 128, 0, s>>>(D.dev, x);
  HHG_CUDA(cudaGetLastError());
  // diagonal (1 at Dirichlet nodes, where x = 0)
  op(m, depth, HHG_F64, OP_DIAG, x, nullptr, dg, nullptr, nullptr, 0, 0, 0, false, s);
  const long long n = D.n_stored;
  const int gv = grid_for(n, 256, 4096);
  for (int it = 0; it < its; ++it) {
    apply_scaled(m, depth, HHG_F64, x, y, s);  // y = A x
    div_kernel<<<gv, 256, 0, s>>>(y, dg, n);     // y = D^-1 A x
    dot(m, depth, HHG_F64, y, y, 10, RED_STORE, false, s);
    std::swap(x, y);
    scale_kernel<double><<<gv, 256, 0, s>>>(x, n, m.d_scalars, 10, 0);
  }
  apply_scaled(m, depth, HHG_F64, x, y, s);
  dot(m, depth, HHG_F64, x, y, 11, RED_STORE, false, s);
  mul_kernel<double><<<gv, 256, 0, s>>>(dg, x, t, n);
  dot(m, depth, HHG_F64, x, t, 12, RED_STORE, false, s);
  HHG_CUDA(cudaMemcpyAsync(m.h_pinned, m.d_scalars + 11, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  HHG_CUDA(cudaStreamSynchronize(s));
  D.lam = m.h_pinned[0] / m.h_pinned[1];
  return D.lam;
}

// ---------------------------------------------------------------------------
// V-cycle (depth-aligned: depth d holds every tet at level_t - d; a component
// reaching the coarsest level is solved directly)
// ---------------------------------------------------------------------------
void vcycle(Mesh& m, int dtype, int nu1, int nu2, int smoother, double omega, const void* f0, void* u0,
            cudaStream_t s) {
  const int pr = prec_of(dtype);
  const int nd = m.ndepth;
  std::vector<void*> F(nd), U(nd);
  F[0] = const_cast<void*>(f0);
  U[0] = u0;
  for (int d = 1; d < nd; ++d) {
    F[d] = workspace(m, d, pr, 0);
    U[d] = workspace(m, d, pr, 1);
  }
  if (smoother == HHG_SMOOTH_CHEBYSHEV)
    for (int d = 0; d < nd; ++d)
      if (m.depth[d].n_slots_nc) lambda_max(m, d, m.power_its, s);
  for (int d = 0; d + 1 < nd; ++d) {
    const Depth& D = m.depth[d];
    if (!D.n_slots_nc) continue;
    void* r = workspace(m, d, pr, 2);
    smooth(m, d, dtype, smoother, nu1, omega, F[d], U[d], true, s, false);
    residual(m, d, dtype, F[d], U[d], r, true, s);
    restrict_residual(m, d, dtype, r, F[d + 1], s);
    HHG_CUDA(cudaMemsetAsync(U[d + 1], 0, m.depth[d + 1].n_stored * elem_size(dtype), s));
  }
  coarse_solve(m, dtype, F.data(), U.data(), s);
  for (int d = nd - 2; d >= 0; --d) {
    const Depth& D = m.depth[d];
    if (!D.n_slots_nc) continue;
    prolongate_add(m, d, dtype, U[d + 1], U[d], s);
    smooth(m, d, dtype, smoother, nu2, omega, F[d], U[d], true, s, true);
  }
}

}  // namespace hhg
