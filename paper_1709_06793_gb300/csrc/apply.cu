// Operator kernels: the stencil-scaled apply (Sec. 6.1) fused with residual,
// damped Jacobi and Chebyshev updates, and the nodal-integration apply
// (eq. "onTheFlyStencil", Sec. 6.2).
//
// Scaled operator, row of node x:
//     (A u)_x = sum_{d} c_d^{prim(x)} (k_x + k_{x+w_d}) (u_{x+w_d} - u_x)
// with c = (1/2) reference stencil of x's primitive (the factor 1/2 folded in
// at setup, Sec. 6.1) and the diagonal -sum_d c_d (k_x + k_{x+w_d}) implied by
// the zero row sum.  Written per edge (x, x+w): the flux
//     F = c_w (k_x + k_{x+w}) (u_{x+w} - u_x)
// enters row x with + and row x+w with - (c is symmetric on the volume).
//
// Volume kernel (nodes strictly inside a macro tet).  A warp owns 4 tiles of
// 8 consecutive i x 4 rows j; lane (g, l) owns column i = i0_g + l, rows
// j0_g .. j0_g+3, and marches along k.  When plane q arrives it computes every
// edge between planes q-1 and q and every edge inside plane q that touches its
// nodes; after that the rows of plane q-1 are complete and are written.  Only
// two planes of u and k live in registers; the neighbour columns i-1, i+1 are
// loaded directly (L1 hits: the 8 lanes of a tile read contiguous memory).
// Tiles of one warp share i0+j0 (anti-diagonal), so all 4 march equally far.
#include "hhg_internal.h"

namespace hhg {

template <class T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};

__device__ __forceinline__ float ldk(const float* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ double ldk(const double* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ float ldk(const __nv_bfloat16* p, long long i) { return __bfloat162float(__ldg(p + i)); }

// (u_b - u_a, k_b + k_a) in one packed FMA for fp32.
__device__ __forceinline__ float2 diffsum(float2 a, float2 b) { return __ffma2_rn(a, make_float2(-1.f, 1.f), b); }
__device__ __forceinline__ double2 diffsum(double2 a, double2 b) { return make_double2(b.x - a.x, b.y + a.y); }

template <class T, bool DIAG>
struct Acc {
  T y = 0;
  T d = 0;
};

// Edge contribution to row a only.
template <class T, bool DIAG, class P2>
__device__ __forceinline__ void edge1(P2 a, P2 b, T c, Acc<T, DIAG>& A) {
  const P2 t = diffsum(a, b);
  const T s = c * t.y;
  A.y = fma(s, t.x, A.y);
  if (DIAG) A.d -= s;
}
// Edge contribution to rows a (+F) and b (-F).
template <class T, bool DIAG, class P2>
__device__ __forceinline__ void edge2(P2 a, P2 b, T c, Acc<T, DIAG>& A, Acc<T, DIAG>& B) {
  const P2 t = diffsum(a, b);
  const T s = c * t.y;
  A.y = fma(s, t.x, A.y);
  B.y = fma(-s, t.x, B.y);
  if (DIAG) {
    A.d -= s;
    B.d -= s;
  }
}

// Register state of one plane of a lane's column footprint: rows m = 0..kTJ+1
// (j = j0-1+m) at column offsets 0, +1 (m = 0..kTJ) and -1 (m = 1..kTJ+1).
template <class T>
struct Plane {
  typename Pair<T>::type c0[kTJ + 2];
  typename Pair<T>::type cp[kTJ + 1];
  typename Pair<T>::type cm[kTJ + 2];
};

struct OpPtrs {
  const void* u;
  const void* k;
  const void* f;
  void* out;
  const void* d_in;
  void* d_out;
  double omega, ca, cb;
};

template <class T, int MODE>
__device__ __forceinline__ void finish_node(T y, T diag, T ux, long long idx, const OpPtrs& p) {
  if (MODE == OP_APPLY) {
    static_cast<T*>(p.out)[idx] = y;
  } else if (MODE == OP_RESID) {
    static_cast<T*>(p.out)[idx] = __ldg(static_cast<const T*>(p.f) + idx) - y;
  } else if (MODE == OP_JACOBI) {
    const T r = __ldg(static_cast<const T*>(p.f) + idx) - y;
    static_cast<T*>(p.out)[idx] = ux + (T)p.omega * r / diag;
  } else if (MODE == OP_CHEB) {
    const T r = __ldg(static_cast<const T*>(p.f) + idx) - y;
    const T prev = p.ca != 0.0 ? (T)p.ca * __ldg(static_cast<const T*>(p.d_in) + idx) : (T)0;
    const T dn = prev + (T)p.cb * r / diag;
    static_cast<T*>(p.d_out)[idx] = dn;
    static_cast<T*>(p.out)[idx] = ux + dn;
  } else {  // OP_DIAG
    static_cast<T*>(p.out)[idx] = diag;
  }
}

template <class T, class KT>
__device__ __forceinline__ void load_plane(Plane<T>& Q, const T* __restrict__ u, const KT* __restrict__ k,
                                           int idx0, int A, int s) {
  using P2 = typename Pair<T>::type;
#pragma unroll
  for (int m = 0; m < kTJ + 2; ++m) {
    const int row = idx0 + m * A - m * (m - 1) / 2;  // (i, j0-1+m, q)
    if (m <= s) Q.c0[m] = P2{u[row], ldk(k, row)};
    if (m <= kTJ && m + 1 <= s) Q.cp[m] = P2{u[row + 1], ldk(k, row + 1)};
    if (m >= 1 && m - 1 <= s) Q.cm[m] = P2{u[row - 1], ldk(k, row - 1)};
  }
}

// One march step: plane P (q-1) is complete in registers, plane Q (q) was
// just loaded.  Adds all edges P-Q touching the lane's nodes and all in-plane
// edges of Q; yP (rows of plane q-1) becomes final, yQ gets its first part.
template <class T, bool DIAG>
__device__ __forceinline__ void step_edges(const Plane<T>& P, const Plane<T>& Q, const T (&c)[7],
                                           Acc<T, DIAG> (&yP)[kTJ], Acc<T, DIAG> (&yQ)[kTJ]) {
  const T c1 = c[0], c2 = c[1], c3 = c[2], c12 = c[3], c13 = c[4], c23 = c[5], cg = c[6];
#pragma unroll
  for (int r = 0; r < kTJ; ++r) yQ[r] = Acc<T, DIAG>{};
  // (A) edges between planes q-1 and q
#pragma unroll
  for (int r = 0; r < kTJ; ++r) {
    const int m = r + 1;
    edge2(P.c0[m], Q.c0[m], c3, yP[r], yQ[r]);  // +e3
    edge1(P.c0[m], Q.cm[m], c13, yP[r]);        // -(e1-e3)
    if (r >= 1)
      edge2(P.c0[m], Q.c0[m - 1], c23, yP[r], yQ[r - 1]);  // -(e2-e3)
    else
      edge1(P.c0[m], Q.c0[m - 1], c23, yP[r]);
    edge1(P.c0[m], Q.cp[m - 1], cg, yP[r]);  // e1-e2+e3
  }
#pragma unroll
  for (int r = 0; r < kTJ; ++r) {
    const int m = r + 1;
    edge1(Q.c0[m], P.cp[m], c13, yQ[r]);                  // e1-e3
    if (r == kTJ - 1) edge1(Q.c0[m], P.c0[m + 1], c23, yQ[r]);  // e2-e3
    edge1(Q.c0[m], P.cm[m + 1], cg, yQ[r]);               // -(e1-e2+e3)
  }
  // (B) edges inside plane q
#pragma unroll
  for (int r = 0; r < kTJ; ++r) {
    const int m = r + 1;
    edge1(Q.c0[m], Q.cp[m], c1, yQ[r]);  // +e1
    edge1(Q.c0[m], Q.cm[m], c1, yQ[r]);  // -e1
    if (r + 1 < kTJ)
      edge2(Q.c0[m], Q.c0[m + 1], c2, yQ[r], yQ[r + 1]);  // +e2
    else
      edge1(Q.c0[m], Q.c0[m + 1], c2, yQ[r]);
    if (r == 0) edge1(Q.c0[m], Q.c0[m - 1], c2, yQ[r]);  // -e2
    edge1(Q.c0[m], Q.cp[m - 1], c12, yQ[r]);             // e1-e2
    edge1(Q.c0[m], Q.cm[m + 1], c12, yQ[r]);             // -(e1-e2)
  }
}

template <class T, class KT, int MODE>
__device__ void volume_item(const DepthDev& D, const T* __restrict__ sten, uint4 item, int lane, const OpPtrs& p) {
  constexpr bool DIAG = (MODE == OP_JACOBI || MODE == OP_CHEB || MODE == OP_DIAG);
  const int g = lane >> 3, l = lane & 7;
  const unsigned tile = g == 0 ? item.x : (g == 1 ? item.y : (g == 2 ? item.z : item.w));
  const int slot = (int)(item.x >> 20);
  const int j0 = (int)((tile >> 10) & 1023u), i0 = (int)(tile & 1023u);
  const TetDev td = D.tets[slot];
  const int N = td.N;
  const int i = i0 + l;
  // the warp marches until the tile with the smallest i0+j0 is done
  int hmin = 2047;
  hmin = min(hmin, (int)((item.x >> 10) & 1023u) + (int)(item.x & 1023u));
  hmin = min(hmin, (int)((item.y >> 10) & 1023u) + (int)(item.y & 1023u));
  hmin = min(hmin, (int)((item.z >> 10) & 1023u) + (int)(item.z & 1023u));
  hmin = min(hmin, (int)((item.w >> 10) & 1023u) + (int)(item.w & 1023u));
  const int qend = N - hmin;
  T c[7];
#pragma unroll
  for (int d = 0; d < 7; ++d) c[d] = sten[slot * 16 * kNDir + d];  // volume row (mask 0)
  const T* u = static_cast<const T*>(p.u) + td.base;
  const KT* k = static_cast<const KT*>(p.k) + td.base;
  OpPtrs q = p;
  q.out = static_cast<T*>(p.out) + td.base;
  if (MODE != OP_APPLY) q.f = static_cast<const T*>(p.f) + td.base;
  if (MODE == OP_CHEB) {
    q.d_in = static_cast<const T*>(p.d_in) + td.base;
    q.d_out = static_cast<T*>(p.d_out) + td.base;
  }
  // plane 0
  int Psz = (N + 1) * (N + 2) / 2;                          // nodes in plane q
  int A = N - j0 + 2;                                        // length of row j0-1 in plane q
  int idx0 = (j0 - 1) * (N + 1) - (j0 - 1) * (j0 - 2) / 2 + i;  // (i, j0-1, q)
  int s = N - i - j0 + 1;                                    // valid iff c + m <= s
  Plane<T> PA, PB;
#pragma unroll
  for (int m = 0; m < kTJ + 2; ++m) {
    PA.c0[m] = PB.c0[m] = {0, 0};
    PA.cm[m] = PB.cm[m] = {0, 0};
  }
#pragma unroll
  for (int m = 0; m < kTJ + 1; ++m) PA.cp[m] = PB.cp[m] = {0, 0};
  load_plane<T, KT>(PA, u, k, idx0, A, s);
  Acc<T, DIAG> yA[kTJ], yB[kTJ];
  int prev_idx0 = idx0, prev_A = A;
  auto advance = [&](int qn) {  // move the plane state from qn-1 to qn
    prev_idx0 = idx0;
    prev_A = A;
    idx0 += Psz - (j0 - 1);
    Psz -= N - qn + 2;
    A -= 1;
    s -= 1;
  };
  auto store = [&](const Plane<T>& P, Acc<T, DIAG>(&y)[kTJ], int pl) {
    if (pl < 1) return;
#pragma unroll
    for (int r = 0; r < kTJ; ++r) {
      if (i + j0 + r + pl <= N - 1) {
        const int m = r + 1;
        const long long idx = prev_idx0 + m * prev_A - m * (m - 1) / 2;
        finish_node<T, MODE>(y[r].y, y[r].d, P.c0[m].x, idx, q);
      }
    }
  };
  for (int qq = 1; qq <= qend; qq += 2) {
    advance(qq);
    load_plane<T, KT>(PB, u, k, idx0, A, s);
    step_edges<T, DIAG>(PA, PB, c, yA, yB);
    store(PA, yA, qq - 1);
    if (qq + 1 > qend) break;
    advance(qq + 1);
    load_plane<T, KT>(PA, u, k, idx0, A, s);
    step_edges<T, DIAG>(PB, PA, c, yB, yA);
    store(PB, yB, qq);
  }
}

// Partial row of one stored copy (its tet's micro-elements only).
template <class T, class KT>
__device__ __forceinline__ void scaled_partial(const DepthDev& D, const T* __restrict__ sten, const BCopy& cp,
                                               const T* __restrict__ u, const KT* __restrict__ k, T& y, T& diag) {
  const TetDev td = D.tets[cp.slot];
  const int N = td.N;
  const T* st = sten + (cp.slot * 16 + cp.mask) * kNDir;
  const T ux = u[cp.idx];
  const T kx = ldk(k, cp.idx);
#pragma unroll
  for (int d = 0; d < kNDir; ++d) {
    int di, dj, dk;
    dir_of(d, di, dj, dk);
    const int a = cp.i + di, b = cp.j + dj, cc = cp.k + dk;
    if (a < 0 || b < 0 || cc < 0 || a + b + cc > N) continue;
    const long long idx = td.base + node_offset(N, a, b, cc);
    const T sv = st[d] * (kx + (T)ldk(k, idx));
    y = fma(sv, u[idx] - ux, y);
    diag -= sv;
  }
}

template <class T, class KT, int MODE>
__device__ void boundary_node(const DepthDev& D, const T* __restrict__ sten, int b, const OpPtrs& p) {
  const int lo = D.bstart[b], hi = D.bstart[b + 1];
  T* out = static_cast<T*>(p.out);
  if (D.bdir[b]) {
    for (int q = lo; q < hi; ++q) {
      const long long idx = D.bcopies[q].idx;
      out[idx] = MODE == OP_DIAG ? (T)1 : (T)0;
      if (MODE == OP_CHEB) static_cast<T*>(p.d_out)[idx] = 0;
    }
    return;
  }
  const T* u = static_cast<const T*>(p.u);
  const KT* k = static_cast<const KT*>(p.k);
  T y = 0, diag = 0;
  for (int q = lo; q < hi; ++q) {
    const BCopy cp = D.bcopies[q];
    scaled_partial<T, KT>(D, sten, cp, u, k, y, diag);
  }
  const long long i0 = D.bcopies[lo].idx;
  const T ux = u[i0];
  T val = y, dval = 0;
  if (MODE == OP_RESID) {
    val = __ldg(static_cast<const T*>(p.f) + i0) - y;
  } else if (MODE == OP_JACOBI) {
    val = ux + (T)p.omega * (__ldg(static_cast<const T*>(p.f) + i0) - y) / diag;
  } else if (MODE == OP_CHEB) {
    const T prev = p.ca != 0.0 ? (T)p.ca * __ldg(static_cast<const T*>(p.d_in) + i0) : (T)0;
    dval = prev + (T)p.cb * (__ldg(static_cast<const T*>(p.f) + i0) - y) / diag;
    val = ux + dval;
  } else if (MODE == OP_DIAG) {
    val = diag;
  }
  for (int q = lo; q < hi; ++q) {
    const long long idx = D.bcopies[q].idx;
    out[idx] = val;
    if (MODE == OP_CHEB) static_cast<T*>(p.d_out)[idx] = dval;
  }
}

// Persistent kernel: warps take volume items (longest first), then chunks of
// 32 interface nodes.
template <class T, class KT, int MODE>
__global__ void __launch_bounds__(128) scaled_op_kernel(DepthDev D, OpPtrs p, int n_items, int n_bnodes) {
  const T* sten = nullptr;
  if constexpr (sizeof(T) == 8)
    sten = reinterpret_cast<const T*>(D.sten64);
  else
    sten = reinterpret_cast<const T*>(D.sten32);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int nchunks = (n_bnodes + 31) / 32;
  for (int it = warp; it < n_items + nchunks; it += nwarps) {
    if (it < n_items) {
      volume_item<T, KT, MODE>(D, sten, D.items[it], lane, p);
    } else {
      const int b = (it - n_items) * 32 + lane;
      if (b < n_bnodes) boundary_node<T, KT, MODE>(D, sten, b, p);
    }
  }
}

template <class T, class KT, int MODE>
static int occupancy() {
  static int occ = 0;
  if (!occ) {
    HHG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, scaled_op_kernel<T, KT, MODE>, 128, 0));
    if (occ < 1) occ = 1;
  }
  return occ;
}

template <class T, class KT>
static void init_typed() {
  occupancy<T, KT, OP_APPLY>();
  occupancy<T, KT, OP_RESID>();
  occupancy<T, KT, OP_JACOBI>();
  occupancy<T, KT, OP_CHEB>();
  occupancy<T, KT, OP_DIAG>();
}

// Launch configurations are computed once, outside any stream capture.
void init_launch_configs(int dtype) {
  if (dtype == HHG_F64 || dtype == kF64KBF16)
    init_typed<double, double>();
  else if (dtype == HHG_F32)
    init_typed<float, float>();
  else
    init_typed<float, __nv_bfloat16>();
}

template <class T, class KT, int MODE>
static void launch_typed(const Mesh& m, int depth, const OpArgs& a, const void* kptr, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  const DepthDev& D = Dh.dev;
  const int n_items = a.nc_only ? D.n_items_nc : D.n_items;
  const int n_b = a.nc_only ? D.n_bnodes_nc : D.n_bnodes;
  const int work = n_items + (n_b + 31) / 32;
  if (work == 0) return;
  const int occ = occupancy<T, KT, MODE>();
  const int blocks = std::min((work + 3) / 4, m.num_sms * occ);
  OpPtrs p{a.u, kptr, a.f, a.out, a.d_in, a.d_out, a.omega, a.ca, a.cb};
  scaled_op_kernel<T, KT, MODE><<<blocks, 128, 0, s>>>(D, p, n_items, n_b);
  HHG_CUDA(cudaGetLastError());
}

template <int MODE>
static void launch_mode(const Mesh& m, int depth, int dtype, const OpArgs& a, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  if (dtype == HHG_F64)
    launch_typed<double, double, MODE>(m, depth, a, Dh.k64, s);
  else if (dtype == kF64KBF16)
    launch_typed<double, double, MODE>(m, depth, a, Dh.k16d, s);
  else if (dtype == HHG_F32)
    launch_typed<float, float, MODE>(m, depth, a, Dh.k32, s);
  else
    launch_typed<float, __nv_bfloat16, MODE>(m, depth, a, Dh.k16, s);
}

void launch_scaled_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, cudaStream_t s) {
  switch (mode) {
    case OP_APPLY: launch_mode<OP_APPLY>(m, depth, dtype, a, s); break;
    case OP_RESID: launch_mode<OP_RESID>(m, depth, dtype, a, s); break;
    case OP_JACOBI: launch_mode<OP_JACOBI>(m, depth, dtype, a, s); break;
    case OP_CHEB: launch_mode<OP_CHEB>(m, depth, dtype, a, s); break;
    case OP_DIAG: launch_mode<OP_DIAG>(m, depth, dtype, a, s); break;
  }
}

// ---------------------------------------------------------------------------
// Nodal-integration apply (eq. "standardfe"): y_x = sum over the micro tets t
// at x of kbar_t * sum_w A_t[x][w] (u_w - u_x), kbar_t = (1/4) sum of k at the
// 4 vertices (the 1/4 is folded into the stored element matrices).  The 24
// micro tets at a node are the Freudenthal simplices of the 8 unit cubes at
// the node (Kuhn coordinates (i+j+k, j+k, k)) whose path passes the node.
// ---------------------------------------------------------------------------
struct NodalEntry {
  int sigma, v;
  int off[4][3];  // index-space offsets of the 4 vertices relative to the node
};
struct NodalTable {
  NodalEntry e[24];
};

constexpr NodalTable make_nodal_table() {
  NodalTable t{};
  const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  int n = 0;
  for (int dm = 0; dm < 8; ++dm) {
    const int delta[3] = {(dm >> 2) & 1, (dm >> 1) & 1, dm & 1};
    for (int s = 0; s < 6; ++s) {
      int cur[3] = {0, 0, 0};
      int path[4][3] = {};
      int v = -1;
      for (int q = 0; q < 4; ++q) {
        if (q > 0) cur[perm[s][q - 1]] += 1;
        path[q][0] = cur[0];
        path[q][1] = cur[1];
        path[q][2] = cur[2];
        if (cur[0] == delta[0] && cur[1] == delta[1] && cur[2] == delta[2]) v = q;
      }
      if (v < 0) continue;
      t.e[n].sigma = s;
      t.e[n].v = v;
      for (int q = 0; q < 4; ++q) {
        const int a = path[q][0] - delta[0], b = path[q][1] - delta[1], c = path[q][2] - delta[2];
        t.e[n].off[q][0] = a - b;  // Kuhn -> index coordinates
        t.e[n].off[q][1] = b - c;
        t.e[n].off[q][2] = c;
      }
      ++n;
    }
  }
  return t;
}

__constant__ NodalTable kNodal = make_nodal_table();

template <class T, class KT>
__device__ __forceinline__ T nodal_partial(const TetDev& td, const T* __restrict__ elem, int i, int j, int k,
                                           const T* __restrict__ u, const KT* __restrict__ kk, bool check) {
  const int N = td.N;
  const long long x = td.base + node_offset(N, i, j, k);
  const T ux = u[x], kx = (T)ldk(kk, x);
  T y = 0;
#pragma unroll 4
  for (int e = 0; e < 24; ++e) {
    const NodalEntry& E = kNodal.e[e];
    bool ok = true;
    long long idx[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int a = i + E.off[q][0], b = j + E.off[q][1], c = k + E.off[q][2];
      if (check && (a < 0 || b < 0 || c < 0 || a + b + c > N)) ok = false;
      idx[q] = td.base + node_offset(N, a, b, c);
    }
    if (!ok) continue;
    T ksum = 0, inner = 0;
    const T* A = elem + E.sigma * 16 + E.v * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q == E.v) {
        ksum += kx;
      } else {
        ksum += (T)ldk(kk, idx[q]);
        inner = fma(A[q], u[idx[q]] - ux, inner);
      }
    }
    y = fma(ksum, inner, y);
  }
  return y;
}

template <class T, class KT>
__global__ void __launch_bounds__(256) nodal_volume_kernel(DepthDev D, const T* __restrict__ u,
                                                           const KT* __restrict__ kk, T* __restrict__ y) {
  const T* elem;
  if constexpr (sizeof(T) == 8)
    elem = reinterpret_cast<const T*>(D.elem64);
  else
    elem = reinterpret_cast<const T*>(D.elem32);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < D.n_rows; r += nwarps) {
    const int4 row = D.rows[r];
    const TetDev td = D.tets[row.x];
    const int N = td.N, j = row.y, k = row.z;
    if (j == 0 || k == 0 || j + k >= N - 1) continue;
    const T* el = elem + row.x * 96;
    for (int i = 1 + lane; i + j + k <= N - 1; i += 32) {
      const T v = nodal_partial<T, KT>(td, el, i, j, k, u, kk, false);
      y[td.base + node_offset(N, i, j, k)] = v;
    }
  }
}

template <class T, class KT>
__global__ void nodal_boundary_kernel(DepthDev D, const T* __restrict__ u, const KT* __restrict__ kk,
                                      T* __restrict__ y) {
  const T* elem;
  if constexpr (sizeof(T) == 8)
    elem = reinterpret_cast<const T*>(D.elem64);
  else
    elem = reinterpret_cast<const T*>(D.elem32);
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= D.n_bnodes) return;
  const int lo = D.bstart[b], hi = D.bstart[b + 1];
  T v = 0;
  if (!D.bdir[b]) {
    for (int q = lo; q < hi; ++q) {
      const BCopy cp = D.bcopies[q];
      v += nodal_partial<T, KT>(D.tets[cp.slot], elem + cp.slot * 96, cp.i, cp.j, cp.k, u, kk, true);
    }
  }
  for (int q = lo; q < hi; ++q) y[D.bcopies[q].idx] = v;
}

template <class T, class KT>
static void nodal_typed(const Mesh& m, int depth, const void* u, const void* kk, void* y, cudaStream_t s) {
  const DepthDev& D = m.depth[depth].dev;
  if (D.n_rows > 0) {
    const int blocks = std::min((D.n_rows + 7) / 8, m.num_sms * 8);
    nodal_volume_kernel<T, KT><<<blocks, 256, 0, s>>>(D, static_cast<const T*>(u), static_cast<const KT*>(kk),
                                                       static_cast<T*>(y));
    HHG_CUDA(cudaGetLastError());
  }
  if (D.n_bnodes > 0) {
    nodal_boundary_kernel<T, KT><<<(D.n_bnodes + 127) / 128, 128, 0, s>>>(
        D, static_cast<const T*>(u), static_cast<const KT*>(kk), static_cast<T*>(y));
    HHG_CUDA(cudaGetLastError());
  }
}

void launch_nodal_apply(const Mesh& m, int depth, int dtype, const void* u, void* y, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  if (dtype == HHG_F64)
    nodal_typed<double, double>(m, depth, u, Dh.k64, y, s);
  else if (dtype == HHG_F32)
    nodal_typed<float, float>(m, depth, u, Dh.k32, y, s);
  else
    nodal_typed<float, __nv_bfloat16>(m, depth, u, Dh.k16, y, s);
}

}  // namespace hhg
