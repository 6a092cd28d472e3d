// Operator of a tensor coefficient (M = 6; eq. "integral", eq. "meshdep"
// with M > 1, Sec. 7.3) in the modes of the scaled kernel.
#include <algorithm>

#include "hhg_internal.h"

namespace hhg {

// stride between the seven edge-weight arrays: n rounded up to 16 elements
long long tensor_weight_stride(long long n) { return (std::max<long long>(n, 1) + 15) / 16 * 16; }

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
// of x's primitive.  Both kinds of rows read weights precomputed with the
// coefficient: volume rows the edge weights of the volume stencil (a column
// march over the macro tets), rows of nodes on macro faces, edges and
// vertices the 14 weights of each copy (one thread per unique node sums its
// copies' partial rows, on a side stream concurrent with the march).
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

// Edge weights of the volume rows.  Every term's volume stencil is point
// symmetric (c^m_{-d} = c^m_d), so the weight of a volume row's edge
// (x, x+w_e) is
//     sum_m c^m_e (k_m(x) + k_m(x+w_e)) = B_e(x) + B_e(x+w_e) =: W_e(x),
//     B_e(z) = sum_m c^m_e k_m(z)   (e = the 7 positive directions),
// with c^m the volume stencil of the tet (also where x+w_e lies on a face).
// W_e(x) is stored for every node whose neighbour x+w_e is in the tet (0
// otherwise), direction major with a stride of n rounded up to 16 elements,
// so that element x of every direction has the same 16-byte alignment.
__global__ void tensor_weights_kernel(DepthDev D, const double* __restrict__ tsten, const double* __restrict__ km,
                                      long long ns, double* __restrict__ w64, float* __restrict__ w32) {
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
      for (int e = 0; e < 7; ++e) {
        int di, dj, dk;
        dir_of(e, di, dj, dk);
        const int a = i + di, b = j + dj, c = k + dk;
        double w = 0;
        if (a >= 0 && b >= 0 && c >= 0 && a + b + c <= N) {
          double ky[6];
          load6(km + 6 * (td.base + node_offset(N, a, b, c)), ky);
#pragma unroll
          for (int m = 0; m < 6; ++m) w = fma(st[m * 16 * kNDir + e], kx[m] + ky[m], w);
        }
        w64[e * ns + x] = w;
        w32[e * ns + x] = (float)w;
      }
    }
  }
}

// Weights of the interface rows: for boundary copy q and direction d,
//     sum_m c^m_{mask,d} (k_m(x) + k_m(x+w_d))
// with the term stencils of the copy's primitive (0 where x+w_d is outside
// the tet); stored at wb[d * n_copies + q].
__global__ void tensor_bweights_kernel(DepthDev D, const double* __restrict__ tsten, const double* __restrict__ km,
                                       int n_copies, double* __restrict__ w64, float* __restrict__ w32) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_copies; q += gridDim.x * blockDim.x) {
    const BCopy cp = D.bcopies[q];
    const TetDev td = D.tets[cp.slot];
    const int N = td.N;
    const double* st = tsten + (size_t)cp.slot * 6 * 16 * kNDir;
    double kx[6];
    load6(km + 6 * cp.idx, kx);
    for (int d = 0; d < kNDir; ++d) {
      int di, dj, dk;
      dir_of(d, di, dj, dk);
      const int a = cp.i + di, b = cp.j + dj, c = cp.k + dk;
      double w = 0;
      if (a >= 0 && b >= 0 && c >= 0 && a + b + c <= N) {
        double ky[6];
        load6(km + 6 * (td.base + node_offset(N, a, b, c)), ky);
#pragma unroll
        for (int m = 0; m < 6; ++m) w = fma(st[(m * 16 + cp.mask) * kNDir + d], kx[m] + ky[m], w);
      }
      w64[(size_t)d * n_copies + q] = w;
      w32[(size_t)d * n_copies + q] = (float)w;
    }
  }
}

void compute_tensor_weights(Mesh& m, cudaStream_t s) {
  for (int d = 0; d < m.ndepth; ++d) {
    Depth& D = m.depth[d];
    if (D.n_rows == 0) continue;
    const long long ns = tensor_weight_stride(D.n_stored);
    if (!D.tb64) {
      D.tb64 = static_cast<double*>(dalloc(D, 7 * ns * 8 + kCoefPad));
      D.tb32 = static_cast<float*>(dalloc(D, 7 * ns * 4 + kCoefPad));
      HHG_CUDA(cudaMemsetAsync(D.tb64, 0, 7 * ns * 8 + kCoefPad, s));
      HHG_CUDA(cudaMemsetAsync(D.tb32, 0, 7 * ns * 4 + kCoefPad, s));
    }
    const int g = std::max(1, std::min((D.n_rows + 7) / 8, 16 * m.num_sms));
    tensor_weights_kernel<<<g, 256, 0, s>>>(D.dev, D.tsten64, D.km64, ns, D.tb64, D.tb32);
    HHG_CUDA(cudaGetLastError());
    const int nc = (int)D.h_bcopies.size();
    if (nc > 0) {
      if (!D.twb64) {
        D.twb64 = static_cast<double*>(dalloc(D, (size_t)kNDir * nc * 8));
        D.twb32 = static_cast<float*>(dalloc(D, (size_t)kNDir * nc * 4));
      }
      tensor_bweights_kernel<<<std::min((nc + 255) / 256, 16 * m.num_sms), 256, 0, s>>>(D.dev, D.tsten64, D.km64, nc,
                                                                                       D.twb64, D.twb32);
      HHG_CUDA(cudaGetLastError());
    }
  }
}


// ---------------------------------------------------------------------------
// Volume rows: the column march of the scalar operator (csrc/march.cu) with
// the edge weights in place of c_e (k_x + k_y):
//     (A u)_x = sum_e [W_e(x) (u_{x+e} - u_x) - W_e(x-e) (u_x - u_{x-e})].
// A block of 4 warps takes a tile of 30 columns (lane L holds column
// i0-1+L) x 16 rows (warp w owns rows j0+4w .. j0+4w+3) of one tet and
// marches along k; each plane's 18 rows of u and of the 7 weight arrays (and
// 16 rows of f) are copied into a ring of plane stages with 16-byte
// cp.async chunks, one commit group per plane; a plane is read after
// cp.async.wait_group and a block barrier.  Forward fluxes are formed once
// at the node they leave; right neighbours come by shuffle, the fluxes a
// node receives from column i-1 are summed in lane L-1 and shuffled up.
// ---------------------------------------------------------------------------
namespace {

constexpr int kTW = 4;                 // warps per block, stacked in j
constexpr int kTRowsW = 4;             // owned rows per warp
constexpr int kTRowsM = kTRowsW + 2;   // rows a warp reads
constexpr int kTRowsB = kTW * kTRowsW + 2;  // staged rows per plane
constexpr int kTRowsF = kTW * kTRowsW;      // staged f rows per plane
constexpr int kTCols = 30;
constexpr int kTThreads = kTW * 32;

template <class T, int MODE>
struct TGeo {
  static constexpr int V = 16 / (int)sizeof(T);
  static constexpr int W = 32 + V;            // elements of a staged row
  static constexpr int R = W * (int)sizeof(T);  // bytes of a staged row
  static constexpr int CH = W / V;            // 16-byte chunks of a row
  static constexpr bool F = MODE == OP_RESID || MODE == OP_JACOBI;
  static constexpr int OFF_W = kTRowsB * R;              // 7 weight arrays after u
  static constexpr int OFF_F = OFF_W + 7 * kTRowsB * R;
  static constexpr int SB = OFF_F + (F ? kTRowsF * R : 0);
  static constexpr int SL = (kTRowsB * CH + kTThreads - 1) / kTThreads;  // copy slots per thread and array
  // stages: FP32 three (three blocks per SM), FP64 four (one block per SM)
  static constexpr int S = sizeof(T) == 8 ? 4 : 3;
  static constexpr int SMEM = S * SB;
};

__device__ __forceinline__ unsigned tsaddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void tcp16(unsigned dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void tcp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void tcp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ int trow(int N, int q, int j) {
  const int M = N - q;
  const int pl = (N + 1) * (N + 2) * (N + 3) / 6 - (M + 1) * (M + 2) * (M + 3) / 6;
  return pl + j * (M + 1) - j * (j - 1) / 2;
}

struct TMarchPtrs {
  const void* u;
  const void* w;  // the 7 edge-weight arrays, stride ws
  const void* f;
  void* out;
  double omega;
  long long lim_u;  // elements of u / f / out
  long long ws;     // stride between the weight arrays
  long long lim_w;  // elements of the weight allocation
};

template <class T, int MODE>
__global__ void __launch_bounds__(kTThreads, sizeof(T) == 8 ? 1 : 3)
    tensor_march_kernel(DepthDev D, TMarchPtrs p, int n_items) {
  using G = TGeo<T, MODE>;
  constexpr int S = G::S;
  constexpr int E = (int)sizeof(T);
  constexpr bool DIAG = MODE == OP_JACOBI || MODE == OP_DIAG;
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const unsigned ring_s = tsaddr(smem);
  int st_i = 0;
  int sr[G::SL], sc[G::SL];  // this thread's copy slots: staged row, chunk (the same for every array)
#pragma unroll
  for (int s = 0; s < G::SL; ++s) {
    const int x = tid + kTThreads * s;
    sr[s] = x < kTRowsB * G::CH ? x / G::CH : -1;
    sc[s] = x - (x / G::CH) * G::CH;
  }
  const bool own_lane = lane >= 1 && lane <= kTCols;
  const T* gu = static_cast<const T*>(p.u);
  const T* gw = static_cast<const T*>(p.w);
  const T* gf = static_cast<const T*>(p.f);

  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4 item = D.sitems[it];
    const TetDev td = D.tets[D.pairs[item.x].x];
    const int N = td.N;
    const int i0 = item.y & 0xffff, j0 = item.y >> 16, k0 = item.z, k1 = item.w;
    const int jw = j0 + kTRowsW * w;
    const int q_first = k0 - 1;
    const long long tb = td.base + i0 - 1;
    const int tl = (int)(tb & 15);
    const long long reach = tb + (long long)(N + 1) * (N + 2) * (N + 3) / 6 + 48;
    const bool inside = reach <= p.lim_u && reach + 6 * p.ws <= p.lim_w;
    // one 16-byte chunk c16 of the row at offset r of the array at base (element tb - tl of it)
    auto chunk = [&](unsigned dst, const T* base, long long lim, int r, int c16) {
      const int al = (tl + r) & ~(G::V - 1);
      const unsigned char* src = reinterpret_cast<const unsigned char*>(base + (tb - tl) + al) + c16;
      if (inside) {
        tcp16(dst, src, 16);
      } else {
        const long long left = (lim - (tb - tl + al)) * E - c16;
        const int nb = left >= 16 ? 16 : (left > 0 ? (int)left : 0);
        tcp16(dst, nb ? (const void*)src : p.u, nb);
      }
    };
    int qi = q_first;
    int o0 = trow(N, qi, j0 - 1), d0 = N - qi + 1 - (j0 - 1);
    int of0 = trow(N, qi - 1, j0 - 1), df0 = N - qi + 2 - (j0 - 1);
    int Pu = (N - qi + 1) * (N - qi + 2) / 2, Pf = (N - qi + 2) * (N - qi + 3) / 2;
    // plane qi's u and weight rows, f rows of plane qi-1; one commit group
    auto issue = [&]() {
      const unsigned st = ring_s + st_i * G::SB;
      if (qi <= k1 + 1) {
#pragma unroll
        for (int s = 0; s < G::SL; ++s)
          if (sr[s] >= 0 && sr[s] < d0) {
            const int r = o0 + sr[s] * d0 - sr[s] * (sr[s] - 1) / 2;
            const unsigned dst = st + sr[s] * G::R + 16 * sc[s];
            chunk(dst, gu, p.lim_u, r, 16 * sc[s]);
#pragma unroll
            for (int e = 0; e < 7; ++e)
              chunk(dst + G::OFF_W + e * kTRowsB * G::R, gw + e * p.ws, p.lim_w - e * p.ws, r, 16 * sc[s]);
          }
        if (G::F && qi - 1 >= k0) {
#pragma unroll
          for (int s = 0; s < G::SL; ++s)
            if (sr[s] >= 0 && sr[s] < kTRowsF && sr[s] + 1 < df0) {
              const int rr = sr[s] + 1;
              chunk(st + G::OFF_F + sr[s] * G::R + 16 * sc[s], gf, p.lim_u, of0 + rr * df0 - rr * (rr - 1) / 2,
                    16 * sc[s]);
            }
        }
      }
      tcp_commit();
      st_i = st_i + 1 == S ? 0 : st_i + 1;
      o0 += Pu - (j0 - 1);
      of0 += Pf - (j0 - 1);
      --d0;
      --df0;
      Pf = Pu;
      Pu -= N - qi + 1;
      ++qi;
    };
    int st_c = st_i;
    __syncthreads();  // every warp is done with the previous item's stages
#pragma unroll
    for (int t = 0; t < S - 1; ++t) issue();

    T ua[2][kTRowsM];  // u of two planes (roles alternate)
    int rs[kTRowsM];
#pragma unroll
    for (int m = 0; m < kTRowsM; ++m) rs[m] = trow(N, q_first, jw - 1 + m);
    auto dlt_of = [&](int q) { return (N - q + 1) * (N - q + 2) / 2 - (jw - 1); };
    const unsigned char* sb_last = smem;  // stage of the plane read last
    auto consume = [&](int b, int dl, int dm) {
      tcp_wait<S - 2>();
      __syncthreads();
      sb_last = smem + st_c * G::SB;
      st_c = st_c + 1 == S ? 0 : st_c + 1;
#pragma unroll
      for (int m = 0; m < kTRowsM; ++m) {
        const int t = tl + rs[m] + dl - dm * m;
        ua[b][m] = reinterpret_cast<const T*>(sb_last + (kTRowsW * w + m) * G::R)[(t & (G::V - 1)) + lane];
      }
    };
    // weight e at row m of the plane staged in sb, row offsets rs[m] + dl - dm m
    auto wt = [&](const unsigned char* sb, int e, int m, int dl, int dm) -> T {
      const int t = tl + rs[m] + dl - dm * m;
      return reinterpret_cast<const T*>(sb + G::OFF_W + (e * kTRowsB + kTRowsW * w + m) * G::R)[(t & (G::V - 1)) +
                                                                                                   lane];
    };
    auto f_at = [&](int m) -> T {
      const int t = tl + rs[m];
      return reinterpret_cast<const T*>(sb_last + G::OFF_F + (kTRowsW * w + m - 1) * G::R)[(t & (G::V - 1)) + lane];
    };
    auto advance_rows = [&](int dl) {
#pragma unroll
      for (int m = 0; m < kTRowsM; ++m) rs[m] += dl - m;
    };
    T* __restrict__ po = static_cast<T*>(p.out) + tb + lane;
    T F2p[4], F4c[4], F5c[4], F6p[5];  // carried fluxes
    // Weights of the plane being computed, read from its stage while that
    // stage is the newest one (a stage is refilled one step after it was
    // newest): W0, W2 rows 1..4, W1 rows 0..4, W3, W6 rows 1..5; for the
    // diagonal also W4, W5 rows 1..4.
    T Wq0[4], Wq1[5], Wq2[4], Wq3[5], Wq6[5], Wq4[4], Wq5[4];
    T W2p[4], W6p[5];  // the previous plane's W2 (rows 1..4) and W6 (rows 1..5), for the diagonal
    auto load_plane_weights = [&](const unsigned char* sb, int dl, int dm) {
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        Wq1[m] = wt(sb, 1, m, dl, dm);
        Wq3[m] = wt(sb, 3, m + 1, dl, dm);
        Wq6[m] = wt(sb, 6, m + 1, dl, dm);
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        Wq0[m] = wt(sb, 0, m + 1, dl, dm);
        Wq2[m] = wt(sb, 2, m + 1, dl, dm);
        if (DIAG) {
          Wq4[m] = wt(sb, 4, m + 1, dl, dm);
          Wq5[m] = wt(sb, 5, m + 1, dl, dm);
        }
      }
    };

    // prologue: planes k0-1 (buffer 0) and k0 (buffer 1)
    consume(0, 0, 0);
    load_plane_weights(sb_last, 0, 0);  // plane k0-1: W2, W6 used below
    issue();
    {
      const int dl = dlt_of(q_first);
      consume(1, dl, 1);
      issue();  // refills the stage of plane k0-1: every warp has read it (barrier in consume)
#pragma unroll
      for (int m = 1; m <= 4; ++m) {
        const T d0u = __shfl_down_sync(0xffffffffu, ua[0][m], 1);
        const T d1u = __shfl_down_sync(0xffffffffu, ua[1][m - 1], 1);
        F2p[m - 1] = Wq2[m - 1] * (ua[1][m] - ua[0][m]);
        F6p[m - 1] = Wq6[m - 1] * (d1u - ua[0][m]);
        F4c[m - 1] = wt(sb_last, 4, m, dl, 1) * (d0u - ua[1][m]);
        F5c[m - 1] = wt(sb_last, 5, m, dl, 1) * (ua[0][m + 1] - ua[1][m]);
      }
      F6p[4] = Wq6[4] * (__shfl_down_sync(0xffffffffu, ua[1][4], 1) - ua[0][5]);
      if (DIAG) {
#pragma unroll
        for (int m = 0; m < 4; ++m) W2p[m] = Wq2[m];
#pragma unroll
        for (int m = 0; m < 5; ++m) W6p[m] = Wq6[m];
      }
      load_plane_weights(sb_last, dl, 1);  // plane k0
      advance_rows(dl);
    }

    // step of plane q: buffer a holds plane q, buffer b receives plane q+1
    // (its stage is sb_last after consume)
    auto step = [&](auto ac, int q) {
      constexpr int a = decltype(ac)::value, b = 1 - a;
      const int dl = dlt_of(q);
      consume(b, dl, 1);
      const unsigned char* sn = sb_last;
      // row m of this lane holds a volume node iff m <= mlim
      const int mlim = N - q - (i0 - 1 + lane) - (jw - 1) - 1;
      T F1prev = Wq1[0] * (ua[a][1] - ua[a][0]);
      T w5prev = wt(sn, 5, 0, dl, 1);
      T F5prev = w5prev * (ua[a][1] - ua[b][0]);
      T F3cur = Wq3[0] * (__shfl_down_sync(0xffffffffu, ua[a][0], 1) - ua[a][1]);
#pragma unroll
      for (int m = 1; m <= 4; ++m) {
        const T dau = __shfl_down_sync(0xffffffffu, ua[a][m], 1);      // (i+1, row m), plane q
        const T dbu = __shfl_down_sync(0xffffffffu, ua[b][m - 1], 1);  // (i+1, row m-1), plane q+1
        const T w4n = wt(sn, 4, m, dl, 1), w5n = wt(sn, 5, m, dl, 1);
        const T F0 = Wq0[m - 1] * (dau - ua[a][m]);
        const T F1 = Wq1[m] * (ua[a][m + 1] - ua[a][m]);
        const T F2 = Wq2[m - 1] * (ua[b][m] - ua[a][m]);
        const T F3n = Wq3[m] * (dau - ua[a][m + 1]);
        const T F6 = Wq6[m - 1] * (dbu - ua[a][m]);
        const T F4n = w4n * (dau - ua[b][m]);
        const T F5n = w5n * (ua[a][m + 1] - ua[b][m]);
        // fluxes that node (i+1, row m) of plane q receives from column i
        const T H = F0 + F3n + F4n + F6p[m];  // F6p[m] holds row m+1
        T y = F0 + (F1 - F1prev) + (F2 - F2p[m - 1]) + F3cur + F4c[m - 1] + (F5c[m - 1] - F5prev) + F6;
        y -= __shfl_up_sync(0xffffffffu, H, 1);
        T dg = 0;
        if (DIAG) {
          // diagonal: -(sum_e W_e(x) + sum_e W_e(x - e))
          const T own = Wq0[m - 1] + Wq1[m] + Wq2[m - 1] + Wq3[m - 1] + Wq4[m - 1] + Wq5[m - 1] + Wq6[m - 1];
          const T back = Wq1[m - 1] + W2p[m - 1] + w5prev;
          const T hd = Wq0[m - 1] + Wq3[m] + w4n + W6p[m];  // from column i to node (i+1, row m)
          dg = -(own + back + __shfl_up_sync(0xffffffffu, hd, 1));
        }
        F2p[m - 1] = F2;
        F4c[m - 1] = F4n;
        F5c[m - 1] = F5n;
        F6p[m - 1] = F6;
        F1prev = F1;
        F5prev = F5n;
        w5prev = w5n;
        F3cur = F3n;
        // epilogue: owned lanes, volume nodes only
        if (own_lane && m <= mlim) {
          T* o = po + rs[m];
          if (MODE == OP_APPLY)
            *o = y;
          else if (MODE == OP_RESID)
            *o = f_at(m) - y;
          else if (MODE == OP_JACOBI)
            *o = ua[a][m] + (T)p.omega * (f_at(m) - y) / dg;
          else
            *o = dg;
        }
      }
      F6p[4] = Wq6[4] * (__shfl_down_sync(0xffffffffu, ua[b][4], 1) - ua[a][5]);
      if (DIAG) {
#pragma unroll
        for (int m = 0; m < 4; ++m) W2p[m] = Wq2[m];
#pragma unroll
        for (int m = 0; m < 5; ++m) W6p[m] = Wq6[m];
      }
      load_plane_weights(sn, dl, 1);  // plane q+1
      advance_rows(dl);
      issue();  // refills the stage of plane q, which every warp read last in the previous step
    };
    for (int q = k0; q <= k1; q += 2) {
      step(std::integral_constant<int, 1>{}, q);
      if (q + 1 > k1) break;
      step(std::integral_constant<int, 0>{}, q + 1);
    }
  }
  tcp_wait<0>();
}

template <class T, int MODE>
int tensor_march_occupancy() {
  static int occ = 0;
  if (!occ) {
    using G = TGeo<T, MODE>;
    HHG_CUDA(cudaFuncSetAttribute(tensor_march_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM));
    HHG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tensor_march_kernel<T, MODE>, kTThreads, G::SMEM));
    if (occ < 1) occ = 1;
  }
  return occ;
}

}  // namespace

void init_tensor_configs() {
  tensor_march_occupancy<float, OP_APPLY>();
  tensor_march_occupancy<float, OP_RESID>();
  tensor_march_occupancy<float, OP_JACOBI>();
  tensor_march_occupancy<float, OP_DIAG>();
  tensor_march_occupancy<double, OP_APPLY>();
  tensor_march_occupancy<double, OP_RESID>();
  tensor_march_occupancy<double, OP_JACOBI>();
  tensor_march_occupancy<double, OP_DIAG>();
}

// Interface rows: one thread per unique boundary node sums, over its copies
// and their 14 directions, the precomputed weight times u_y - u_x, applies
// the epilogue and writes every copy (Dirichlet: 0).
template <class T, int MODE>
__global__ void tensor_bnodes_kernel(DepthDev D, const T* __restrict__ wb, int n_copies, TensorPtrs p, int n_b) {
  const T* __restrict__ u = static_cast<const T*>(p.u);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_b; b += gridDim.x * blockDim.x) {
    const int lo = D.bstart[b], hi = D.bstart[b + 1];
    T val;
    if (D.bdir[b]) {
      val = MODE == OP_DIAG ? (T)1 : (T)0;
    } else {
      T y = 0, dg = 0;
      const T ux = u[D.bcopies[lo].idx];
      for (int q = lo; q < hi; ++q) {
        const BCopy cp = D.bcopies[q];
        const TetDev td = D.tets[cp.slot];
        const int N = td.N;
#pragma unroll
        for (int d = 0; d < kNDir; ++d) {
          int di, dj, dk;
          dir_of(d, di, dj, dk);
          const int a = cp.i + di, bb = cp.j + dj, c = cp.k + dk;
          if (a < 0 || bb < 0 || c < 0 || a + bb + c > N) continue;
          const T w = __ldg(wb + (size_t)d * n_copies + q);
          y = fma(w, __ldg(u + td.base + node_offset(N, a, bb, c)) - ux, y);
          dg -= w;
        }
      }
      val = tensor_finish<T, MODE>(y, dg, ux, D.bcopies[lo].idx, p);
    }
    for (int q = lo; q < hi; ++q) static_cast<T*>(p.out)[D.bcopies[q].idx] = val;
  }
}

template <class T, int MODE>
static void tensor_typed(const Mesh& m, int depth, const OpArgs& a, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  const DepthDev& D = Dh.dev;
  const int n_b = a.nc_only ? D.n_bnodes_nc : D.n_bnodes;
  const T* tb;
  const T* wb;
  if constexpr (sizeof(T) == 8) {
    tb = Dh.tb64;
    wb = Dh.twb64;
  } else {
    tb = Dh.tb32;
    wb = Dh.twb32;
  }
  TensorPtrs p{a.u, a.f, a.out, a.omega};
  const int n_items = a.nc_only ? D.n_sitems_nc : D.n_sitems;
  const int n_copies = (int)Dh.h_bcopies.size();
  // interface rows on the side stream, concurrent with the volume march;
  // joined before returning (also valid inside a stream capture)
  const bool fork = n_items > 0 && n_b > 0 && m.side;
  if (fork) {
    HHG_CUDA(cudaEventRecord(m.side_fork, s));
    HHG_CUDA(cudaStreamWaitEvent(m.side, m.side_fork, 0));
    tensor_bnodes_kernel<T, MODE><<<std::min((n_b + 127) / 128, 16 * m.num_sms), 128, 0, m.side>>>(D, wb, n_copies, p,
                                                                                                   n_b);
    HHG_CUDA(cudaGetLastError());
    HHG_CUDA(cudaEventRecord(m.side_join, m.side));
  }
  if (n_items > 0) {
    const long long ws = tensor_weight_stride(Dh.n_stored);
    TMarchPtrs mp{a.u, tb, a.f, a.out, a.omega, Dh.n_stored, ws, 7 * ws + kCoefPad / (long long)sizeof(T)};
    const int blocks = std::min(n_items, m.num_sms * tensor_march_occupancy<T, MODE>());
    tensor_march_kernel<T, MODE><<<blocks, kTThreads, TGeo<T, MODE>::SMEM, s>>>(D, mp, n_items);
    HHG_CUDA(cudaGetLastError());
  }
  if (fork) {
    HHG_CUDA(cudaStreamWaitEvent(s, m.side_join, 0));
  } else if (n_b > 0) {
    tensor_bnodes_kernel<T, MODE><<<std::min((n_b + 127) / 128, 16 * m.num_sms), 128, 0, s>>>(D, wb, n_copies, p, n_b);
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
