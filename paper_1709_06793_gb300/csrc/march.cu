// Volume kernel of the scaled operator (Sec. 6.1): a column march over tiles
// of 30 columns x 16 rows, the rows of each plane staged once per block.
//
// Rows of the volume (nodes strictly inside a macro tet: i, j, k >= 1 and
// i + j + k <= N - 1).  With the flux of an edge (a, b)
//     F(a, b) = (k_a + k_b) (u_b - u_a)
// and the 7 positive directions e_0..e_6 of the refined mesh (dir_of: e1,
// e2, e3, e1-e2, e1-e3, e2-e3, e1-e2+e3), the row of node x is
//     (A u)_x = sum_e c_e [F(x, x+e) - F(x-e, x)],
// c = (1/2) reference stencil of the volume primitive, the same for +e and
// -e (the volume stencil is symmetric).  Every flux is formed once, at the
// node it leaves.
//
// Work: a block item is a tile of one macro tet: columns i0-1 .. i0+30 (lane
// L of every warp holds column i0-1+L; lanes 1..30 own rows, lanes 0 and 31
// are the halo), rows j0 .. j0+15 (warp w owns rows j0+4w .. j0+4w+3 and
// reads rows j0+4w-1 .. j0+4w+4 of a plane, thread rows m = 0..5), planes
// k0..k1 of the k-march.  The right neighbour column comes from lane L+1 by
// a shuffle; the fluxes that node x receives from column i-1 (directions
// with di = 1) are summed in lane L-1 and shuffled up as one value.
//
// Staging: the tile's 18 rows of a plane (those that exist: rows past the
// plane's last row are skipped, their staged values are never used by a
// volume row) are contiguous segments of u, k
// (and f) in the packed layout.  The block's threads copy them with cp.async
// in 16-byte chunks from each segment's 16-byte boundary into a ring of S
// plane stages (rows shared by neighbouring warps are fetched once); one
// commit group per plane keeps S-1 planes in flight, and the block waits for
// its plane's group (cp.async.wait_group + __syncthreads).  No spin loop
// waits on memory.
//
// The FP32 apply and diagonal also run with two column sets per lane (P =
// 2): lane L holds columns i0-1+L and i0+29+L of a 60-column tile, and the
// flux and row arithmetic of both columns is one packed FP32x2 instruction
// (add / mul / fma .f32x2), which halves the issued arithmetic per node;
// copies, shared loads and shuffles stay per column, the row addressing is
// shared by both.
#include <algorithm>

#include "hhg_internal.h"

namespace hhg {

namespace {

template <class E>
__device__ __forceinline__ float to_f32(E v) {
  return (float)v;
}
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
// coefficient element -> arithmetic type (no detour through float for FP64)
template <class T, class E>
__device__ __forceinline__ T to_t(E v) {
  if constexpr (sizeof(T) == 8)
    return (T)v;
  else
    return to_f32(v);
}

__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// copy 16 bytes, of which the first src_bytes come from global memory (the
// rest is zero-filled; src_bytes = 0 reads nothing)
__device__ __forceinline__ void cp16(unsigned dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kWarps = 4;                    // warps per block, stacked in j
constexpr int kRowsW = 4;                    // owned rows per warp
constexpr int kRowsM = kRowsW + 2;           // rows a warp reads
constexpr int kRowsB = kWarps * kRowsW + 2;  // rows staged per plane (j0-1 .. j0+16)
constexpr int kRowsF = kWarps * kRowsW;      // f rows staged per plane (j0 .. j0+15)
constexpr int kCols = 30;                    // owned columns per tile (per column set)
constexpr int kSet = 30;                     // column distance of a lane's two column sets
constexpr int kThreads = kWarps * 32;

template <class T, class KT, int MODE, int P = 1>
struct Geo {
  static constexpr int VU = 16 / (int)sizeof(T);
  static constexpr int VK = 16 / (int)sizeof(KT);
  static constexpr int COLS = 32 + kSet * (P - 1);  // columns a warp reads
  // elements of a staged u / f row (whole chunks, one chunk of head room)
  static constexpr int WU = (COLS + VU - 1) / VU * VU + VU;
  static constexpr int WK = (COLS + VK - 1) / VK * VK + VK;
  static constexpr int RU = WU * (int)sizeof(T);
  static constexpr int RK = WK * (int)sizeof(KT);
  static constexpr bool F = MODE == OP_RESID || MODE == OP_JACOBI || MODE == OP_CHEB;
  static constexpr int OFF_K = kRowsB * RU;
  static constexpr int OFF_F = OFF_K + kRowsB * RK;
  static constexpr int SB = OFF_F + (F ? kRowsF * RU : 0);  // bytes of one plane stage
  static constexpr int CHU = WU / VU;                       // 16-byte chunks of a u / f row
  static constexpr int CHK = WK / VK;                       // ... of a k row
  static constexpr int SU = (kRowsB * CHU + kThreads - 1) / kThreads;  // copy slots per thread: u
  static constexpr int SK = (kRowsB * CHK + kThreads - 1) / kThreads;  // k
  static constexpr int SF = F ? (kRowsF * CHU + kThreads - 1) / kThreads : 0;  // f
  static constexpr int S = sizeof(T) == 8 ? 4 : 5;  // stages (S-1 planes in flight)
  static constexpr int REACH = (WU > WK ? WU : WK) + 16;  // elements a row's chunks reach past its start
  static constexpr int SMEM = S * SB;
  static_assert(RU % 16 == 0 && RK % 16 == 0, "staged rows must keep 16-byte alignment");
};

struct MarchPtrs {
  const void* u;
  const void* k;
  const void* f;
  void* out;
  const void* d_in;
  void* d_out;
  double omega, ca, cb;
  long long lim_u;  // elements of u / f / out (depth vector length)
  long long lim_k;  // elements of the coefficient array (padded allocation)
};

// offset of row j of plane q in a tet with N = 2^level
__device__ __forceinline__ int row_offset(int N, int q, int j) {
  const int M = N - q;
  const int pl = (N + 1) * (N + 2) * (N + 3) / 6 - (M + 1) * (M + 2) * (M + 3) / 6;
  return pl + j * (M + 1) - j * (j - 1) / 2;
}

template <class T>
__device__ __forceinline__ T qdiv(T a, T b) {
  return a / b;
}
template <>
__device__ __forceinline__ float qdiv<float>(float a, float b) {
  return __fdividef(a, b);  // preconditioner step: the outer FP64 residual decides convergence
}

template <class T>
__device__ __forceinline__ T shdown(T a) {
  return __shfl_down_sync(0xffffffffu, a, 1);
}
template <class T>
__device__ __forceinline__ T shup(T a) {
  return __shfl_up_sync(0xffffffffu, a, 1);
}
// The flux product is rounded on its own (no contraction into a following
// add), so the one- and two-column-set kernels round every node alike.
__device__ __forceinline__ float flux(float ua, float ka, float ub, float kb) {
  return __fmul_rn(ka + kb, ub - ua);
}
__device__ __forceinline__ double flux(double ua, double ka, double ub, double kb) {
  return __dmul_rn(ka + kb, ub - ua);
}

// packed pairs (two column sets per lane): one FP32x2 instruction per
// operation, each component rounded as the scalar operation would be
// (a - b as fma(b, -1, a): the product is exact, one rounding of a - b)
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2& operator+=(float2& a, float2 b) { return a = a + b; }
__device__ __forceinline__ float2& operator-=(float2& a, float2 b) { return a = a - b; }
using ::fma;
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 flux(float2 ua, float2 ka, float2 ub, float2 kb) { return (ka + kb) * (ub - ua); }
template <>
__device__ __forceinline__ float2 shdown<float2>(float2 a) {
  return make_float2(__shfl_down_sync(0xffffffffu, a.x, 1), __shfl_down_sync(0xffffffffu, a.y, 1));
}
template <>
__device__ __forceinline__ float2 shup<float2>(float2 a) {
  return make_float2(__shfl_up_sync(0xffffffffu, a.x, 1), __shfl_up_sync(0xffffffffu, a.y, 1));
}

// value type of P column sets per lane
template <class T, int P>
struct Lanes {
  using V = T;
  static __device__ __forceinline__ V splat(T x) { return x; }
  static __device__ __forceinline__ T comp(V v, int) { return v; }
  template <class E>
  static __device__ __forceinline__ V ld(const E* row, int i) {
    return to_t<T, E>(row[i]);
  }
};
template <>
struct Lanes<float, 2> {
  using V = float2;
  static __device__ __forceinline__ V splat(float x) { return make_float2(x, x); }
  static __device__ __forceinline__ float comp(V v, int h) { return h ? v.y : v.x; }
  template <class E>
  static __device__ __forceinline__ V ld(const E* row, int i) {
    return make_float2(to_f32(row[i]), to_f32(row[i + kSet]));
  }
};

// resident blocks per SM the registers are budgeted for (every variant
// without spills): more warps hide the latency of the dependent flux chains
constexpr int march_min_blocks(size_t es, int mode, int p) {
  return es == 8 ? 2
         : p == 2 ? (mode == OP_JACOBI || mode == OP_CHEB || mode == OP_RESID ? 3 : 4)
                  : (mode == OP_JACOBI || mode == OP_CHEB ? 3 : 4);
}

template <class T, class KT, int MODE, int P>
__global__ void __launch_bounds__(kThreads, march_min_blocks(sizeof(T), MODE, P))
    march_kernel(DepthDev D, const T* __restrict__ sten, MarchPtrs p, int n_items) {
  using G = Geo<T, KT, MODE, P>;
  using L = Lanes<T, P>;
  using V = typename L::V;
  constexpr int S = G::S;
  constexpr bool DIAG = MODE == OP_JACOBI || MODE == OP_CHEB || MODE == OP_DIAG;
  constexpr int EU = (int)sizeof(T), EK = (int)sizeof(KT);
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const unsigned ring_s = saddr(smem);
  int st_i = 0;  // stage of the next commit group (groups fill the ring in order)
  // this thread's copy slots: staged row and 16-byte chunk
  int ur[G::SU], uc[G::SU], kr[G::SK], kc[G::SK], fr[G::SF > 0 ? G::SF : 1], fc[G::SF > 0 ? G::SF : 1];
#pragma unroll
  for (int s = 0; s < G::SU; ++s) {
    const int x = tid + kThreads * s;
    ur[s] = x < kRowsB * G::CHU ? x / G::CHU : -1;
    uc[s] = x - (x / G::CHU) * G::CHU;
  }
#pragma unroll
  for (int s = 0; s < G::SK; ++s) {
    const int x = tid + kThreads * s;
    kr[s] = x < kRowsB * G::CHK ? x / G::CHK : -1;
    kc[s] = x - (x / G::CHK) * G::CHK;
  }
#pragma unroll
  for (int s = 0; s < G::SF; ++s) {
    const int x = tid + kThreads * s;
    fr[s] = x < kRowsF * G::CHU ? x / G::CHU : -1;
    fc[s] = x - (x / G::CHU) * G::CHU;
  }
  const bool own_lane = lane >= 1 && lane <= kCols;

  const int4* __restrict__ items = P == 2 ? D.mitems : D.sitems;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4 item = items[it];
    const int slot = D.pairs[item.x].x;
    const TetDev td = D.tets[slot];
    const int N = td.N;
    const int i0 = item.y & 0xffff, j0 = item.y >> 16, k0 = item.z, k1 = item.w;
    const int jw = j0 + kRowsW * w;  // first owned row of this warp
    V c[7];
    T cs = 0;
#pragma unroll
    for (int e = 0; e < 7; ++e) {
      const T ce = sten[slot * 16 * kNDir + e];
      c[e] = L::splat(ce);
      cs = e ? cs + ce : ce;
    }
    const V csum = L::splat(cs + cs);
    const int q_first = k0 - 1;

    // Element tb + r is node (i0-1, row offset r) of the tet.  Its 16-byte
    // chunk starts at the aligned element tb - tl + ((tl + r) & ~(V-1)),
    // tl = tb mod 16 elements.
    const long long tb = td.base + i0 - 1;
    const int tl = (int)(tb & 15);
    // every chunk of the tile lies before the end of the arrays (then no copy
    // needs clipping): the tet's nodes + a staged row's width + 16 elements
    const long long reach = tb + (long long)(N + 1) * (N + 2) * (N + 3) / 6 + G::REACH;
    const bool inside = reach <= p.lim_u && reach <= p.lim_k;
    const unsigned char* bu = reinterpret_cast<const unsigned char*>(static_cast<const T*>(p.u) + (tb - tl));
    const unsigned char* bk = reinterpret_cast<const unsigned char*>(static_cast<const KT*>(p.k) + (tb - tl));
    const unsigned char* bf =
        G::F ? reinterpret_cast<const unsigned char*>(static_cast<const T*>(p.f) + (tb - tl)) : nullptr;
    // one 16-byte chunk c of the row at offset r (array of element size es, lim elements)
    auto chunk = [&](unsigned dst, const unsigned char* b, int es, long long lim, int r, int c16) {
      const int al = (tl + r) & ~(16 / es - 1);
      const unsigned char* src = b + (long long)al * es + c16;
      if (inside) {
        cp16(dst, src, 16);
      } else {
        const long long left = (lim - (tb - tl + al)) * es - c16;
        const int sb = left >= 16 ? 16 : (left > 0 ? (int)left : 0);
        cp16(dst, sb ? (const void*)src : p.u, sb);
      }
    };

    // copy state: the plane to issue (qi), the offset and length of staged
    // row 0 (j0-1) there and in plane qi-1 (f rows), and the plane sizes
    int qi = q_first;
    int o0 = row_offset(N, qi, j0 - 1), d0 = N - qi + 1 - (j0 - 1);
    int of0 = row_offset(N, qi - 1, j0 - 1), df0 = N - qi + 2 - (j0 - 1);
    int Pu = (N - qi + 1) * (N - qi + 2) / 2, Pf = (N - qi + 2) * (N - qi + 3) / 2;
    // copies of plane qi (u, k) and of f of plane qi-1 into the next stage;
    // always one commit group (empty past the item's last plane)
    auto issue = [&]() {
      const unsigned st = ring_s + st_i * G::SB;
      if (qi <= k1 + 1) {
#pragma unroll
        for (int s = 0; s < G::SU; ++s)
          if (ur[s] >= 0 && ur[s] < d0)  // rows past the plane's last row are not fetched
            chunk(st + ur[s] * G::RU + 16 * uc[s], bu, EU, p.lim_u, o0 + ur[s] * d0 - ur[s] * (ur[s] - 1) / 2,
                  16 * uc[s]);
#pragma unroll
        for (int s = 0; s < G::SK; ++s)
          if (kr[s] >= 0 && kr[s] < d0)
            chunk(st + G::OFF_K + kr[s] * G::RK + 16 * kc[s], bk, EK, p.lim_k,
                  o0 + kr[s] * d0 - kr[s] * (kr[s] - 1) / 2, 16 * kc[s]);
        if (G::F && qi - 1 >= k0) {
#pragma unroll
          for (int s = 0; s < G::SF; ++s)
            if (fr[s] >= 0 && fr[s] + 1 < df0) {
              const int r = fr[s] + 1;  // staged f row s holds row j0 + fr
              chunk(st + G::OFF_F + fr[s] * G::RU + 16 * fc[s], bf, EU, p.lim_u, of0 + r * df0 - r * (r - 1) / 2,
                    16 * fc[s]);
            }
        }
      }
      cp_commit();
      st_i = st_i + 1 == S ? 0 : st_i + 1;
      // plane qi+1: row j moves by the plane size - j, rows get one shorter
      o0 += Pu - (j0 - 1);
      of0 += Pf - (j0 - 1);
      --d0;
      --df0;
      Pf = Pu;
      Pu -= N - qi + 1;
      ++qi;
    };

    int st_c = st_i;  // stage of the next plane to read (plane q_first)
    // every warp is done with the previous item's stages (the last one read
    // is the first one this item fills)
    __syncthreads();
#pragma unroll
    for (int t = 0; t < S - 1; ++t) issue();

    // thread state
    V xu[2][kRowsM], xk[2][kRowsM];  // planes (two buffers, roles alternate)
    int rs[kRowsM];                  // row offsets (rows jw-1+m) of the plane being computed
    V F2p[4], F4c[4], F5c[4], F6p[5];  // carried fluxes
    V kp[5], dkp[4];                   // plane q-1: own k (rows 1..5), right k (rows 1..4)
#pragma unroll
    for (int m = 0; m < kRowsM; ++m) rs[m] = row_offset(N, q_first, jw - 1 + m);
    // row m of plane q+1 starts at rs[m] + dlt(q) - m
    auto dlt_of = [&](int q) { return (N - q + 1) * (N - q + 2) / 2 - (jw - 1); };
    const unsigned char* sb_last = smem;  // stage read last (plane q+1 during the step of plane q)

    // wait for the next plane, then read this warp's rows (staged rows 4w + m)
    auto consume = [&](int b, int dl, int dm) {  // row m of the plane at rs[m] + dl - dm m
      cp_wait<S - 2>();  // this thread's copies of the plane have landed
      __syncthreads();   // ... and every other thread's (and every warp is done with the previous step)
      const unsigned char* sb = smem + st_c * G::SB;
      sb_last = sb;
      st_c = st_c + 1 == S ? 0 : st_c + 1;
#pragma unroll
      for (int m = 0; m < kRowsM; ++m) {
        const int t = tl + rs[m] + dl - dm * m;
        const int r = kRowsW * w + m;
        xu[b][m] = L::ld(reinterpret_cast<const T*>(sb + r * G::RU), (t & (G::VU - 1)) + lane);
        xk[b][m] = L::ld(reinterpret_cast<const KT*>(sb + G::OFF_K + r * G::RK), (t & (G::VK - 1)) + lane);
      }
    };
    auto advance_rows = [&](int dl) {
#pragma unroll
      for (int m = 0; m < kRowsM; ++m) rs[m] += dl - m;
    };
    // f at owned row m of the plane being computed (carried by the stage of the next plane)
    auto f_at = [&](int m) -> V {
      const int t = tl + rs[m];
      return L::ld(reinterpret_cast<const T*>(sb_last + G::OFF_F + (kRowsW * w + m - 1) * G::RU), (t & (G::VU - 1)) + lane);
    };
    T* __restrict__ po = static_cast<T*>(p.out) + tb + lane;

    // prologue: planes k0-1 (buffer 0) and k0 (buffer 1); carried fluxes of plane k0
    consume(0, 0, 0);
    issue();
    {
      const int dl = dlt_of(q_first);
      consume(1, dl, 1);
      issue();
      advance_rows(dl);
    }
    // right neighbours (lane L+1) are shuffled where they are used
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
      const V d0u = shdown(xu[0][m]), d0k = shdown(xk[0][m]);
      const V d1u = shdown(xu[1][m - 1]), d1k = shdown(xk[1][m - 1]);
      F2p[m - 1] = flux(xu[0][m], xk[0][m], xu[1][m], xk[1][m]);
      F6p[m - 1] = flux(xu[0][m], xk[0][m], d1u, d1k);
      F4c[m - 1] = flux(xu[1][m], xk[1][m], d0u, d0k);
      F5c[m - 1] = flux(xu[1][m], xk[1][m], xu[0][m + 1], xk[0][m + 1]);
      if (DIAG) dkp[m - 1] = d0k;
    }
    F6p[4] = flux(xu[0][5], xk[0][5], shdown(xu[1][4]), shdown(xk[1][4]));
    if (DIAG) {
#pragma unroll
      for (int m = 1; m <= 5; ++m) kp[m - 1] = xk[0][m];
    }

    // step of plane q: buffer a holds plane q, buffer b receives plane q+1
    auto step = [&](auto ac, int q) {
      constexpr int a = decltype(ac)::value, b = 1 - a;
      const int dl = dlt_of(q);
      consume(b, dl, 1);
      // row m of this lane holds a volume node iff m <= mlim
      const int mlim = N - q - (i0 - 1 + lane) - (jw - 1) - 1;
      V F1prev = flux(xu[a][0], xk[a][0], xu[a][1], xk[a][1]);
      V F5prev = flux(xu[b][0], xk[b][0], xu[a][1], xk[a][1]);
      V dak = shdown(xk[a][0]);  // k at (i+1, row m-1) of plane q
      V F3cur = flux(xu[a][1], xk[a][1], shdown(xu[a][0]), dak);
#pragma unroll
      for (int m = 1; m <= 4; ++m) {
        const V dau = shdown(xu[a][m]), dakm = shdown(xk[a][m]);          // (i+1, row m), plane q
        const V dbu = shdown(xu[b][m - 1]), dbk = shdown(xk[b][m - 1]);  // (i+1, row m-1), plane q+1
        const V F0 = flux(xu[a][m], xk[a][m], dau, dakm);
        const V F1 = flux(xu[a][m], xk[a][m], xu[a][m + 1], xk[a][m + 1]);
        const V F2 = flux(xu[a][m], xk[a][m], xu[b][m], xk[b][m]);
        const V F3n = flux(xu[a][m + 1], xk[a][m + 1], dau, dakm);
        const V F6 = flux(xu[a][m], xk[a][m], dbu, dbk);
        const V F4n = flux(xu[b][m], xk[b][m], dau, dakm);
        const V F5n = flux(xu[b][m], xk[b][m], xu[a][m + 1], xk[a][m + 1]);
        const V t0 = c[0] * F0;
        V H = fma(c[3], F3n, t0);
        H = fma(c[4], F4n, H);
        H = fma(c[6], F6p[m], H);  // F6p[m] holds row m+1
        V y = fma(c[1], F1 - F1prev, t0);
        y = fma(c[2], F2 - F2p[m - 1], y);
        y = fma(c[3], F3cur, y);
        y = fma(c[4], F4c[m - 1], y);
        y = fma(c[5], F5c[m - 1] - F5prev, y);
        y = fma(c[6], F6, y);
        y -= shup(H);
        V dg = y;
        if (DIAG) {
          V sk = c[0] * dakm;
          sk = fma(c[1], xk[a][m + 1] + xk[a][m - 1], sk);
          sk = fma(c[2], xk[b][m] + kp[m - 1], sk);
          sk = fma(c[3], dak, sk);
          sk = fma(c[4], dkp[m - 1], sk);
          sk = fma(c[5], kp[m] + xk[b][m - 1], sk);
          sk = fma(c[6], dbk, sk);
          V hd = c[0] * xk[a][m];
          hd = fma(c[3], xk[a][m + 1], hd);
          hd = fma(c[4], xk[b][m], hd);
          hd = fma(c[6], kp[m], hd);
          sk += shup(hd);
          dg = fma(csum, xk[a][m], sk);  // -diagonal
        }
        F2p[m - 1] = F2;
        F4c[m - 1] = F4n;
        F5c[m - 1] = F5n;
        F6p[m - 1] = F6;
        F1prev = F1;
        F5prev = F5n;
        F3cur = F3n;
        if (DIAG) dkp[m - 1] = dakm;
        dak = dakm;
        // epilogue: owned lanes, volume nodes only (column set h at +30 h)
        if (own_lane) {
          V fv;
          if (G::F) fv = f_at(m);
#pragma unroll
          for (int h = 0; h < P; ++h) {
            if (m > mlim - kSet * h) continue;
            T* o = po + rs[m] + kSet * h;
            const T yv = L::comp(y, h);
            if (MODE == OP_APPLY) {
              *o = yv;
            } else if (MODE == OP_RESID) {
              *o = L::comp(fv, h) - yv;
            } else if (MODE == OP_JACOBI) {
              *o = L::comp(xu[a][m], h) + qdiv((T)p.omega * (L::comp(fv, h) - yv), -L::comp(dg, h));
            } else if (MODE == OP_CHEB) {
              const long long idx = o - static_cast<T*>(p.out);
              const T prev = p.ca != 0.0 ? (T)p.ca * __ldg(static_cast<const T*>(p.d_in) + idx) : (T)0;
              const T dn = prev + (T)p.cb * (L::comp(fv, h) - yv) / -L::comp(dg, h);
              static_cast<T*>(p.d_out)[idx] = dn;
              *o = L::comp(xu[a][m], h) + dn;
            } else {  // OP_DIAG
              *o = -L::comp(dg, h);
            }
          }
        }
      }
      F6p[4] = flux(xu[a][5], xk[a][5], shdown(xu[b][4]), shdown(xk[b][4]));
      if (DIAG) {
#pragma unroll
        for (int m = 1; m <= 5; ++m) kp[m - 1] = xk[a][m];
      }
      advance_rows(dl);
      issue();  // the stage read in the previous step is free (every warp passed this step's barrier)
    };

    for (int q = k0; q <= k1; q += 2) {
      step(std::integral_constant<int, 1>{}, q);
      if (q + 1 > k1) break;
      step(std::integral_constant<int, 0>{}, q + 1);
    }
  }
  cp_wait<0>();
}

template <class T, class KT, int MODE, int P>
int march_occupancy() {
  static int occ = 0;
  if (!occ) {
    using G = Geo<T, KT, MODE, P>;
    HHG_CUDA(cudaFuncSetAttribute(march_kernel<T, KT, MODE, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM));
    HHG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, march_kernel<T, KT, MODE, P>, kThreads, G::SMEM));
    if (occ < 1) occ = 1;
  }
  return occ;
}

template <class T, class KT, int MODE, int P>
void launch_t(const Mesh& m, int depth, const OpArgs& a, const void* kptr, long long lim_k, int n_items,
              cudaStream_t s) {
  using G = Geo<T, KT, MODE, P>;
  const Depth& Dh = m.depth[depth];
  const int occ = march_occupancy<T, KT, MODE, P>();
  const int blocks = std::min(n_items, m.num_sms * occ);
  MarchPtrs p{a.u, kptr, a.f, a.out, a.d_in, a.d_out, a.omega, a.ca, a.cb, Dh.n_stored, lim_k};
  const T* sten = sizeof(T) == 8 ? reinterpret_cast<const T*>(Dh.dev.sten64) : reinterpret_cast<const T*>(Dh.dev.sten32);
  march_kernel<T, KT, MODE, P><<<blocks, kThreads, G::SMEM, s>>>(Dh.dev, sten, p, n_items);
  HHG_CUDA(cudaGetLastError());
}

template <int MODE>
void launch_mode(const Mesh& m, int depth, int dtype, const OpArgs& a, bool wide, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  const DepthDev& D = Dh.dev;
  const long long n = Dh.n_stored;
  const int n1 = a.nc_only ? D.n_sitems_nc : D.n_sitems;
  const int n2 = a.nc_only ? D.n_mitems_nc : D.n_mitems;
  if (dtype == HHG_F64) {
    if (n1) launch_t<double, double, MODE, 1>(m, depth, a, Dh.k64, n + kCoefPad / 8, n1, s);
  } else if (dtype == kF64KBF16) {
    if (n1) launch_t<double, double, MODE, 1>(m, depth, a, Dh.k16d, n + kCoefPad / 8, n1, s);
  } else if (dtype == HHG_F32) {
    if (wide) {
      if (n2) launch_t<float, float, MODE, 2>(m, depth, a, Dh.k32, n + kCoefPad / 4, n2, s);
    } else if (n1) {
      launch_t<float, float, MODE, 1>(m, depth, a, Dh.k32, n + kCoefPad / 4, n1, s);
    }
  } else {
    if (wide) {
      if (n2) launch_t<float, __nv_bfloat16, MODE, 2>(m, depth, a, Dh.k16, n + kCoefPad / 2, n2, s);
    } else if (n1) {
      launch_t<float, __nv_bfloat16, MODE, 1>(m, depth, a, Dh.k16, n + kCoefPad / 2, n1, s);
    }
  }
}

template <class T, class KT, int P>
void init_t() {
  march_occupancy<T, KT, OP_APPLY, P>();
  march_occupancy<T, KT, OP_RESID, P>();
  march_occupancy<T, KT, OP_JACOBI, P>();
  march_occupancy<T, KT, OP_CHEB, P>();
  march_occupancy<T, KT, OP_DIAG, P>();
}

}  // namespace

void init_march_configs(int dtype) {
  if (dtype == HHG_F64 || dtype == kF64KBF16) {
    init_t<double, double, 1>();
  } else if (dtype == HHG_F32) {
    init_t<float, float, 1>();
    init_t<float, float, 2>();
  } else {
    init_t<float, __nv_bfloat16, 1>();
    init_t<float, __nv_bfloat16, 2>();
  }
}

// vkernel 2: the FP32 apply (and diagonal) run the march with two column
// sets per lane; the modes that also stream f (residual, Jacobi, Chebyshev)
// keep one, which measures faster for them; FP64 keeps one
void launch_march(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, cudaStream_t s) {
  const bool wide = m.vkernel == 2 && (mode == OP_APPLY || mode == OP_DIAG);
  switch (mode) {
    case OP_APPLY: launch_mode<OP_APPLY>(m, depth, dtype, a, wide, s); break;
    case OP_RESID: launch_mode<OP_RESID>(m, depth, dtype, a, wide, s); break;
    case OP_JACOBI: launch_mode<OP_JACOBI>(m, depth, dtype, a, wide, s); break;
    case OP_CHEB: launch_mode<OP_CHEB>(m, depth, dtype, a, wide, s); break;
    case OP_DIAG: launch_mode<OP_DIAG>(m, depth, dtype, a, wide, s); break;
  }
}

// Work lists of the march: per tet (those above the coarsest level first),
// tiles (i0, j0) of 30 columns (sitems; 60 for the two-column-set kernel:
// mitems) x 16 rows, each tile's planes 1 .. N-1-i0-j0 cut into segments of
// kseg planes; longest segment first within a class (korder 1: by plane
// window).  kseg is halved (down to 4) while a class would have fewer items
// than two per resident block.
static void march_items(const Mesh& m, Depth& D, int cols, std::vector<int4>& out, int& n_nc) {
  const int ns = (int)D.slot_tet.size();
  const long long target = (long long)(m.num_sms > 0 ? m.num_sms : 152) * 3 * 2;
  constexpr int kTileJ = kWarps * kRowsW;
  std::vector<int4> lists[2];
  for (int cls = 0; cls < 2; ++cls) {
    std::vector<int> slots;
    for (int s = 0; s < ns; ++s)
      if ((s < D.n_slots_nc) == (cls == 0)) slots.push_back(s);
    auto count = [&](int ks) {
      long long c = 0;
      for (int s : slots) {
        const int N = D.h_tets[s].N;
        for (int j0 = 1; j0 <= N - 2; j0 += kTileJ)
          for (int i0 = 1; i0 + j0 <= N - 2; i0 += cols) c += (N - 1 - (i0 + j0) + ks - 1) / ks;
      }
      return c;
    };
    int ks = std::max(1, m.kseg);
    while (ks > 4 && count(ks) < target) ks /= 2;
    std::vector<std::pair<long long, int4>> its;
    for (int s : slots) {
      const int N = D.h_tets[s].N;
      for (int j0 = 1; j0 <= N - 2; j0 += kTileJ)
        for (int i0 = 1; i0 + j0 <= N - 2; i0 += cols) {
          const int top = N - 1 - (i0 + j0);
          for (int k0 = 1; k0 <= top; k0 += ks) {
            const int k1 = std::min(top, k0 + ks - 1);
            const long long key = m.korder == 1 ? ((long long)k0 << 42) | ((long long)s << 22) |
                                                      ((long long)j0 << 11) | i0
                                                : -(long long)(k1 - k0 + 1);
            its.push_back({key, make_int4(s, i0 | j0 << 16, k0, k1)});
          }
        }
    }
    std::stable_sort(its.begin(), its.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    for (auto& e : its) lists[cls].push_back(e.second);
  }
  out = lists[0];
  n_nc = (int)lists[0].size();
  out.insert(out.end(), lists[1].begin(), lists[1].end());
}

void build_march_items(const Mesh& m, Depth& D) {
  const int ns = (int)D.slot_tet.size();
  D.h_pairs.clear();
  for (int s = 0; s < ns; ++s) D.h_pairs.push_back(make_int2(s, -1));
  march_items(m, D, kCols, D.h_sitems, D.n_sitems_nc);
  D.n_sitems = (int)D.h_sitems.size();
  march_items(m, D, kCols + kSet, D.h_mitems, D.n_mitems_nc);
  D.n_mitems = (int)D.h_mitems.size();
}

}  // namespace hhg
