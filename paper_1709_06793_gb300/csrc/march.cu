// Volume kernel of the scaled operator (Sec. 6.1): a column march with
// bulk-copied row segments.
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
// Work: a warp item is a tile of one pair of macro tets with the same level
// (the two tets ride in the two halves of packed FP32x2 registers; FP64 and
// unpaired tets use one half): columns i0-1 .. i0+30 (lane L holds column
// i0-1+L; lanes 1..30 own rows, lanes 0 and 31 are the halo), rows j0-1 ..
// j0+4 (thread rows m = 0..5; m = 1..4 are owned), planes k0..k1 of the
// k-march.  The right neighbour column comes from lane L+1 by a shuffle; the
// fluxes that node x receives from column i-1 (directions with di = 1) are
// summed in lane L-1 and shuffled up as one value.
//
// Staging: the tile's rows of a plane are contiguous segments of u, k (and f)
// in the packed layout.  The lanes copy them with cp.async in 16-byte chunks
// from each segment's 16-byte boundary into the warp's ring of S plane
// stages (a row's chunks side by side in one instruction, several rows per
// instruction); one commit group per plane keeps S-1 planes in flight, and a
// consumer waits for its plane's group (cp.async.wait_group) and the warp
// (__syncwarp).  No spin loop waits on memory.
#include <algorithm>
#include <map>

#include "hhg_internal.h"

namespace hhg {

namespace {

// ---- arithmetic on the P tets of a pair ------------------------------------
template <class T, int P>
struct VT;
template <>
struct VT<float, 2> {
  using t = float2;
  static __device__ __forceinline__ t add(t a, t b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ t sub(t a, t b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
  static __device__ __forceinline__ t mul(t a, t b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ t fma(t a, t b, t c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ t down(t a) {
    return make_float2(__shfl_down_sync(0xffffffffu, a.x, 1), __shfl_down_sync(0xffffffffu, a.y, 1));
  }
  static __device__ __forceinline__ t up(t a) {
    return make_float2(__shfl_up_sync(0xffffffffu, a.x, 1), __shfl_up_sync(0xffffffffu, a.y, 1));
  }
  static __device__ __forceinline__ t make(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ float get(t a, int h) { return h ? a.y : a.x; }
};
template <class T>
struct VT<T, 1> {
  using t = T;
  static __device__ __forceinline__ t add(t a, t b) { return a + b; }
  static __device__ __forceinline__ t sub(t a, t b) { return a - b; }
  static __device__ __forceinline__ t mul(t a, t b) { return a * b; }
  static __device__ __forceinline__ t fma(t a, t b, t c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ t down(t a) { return __shfl_down_sync(0xffffffffu, a, 1); }
  static __device__ __forceinline__ t up(t a) { return __shfl_up_sync(0xffffffffu, a, 1); }
  static __device__ __forceinline__ t make(T a, T) { return a; }
  static __device__ __forceinline__ T get(t a, int) { return a; }
};

// coefficient element -> arithmetic type (no detour through float for FP64)
template <class T, class E>
__device__ __forceinline__ T to_t(E v) {
  return (T)v;
}
template <>
__device__ __forceinline__ float to_t<float, __nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

// ---- 16-byte asynchronous copies (inline PTX) -------------------------------
__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// copy 16 bytes, of which the first src_bytes come from global memory (the
// rest is zero-filled; src_bytes = 0 reads nothing)
__device__ __forceinline__ void cp16(unsigned dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kWarps = 4;                        // warps per block
constexpr int kRowsM = 6;                        // thread rows m = 0..5 (j0-1 .. j0+4)
constexpr int kCols = 30;                        // owned columns per warp tile

template <class T, class KT, int P, int MODE>
struct Geo {
  static constexpr int VU = 16 / (int)sizeof(T);
  static constexpr int VK = 16 / (int)sizeof(KT);
  static constexpr int WU = 32 + VU;  // elements of a staged u / f row (one 16-byte chunk of head room)
  static constexpr int WK = 32 + VK;
  static constexpr int RU = WU * (int)sizeof(T);
  static constexpr int RK = WK * (int)sizeof(KT);
  static constexpr bool F = MODE == OP_RESID || MODE == OP_JACOBI || MODE == OP_CHEB;
  static constexpr int NF = F ? 4 : 0;  // f rows per tet (the owned rows)
  static constexpr int OFF_K = P * kRowsM * RU;
  static constexpr int OFF_F = OFF_K + P * kRowsM * RK;
  static constexpr int SB = OFF_F + P * NF * RU;  // bytes of one plane stage
  static constexpr int CHU = WU / VU;   // 16-byte chunks of a u / f row
  static constexpr int CHK = WK / VK;   // ... of a k row
  static constexpr int RPU = 32 / CHU;  // u / f rows per copy instruction
  static constexpr int RPK = 32 / CHK;  // k rows per copy instruction
  static constexpr int S = sizeof(T) == 8 ? 4 : 5;  // stages per warp (S-1 planes in flight)
  static constexpr int WARP_BYTES = S * SB;
  static constexpr int SMEM = kWarps * WARP_BYTES;
  static_assert(RU % 16 == 0 && RK % 16 == 0, "staged rows must keep 16-byte alignment");
  static_assert(RPU >= 1 && RPK >= 1, "a row fits one copy instruction");
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

#ifndef HHG_MARCH_MINB
#define HHG_MARCH_MINB 3
#endif
template <class T, class KT, int P, int MODE>
__global__ void __launch_bounds__(kWarps * 32, sizeof(T) == 8 || MODE == OP_JACOBI || MODE == OP_CHEB || MODE == OP_RESID ? 2 : HHG_MARCH_MINB)
    march_kernel(DepthDev D, const T* __restrict__ sten, MarchPtrs p, int n_items) {
  using G = Geo<T, KT, P, MODE>;
  using V = VT<T, P>;
  using PT = typename V::t;
  constexpr int S = G::S;
  constexpr bool DIAG = MODE == OP_JACOBI || MODE == OP_CHEB || MODE == OP_DIAG;
  constexpr int EU = (int)sizeof(T), EK = (int)sizeof(KT);
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned char* ring = smem + wib * G::WARP_BYTES;
  const unsigned ring_s = saddr(ring);
  unsigned g = 0;  // commit groups of this warp so far (plane stage = group mod S)
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  // this lane's chunk of the copy instructions: row pu (pk) of each round, chunk cu (ck)
  const int pu = lane / G::CHU, cu = lane - pu * G::CHU;
  const int pk = lane / G::CHK, ck = lane - pk * G::CHK;
  const bool cpu_on = pu < G::RPU, cpk_on = pk < G::RPK;

  for (int it = gw; it < n_items; it += nw) {
    const int4 item = P == 2 ? D.mitems[it] : D.sitems[it];
    const int2 pr = D.pairs[item.x];
    const bool hasB = P == 2 && pr.y >= 0;
    const int slotA = pr.x, slotB = pr.y >= 0 ? pr.y : pr.x;
    const TetDev ta = D.tets[slotA], tb = D.tets[slotB];
    const int N = ta.N;
    const int i0 = item.y & 0xffff, j0 = item.y >> 16, k0 = item.z, k1 = item.w;
    PT c[7];
#pragma unroll
    for (int e = 0; e < 7; ++e) c[e] = V::make(sten[slotA * 16 * kNDir + e], sten[slotB * 16 * kNDir + e]);
    PT csum = V::add(c[0], c[1]);
#pragma unroll
    for (int e = 2; e < 7; ++e) csum = V::add(csum, c[e]);
    csum = V::add(csum, csum);
    const int q_first = k0 - 1;

    // Element e = tbase[h] + r is node (i0-1, row r) of tet h (r a row offset
    // in the tet).  Its 16-byte chunk starts at the aligned element
    // tbase - tl + ((tl + r) & ~(V-1)), tl = tbase mod 16 elements.
    long long tbase[2];
    int tl[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      tbase[h] = (h ? tb.base : ta.base) + i0 - 1;
      tl[h] = (int)(tbase[h] & 15);
    }
    // every chunk of the tile lies before the end of the arrays (then no copy
    // needs clipping): the tet's nodes + 48 elements of head room
    const long long tet_end = tbase[0] > tbase[1] ? tbase[0] : tbase[1];
    const bool inside = tet_end + (long long)(N + 1) * (N + 2) * (N + 3) / 6 + 48 <= p.lim_u &&
                        tet_end + (long long)(N + 1) * (N + 2) * (N + 3) / 6 + 48 <= p.lim_k;
    // aligned chunk bases of this lane (u / f and k), per tet half
    const unsigned char* bu[2];
    const unsigned char* bk[2];
    const unsigned char* bf[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      bu[h] = reinterpret_cast<const unsigned char*>(static_cast<const T*>(p.u) + (tbase[h] - tl[h])) + 16 * cu;
      bk[h] = reinterpret_cast<const unsigned char*>(static_cast<const KT*>(p.k) + (tbase[h] - tl[h])) + 16 * ck;
      bf[h] = G::F ? reinterpret_cast<const unsigned char*>(static_cast<const T*>(p.f) + (tbase[h] - tl[h])) + 16 * cu
                   : nullptr;
    }
    // one 16-byte chunk: row offset r of tet half h, from lane base b (array
    // of element size es, lim elements); clipped copies only outside `inside`
    auto chunk = [&](unsigned dst, const unsigned char* b, int es, long long lim, int h, int r, int c16) {
      const int al = (tl[h] + r) & ~(16 / es - 1);  // aligned element offset from tbase - tl
      const unsigned char* src = b + (long long)al * es;
      if (inside) {
        cp16(dst, src, 16);
      } else {
        const long long left = (lim - (tbase[h] - tl[h] + al)) * es - c16;
        const int sb = left >= 16 ? 16 : (left > 0 ? (int)left : 0);
        cp16(dst, sb ? (const void*)src : p.u, sb);
      }
    };

    // copy state of the plane to issue next: row offsets of this lane's rows
    // (u/k rows j0-1+pu / j0-1+pk of plane qi, f row j0+pu of plane qi-1), the
    // row lengths there, and the plane sizes of qi and qi-1
    int qi = q_first;
    int ou = row_offset(N, qi, j0 - 1 + pu), ok_ = row_offset(N, qi, j0 - 1 + pk), of = row_offset(N, qi - 1, j0 + pu);
    int du = N - qi + 1 - (j0 - 1 + pu), dk_ = N - qi + 1 - (j0 - 1 + pk), df = N - qi + 2 - (j0 + pu);
    int Pu = (N - qi + 1) * (N - qi + 2) / 2, Pf = (N - qi + 2) * (N - qi + 3) / 2;
    // copies of plane qi (u, k) and of f of plane qi-1 into the next stage;
    // always one commit group (empty past the item's last plane)
    auto issue = [&]() {
      const unsigned st = ring_s + (g % S) * G::SB;
      if (qi <= k1 + 1) {
#pragma unroll
        for (int h = 0; h < P; ++h) {
#pragma unroll
          for (int Q = 0; Q < kRowsM; Q += G::RPU)
            if (cpu_on && pu + Q < kRowsM)
              chunk(st + (h * kRowsM + pu + Q) * G::RU + 16 * cu, bu[h], EU, p.lim_u, h, ou + Q * du - Q * (Q - 1) / 2,
                    16 * cu);
#pragma unroll
          for (int Q = 0; Q < kRowsM; Q += G::RPK)
            if (cpk_on && pk + Q < kRowsM)
              chunk(st + G::OFF_K + (h * kRowsM + pk + Q) * G::RK + 16 * ck, bk[h], EK, p.lim_k, h,
                    ok_ + Q * dk_ - Q * (Q - 1) / 2, 16 * ck);
          if (G::F && qi - 1 >= k0) {
#pragma unroll
            for (int Q = 0; Q < 4; Q += G::RPU)
              if (cpu_on && pu + Q < 4)
                chunk(st + G::OFF_F + (h * 4 + pu + Q) * G::RU + 16 * cu, bf[h], EU, p.lim_u, h,
                      of + Q * df - Q * (Q - 1) / 2, 16 * cu);
          }
        }
      }
      cp_commit();
      ++g;
      // advance to plane qi+1 (row offset of row j grows by the plane size - j)
      ou += Pu - (j0 - 1 + pu);
      ok_ += Pu - (j0 - 1 + pk);
      of += Pf - (j0 + pu);
      --du;
      --dk_;
      --df;
      Pf = Pu;
      Pu -= N - qi + 1;
      ++qi;
    };

    const unsigned g_item = g;  // group of plane q_first
#pragma unroll
    for (int t = 0; t < S - 1; ++t) issue();

    // thread state
    PT xu[2][kRowsM], xk[2][kRowsM];  // planes (two buffers, roles alternate)
    int rs[kRowsM];                   // row offsets in the tet of the plane being computed
    PT F2p[4], F4c[4], F5c[4], F6p[5];  // carried fluxes
    PT kp[5], dkp[4];                   // plane q-1: own k (rows 1..5), right k (rows 1..4)
#pragma unroll
    for (int m = 0; m < kRowsM; ++m) rs[m] = row_offset(N, q_first, j0 - 1 + m);
    // row m of plane q+1 starts at rs[m] + dlt(q) - m
    auto dlt_of = [&](int q) { return (N - q + 1) * (N - q + 2) / 2 - (j0 - 1); };

    // read plane q into buffer b (its stage stays valid until the next release)
    auto stage_of = [&](int q) { return ring + ((g_item + (unsigned)(q - q_first)) % S) * G::SB; };
    auto consume = [&](int b, int q, int dl, int dm) {  // rows of plane q at rs[m] + dl - dm m
      cp_wait<S - 2>();  // this lane's copies of plane q have landed
      __syncwarp();      // ... and every other lane's
      const unsigned char* sb = stage_of(q);
#pragma unroll
      for (int m = 0; m < kRowsM; ++m) {
        T uv[2], kv[2];
#pragma unroll
        for (int h = 0; h < P; ++h) {
          const int t = tl[h] + rs[m] + dl - dm * m;
          uv[h] = reinterpret_cast<const T*>(sb + (h * kRowsM + m) * G::RU)[(t & (G::VU - 1)) + lane];
          kv[h] = to_t<T, KT>(reinterpret_cast<const KT*>(sb + G::OFF_K + (h * kRowsM + m) * G::RK)[(t & (G::VK - 1)) + lane]);
        }
        xu[b][m] = V::make(uv[0], uv[P - 1]);
        xk[b][m] = V::make(kv[0], kv[P - 1]);
      }
    };
    auto advance_rows = [&](int dl) {
#pragma unroll
      for (int m = 0; m < kRowsM; ++m) rs[m] += dl - m;
    };
    // the stage read before the last one is free: refill it with the next plane
    auto release = [&]() {
      __syncwarp();  // every lane is done with the stages it has read
      issue();
    };
    // f at row m of plane q (buffer a's rows), tet half h: carried by the
    // stage of plane q+1
    auto f_at = [&](int q, int m, int h) -> T {
      const unsigned char* sb = stage_of(q + 1);
      const int t = tl[h] + rs[m];
      return reinterpret_cast<const T*>(sb + G::OFF_F + (h * 4 + m - 1) * G::RU)[(t & (G::VU - 1)) + lane];
    };
    auto flux = [&](PT ua, PT ka, PT ub, PT kb) { return V::mul(V::add(ka, kb), V::sub(ub, ua)); };
    T* __restrict__ po[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) po[h] = static_cast<T*>(p.out) + tbase[h] + lane;
    const bool own_lane = lane >= 1 && lane <= kCols;

    // prologue: planes k0-1 (buffer 0) and k0 (buffer 1); carried fluxes of plane k0
    consume(0, q_first, 0, 0);
    release();
    {
      const int dl = dlt_of(q_first);
      consume(1, k0, dl, 1);
      release();
      advance_rows(dl);
    }
    // right neighbours (lane L+1) are shuffled where they are used
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
      const PT d0u = V::down(xu[0][m]), d0k = V::down(xk[0][m]);
      const PT d1u = V::down(xu[1][m - 1]), d1k = V::down(xk[1][m - 1]);
      F2p[m - 1] = flux(xu[0][m], xk[0][m], xu[1][m], xk[1][m]);
      F6p[m - 1] = flux(xu[0][m], xk[0][m], d1u, d1k);
      F4c[m - 1] = flux(xu[1][m], xk[1][m], d0u, d0k);
      F5c[m - 1] = flux(xu[1][m], xk[1][m], xu[0][m + 1], xk[0][m + 1]);
      if (DIAG) dkp[m - 1] = d0k;
    }
    F6p[4] = flux(xu[0][5], xk[0][5], V::down(xu[1][4]), V::down(xk[1][4]));
    if (DIAG) {
#pragma unroll
      for (int m = 1; m <= 5; ++m) kp[m - 1] = xk[0][m];
    }

    // step of plane q: buffer a holds plane q, buffer b receives plane q+1
    auto step = [&](auto ac, int q) {
      constexpr int a = decltype(ac)::value, b = 1 - a;
      const int dl = dlt_of(q);
      consume(b, q + 1, dl, 1);
      // row m of this lane holds a volume node iff m <= mlim
      const int mlim = N - q - (i0 - 1 + lane) - (j0 - 1) - 1;
      PT F1prev = flux(xu[a][0], xk[a][0], xu[a][1], xk[a][1]);
      PT F5prev = flux(xu[b][0], xk[b][0], xu[a][1], xk[a][1]);
      PT dak = V::down(xk[a][0]);  // k at (i+1, row m-1) of plane q
      PT F3cur = flux(xu[a][1], xk[a][1], V::down(xu[a][0]), dak);
#pragma unroll
      for (int m = 1; m <= 4; ++m) {
        const PT dau = V::down(xu[a][m]), dakm = V::down(xk[a][m]);          // (i+1, row m), plane q
        const PT dbu = V::down(xu[b][m - 1]), dbk = V::down(xk[b][m - 1]);  // (i+1, row m-1), plane q+1
        const PT F0 = flux(xu[a][m], xk[a][m], dau, dakm);
        const PT F1 = flux(xu[a][m], xk[a][m], xu[a][m + 1], xk[a][m + 1]);
        const PT F2 = flux(xu[a][m], xk[a][m], xu[b][m], xk[b][m]);
        const PT F3n = flux(xu[a][m + 1], xk[a][m + 1], dau, dakm);
        const PT F6 = flux(xu[a][m], xk[a][m], dbu, dbk);
        const PT F4n = flux(xu[b][m], xk[b][m], dau, dakm);
        const PT F5n = flux(xu[b][m], xk[b][m], xu[a][m + 1], xk[a][m + 1]);
        const PT t0 = V::mul(c[0], F0);
        PT H = V::fma(c[3], F3n, t0);
        H = V::fma(c[4], F4n, H);
        H = V::fma(c[6], F6p[m], H);  // F6p[m] holds row m+1
        PT y = V::fma(c[1], V::sub(F1, F1prev), t0);
        y = V::fma(c[2], V::sub(F2, F2p[m - 1]), y);
        y = V::fma(c[3], F3cur, y);
        y = V::fma(c[4], F4c[m - 1], y);
        y = V::fma(c[5], V::sub(F5c[m - 1], F5prev), y);
        y = V::fma(c[6], F6, y);
        y = V::sub(y, V::up(H));
        PT dg = y;
        if (DIAG) {
          PT sk = V::mul(c[0], dakm);
          sk = V::fma(c[1], V::add(xk[a][m + 1], xk[a][m - 1]), sk);
          sk = V::fma(c[2], V::add(xk[b][m], kp[m - 1]), sk);
          sk = V::fma(c[3], dak, sk);
          sk = V::fma(c[4], dkp[m - 1], sk);
          sk = V::fma(c[5], V::add(kp[m], xk[b][m - 1]), sk);
          sk = V::fma(c[6], dbk, sk);
          PT hd = V::mul(c[0], xk[a][m]);
          hd = V::fma(c[3], xk[a][m + 1], hd);
          hd = V::fma(c[4], xk[b][m], hd);
          hd = V::fma(c[6], kp[m], hd);
          sk = V::add(sk, V::up(hd));
          dg = V::fma(csum, xk[a][m], sk);  // -diagonal
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
        // epilogue: owned lanes, volume nodes only
        if (own_lane && m <= mlim) {
#pragma unroll
          for (int h = 0; h < P; ++h) {
            if (h == 1 && !hasB) break;
            T* o = po[h] + rs[m];
            const T yv = V::get(y, h);
            if (MODE == OP_APPLY) {
              *o = yv;
            } else if (MODE == OP_RESID) {
              *o = f_at(q, m, h) - yv;
            } else if (MODE == OP_JACOBI) {
              const T diag = -V::get(dg, h);
              *o = V::get(xu[a][m], h) + qdiv((T)p.omega * (f_at(q, m, h) - yv), diag);
            } else if (MODE == OP_CHEB) {
              const T diag = -V::get(dg, h);
              const long long idx = o - static_cast<T*>(p.out);
              const T prev = p.ca != 0.0 ? (T)p.ca * __ldg(static_cast<const T*>(p.d_in) + idx) : (T)0;
              const T dn = prev + (T)p.cb * (f_at(q, m, h) - yv) / diag;
              static_cast<T*>(p.d_out)[idx] = dn;
              *o = V::get(xu[a][m], h) + dn;
            } else {  // OP_DIAG
              *o = -V::get(dg, h);
            }
          }
        }
      }
      F6p[4] = flux(xu[a][5], xk[a][5], V::down(xu[b][4]), V::down(xk[b][4]));
      if (DIAG) {
#pragma unroll
        for (int m = 1; m <= 5; ++m) kp[m - 1] = xk[a][m];
      }
      advance_rows(dl);
      release();
    };

    for (int q = k0; q <= k1; q += 2) {
      step(std::integral_constant<int, 1>{}, q);
      if (q + 1 > k1) break;
      step(std::integral_constant<int, 0>{}, q + 1);
    }
  }
  cp_wait<0>();
}

template <class T, class KT, int P, int MODE>
int march_occupancy() {
  static int occ = 0;
  if (!occ) {
    using G = Geo<T, KT, P, MODE>;
    HHG_CUDA(cudaFuncSetAttribute(march_kernel<T, KT, P, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM));
    HHG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, march_kernel<T, KT, P, MODE>, kWarps * 32, G::SMEM));
    if (occ < 1) occ = 1;
  }
  return occ;
}

template <class T, class KT, int P, int MODE>
void launch_t(const Mesh& m, int depth, const OpArgs& a, const void* kptr, long long lim_k, int n_items,
              cudaStream_t s) {
  using G = Geo<T, KT, P, MODE>;
  const Depth& Dh = m.depth[depth];
  const int occ = march_occupancy<T, KT, P, MODE>();
  const int blocks = std::min((n_items + kWarps - 1) / kWarps, m.num_sms * occ);
  MarchPtrs p{a.u, kptr, a.f, a.out, a.d_in, a.d_out, a.omega, a.ca, a.cb, Dh.n_stored, lim_k};
  const T* sten = sizeof(T) == 8 ? reinterpret_cast<const T*>(Dh.dev.sten64) : reinterpret_cast<const T*>(Dh.dev.sten32);
  march_kernel<T, KT, P, MODE><<<blocks, kWarps * 32, G::SMEM, s>>>(Dh.dev, sten, p, n_items);
  HHG_CUDA(cudaGetLastError());
}

template <int MODE>
void launch_mode(const Mesh& m, int depth, int dtype, const OpArgs& a, int n_items, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  const long long n = Dh.n_stored;
  if (dtype == HHG_F64)
    launch_t<double, double, 1, MODE>(m, depth, a, Dh.k64, n + kCoefPad / 8, n_items, s);
  else if (dtype == kF64KBF16)
    launch_t<double, double, 1, MODE>(m, depth, a, Dh.k16d, n + kCoefPad / 8, n_items, s);
  else if (dtype == HHG_F32)
    (m.vkernel == 1 ? launch_t<float, float, 2, MODE> : launch_t<float, float, 1, MODE>)(m, depth, a, Dh.k32,
                                                                                          n + kCoefPad / 4, n_items, s);
  else
    (m.vkernel == 1 ? launch_t<float, __nv_bfloat16, 2, MODE>
                    : launch_t<float, __nv_bfloat16, 1, MODE>)(m, depth, a, Dh.k16, n + kCoefPad / 2, n_items, s);
}

template <class T, class KT, int P>
void init_t() {
  march_occupancy<T, KT, P, OP_APPLY>();
  march_occupancy<T, KT, P, OP_RESID>();
  march_occupancy<T, KT, P, OP_JACOBI>();
  march_occupancy<T, KT, P, OP_CHEB>();
  march_occupancy<T, KT, P, OP_DIAG>();
}

}  // namespace

void init_march_configs(int dtype) {
  if (dtype == HHG_F64 || dtype == kF64KBF16)
    init_t<double, double, 1>();
  else if (dtype == HHG_F32) {
    init_t<float, float, 2>();
    init_t<float, float, 1>();
  } else {
    init_t<float, __nv_bfloat16, 2>();
    init_t<float, __nv_bfloat16, 1>();
  }
}

void launch_march(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, cudaStream_t s) {
  const DepthDev& D = m.depth[depth].dev;
  const bool paired = (dtype == HHG_F32 || dtype == HHG_F32_KBF16) && m.vkernel == 1;
  const int n_items = paired ? (a.nc_only ? D.n_mitems_nc : D.n_mitems) : (a.nc_only ? D.n_sitems_nc : D.n_sitems);
  if (n_items == 0) return;
  switch (mode) {
    case OP_APPLY: launch_mode<OP_APPLY>(m, depth, dtype, a, n_items, s); break;
    case OP_RESID: launch_mode<OP_RESID>(m, depth, dtype, a, n_items, s); break;
    case OP_JACOBI: launch_mode<OP_JACOBI>(m, depth, dtype, a, n_items, s); break;
    case OP_CHEB: launch_mode<OP_CHEB>(m, depth, dtype, a, n_items, s); break;
    case OP_DIAG: launch_mode<OP_DIAG>(m, depth, dtype, a, n_items, s); break;
  }
}

// Work lists of the march.  Pairs: tets paired by class (above the coarsest
// level first) and level, an odd one out alone; singles: every tet alone.
// Per pair (or single), tiles (i0, j0) of 30 columns x 4 rows, each tile's
// planes 1 .. N-1-i0-j0 cut into segments of kseg planes; longest segment
// first within a class.  kseg is halved (down to 4) while a class would have
// fewer items than resident warps.
void build_march_items(const Mesh& m, Depth& D) {
  const int ns = (int)D.slot_tet.size();
  D.h_pairs.clear();
  const long long target = (long long)(m.num_sms > 0 ? m.num_sms : 152) * 12;
  std::vector<int4> lists[2][2];  // [paired][class]
  for (int paired = 1; paired >= 0; --paired)
    for (int cls = 0; cls < 2; ++cls) {
      std::map<int, std::vector<int>> by_n;
      for (int s = 0; s < ns; ++s)
        if ((s < D.n_slots_nc) == (cls == 0)) by_n[D.h_tets[s].N].push_back(s);
      std::vector<std::pair<int, int>> prs;  // (pair index, N)
      const size_t step = paired ? 2 : 1;
      for (auto& kv : by_n)
        for (size_t a = 0; a < kv.second.size(); a += step) {
          const int sb = paired && a + 1 < kv.second.size() ? kv.second[a + 1] : -1;
          prs.push_back({(int)D.h_pairs.size(), kv.first});
          D.h_pairs.push_back(make_int2(kv.second[a], sb));
        }
      auto count = [&](int ks) {
        long long c = 0;
        for (auto& pn : prs) {
          const int N = pn.second;
          for (int j0 = 1; j0 <= N - 2; j0 += 4)
            for (int i0 = 1; i0 + j0 <= N - 2; i0 += kCols) c += (N - 1 - (i0 + j0) + ks - 1) / ks;
        }
        return c;
      };
      int ks = std::max(1, m.kseg);
      while (ks > 4 && count(ks) < target) ks /= 2;
      std::vector<std::pair<int, int4>> its;
      for (auto& pn : prs) {
        const int N = pn.second;
        for (int j0 = 1; j0 <= N - 2; j0 += 4)
          for (int i0 = 1; i0 + j0 <= N - 2; i0 += kCols) {
            const int top = N - 1 - (i0 + j0);
            for (int k0 = 1; k0 <= top; k0 += ks) {
              const int k1 = std::min(top, k0 + ks - 1);
              its.push_back({-(k1 - k0 + 1), make_int4(pn.first, i0 | j0 << 16, k0, k1)});
            }
          }
      }
      std::stable_sort(its.begin(), its.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
      for (auto& e : its) lists[paired][cls].push_back(e.second);
    }
  D.h_mitems = lists[1][0];
  D.n_mitems_nc = (int)lists[1][0].size();
  D.h_mitems.insert(D.h_mitems.end(), lists[1][1].begin(), lists[1][1].end());
  D.n_mitems = (int)D.h_mitems.size();
  D.h_sitems = lists[0][0];
  D.n_sitems_nc = (int)lists[0][0].size();
  D.h_sitems.insert(D.h_sitems.end(), lists[0][1].begin(), lists[0][1].end());
  D.n_sitems = (int)D.h_sitems.size();
}

}  // namespace hhg
