// Stencil-scaled operator (Sec. 6.1, eq. "discrete"), fused with the residual,
// damped Jacobi and Chebyshev updates.
//
// Row of node x of macro tet T (partial row if x lies on a macro face):
//     (A u)_x = sum_d c_d^{prim(x)} (k_x + k_{x+w_d}) (u_{x+w_d} - u_x)
// with c = (1/2) reference stencil of x's primitive and the diagonal implied
// by the zero row sum.  Written per edge (x, x+w): F = c_w (k_x + k_{x+w})
// (u_{x+w} - u_x) enters row x with + and row x+w with -.  The coefficient of
// an edge is the volume stencil's unless both ends lie on a common macro face
// (then it is that face primitive's entry) or one end lies outside T (0).
//
// One apply is three launches:
//  1. tile kernel: every volume row, the partial rows of the copies on the
//     macro face i = 0 (away from the faces j = 0, k = 0), and the Dirichlet
//     zeros of the face i + j + k = N it passes;
//  2. copy kernel (concurrent, side stream): partial rows (or Dirichlet
//     zeros) of all other macro-face, edge and vertex copies;
//  3. sum kernel: every non-Dirichlet interface node adds the partial rows of
//     its copies, applies the mode's epilogue and writes all copies.
//
// Tile kernel.  A work item is a 16 (i) x 8 (j) tile of TWO macro tets of the
// same level, marched along k over a segment of planes: all index arithmetic
// is shared by the two tets and FP32 work runs in packed f32x2 instructions,
// one half per tet (FP64: one tet at a time).  Lane (li, lj) = (lane % 8,
// lane / 8) owns the 2 x 2 nodes i0 + 2li + {0,1}, j0 + 2lj + {0,1} of each
// tet.  The tile's footprint of every plane (rows j0-1 .. j0+8, columns
// i0-1 .. i0+16, u and k of both tets) is staged in a 4-plane shared-memory
// ring per warp with 16-byte cp.async copies (two planes in flight, completion
// by cp.async groups: no spin loop).  When plane q has landed, each lane
// computes every edge between planes q-1 and q and inside plane q that
// touches its nodes; plane q-1's rows are then complete and stored.
#include <algorithm>
#include <map>
#include <utility>

#include "hhg_internal.h"

namespace hhg {

size_t elem_size(int dtype);

namespace {

constexpr int kTI = 16;          // tile columns
constexpr int kTJ2 = 8;          // tile rows
constexpr int kSR = kTJ2 + 2;    // staged rows j0-1 .. j0+8
#ifndef HHG_TSTAGES
#define HHG_TSTAGES 4
#endif
#ifndef HHG_TMINB
#define HHG_TMINB 3
#endif
constexpr int kNS = HHG_TSTAGES;  // ring stages per warp (kNS - 2 planes in flight)
static_assert(kNS >= 3, "the ring needs a stage being read, one being filled and one in flight");
#ifndef HHG_TPIN
#define HHG_TPIN 1
#endif

// Staged row geometry of element type E: a row copy starts at the 16-byte
// boundary at or below column i0-1 and covers columns i0-1 .. i0+16.
template <class E>
struct SG {
  static constexpr int V = 16 / (int)sizeof(E);                  // elements per chunk
  static constexpr int CH = (kTI + 2 + 2 * (V - 1) + V - 1) / V;  // chunks a row may need
  static constexpr int R = 32 / CH;                              // rows per copy round
  static constexpr int PITCH = sizeof(E) == 4 ? 28 : (sizeof(E) == 8 ? 24 : 48);  // elements per staged row
  static constexpr int PB = PITCH * (int)sizeof(E);
  static constexpr int BYTES = kSR * PB;
  static_assert(CH * V <= PITCH, "staged row too short");
};

// lane vector: two tets in the halves of an f32x2 (FP32), one tet (FP64)
template <class T>
struct LaneV;
template <>
struct LaneV<float> {
  using V = float2;
  static constexpr int NT = 2;
};
template <>
struct LaneV<double> {
  using V = double;
  static constexpr int NT = 1;
};

__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vnfma(float2 a, float2 b, float2 c) {
  return __ffma2_rn(make_float2(-a.x, -a.y), b, c);
}
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ double vmul(double a, double b) { return a * b; }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double vnfma(double a, double b, double c) { return fma(-a, b, c); }

template <class V>
__device__ __forceinline__ V vzero();
template <>
__device__ __forceinline__ float2 vzero<float2>() {
  return make_float2(0.f, 0.f);
}
template <>
__device__ __forceinline__ double vzero<double>() {
  return 0.0;
}

// component t of a lane vector
__device__ __forceinline__ float& comp(float2& v, int t) { return t ? v.y : v.x; }
__device__ __forceinline__ float comp(const float2& v, int t) { return t ? v.y : v.x; }
__device__ __forceinline__ double& comp(double& v, int) { return v; }
__device__ __forceinline__ double comp(const double& v, int) { return v; }

template <class V>
struct NV {
  V u, k;
};

template <class V, bool DIAG>
struct Acc {
  V y, d;
};

// Edge from a to b, coefficient c: row a only.
template <class V, bool DIAG>
__device__ __forceinline__ void edge1(const NV<V>& a, const NV<V>& b, V c, Acc<V, DIAG>& A) {
  const V du = vsub(b.u, a.u);
  const V s = vmul(c, vadd(b.k, a.k));
  A.y = vfma(s, du, A.y);
  if (DIAG) A.d = vsub(A.d, s);
}
// Edge from a to b: rows a (+F) and b (-F).
template <class V, bool DIAG>
__device__ __forceinline__ void edge2(const NV<V>& a, const NV<V>& b, V c, Acc<V, DIAG>& A, Acc<V, DIAG>& B) {
  const V du = vsub(b.u, a.u);
  const V s = vmul(c, vadd(b.k, a.k));
  A.y = vfma(s, du, A.y);
  B.y = vnfma(s, du, B.y);
  if (DIAG) {
    A.d = vsub(A.d, s);
    B.d = vsub(B.d, s);
  }
}

// Register state of one plane: v[row + 1][col + 1] for rows -1..2 and columns
// -1..2 around the lane's patch (14 positions are read; P keeps 10 of them),
// the tet-local offsets of (i0-1, row) for rows 0 and 1 (stores), and f (and
// the previous Chebyshev update) at the lane's nodes, read one step ahead.
template <class V>
struct PlaneR {
  NV<V> v[4][4];
  int off[2];
  V fv[2][2], dv[2][2];
};

// Coefficients of the lane's edge slots.  Column a = 0 of the patch is the
// macro face i = 0 for lane li = 0 of tiles with i0 = 0 ("col" lanes): there
// the edges inside the column (e2, e3, e2-e3) take the face primitive's
// entries (c2F, c3F, c23F) and the edges leaving T towards i = -1 are 0 (c1M,
// c12M, c13M, cgM); every other slot takes the volume stencil.
template <class V>
struct Coef {
  V c1, c2, c3, c12, c13, c23, cg;
  V c2F, c3F, c23F, c1M, c12M, c13M, cgM;
};

// Read head of a plane: tet-local offset e0 of (i0-1, jr, q), length A of row
// jr in plane q, nodes Psz in plane q.
struct PHead {
  int e0, A, Psz, q;
  __device__ __forceinline__ void next(int N, int jr) {
    e0 += Psz - jr;
    Psz -= N - q + 1;
    A -= 1;
    ++q;
  }
  __device__ __forceinline__ void init(int N, int jr, int i0, int q0) {
    const int M = N - q0;
    q = q0;
    Psz = (M + 1) * (M + 2) / 2;
    A = M - jr + 1;
    const int pl = (int)(tetnum(N + 1) - tetnum(N + 1 - q0));
    e0 = pl + jr * (M + 1) - jr * (jr - 1) / 2 + (i0 - 1);
  }
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cpa16(unsigned dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
template <int OFF>
__device__ __forceinline__ void cpa16_if(bool pred, unsigned dst, const void* src) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n @p cp.async.cg.shared.global [%0+%3], [%1], 16;\n}\n" ::"r"(dst),
      "l"(src), "r"((int)pred), "n"(OFF)
      : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copies of one array of one tet for staged plane H.q.  Lane = CH p + c
// copies chunk c of rows p, p + R, ... (one instruction moves consecutive
// chunks of R rows).  base = the array at the tet base minus bm elements (a
// 16-byte boundary); offb = tet-local offset of (i0-1, j0-1, q) plus bm.
// Fast path (inside): every chunk of the footprint lies in the vector; the
// others check each chunk against [0, lim) of the vector (lim counted from
// the boundary below the tet base) and zero-fill what lies outside.
// Per-lane constants of the copy rounds of element type E: lane = CH p + c
// copies chunk c of rows p, p + R, p + 2R, ... of the footprint.
template <class E>
struct CopyLane {
  static constexpr int NR = (kSR + SG<E>::R - 1) / SG<E>::R;  // rounds
  int p, c;
  int rowc[NR];  // row (row - 1) / 2 for the row of round r
  unsigned act;  // bit r: the lane copies a row in round r
  __device__ __forceinline__ void init(int lane) {
    using G = SG<E>;
    p = lane / G::CH;
    c = lane - p * G::CH;
    act = 0;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int row = p + r * G::R;
      rowc[r] = row * (row - 1) / 2;
      if (p < G::R && row < kSR) act |= 1u << r;
    }
  }
};

// Fast path: every chunk of the item's footprint lies in the vector (checked
// once per item), so each lane copies its CH-th share of every row without a
// test (the chunk past the footprint's end, when a row starts on a 16-byte
// boundary, is copied too).  Row offsets are tet-local and shared by the tets
// of the item; only the chunk alignment (bm) differs between them.
// dst = the stage plus the lane's row p and chunk c; g[t] = the array of tet
// t at its base minus bm[t], plus the lane's chunk.
template <class E, int RB, int TB, int NT, int R, int T0 = 0>
__device__ __forceinline__ void copy_round(const CopyLane<E>& cl, int rowoff, unsigned dst, const E* const (&g)[NT],
                                           const int (&bm)[NT]) {
  if constexpr (T0 < NT) {
    using G = SG<E>;
    const bool on = (cl.act >> R) & 1u;
    const int a = (rowoff + bm[T0]) & ~(G::V - 1);
    cpa16_if<RB + T0 * TB + R * G::R * G::PB>(on, dst, g[T0] + a);
    copy_round<E, RB, TB, NT, R, T0 + 1>(cl, rowoff, dst, g, bm);
  }
}
template <class E, class E2, int RB, int RB2, int TB, int NT, int R, int T0 = 0>
__device__ __forceinline__ void copy_round2(const CopyLane<E>& cl, int rowoff, unsigned dst, const E* const (&g)[NT],
                                            const E2* const (&g2)[NT], const int (&bm)[NT]) {
  if constexpr (T0 < NT) {
    using G = SG<E>;
    const bool on = (cl.act >> R) & 1u;
    const int a = (rowoff + bm[T0]) & ~(G::V - 1);
    cpa16_if<RB + T0 * TB + R * G::R * G::PB>(on, dst, g[T0] + a);
    cpa16_if<RB2 + T0 * TB + R * G::R * G::PB>(on, dst, reinterpret_cast<const E*>(g2[T0]) + a);
    copy_round2<E, E2, RB, RB2, TB, NT, R, T0 + 1>(cl, rowoff, dst, g, g2, bm);
  }
}
template <class E, int R>
__device__ __forceinline__ int round_off(const CopyLane<E>& cl, int pA, const PHead& H) {
  // tet-local offset of (i0-1, j0-1+row, q), row = p + R*SG<E>::R
  return H.e0 + pA + R * SG<E>::R * H.A - cl.rowc[R];
}

template <class E>
__device__ __noinline__ void copy_rows_checked(int offb, int A, int p, int c, unsigned dst, const E* base, int lo,
                                               int hi) {
  using G = SG<E>;
#pragma unroll
  for (int Q = 0; Q < kSR; Q += G::R) {
    const int row = p + Q;
    const int eb = offb + row * A - row * (row - 1) / 2;
    const int mis = eb & (G::V - 1);
    if (p < G::R && row < kSR && mis >= c * G::V - (kTI + 1)) {
      const int a = eb - mis + c * G::V;  // chunk start, elements from base
      const unsigned d = dst + Q * G::PB;
      if (a < lo) {
        cpa16(d, base, 0);  // before the vector: zero-fill
      } else {
        const int rem = hi - a;  // elements of the vector from the chunk start on
        if (rem >= G::V)
          cpa16(d, base + a, 16);
        else
          cpa16(d, rem > 0 ? (const void*)(base + a) : (const void*)(base + lo), rem > 0 ? rem * (int)sizeof(E) : 0);
      }
    }
  }
}

template <class T, class KT>
struct Stage {
  static constexpr int NT = LaneV<T>::NT;
  static constexpr int UB = SG<T>::BYTES;
  static constexpr int KB = SG<KT>::BYTES;
  static constexpr int TB = UB + KB;  // one tet
  static constexpr int SB = NT * TB;  // one stage
  static constexpr int WB = kNS * SB;  // one warp's ring
};

// Per-tet data of an item (vectors hold fewer than 2^31 entries).
template <class T, class KT>
struct TetPtrs {
  const T* u;   // u at the tet base minus bm = base mod (elements per chunk of T)
  const KT* k;  // k at the tet base minus bmk = base mod (elements per chunk of KT)
  int base;     // tet base in the depth vector
  __device__ __forceinline__ int bm() const { return base & (SG<T>::V - 1); }
  __device__ __forceinline__ int bmk() const { return base & (SG<KT>::V - 1); }
};

// Stage plane H.q of both tets (nothing if !want).  fast: the item's whole
// footprint lies inside the vector (decided once per item); otherwise every
// chunk is checked against the vector's ends.  du/dk = the stage plus the
// lane's copy slot for u and k; gu/gk = the tets' arrays plus the lane's chunk.
template <class T, class KT>
__device__ __forceinline__ void issue_plane(unsigned stage, const PHead& H, const CopyLane<T>& cu,
                                            const CopyLane<KT>& ckl, int nst,
                                            const TetPtrs<T, KT> (&tp)[LaneV<T>::NT], const T* const (&gu)[LaneV<T>::NT],
                                            const KT* const (&gk)[LaneV<T>::NT], bool want, bool fast) {
  using S = Stage<T, KT>;
  using GU = SG<T>;
  using GK = SG<KT>;
  constexpr int NT = S::NT;
  if (!want) return;
  const unsigned du = stage + cu.p * GU::PB + 16 * cu.c;
  int bm[NT], bmk[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    bm[t] = tp[t].bm();
    bmk[t] = tp[t].bmk();
  }
  if (fast) {
    const int pA = cu.p * H.A;
    if constexpr (sizeof(T) == sizeof(KT)) {
      copy_round2<T, KT, 0, S::UB, S::TB, NT, 0>(cu, round_off<T, 0>(cu, pA, H), du, gu, gk, bm);
      if constexpr (CopyLane<T>::NR > 1) copy_round2<T, KT, 0, S::UB, S::TB, NT, 1>(cu, round_off<T, 1>(cu, pA, H), du, gu, gk, bm);
      if constexpr (CopyLane<T>::NR > 2) copy_round2<T, KT, 0, S::UB, S::TB, NT, 2>(cu, round_off<T, 2>(cu, pA, H), du, gu, gk, bm);
      if constexpr (CopyLane<T>::NR > 3) copy_round2<T, KT, 0, S::UB, S::TB, NT, 3>(cu, round_off<T, 3>(cu, pA, H), du, gu, gk, bm);
      static_assert(CopyLane<T>::NR <= 4, "copy rounds");
    } else {
      copy_round<T, 0, S::TB, NT, 0>(cu, round_off<T, 0>(cu, pA, H), du, gu, bm);
      copy_round<T, 0, S::TB, NT, 1>(cu, round_off<T, 1>(cu, pA, H), du, gu, bm);
      static_assert(CopyLane<T>::NR == 2 && CopyLane<KT>::NR == 2, "copy rounds");
      const unsigned dk = stage + ckl.p * GK::PB + 16 * ckl.c;
      const int pAk = ckl.p * H.A;
      copy_round<KT, S::UB, S::TB, NT, 0>(ckl, round_off<KT, 0>(ckl, pAk, H), dk, gk, bmk);
      copy_round<KT, S::UB, S::TB, NT, 1>(ckl, round_off<KT, 1>(ckl, pAk, H), dk, gk, bmk);
    }
    return;
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int lo = bm[t] - tp[t].base, hi = nst - tp[t].base + bm[t];
    const int lok = bmk[t] - tp[t].base, hik = nst - tp[t].base + bmk[t];
    copy_rows_checked<T>(H.e0 + bm[t], H.A, cu.p, cu.c, du + t * S::TB, tp[t].u, lo, hi);
    const unsigned dk = stage + ckl.p * GK::PB + 16 * ckl.c + S::UB + t * S::TB;
    copy_rows_checked<KT>(H.e0 + bmk[t], H.A, ckl.p, ckl.c, dk, tp[t].k, lok, hik);
  }
}

// Does the footprint of planes q0 .. q1 of tile (i0, j0) lie inside the
// vector for array geometry G (b = tet base mod G::V)?  Row r of plane q
// starts at e0(q) + r A(q) - r (r - 1) / 2: e0 grows with q, the row term is
// concave in r and shrinks with A, so the lowest start is row 0 or kSR-1 of
// the last plane's shape at the first plane and the highest end is the first
// plane's widest row at the last plane.
template <class G>
__device__ __forceinline__ bool footprint_inside(int N, int i0, int j0, int q0, int q1, int base, int nst) {
  PHead a, b;
  a.init(N, j0 - 1, i0, q0);
  b.init(N, j0 - 1, i0, q1);
  const int bm = base & (G::V - 1);
  const int fmin = min(0, (kSR - 1) * b.A - (kSR - 1) * (kSR - 2) / 2);
  const int rmax = min(kSR - 1, max(a.A, 0));
  const int fmax = rmax * a.A - rmax * (rmax - 1) / 2;
  const long long first = (long long)base - bm + ((a.e0 + bm + fmin) & ~(G::V - 1));
  const long long last = (long long)base + b.e0 + fmax + G::CH * G::V;
  return first >= 0 && last <= nst;
}

// a staged coefficient in the arithmetic type T (bfloat16 widened to FP32)
template <class T, class E>
__device__ __forceinline__ T ldsk(const E* p) {
  if constexpr (sizeof(E) == 2)
    return (T)__bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
  else
    return (T)*p;
}

// Read the lane's positions of a staged plane (ring = the warp's ring); rows
// m = 0..3 are rows jb-1+m, the lane's columns start 2 li after column i0-1.
template <class T, class KT>
__device__ __forceinline__ void read_plane(PlaneR<typename LaneV<T>::V>& P, const unsigned char* stage, int li, int lj,
                                           const PHead& rh, const TetPtrs<T, KT> (&tp)[LaneV<T>::NT]) {
  using S = Stage<T, KT>;
  using GU = SG<T>;
  using GK = SG<KT>;
  int o[4];
  o[0] = rh.e0;
  o[1] = o[0] + rh.A;
  o[2] = o[1] + rh.A - 1;
  o[3] = o[2] + rh.A - 2;
  P.off[0] = o[1];
  P.off[1] = o[2];
#pragma unroll
  for (int t = 0; t < S::NT; ++t) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int mis = (o[m] + tp[t].bm()) & (GU::V - 1);
      const T* us = reinterpret_cast<const T*>(stage + t * S::TB + (2 * lj + m) * GU::PB) + mis + 2 * li;
      const KT* ks;
      if constexpr (sizeof(KT) == sizeof(T))
        ks = reinterpret_cast<const KT*>(reinterpret_cast<const unsigned char*>(us) + S::UB);
      else
        ks = reinterpret_cast<const KT*>(stage + t * S::TB + S::UB + (2 * lj + m) * GK::PB) +
             ((o[m] + tp[t].bmk()) & (GK::V - 1)) + 2 * li;
      const int c_lo = m == 0 ? 1 : 0, c_hi = m == 3 ? 2 : 3;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        if (cc < c_lo || cc > c_hi) continue;
        comp(P.v[m][cc].u, t) = us[cc];
        comp(P.v[m][cc].k, t) = ldsk<T>(ks + cc);
      }
    }
  }
}

// Keep the positions the next step uses as its plane q-1 in registers (the
// compiler would otherwise re-read them from the staged plane).
__device__ __forceinline__ void pin(float2& v) { asm volatile("" : "+f"(v.x), "+f"(v.y)); }
__device__ __forceinline__ void pin(double& v) { asm volatile("" : "+d"(v)); }
template <class V>
__device__ __forceinline__ void pin_kept(PlaneR<V>& Q) {
#pragma unroll
  for (int m = 1; m < 4; ++m)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      if ((m == 1 && cc == 0) || (m == 3 && cc == 3)) continue;
      pin(Q.v[m][cc].u);
      pin(Q.v[m][cc].k);
    }
}

// All edges of one march step (P = plane q-1, Q = plane q); see the header.
template <class V, bool DIAG>
__device__ __forceinline__ void step_edges(const PlaneR<V>& P, const PlaneR<V>& Q, const Coef<V>& c,
                                           Acc<V, DIAG> (&yP)[2][2], Acc<V, DIAG> (&yQ)[2][2]) {
#define PV(a, b) P.v[(b) + 1][(a) + 1]
#define QV(a, b) Q.v[(b) + 1][(a) + 1]
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      yQ[a][b].y = vzero<V>();
      if (DIAG) yQ[a][b].d = vzero<V>();
    }
  // (A) edges between planes q-1 and q
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    edge2(PV(0, b), QV(0, b), c.c3F, yP[0][b], yQ[0][b]);  // e3
    edge2(PV(1, b), QV(1, b), c.c3, yP[1][b], yQ[1][b]);
    edge2(PV(1, b), QV(0, b), c.c13, yP[1][b], yQ[0][b]);  // -(e1-e3) from P(1,b) = e1-e3 from Q(0,b)
    edge1(PV(0, b), QV(-1, b), c.c13M, yP[0][b]);           // -(e1-e3) from P(0,b)
  }
  edge2(PV(0, 1), QV(0, 0), c.c23F, yP[0][1], yQ[0][0]);  // -(e2-e3) from P(a,1) = e2-e3 from Q(a,0)
  edge2(PV(1, 1), QV(1, 0), c.c23, yP[1][1], yQ[1][0]);
  edge1(PV(0, 0), QV(0, -1), c.c23F, yP[0][0]);  // -(e2-e3) from P(a,0)
  edge1(PV(1, 0), QV(1, -1), c.c23, yP[1][0]);
  edge2(PV(0, 1), QV(1, 0), c.cg, yP[0][1], yQ[1][0]);  // e1-e2+e3 from P(0,1) = -(e1-e2+e3) from Q(1,0)
  edge1(PV(0, 0), QV(1, -1), c.cg, yP[0][0]);            // e1-e2+e3 from P(a,b), other ends outside the patch
  edge1(PV(1, 0), QV(2, -1), c.cg, yP[1][0]);
  edge1(PV(1, 1), QV(2, 0), c.cg, yP[1][1]);
  // (A') the remaining edges from plane q down to q-1
#pragma unroll
  for (int b = 0; b < 2; ++b) edge1(QV(1, b), PV(2, b), c.c13, yQ[1][b]);  // e1-e3 from Q(1,b)
  edge1(QV(0, 1), PV(0, 2), c.c23F, yQ[0][1]);                               // e2-e3 from Q(a,1)
  edge1(QV(1, 1), PV(1, 2), c.c23, yQ[1][1]);
#pragma unroll
  for (int b = 0; b < 2; ++b) edge1(QV(0, b), PV(-1, b + 1), c.cgM, yQ[0][b]);  // -(e1-e2+e3) from Q(0,b)
  edge1(QV(1, 1), PV(0, 2), c.cg, yQ[1][1]);                                       // -(e1-e2+e3) from Q(1,1)
  // (B) edges inside plane q
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    edge2(QV(0, b), QV(1, b), c.c1, yQ[0][b], yQ[1][b]);  // e1
    edge1(QV(1, b), QV(2, b), c.c1, yQ[1][b]);
    edge1(QV(0, b), QV(-1, b), c.c1M, yQ[0][b]);  // -e1
  }
  edge2(QV(0, 0), QV(0, 1), c.c2F, yQ[0][0], yQ[0][1]);  // e2
  edge2(QV(1, 0), QV(1, 1), c.c2, yQ[1][0], yQ[1][1]);
  edge1(QV(0, 1), QV(0, 2), c.c2F, yQ[0][1]);
  edge1(QV(1, 1), QV(1, 2), c.c2, yQ[1][1]);
  edge1(QV(0, 0), QV(0, -1), c.c2F, yQ[0][0]);  // -e2
  edge1(QV(1, 0), QV(1, -1), c.c2, yQ[1][0]);
  edge2(QV(0, 1), QV(1, 0), c.c12, yQ[0][1], yQ[1][0]);  // e1-e2 from Q(0,1) = -(e1-e2) from Q(1,0)
  edge1(QV(0, 0), QV(1, -1), c.c12, yQ[0][0]);           // e1-e2
  edge1(QV(1, 0), QV(2, -1), c.c12, yQ[1][0]);
  edge1(QV(1, 1), QV(2, 0), c.c12, yQ[1][1]);
  edge1(QV(0, 0), QV(-1, 1), c.c12M, yQ[0][0]);  // -(e1-e2)
  edge1(QV(0, 1), QV(-1, 2), c.c12M, yQ[0][1]);
  edge1(QV(1, 1), QV(0, 2), c.c12, yQ[1][1]);
#undef PV
#undef QV
}

// Quotient of the damped Jacobi update: the fast division intrinsic in FP32
// (within 2 ulp; the sweep is a preconditioner step and the outer FP64
// residual decides convergence), the correctly rounded one in FP64.
__device__ __forceinline__ float sdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sdiv(double a, double b) { return a / b; }

struct OpPtrs {
  const void* u;
  const void* k;
  const void* f;
  void* out;
  const void* d_in;
  void* d_out;
  double omega, ca, cb;
};

// Final value (and Chebyshev update) of a complete row.
template <class T, int MODE>
__device__ __forceinline__ void final_value(T y, T diag, T ux, T fv, T dv, const OpPtrs& p, T& val, T& dval) {
  dval = 0;
  if (MODE == OP_APPLY) {
    val = y;
  } else if (MODE == OP_RESID) {
    val = fv - y;
  } else if (MODE == OP_JACOBI) {
    val = ux + sdiv((T)p.omega * (fv - y), diag);
  } else if (MODE == OP_CHEB) {
    const T prev = p.ca != 0.0 ? (T)p.ca * dv : (T)0;
    dval = prev + (T)p.cb * (fv - y) / diag;
    val = ux + dval;
  } else {
    val = diag;
  }
}
// Partial row of an interface copy (summed by the sum kernel).
template <class T, int MODE>
__device__ __forceinline__ void store_partial(T y, T diag, T* out) {
  *out = MODE == OP_DIAG ? diag : y;
}
// Row of a Dirichlet node.
template <class T, int MODE>
__device__ __forceinline__ void store_dirichlet(T* out, T* dout) {
  *out = MODE == OP_DIAG ? (T)1 : (T)0;
  if (MODE == OP_CHEB) *dout = (T)0;
}

template <class T>
__device__ __forceinline__ const T* sten_of(const DepthDev& D) {
  if constexpr (sizeof(T) == 8)
    return reinterpret_cast<const T*>(D.sten64);
  else
    return reinterpret_cast<const T*>(D.sten32);
}

// One work item: tile (i0, j0) of the tets in `slots` (NT of them), planes k0..k1.
template <class T, class KT, int MODE>
__device__ void tile_item(const DepthDev& D, const int (&slots)[LaneV<T>::NT], int i0, int j0, int k0,
                          int k1, int lane, const OpPtrs& p, unsigned char* ring, unsigned ring_s) {
  using V = typename LaneV<T>::V;
  constexpr int NT = LaneV<T>::NT;
  constexpr bool DIAG = (MODE == OP_JACOBI || MODE == OP_CHEB || MODE == OP_DIAG);
  constexpr bool PREF = (MODE == OP_RESID || MODE == OP_JACOBI || MODE == OP_CHEB);
  const int N = D.tets[slots[0]].N;
  const int qend = min(k1 + 1, N - (i0 + j0));
  const int li = lane & 7, lj = lane >> 3;
  const int x0 = i0 + 2 * li;
  const int jb = j0 + 2 * lj;
  const bool col = i0 == 0 && li == 0;
  const T* sten = sten_of<T>(D);
  Coef<V> c;
  TetPtrs<T, KT> tp[NT];
  int lb[NT];  // node (x0, row) of plane pl is at lb + (offset of (i0-1, row, pl))
  unsigned dm[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int s = slots[t];
    const T* s0 = sten + s * 16 * kNDir;       // volume row (mask 0)
    const T* s2 = sten + (s * 16 + 2) * kNDir;  // face i = 0 (mask 2)
    comp(c.c1, t) = s0[0];
    comp(c.c2, t) = s0[1];
    comp(c.c3, t) = s0[2];
    comp(c.c12, t) = s0[3];
    comp(c.c13, t) = s0[4];
    comp(c.c23, t) = s0[5];
    comp(c.cg, t) = s0[6];
    comp(c.c2F, t) = col ? s2[1] : s0[1];
    comp(c.c3F, t) = col ? s2[2] : s0[2];
    comp(c.c23F, t) = col ? s2[5] : s0[5];
    comp(c.c1M, t) = col ? (T)0 : s0[0];
    comp(c.c12M, t) = col ? (T)0 : s0[3];
    comp(c.c13M, t) = col ? (T)0 : s0[4];
    comp(c.cgM, t) = col ? (T)0 : s0[6];
    const int base = (int)D.tets[s].base;
    tp[t].base = base;
    tp[t].u = static_cast<const T*>(p.u) + (base - tp[t].bm());
    tp[t].k = static_cast<const KT*>(p.k) + (base - tp[t].bmk());
    lb[t] = base + x0 + 1 - i0;
    dm[t] = D.dmask[s];
  }
  const int nst = (int)D.n_stored;
  T* const out = static_cast<T*>(p.out);
  T* const dout = static_cast<T*>(p.d_out);
  const T* const fvec = static_cast<const T*>(p.f);
  const T* const dinv = static_cast<const T*>(p.d_in);
  PHead ch, rh;
  ch.init(N, j0 - 1, i0, k0 - 1);
  rh.init(N, jb - 1, i0, k0 - 1);
  using S = Stage<T, KT>;
  bool fast = true;
#pragma unroll
  for (int t = 0; t < NT; ++t)
    fast = fast && footprint_inside<SG<T>>(N, i0, j0, k0 - 1, qend, tp[t].base, nst) &&
           footprint_inside<SG<KT>>(N, i0, j0, k0 - 1, qend, tp[t].base, nst);
  CopyLane<T> clu;
  CopyLane<KT> clk;
  clu.init(lane);
  clk.init(lane);
  const T* gu[NT];
  const KT* gk[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    gu[t] = tp[t].u + clu.c * SG<T>::V;
    gk[t] = tp[t].k + (sizeof(T) == sizeof(KT) ? clu.c : clk.c) * SG<KT>::V;
  }
  auto issue_next = [&](int st) {
    issue_plane<T, KT>(ring_s + st * S::SB, ch, clu, clk, nst, tp, gu, gk, ch.q <= qend, fast);
    cpa_commit();
    ch.next(N, j0 - 1);
  };
  auto read_next = [&](int st, PlaneR<V>& P) {
    read_plane<T, KT>(P, ring + st * S::SB, li, lj, rh, tp);
    if constexpr (PREF) {
      const int pl = rh.q;
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const bool ok = pl >= k0 && N - 1 - (x0 + a) - (jb + b) - pl >= 0;
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const int o = lb[t] + P.off[b] + a;
            comp(P.fv[a][b], t) = ok ? __ldg(fvec + o) : (T)0;
            if (MODE == OP_CHEB) comp(P.dv[a][b], t) = ok && p.ca != 0.0 ? __ldg(dinv + o) : (T)0;
          }
        }
    }
    rh.next(N, jb - 1);
  };
  // store the completed plane pl (rows of P)
  auto store = [&](const PlaneR<V>& P, Acc<V, DIAG> (&y)[2][2], int pl) {
    const bool interior = i0 > 0 && (i0 + kTI - 1) + (j0 + kTJ2 - 1) + pl <= N - 1;
    if (interior) {
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const int o = lb[t] + P.off[b] + a;
            T val, dval;
            final_value<T, MODE>(comp(y[a][b].y, t), DIAG ? comp(y[a][b].d, t) : (T)0, comp(P.v[b + 1][a + 1].u, t),
                                 PREF ? comp(P.fv[a][b], t) : (T)0, MODE == OP_CHEB ? comp(P.dv[a][b], t) : (T)0, p,
                                 val, dval);
            out[o] = val;
            if (MODE == OP_CHEB) dout[o] = dval;
          }
      return;
    }
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int x = x0 + a;
        const int s = N - 1 - x - (jb + b) - pl;  // >= 0: row in T; -1: on the face i + j + k = N
        const bool row = s >= 0, diag = s == -1;
        const int mask = diag ? (x == 0 ? 3 : 1) : 2;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const int o = lb[t] + P.off[b] + a;
          const bool dir = (dm[t] >> mask) & 1u;
          // volume rows: the final value; face i = 0: the partial row (or the
          // Dirichlet value); face i + j + k = N: the Dirichlet value only
          const bool vol = row && x > 0;
          const bool zero = (row || diag) && !vol && dir;
          const bool part = row && !vol && !dir;
          T val, dval;
          final_value<T, MODE>(comp(y[a][b].y, t), DIAG ? comp(y[a][b].d, t) : (T)0, comp(P.v[b + 1][a + 1].u, t),
                               PREF ? comp(P.fv[a][b], t) : (T)0, MODE == OP_CHEB ? comp(P.dv[a][b], t) : (T)0, p,
                               val, dval);
          if (part) val = MODE == OP_DIAG ? comp(y[a][b].d, t) : comp(y[a][b].y, t);
          if (zero) {
            val = MODE == OP_DIAG ? (T)1 : (T)0;
            dval = 0;
          }
          if (vol || zero || part) out[o] = val;
          if (MODE == OP_CHEB && (vol || zero)) dout[o] = dval;
        }
      }
  };
#pragma unroll
  for (int st = 0; st < kNS - 1; ++st) issue_next(st);  // planes k0-1 .. k0+kNS-3
  cpa_wait<kNS - 2>();
  __syncwarp();
  PlaneR<V> X, Y;
  read_next(0, X);  // plane k0-1
  Acc<V, DIAG> yX[2][2], yY[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      yX[a][b].y = vzero<V>();
      yX[a][b].d = vzero<V>();
    }
  // one march step: plane qq + kNS - 2 goes into the stage of plane qq - 2
  // (stage sc), plane qq is read from stage sr
  int sc = kNS - 1, sr = 1;
  auto step = [&](PlaneR<V>& P, PlaneR<V>& Q, Acc<V, DIAG>(&yP)[2][2], Acc<V, DIAG>(&yQ)[2][2], int qq) {
    __syncwarp();    // every lane has read plane qq-2 before its stage is refilled
    issue_next(sc);  // plane qq + kNS - 2
    sc = sc + 1 == kNS ? 0 : sc + 1;
    cpa_wait<kNS - 2>();  // this lane's copies of plane qq have landed
    __syncwarp();         // ... and every other lane's
    read_next(sr, Q);     // plane qq
    sr = sr + 1 == kNS ? 0 : sr + 1;
    step_edges<V, DIAG>(P, Q, c, yP, yQ);
    if (qq - 1 >= k0) store(P, yP, qq - 1);
    if (HHG_TPIN) pin_kept(Q);  // the next step's plane q-1 stays in registers
  };
  for (int qq = k0; qq <= qend; qq += 2) {
    step(X, Y, yX, yY, qq);
    if (qq + 1 > qend) break;
    step(Y, X, yY, yX, qq + 1);
  }
  cpa_wait<0>();
  __syncwarp();
}

// Persistent tile kernel: warps take items in list order (longest first).
// One warp per block, so that an item and everything derived from it is
// uniform in the block.
template <class T, class KT, int MODE>
__global__ void __launch_bounds__(32, sizeof(T) == 8 ? 8 : 4 * HHG_TMINB)
    tile_kernel(DepthDev D, OpPtrs p, int n_items) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x;
  unsigned char* ring = smem_raw;
  const unsigned ring_s = smem_u32(ring);
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4 item = D.pitems[it];
    if (item.z < item.y) continue;
    const int sa = (int)((unsigned)item.x >> 20);
    const int j0 = (item.x >> 10) & 1023, i0 = item.x & 1023;
    const bool single = (item.w & kPairSingle) != 0;
    const int sb = item.w & 0xfffff;
    if constexpr (LaneV<T>::NT == 2) {
      const int sl[2] = {sa, single ? sa : sb};
      tile_item<T, KT, MODE>(D, sl, i0, j0, item.y, item.z, lane, p, ring, ring_s);
    } else {
      const int s1[1] = {sa};
      tile_item<T, KT, MODE>(D, s1, i0, j0, item.y, item.z, lane, p, ring, ring_s);
      if (!single) {
        const int s2[1] = {sb};
        tile_item<T, KT, MODE>(D, s2, i0, j0, item.y, item.z, lane, p, ring, ring_s);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Copies the tile kernel does not write: one thread each.  Dirichlet: the
// mode's boundary value; otherwise the copy's partial row from its tet.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ldg_k(const float* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ double ldg_k(const double* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ float ldg_k(const __nv_bfloat16* p, long long i) { return __bfloat162float(__ldg(p + i)); }

template <class T, class KT>
__device__ __forceinline__ void copy_partial(const DepthDev& D, const T* __restrict__ sten, const BCopy& cp,
                                             const T* __restrict__ u, const KT* __restrict__ k, T& y, T& diag) {
  const TetDev td = D.tets[cp.slot];
  const int N = td.N;
  const T* st = sten + (cp.slot * 16 + (cp.mask & 15)) * kNDir;
  const T* ut = u + td.base;
  const KT* kt = k + td.base;
  const int ci = cp.i, cj = cp.j, ck = cp.k;
  auto pstart = [&](int kk) { return (int)(tetnum(N + 1) - tetnum(N + 1 - kk)); };
  auto rstart = [&](int pk, int kk, int jj) { return pk + jj * (N - kk + 1) - jj * (jj - 1) / 2; };
  const int p0 = pstart(ck);
  const int pm = ck > 0 ? pstart(ck - 1) : 0;
  const int pp = ck < N ? pstart(ck + 1) : 0;
  const int x = rstart(p0, ck, cj) + ci;
  const T ux = __ldg(ut + x);
  const T kx = (T)ldg_k(kt, x);
#pragma unroll
  for (int d = 0; d < kNDir; ++d) {
    int di, dj, dk;
    dir_of(d, di, dj, dk);
    const int a = ci + di, b = cj + dj, cc = ck + dk;
    if (a < 0 || b < 0 || cc < 0 || a + b + cc > N) continue;
    const int ps = dk == 0 ? p0 : (dk < 0 ? pm : pp);
    const int idx = rstart(ps, cc, b) + a;
    const T sv = st[d] * (kx + (T)ldg_k(kt, idx));
    y = fma(sv, __ldg(ut + idx) - ux, y);
    diag -= sv;
  }
}

template <class T, class KT, int MODE>
__global__ void __launch_bounds__(128) copies_kernel(DepthDev D, OpPtrs p, int n) {
  const T* sten = sten_of<T>(D);
  T* out = static_cast<T*>(p.out);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const BCopy cp = D.fcopies[q];
    if (cp.mask & kCopyDirichlet) {
      store_dirichlet<T, MODE>(out + cp.idx, MODE == OP_CHEB ? static_cast<T*>(p.d_out) + cp.idx : nullptr);
      continue;
    }
    T y = 0, dg = 0;
    copy_partial<T, KT>(D, sten, cp, static_cast<const T*>(p.u), static_cast<const KT*>(p.k), y, dg);
    store_partial<T, MODE>(y, dg, out + cp.idx);
  }
}

// ---------------------------------------------------------------------------
// Interface sums: node isum[t] adds its copies' partial rows (left in out by
// the two kernels above), applies the mode's epilogue with the summed
// diagonal dsum[t], and writes every copy.  In OP_DIAG the sums are the
// diagonal itself (written to dsum_out when given).
// ---------------------------------------------------------------------------
template <class T, int MODE>
__global__ void __launch_bounds__(128) sum_kernel(DepthDev D, OpPtrs p, int n, const T* __restrict__ dsum,
                                                  T* __restrict__ dsum_out) {
  T* out = static_cast<T*>(p.out);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int lo = D.sstart[t], hi = D.sstart[t + 1];
    T y = 0;
    for (int q = lo; q < hi; ++q) y += out[D.sidx[q]];
    const int i0 = D.sidx[lo];
    T val = y, dval = 0;
    if (MODE == OP_RESID) {
      val = __ldg(static_cast<const T*>(p.f) + i0) - y;
    } else if (MODE == OP_JACOBI) {
      val = __ldg(static_cast<const T*>(p.u) + i0) +
            sdiv((T)p.omega * (__ldg(static_cast<const T*>(p.f) + i0) - y), dsum[t]);
    } else if (MODE == OP_CHEB) {
      const T prev = p.ca != 0.0 ? (T)p.ca * __ldg(static_cast<const T*>(p.d_in) + i0) : (T)0;
      dval = prev + (T)p.cb * (__ldg(static_cast<const T*>(p.f) + i0) - y) / dsum[t];
      val = __ldg(static_cast<const T*>(p.u) + i0) + dval;
    } else if (MODE == OP_DIAG) {
      if (dsum_out) dsum_out[t] = y;
    }
    for (int q = lo; q < hi; ++q) {
      const int idx = D.sidx[q];
      out[idx] = val;
      if (MODE == OP_CHEB) static_cast<T*>(p.d_out)[idx] = dval;
    }
  }
}

template <class T, class KT>
constexpr int ring_bytes() {
  return Stage<T, KT>::WB;  // one warp per block
}

template <class T, class KT, int MODE>
static int occupancy() {
  static int occ = 0;
  if (!occ) {
    HHG_CUDA(cudaFuncSetAttribute(tile_kernel<T, KT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ring_bytes<T, KT>()));
    HHG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tile_kernel<T, KT, MODE>, 32, ring_bytes<T, KT>()));
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

// dsum slot of an internal dtype
static int dsum_slot(int dtype) {
  return dtype == HHG_F64 ? 0 : (dtype == HHG_F32 ? 1 : (dtype == HHG_F32_KBF16 ? 2 : 3));
}

template <class T, class KT, int MODE>
static void launch_typed(const Mesh& m, int depth, int dtype, const OpArgs& a, const void* kptr, void* dsum_out,
                         cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  const DepthDev& D = Dh.dev;
  const int n_items = a.nc_only ? D.n_pitems_nc : D.n_pitems;
  const int n_f = a.nc_only ? D.n_fcopies_nc : D.n_fcopies;
  const int n_s = a.nc_only ? D.n_isum_nc : D.n_isum;
  OpPtrs p{a.u, kptr, a.f, a.out, a.d_in, a.d_out, a.omega, a.ca, a.cb};
  const T* dsum = static_cast<const T*>(Dh.dsum[dsum_slot(dtype)]);
  if ((MODE == OP_JACOBI || MODE == OP_CHEB) && n_s > 0)
    HHG_REQUIRE(dsum, "internal: interface diagonals not computed (hhg_set_coefficient)");
  const bool fork = n_items > 0 && n_f > 0 && m.side;
  if (fork) {
    HHG_CUDA(cudaEventRecord(m.side_fork, s));
    HHG_CUDA(cudaStreamWaitEvent(m.side, m.side_fork, 0));
  }
  if (n_f > 0) {
    copies_kernel<T, KT, MODE><<<std::min((n_f + 127) / 128, 16 * m.num_sms), 128, 0, fork ? m.side : s>>>(D, p, n_f);
    HHG_CUDA(cudaGetLastError());
  }
  if (fork) HHG_CUDA(cudaEventRecord(m.side_join, m.side));
  if (n_items > 0) {
    const int occ = occupancy<T, KT, MODE>();
    const int blocks = std::min(n_items, m.num_sms * occ);
    tile_kernel<T, KT, MODE><<<blocks, 32, ring_bytes<T, KT>(), s>>>(D, p, n_items);
    HHG_CUDA(cudaGetLastError());
  }
  if (fork) HHG_CUDA(cudaStreamWaitEvent(s, m.side_join, 0));
  if (n_s > 0) {
    sum_kernel<T, MODE><<<std::min((n_s + 127) / 128, 16 * m.num_sms), 128, 0, s>>>(
        D, p, n_s, dsum, static_cast<T*>(dsum_out));
    HHG_CUDA(cudaGetLastError());
  }
}

template <int MODE>
static void launch_mode(const Mesh& m, int depth, int dtype, const OpArgs& a, void* dsum_out, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  if (dtype == HHG_F64)
    launch_typed<double, double, MODE>(m, depth, dtype, a, Dh.k64, dsum_out, s);
  else if (dtype == kF64KBF16)
    launch_typed<double, double, MODE>(m, depth, dtype, a, Dh.k16d, dsum_out, s);
  else if (dtype == HHG_F32)
    launch_typed<float, float, MODE>(m, depth, dtype, a, Dh.k32, dsum_out, s);
  else
    launch_typed<float, __nv_bfloat16, MODE>(m, depth, dtype, a, Dh.k16, dsum_out, s);
}

static void launch_any(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, void* dsum_out,
                       cudaStream_t s) {
  switch (mode) {
    case OP_APPLY: launch_mode<OP_APPLY>(m, depth, dtype, a, dsum_out, s); break;
    case OP_RESID: launch_mode<OP_RESID>(m, depth, dtype, a, dsum_out, s); break;
    case OP_JACOBI: launch_mode<OP_JACOBI>(m, depth, dtype, a, dsum_out, s); break;
    case OP_CHEB: launch_mode<OP_CHEB>(m, depth, dtype, a, dsum_out, s); break;
    case OP_DIAG: launch_mode<OP_DIAG>(m, depth, dtype, a, dsum_out, s); break;
  }
}

}  // namespace

// Launch configurations are computed once, outside any stream capture.
void init_launch_configs(int dtype) {
  if (dtype == HHG_F64 || dtype == kF64KBF16)
    init_typed<double, double>();
  else if (dtype == HHG_F32)
    init_typed<float, float>();
  else
    init_typed<float, __nv_bfloat16>();
}

void launch_scaled_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, cudaStream_t s) {
  launch_any(m, depth, dtype, mode, a, nullptr, s);
}

// Summed diagonals of the unique non-Dirichlet interface nodes, for every
// depth and dtype: the operator in OP_DIAG mode into a scratch vector, whose
// sum pass records them.
void compute_interface_diagonals(Mesh& m, cudaStream_t s) {
  const int dtypes[4] = {HHG_F64, HHG_F32, HHG_F32_KBF16, kF64KBF16};
  for (int dt : dtypes) init_launch_configs(dt);
  for (int d = 0; d < m.ndepth; ++d) {
    Depth& D = m.depth[d];
    for (int dt : dtypes) {
      const size_t es = elem_size(dt);
      if (!D.dsum[dsum_slot(dt)]) D.dsum[dsum_slot(dt)] = dalloc(D, std::max(D.n_isum, 1) * es);
    }
    if (D.n_isum == 0) continue;
    void* tmp = nullptr;
    const cudaError_t e = cudaMalloc(&tmp, (size_t)std::max<long long>(D.n_stored, 1) * 8);
    if (e != cudaSuccess) throw Error{HHG_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
    for (int dt : dtypes) {
      OpArgs a{nullptr, nullptr, tmp, nullptr, nullptr, 0, 0, 0, 0};
      // OP_DIAG reads no u, but the tile kernel stages it: give it the coefficient's own array
      a.u = dt == HHG_F64 ? (const void*)D.k64
                          : (dt == kF64KBF16 ? (const void*)D.k16d : (const void*)D.k32);
      launch_any(m, d, dt, OP_DIAG, a, D.dsum[dsum_slot(dt)], s);
    }
    const cudaError_t es = cudaStreamSynchronize(s);
    cudaFree(tmp);
    HHG_CUDA(es);
  }
}

// ---------------------------------------------------------------------------
// Host: work lists of the scaled operator for one depth.
// ---------------------------------------------------------------------------
namespace {

// Does the tile kernel write this copy (tile rule mirrored from tile_item)?
bool tile_writes(int N, int i, int j, int k, bool dir) {
  if (j < 1 || k < 1) return false;
  const int i0 = (i / kTI) * kTI, j0 = 1 + ((j - 1) / kTJ2) * kTJ2;
  if (i0 + j0 > N - 2) return false;
  if (k > N - 1 - (i0 + j0)) return false;
  const int s = N - 1 - i - j - k;
  if (s >= 0) return true;
  return s == -1 && dir;
}

// slot pairs: equal level, same class (above the coarsest level or not)
std::vector<std::pair<int, int>> slot_pairs(const Depth& D) {
  std::vector<std::pair<int, int>> out;
  const int ns = (int)D.slot_tet.size();
  for (int cls = 0; cls < 2; ++cls) {
    std::map<int, std::vector<int>> byN;
    for (int s = 0; s < ns; ++s)
      if ((s < D.n_slots_nc) == (cls == 0)) byN[D.h_tets[s].N].push_back(s);
    for (auto& kv : byN) {
      const auto& v = kv.second;
      for (size_t a = 0; a < v.size(); a += 2) out.push_back({v[a], a + 1 < v.size() ? v[a + 1] : -1});
    }
  }
  return out;
}

int count_items(const Depth& D, const std::vector<std::pair<int, int>>& pairs, int ks) {
  long long c = 0;
  for (auto& pr : pairs) {
    const int N = D.h_tets[pr.first].N;
    for (int j0 = 1; j0 <= N - 2; j0 += kTJ2)
      for (int i0 = 0; i0 + j0 <= N - 2; i0 += kTI) c += (N - 1 - (i0 + j0) + ks - 1) / ks;
  }
  return (int)std::min<long long>(c, 1 << 30);
}

}  // namespace

void build_pair_items(const Mesh& m, Depth& D) {
  const auto pairs = slot_pairs(D);
  // k-segment length: the mesh's, halved (down to 4 planes) while the depth
  // has fewer items than resident warps (12 per SM)
  const int target = (m.num_sms > 0 ? m.num_sms : 152) * 12;
  int ks = m.kseg;
  while (ks > 4 && count_items(D, pairs, ks) < target) ks /= 2;
  std::vector<std::pair<long long, int4>> its[2];
  for (auto& pr : pairs) {
    const int sa = pr.first;
    const int cls = sa < D.n_slots_nc ? 0 : 1;
    const int N = D.h_tets[sa].N;
    const int w = pr.second >= 0 ? pr.second : kPairSingle;
    for (int j0 = 1; j0 <= N - 2; j0 += kTJ2)
      for (int i0 = 0; i0 + j0 <= N - 2; i0 += kTI) {
        const int top = N - 1 - (i0 + j0);
        for (int k0 = 1; k0 <= top; k0 += ks) {
          const int k1 = std::min(top, k0 + ks - 1);
          const long long key = m.korder == 1 ? k0 : -(long long)(k1 - k0 + 1);
          its[cls].push_back({key, make_int4(sa << 20 | j0 << 10 | i0, k0, k1, w)});
        }
      }
  }
  D.h_pitems.clear();
  for (int cls = 0; cls < 2; ++cls) {
    std::stable_sort(its[cls].begin(), its[cls].end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    for (auto& p : its[cls]) D.h_pitems.push_back(p.second);
    if (cls == 0) D.n_pitems_nc = (int)D.h_pitems.size();
  }
  D.n_pitems = (int)D.h_pitems.size();
}

void build_scaled_lists(const Mesh& m, Depth& D) {
  const int ns = (int)D.slot_tet.size();
  HHG_REQUIRE(ns < (1 << 11), "too many macro tets in one depth (max 2047)");
  HHG_REQUIRE(D.n_stored < (1LL << 31) - (1LL << 20), "a depth vector must hold fewer than 2^31 - 2^20 nodes");
  // the tile kernel's column-0 slots assume: face i = 0 entries equal the
  // volume ones for edges leaving the face, 0 for edges leaving the tet, and
  // the same for +w and -w inside the face
  for (int s = 0; s < ns; ++s) {
    if (D.h_tets[s].N < 4) continue;
    const double* s0 = &D.h_sten[(size_t)s * 16 * kNDir];
    const double* s2 = s0 + 2 * kNDir;
    double scale = 0;
    for (int d = 0; d < kNDir; ++d) scale = std::max(scale, std::fabs(s0[d]));
    auto near = [&](double a, double b) { return std::fabs(a - b) <= 1e-12 * scale; };
    const int inward[4] = {0, 3, 4, 6}, outward[4] = {7, 10, 11, 13}, inface[3] = {1, 2, 5};
    for (int d : inward) HHG_REQUIRE(near(s2[d], s0[d]), "internal: face stencil differs from the volume stencil");
    for (int d : outward) HHG_REQUIRE(near(s2[d], 0.0), "internal: face stencil reaches outside its tet");
    for (int d : inface) HHG_REQUIRE(near(s2[d], s2[d + 7]), "internal: face stencil not symmetric in the face");
    for (int d = 0; d < 7; ++d) HHG_REQUIRE(near(s0[d], s0[d + 7]), "internal: volume stencil not symmetric");
  }
  // Dirichlet status of each face mask per slot
  D.h_dmask.assign(std::max(ns, 1), 0);
  for (int b = 0; b < D.n_bnodes; ++b)
    if (D.h_bdir[b])
      for (int q = D.h_bstart[b]; q < D.h_bstart[b + 1]; ++q) {
        const BCopy& c = D.h_bcopies[q];
        D.h_dmask[c.slot] |= (unsigned short)(1u << c.mask);
      }
  // copies the tile kernel does not write, in stored order
  D.h_fcopies.clear();
  D.n_fcopies_nc = 0;
  for (int b = 0; b < D.n_bnodes; ++b)
    for (int q = D.h_bstart[b]; q < D.h_bstart[b + 1]; ++q) {
      BCopy c = D.h_bcopies[q];
      const int N = D.h_tets[c.slot].N;
      const bool dir = D.h_bdir[b] != 0;
      HHG_REQUIRE(((D.h_dmask[c.slot] >> c.mask) & 1u) == (dir ? 1u : 0u),
                  "internal: Dirichlet status differs between nodes of one primitive");
      if (tile_writes(N, c.i, c.j, c.k, dir)) continue;
      if (dir) c.mask |= kCopyDirichlet;
      D.h_fcopies.push_back(c);
    }
  std::sort(D.h_fcopies.begin(), D.h_fcopies.end(), [](const BCopy& a, const BCopy& b) { return a.idx < b.idx; });
  D.n_fcopies = (int)D.h_fcopies.size();
  for (const BCopy& c : D.h_fcopies)
    if (c.slot < D.n_slots_nc) ++D.n_fcopies_nc;
  // unique interface nodes whose copies are summed, with their copies'
  // stored indices
  D.h_isum.clear();
  D.h_sstart.assign(1, 0);
  D.h_sidx.clear();
  D.n_isum_nc = 0;
  for (int b = 0; b < D.n_bnodes; ++b) {
    if (D.h_bdir[b]) continue;
    D.h_isum.push_back(b);
    for (int q = D.h_bstart[b]; q < D.h_bstart[b + 1]; ++q) D.h_sidx.push_back((int)D.h_bcopies[q].idx);
    D.h_sstart.push_back((int)D.h_sidx.size());
    if (b < D.n_bnodes_nc) D.n_isum_nc = (int)D.h_isum.size();
  }
  D.n_isum = (int)D.h_isum.size();
  build_pair_items(m, D);
}

template <class T>
static T* upload_vec(Depth& d, const std::vector<T>& h) {
  T* p = static_cast<T*>(dalloc(d, std::max<size_t>(h.size(), 1) * sizeof(T)));
  if (!h.empty()) HHG_CUDA(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return p;
}

void upload_pair_items(Depth& D) {
  if (D.dev.pitems) {
    cudaFree(const_cast<int4*>(D.dev.pitems));
    D.allocations.erase(std::remove(D.allocations.begin(), D.allocations.end(), (void*)D.dev.pitems),
                        D.allocations.end());
  }
  D.dev.pitems = upload_vec(D, D.h_pitems);
  D.dev.n_pitems = D.n_pitems;
  D.dev.n_pitems_nc = D.n_pitems_nc;
}

void upload_scaled_lists(Depth& D) {
  D.dev.pitems = nullptr;
  upload_pair_items(D);
  D.dev.dmask = upload_vec(D, D.h_dmask);
  D.dev.fcopies = upload_vec(D, D.h_fcopies);
  D.dev.n_fcopies = D.n_fcopies;
  D.dev.n_fcopies_nc = D.n_fcopies_nc;
  D.dev.isum = upload_vec(D, D.h_isum);
  D.dev.sstart = upload_vec(D, D.h_sstart);
  D.dev.sidx = upload_vec(D, D.h_sidx);
  D.dev.n_isum = D.n_isum;
  D.dev.n_isum_nc = D.n_isum_nc;
}

}  // namespace hhg
