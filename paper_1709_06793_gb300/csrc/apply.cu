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
// Volume kernel (nodes strictly inside a macro tet).  A warp owns a tile of
// 16 consecutive i x 8 rows j and marches along k; lane (h, l) owns column
// i = i0 + l, rows j0+4h .. j0+4h+3.  The tile's footprint of each plane is
// staged in shared memory (see the staging section below).  When plane q
// arrives a lane computes every edge between planes q-1 and q and every edge
// inside plane q that touches its nodes; after that the rows of plane q-1 are
// complete and are written.  Two planes of the lane's footprint live in
// registers.
#include <utility>

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
// Two edges of row a with the same coefficient (opposite directions):
// c [(k_a + k_b1)(u_b1 - u_a) + (k_a + k_b2)(u_b2 - u_a)] with one scaling.
template <class T, bool DIAG, class P2>
__device__ __forceinline__ void edge1x2(P2 a, P2 b1, P2 b2, T c, Acc<T, DIAG>& A) {
  const P2 t1 = diffsum(a, b1);
  const P2 t2 = diffsum(a, b2);
  const T w = fma(t2.y, t2.x, t1.y * t1.x);
  A.y = fma(c, w, A.y);
  if (DIAG) A.d = fma(-c, t1.y + t2.y, A.d);
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
  int off[kTJ];  // tet-local offset of (i0-1, row) for the lane's rows (stores)
  T fv[kTJ];     // f (and the previous Chebyshev update) at the lane's nodes,
  T dv[kTJ];     // loaded when the plane is read, used when it is stored
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

// Quotient of the damped Jacobi update: FP32 uses the fast division
// intrinsic (within 2 ulp; the sweep is a preconditioner step, the outer
// FP64 residual decides convergence), FP64 the correctly rounded one.
__device__ __forceinline__ float sdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sdiv(double a, double b) { return a / b; }

// fv, dv: f and the previous Chebyshev update at the node (prefetched)
template <class T, int MODE>
__device__ __forceinline__ void finish_node(T y, T diag, T ux, long long idx, const OpPtrs& p, T fv, T dv) {
  if (MODE == OP_APPLY) {
    static_cast<T*>(p.out)[idx] = y;
  } else if (MODE == OP_RESID) {
    static_cast<T*>(p.out)[idx] = fv - y;
  } else if (MODE == OP_JACOBI) {
    const T r = fv - y;
    static_cast<T*>(p.out)[idx] = ux + sdiv((T)p.omega * r, diag);
  } else if (MODE == OP_CHEB) {
    const T r = fv - y;
    const T prev = p.ca != 0.0 ? (T)p.ca * dv : (T)0;
    const T dn = prev + (T)p.cb * r / diag;
    static_cast<T*>(p.d_out)[idx] = dn;
    static_cast<T*>(p.out)[idx] = ux + dn;
  } else {  // OP_DIAG
    static_cast<T*>(p.out)[idx] = diag;
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
    edge1x2(Q.c0[m], Q.cp[m], Q.cm[m], c1, yQ[r]);  // +e1, -e1
    if (r + 1 < kTJ)
      edge2(Q.c0[m], Q.c0[m + 1], c2, yQ[r], yQ[r + 1]);  // +e2
    else
      edge1(Q.c0[m], Q.c0[m + 1], c2, yQ[r]);
    if (r == 0) edge1(Q.c0[m], Q.c0[m - 1], c2, yQ[r]);  // -e2
    edge1x2(Q.c0[m], Q.cp[m - 1], Q.cm[m + 1], c12, yQ[r]);  // e1-e2, -(e1-e2)
  }
}

// ---------------------------------------------------------------------------
// Volume kernel with shared-memory staging.
//
// A warp owns a tile of 16 columns i0..i0+15 x 8 rows j0..j0+7 of one tet and
// marches along k; half-warp h = lane/16 owns rows j0+4h .. j0+4h+3 of column
// i = i0 + lane%16.  The tile's footprint in plane q is rows j0-1 .. j0+8 (m =
// 0..9) x columns i0-1 .. i0+16 of u and k: 20 contiguous row segments.
// Each segment is copied from its 16-byte-aligned start in 16-byte chunks
// with cp.async (all lanes copy chunks in parallel; chunks past the end of
// the vector are zero-filled, so no read leaves the vector).  A ring of
// kStages planes per warp keeps kStages-2 planes in flight; completion is
// tracked by cp.async groups (no spin loop).
// ---------------------------------------------------------------------------
#ifndef HHG_STAGES
#define HHG_STAGES 4
#endif
constexpr int kStages = HHG_STAGES;  // staged planes per warp (kStages-2 in flight)
constexpr int kTileI = kWarpTileI;  // columns per warp tile
constexpr int kTileJ = kWarpTileJ;  // rows per warp tile (32/kTileI row groups x kTJ)
constexpr int kRows = kTileJ + 2;

template <class E>
struct RowGeom {
  static constexpr int V = 16 / (int)sizeof(E);                        // elements per 16-byte chunk
  static constexpr int chunks = (kTileI + 2 + 2 * (V - 1) + V - 1) / V;  // max chunks per row
  // row stride in elements: with two row groups, rows 4 apart land 16 banks
  // apart for 4-byte data; with one group any 16-byte-multiple stride will do
  static constexpr int stride =
      kTileI == 16 ? (sizeof(E) == 4 ? 28 : (sizeof(E) == 8 ? 24 : 48)) : chunks * V + (sizeof(E) == 2 ? 8 : 4);
  static constexpr int bytes = kRows * stride * (int)sizeof(E);
  static_assert(chunks * V <= stride, "row buffer too small");
};

template <class T, class KT>
struct Stage {
  static constexpr int u_bytes = RowGeom<T>::bytes;
  static constexpr int k_bytes = RowGeom<KT>::bytes;
  static constexpr int bytes = u_bytes + k_bytes;
  static constexpr int warp_bytes = kStages * bytes;
  static constexpr int u_chunks = kRows * RowGeom<T>::chunks;
  static constexpr int n_chunks = u_chunks + kRows * RowGeom<KT>::chunks;
  static constexpr int rounds = (n_chunks + 31) / 32;
};

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(unsigned dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Row heads.  Offsets are tet-local (32-bit: a tet holds < 2^31 nodes); the
// tet base is applied to the pointers once per item.  For plane q the head is
// the offset of (i0-1, jr, q) and A the length of row jr (jr = j0-1 for the
// tile, jb-1 for a half-warp); row jr+m starts m*A - m(m-1)/2 later.
struct Head {
  int e0;   // offset of (i0-1, jr, q) in the tet
  int A;    // length of row jr in plane q
  int Psz;  // nodes in plane q
  int q;
  __device__ __forceinline__ void next(int N, int jr) {  // plane q -> q+1
    e0 += Psz - jr;
    Psz -= N - q + 1;
    A -= 1;
    ++q;
  }
};

// Copy assignment.  The tile's footprint in a plane is kRows row segments of
// u and kRows of k.  For each array, lane = CH p + c (CH = chunks per row at
// the worst alignment) copies chunk c of rows p, p + R, p + 2R, ... (R = 32 /
// CH rows per round), so the 32 chunks of one cp.async instruction are
// consecutive chunks of R rows (a few cache lines per instruction) rather
// than one chunk of every row.
struct CopyLane {
  int lane;
};

template <class T, class KT>
__device__ __forceinline__ CopyLane copy_lane(int lane) {
  return CopyLane{lane};
}

// elements a staged row can reach past its start (the last chunk's end)
template <class T, class KT>
constexpr int max_reach() {
  return RowGeom<T>::chunks * RowGeom<T>::V > RowGeom<KT>::chunks * RowGeom<KT>::V ? RowGeom<T>::chunks * RowGeom<T>::V
                                                                                   : RowGeom<KT>::chunks * RowGeom<KT>::V;
}

// 16-byte copy issued only where pred is set (no branch around it); the
// destination is dst + OFF bytes.
template <int OFF>
__device__ __forceinline__ void cp_async16_if(bool pred, unsigned dst, const void* src) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n @p cp.async.cg.shared.global [%0+%3], [%1], 16;\n}\n" ::"r"(dst),
      "l"(src), "r"((int)pred), "n"(OFF)
      : "memory");
}

// The copy rounds of issue_rows on the fast path: rows p + Q, Q = 0, R, 2R, ...
template <class E, int RB, int Q>
__device__ __forceinline__ void copy_rounds(int eb, int d, int pm, int thr, unsigned dst0, const E* lane_src) {
  if constexpr (Q < kRows) {
    constexpr int V = RowGeom<E>::V, R = 32 / RowGeom<E>::chunks;
    constexpr int PITCH = RowGeom<E>::stride * (int)sizeof(E);
    const int eg = eb + Q * d - Q * (Q - 1) / 2;  // row p + Q: element (i0-1, j, q)
    const int mis = eg & (V - 1);
    cp_async16_if<Q * PITCH>(pm + Q <= 0 && mis >= thr, dst0, lane_src + (eg - mis));
    copy_rounds<E, RB, Q + R>(eb, d, pm, thr, dst0, lane_src);
  }
}

// The same with u and k of one element size: the row geometry (and the tet
// base's alignment) is shared, so one set of row arithmetic drives both copies.
template <class E, int RBK, int Q>
__device__ __forceinline__ void copy_rounds2(int eb, int d, int pm, int thr, unsigned dst0, const E* src_u,
                                             const E* src_k) {
  if constexpr (Q < kRows) {
    constexpr int V = RowGeom<E>::V, R = 32 / RowGeom<E>::chunks;
    constexpr int PITCH = RowGeom<E>::stride * (int)sizeof(E);
    const int eg = eb + Q * d - Q * (Q - 1) / 2;
    const int a = eg & ~(V - 1);
    const bool pred = pm + Q <= 0 && eg - a >= thr;
    cp_async16_if<Q * PITCH>(pred, dst0, src_u + a);
    cp_async16_if<RBK + Q * PITCH>(pred, dst0, src_k + a);
    copy_rounds2<E, RBK, Q + R>(eb, d, pm, thr, dst0, src_u, src_k);
  }
}

// Rows m = 0..kRows-1 of one array (row m at byte offset RB + m * pitch of a
// stage); rows m > mrows are absent from the plane.  Indices are counted
// from the 16-byte boundary at or below the tet base (bm elements below it),
// so a chunk's start is the row start rounded down to a multiple of V.
// inside = every chunk of the footprint ends before the end of the vector
// (then no chunk needs cutting, and the copies are predicated, branch-free).
template <class E, int RB>
__device__ __forceinline__ void issue_rows(unsigned stage, const Head& H, int lane, int mrows, int lim, int bm,
                                           const unsigned char* __restrict__ base, bool inside) {
  constexpr int CH = RowGeom<E>::chunks, R = 32 / CH, V = RowGeom<E>::V;
  constexpr int PITCH = RowGeom<E>::stride * (int)sizeof(E);
  const int p = lane / CH, c = lane - p * CH;
  // row p + Q starts Q (A - p) - Q (Q - 1) / 2 after row p
  const int eb = H.e0 + p * H.A - p * (p - 1) / 2 + bm;
  const int d = H.A - p;
  // row p + Q is staged iff pm + Q <= 0 (lanes left over by the row size never)
  const int pm = p < R ? p - min(mrows, kRows - 1) : kRows;
  const int thr = c * V - (kTileI + 1);  // chunk c reaches column i0+kTileI iff mis >= thr
  const E* lane_src = reinterpret_cast<const E*>(base - bm * (int)sizeof(E) + 16 * c);
  const unsigned dst0 = stage + (unsigned)(RB + p * PITCH + 16 * c);
  if (inside) {
    copy_rounds<E, RB, 0>(eb, d, pm, thr, dst0, lane_src);
  } else {
#pragma unroll
    for (int r = 0; r * R < kRows; ++r) {
      const int Q = r * R;
      const int eg = eb + Q * d - Q * (Q - 1) / 2;
      const int mis = eg & (V - 1);
      if (pm + Q <= 0 && mis >= thr) {
        const int a = eg - mis;
        const long long left = ((long long)lim + bm - a - c * V) * (int)sizeof(E);  // bytes of the vector from the chunk on
        const unsigned dst = dst0 + Q * PITCH;
        if (left >= 16)
          cp_async16(dst, lane_src + a, 16);
        else
          cp_async16(dst, left > 0 ? (const void*)(lane_src + a) : (const void*)base, left > 0 ? (int)left : 0);
      }
    }
  }
}

// Stage plane H.q: row m (j = jm1 + m) of u and of k, from the aligned start
// at or before column i0-1 through column i0+kTileI.  base_u / base_k = the
// arrays at the tet base, in bytes; bm_u / bm_k = tet base mod V (elements
// per chunk); lim = elements of the vector from the tet base on (chunks are
// cut there and zero-filled beyond it).
template <class T, class KT>
// want = the march needs this plane (otherwise nothing is copied; the
// arithmetic runs predicated off rather than behind a branch).
__device__ __forceinline__ void issue_plane(unsigned stage, const Head& H, const CopyLane& cl, int N, int jm1,
                                            int lim, int bm_u, int bm_k, const unsigned char* __restrict__ base_u,
                                            const unsigned char* __restrict__ base_k, bool want) {
  const int mrows = want ? N - H.q - jm1 : -1;
  // row starts grow by at most A per row; a chunk ends < CH V elements after its row's start
  constexpr int reach = max_reach<T, KT>();
  const bool inside = H.e0 + (kRows - 1) * H.A + reach <= lim;
  if constexpr (sizeof(T) == sizeof(KT)) {
    // one lane assignment for both arrays (bm_u == bm_k); only a footprint
    // that reaches the end of the vector takes the checked path below
    constexpr int CH = RowGeom<T>::chunks, R = 32 / CH, V = RowGeom<T>::V;
    constexpr int PITCH = RowGeom<T>::stride * (int)sizeof(T);
    const int p = cl.lane / CH, c = cl.lane - p * CH;
    const int eb = H.e0 + p * H.A - p * (p - 1) / 2 + bm_u;
    const int pm = p < R && inside ? p - min(mrows, kRows - 1) : kRows;
    const int shift = 16 * c - bm_u * (int)sizeof(T);
    copy_rounds2<T, Stage<T, KT>::u_bytes, 0>(eb, H.A - p, pm, c * V - (kTileI + 1), stage + (unsigned)(p * PITCH + 16 * c),
                                              reinterpret_cast<const T*>(base_u + shift),
                                              reinterpret_cast<const T*>(base_k + shift));
    if (inside) return;
  }
  issue_rows<T, 0>(stage, H, cl.lane, mrows, lim, bm_u, base_u, inside);
  issue_rows<KT, Stage<T, KT>::u_bytes>(stage, H, cl.lane, mrows, lim, bm_k, base_k, inside);
}

template <class E>
__device__ __forceinline__ float elem_f(const E* p) {
  if constexpr (sizeof(E) == 2)
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
  else
    return (float)*p;
}

// Lane's footprint (rows jb-1 .. jb+4, columns i-1, i, i+1) from a staged
// plane.  hh = the half-warp's head (row jb-1); stage_lane_u / _k = the
// lane's shared-memory bases (row 4h, column l).  Keeps the offsets of rows
// jb .. jb+3 for the stores.
template <class T, class KT>
__device__ __forceinline__ void read_plane(Plane<T>& Q, const unsigned char* stage_lane_u,
                                           const unsigned char* stage_lane_k, const Head& hh, int bmod_u,
                                           int bmod_k) {
  using P2 = typename Pair<T>::type;
  using GU = RowGeom<T>;
  using GK = RowGeom<KT>;
#pragma unroll
  for (int mm = 0; mm < kTJ + 2; ++mm) {
    const int off = hh.e0 + mm * hh.A - mm * (mm - 1) / 2;  // (i0-1, jb-1+mm, q)
    if (mm >= 1 && mm <= kTJ) Q.off[mm - 1] = off;
    const int mis_u = (off + bmod_u) & (GU::V - 1);
    const T* us = reinterpret_cast<const T*>(stage_lane_u) + mm * GU::stride + mis_u;
    const KT* ks;
    if constexpr (sizeof(KT) == sizeof(T) && GK::stride == GU::stride)  // same alignment: reuse mis
      ks = reinterpret_cast<const KT*>(stage_lane_k) + mm * GK::stride + mis_u;
    else
      ks = reinterpret_cast<const KT*>(stage_lane_k) + mm * GK::stride + ((off + bmod_k) & (GK::V - 1));
    T kv0, kv1, kv2;
    if constexpr (sizeof(KT) == 2) {
      kv0 = (T)elem_f(ks);
      kv1 = (T)elem_f(ks + 1);
      kv2 = (T)elem_f(ks + 2);
    } else {
      kv0 = (T)ks[0];
      kv1 = (T)ks[1];
      kv2 = (T)ks[2];
    }
    if (mm >= 1) Q.cm[mm] = P2{us[0], kv0};
    Q.c0[mm] = P2{us[1], kv1};
    if (mm <= kTJ) Q.cp[mm] = P2{us[2], kv2};
  }
}

// One warp item: tile (i0, j0) of one tet, planes k0..k1 of its k-march.
template <class T, class KT, int MODE>
__device__ void volume_item(const DepthDev& D, const T* __restrict__ sten, int4 item, int lane, const OpPtrs& p,
                            unsigned char* ring, unsigned ring_s, const CopyLane& cl) {
  constexpr bool DIAG = (MODE == OP_JACOBI || MODE == OP_CHEB || MODE == OP_DIAG);
  if (item.z < item.y) return;  // padding item: no planes
  const unsigned tile = (unsigned)item.x;
  const int slot = (int)(tile >> 20);
  const int j0 = (int)((tile >> 10) & 1023u), i0 = (int)(tile & 1023u);
  const int k0 = item.y;
  const TetDev td = D.tets[slot];
  const int N = td.N;
  const int qend = min(item.z + 1, N - (i0 + j0));
  const int h = lane / kTileI, l = lane % kTileI;
  const int i = i0 + l;
  const int jb = j0 + kTJ * h;  // first row of this row group
  T c[7];
#pragma unroll
  for (int d = 0; d < 7; ++d) c[d] = sten[slot * 16 * kNDir + d];  // volume row (mask 0)
  const T* u = static_cast<const T*>(p.u) + td.base;
  const KT* k = static_cast<const KT*>(p.k) + td.base;
  const int bmod_u = (int)(td.base & (RowGeom<T>::V - 1));
  const int bmod_k = (int)(td.base & (RowGeom<KT>::V - 1));
  const long long lim64 = D.n_stored - td.base;
  const int lim = lim64 > 0x7fffffffLL ? 0x7fffffff : (int)lim64;
  // The read head counts elements from the 16-byte boundary at or below the
  // tet base (bmod_u below it), so a staged row's misalignment is its head
  // offset mod V; the node pointers carry the matching shift and the lane's
  // column, so node (i, row) of a plane is ptr[row head offset].
  const long long lb = td.base + l + 1 - bmod_u;
  OpPtrs q = p;
  q.out = static_cast<T*>(p.out) + lb;
  if (MODE != OP_APPLY && MODE != OP_DIAG) q.f = static_cast<const T*>(p.f) + lb;
  if (MODE == OP_CHEB) {
    q.d_in = static_cast<const T*>(p.d_in) + lb;
    q.d_out = static_cast<T*>(p.d_out) + lb;
  }
  // copy head (tile rows from j0-1) and read head (this half's rows from jb-1) at plane k0-1
  Head ch, rh;
  {
    const int qq = k0 - 1;
    const int M = N - qq;
    ch.q = rh.q = qq;
    ch.Psz = rh.Psz = (M + 1) * (M + 2) / 2;
    const int pl = (int)(tetnum(N + 1) - tetnum(N + 1 - qq));
    ch.A = M - j0 + 2;
    ch.e0 = pl + (j0 - 1) * (M + 1) - (j0 - 1) * (j0 - 2) / 2 + (i0 - 1);
    rh.A = M - jb + 2;
    rh.e0 = pl + (jb - 1) * (M + 1) - (jb - 1) * (jb - 2) / 2 + (i0 - 1) + bmod_u;
  }
  constexpr int SB = Stage<T, KT>::bytes;
  static_assert(kStages == 4, "the march below is unrolled over a ring of 4 stages");
  const unsigned char* cbase_u = reinterpret_cast<const unsigned char*>(u);
  const unsigned char* cbase_k = reinterpret_cast<const unsigned char*>(k);
  const int lane_u = (kTJ * h * RowGeom<T>::stride + l) * (int)sizeof(T);  // row 4h, column l
  const int lane_k = Stage<T, KT>::u_bytes + (kTJ * h * RowGeom<KT>::stride + l) * (int)sizeof(KT);
  const unsigned char* ring_u = ring + lane_u;
  const unsigned char* ring_k = ring + lane_k;
  const int dk = bmod_k - bmod_u;
  // stage plane ch.q into stage st if the march needs it; one group per plane
  auto issue_next = [&](int st) {
    issue_plane<T, KT>(ring_s + st * SB, ch, cl, N, j0 - 1, lim, bmod_u, bmod_k, cbase_u, cbase_k, ch.q <= qend);
    cp_async_commit();
    ch.next(N, j0 - 1);
  };
  auto read_next = [&](Plane<T>& P, int st) {
    const int pl = rh.q;
    read_plane<T, KT>(P, ring_u + st * SB, ring_k + st * SB, rh, 0, dk);
    if (MODE == OP_RESID || MODE == OP_JACOBI || MODE == OP_CHEB) {
      // f (and d_in) at the lane's nodes of this plane, needed one step later
      const int lim_r = N - 1 - i - jb - pl;
#pragma unroll
      for (int r = 0; r < kTJ; ++r) {
        const bool ok = r <= lim_r && pl >= k0;
        P.fv[r] = ok ? __ldg(static_cast<const T*>(q.f) + P.off[r]) : (T)0;
        if (MODE == OP_CHEB) P.dv[r] = ok && q.ca != 0.0 ? __ldg(static_cast<const T*>(q.d_in) + P.off[r]) : (T)0;
      }
    }
    rh.next(N, jb - 1);
  };
  // planes k0-1 .. k0+1 into stages 0..2; the step for plane k0+t (t mod 4)
  // then copies plane k0+t+2 into stage (3+t) mod 4 and reads stage (1+t) mod 4
  issue_next(0);
  issue_next(1);
  issue_next(2);
  cp_async_wait<kStages - 2>();
  __syncwarp();
  Plane<T> X, Y;
  read_next(X, 0);  // plane k0-1
  Acc<T, DIAG> yX[kTJ], yY[kTJ];
  auto store = [&](const Plane<T>& P, Acc<T, DIAG>(&y)[kTJ], int pl) {
    const int lim_r = N - 1 - i - jb - pl;  // row r holds a volume node iff r <= lim_r
#pragma unroll
    for (int r = 0; r < kTJ; ++r)
      if (r <= lim_r) finish_node<T, MODE>(y[r].y, y[r].d, P.c0[r + 1].x, P.off[r], q, P.fv[r], P.dv[r]);
  };
  auto step = [&](auto tc, Plane<T>& P, Plane<T>& Q, Acc<T, DIAG>(&yP)[kTJ], Acc<T, DIAG>(&yQ)[kTJ], int qq) {
    constexpr int t = decltype(tc)::value;
    __syncwarp();                  // every lane has read plane qq-2 before its stage is refilled
    issue_next((3 + t) & 3);       // plane qq + 2
    cp_async_wait<kStages - 2>();  // this lane's copies of plane qq have landed
    __syncwarp();                  // ... and every other lane's
    read_next(Q, (1 + t) & 3);     // plane qq
    step_edges<T, DIAG>(P, Q, c, yP, yQ);
    if (t != 0 || qq - 1 >= k0) store(P, yP, qq - 1);
  };
  for (int qq = k0; qq <= qend; qq += 4) {
    step(std::integral_constant<int, 0>{}, X, Y, yX, yY, qq);
    if (qq + 1 > qend) break;
    step(std::integral_constant<int, 1>{}, Y, X, yY, yX, qq + 1);
    if (qq + 2 > qend) break;
    step(std::integral_constant<int, 2>{}, X, Y, yX, yY, qq + 2);
    if (qq + 3 > qend) break;
    step(std::integral_constant<int, 3>{}, Y, X, yY, yX, qq + 3);
  }
  cp_async_wait<0>();
  __syncwarp();
}

// Partial row of one stored copy (its tet's micro-elements only).  Neighbour
// offsets: plane starts P(k) and row starts within planes k-1, k, k+1 are
// formed once; the 14 directions then only add constants.
template <class T, class KT>
__device__ __forceinline__ void scaled_partial(const DepthDev& D, const T* __restrict__ sten, const BCopy& cp,
                                               const T* __restrict__ u, const KT* __restrict__ k, T& y, T& diag) {
  const TetDev td = D.tets[cp.slot];
  const int N = td.N;
  const T* st = sten + (cp.slot * 16 + cp.mask) * kNDir;
  const T* ut = u + td.base;
  const KT* kt = k + td.base;
  const int ci = cp.i, cj = cp.j, ck = cp.k;
  // plane start of plane kk and start of row jj in it
  auto pstart = [&](int kk) { return (int)(tetnum(N + 1) - tetnum(N + 1 - kk)); };
  auto rstart = [&](int pk, int kk, int jj) { return pk + jj * (N - kk + 1) - jj * (jj - 1) / 2; };
  const int p0 = pstart(ck);
  const int pm = ck > 0 ? pstart(ck - 1) : 0;
  const int pp = ck < N ? pstart(ck + 1) : 0;
  const int x = rstart(p0, ck, cj) + ci;
  const T ux = ut[x];
  const T kx = (T)ldk(kt, x);
#pragma unroll
  for (int d = 0; d < kNDir; ++d) {
    int di, dj, dk;
    dir_of(d, di, dj, dk);
    const int a = ci + di, b = cj + dj, cc = ck + dk;
    if (a < 0 || b < 0 || cc < 0 || a + b + cc > N) continue;
    const int ps = dk == 0 ? p0 : (dk < 0 ? pm : pp);
    const int idx = rstart(ps, cc, b) + a;
    const T sv = st[d] * (kx + (T)ldk(kt, idx));
    y = fma(sv, ut[idx] - ux, y);
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
    val = ux + sdiv((T)p.omega * (__ldg(static_cast<const T*>(p.f) + i0) - y), diag);
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
// 32 interface nodes.  Dynamic shared memory: one staging ring per warp.
template <class T, class KT, int MODE>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 2 : 4) scaled_op_kernel(DepthDev D, OpPtrs p, int n_items, int n_bnodes,
                                                            unsigned* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  (void)err;
  const T* sten = nullptr;
  if constexpr (sizeof(T) == 8)
    sten = reinterpret_cast<const T*>(D.sten64);
  else
    sten = reinterpret_cast<const T*>(D.sten32);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned char* ring = smem_raw + wib * Stage<T, KT>::warp_bytes;
  const unsigned ring_s = smem_addr(ring);
  const CopyLane cl = copy_lane<T, KT>(lane);
  // Work in quads of 4 positions (one per warp of a block): volume quads
  // (4 consecutive items: the work list groups j-stacked tiles in fours) and
  // interface quads (4 chunks of 32 nodes) spread evenly among them.
  const int nchunks = (n_bnodes + 31) / 32;
  const int vq = (n_items + 3) / 4, bq = (nchunks + 3) / 4;
  const int totq = vq + bq;
  const int R = bq ? max(1, totq / bq) : totq + 1;
  for (int it = warp; it < 4 * totq; it += nwarps) {
    const int qd = it >> 2, sub = it & 3;
    const int before = min(bq, qd / R);  // interface quads before this one
    if (qd % R == R - 1 && qd / R < bq) {
      const int b = ((qd / R) * 4 + sub) * 32 + lane;
      if (b < n_bnodes) boundary_node<T, KT, MODE>(D, sten, b, p);
    } else {
      const int v = (qd - before) * 4 + sub;
      if (v < n_items) volume_item<T, KT, MODE>(D, sten, D.items[v], lane, p, ring, ring_s, cl);
    }
  }
}

// Interface rows on their own: one thread per unique boundary node, launched
// on the mesh's side stream ahead of the volume kernel (its blocks take the
// SMs first and the persistent volume blocks start as they drain), instead
// of as chunks inside the volume kernel's loop.
template <class T, class KT, int MODE>
__global__ void __launch_bounds__(128) boundary_only_kernel(DepthDev D, OpPtrs p, int n_b) {
  const T* sten;
  if constexpr (sizeof(T) == 8)
    sten = reinterpret_cast<const T*>(D.sten64);
  else
    sten = reinterpret_cast<const T*>(D.sten32);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_b; b += gridDim.x * blockDim.x)
    boundary_node<T, KT, MODE>(D, sten, b, p);
}

template <class T, class KT>
constexpr int ring_bytes() {
  return 4 * Stage<T, KT>::warp_bytes;  // 4 warps per block
}

template <class T, class KT, int MODE>
static int occupancy() {
  static int occ = 0;
  if (!occ) {
    HHG_CUDA(cudaFuncSetAttribute(scaled_op_kernel<T, KT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ring_bytes<T, KT>()));
    HHG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, scaled_op_kernel<T, KT, MODE>, 128,
                                                           ring_bytes<T, KT>()));
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
  init_march_configs(dtype);
  if (dtype == HHG_F64 || dtype == kF64KBF16)
    init_typed<double, double>();
  else if (dtype == HHG_F32)
    init_typed<float, float>();
  else
    init_typed<float, __nv_bfloat16>();
}

template <class T, class KT, int MODE>
static void launch_typed(const Mesh& m, int depth, int dtype, const OpArgs& a, const void* kptr, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  const DepthDev& D = Dh.dev;
  const int n_items = a.nc_only ? D.n_items_nc : D.n_items;
  const int n_b = a.nc_only ? D.n_bnodes_nc : D.n_bnodes;
  const int work = n_items + (n_b + 31) / 32;
  if (work == 0) return;
  const int occ = occupancy<T, KT, MODE>();
  OpPtrs p{a.u, kptr, a.f, a.out, a.d_in, a.d_out, a.omega, a.ca, a.cb};
  if (n_items > 0 && n_b > 0 && m.side) {
    // fork: interface rows on the side stream, volume rows here; join before
    // returning (also valid inside a stream capture)
    HHG_CUDA(cudaEventRecord(m.side_fork, s));
    HHG_CUDA(cudaStreamWaitEvent(m.side, m.side_fork, 0));
    boundary_only_kernel<T, KT, MODE><<<(n_b + 127) / 128, 128, 0, m.side>>>(D, p, n_b);
    HHG_CUDA(cudaGetLastError());
    HHG_CUDA(cudaEventRecord(m.side_join, m.side));
    if (m.vkernel >= 1) {
      launch_march(m, depth, dtype, (OpMode)MODE, a, s);
    } else {
      const int blocks = std::min((n_items + 3) / 4, m.num_sms * occ);
      scaled_op_kernel<T, KT, MODE><<<blocks, 128, ring_bytes<T, KT>(), s>>>(D, p, n_items, 0, m.d_error);
      HHG_CUDA(cudaGetLastError());
    }
    HHG_CUDA(cudaStreamWaitEvent(s, m.side_join, 0));
    return;
  }
  if (m.vkernel >= 1 && n_items > 0) {
    launch_march(m, depth, dtype, (OpMode)MODE, a, s);
    if (n_b > 0) {
      boundary_only_kernel<T, KT, MODE><<<(n_b + 127) / 128, 128, 0, s>>>(D, p, n_b);
      HHG_CUDA(cudaGetLastError());
    }
    return;
  }
  const int blocks = std::min((work + 3) / 4, m.num_sms * occ);
  scaled_op_kernel<T, KT, MODE><<<blocks, 128, ring_bytes<T, KT>(), s>>>(D, p, n_items, n_b, m.d_error);
  HHG_CUDA(cudaGetLastError());
}

template <int MODE>
static void launch_mode(const Mesh& m, int depth, int dtype, const OpArgs& a, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  if (dtype == HHG_F64)
    launch_typed<double, double, MODE>(m, depth, dtype, a, Dh.k64, s);
  else if (dtype == kF64KBF16)
    launch_typed<double, double, MODE>(m, depth, dtype, a, Dh.k16d, s);
  else if (dtype == HHG_F32)
    launch_typed<float, float, MODE>(m, depth, dtype, a, Dh.k32, s);
  else
    launch_typed<float, __nv_bfloat16, MODE>(m, depth, dtype, a, Dh.k16, s);
}

void launch_scaled_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, cudaStream_t s) {
  if (m.kappa) {  // the pre-asymptotic modification of Sec. 4 (kappa.cu)
    launch_kappa_op(m, depth, dtype, mode, a, s);
    return;
  }
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

// Partial nodal-integration row of one copy; with DIAG the copy's part of the
// diagonal (-sum of the off-diagonal entries) is subtracted into *dg.
template <class T, class KT, bool DIAG = false>
__device__ __forceinline__ T nodal_partial(const TetDev& td, const T* __restrict__ elem, int i, int j, int k,
                                           const T* __restrict__ u, const KT* __restrict__ kk, bool check,
                                           T* dg = nullptr) {
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
    T ksum = 0, inner = 0, asum = 0;
    const T* A = elem + E.sigma * 16 + E.v * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q == E.v) {
        ksum += kx;
      } else {
        ksum += (T)ldk(kk, idx[q]);
        inner = fma(A[q], u[idx[q]] - ux, inner);
        if (DIAG) asum += A[q];
      }
    }
    y = fma(ksum, inner, y);
    if (DIAG) *dg = fma(-ksum, asum, *dg);
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

// Staged nodal-integration volume kernel: the same tiles, work list and
// shared-memory staging as the scaled kernel, but three planes in registers
// (q-2, q-1, q): the 24 micro tets around a node of plane q-1 span planes
// q-2 .. q.  The tet's element matrices (6 Kuhn types, symmetric, 36 distinct
// off-diagonal entries of (1/4) A_t) are held in registers; every micro tet
// of every node is unrolled at compile time.
constexpr NodalTable kNodalC = make_nodal_table();

template <int S, int V, int W>
struct EIdx {  // register slot of (1/4) A_sigma[v][w], v != w (symmetric pairs share a slot)
  static constexpr int a = V < W ? V : W, b = V < W ? W : V;
  static constexpr int pair = a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);  // (0,1)..(0,3)->0..2, (1,2)->3, (1,3)->4, (2,3)->5
  static constexpr int value = S * 6 + pair;
};

template <int DI, int MM, class P2, class T>
__device__ __forceinline__ P2 plane_at(const Plane<T>& P) {
  if constexpr (DI == 0)
    return P.c0[MM];
  else if constexpr (DI > 0)
    return P.cp[MM];
  else
    return P.cm[MM];
}

template <int DK, int DI, int MM, class T>
__device__ __forceinline__ typename Pair<T>::type at3(const Plane<T>& A, const Plane<T>& B, const Plane<T>& C) {
  using P2 = typename Pair<T>::type;
  if constexpr (DK < 0)
    return plane_at<DI, MM, P2>(A);
  else if constexpr (DK == 0)
    return plane_at<DI, MM, P2>(B);
  else
    return plane_at<DI, MM, P2>(C);
}

// contribution of micro tet E of node row R: ksum * sum_w A[v][w] (u_w - u_x)
template <int E, int R, class T>
__device__ __forceinline__ T nodal_term(const Plane<T>& A, const Plane<T>& B, const Plane<T>& C, const T (&el)[36],
                                        T ux, T kx) {
  constexpr NodalEntry en = kNodalC.e[E];
  constexpr int v = en.v;
  T ks = kx, inner = 0;
#define HHG_NODAL_VERT(QQ)                                                                              \
  if constexpr (QQ != v) {                                                                            \
    constexpr int di = en.off[QQ][0], dj = en.off[QQ][1], dk = en.off[QQ][2];                          \
    const auto w = at3<dk, di, R + 1 + dj, T>(A, B, C);                                                 \
    ks += w.y;                                                                                          \
    inner = fma(el[EIdx<en.sigma, v, QQ>::value], w.x - ux, inner);                                    \
  }
  HHG_NODAL_VERT(0)
  HHG_NODAL_VERT(1)
  HHG_NODAL_VERT(2)
  HHG_NODAL_VERT(3)
#undef HHG_NODAL_VERT
  return ks * inner;
}

template <int R, class T, int... E>
__device__ __forceinline__ T nodal_row(const Plane<T>& A, const Plane<T>& B, const Plane<T>& C, const T (&el)[36],
                                       std::integer_sequence<int, E...>) {
  const T ux = B.c0[R + 1].x, kx = B.c0[R + 1].y;
  T y = 0;
  ((y += nodal_term<E, R, T>(A, B, C, el, ux, kx)), ...);
  return y;
}

template <class T, class KT>
__device__ void nodal_item(const DepthDev& D, const T* __restrict__ elem, int4 item, int lane, const OpPtrs& p,
                           unsigned char* ring, unsigned ring_s, const CopyLane& cl) {
  if (item.z < item.y) return;  // padding item: no planes
  const unsigned tile = (unsigned)item.x;
  const int slot = (int)(tile >> 20);
  const int j0 = (int)((tile >> 10) & 1023u), i0 = (int)(tile & 1023u);
  const int k0 = item.y;
  const TetDev td = D.tets[slot];
  const int N = td.N;
  const int qend = min(item.z + 1, N - (i0 + j0));
  const int h = lane / kTileI, l = lane % kTileI;
  const int i = i0 + l;
  const int jb = j0 + kTJ * h;
  T el[36];
#pragma unroll
  for (int s6 = 0; s6 < 6; ++s6) {
    const T* E = elem + slot * 96 + s6 * 16;
    el[s6 * 6 + 0] = E[1];
    el[s6 * 6 + 1] = E[2];
    el[s6 * 6 + 2] = E[3];
    el[s6 * 6 + 3] = E[6];
    el[s6 * 6 + 4] = E[7];
    el[s6 * 6 + 5] = E[11];
  }
  const T* u = static_cast<const T*>(p.u) + td.base;
  const KT* k = static_cast<const KT*>(p.k) + td.base;
  T* out = static_cast<T*>(p.out) + td.base;
  const int bmod_u = (int)(td.base & (RowGeom<T>::V - 1));
  const int bmod_k = (int)(td.base & (RowGeom<KT>::V - 1));
  const long long lim64 = D.n_stored - td.base;
  const int lim = lim64 > 0x7fffffffLL ? 0x7fffffff : (int)lim64;
  Head ch, rh;
  {
    const int qq = k0 - 1;
    const int M = N - qq;
    ch.q = rh.q = qq;
    ch.Psz = rh.Psz = (M + 1) * (M + 2) / 2;
    const int pl = (int)(tetnum(N + 1) - tetnum(N + 1 - qq));
    ch.A = M - j0 + 2;
    ch.e0 = pl + (j0 - 1) * (M + 1) - (j0 - 1) * (j0 - 2) / 2 + (i0 - 1);
    rh.A = M - jb + 2;
    rh.e0 = pl + (jb - 1) * (M + 1) - (jb - 1) * (jb - 2) / 2 + (i0 - 1);
  }
  constexpr int SB = Stage<T, KT>::bytes;
  const unsigned char* cbase_u = reinterpret_cast<const unsigned char*>(u);
  const unsigned char* cbase_k = reinterpret_cast<const unsigned char*>(k);
  const int lane_u = (kTJ * h * RowGeom<T>::stride + l) * (int)sizeof(T);
  const int lane_k = Stage<T, KT>::u_bytes + (kTJ * h * RowGeom<KT>::stride + l) * (int)sizeof(KT);
  int st_c = 0, st_r = 0;
  auto issue_next = [&]() {
    if (ch.q <= qend) issue_plane<T, KT>(ring_s + st_c * SB, ch, cl, N, j0 - 1, lim, bmod_u, bmod_k, cbase_u, cbase_k, true);
    cp_async_commit();
    ch.next(N, j0 - 1);
    st_c = st_c + 1 == kStages ? 0 : st_c + 1;
  };
  auto read_next = [&](Plane<T>& P) {
    const unsigned char* sb = ring + st_r * SB;
    read_plane<T, KT>(P, sb + lane_u, sb + lane_k, rh, bmod_u, bmod_k);
    rh.next(N, jb - 1);
    st_r = st_r + 1 == kStages ? 0 : st_r + 1;
  };
#pragma unroll
  for (int t = 0; t < kStages - 1; ++t) issue_next();
  Plane<T> X, Y, Z;
  cp_async_wait<kStages - 2>();
  __syncwarp();
  read_next(X);  // plane k0-1
  __syncwarp();
  issue_next();
  cp_async_wait<kStages - 2>();
  __syncwarp();
  read_next(Y);  // plane k0
  auto step = [&](const Plane<T>& A, const Plane<T>& B, Plane<T>& C, int qq) {
    __syncwarp();
    issue_next();
    cp_async_wait<kStages - 2>();
    __syncwarp();
    read_next(C);  // plane qq
    const int pl = qq - 1;
    const int lim_r = N - 1 - i - jb - pl;
    constexpr auto seq = std::make_integer_sequence<int, 24>{};
    const T y0 = nodal_row<0>(A, B, C, el, seq);
    const T y1 = nodal_row<1>(A, B, C, el, seq);
    const T y2 = nodal_row<2>(A, B, C, el, seq);
    const T y3 = nodal_row<3>(A, B, C, el, seq);
    if (0 <= lim_r) out[B.off[0] + l + 1] = y0;
    if (1 <= lim_r) out[B.off[1] + l + 1] = y1;
    if (2 <= lim_r) out[B.off[2] + l + 1] = y2;
    if (3 <= lim_r) out[B.off[3] + l + 1] = y3;
  };
  for (int qq = k0 + 1; qq <= qend; qq += 3) {
    step(X, Y, Z, qq);
    if (qq + 1 > qend) break;
    step(Y, Z, X, qq + 1);
    if (qq + 2 > qend) break;
    step(Z, X, Y, qq + 2);
  }
  cp_async_wait<0>();
  __syncwarp();
}

template <class T, class KT>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 2 : 3) nodal_staged_kernel(DepthDev D, OpPtrs p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const T* elem;
  if constexpr (sizeof(T) == 8)
    elem = reinterpret_cast<const T*>(D.elem64);
  else
    elem = reinterpret_cast<const T*>(D.elem32);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned char* ring = smem_raw + wib * Stage<T, KT>::warp_bytes;
  const unsigned ring_s = smem_addr(ring);
  const CopyLane cl = copy_lane<T, KT>(lane);
  for (int it = warp; it < D.n_items; it += nwarps) nodal_item<T, KT>(D, elem, D.items[it], lane, p, ring, ring_s, cl);
}

template <class T, class KT>
static void nodal_typed(const Mesh& m, int depth, const void* u, const void* kk, void* y, cudaStream_t s) {
  const DepthDev& D = m.depth[depth].dev;
  // interface rows on the side stream, concurrent with the volume kernel
  const bool fork = D.n_items > 0 && D.n_bnodes > 0 && m.side;
  if (fork) {
    HHG_CUDA(cudaEventRecord(m.side_fork, s));
    HHG_CUDA(cudaStreamWaitEvent(m.side, m.side_fork, 0));
    nodal_boundary_kernel<T, KT><<<(D.n_bnodes + 127) / 128, 128, 0, m.side>>>(
        D, static_cast<const T*>(u), static_cast<const KT*>(kk), static_cast<T*>(y));
    HHG_CUDA(cudaGetLastError());
    HHG_CUDA(cudaEventRecord(m.side_join, m.side));
  }
  if (D.n_items > 0) {
    static int occ = 0;
    const int smem = 4 * Stage<T, KT>::warp_bytes;
    if (!occ) {
      HHG_CUDA(cudaFuncSetAttribute(nodal_staged_kernel<T, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      HHG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, nodal_staged_kernel<T, KT>, 128, smem));
      if (occ < 1) occ = 1;
    }
    const int blocks = std::min((D.n_items + 3) / 4, m.num_sms * occ);
    OpPtrs p{u, kk, nullptr, y, nullptr, nullptr, 0, 0, 0};
    nodal_staged_kernel<T, KT><<<blocks, 128, smem, s>>>(D, p);
    HHG_CUDA(cudaGetLastError());
  }
  if (fork) {
    HHG_CUDA(cudaStreamWaitEvent(s, m.side_join, 0));
  } else if (D.n_bnodes > 0) {
    nodal_boundary_kernel<T, KT><<<(D.n_bnodes + 127) / 128, 128, 0, s>>>(
        D, static_cast<const T*>(u), static_cast<const KT*>(kk), static_cast<T*>(y));
    HHG_CUDA(cudaGetLastError());
  }
}

// ---------------------------------------------------------------------------
// Diagonal of the nodal-integration operator: sum over the micro tets at a
// node of kbar_t A_t[x][x] = -kbar_t sum_{w != x} A_t[x][w] (zero row sums),
// summed over the copies of interface nodes; written as 1/diag, 0 on
// Dirichlet nodes (Jacobi then leaves them unchanged).
// ---------------------------------------------------------------------------
template <class T, class KT>
__device__ __forceinline__ T nodal_diag_partial(const TetDev& td, const T* __restrict__ elem, int i, int j, int k,
                                                const KT* __restrict__ kk, bool check) {
  const int N = td.N;
  const T kx = (T)ldk(kk, td.base + node_offset(N, i, j, k));
  T dg = 0;
  for (int e = 0; e < 24; ++e) {
    const NodalEntry& E = kNodal.e[e];
    bool ok = true;
    T ksum = 0, asum = 0;
    const T* A = elem + E.sigma * 16 + E.v * 4;
    for (int q = 0; q < 4; ++q) {
      const int a = i + E.off[q][0], b = j + E.off[q][1], c = k + E.off[q][2];
      if (check && (a < 0 || b < 0 || c < 0 || a + b + c > N)) ok = false;
      if (!ok) break;
      if (q == E.v) {
        ksum += kx;
      } else {
        ksum += (T)ldk(kk, td.base + node_offset(N, a, b, c));
        asum += A[q];
      }
    }
    if (ok) dg -= ksum * asum;
  }
  return dg;
}

template <class T, class KT>
__global__ void nodal_dinv_kernel(DepthDev D, const KT* __restrict__ kk, T* __restrict__ dinv) {
  const T* elem;
  if constexpr (sizeof(T) == 8)
    elem = reinterpret_cast<const T*>(D.elem64);
  else
    elem = reinterpret_cast<const T*>(D.elem32);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < D.n_rows; r += nwarps) {  // volume nodes
    const int4 row = D.rows[r];
    const TetDev td = D.tets[row.x];
    const int N = td.N, j = row.y, k = row.z;
    if (j == 0 || k == 0 || j + k >= N - 1) continue;
    for (int i = 1 + lane; i + j + k <= N - 1; i += 32)
      dinv[td.base + node_offset(N, i, j, k)] = (T)1 / nodal_diag_partial<T, KT>(td, elem + row.x * 96, i, j, k, kk, false);
  }
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < D.n_bnodes; b += gridDim.x * blockDim.x) {
    const int lo = D.bstart[b], hi = D.bstart[b + 1];
    T v = 0;
    if (!D.bdir[b]) {
      T dg = 0;
      for (int q = lo; q < hi; ++q) {
        const BCopy cp = D.bcopies[q];
        dg += nodal_diag_partial<T, KT>(D.tets[cp.slot], elem + cp.slot * 96, cp.i, cp.j, cp.k, kk, true);
      }
      v = (T)1 / dg;
    }
    for (int q = lo; q < hi; ++q) dinv[D.bcopies[q].idx] = v;
  }
}

// residual / Jacobi / diagonal epilogue of the nodal operator from y = A_n u
template <class T, int MODE>
__global__ void nodal_epilogue_kernel(const T* __restrict__ y, const T* __restrict__ u, const T* __restrict__ f,
                                      const T* __restrict__ dinv, T* __restrict__ out, double omega, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const bool dir = dinv[i] == (T)0;
    if (MODE == OP_RESID) {
      out[i] = dir ? (T)0 : f[i] - y[i];
    } else if (MODE == OP_JACOBI) {
      out[i] = dir ? (T)0 : u[i] + (T)omega * (f[i] - y[i]) * dinv[i];
    } else {  // OP_DIAG
      out[i] = dir ? (T)1 : (T)1 / dinv[i];
    }
  }
}

template <class T, class KT>
static void nodal_dinv_typed(const Mesh& m, int depth, const void* kk, void* dinv, cudaStream_t s) {
  const DepthDev& D = m.depth[depth].dev;
  const int g = std::max(1, std::min(8 * m.num_sms, std::max((D.n_rows + 7) / 8, (D.n_bnodes + 255) / 256)));
  nodal_dinv_kernel<T, KT><<<g, 256, 0, s>>>(D, static_cast<const KT*>(kk), static_cast<T*>(dinv));
  HHG_CUDA(cudaGetLastError());
}

void launch_nodal_dinv(const Mesh& m, int depth, int dtype, void* dinv, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  if (dtype == HHG_F64)
    nodal_dinv_typed<double, double>(m, depth, Dh.k64, dinv, s);
  else if (dtype == kF64KBF16)
    nodal_dinv_typed<double, double>(m, depth, Dh.k16d, dinv, s);
  else if (dtype == HHG_F32)
    nodal_dinv_typed<float, float>(m, depth, Dh.k32, dinv, s);
  else
    nodal_dinv_typed<float, __nv_bfloat16>(m, depth, Dh.k16, dinv, s);
}

// Nodal-integration operator with the scaled kernel's modes: y = A_n u into
// `tmp` (the fast staged kernels), then the pointwise epilogue with 1/diag.
void launch_nodal_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, const void* dinv, void* tmp,
                     cudaStream_t s) {
  HHG_REQUIRE(mode == OP_APPLY || mode == OP_RESID || mode == OP_JACOBI || mode == OP_DIAG,
              "the nodal operator has no Chebyshev mode");
  const long long n = a.nc_only ? m.depth[depth].n_stored_nc : m.depth[depth].n_stored;
  if (mode == OP_APPLY) {
    launch_nodal_apply(m, depth, dtype, a.u, a.out, s);
    return;
  }
  if (mode != OP_DIAG) launch_nodal_apply(m, depth, dtype, a.u, tmp, s);
  if (n == 0) return;
  const int g = (int)std::min<long long>((n + 255) / 256, 8LL * m.num_sms);
  const bool f64 = dtype == HHG_F64 || dtype == kF64KBF16;
#define HHG_EPI(T, MD)                                                                                          \
  nodal_epilogue_kernel<T, MD><<<g, 256, 0, s>>>(static_cast<const T*>(tmp), static_cast<const T*>(a.u),      \
                                                 static_cast<const T*>(a.f), static_cast<const T*>(dinv),     \
                                                 static_cast<T*>(a.out), a.omega, n)
  if (mode == OP_RESID) {
    if (f64) HHG_EPI(double, OP_RESID); else HHG_EPI(float, OP_RESID);
  } else if (mode == OP_JACOBI) {
    if (f64) HHG_EPI(double, OP_JACOBI); else HHG_EPI(float, OP_JACOBI);
  } else {
    if (f64) HHG_EPI(double, OP_DIAG); else HHG_EPI(float, OP_DIAG);
  }
#undef HHG_EPI
  HHG_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// "Scale Vol+Face" (Sec. 5, eq. "modst" with I = W_V u W_E): after the scaled
// launch, the rows of nodes on macro vertices and edges (face mask with two or
// more bits in every containing tet) are replaced by their nodal-integration
// rows, summed over the copies and written to every copy, with the same
// residual / Jacobi / diagonal epilogue as the scaled kernel.
// ---------------------------------------------------------------------------
// One warp per listed node: lanes take the (copy, micro tet) pairs, the warp
// sums the row and its diagonal, the lanes write the copies.
template <class T, class KT, int MODE>
__global__ void __launch_bounds__(128) volface_fixup_kernel(DepthDev D, OpPtrs p, int n_vf) {
  const T* elem;
  if constexpr (sizeof(T) == 8)
    elem = reinterpret_cast<const T*>(D.elem64);
  else
    elem = reinterpret_cast<const T*>(D.elem32);
  const T* u = static_cast<const T*>(p.u);
  const KT* kk = static_cast<const KT*>(p.k);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int w = warp; w < n_vf; w += nwarps) {
    const int b = D.vf[w];
    const int lo = D.bstart[b], hi = D.bstart[b + 1];
    T y = 0, dg = 0;
    for (int pr = lane; pr < (hi - lo) * 24; pr += 32) {
      const BCopy cp = D.bcopies[lo + pr / 24];
      const TetDev td = D.tets[cp.slot];
      const int N = td.N;
      const NodalEntry& E = kNodal.e[pr % 24];
      const long long x = td.base + node_offset(N, cp.i, cp.j, cp.k);
      const T ux = u[x], kx = (T)ldk(kk, x);
      const T* A = elem + cp.slot * 96 + E.sigma * 16 + E.v * 4;
      bool ok = true;
      T ksum = 0, inner = 0, asum = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = cp.i + E.off[q][0], bb = cp.j + E.off[q][1], c = cp.k + E.off[q][2];
        if (a < 0 || bb < 0 || c < 0 || a + bb + c > N) ok = false;
        if (!ok) continue;
        if (q == E.v) {
          ksum += kx;
        } else {
          const long long idx = td.base + node_offset(N, a, bb, c);
          ksum += (T)ldk(kk, idx);
          inner = fma(A[q], u[idx] - ux, inner);
          asum += A[q];
        }
      }
      if (ok) {
        y = fma(ksum, inner, y);
        dg = fma(-ksum, asum, dg);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      y += __shfl_xor_sync(0xffffffffu, y, o);
      dg += __shfl_xor_sync(0xffffffffu, dg, o);
    }
    const long long i0 = D.bcopies[lo].idx;
    T val = y;
    if (MODE == OP_RESID) {
      val = static_cast<const T*>(p.f)[i0] - y;
    } else if (MODE == OP_JACOBI) {
      val = u[i0] + (T)p.omega * (static_cast<const T*>(p.f)[i0] - y) / dg;
    } else if (MODE == OP_DIAG) {
      val = dg;
    }
    for (int q = lo + lane; q < hi; q += 32) static_cast<T*>(p.out)[D.bcopies[q].idx] = val;
  }
}

template <class T, class KT, int MODE>
static void volface_typed(const Mesh& m, int depth, const OpArgs& a, const void* kptr, cudaStream_t s) {
  const DepthDev& D = m.depth[depth].dev;
  const int n_vf = a.nc_only ? D.n_vf_nc : D.n_vf;
  if (n_vf == 0) return;
  OpPtrs p{a.u, kptr, a.f, a.out, nullptr, nullptr, a.omega, 0, 0};
  volface_fixup_kernel<T, KT, MODE><<<std::min((n_vf + 3) / 4, 16 * m.num_sms), 128, 0, s>>>(D, p, n_vf);
  HHG_CUDA(cudaGetLastError());
}

template <int MODE>
static void volface_mode(const Mesh& m, int depth, int dtype, const OpArgs& a, cudaStream_t s) {
  const Depth& Dh = m.depth[depth];
  if (dtype == HHG_F64)
    volface_typed<double, double, MODE>(m, depth, a, Dh.k64, s);
  else if (dtype == kF64KBF16)
    volface_typed<double, double, MODE>(m, depth, a, Dh.k16d, s);
  else if (dtype == HHG_F32)
    volface_typed<float, float, MODE>(m, depth, a, Dh.k32, s);
  else
    volface_typed<float, __nv_bfloat16, MODE>(m, depth, a, Dh.k16, s);
}

void launch_volface_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, cudaStream_t s) {
  HHG_REQUIRE(mode != OP_CHEB, "the Vol+Face operator has no Chebyshev mode");
  launch_scaled_op(m, depth, dtype, mode, a, s);
  switch (mode) {
    case OP_APPLY: volface_mode<OP_APPLY>(m, depth, dtype, a, s); break;
    case OP_RESID: volface_mode<OP_RESID>(m, depth, dtype, a, s); break;
    case OP_JACOBI: volface_mode<OP_JACOBI>(m, depth, dtype, a, s); break;
    case OP_DIAG: volface_mode<OP_DIAG>(m, depth, dtype, a, s); break;
    default: break;
  }
}

// ---------------------------------------------------------------------------
// Consistent mass matrix y = M u (setup of the right-hand side M I_h f,
// Sec. 7.2): per-primitive stencils, every input entry used (including
// Dirichlet nodes), Dirichlet rows set to 0.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T mass_partial(const TetDev& td, const T* __restrict__ ms, int i, int j, int k,
                                          const T* __restrict__ u) {
  const int N = td.N;
  T y = ms[14] * u[td.base + node_offset(N, i, j, k)];
#pragma unroll
  for (int d = 0; d < kNDir; ++d) {
    int di, dj, dk;
    dir_of(d, di, dj, dk);
    const int a = i + di, b = j + dj, c = k + dk;
    if (a < 0 || b < 0 || c < 0 || a + b + c > N) continue;
    y = fma(ms[d], u[td.base + node_offset(N, a, b, c)], y);
  }
  return y;
}

template <class T>
__global__ void mass_volume_kernel(DepthDev D, const T* __restrict__ mass, const T* __restrict__ u, T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < D.n_rows; r += nwarps) {
    const int4 row = D.rows[r];
    const TetDev td = D.tets[row.x];
    const int N = td.N, j = row.y, k = row.z;
    if (j == 0 || k == 0 || j + k >= N - 1) continue;
    const T* ms = mass + row.x * 16 * 15;  // volume row (mask 0)
    for (int i = 1 + lane; i + j + k <= N - 1; i += 32)
      y[td.base + node_offset(N, i, j, k)] = mass_partial<T>(td, ms, i, j, k, u);
  }
}

template <class T>
__global__ void mass_boundary_kernel(DepthDev D, const T* __restrict__ mass, const T* __restrict__ u, T* __restrict__ y) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= D.n_bnodes) return;
  const int lo = D.bstart[b], hi = D.bstart[b + 1];
  T v = 0;
  if (!D.bdir[b])
    for (int q = lo; q < hi; ++q) {
      const BCopy cp = D.bcopies[q];
      v += mass_partial<T>(D.tets[cp.slot], mass + (cp.slot * 16 + cp.mask) * 15, cp.i, cp.j, cp.k, u);
    }
  for (int q = lo; q < hi; ++q) y[D.bcopies[q].idx] = v;
}

template <class T>
static void mass_typed(const Mesh& m, int depth, const T* mass, const void* u, void* y, cudaStream_t s) {
  const DepthDev& D = m.depth[depth].dev;
  if (D.n_rows > 0) {
    const int blocks = std::min((D.n_rows + 7) / 8, m.num_sms * 8);
    mass_volume_kernel<T><<<blocks, 256, 0, s>>>(D, mass, static_cast<const T*>(u), static_cast<T*>(y));
    HHG_CUDA(cudaGetLastError());
  }
  if (D.n_bnodes > 0) {
    mass_boundary_kernel<T><<<(D.n_bnodes + 127) / 128, 128, 0, s>>>(D, mass, static_cast<const T*>(u),
                                                                      static_cast<T*>(y));
    HHG_CUDA(cudaGetLastError());
  }
}

void launch_mass_apply(const Mesh& m, int depth, int dtype, const void* u, void* y, cudaStream_t s) {
  const DepthDev& D = m.depth[depth].dev;
  if (dtype == HHG_F64)
    mass_typed<double>(m, depth, D.mass64, u, y, s);
  else
    mass_typed<float>(m, depth, D.mass32, u, y, s);
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
