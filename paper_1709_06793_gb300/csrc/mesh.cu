// Host-side construction of the hierarchical hybrid grid: index spaces, the
// 15 reference stencils per macro tet and level, micro-element matrices,
// interface (face/edge/vertex) copy maps, work lists and coarse problems.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>

#include "hhg_internal.h"

namespace hhg {

void* dalloc(Depth& d, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) throw Error{HHG_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
  d.allocations.push_back(p);
  return p;
}

template <class T>
static T* upload(Depth& d, const std::vector<T>& h) {
  T* p = static_cast<T*>(dalloc(d, h.size() * sizeof(T)));
  if (!h.empty()) HHG_CUDA(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return p;
}

// ---------------------------------------------------------------------------
// Micro tetrahedra around a node.  Uniform refinement by Bey's rule with the
// vertex order kept is, in the coordinates (a,b,c) = (i+j+k, j+k, k), the
// Freudenthal triangulation of the simplex N >= a >= b >= c >= 0: every unit
// cube [B, B+1] splits into the 6 simplices B, B+e_s0, B+e_s0+e_s1, B+1 over
// the permutations s.  (The oracle refines recursively; the tests check both
// agree.)
// ---------------------------------------------------------------------------
static const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

struct Micro {
  int sigma;          // Kuhn type (permutation index)
  int v;              // local vertex index of the centre node
  int ijk[4][3];      // index coordinates of the 4 vertices (path order)
};

static void kuhn_to_index(const int abc[3], int out[3]) {
  out[0] = abc[0] - abc[1];
  out[1] = abc[1] - abc[2];
  out[2] = abc[2];
}

// Micro tets of a tet with N = 2^level that have node (i,j,k) as a vertex.
static std::vector<Micro> micro_at(int N, int i, int j, int k) {
  std::vector<Micro> out;
  const int P[3] = {i + j + k, j + k, k};
  for (int dm = 0; dm < 8; ++dm) {
    const int delta[3] = {(dm >> 2) & 1, (dm >> 1) & 1, dm & 1};
    const int B[3] = {P[0] - delta[0], P[1] - delta[1], P[2] - delta[2]};
    for (int s = 0; s < 6; ++s) {
      int cur[3] = {B[0], B[1], B[2]};
      int verts[4][3];
      for (int q = 0; q < 4; ++q) {
        if (q > 0) cur[kPerm[s][q - 1]] += 1;
        verts[q][0] = cur[0];
        verts[q][1] = cur[1];
        verts[q][2] = cur[2];
      }
      int v = -1;
      bool inside = true;
      for (int q = 0; q < 4; ++q) {
        if (verts[q][0] == P[0] && verts[q][1] == P[1] && verts[q][2] == P[2]) v = q;
        if (!(N >= verts[q][0] && verts[q][0] >= verts[q][1] && verts[q][1] >= verts[q][2] && verts[q][2] >= 0))
          inside = false;
      }
      if (v < 0 || !inside) continue;
      Micro m;
      m.sigma = s;
      m.v = v;
      for (int q = 0; q < 4; ++q) kuhn_to_index(verts[q], m.ijk[q]);
      out.push_back(m);
    }
  }
  return out;
}

// P1 stiffness matrix of the tetrahedron X[4][3]: vol * grad phi_a . grad phi_b;
// with a direction d: vol * (d . grad phi_a)(d . grad phi_b) (one term of the
// tensor coefficient's split).
static void p1_stiffness(const double X[4][3], double A[4][4], const double* d = nullptr) {
  double J[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) J[r][c] = X[c + 1][r] - X[0][r];  // columns = edge vectors
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  HHG_REQUIRE(std::fabs(det) > 0.0, "degenerate tetrahedron");
  double Ji[3][3];  // inverse of J; grad phi_a (a=1..3) = row a-1 of J^-1
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  double G[4][3];
  for (int c = 0; c < 3; ++c) {
    G[1][c] = Ji[0][c];
    G[2][c] = Ji[1][c];
    G[3][c] = Ji[2][c];
    G[0][c] = -(G[1][c] + G[2][c] + G[3][c]);
  }
  const double vol = std::fabs(det) / 6.0;
  if (d) {
    double gd[4];
    for (int a = 0; a < 4; ++a) gd[a] = G[a][0] * d[0] + G[a][1] * d[1] + G[a][2] * d[2];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) A[a][b] = vol * gd[a] * gd[b];
    return;
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) A[a][b] = vol * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]);
}

static void index_to_phys(const Mesh& m, int tet, int N, const int ijk[3], double x[3]) {
  const int* g = &m.T[4 * tet];
  for (int r = 0; r < 3; ++r) {
    const double x0 = m.V[3 * g[0] + r];
    x[r] = x0 + (ijk[0] * (m.V[3 * g[1] + r] - x0) + ijk[1] * (m.V[3 * g[2] + r] - x0) +
                 ijk[2] * (m.V[3 * g[3] + r] - x0)) /
                    N;
  }
}

static int dir_index(int di, int dj, int dk) {
  for (int d = 0; d < kNDir; ++d) {
    int a, b, c;
    dir_of(d, a, b, c);
    if (a == di && b == dj && c == dk) return d;
  }
  return -1;
}

// A node of the given face-bit mask, if the level has one.
static bool representative(int N, int mask, int rep[3]) {
  const int cand[6] = {0, 1, 2, N - 2, N - 1, N};
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b)
      for (int c = 0; c < 6; ++c) {
        const int i = cand[a], j = cand[b], k = cand[c];
        if (i < 0 || j < 0 || k < 0 || i + j + k > N) continue;
        if (face_mask(N, i, j, k) == mask) {
          rep[0] = i;
          rep[1] = j;
          rep[2] = k;
          return true;
        }
      }
  return false;
}

// (1/2) reference stencil of each primitive (Sec. 2.2): column d of row `mask`
// = (1/2) sum over micro tets t in T containing x and x+w_d of int_t grad
// phi_x . grad phi_(x+w_d), x any node of that primitive.
void stencils_for(const Mesh& m, int tet, int level, double* out) {
  const int N = 1 << level;
  std::fill(out, out + 16 * kNDir, 0.0);
  for (int mask = 0; mask < 16; ++mask) {
    int rep[3];
    if (!representative(N, mask, rep)) continue;
    for (const Micro& mt : micro_at(N, rep[0], rep[1], rep[2])) {
      double X[4][3], A[4][4];
      for (int q = 0; q < 4; ++q) index_to_phys(m, tet, N, mt.ijk[q], X[q]);
      p1_stiffness(X, A);
      for (int q = 0; q < 4; ++q) {
        if (q == mt.v) continue;
        const int d = dir_index(mt.ijk[q][0] - rep[0], mt.ijk[q][1] - rep[1], mt.ijk[q][2] - rep[2]);
        HHG_REQUIRE(d >= 0, "internal: micro-tet edge not in the 15-point pattern");
        out[mask * kNDir + d] += 0.5 * A[mt.v][q];
      }
    }
  }
}

// Reference stencils of the six terms of a tensor coefficient (directions e1,
// e2, e3, e1-e2, e1-e3, e2-e3): out[m][mask][d] = (1/2) sum over the micro
// tets at the primitive's node of vol (d_m . grad phi_x)(d_m . grad phi_y).
void tensor_stencils_for(const Mesh& m, int tet, int level, double* out) {
  static const double dirs[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, -1, 0}, {1, 0, -1}, {0, 1, -1}};
  const int N = 1 << level;
  std::fill(out, out + 6 * 16 * kNDir, 0.0);
  for (int mask = 0; mask < 16; ++mask) {
    int rep[3];
    if (!representative(N, mask, rep)) continue;
    for (const Micro& mt : micro_at(N, rep[0], rep[1], rep[2])) {
      double X[4][3];
      for (int q = 0; q < 4; ++q) index_to_phys(m, tet, N, mt.ijk[q], X[q]);
      for (int t = 0; t < 6; ++t) {
        double A[4][4];
        p1_stiffness(X, A, dirs[t]);
        for (int q = 0; q < 4; ++q) {
          if (q == mt.v) continue;
          const int d = dir_index(mt.ijk[q][0] - rep[0], mt.ijk[q][1] - rep[1], mt.ijk[q][2] - rep[2]);
          HHG_REQUIRE(d >= 0, "internal: micro-tet edge not in the 15-point pattern");
          out[(t * 16 + mask) * kNDir + d] += 0.5 * A[mt.v][q];
        }
      }
    }
  }
}

// Device copies of the tensor stencils of every depth (built on first use).
void ensure_tensor_stencils(Mesh& m) {
  for (Depth& D : m.depth) {
    if (D.tsten64) continue;
    const int ns = (int)D.slot_tet.size();
    std::vector<double> h((size_t)std::max(ns, 1) * 6 * 16 * kNDir, 0.0);
    for (int s = 0; s < ns; ++s) {
      const int t = D.slot_tet[s];
      tensor_stencils_for(m, t, D.tet_level[t], &h[(size_t)s * 6 * 16 * kNDir]);
    }
    std::vector<float> h32(h.begin(), h.end());
    D.tsten64 = upload(D, h);
    D.tsten32 = upload(D, h32);
  }
}

// Consistent P1 mass matrix (|t|/20 (1 + delta_ab) per micro tet) in stencil
// form per primitive: column 14 = centre, columns 0..13 the directions.
void mass_stencils_for(const Mesh& m, int tet, int level, double* out) {
  const int N = 1 << level;
  std::fill(out, out + 16 * 15, 0.0);
  for (int mask = 0; mask < 16; ++mask) {
    int rep[3];
    if (!representative(N, mask, rep)) continue;
    for (const Micro& mt : micro_at(N, rep[0], rep[1], rep[2])) {
      double X[4][3];
      for (int q = 0; q < 4; ++q) index_to_phys(m, tet, N, mt.ijk[q], X[q]);
      double J[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) J[r][c] = X[c + 1][r] - X[0][r];
      const double vol = std::fabs(J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                   J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                   J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0])) / 6.0;
      out[mask * 15 + 14] += vol / 10.0;
      for (int q = 0; q < 4; ++q) {
        if (q == mt.v) continue;
        const int d = dir_index(mt.ijk[q][0] - rep[0], mt.ijk[q][1] - rep[1], mt.ijk[q][2] - rep[2]);
        HHG_REQUIRE(d >= 0, "internal: micro-tet edge not in the 15-point pattern");
        out[mask * 15 + d] += vol / 20.0;
      }
    }
  }
}

// (1/4) P1 stiffness matrix of the 6 Kuhn types of micro tet (vertices in
// path order), for the nodal-integration operator k_bar_t * A_t with
// k_bar_t = (1/4) sum of the vertex values (eq. "standardfe").
void elements_for(const Mesh& m, int tet, int level, double* out) {
  const int N = 1 << level;
  for (int s = 0; s < 6; ++s) {
    int abc[3] = {0, 0, 0};
    double X[4][3], A[4][4];
    for (int q = 0; q < 4; ++q) {
      if (q > 0) abc[kPerm[s][q - 1]] += 1;
      int ijk[3];
      kuhn_to_index(abc, ijk);
      index_to_phys(m, tet, N, ijk, X[q]);
    }
    p1_stiffness(X, A);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) out[s * 16 + a * 4 + b] = 0.25 * A[a][b];
  }
}

// ---------------------------------------------------------------------------
// Node identity: barycentric support in the macro mesh (vertex ids with
// non-zero integer weights), packed into 128 bits.
// ---------------------------------------------------------------------------
struct Key {
  uint64_t a, b;
  bool operator<(const Key& o) const { return a < o.a || (a == o.a && b < o.b); }
  bool operator==(const Key& o) const { return a == o.a && b == o.b; }
};

static Key node_key(const Mesh& m, int tet, int N, int i, int j, int k) {
  const int* g = &m.T[4 * tet];
  std::array<std::pair<int, int>, 4> p = {{{g[0], N - i - j - k}, {g[1], i}, {g[2], j}, {g[3], k}}};
  for (auto& q : p)
    if (q.second == 0) q.first = 0x7fffffff;
  std::sort(p.begin(), p.end());
  uint64_t w[4];
  for (int a = 0; a < 4; ++a)
    w[a] = p[a].second == 0 ? 0 : ((uint64_t)(uint32_t)p[a].first << 11) | (uint64_t)p[a].second;
  return Key{(w[0] << 32) | w[1], (w[2] << 32) | w[3]};
}

void node_coords(const Mesh& m, int depth, std::vector<double>& xyz) {
  const Depth& D = m.depth[depth];
  xyz.assign(3 * D.n_stored, 0.0);
  for (size_t s = 0; s < D.slot_tet.size(); ++s) {
    const int t = D.slot_tet[s];
    const int N = D.h_tets[s].N;
    const int* g = &m.T[4 * t];
    long long idx = D.h_tets[s].base;
    for (int k = 0; k <= N; ++k)
      for (int j = 0; j <= N - k; ++j)
        for (int i = 0; i <= N - j - k; ++i, ++idx) {
          std::array<std::pair<int, int>, 4> p = {{{g[0], N - i - j - k}, {g[1], i}, {g[2], j}, {g[3], k}}};
          std::sort(p.begin(), p.end());
          for (int r = 0; r < 3; ++r) {
            double x = 0.0;
            for (int a = 0; a < 4; ++a)
              if (p[a].second) x += ((double)p[a].second / N) * m.V[3 * p[a].first + r];
            xyz[3 * idx + r] = x;
          }
        }
  }
}

// ---------------------------------------------------------------------------
// Mesh construction
// ---------------------------------------------------------------------------
static int find(std::vector<int>& p, int x) {
  while (p[x] != x) x = p[x] = p[p[x]];
  return x;
}

// Volume work list: tiles of kTI x kTJ columns (i0, j0), 4 per warp item (one
// tet per item, equal i0+j0 where possible), each tile's k-march cut into
// segments of m.kseg planes; longest item first.
// k-segment length of a depth: the mesh's kseg, halved (down to 4) while the
// depth would have fewer volume items than resident warps (16 per SM), so
// that small depths still spread over the whole GPU
static int depth_kseg(const Mesh& m, const Depth& D) {
  const long long target = (long long)(m.num_sms > 0 ? m.num_sms : 152) * 16;
  auto count = [&](int ks) {
    long long c = 0;
    for (size_t s = 0; s < D.h_tets.size(); ++s) {
      const int N = D.h_tets[s].N;
      for (int j0 = 1; j0 <= N - 2; j0 += kWarpTileJ)
        for (int i0 = 1; i0 + j0 <= N - 2; i0 += kWarpTileI) c += (N - 1 - (i0 + j0) + ks - 1) / ks;
    }
    return c;
  };
  int ks = m.kseg;
  while (ks > 4 && count(ks) < target) ks /= 2;
  return ks;
}

void build_items(const Mesh& m, Depth& D) {
  const int ns = (int)D.slot_tet.size();
  const int empty_tile = 1023 << 10 | 1023;
  const int kseg = depth_kseg(m, D);
  std::vector<std::vector<int4>> by_class(2);
  for (int cls = 0; cls < 2; ++cls) {
    std::vector<std::pair<long long, int4>> its;  // (sort key, item)
    for (int s = 0; s < ns; ++s) {
      if ((s < D.n_slots_nc) != (cls == 0)) continue;
      const int N = D.h_tets[s].N;
      if (m.korder == 2) {
        // quads: the 4 warps of a block take 4 tiles stacked in j (same i0,
        // same plane window), so the halo rows they share are fetched once
        const int jstack = 4 * kWarpTileJ;
        for (int k0 = 1; k0 <= N - 3; k0 += kseg)
          for (int jg = 1; jg <= N - 2; jg += jstack)
            for (int i0 = 1; i0 + jg <= N - 2; i0 += kWarpTileI) {
              int4 q[4];
              int live = 0;
              for (int w = 0; w < 4; ++w) {
                const int j0 = jg + w * kWarpTileJ;
                const int top = N - 1 - (i0 + j0);
                if (j0 <= N - 2 && top >= k0) {
                  q[w] = make_int4(s << 20 | j0 << 10 | i0, k0, std::min(top, k0 + kseg - 1), 0);
                  ++live;
                } else {
                  q[w] = make_int4(s << 20 | empty_tile, 1, 0, 0);  // no planes
                }
              }
              if (!live) continue;
              const long long key = ((long long)k0 << 40) | ((long long)s << 28) | ((long long)i0 << 14) | jg;
              for (int w = 0; w < 4; ++w) its.push_back({key, q[w]});
            }
      } else {
        for (int j0 = 1; j0 <= N - 2; j0 += kWarpTileJ)
          for (int i0 = 1; i0 + j0 <= N - 2; i0 += kWarpTileI) {
            const int tile = s << 20 | j0 << 10 | i0;
            const int top = N - 1 - (i0 + j0);  // last plane with a volume node in the tile
            for (int k0 = 1; k0 <= top; k0 += kseg) {
              const int k1 = std::min(top, k0 + kseg - 1);
              const long long key = m.korder == 1 ? k0 : -(long long)(k1 - k0 + 1);
              its.push_back({key, make_int4(tile, k0, k1, 0)});
            }
          }
        while (its.size() % 4) its.push_back({its.empty() ? 0 : its.back().first, make_int4(s << 20 | empty_tile, 1, 0, 0)});
      }
    }
    std::stable_sort(its.begin(), its.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    for (auto& p : its) by_class[cls].push_back(p.second);
  }
  D.h_items = by_class[0];
  D.n_items_nc = (int)D.h_items.size();
  D.h_items.insert(D.h_items.end(), by_class[1].begin(), by_class[1].end());
  D.n_items = (int)D.h_items.size();
  build_march_items(m, D);
}

static void build_depth(Mesh& m, int d) {
  Depth& D = m.depth[d];
  const int nt = m.nt;
  D.tet_slot.assign(nt, -1);
  D.tet_level.assign(nt, -1);
  // slots: tets above the coarsest level first, then those at it
  for (int pass = 0; pass < 2; ++pass)
    for (int t = 0; t < nt; ++t) {
      const int l = m.level[t] - d;
      if (l < m.coarsest) continue;
      const bool nc = l > m.coarsest;
      if ((pass == 0) != nc) continue;
      D.tet_slot[t] = (int)D.slot_tet.size();
      D.tet_level[t] = l;
      D.slot_tet.push_back(t);
    }
  const int ns = (int)D.slot_tet.size();
  D.n_slots_nc = 0;
  for (int s = 0; s < ns; ++s)
    if (D.tet_level[D.slot_tet[s]] > m.coarsest) D.n_slots_nc = s + 1;
  D.h_tets.resize(ns);
  long long off = 0;
  for (int s = 0; s < ns; ++s) {
    const int t = D.slot_tet[s];
    const int N = 1 << D.tet_level[t];
    D.h_tets[s] = TetDev{off, N, t};
    off += tetnum(N + 1);
    if (s + 1 == D.n_slots_nc) D.n_stored_nc = off;
  }
  D.n_stored = off;
  if (D.n_slots_nc == 0) D.n_stored_nc = 0;
  D.tet_offset.assign(nt + 1, 0);
  {
    // offsets per tet index (inactive tets: empty range at the next start)
    std::vector<long long> start(nt, -1);
    for (int s = 0; s < ns; ++s) start[D.slot_tet[s]] = D.h_tets[s].base;
    long long cur = D.n_stored;
    for (int t = nt - 1; t >= 0; --t) {
      if (start[t] >= 0) cur = start[t];
      D.tet_offset[t] = start[t] >= 0 ? start[t] : cur;
    }
    D.tet_offset[nt] = D.n_stored;
  }
  // stencils and element matrices
  D.h_sten.assign((size_t)ns * 16 * kNDir, 0.0);
  D.h_elem.assign((size_t)ns * 6 * 16, 0.0);
  D.h_mass.assign((size_t)ns * 16 * 15, 0.0);
  for (int s = 0; s < ns; ++s) {
    const int t = D.slot_tet[s];
    stencils_for(m, t, D.tet_level[t], &D.h_sten[(size_t)s * 16 * kNDir]);
    elements_for(m, t, D.tet_level[t], &D.h_elem[(size_t)s * 96]);
    mass_stencils_for(m, t, D.tet_level[t], &D.h_mass[(size_t)s * 16 * 15]);
  }
  build_items(m, D);
  // rows (slot, j, k)
  D.h_rows.clear();
  for (int s = 0; s < ns; ++s) {
    const int N = D.h_tets[s].N;
    for (int k = 0; k <= N; ++k)
      for (int j = 0; j <= N - k; ++j) D.h_rows.push_back(make_int4(s, j, k, 0));
    if (s + 1 == D.n_slots_nc) D.n_rows_nc = (int)D.h_rows.size();
  }
  D.n_rows = (int)D.h_rows.size();
  if (D.n_slots_nc == 0) D.n_rows_nc = 0;
  // boundary (interface) nodes: all copies of nodes on macro faces/edges/vertices
  struct Rec {
    Key key;
    BCopy c;
    bool dir;
  };
  std::vector<Rec> recs;
  for (int s = 0; s < ns; ++s) {
    const int t = D.slot_tet[s];
    const int N = D.h_tets[s].N;
    const long long base = D.h_tets[s].base;
    for (int k = 0; k <= N; ++k)
      for (int j = 0; j <= N - k; ++j)
        for (int i = 0; i <= N - j - k; ++i) {
          const int mask = face_mask(N, i, j, k);
          if (!mask) continue;
          bool dir = false;
          for (int f = 0; f < 4; ++f)
            if ((mask >> f) & 1 && m.face_boundary[t][f]) dir = true;
          BCopy c;
          c.idx = base + node_offset(N, i, j, k);
          c.slot = s;
          c.i = (short)i;
          c.j = (short)j;
          c.k = (short)k;
          c.mask = (short)mask;
          recs.push_back({node_key(m, t, N, i, j, k), c, dir});
        }
  }
  std::sort(recs.begin(), recs.end(), [](const Rec& a, const Rec& b) {
    if (a.key == b.key) return a.c.idx < b.c.idx;
    return a.key < b.key;
  });
  struct Group {
    size_t lo, hi;
    long long owner;
    bool dir;
  };
  std::vector<Group> groups;
  for (size_t a = 0; a < recs.size();) {
    size_t b = a;
    bool dir = false;
    while (b < recs.size() && recs[b].key == recs[a].key) dir |= recs[b++].dir;
    groups.push_back({a, b, recs[a].c.idx, dir});
    a = b;
  }
  std::stable_sort(groups.begin(), groups.end(), [](const Group& a, const Group& b) { return a.owner < b.owner; });
  D.h_bstart.assign(1, 0);
  D.h_bcopies.clear();
  D.h_bdir.clear();
  D.h_extra.clear();
  D.n_bnodes_nc = 0;
  D.n_extra_nc = 0;
  for (const Group& g : groups) {
    for (size_t q = g.lo; q < g.hi; ++q) {
      D.h_bcopies.push_back(recs[q].c);
      if (q > g.lo && !g.dir) D.h_extra.push_back(recs[q].c.idx);
    }
    D.h_bstart.push_back((int)D.h_bcopies.size());
    D.h_bdir.push_back(g.dir ? 1 : 0);
    if (recs[g.lo].c.slot < D.n_slots_nc) {
      D.n_bnodes_nc = (int)D.h_bdir.size();
      D.n_extra_nc = (int)D.h_extra.size();
    }
  }
  D.n_bnodes = (int)D.h_bdir.size();
  D.n_extra = (int)D.h_extra.size();
  // interface nodes whose rows the "scale Vol+Face" operator takes from nodal
  // integration: two or more face bits (macro edge or vertex), not Dirichlet
  D.h_vf.clear();
  D.n_vf_nc = 0;
  for (int b = 0; b < D.n_bnodes; ++b) {
    const int mask = D.h_bcopies[D.h_bstart[b]].mask;
    if (D.h_bdir[b] || __builtin_popcount((unsigned)mask) < 2) continue;
    D.h_vf.push_back(b);
    if (b < D.n_bnodes_nc) D.n_vf_nc = (int)D.h_vf.size();
  }
  D.n_vf = (int)D.h_vf.size();
  // slot of the same tet one depth finer; copies per (slot, face mask)
  D.h_fslot.assign(ns, -1);
  if (d > 0)
    for (int s = 0; s < ns; ++s) D.h_fslot[s] = m.depth[d - 1].tet_slot[D.slot_tet[s]];
  D.h_mult.assign((size_t)ns * 16, 1);
  for (int b = 0; b < D.n_bnodes; ++b)
    for (int q = D.h_bstart[b]; q < D.h_bstart[b + 1]; ++q) {
      const BCopy& c = D.h_bcopies[q];
      D.h_mult[(size_t)c.slot * 16 + c.mask] = (unsigned char)(D.h_bstart[b + 1] - D.h_bstart[b]);
    }
}

template <class T>
static T* reupload(Depth& d, T* old, const std::vector<T>& h) {
  if (old) {
    cudaFree(old);
    d.allocations.erase(std::remove(d.allocations.begin(), d.allocations.end(), (void*)old), d.allocations.end());
  }
  return upload(d, h);
}

void set_kseg(Mesh& m, int kseg, int korder) {
  drop_graphs(m);
  HHG_REQUIRE(kseg >= 1 && kseg <= 1024, "kseg must be in [1, 1024]");
  HHG_REQUIRE(korder >= 0 && korder <= 2, "korder must be 0, 1 or 2");
  m.kseg = kseg;
  m.korder = korder;
  for (Depth& D : m.depth) {
    build_items(m, D);
    if (m.device) {
      HHG_CUDA(cudaDeviceSynchronize());
      D.dev.items = reupload(D, const_cast<int4*>(D.dev.items), D.h_items);
      D.dev.n_items = D.n_items;
      D.dev.n_items_nc = D.n_items_nc;
      D.dev.mitems = reupload(D, const_cast<int4*>(D.dev.mitems), D.h_mitems);
      D.dev.sitems = reupload(D, const_cast<int4*>(D.dev.sitems), D.h_sitems);
      D.dev.pairs = reupload(D, const_cast<int2*>(D.dev.pairs), D.h_pairs);
      D.dev.n_mitems = D.n_mitems;
      D.dev.n_mitems_nc = D.n_mitems_nc;
      D.dev.n_sitems = D.n_sitems;
      D.dev.n_sitems_nc = D.n_sitems_nc;
    }
  }
}

static void upload_depth(Depth& D) {
  D.dev.tets = upload(D, D.h_tets);
  // gray directions of each slot's volume stencil (positive off-centre
  // entries, Sec. 4.2), relative to the stencil's largest entry
  D.h_gray.assign(D.h_tets.size(), 0u);
  for (size_t sl = 0; sl < D.h_tets.size(); ++sl) {
    const double* st = &D.h_sten[sl * 16 * kNDir];  // mask 0: the volume row
    double mx = 0;
    for (int d = 0; d < kNDir; ++d) mx = std::max(mx, std::abs(st[d]));
    for (int d = 0; d < kNDir; ++d)
      if (st[d] > 1e-12 * mx) D.h_gray[sl] |= 1u << d;
  }
  D.dev.gray = upload(D, D.h_gray);
  D.dev.sten64 = upload(D, D.h_sten);
  std::vector<float> s32(D.h_sten.begin(), D.h_sten.end());
  D.dev.sten32 = upload(D, s32);
  D.dev.elem64 = upload(D, D.h_elem);
  D.dev.mass64 = upload(D, D.h_mass);
  std::vector<float> m32(D.h_mass.begin(), D.h_mass.end());
  D.dev.mass32 = upload(D, m32);
  std::vector<float> e32(D.h_elem.begin(), D.h_elem.end());
  D.dev.elem32 = upload(D, e32);
  D.dev.items = upload(D, D.h_items);
  D.dev.n_items = D.n_items;
  D.dev.n_items_nc = D.n_items_nc;
  D.dev.mitems = upload(D, D.h_mitems);
  D.dev.sitems = upload(D, D.h_sitems);
  D.dev.pairs = upload(D, D.h_pairs);
  D.dev.n_mitems = D.n_mitems;
  D.dev.n_mitems_nc = D.n_mitems_nc;
  D.dev.n_sitems = D.n_sitems;
  D.dev.n_sitems_nc = D.n_sitems_nc;
  D.dev.bstart = upload(D, D.h_bstart);
  D.dev.bcopies = upload(D, D.h_bcopies);
  D.dev.bdir = upload(D, D.h_bdir);
  D.dev.n_bnodes = D.n_bnodes;
  D.dev.n_bnodes_nc = D.n_bnodes_nc;
  D.dev.vf = upload(D, D.h_vf);
  D.dev.n_vf = D.n_vf;
  D.dev.n_vf_nc = D.n_vf_nc;
  D.dev.rows = upload(D, D.h_rows);
  D.dev.n_rows = D.n_rows;
  D.dev.n_rows_nc = D.n_rows_nc;
  D.dev.extra = upload(D, D.h_extra);
  D.dev.n_extra = D.n_extra;
  D.dev.n_extra_nc = D.n_extra_nc;
  D.dev.n_stored = D.n_stored;
  D.dev.n_stored_nc = D.n_stored_nc;
  D.dev.fslot = upload(D, D.h_fslot);
  D.dev.mult = upload(D, D.h_mult);
}

// Unknowns of every component at the depth where it reaches the coarsest level.
static void build_coarse(Mesh& m) {
  m.coarse.assign(m.ncomp, CoarseComp{});
  for (int c = 0; c < m.ncomp; ++c) {
    CoarseComp& C = m.coarse[c];
    C.depth = m.comp_level[c] - m.coarsest;
    const Depth& D = m.depth[C.depth];
    C.h_cstart.assign(1, 0);
    // volume nodes of the component's tets
    for (size_t s = 0; s < D.slot_tet.size(); ++s) {
      const int t = D.slot_tet[s];
      if (m.comp[t] != c) continue;
      const int N = D.h_tets[s].N;
      for (int k = 1; k <= N; ++k)
        for (int j = 1; j <= N - k; ++j)
          for (int i = 1; i + j + k <= N - 1; ++i) {
            const long long idx = D.h_tets[s].base + node_offset(N, i, j, k);
            C.h_rep.push_back((int)idx);
            C.h_copies.push_back(idx);
            C.h_cstart.push_back((int)C.h_copies.size());
          }
    }
    // interface nodes (not Dirichlet)
    for (int b = 0; b < D.n_bnodes; ++b) {
      const BCopy& c0 = D.h_bcopies[D.h_bstart[b]];
      if (m.comp[D.slot_tet[c0.slot]] != c || D.h_bdir[b]) continue;
      C.h_rep.push_back((int)c0.idx);
      for (int q = D.h_bstart[b]; q < D.h_bstart[b + 1]; ++q) C.h_copies.push_back(D.h_bcopies[q].idx);
      C.h_cstart.push_back((int)C.h_copies.size());
    }
    C.n = (int)C.h_rep.size();
  }
}

Mesh* build_mesh(const double* verts, int nv, const int* tets, int nt, const int* levels, int coarsest,
                 bool device) {
  HHG_REQUIRE(verts && tets && levels, "null mesh array");
  HHG_REQUIRE(nv >= 4 && nt >= 1, "need at least 4 vertices and 1 tet");
  HHG_REQUIRE(nv < (1 << 20), "too many vertices (max 2^20 - 1)");
  HHG_REQUIRE(coarsest >= 1 && coarsest <= kMaxLevel, "coarsest_level must be in [1, 10]");
  auto m = new Mesh();
  try {
    m->nv = nv;
    m->nt = nt;
    m->coarsest = coarsest;
    m->V.assign(verts, verts + 3 * nv);
    m->T.assign(tets, tets + 4 * nt);
    m->level.assign(levels, levels + nt);
    for (int t = 0; t < nt; ++t) {
      HHG_REQUIRE(levels[t] >= coarsest && levels[t] <= kMaxLevel,
                  "tet " + std::to_string(t) + ": level must be in [coarsest_level, 10]");
      for (int a = 0; a < 4; ++a) {
        HHG_REQUIRE(tets[4 * t + a] >= 0 && tets[4 * t + a] < nv, "tet " + std::to_string(t) + ": vertex id out of range");
        for (int b = 0; b < a; ++b)
          HHG_REQUIRE(tets[4 * t + a] != tets[4 * t + b], "tet " + std::to_string(t) + ": repeated vertex");
      }
      double X[4][3], A[4][4];
      for (int a = 0; a < 4; ++a)
        for (int r = 0; r < 3; ++r) X[a][r] = verts[3 * tets[4 * t + a] + r];
      p1_stiffness(X, A);  // throws on a degenerate tet
    }
    // components through shared vertices
    std::vector<int> par(nv);
    std::iota(par.begin(), par.end(), 0);
    for (int t = 0; t < nt; ++t)
      for (int a = 1; a < 4; ++a) par[find(par, tets[4 * t + a])] = find(par, tets[4 * t]);
    std::map<int, int> cid;
    m->comp.resize(nt);
    for (int t = 0; t < nt; ++t) {
      const int r = find(par, tets[4 * t]);
      if (!cid.count(r)) cid[r] = (int)cid.size();
      m->comp[t] = cid[r];
    }
    m->ncomp = (int)cid.size();
    m->comp_level.assign(m->ncomp, -1);
    for (int t = 0; t < nt; ++t) {
      int& l = m->comp_level[m->comp[t]];
      HHG_REQUIRE(l < 0 || l == levels[t], "tets sharing a vertex must have the same level");
      l = levels[t];
    }
    // boundary faces
    std::map<std::array<int, 3>, int> fcount;
    auto face_of = [&](int t, int f) {
      std::array<int, 3> q;
      int n = 0;
      for (int a = 0; a < 4; ++a)
        if (a != f) q[n++] = tets[4 * t + a];
      std::sort(q.begin(), q.end());
      return q;
    };
    for (int t = 0; t < nt; ++t)
      for (int f = 0; f < 4; ++f) fcount[face_of(t, f)]++;
    m->face_boundary.assign(nt, std::vector<int>(4, 0));
    for (int t = 0; t < nt; ++t)
      for (int f = 0; f < 4; ++f) {
        const int c = fcount[face_of(t, f)];
        HHG_REQUIRE(c <= 2, "a face is shared by more than two tets");
        m->face_boundary[t][f] = c == 1;
      }
    int maxd = 0;
    for (int t = 0; t < nt; ++t) maxd = std::max(maxd, levels[t] - coarsest);
    m->ndepth = maxd + 1;
    m->depth.resize(m->ndepth);
    if (device) {  // the SM count sizes the work lists
      int dev = 0;
      HHG_CUDA(cudaGetDevice(&dev));
      HHG_CUDA(cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    for (int d = 0; d < m->ndepth; ++d) build_depth(*m, d);
    build_coarse(*m);
    m->device = device;
    if (!device) return m;
    for (int d = 0; d < m->ndepth; ++d) upload_depth(m->depth[d]);
    HHG_CUDA(cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking));
    HHG_CUDA(cudaEventCreateWithFlags(&m->side_fork, cudaEventDisableTiming));
    HHG_CUDA(cudaEventCreateWithFlags(&m->side_join, cudaEventDisableTiming));
    Depth& D0 = m->depth[0];
    m->d_red = static_cast<double*>(dalloc(D0, 4096 * sizeof(double)));
    m->d_counter = static_cast<unsigned*>(dalloc(D0, 64 * sizeof(unsigned)));
    HHG_CUDA(cudaMemset(m->d_counter, 0, 64 * sizeof(unsigned)));
    m->d_error = m->d_counter + 32;
    m->d_scalars = static_cast<double*>(dalloc(D0, 64 * sizeof(double)));
    HHG_CUDA(cudaMemset(m->d_scalars, 0, 64 * sizeof(double)));
    HHG_CUDA(cudaMallocHost(&m->h_pinned, 64 * sizeof(double)));
  } catch (...) {
    free_mesh(m);
    throw;
  }
  return m;
}

void free_learned(Mesh* m);

void free_mesh(Mesh* m) {
  if (!m) return;
  drop_graphs(*m);
  free_learned(m);
  if (m->side) {
    cudaStreamSynchronize(m->side);
    cudaStreamDestroy(m->side);
  }
  if (m->side_fork) cudaEventDestroy(m->side_fork);
  if (m->side_join) cudaEventDestroy(m->side_join);
  for (Depth& d : m->depth) {
    for (void* p : d.allocations) cudaFree(p);
    d.allocations.clear();
  }
  if (m->h_pinned) cudaFreeHost(m->h_pinned);
  delete m;
}

}  // namespace hhg
