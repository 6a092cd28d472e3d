// Internal structures of the hhg library (host + device).  Not part of the ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hhg.h"

namespace hhg {

constexpr int kNDir = 14;     // stencil directions (without the centre)
constexpr int kMaxLevel = 10; // N <= 1024: i, j, k fit in 11 bits
constexpr int kTJ = 4;        // rows per thread in the volume kernels
#ifndef HHG_TILE_I
#define HHG_TILE_I 16
#endif
constexpr int kWarpTileI = HHG_TILE_I;       // columns of a volume warp tile (16 or 32)
constexpr int kWarpTileJ = 32 / HHG_TILE_I * kTJ;  // rows of a volume warp tile

// Direction d = (di, dj, dk) in the index space of a macro tet.
// 0..6: e1, e2, e3, e1-e2, e1-e3, e2-e3, e1-e2+e3 (the 7 edge directions of
// the refined mesh, Sec. 2.2 / Fig. "stencildir"); 7..13: their negatives.
__host__ __device__ inline void dir_of(int d, int& di, int& dj, int& dk) {
  const int s = d < 7 ? 1 : -1;
  const int b = d < 7 ? d : d - 7;
  di = (b == 0 || b == 3 || b == 4 || b == 6) ? s : 0;
  dj = (b == 1 || b == 5) ? s : ((b == 3 || b == 6) ? -s : 0);
  dk = (b == 2 || b == 6) ? s : ((b == 4 || b == 5) ? -s : 0);
}

// Number of nodes of a tetrahedral index space with n nodes per edge.
__host__ __device__ inline long long tetnum(long long n) { return n * (n + 1) * (n + 2) / 6; }

// Offset of node (i,j,k) in the packed array of a tet with N = 2^level.
__host__ __device__ inline long long node_offset(int N, int i, int j, int k) {
  const long long M = N - k;
  return tetnum(N + 1) - tetnum(N + 1 - k) + (long long)j * (M + 1) - (long long)j * (j - 1) / 2 + i;
}

// Face-bit mask of a node: bit f set iff the node lies on the face opposite
// vertex f (f=0: i+j+k=N, 1: i=0, 2: j=0, 3: k=0).  0 = volume primitive.
__host__ __device__ inline int face_mask(int N, int i, int j, int k) {
  return (i + j + k == N ? 1 : 0) | (i == 0 ? 2 : 0) | (j == 0 ? 4 : 0) | (k == 0 ? 8 : 0);
}

// Per active tet at one depth (device table, indexed by slot).
struct TetDev {
  long long base;  // offset of the tet's packed array in the depth vector
  int N;           // 2^level at this depth
  int tet;         // macro tet index
};

// One stored copy of a node on a macro face/edge/vertex.
struct BCopy {
  long long idx;   // index in the depth vector
  int slot;        // active-tet slot
  short i, j, k;   // index-space position in that tet
  short mask;      // face-bit mask (primitive) in that tet
};

// Everything the kernels of one depth need (device pointers + counts).
struct DepthDev {
  const TetDev* tets;
  const double* sten64;  // [slot][16][14]  (1/2) reference stencil per primitive
  const float* sten32;
  const double* elem64;  // [slot][6][16]   (1/4)*micro-element stiffness per Kuhn type
  const float* elem32;
  const double* mass64;  // [slot][16][15]  consistent mass stencil per primitive (col 14 = centre)
  const float* mass32;
  const int4* items;     // volume work: (tile = slot<<20 | j0<<10 | i0, k0, k1, -) per warp item
  int n_items;           // items of all active tets
  int n_items_nc;        // items of tets above the coarsest level (prefix)
  const int4* mitems;    // column-march work, 60-column tiles: (slot index, i0 | j0<<16, k0, k1) per block item
  const int2* pairs;     // (slot, -1) per active slot
  int n_mitems;          // items of the two-column-set (FP32x2) march
  int n_mitems_nc;       // of those, items of tets above the coarsest level (prefix)
  const int4* sitems;    // the same over 30-column tiles (one column set per lane)
  int n_sitems;
  int n_sitems_nc;
  const int* bstart;     // boundary unique nodes: copies bstart[b]..bstart[b+1]
  const BCopy* bcopies;
  const unsigned char* bdir;  // 1 = Dirichlet
  int n_bnodes;
  int n_bnodes_nc;
  const int4* rows;      // (slot, j, k, -) per stored row of active tets
  int n_rows;
  int n_rows_nc;
  const long long* extra;  // non-owner interface copies (excluded from dots)
  int n_extra;
  int n_extra_nc;
  long long n_stored;
  long long n_stored_nc;
  const int* vf;               // interface nodes on macro vertices/edges (not Dirichlet): indices into bstart
  int n_vf;
  int n_vf_nc;
  const unsigned* gray;         // [slot] bit d set: direction d of the volume stencil is of gray type (> 0)
  const int* fslot;            // slot of the same tet at depth-1 (-1 at depth 0)
  const unsigned char* mult;   // [slot][16] copies of a node of that face mask
};

// Host-side description of one depth.
struct Depth {
  std::vector<int> slot_tet;          // slot -> macro tet
  std::vector<int> tet_slot;          // macro tet -> slot or -1
  std::vector<long long> tet_offset;  // nt+1 (inactive: empty range)
  std::vector<int> tet_level;         // level at this depth or -1
  int n_slots_nc = 0;                 // slots [0, n_slots_nc) are above the coarsest level
  long long n_stored = 0, n_stored_nc = 0;
  std::vector<TetDev> h_tets;
  std::vector<double> h_sten;         // [slot][16][14]
  std::vector<double> h_elem;         // [slot][6][16]
  std::vector<double> h_mass;         // [slot][16][15]
  std::vector<int4> h_items;
  int n_items = 0, n_items_nc = 0;
  std::vector<int4> h_mitems, h_sitems;
  std::vector<int2> h_pairs;
  int n_mitems = 0, n_mitems_nc = 0, n_sitems = 0, n_sitems_nc = 0;
  std::vector<int> h_bstart;
  std::vector<BCopy> h_bcopies;
  std::vector<unsigned char> h_bdir;
  int n_bnodes = 0, n_bnodes_nc = 0;
  std::vector<int4> h_rows;
  int n_rows = 0, n_rows_nc = 0;
  std::vector<long long> h_extra;
  int n_extra = 0, n_extra_nc = 0;
  std::vector<int> h_vf;
  int n_vf = 0, n_vf_nc = 0;
  std::vector<int> h_fslot;
  std::vector<unsigned char> h_mult;
  DepthDev dev{};
  // device allocations owned by this depth
  std::vector<void*> allocations;
  // coefficient copies at this depth
  double* k16d = nullptr;  // bfloat16-rounded k held in double (outer residual of the bf16 solve)
  // tensor coefficient (six terms, node major: n_stored x 6) and the
  // six terms' reference stencils [slot][6][16][14] (set on first use)
  double* km64 = nullptr;
  float* km32 = nullptr;
  const double* tsten64 = nullptr;
  const float* tsten32 = nullptr;
  // edge weights of the tensor operator's volume rows (W_e(x) = sum_m
  // c^m_e (k_m(x) + k_m(x+w_e)) for the 7 positive directions e of the volume
  // stencil; direction major, stride n_stored rounded up to 16), and of its
  // interface rows (per boundary copy and each of the 14 directions, with
  // the stencils of the copy's primitive; direction major, stride the copy
  // count), set with the tensor coefficient
  double* tb64 = nullptr;
  float* tb32 = nullptr;
  double* twb64 = nullptr;
  float* twb32 = nullptr;
  double* k64 = nullptr;
  float* k32 = nullptr;
  __nv_bfloat16* k16 = nullptr;
  // k_min of eq. "defKmin" per stored copy (the minimum over the copy's
  // neighbourhood inside its own tet), per precision; set while the mesh's
  // kappa option is on
  double* kmin64 = nullptr;
  double* kmin16d = nullptr;
  float* kmin32 = nullptr;
  __nv_bfloat16* kmin16 = nullptr;
  std::vector<unsigned> h_gray;
  // multigrid workspace per precision (allocated lazily): 0 = f64, 1 = f32
  // slots: 0 F (depth>0) / CG r (depth 0), 1 U / CG z, 2 V-cycle residual,
  // 3 CG p, 4 smoother ping-pong, 5-6 Chebyshev updates, 7 CG q, 8 inner solution
  // 9 inner solution, 10 operator scratch (nodal modes), 11 spare
  void* ws[2][14] = {{nullptr}};
  void* ndinv[4] = {nullptr, nullptr, nullptr, nullptr};  // nodal operator 1/diag per dtype (0 on Dirichlet)
  int* cslot_map = nullptr;  // slot at depth+1 of each slot (prolongation)
  double lam = 0.0;  // lambda_max of D^-1 A (FP64, 0 = not yet estimated)
};

// Coarse problem of one connected component at its coarsest depth.
struct CoarseComp {
  int depth;                    // depth at which the component is at the coarsest level
  int n;                        // unknowns
  std::vector<int> h_rep;       // n: owner-copy index (int) of each unknown in the depth vector
  std::vector<int> h_cstart;    // n+1: copies of each unknown
  std::vector<long long> h_copies;
};

struct Mesh {
  int nv = 0, nt = 0, coarsest = 0;
  std::vector<double> V;
  std::vector<int> T;
  std::vector<int> level;        // finest level per tet
  std::vector<int> comp;         // component per tet
  int ncomp = 0;
  std::vector<int> comp_level;   // finest level per component
  std::vector<std::vector<int>> face_boundary;  // [tet][face] 1 if on the domain boundary
  int ndepth = 0;
  std::vector<Depth> depth;
  std::vector<CoarseComp> coarse;
  // coarse solve device data (all components packed)
  long long* d_cinv_off = nullptr;
  int* d_cn = nullptr;
  int* d_cdepth = nullptr;
  int* d_crep = nullptr;          // owner copy index per unknown (packed)
  int* d_crep_off = nullptr;
  int* d_ccstart = nullptr;       // copy ranges (packed, per component offset by d_crep_off)
  long long* d_ccopies = nullptr;
  int* d_ccopies_off = nullptr;
  bool device = true;            // false: host-only inspection mesh
  bool coef_set = false;
  // operator of the multigrid internals (V-cycle, smoothers, residuals, coarse
  // solve): 0 scaled, 1 "scale Vol+Face", 2 nodal integration; set by the
  // multigrid solve for its duration, 0 otherwise
  int opk = 0;                        // 3: scaled tensor coefficient (M = 6)
  bool tensor_set = false;
  bool cinv_ready[4][4] = {};         // per operator and dtype
  double* d_cinv[4][4] = {};          // dense coarse inverses (packed)
  std::vector<long long> cinv_off;  // per component offset into d_cinv
  // scratch
  double* d_red = nullptr;        // reduction partials
  unsigned* d_counter = nullptr;
  unsigned* d_error = nullptr;    // set by a kernel whose bounded wait ran out
  double* d_scalars = nullptr;    // device scalars for CG
  double* h_pinned = nullptr;     // pinned host scalars
  double* d_geom = nullptr;       // macro vertices (double) followed by tets (int)
  int num_sms = 0;
  // side stream of the operator launches (interface rows concurrent with the
  // volume kernel) and its fork/join events
  cudaStream_t side = nullptr;
  cudaEvent_t side_fork = nullptr, side_join = nullptr;
  int cheb_degree = 2;
  double cheb_lo = 0.3, cheb_hi = 1.1;
  int power_its = 15;
  int kseg = 32;                  // planes per volume work item (k-march segment)
  int vkernel = 1;                // volume kernel: 1 column march (march.cu), 2 the same with two column
                                  // sets per lane in FP32, 0 tile march (apply.cu)
  bool kappa = false;             // scaled operator with k_min on gray directions (eq. "defKmin", kappa.cu)
  int korder = 0;                 // work order: 0 longest first, 1 by plane window, 2 j-stacked quads by window
  // learned smoother state (opaque)
  void* learned = nullptr;
  // instantiated CG-iteration graphs, keyed by their arguments; dropped when
  // work lists, coefficients or options change (kernel parameters embed them)
  struct GraphEntry {
    int dtype, smoother, nu1, nu2;
    double omega;
    const void *x, *r;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
};

void drop_graphs(Mesh& m);
// learned smoother (learned.cu)
void learned_invalidate(Mesh& m);  // coefficient changed: recompute the input features
void learned_step(Mesh& m, int d, int dtype, const void* f, const void* src, void* dst, bool nc_only, cudaStream_t s);

// ---- error handling --------------------------------------------------------
void set_error(const std::string& msg);
struct Error {
  int code;
  std::string msg;
};

#define HHG_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      throw ::hhg::Error{HHG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define HHG_REQUIRE(cond, msg)                                 \
  do {                                                         \
    if (!(cond)) throw ::hhg::Error{HHG_ERR_ARG, std::string(msg)}; \
  } while (0)

// ---- host setup (mesh.cu) ---------------------------------------------------
Mesh* build_mesh(const double* verts, int nv, const int* tets, int nt, const int* levels, int coarsest,
                 bool device);
void free_mesh(Mesh* m);
void node_coords(const Mesh& m, int depth, std::vector<double>& xyz);
void stencils_for(const Mesh& m, int tet, int level, double* out16x14);
void elements_for(const Mesh& m, int tet, int level, double* out6x16);
void* dalloc(Depth& d, size_t bytes);
void build_items(const Mesh& m, Depth& D);
void build_march_items(const Mesh& m, Depth& D);
void set_kseg(Mesh& m, int kseg, int korder);

// ---- kernels (apply.cu / mg.cu) ----------------------------------------------
enum OpMode { OP_APPLY = 0, OP_RESID = 1, OP_JACOBI = 2, OP_CHEB = 3, OP_DIAG = 4 };
// internal dtype: FP64 arithmetic with the bfloat16-rounded coefficient
constexpr int kF64KBF16 = 3;

struct OpArgs {
  const void* u;   // input vector (neighbours read)
  const void* f;   // right-hand side (RESID/JACOBI/CHEB)
  void* out;       // y, r, or u_new
  const void* d_in;  // CHEB: previous update
  void* d_out;       // CHEB: new update
  double omega;      // JACOBI damping
  double ca, cb;     // CHEB: d_new = ca d_old + cb D^-1 (f - A u)
  int nc_only;       // 1: tets above the coarsest level only
};

void launch_scaled_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, cudaStream_t s);
// volume rows of the scaled operator by the column march (march.cu)
void launch_march(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, cudaStream_t s);
void init_march_configs(int dtype);
// bytes past the end of every coefficient array (bulk copies of whole 16-byte
// chunks may reach into it)
constexpr int kCoefPad = 64;
void launch_nodal_apply(const Mesh& m, int depth, int dtype, const void* u, void* y, cudaStream_t s);
// scaled launch followed by the nodal-integration rows of macro vertices and edges (eq. "modst")
void launch_volface_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, cudaStream_t s);
// nodal-integration operator in the modes above (dinv: 1/diag, 0 on Dirichlet nodes; tmp: a scratch vector)
void launch_nodal_dinv(const Mesh& m, int depth, int dtype, void* dinv, cudaStream_t s);
// scaled operator of the tensor coefficient (M = 6) in the modes above
void compute_tensor_weights(Mesh& m, cudaStream_t s);
void init_tensor_configs();  // shared-memory limits of the tensor march kernels
void launch_tensor_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a,
                      cudaStream_t s);
void ensure_tensor_stencils(Mesh& m);
void launch_nodal_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, const void* dinv, void* tmp,
                     cudaStream_t s);
void launch_mass_apply(const Mesh& m, int depth, int dtype, const void* u, void* y, cudaStream_t s);
// scaled operator with the pre-asymptotic modification (kappa.cu)
void compute_kmin(Mesh& m, cudaStream_t s);
void launch_kappa_op(const Mesh& m, int depth, int dtype, OpMode mode, const OpArgs& a, cudaStream_t s);

}  // namespace hhg
