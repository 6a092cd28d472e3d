/*
 * hhg.h -- C ABI of the GB300 (sm_103a) library for the stencil-scaled P1
 * operator -div(k grad u) on hierarchical hybrid grids.
 *
 * Method: a macro mesh of tetrahedra is refined uniformly (Bey's rule, paper
 * Sec. 2.1); inside each macro tetrahedron T the nodes form the structured
 * index space (i,j,k), i+j+k <= N = 2^level.  The operator row of a node x is
 * its macro primitive's constant-coefficient reference stencil with every
 * off-diagonal entry scaled by (k(x)+k(x+w))/2 and the diagonal set by the
 * zero row sum (paper Sec. 6.1, "Cost for stencil scaling"; the bilinear form
 * is eq. "discrete" of Sec. 2.1).  The nodal-integration operator of eq.
 * "standardfe" / eq. "onTheFlyStencil" (Sec. 6.2) is the cost comparison.
 *
 * Conventions shared by every entry point
 *  - Pointers named *_dev are CUDA device pointers that the CALLER owns; all
 *    other pointers are host pointers the caller owns.  The library owns only
 *    the mesh object and the workspace it allocates (at create, at
 *    hhg_set_coefficient, or at the first call that needs it).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  All calls are
 *    stream-ordered and asynchronous unless stated otherwise.
 *  - Vectors use the STORED layout at a given depth: the macro tetrahedra
 *    active at that depth (first those above the coarsest level at that
 *    depth, then those at it, each group in increasing tet index), each as a
 *    packed array of its nodes ordered by k (slowest), then j, then i
 *    (fastest); node (i,j,k)
 *    of a tet with N = 2^level sits at
 *        planeoff(k) + j*(N-k+1) - j*(j-1)/2 + i,
 *        planeoff(k) = tet(N+1) - tet(N+1-k),  tet(n) = n(n+1)(n+2)/6.
 *    Nodes on macro faces, edges and vertices are stored once per macro
 *    tetrahedron that contains them (paper Sec. 2.1); every copy of a node
 *    holds the same value in every input and output.  hhg_layout gives the
 *    tet offsets.
 *  - Depth d means refinement level level_t - d of every tet t (0 = finest).
 *    All tets connected through a shared vertex must have the same finest
 *    level; independent components may differ (a batch of problems).
 *  - Device vectors must be 16-byte aligned (they are staged with bulk copies);
 *    allocations from cudaMalloc or PyTorch are.
 *  - Dirichlet: nodes on faces that belong to exactly one macro tetrahedron
 *    form the domain boundary with u = 0.  Inputs must hold 0 there (outputs
 *    of this library always do); outputs are 0 there.
 *  - Every entry point returns an hhg_status; on error, hhg_last_error()
 *    gives a message (per calling thread).  No C++ exception crosses the ABI.
 */
#ifndef HHG_H
#define HHG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hhg_mesh_s* hhg_mesh;

/* Arithmetic of a call: vector element type and coefficient (k) type. */
typedef enum {
    HHG_F64 = 0,       /* double vectors, double k */
    HHG_F32 = 1,       /* float vectors, float k (k rounded once from the double input) */
    HHG_F32_KBF16 = 2  /* float vectors, bfloat16 k (k rounded once, RN) */
} hhg_dtype;

typedef enum {
    HHG_OK = 0,
    HHG_ERR_ARG = -1,           /* invalid argument (message says which) */
    HHG_ERR_CUDA = -2,          /* a CUDA runtime call failed */
    HHG_ERR_NOMEM = -3,         /* device or host allocation failed */
    HHG_ERR_NOT_CONVERGED = -4, /* solver hit its iteration limit */
    HHG_ERR_TIMEOUT = -5,       /* reserved for a bounded device wait running out (no kernel waits today) */
    HHG_ERR_STATE = -6          /* call order violated (e.g. no coefficient set) */
} hhg_status;

typedef enum {
    HHG_SMOOTH_JACOBI = 0,     /* damped Jacobi, u += omega D^-1 (f - A u) */
    HHG_SMOOTH_CHEBYSHEV = 1,  /* Chebyshev on D^-1 A, interval [lo, hi] * lambda_max */
    HHG_SMOOTH_LEARNED = 2     /* damped Jacobi sweeps alternating with learned steps (see hhg_learned_train) */
} hhg_smoother;

typedef enum {
    HHG_SOLVE_FP64 = 0,        /* plain FP64 GMG-preconditioned CG */
    HHG_SOLVE_MIXED = 1,       /* FP64 iterative refinement around FP32 GMG-CG */
    HHG_SOLVE_MIXED_KBF16 = 2, /* as MIXED with k rounded to bfloat16 everywhere: the FP32 inner solve and
                                  the FP64 outer residual, so u is the discrete solution of the rounded k */
    HHG_SOLVE_MG = 3,          /* FP64 multigrid as the solver: u <- V(nu1,nu2)(f, u) (Sec. 7.2) */
    HHG_SOLVE_MIXED_KBF16_INNER = 4 /* bfloat16 k in the FP32 inner solve only, the FP64 k in the outer
                                  residual: u is the discrete solution of the FP64 k */
} hhg_solve_mode;

typedef enum {
    HHG_OP_SCALED = 0,         /* stencil scaling on every row (eq. "discrete") */
    HHG_OP_VOLFACE = 1,        /* "scale Vol+Face": nodal rows on macro vertices/edges (eq. "modst") */
    HHG_OP_NODAL = 2,          /* nodal integration on every row (eq. "standardfe") */
    HHG_OP_TENSOR = 3          /* stencil scaling of the tensor coefficient (M = 6, hhg_set_tensor_coefficient) */
} hhg_operator;

typedef struct {
    double tol;          /* stop when ||f - A u||_2 / ||f||_2 <= tol (unique unknowns) */
    int maxit;           /* max CG iterations (FP64 mode) or total inner iterations */
    int mode;            /* hhg_solve_mode */
    int smoother;        /* hhg_smoother */
    int nu1, nu2;        /* pre/post smoothing steps of the V-cycle */
    double omega;        /* Jacobi damping (default 2/3 if <= 0) */
    double inner_rtol;   /* MIXED: relative residual reduction of each inner solve (default 3e-5; never
                            below half the outer tolerance) */
    int max_outer;       /* MIXED: max refinement steps (default 20) */
    int use_graph;       /* capture each CG iteration in a CUDA graph (1) or launch eagerly (0) */
    int op;              /* hhg_operator; HHG_OP_VOLFACE, HHG_OP_NODAL, HHG_OP_TENSOR need mode HHG_SOLVE_MG
                            and Jacobi smoothing (coarsest level: dense LU of that operator) */
} hhg_solve_params;

typedef struct {
    int iterations;      /* CG iterations (sum over refinement steps in MIXED) */
    int outer;           /* refinement steps (1 in FP64 mode) */
    double rel_residual; /* final ||f - A u|| / ||f|| in FP64 */
    double time_ms;      /* wall time of the call */
    int smoother_used;   /* smoother of the last inner solve (HHG_SMOOTH_JACOBI if a
                            requested learned smoother was not accepted or diverged) */
    double rho;          /* HHG_SOLVE_MG: convergence rate (r^(i*) / r^(5))^(1/(i*-5)) of the
                            residual 2-norms, i* = cycles taken (Sec. 7); 0 otherwise */
} hhg_solve_stats;

/* Training of the learned smoother (hhg_learned_train); fields <= 0 take the
 * default in brackets. */
typedef struct {
    int steps;               /* Adam steps [150] */
    int pairs;               /* residual/error pairs per step, gradients summed [4] */
    double lr;               /* Adam learning rate [3e-3] */
    double omega;            /* damping of the Jacobi sweep before each learned step [2/3] */
    int max_depth;           /* pairs come from the smoothed depths 0..max_depth [0] */
    int vcycle_pairs;        /* pairs per step whose error is the one a plain V-cycle leaves [0] */
    double init_noise;       /* size of the random part of the initial weights [0] */
    unsigned long long seed; /* initial weights and random errors */
    int weights_bf16;        /* 1: kernels read BF16 weights; 0: FP32 weights */
    int validate_its;        /* PCG iterations of the convergence check [8] */
    int resume;              /* 1: continue from the current weights and Adam state */
} hhg_learn_params;

typedef struct {
    double loss_jacobi;  /* validation loss of the network equal to damped Jacobi */
    double loss_init;    /* validation loss of the initial weights */
    double loss_final;   /* validation loss after training */
    double rho_plain;    /* FP32 PCG residual reduction per iteration, plain Jacobi V(2,2) */
    double rho_learned;  /* the same with the learned smoother */
    int accepted;        /* 1 if rho_learned < rho_plain: solves may use the network */
    int steps;           /* Adam steps taken */
    double time_ms;      /* wall time of the training */
} hhg_learn_stats;

/* Create a macro mesh.  verts: nv*3 doubles; tets: nt*4 vertex ids, the order
 * of a tet's vertices is its refinement order (Bey's rule, Sec. 2.1);
 * levels: finest refinement level per tet (coarsest_level <= level <= 10);
 * coarsest_level: level of the dense coarse solve (>= 1).  Builds the index
 * spaces, the 15 reference stencils per tet and level (paper Sec. 2.2, one
 * per primitive: 4 vertices, 6 edges, 4 faces, 1 volume), the interface maps
 * and the volume work lists, and allocates their device copies.  Errors:
 * HHG_ERR_ARG (bad ids, degenerate tet, level mismatch across a shared
 * vertex), HHG_ERR_NOMEM, HHG_ERR_CUDA.  Synchronous. */
int hhg_create_macromesh(const double* verts, int nv, const int* tets, int nt,
                         const int* levels, int coarsest_level, hhg_mesh* out);

/* As hhg_create_macromesh but builds the host-side structures only (no GPU
 * needed): hhg_num_depths, hhg_layout, hhg_node_coords and hhg_get_stencils
 * work on it; every operator call returns HHG_ERR_STATE.  For inspection and
 * for tests on machines without a GPU. */
int hhg_create_macromesh_host(const double* verts, int nv, const int* tets, int nt,
                              const int* levels, int coarsest_level, hhg_mesh* out);

/* Free the mesh and every device buffer it owns.  Synchronous; NULL is a no-op. */
int hhg_destroy_macromesh(hhg_mesh mesh);

/* Number of depths (0 .. n-1) of the multigrid hierarchy. */
int hhg_num_depths(hhg_mesh mesh, int* n);

/* Stored layout at a depth.  tet_offsets: nt+1 int64 (host), offset of tet t's
 * array (inactive tets get an empty range); tet_levels: nt ints (host), the
 * level of tet t at this depth or -1 if inactive (either may be NULL);
 * n_stored: total length. */
int hhg_layout(hhg_mesh mesh, int depth, int64_t* tet_offsets, int* tet_levels, int64_t* n_stored);

/* Node coordinates (host, n_stored*3 doubles) at a depth, computed from the
 * macro vertices in increasing vertex-id order so that all copies of a node
 * get bitwise identical coordinates. */
int hhg_node_coords(hhg_mesh mesh, int depth, double* xyz);

/* Reference stencils of tet t at a depth (host out: 16*14 doubles): row m is
 * the primitive whose nodes lie exactly on the tet faces of bit mask m (bit f
 * = face opposite vertex f; m = 0 is the volume), column d the direction
 * (index space) 0..6 = e1, e2, e3, e1-e2, e1-e3, e2-e3, e1-e2+e3 and 7..13 the
 * negatives; the value is (1/2) int_T grad phi_x . grad phi_(x+w_d), the
 * factor 1/2 of Sec. 6.1 folded in.  Rows of absent primitives are 0. */
int hhg_get_stencils(hhg_mesh mesh, int tet, int depth, double* out);

/* Set the coefficient: k_dev is a device array of doubles in the depth-0
 * layout, positive and equal on all copies of a node.  The library keeps
 * its own FP64, FP32 and BF16 copies and injects them to every depth
 * (coarse nodal value = fine nodal value at the same point).  Must precede
 * any operator call.  Allocates on first call.  Every entry is checked on the
 * device first: HHG_ERR_ARG (and nothing changed) if one is NaN, infinite,
 * zero or negative; the check synchronises `stream`. */
int hhg_set_coefficient(hhg_mesh mesh, const double* k_dev, void* stream);

/* y = A_s(k) u: the scaled operator (Sec. 6.1) at `depth` on all active tets.
 * u_dev, y_dev: device arrays of the depth's stored length, element type of
 * `dtype`; they must not overlap.  Rows of Dirichlet nodes are 0 and all
 * copies of an interface node get the same value.  The interface rows run on
 * a library stream forked from `stream` with an event and joined to it before
 * the call returns (so the call may be captured in a CUDA graph); one mesh
 * must not be used from two streams at once. */
int hhg_apply_scaled(hhg_mesh mesh, int depth, const void* u_dev, void* y_dev, int dtype, void* stream);

/* y = A_n(k) u: the nodal-integration operator of eq. "standardfe", computed
 * on the fly from the precomputed micro-element stiffness matrices (Sec. 6.2,
 * eq. "onTheFlyStencil").  Same arguments as hhg_apply_scaled. */
int hhg_apply_nodal(hhg_mesh mesh, int depth, const void* u_dev, void* y_dev, int dtype, void* stream);

/* y = M u with M the consistent P1 mass matrix (|t|/20 (1 + delta_ab) per
 * micro tetrahedron), for the right-hand side f_h = M I_h f of Sec. 7.2:
 * every entry of u is used (Dirichlet nodes included, u holds the nodal
 * interpolant of f); rows of Dirichlet nodes are set to 0.  dtype HHG_F64 or
 * HHG_F32. */
int hhg_apply_mass(hhg_mesh mesh, int depth, const void* u_dev, void* y_dev, int dtype, void* stream);

/* Autotune the volume work for `dtype` (not part of the method): time the
 * scaled apply on depth 0 for every candidate volume kernel (the "vkernel"
 * option: 1 column march, 2 column march with two column sets per lane --
 * FP32 dtypes only --, 0 tile march), k-segment length (16, 32, 64) and
 * work order (0, 1), keep the fastest on the mesh, and report its kseg and
 * korder (the kernel: hhg_get_option "vkernel").
 * cache_path (may be NULL): a text file of earlier results keyed by the mesh
 * shape and dtype; a hit skips the search, a miss appends the new result.
 * Synchronous.  kseg, korder, best_ms may be NULL (best_ms < 0 on a hit). */
int hhg_autotune(hhg_mesh mesh, int dtype, const char* cache_path, int* kseg, int* korder, double* best_ms,
                 void* stream);

/* y = A_I(k) u, the "scale Vol+Face" operator of Sec. 5 (eq. "modst" with
 * I = W_V u W_E): rows of nodes on macro vertices and edges are the
 * nodal-integration rows of eq. "standardfe", all other rows the scaled rows
 * of hhg_apply_scaled.  Reproduces affine solutions for affine k (Lemma
 * "repro"); not symmetric (the asymmetry is O(h^2)).  Arguments, layout and
 * errors as hhg_apply_scaled; u_dev and y_dev must not overlap. */
int hhg_apply_volface(hhg_mesh mesh, int depth, const void* u_dev, void* y_dev, int dtype, void* stream);

/* Tensor coefficient K (Sec. 7.3; eq. "integral" and eq. "meshdep" with
 * M = 6).  K6_dev: FP64 device array of 6 x n_stored(depth 0), component
 * major: K11, K22, K33, K12, K13, K23 at every stored node.  The library
 * splits K = sum_m k_m d_m d_m^T along d = e1, e2, e3, e1-e2, e1-e3, e2-e3
 * (k_i = K_ii + sum_{j != i} K_ij, k_ij = -K_ij; all k_m >= 0 when the
 * off-diagonal entries of K are <= 0, as in the paper's test), injects the
 * k_m to every depth and builds the six terms' reference stencils on first
 * use.  Independent of hhg_set_coefficient. */
int hhg_set_tensor_coefficient(hhg_mesh mesh, const void* K6_dev, void* stream);

/* y = A_K u: every row sum_m sum_d c^m_d (k_m(x) + k_m(x+w_d)) (u_{x+w_d} - u_x)
 * with c^m the (1/2) reference stencil of (d_m . grad)(d_m . grad).  dtype
 * HHG_F64 or HHG_F32; u_dev and y_dev must not overlap; HHG_ERR_STATE without
 * a tensor coefficient. */
int hhg_apply_tensor(hhg_mesh mesh, int depth, const void* u_dev, void* y_dev, int dtype, void* stream);

/* r = f - A_s(k) u at `depth` (the residual of the paper's benchmark, Sec. 7.4). */
int hhg_residual(hhg_mesh mesh, int depth, const void* f_dev, const void* u_dev, void* r_dev,
                 int dtype, void* stream);

/* `sweeps` smoothing steps on A_s u = f at `depth`, in place on u_dev:
 * Jacobi u += omega D^-1 (f - A u) with D the operator diagonal
 * (-sum of the scaled off-diagonals, computed on the fly), or Chebyshev of
 * the mesh's degree on D^-1 A.  Uses library workspace. */
int hhg_smooth(hhg_mesh mesh, int depth, int kind, int sweeps, double omega,
               const void* f_dev, void* u_dev, int dtype, void* stream);

/* Damped-Jacobi smoothing like hhg_smooth(kind = HHG_SMOOTH_JACOBI) that
 * never allocates.  The paper has no counterpart: this exists for callers
 * that must not trigger a device allocation during the call (hhg_smooth
 * allocates its ping-pong vector on first use of a depth), e.g. code whose
 * memory budget is fixed before the solve or that runs where cudaMalloc is
 * not allowed.  The ping-pong vector lives in one fixed array of 16 MiB
 * inside the library image (held on every GPU that loads the library until
 * the process exits); a depth whose vector needs more than 16 MiB (more than
 * 2^21 FP64 or 2^22 FP32 stored nodes) is rejected with HHG_ERR_ARG.  The
 * first call on a device looks the array's device address up
 * (cudaGetSymbolAddress); make that first call outside any stream capture.
 * All calls share the array: calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  Each sweep
 * overwrites the whole vector, so nothing needs clearing between calls.
 * Arguments as for hhg_smooth; u_dev holds the result. */
int hhg_smooth_noalloc(hhg_mesh mesh, int depth, int sweeps, double omega, const void* f_dev, void* u_dev,
                       int dtype, void* stream);

/* ---- learned smoother ------------------------------------------------------
 * The paper has no learned component; this is an addition to its multigrid.
 * A network of two 3x3x3 convolutions in the (i,j,k) index space of each
 * macro tet (2 -> 16 -> 1 channels, ReLU, no biases) maps the residual to a
 * correction c.  Inputs: a0 = r / D (0 on Dirichlet nodes), a1 = a0 log k;
 * values outside a tet's index set are zero; a node shared by several macro
 * tets takes the mean of their values; Dirichlet nodes get 0.  Weights: 1296
 * floats, W1[t][a][c] (27 x 2 x 16) then W2[t][c] (27 x 16), tap
 * t = 9 (dk+1) + 3 (dj+1) + (di+1) for the offset (di,dj,dk).  In a V-cycle
 * (HHG_SMOOTH_LEARNED) each pre-smoothing block runs Jacobi, learned, Jacobi,
 * ... and each post-smoothing block learned, Jacobi, ...; a learned step is
 * u += c(f - A u).  The step is nonlinear, so CG switches to its flexible
 * form (beta = z_new.(r_new - r_old) / z_old.r_old).  Learned steps run on
 * FP32 vectors only (dtype HHG_F32 or HHG_F32_KBF16; hhg_solve modes MIXED
 * and MIXED_KBF16). */

/* Train the network on the GPU for the mesh's current coefficient.  Pairs
 * (r, e) with r = A e: e a random vector (or the error one plain V-cycle
 * leaves of it), after the damped Jacobi sweep that precedes a learned step.
 * Loss (e - c)^T A (e - c) / e^T r, the relative energy error after the step;
 * Adam.  The initial weights are the network equal to damped Jacobi plus
 * uniform noise of size init_noise.  Afterwards the plain V-cycle judges the
 * result: the network is accepted only if FP32 PCG with it reduces the
 * residual faster per iteration than with the plain V(2,2) cycle.
 * Synchronous.  HHG_ERR_STATE without a coefficient. */
int hhg_learned_train(hhg_mesh mesh, const hhg_learn_params* p, hhg_learn_stats* stats, void* stream);

/* Set (host in, 1296 floats) or read (host out) the FP32 master weights.
 * Setting marks the network accepted; weights_bf16 selects BF16 (1) or FP32
 * (0) weights in the kernels.  Synchronous. */
int hhg_learned_set_weights(hhg_mesh mesh, const float* w_host, int weights_bf16);
int hhg_learned_get_weights(hhg_mesh mesh, float* w_host);

/* c = network(r) at a smoothed depth (FP32 device vectors, stored layout;
 * consistent on interface copies, 0 on Dirichlet nodes). */
int hhg_learned_forward(hhg_mesh mesh, int depth, const void* r_dev, void* c_dev, void* stream);

/* Loss of one pair and its gradient with respect to the 1296 weights (host
 * out, FP64; FP32 products, FP64 sums over tiles).  r_dev, e_dev: FP32
 * device vectors with r = A e.  Synchronous. */
int hhg_learned_loss_grad(hhg_mesh mesh, int depth, const void* r_dev, const void* e_dev, double* loss,
                          double* grad_host, void* stream);

/* rc = P^T rf (restriction, depth -> depth+1) and uf += P ec (prolongation,
 * depth+1 -> depth), P = linear interpolation between nested P1 spaces. */
int hhg_restrict(hhg_mesh mesh, int depth, const void* rf_dev, void* rc_dev, int dtype, void* stream);
int hhg_prolongate_add(hhg_mesh mesh, int depth, const void* ec_dev, void* uf_dev, int dtype, void* stream);

/* One symmetric V(nu1,nu2) cycle for A_s u = f at depth 0, in place on u_dev. */
int hhg_vcycle(hhg_mesh mesh, int nu1, int nu2, int smoother, const void* f_dev, void* u_dev,
               int dtype, void* stream);

/* Largest eigenvalue estimate of D^-1 A at a depth (power iteration from
 * cos(pi N (x+y+z)) + 1/4, `its` steps, Rayleigh quotient); host out. */
int hhg_lambda_max(hhg_mesh mesh, int depth, int its, int dtype, double* out, void* stream);

/* FP64 dot product over unique unknowns (each interface node counted once). */
int hhg_dot(hhg_mesh mesh, int depth, const void* x_dev, const void* y_dev, int dtype,
            double* out, void* stream);

/* Solve A_s(k) u = f to ||f - A u|| / ||f|| <= p->tol with GMG-preconditioned
 * CG (FP64) or FP64 iterative refinement around FP32 GMG-CG.  f_dev, u_dev:
 * FP64 device arrays, depth-0 layout; u_dev is the initial guess on entry and
 * the solution on exit.  Synchronous (reads residual norms back).  Returns
 * HHG_ERR_NOT_CONVERGED (with stats filled) if the limits are hit. */
int hhg_solve(hhg_mesh mesh, const hhg_solve_params* p, const double* f_dev, double* u_dev,
              hhg_solve_stats* stats, void* stream);

/* Options of a mesh.  The method: "kappa" (0 or 1): 1 scales every
 * direction of gray type (a positive entry of the macro tetrahedron's
 * reference volume stencil, Sec. 4.2) with (k_min(x) + k_min(y))/2 instead
 * of (k_x + k_y)/2, k_min(x) the minimum of k over x and its edge neighbours
 * inside that macro tetrahedron (Sec. 4, eq. "defKmin": the pre-asymptotic
 * modification that keeps the form coercive); all modes of the scaled
 * operator and the solvers use it; synchronises the device.  Tuning (not
 * part of the method): "kseg" planes per volume work item of the k-march and
 * "korder" (0: longest item first, 1: items ordered by plane window) -- both
 * rebuild the work lists and synchronise the device --, "vkernel" (1: the
 * column-march volume kernel, 2: the same with two column sets per lane in
 * packed FP32x2 arithmetic for the FP32 apply, the other modes and FP64
 * running as 1; 0: the tile-march one), "cheb_degree",
 * "cheb_lo", "cheb_hi" (Chebyshev interval as fractions of lambda_max) and
 * "power_its" (lambda_max estimate).  Unknown keys or out-of-range values:
 * HHG_ERR_ARG. */
int hhg_set_option(hhg_mesh mesh, const char* key, double value);
int hhg_get_option(hhg_mesh mesh, const char* key, double* value);

/* Device-side error word of the mesh: HHG_ERR_TIMEOUT if a kernel had set it
 * since the last check, HHG_OK otherwise.  No kernel of this library waits on
 * memory written by another block or launch (the staging waits are cp.async
 * groups), so none sets it and the call returns HHG_OK; it is kept for kernels
 * with bounded waits.  Synchronous; clears the word. */
int hhg_device_status(hhg_mesh mesh);

/* Arithmetic peak probe (a measurement aid, not part of the method): one
 * launch of `blocks` blocks of 256 threads on `stream`, every thread running
 * 8 independent multiply-add chains for `iters` steps.  kind 0: FP64 fma,
 * 1: FP32 fma, 2: packed FP32x2 fma (two per instruction).  out_dev: device
 * array of at least blocks * 256 doubles (each thread's chain sum, written
 * so nothing is folded away).  *flops receives the floating-point operations
 * the launch performs (2 per multiply-add); divide by the launch's
 * CUDA-event time for the rate.  Asynchronous.  HHG_ERR_ARG for an unknown
 * kind, non-positive sizes or NULL pointers; HHG_ERR_CUDA if the launch
 * fails. */
int hhg_alu_probe(int kind, int blocks, int iters, void* out_dev, double* flops, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* hhg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HHG_H */
