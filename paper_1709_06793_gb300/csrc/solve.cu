// Solver driver: GMG-preconditioned CG (scalars stay on the device, one CG
// iteration captured as a CUDA graph) and FP64 iterative refinement around an
// FP32 inner solve.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "hhg_internal.h"

namespace hhg {

size_t elem_size(int dtype);
void* workspace(Mesh& m, int depth, int prec, int w);
void dot(Mesh& m, int depth, int dtype, const void* x, const void* y, int slot, int post, bool nc_only, cudaStream_t s);
void residual(Mesh& m, int depth, int dtype, const void* f, const void* u, void* r, bool nc_only, cudaStream_t s);
void apply_scaled(Mesh& m, int depth, int dtype, const void* u, void* y, cudaStream_t s);
void vcycle(Mesh& m, int dtype, int nu1, int nu2, int smoother, double omega, const void* f0, void* u0, cudaStream_t s);
double lambda_max(Mesh& m, int depth, int its, cudaStream_t s);
void ensure_coarse(Mesh& m, int dtype, cudaStream_t s);
const int* coarse_slot_map(Mesh& m, int depth);
void init_launch_configs(int dtype);
void learned_prepare(Mesh& m, int dtype, cudaStream_t s);
bool learned_accepted(Mesh& m);
void random_vector(Mesh& m, int d, float* x, unsigned long long key, cudaStream_t s);
const void* nodal_dinv(Mesh& m, int depth, int dtype, cudaStream_t s);

enum { RED_STORE = 0, RED_ALPHA = 1, RED_BETA = 2, RED_FBETA = 3 };

static int prec_of(int dtype) { return elem_size(dtype) == 8 ? 0 : 1; }

static inline int grid_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)std::min<long long>(b, cap);
}

template <class T>
__global__ void cg_update_kernel2(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                  const T* __restrict__ q, long long n, const double* S) {
  const T alpha = (T)S[2];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
  }
}

template <class T>
__global__ void xpay_kernel2(T* __restrict__ p, const T* __restrict__ z, long long n, const double* S) {
  const T beta = (T)S[5];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

__global__ void set_scalar_kernel(double* S, int slot, double v) { S[slot] = v; }

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void add_f32_kernel(double* __restrict__ x, const float* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

void drop_graphs(Mesh& m) {
  for (auto& g : m.graphs) cudaGraphExecDestroy(g.exec);
  m.graphs.clear();
}

// Allocate every buffer and estimate every quantity a V-cycle / CG needs, so
// that afterwards the iteration only enqueues kernels (capturable).
void prepare(Mesh& m, int dtype, int smoother, cudaStream_t s) {
  if (!m.coef_set && m.opk != 3) throw Error{HHG_ERR_STATE, "hhg_set_coefficient must be called first"};
  HHG_REQUIRE(m.opk == 0 || smoother == HHG_SMOOTH_JACOBI,
              "the Vol+Face and nodal operators are smoothed with damped Jacobi");
  const int pr = prec_of(dtype);
  init_launch_configs(dtype);
  init_launch_configs(HHG_F64);
  for (int d = 0; d < m.ndepth; ++d) {
    for (int w : {0, 1, 2, 3, 4, 5, 6, 7, 8}) workspace(m, d, pr, w);
    if (m.opk == 2) nodal_dinv(m, d, dtype, s);
    if (d + 1 < m.ndepth) coarse_slot_map(m, d);
  }
  if (smoother == HHG_SMOOTH_CHEBYSHEV)
    for (int d = 0; d < m.ndepth; ++d)
      if (m.depth[d].n_slots_nc) lambda_max(m, d, m.power_its, s);
  if (smoother == HHG_SMOOTH_LEARNED) learned_prepare(m, dtype, s);
  ensure_coarse(m, dtype == kF64KBF16 ? (int)HHG_F32_KBF16 : dtype, s);
  HHG_CUDA(cudaStreamSynchronize(s));
}

struct PcgResult {
  int its;
  double rr;
};

// One CG iteration from "z = M r" to "rr = r.r" (see pcg()).
static void pcg_body(Mesh& m, int dtype, const hhg_solve_params& p, void* x, void* r, void* z, void* pp, void* q,
                     cudaStream_t s) {
  const Depth& D0 = m.depth[0];
  const long long n = D0.n_stored;
  const int g = grid_for(n, 256, 8 * m.num_sms);
  HHG_CUDA(cudaMemsetAsync(z, 0, n * elem_size(dtype), s));
  vcycle(m, dtype, p.nu1, p.nu2, p.smoother, p.omega, r, z, s);
  if (p.smoother == HHG_SMOOTH_LEARNED) {
    // nonlinear preconditioner: flexible CG, r_new - r_old = -alpha q
    dot(m, 0, dtype, z, q, 8, RED_STORE, false, s);
    dot(m, 0, dtype, r, z, 4, RED_FBETA, false, s);
  } else {
    dot(m, 0, dtype, r, z, 4, RED_BETA, false, s);  // beta = rz_new / rz; rz = rz_new
  }
  if (elem_size(dtype) == 8)
    xpay_kernel2<double><<<g, 256, 0, s>>>((double*)pp, (const double*)z, n, m.d_scalars);
  else
    xpay_kernel2<float><<<g, 256, 0, s>>>((float*)pp, (const float*)z, n, m.d_scalars);
  HHG_CUDA(cudaGetLastError());
  apply_scaled(m, 0, dtype, pp, q, s);
  dot(m, 0, dtype, pp, q, 1, RED_ALPHA, false, s);  // alpha = rz / pq
  if (elem_size(dtype) == 8)
    cg_update_kernel2<double><<<g, 256, 0, s>>>((double*)x, (double*)r, (const double*)pp, (const double*)q, n,
                                                m.d_scalars);
  else
    cg_update_kernel2<float><<<g, 256, 0, s>>>((float*)x, (float*)r, (const float*)pp, (const float*)q, n,
                                               m.d_scalars);
  HHG_CUDA(cudaGetLastError());
  dot(m, 0, dtype, r, r, 3, RED_STORE, false, s);
}

static double read_scalar(Mesh& m, int slot, cudaStream_t s) {
  HHG_CUDA(cudaMemcpyAsync(m.h_pinned, m.d_scalars + slot, sizeof(double), cudaMemcpyDeviceToHost, s));
  HHG_CUDA(cudaStreamSynchronize(s));
  return m.h_pinned[0];
}

// CG on A x = b preconditioned by one V-cycle; x holds the initial guess and
// the result; r must hold b - A x on entry.  Stops when r.r <= tol2.
static PcgResult pcg(Mesh& m, int dtype, const hhg_solve_params& p, void* x, void* r, double tol2, int maxit,
                     cudaStream_t s) {
  const int pr = prec_of(dtype);
  void* z = workspace(m, 0, pr, 1);
  void* pp = workspace(m, 0, pr, 3);
  void* q = workspace(m, 0, pr, 7);
  const long long n = m.depth[0].n_stored;
  dot(m, 0, dtype, r, r, 3, RED_STORE, false, s);
  double rr = read_scalar(m, 3, s);
  if (rr <= tol2) return {0, rr};
  // first iteration: beta = 0 (rz = +inf), p = 0
  HHG_CUDA(cudaMemsetAsync(pp, 0, n * elem_size(dtype), s));
  set_scalar_kernel<<<1, 1, 0, s>>>(m.d_scalars, 0, INFINITY);
  if (p.smoother == HHG_SMOOTH_LEARNED) {  // flexible beta of the first iteration: (rz - 0 * z.0) / inf = 0
    HHG_CUDA(cudaMemsetAsync(q, 0, n * elem_size(dtype), s));
    set_scalar_kernel<<<1, 1, 0, s>>>(m.d_scalars, 2, 0.0);
  }
  cudaGraphExec_t exec = nullptr;
  if (p.use_graph) {
    for (auto& g : m.graphs)
      if (g.dtype == dtype && g.smoother == p.smoother && g.nu1 == p.nu1 && g.nu2 == p.nu2 && g.omega == p.omega &&
          g.x == x && g.r == r)
        exec = g.exec;
    if (!exec) {
      cudaGraph_t graph = nullptr;
      HHG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
      pcg_body(m, dtype, p, x, r, z, pp, q, s);
      HHG_CUDA(cudaStreamEndCapture(s, &graph));
      HHG_CUDA(cudaGraphInstantiate(&exec, graph, 0));
      cudaGraphDestroy(graph);
      m.graphs.push_back({dtype, p.smoother, p.nu1, p.nu2, p.omega, x, r, exec});
    }
  }
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    if (exec)
      HHG_CUDA(cudaGraphLaunch(exec, s));
    else
      pcg_body(m, dtype, p, x, r, z, pp, q, s);
    rr = read_scalar(m, 3, s);
    if (!(rr > tol2)) break;  // also stops on NaN
  }
  return {std::min(it, maxit), rr};
}

// Residual reduction per iteration of `its` FP32 PCG iterations on A x = A e
// (e a consistent random vector) from x = 0.
double pcg_rate(Mesh& m, int dtype, int smoother, int nu1, int nu2, double omega, int its, unsigned long long seed,
                cudaStream_t s) {
  HHG_REQUIRE(elem_size(dtype) == 4, "pcg_rate runs on FP32 vectors");
  prepare(m, dtype, smoother, s);
  float* x = static_cast<float*>(workspace(m, 0, 1, 8));
  float* r = static_cast<float*>(workspace(m, 0, 1, 0));
  float* e = static_cast<float*>(workspace(m, 0, 1, 9));
  random_vector(m, 0, e, seed, s);
  apply_scaled(m, 0, dtype, e, r, s);
  HHG_CUDA(cudaMemsetAsync(x, 0, m.depth[0].n_stored * 4, s));
  dot(m, 0, dtype, r, r, 3, RED_STORE, false, s);
  const double rr0 = read_scalar(m, 3, s);
  hhg_solve_params p{};
  p.smoother = smoother;
  p.nu1 = nu1;
  p.nu2 = nu2;
  p.omega = omega;
  p.use_graph = 0;
  const PcgResult res = pcg(m, dtype, p, x, r, 0.0, its, s);
  if (!(res.rr >= 0) || rr0 <= 0 || res.its <= 0) return INFINITY;
  return std::pow(res.rr / rr0, 0.5 / res.its);
}

// Multigrid as the solver (Sec. 7.2): u <- V(nu1,nu2)(f, u) in FP64 with the
// operator p.op until ||f - A u|| <= tol ||f|| or p.maxit cycles; rho as in
// Sec. 7, (r^(i*) / r^(5))^(1/(i*-5)) (from r^(0) when i* <= 5).
static int solve_mg(Mesh& m, const hhg_solve_params& p, const double* f, double* u, hhg_solve_stats* st,
                    cudaStream_t s) {
  HHG_REQUIRE(p.smoother == HHG_SMOOTH_JACOBI || (p.smoother == HHG_SMOOTH_CHEBYSHEV && p.op == 0),
              "multigrid solve: Jacobi smoothing (Chebyshev for the scaled operator only)");
  const auto t0 = std::chrono::steady_clock::now();
  struct OpGuard {  // the multigrid internals use p.op for this call only
    Mesh& m;
    OpGuard(Mesh& mm, int opk) : m(mm) {
      drop_graphs(m);
      m.opk = opk;
    }
    ~OpGuard() { m.opk = 0; }
  } guard(m, p.op);
  prepare(m, HHG_F64, p.smoother, s);
  double* r = static_cast<double*>(workspace(m, 0, 0, 8));
  dot(m, 0, HHG_F64, f, f, 6, RED_STORE, false, s);
  const double nf = std::sqrt(read_scalar(m, 6, s));
  std::vector<double> hist;
  residual(m, 0, HHG_F64, f, u, r, false, s);
  dot(m, 0, HHG_F64, r, r, 7, RED_STORE, false, s);
  hist.push_back(std::sqrt(read_scalar(m, 7, s)));
  int it = 0;
  while (it < p.maxit && nf > 0 && hist.back() > p.tol * nf && std::isfinite(hist.back())) {
    vcycle(m, HHG_F64, p.nu1, p.nu2, p.smoother, p.omega, f, u, s);
    residual(m, 0, HHG_F64, f, u, r, false, s);
    dot(m, 0, HHG_F64, r, r, 7, RED_STORE, false, s);
    hist.push_back(std::sqrt(read_scalar(m, 7, s)));
    ++it;
  }
  HHG_CUDA(cudaStreamSynchronize(s));
  const double rel = nf > 0 ? hist.back() / nf : 0.0;
  double rho = 0.0;
  if (it > 5 && hist[5] > 0)
    rho = std::pow(hist[it] / hist[5], 1.0 / (it - 5));
  else if (it > 0 && hist[0] > 0)
    rho = std::pow(hist[it] / hist[0], 1.0 / it);
  if (st) {
    st->iterations = it;
    st->outer = 1;
    st->rel_residual = rel;
    st->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    st->smoother_used = p.smoother;
    st->rho = rho;
  }
  return rel <= p.tol ? HHG_OK : HHG_ERR_NOT_CONVERGED;
}

int solve(Mesh& m, const hhg_solve_params& p_in, const double* f, double* u, hhg_solve_stats* st, cudaStream_t s) {
  hhg_solve_params p = p_in;
  if (p.omega <= 0) p.omega = 2.0 / 3.0;
  if (p.inner_rtol <= 0) p.inner_rtol = 3e-5;
  if (p.max_outer <= 0) p.max_outer = 20;
  if (p.maxit <= 0) p.maxit = 200;
  HHG_REQUIRE(p.tol > 0, "tol must be positive");
  HHG_REQUIRE(p.mode >= 0 && p.mode <= 4, "unknown solve mode");
  HHG_REQUIRE(p.op >= 0 && p.op <= 3, "unknown operator");
  HHG_REQUIRE(p.op != 3 || m.tensor_set, "hhg_set_tensor_coefficient must be called first");
  HHG_REQUIRE(p.op == 0 || p.mode == HHG_SOLVE_MG, "the Vol+Face, nodal and tensor operators are solved with HHG_SOLVE_MG");
  if (p.mode == HHG_SOLVE_MG) return solve_mg(m, p, f, u, st, s);
  const auto t0 = std::chrono::steady_clock::now();
  const long long n = m.depth[0].n_stored;
  const int g = grid_for(n, 256, 8 * m.num_sms);
  HHG_REQUIRE(p.smoother != HHG_SMOOTH_LEARNED || p.mode != HHG_SOLVE_FP64,
              "the learned smoother runs in the FP32 inner solve (modes MIXED, MIXED_KBF16)");
  // the plain V-cycle replaces a learned smoother that is missing or was not accepted
  if (p.smoother == HHG_SMOOTH_LEARNED && !learned_accepted(m)) p.smoother = HHG_SMOOTH_JACOBI;
  const int outer_dtype = p.mode == HHG_SOLVE_MIXED_KBF16 ? kF64KBF16 : HHG_F64;
  int inner_dtype = HHG_F64;
  if (p.mode == HHG_SOLVE_MIXED) inner_dtype = HHG_F32;
  if (p.mode == HHG_SOLVE_MIXED_KBF16 || p.mode == HHG_SOLVE_MIXED_KBF16_INNER) inner_dtype = HHG_F32_KBF16;
  prepare(m, inner_dtype, p.smoother, s);
  if (inner_dtype != HHG_F64) prepare(m, HHG_F64, HHG_SMOOTH_JACOBI, s);
  // ||f||
  dot(m, 0, HHG_F64, f, f, 6, RED_STORE, false, s);
  const double nf2 = read_scalar(m, 6, s);
  const double nf = std::sqrt(nf2);
  int total = 0, outer = 0;
  double rel = 0;
  int status = HHG_OK;
  double* r64 = static_cast<double*>(workspace(m, 0, 0, 8));
  if (nf == 0.0) {
    HHG_CUDA(cudaMemsetAsync(u, 0, n * 8, s));
    rel = 0;
  } else if (p.mode == HHG_SOLVE_FP64) {
    double* r = static_cast<double*>(workspace(m, 0, 0, 0));
    residual(m, 0, HHG_F64, f, u, r, false, s);
    const double tol2 = p.tol * p.tol * nf2;
    PcgResult res = pcg(m, HHG_F64, p, u, r, tol2, p.maxit, s);
    total = res.its;
    outer = 1;
    residual(m, 0, HHG_F64, f, u, r64, false, s);
    dot(m, 0, HHG_F64, r64, r64, 7, RED_STORE, false, s);
    rel = std::sqrt(read_scalar(m, 7, s)) / nf;
    if (rel > p.tol) status = HHG_ERR_NOT_CONVERGED;
  } else {
    float* r32 = static_cast<float*>(workspace(m, 0, 1, 0));
    float* d32 = static_cast<float*>(workspace(m, 0, 1, 8));
    residual(m, 0, outer_dtype, f, u, r64, false, s);
    for (outer = 1; outer <= p.max_outer; ++outer) {
      dot(m, 0, HHG_F64, r64, r64, 7, RED_STORE, false, s);
      const double rr = read_scalar(m, 7, s);
      rel = std::sqrt(rr) / nf;
      if (rel <= p.tol || total >= p.maxit) break;
      f64_to_f32_kernel<<<g, 256, 0, s>>>(r64, r32, n);
      HHG_CUDA(cudaMemsetAsync(d32, 0, n * 4, s));
      // inner: reduce the residual by the factor inner_rtol, but not below
      // half the outer tolerance (the last inner solve stops where the outer
      // one can finish instead of over-solving)
      const double target = std::max(p.inner_rtol * p.inner_rtol * rr, 0.25 * p.tol * p.tol * nf2);
      PcgResult res = pcg(m, inner_dtype, p, d32, r32, target, p.maxit - total, s);
      total += res.its;
      if (p.smoother == HHG_SMOOTH_LEARNED && !(res.rr <= rr)) {
        // divergence guard: a learned inner solve that did not reduce the
        // residual is discarded and the plain V-cycle takes over
        p.smoother = HHG_SMOOTH_JACOBI;
        prepare(m, inner_dtype, p.smoother, s);
        continue;
      }
      add_f32_kernel<<<g, 256, 0, s>>>(u, d32, n);
      HHG_CUDA(cudaGetLastError());
      residual(m, 0, outer_dtype, f, u, r64, false, s);
    }
    if (outer > p.max_outer) {
      // the refinement steps ran out: report the residual of the last correction
      outer = p.max_outer;
      dot(m, 0, HHG_F64, r64, r64, 7, RED_STORE, false, s);
      rel = std::sqrt(read_scalar(m, 7, s)) / nf;
    }
    if (rel > p.tol) status = HHG_ERR_NOT_CONVERGED;
  }
  HHG_CUDA(cudaStreamSynchronize(s));
  const auto t1 = std::chrono::steady_clock::now();
  if (st) {
    st->iterations = total;
    st->outer = outer;
    st->rel_residual = rel;
    st->time_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    st->smoother_used = p.smoother;
    st->rho = 0.0;
  }
  return status;
}

}  // namespace hhg
