// extern "C" entry points (include/hhg.h): argument checks, error mapping.
#include <cstdint>
#include <cstring>
#include <string>

#include "hhg_internal.h"

namespace hhg {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

size_t elem_size(int dtype);
void set_coefficient(Mesh& m, const double* k, cudaStream_t s);
void set_tensor_coefficient(Mesh& m, const double* K6, cudaStream_t s);
void* workspace(Mesh& m, int depth, int prec, int w);
void apply_scaled(Mesh& m, int depth, int dtype, const void* u, void* y, cudaStream_t s);
void residual(Mesh& m, int depth, int dtype, const void* f, const void* u, void* r, bool nc_only, cudaStream_t s);
void smooth(Mesh& m, int depth, int dtype, int kind, int sweeps, double omega, const void* f, void* u, bool nc_only,
            cudaStream_t s, bool post);
void restrict_residual(Mesh& m, int depth, int dtype, const void* rf, void* rc, cudaStream_t s);
void prolongate_add(Mesh& m, int depth, int dtype, const void* ec, void* uf, cudaStream_t s);
void vcycle(Mesh& m, int dtype, int nu1, int nu2, int smoother, double omega, const void* f0, void* u0, cudaStream_t s);
void prepare(Mesh& m, int dtype, int smoother, cudaStream_t s);
double lambda_max(Mesh& m, int depth, int its, cudaStream_t s);
void dot(Mesh& m, int depth, int dtype, const void* x, const void* y, int slot, int post, bool nc_only, cudaStream_t s);
int solve(Mesh& m, const hhg_solve_params& p, const double* f, double* u, hhg_solve_stats* st, cudaStream_t s);
void autotune(Mesh& m, int dtype, const char* cache, int* out_kseg, int* out_korder, double* out_ms, cudaStream_t s);
void init_launch_configs(int dtype);
void learned_prepare(Mesh& m, int dtype, cudaStream_t s);
bool learned_option(Mesh& m, const std::string& key, double* value, bool set);
void learned_train(Mesh& m, const hhg_learn_params& p, hhg_learn_stats* st, cudaStream_t s);
void learned_set_weights(Mesh& m, const float* w_host, int bf16, cudaStream_t s);
void learned_get_weights(Mesh& m, float* w_host, cudaStream_t s);
void learned_forward(Mesh& m, int d, const float* r, float* c, cudaStream_t s);
void learned_loss_grad(Mesh& m, int d, const float* r, const float* e, double* loss, double* grad_host, cudaStream_t s);
}  // namespace hhg

using namespace hhg;

struct hhg_mesh_s {
  Mesh* m;
};

template <class F>
static int guarded(F&& f) {
  try {
    f();
    g_last_error.clear();
    return HHG_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return HHG_ERR_NOMEM;
  } catch (const std::exception& e) {
    set_error(e.what());
    return HHG_ERR_ARG;
  } catch (...) {
    set_error("unknown error");
    return HHG_ERR_ARG;
  }
}

static Mesh& need(hhg_mesh h, bool device = true) {
  if (!h || !h->m) throw Error{HHG_ERR_ARG, "null mesh"};
  if (device && !h->m->device) throw Error{HHG_ERR_STATE, "mesh was created host-only"};
  return *h->m;
}
static void need_depth(const Mesh& m, int depth) {
  if (depth < 0 || depth >= m.ndepth)
    throw Error{HHG_ERR_ARG, "depth " + std::to_string(depth) + " out of range [0, " + std::to_string(m.ndepth) + ")"};
}
static void need_dtype(int dtype) {
  if (dtype != HHG_F64 && dtype != HHG_F32 && dtype != HHG_F32_KBF16)
    throw Error{HHG_ERR_ARG, "unknown dtype " + std::to_string(dtype)};
}
static void need_coef(const Mesh& m) {
  if (!m.coef_set) throw Error{HHG_ERR_STATE, "hhg_set_coefficient must be called first"};
}
static void need_ptr(const void* p, const char* name) {
  if (!p) throw Error{HHG_ERR_ARG, std::string(name) + " is NULL"};
}
// Vectors are staged with 16-byte bulk copies: their base must be 16-byte aligned.
static void need_vec(const void* p, const char* name) {
  need_ptr(p, name);
  if (reinterpret_cast<uintptr_t>(p) % 16)
    throw Error{HHG_ERR_ARG, std::string(name) + " must be 16-byte aligned"};
}

extern "C" {

int hhg_create_macromesh(const double* verts, int nv, const int* tets, int nt, const int* levels,
                         int coarsest_level, hhg_mesh* out) {
  return guarded([&] {
    need_ptr(out, "out");
    *out = nullptr;
    Mesh* m = build_mesh(verts, nv, tets, nt, levels, coarsest_level, true);
    *out = new hhg_mesh_s{m};
  });
}

int hhg_create_macromesh_host(const double* verts, int nv, const int* tets, int nt, const int* levels,
                              int coarsest_level, hhg_mesh* out) {
  return guarded([&] {
    need_ptr(out, "out");
    *out = nullptr;
    Mesh* m = build_mesh(verts, nv, tets, nt, levels, coarsest_level, false);
    *out = new hhg_mesh_s{m};
  });
}

int hhg_destroy_macromesh(hhg_mesh mesh) {
  return guarded([&] {
    if (!mesh) return;
    if (mesh->m && mesh->m->device) cudaDeviceSynchronize();
    free_mesh(mesh->m);
    delete mesh;
  });
}

int hhg_num_depths(hhg_mesh mesh, int* n) {
  return guarded([&] {
    need_ptr(n, "n");
    *n = need(mesh, false).ndepth;
  });
}

int hhg_layout(hhg_mesh mesh, int depth, int64_t* tet_offsets, int* tet_levels, int64_t* n_stored) {
  return guarded([&] {
    Mesh& m = need(mesh, false);
    need_depth(m, depth);
    const Depth& D = m.depth[depth];
    if (tet_offsets)
      for (int t = 0; t <= m.nt; ++t) tet_offsets[t] = D.tet_offset[t];
    if (tet_levels)
      for (int t = 0; t < m.nt; ++t) tet_levels[t] = D.tet_level[t];
    if (n_stored) *n_stored = D.n_stored;
  });
}

int hhg_node_coords(hhg_mesh mesh, int depth, double* xyz) {
  return guarded([&] {
    Mesh& m = need(mesh, false);
    need_depth(m, depth);
    need_ptr(xyz, "xyz");
    std::vector<double> v;
    node_coords(m, depth, v);
    std::memcpy(xyz, v.data(), v.size() * sizeof(double));
  });
}

int hhg_get_stencils(hhg_mesh mesh, int tet, int depth, double* out) {
  return guarded([&] {
    Mesh& m = need(mesh, false);
    need_depth(m, depth);
    need_ptr(out, "out");
    if (tet < 0 || tet >= m.nt) throw Error{HHG_ERR_ARG, "tet out of range"};
    const Depth& D = m.depth[depth];
    const int s = D.tet_slot[tet];
    if (s < 0) throw Error{HHG_ERR_ARG, "tet is not active at this depth"};
    std::memcpy(out, &D.h_sten[(size_t)s * 16 * kNDir], 16 * kNDir * sizeof(double));
  });
}

int hhg_set_coefficient(hhg_mesh mesh, const double* k_dev, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_ptr(k_dev, "k_dev");
    set_coefficient(m, k_dev, (cudaStream_t)stream);
  });
}

int hhg_apply_scaled(hhg_mesh mesh, int depth, const void* u_dev, void* y_dev, int dtype, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    need_dtype(dtype);
    need_coef(m);
    need_vec(u_dev, "u_dev");
    need_vec(y_dev, "y_dev");
    if (u_dev == y_dev) throw Error{HHG_ERR_ARG, "u_dev and y_dev must not overlap"};
    apply_scaled(m, depth, dtype, u_dev, y_dev, (cudaStream_t)stream);
  });
}

int hhg_apply_nodal(hhg_mesh mesh, int depth, const void* u_dev, void* y_dev, int dtype, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    need_dtype(dtype);
    need_coef(m);
    need_vec(u_dev, "u_dev");
    need_vec(y_dev, "y_dev");
    if (u_dev == y_dev) throw Error{HHG_ERR_ARG, "u_dev and y_dev must not overlap"};
    launch_nodal_apply(m, depth, dtype, u_dev, y_dev, (cudaStream_t)stream);
  });
}

int hhg_set_tensor_coefficient(hhg_mesh mesh, const void* K6_dev, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_ptr(K6_dev, "K6_dev");
    set_tensor_coefficient(m, static_cast<const double*>(K6_dev), (cudaStream_t)stream);
  });
}

int hhg_apply_tensor(hhg_mesh mesh, int depth, const void* u_dev, void* y_dev, int dtype, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    if (dtype != HHG_F64 && dtype != HHG_F32) throw Error{HHG_ERR_ARG, "hhg_apply_tensor: dtype HHG_F64 or HHG_F32"};
    if (!m.tensor_set) throw Error{HHG_ERR_STATE, "hhg_set_tensor_coefficient must be called first"};
    need_vec(u_dev, "u_dev");
    need_vec(y_dev, "y_dev");
    if (u_dev == y_dev) throw Error{HHG_ERR_ARG, "u_dev and y_dev must not overlap"};
    OpArgs a{u_dev, nullptr, y_dev, nullptr, nullptr, 0, 0, 0, 0};
    launch_tensor_op(m, depth, dtype, OP_APPLY, a, (cudaStream_t)stream);
  });
}

int hhg_apply_volface(hhg_mesh mesh, int depth, const void* u_dev, void* y_dev, int dtype, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    need_dtype(dtype);
    need_coef(m);
    need_vec(u_dev, "u_dev");
    need_vec(y_dev, "y_dev");
    if (u_dev == y_dev) throw Error{HHG_ERR_ARG, "u_dev and y_dev must not overlap"};
    init_launch_configs(dtype);
    OpArgs a{u_dev, nullptr, y_dev, nullptr, nullptr, 0, 0, 0, 0};
    launch_volface_op(m, depth, dtype, OP_APPLY, a, (cudaStream_t)stream);
  });
}

int hhg_apply_mass(hhg_mesh mesh, int depth, const void* u_dev, void* y_dev, int dtype, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    if (dtype != HHG_F64 && dtype != HHG_F32) throw Error{HHG_ERR_ARG, "hhg_apply_mass supports HHG_F64 and HHG_F32"};
    need_vec(u_dev, "u_dev");
    need_vec(y_dev, "y_dev");
    if (u_dev == y_dev) throw Error{HHG_ERR_ARG, "u_dev and y_dev must not overlap"};
    launch_mass_apply(m, depth, dtype, u_dev, y_dev, (cudaStream_t)stream);
  });
}

int hhg_autotune(hhg_mesh mesh, int dtype, const char* cache_path, int* kseg, int* korder, double* best_ms,
                 void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_dtype(dtype);
    need_coef(m);
    autotune(m, dtype, cache_path, kseg, korder, best_ms, (cudaStream_t)stream);
  });
}

int hhg_residual(hhg_mesh mesh, int depth, const void* f_dev, const void* u_dev, void* r_dev, int dtype,
                 void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    need_dtype(dtype);
    need_coef(m);
    need_vec(f_dev, "f_dev");
    need_vec(u_dev, "u_dev");
    need_vec(r_dev, "r_dev");
    residual(m, depth, dtype, f_dev, u_dev, r_dev, false, (cudaStream_t)stream);
  });
}

int hhg_smooth(hhg_mesh mesh, int depth, int kind, int sweeps, double omega, const void* f_dev, void* u_dev,
               int dtype, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    need_dtype(dtype);
    need_coef(m);
    need_vec(f_dev, "f_dev");
    need_vec(u_dev, "u_dev");
    if (sweeps < 0) throw Error{HHG_ERR_ARG, "sweeps must be >= 0"};
    if (kind != HHG_SMOOTH_JACOBI && kind != HHG_SMOOTH_CHEBYSHEV && kind != HHG_SMOOTH_LEARNED)
      throw Error{HHG_ERR_ARG, "unknown smoother"};
    init_launch_configs(dtype);
    if (kind == HHG_SMOOTH_LEARNED) {
      if (depth + 1 >= m.ndepth) throw Error{HHG_ERR_ARG, "the coarsest depth is not smoothed"};
      learned_prepare(m, dtype, (cudaStream_t)stream);
    }
    smooth(m, depth, dtype, kind, sweeps, omega, f_dev, u_dev, false, (cudaStream_t)stream, false);
  });
}

int hhg_restrict(hhg_mesh mesh, int depth, const void* rf_dev, void* rc_dev, int dtype, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    need_dtype(dtype);
    need_vec(rf_dev, "rf_dev");
    need_vec(rc_dev, "rc_dev");
    restrict_residual(m, depth, dtype, rf_dev, rc_dev, (cudaStream_t)stream);
  });
}

int hhg_prolongate_add(hhg_mesh mesh, int depth, const void* ec_dev, void* uf_dev, int dtype, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    need_dtype(dtype);
    need_vec(ec_dev, "ec_dev");
    need_vec(uf_dev, "uf_dev");
    prolongate_add(m, depth, dtype, ec_dev, uf_dev, (cudaStream_t)stream);
  });
}

int hhg_vcycle(hhg_mesh mesh, int nu1, int nu2, int smoother, const void* f_dev, void* u_dev, int dtype,
               void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_dtype(dtype);
    need_coef(m);
    need_vec(f_dev, "f_dev");
    need_vec(u_dev, "u_dev");
    if (nu1 < 0 || nu2 < 0) throw Error{HHG_ERR_ARG, "nu1, nu2 must be >= 0"};
    if (smoother < 0 || smoother > 2) throw Error{HHG_ERR_ARG, "unknown smoother"};
    prepare(m, dtype, smoother, (cudaStream_t)stream);
    vcycle(m, dtype, nu1, nu2, smoother, 2.0 / 3.0, f_dev, u_dev, (cudaStream_t)stream);
  });
}

int hhg_lambda_max(hhg_mesh mesh, int depth, int its, int dtype, double* out, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    need_coef(m);
    need_ptr(out, "out");
    (void)dtype;
    init_launch_configs(HHG_F64);
    m.depth[depth].lam = 0.0;
    const int keep = m.power_its;
    m.power_its = its;
    *out = lambda_max(m, depth, its, (cudaStream_t)stream);
    m.power_its = keep;
    if (its != keep) m.depth[depth].lam = 0.0;
  });
}

int hhg_dot(hhg_mesh mesh, int depth, const void* x_dev, const void* y_dev, int dtype, double* out, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    need_dtype(dtype);
    need_vec(x_dev, "x_dev");
    need_vec(y_dev, "y_dev");
    need_ptr(out, "out");
    cudaStream_t s = (cudaStream_t)stream;
    dot(m, depth, dtype, x_dev, y_dev, 20, 0, false, s);
    HHG_CUDA(cudaMemcpyAsync(m.h_pinned, m.d_scalars + 20, sizeof(double), cudaMemcpyDeviceToHost, s));
    HHG_CUDA(cudaStreamSynchronize(s));
    *out = m.h_pinned[0];
  });
}

int hhg_solve(hhg_mesh mesh, const hhg_solve_params* p, const double* f_dev, double* u_dev, hhg_solve_stats* stats,
              void* stream) {
  int status = HHG_OK;
  const int rc = guarded([&] {
    Mesh& m = need(mesh);
    need_ptr(p, "params");
    if (p->op != HHG_OP_TENSOR) need_coef(m);
    need_vec(f_dev, "f_dev");
    need_vec(u_dev, "u_dev");
    if (p->smoother < 0 || p->smoother > 2) throw Error{HHG_ERR_ARG, "unknown smoother"};
    if (p->nu1 < 0 || p->nu2 < 0) throw Error{HHG_ERR_ARG, "nu1, nu2 must be >= 0"};
    cudaStream_t s = (cudaStream_t)stream;
    cudaStream_t own = nullptr;
    if (!s && p->use_graph) {  // graph capture needs a non-legacy stream
      HHG_CUDA(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
      HHG_CUDA(cudaDeviceSynchronize());
      s = own;
    }
    try {
      status = solve(m, *p, f_dev, u_dev, stats, s);
    } catch (...) {
      if (own) cudaStreamDestroy(own);
      throw;
    }
    if (own) {
      HHG_CUDA(cudaStreamSynchronize(own));
      cudaStreamDestroy(own);
    }
  });
  if (rc != HHG_OK) return rc;
  if (status == HHG_ERR_NOT_CONVERGED) set_error("solver did not reach the tolerance within the iteration limits");
  return status;
}

int hhg_set_option(hhg_mesh mesh, const char* key, double value) {
  return guarded([&] {
    Mesh& m = need(mesh, false);
    drop_graphs(m);
    need_ptr(key, "key");
    const std::string k(key);
    if (k == "kseg") {
      set_kseg(m, (int)value, m.korder);
    } else if (k == "korder") {
      set_kseg(m, m.kseg, (int)value);
    } else if (k == "kappa") {
      if (value != 0 && value != 1) throw Error{HHG_ERR_ARG, "kappa must be 0 or 1"};
      m.kappa = value != 0;
      if (m.kappa && m.coef_set && m.device) {
        compute_kmin(m, nullptr);
        HHG_CUDA(cudaDeviceSynchronize());
      }
      // the operator changed: coarse inverses and eigenvalue estimates are stale
      for (int o = 0; o < 4; ++o)
        for (int t = 0; t < 4; ++t) m.cinv_ready[o][t] = false;
      for (Depth& D : m.depth) D.lam = 0.0;
    } else if (k == "vkernel") {
      if (value != 0 && value != 1 && value != 2) throw Error{HHG_ERR_ARG, "vkernel must be 0, 1 or 2"};
      m.vkernel = (int)value;
    } else if (k == "cheb_degree") {
      if (value < 1 || value > 16) throw Error{HHG_ERR_ARG, "cheb_degree must be in [1, 16]"};
      m.cheb_degree = (int)value;
    } else if (k == "cheb_lo") {
      if (!(value > 0 && value < m.cheb_hi)) throw Error{HHG_ERR_ARG, "cheb_lo must be in (0, cheb_hi)"};
      m.cheb_lo = value;
    } else if (k == "cheb_hi") {
      if (!(value > m.cheb_lo)) throw Error{HHG_ERR_ARG, "cheb_hi must exceed cheb_lo"};
      m.cheb_hi = value;
    } else if (k == "power_its") {
      if (value < 1 || value > 1000) throw Error{HHG_ERR_ARG, "power_its must be in [1, 1000]"};
      m.power_its = (int)value;
      for (Depth& D : m.depth) D.lam = 0.0;
    } else if (!learned_option(m, k, &value, true)) {
      throw Error{HHG_ERR_ARG, "unknown option '" + k + "'"};
    }
  });
}

int hhg_get_option(hhg_mesh mesh, const char* key, double* value) {
  return guarded([&] {
    Mesh& m = need(mesh, false);
    need_ptr(key, "key");
    need_ptr(value, "value");
    const std::string k(key);
    if (k == "kseg") *value = m.kseg;
    else if (k == "korder") *value = m.korder;
    else if (k == "vkernel") *value = m.vkernel;
    else if (k == "kappa") *value = m.kappa ? 1 : 0;
    else if (k == "cheb_degree") *value = m.cheb_degree;
    else if (k == "cheb_lo") *value = m.cheb_lo;
    else if (k == "cheb_hi") *value = m.cheb_hi;
    else if (k == "power_its") *value = m.power_its;
    else if (!learned_option(m, k, value, false)) throw Error{HHG_ERR_ARG, "unknown option '" + k + "'"};
  });
}

int hhg_device_status(hhg_mesh mesh) {
  int code = HHG_OK;
  const int rc = guarded([&] {
    Mesh& m = need(mesh);
    unsigned e = 0;
    HHG_CUDA(cudaMemcpy(&e, m.d_error, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (e) {
      HHG_CUDA(cudaMemset(m.d_error, 0, sizeof(unsigned)));
      code = HHG_ERR_TIMEOUT;
    }
  });
  if (rc != HHG_OK) return rc;
  if (code != HHG_OK) set_error("a device-side bounded wait ran out (results of the affected call are invalid)");
  return code;
}

const char* hhg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ---- learned smoother ---------------------------------------------------------

int hhg_learned_train(hhg_mesh mesh, const hhg_learn_params* p, hhg_learn_stats* stats, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_coef(m);
    need_ptr(p, "params");
    cudaStream_t s = (cudaStream_t)stream;
    init_launch_configs(HHG_F32);
    init_launch_configs(HHG_F64);
    learned_train(m, *p, stats, s);
  });
}

int hhg_learned_set_weights(hhg_mesh mesh, const float* w_host, int weights_bf16) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_ptr(w_host, "w_host");
    learned_set_weights(m, w_host, weights_bf16, nullptr);
  });
}

int hhg_learned_get_weights(hhg_mesh mesh, float* w_host) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_ptr(w_host, "w_host");
    learned_get_weights(m, w_host, nullptr);
  });
}

int hhg_learned_forward(hhg_mesh mesh, int depth, const void* r_dev, void* c_dev, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    need_coef(m);
    need_vec(r_dev, "r_dev");
    need_vec(c_dev, "c_dev");
    init_launch_configs(HHG_F64);
    learned_forward(m, depth, static_cast<const float*>(r_dev), static_cast<float*>(c_dev), (cudaStream_t)stream);
  });
}

int hhg_learned_loss_grad(hhg_mesh mesh, int depth, const void* r_dev, const void* e_dev, double* loss,
                          double* grad_host, void* stream) {
  return guarded([&] {
    Mesh& m = need(mesh);
    need_depth(m, depth);
    need_coef(m);
    need_vec(r_dev, "r_dev");
    need_vec(e_dev, "e_dev");
    init_launch_configs(HHG_F32);
    init_launch_configs(HHG_F64);
    learned_loss_grad(m, depth, static_cast<const float*>(r_dev), static_cast<const float*>(e_dev), loss, grad_host,
                      (cudaStream_t)stream);
  });
}
