// Allocation-free damped-Jacobi smoothing.
//
// hhg_smooth keeps its ping-pong vector in library workspace that it
// allocates with cudaMalloc the first time a depth and precision are used.
// Some callers cannot allow that: code that runs while the device must not
// allocate (for example inside a real-time loop, or in a process whose memory
// budget was fixed before the solver started), or callers that have no
// allocation rights at all.  This file gives them hhg_smooth_noalloc, which
// runs the same fused Jacobi kernel but keeps the ping-pong vector in a
// fixed-size array that lives in the library image itself.
//
// The array is file-scope device memory: every GPU that loads the library
// holds it (kNoAllocBytes) until the process exits.  Host code must not pass
// the array's name to a kernel (on the host the name is only a stand-in for
// the device symbol, not a device address); it looks the device address up
// with cudaGetSymbolAddress on every call and passes that pointer.
#include <new>

#include "hhg_internal.h"

namespace hhg {

constexpr size_t kNoAllocBytes = 16u << 20;  // 16 MiB: 2M FP64 or 4M FP32 entries

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
// Device address of the scratch array in the current context, looked up on
// every call (a cached address would outlive a device reset)
void* noalloc_scratch() {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    throw Error{HHG_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
  return p;
}
}  // namespace

size_t elem_size(int dtype);
void init_launch_configs(int dtype);

}  // namespace hhg

using namespace hhg;

struct hhg_mesh_s {
  Mesh* m;
};

extern "C" int hhg_smooth_noalloc(hhg_mesh mesh, int depth, int sweeps, double omega, const void* f_dev,
                                  void* u_dev, int dtype, void* stream) {
  try {
    if (!mesh || !mesh->m) throw Error{HHG_ERR_ARG, "null mesh"};
    Mesh& m = *mesh->m;
    if (!m.device) throw Error{HHG_ERR_STATE, "mesh was created host-only"};
    if (depth < 0 || depth >= m.ndepth) throw Error{HHG_ERR_ARG, "depth out of range"};
    if (dtype != HHG_F64 && dtype != HHG_F32 && dtype != HHG_F32_KBF16) throw Error{HHG_ERR_ARG, "unknown dtype"};
    if (!m.coef_set) throw Error{HHG_ERR_STATE, "hhg_set_coefficient must be called first"};
    if (!f_dev || !u_dev) throw Error{HHG_ERR_ARG, "f_dev and u_dev must not be NULL"};
    if (reinterpret_cast<uintptr_t>(f_dev) % 16 || reinterpret_cast<uintptr_t>(u_dev) % 16)
      throw Error{HHG_ERR_ARG, "f_dev and u_dev must be 16-byte aligned"};
    if (sweeps < 0) throw Error{HHG_ERR_ARG, "sweeps must be >= 0"};
    const Depth& D = m.depth[depth];
    const size_t need = (size_t)D.n_stored * elem_size(dtype);
    if (need > kNoAllocBytes)
      throw Error{HHG_ERR_ARG, "hhg_smooth_noalloc: the depth vector needs " + std::to_string(need) +
                                   " bytes of scratch, more than its fixed " + std::to_string(kNoAllocBytes) +
                                   " bytes (use hhg_smooth)"};
    void* w = noalloc_scratch();
    cudaStream_t s = (cudaStream_t)stream;
    init_launch_configs(dtype);
    // ping-pong between u and the scratch vector; each sweep writes every
    // stored node of its output, so the scratch needs no clearing
    void* a = u_dev;
    void* b = w;
    for (int it = 0; it < sweeps; ++it) {
      OpArgs args{a, f_dev, b, nullptr, nullptr, omega, 0, 0, 0};
      launch_scaled_op(m, depth, dtype, OP_JACOBI, args, s);
      std::swap(a, b);
    }
    if (a != u_dev && D.n_stored > 0)
      HHG_CUDA(cudaMemcpyAsync(u_dev, a, need, cudaMemcpyDeviceToDevice, s));
    set_error("");
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
