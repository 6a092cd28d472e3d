// Arithmetic peak probes: the denominators of the ALU rooflines of the FP64
// kernels (the FP64 stencil apply, smoother and residual) and of the FP32
// nodal-integration apply.  Not part of the method; hhg_alu_probe in
// include/hhg.h.
//
// Every thread runs 8 independent multiply-add chains a <- a * b + c for
// `iters` steps (8 chains hide the FMA latency at full occupancy) and writes
// the sum of its chains, so nothing can be folded away.  b and c are kernel
// arguments, |b| < 1, so the values stay bounded.
#include "hhg_internal.h"

namespace hhg {

template <class T>
__global__ void __launch_bounds__(256) fma_chain_kernel(T b, T c, int iters, double* __restrict__ out) {
  T a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = (T)(threadIdx.x + 8 * q) * (T)1e-3;
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = fma(a[q], b, c);
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = (double)s;
}

// packed FP32 pairs: one instruction performs two multiply-adds
__global__ void __launch_bounds__(256) ffma2_chain_kernel(float b, float c, int iters, double* __restrict__ out) {
  float2 a[8];
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = make_float2((threadIdx.x + 8 * q) * 1e-3f, (threadIdx.x + 8 * q + 4) * 1e-3f);
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = __ffma2_rn(a[q], bb, cc);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q].x + a[q].y;
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = (double)s;
}

}  // namespace hhg

using namespace hhg;

extern "C" int hhg_alu_probe(int kind, int blocks, int iters, void* out_dev, double* flops, void* stream) {
  if (kind < 0 || kind > 2 || blocks <= 0 || iters <= 0 || !out_dev || !flops) {
    set_error("hhg_alu_probe: kind must be 0..2, blocks and iters positive, out_dev and flops non-NULL");
    return HHG_ERR_ARG;
  }
  constexpr int kThreads = 256;
  cudaStream_t s = (cudaStream_t)stream;
  double* out = (double*)out_dev;
  const double lanes = (double)blocks * kThreads * iters * 8;
  if (kind == 0)
    fma_chain_kernel<double><<<blocks, kThreads, 0, s>>>(0.999999, 1e-7, iters, out);
  else if (kind == 1)
    fma_chain_kernel<float><<<blocks, kThreads, 0, s>>>(0.9999f, 1e-5f, iters, out);
  else
    ffma2_chain_kernel<<<blocks, kThreads, 0, s>>>(0.9999f, 1e-5f, iters, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("hhg_alu_probe: ") + cudaGetErrorString(e));
    return HHG_ERR_CUDA;
  }
  *flops = lanes * (kind == 2 ? 4.0 : 2.0);
  set_error("");
  return HHG_OK;
}
