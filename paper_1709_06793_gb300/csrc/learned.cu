// Learned convolutional smoother: forward and backward kernels, training on
// residual/error pairs drawn from the plain multigrid, and the smoothing step
// used inside the V-cycle.
//
// The paper has no learned component.  The network (2 layers of 3x3x3
// convolutions in the (i,j,k) index space of each macro tetrahedron, 2 -> 16
// -> 1 channels, ReLU, no biases) is defined as follows.
//   inputs    a0 = r / D (0 on Dirichlet nodes), a1 = a0 * log k, where r is
//             the residual and D the diagonal of the scaled operator;
//   layer 1   z_c(p) = sum_tau sum_a W1[tau][a][c] a_a(p + tau);  h = max(z, 0)
//   layer 2   ch(p)  = sum_tau sum_c W2[tau][c] h_c(p + tau)
// with values outside the tetrahedron's index set {i+j+k <= N} taken as zero;
// tau = (di,dj,dk) in {-1,0,1}^3 is numbered 9(dk+1) + 3(dj+1) + (di+1).  A
// node shared by several macro tetrahedra takes the mean of their values;
// Dirichlet nodes get 0.  Without biases the network is positively
// homogeneous, so residuals of any size need no normalisation.
//
// Training minimises, over pairs (r, e) with r = A e, the energy norm of the
// error left after the step relative to the error before it:
//   L = (e - c)^T A (e - c) / (e^T r).
// Weights are held as an FP32 master copy; the kernels read them as BF16 (or
// FP32) and accumulate in FP32.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "hhg_internal.h"

namespace hhg {

size_t elem_size(int dtype);
void* workspace(Mesh& m, int depth, int prec, int w);
void dot(Mesh& m, int depth, int dtype, const void* x, const void* y, int slot, int post, bool nc_only, cudaStream_t s);
void residual(Mesh& m, int depth, int dtype, const void* f, const void* u, void* r, bool nc_only, cudaStream_t s);
void vcycle(Mesh& m, int dtype, int nu1, int nu2, int smoother, double omega, const void* f0, void* u0, cudaStream_t s);
void prepare(Mesh& m, int dtype, int smoother, cudaStream_t s);
double pcg_rate(Mesh& m, int dtype, int smoother, int nu1, int nu2, double omega, int its, unsigned long long seed,
                cudaStream_t s);

namespace {

constexpr int kTaps = 27, kIn = 2, kHid = 16;
constexpr int kNW1 = kTaps * kIn * kHid;  // 864
constexpr int kNW2 = kTaps * kHid;        // 432
constexpr int kNW = kNW1 + kNW2;          // 1296
constexpr int kCentre = 13;
constexpr int kT = 8;                     // tile edge (outputs / hidden points)
constexpr int kBF = kT + 4;               // forward input box edge (halo 2)
constexpr int kBH = kT + 2;               // hidden box edge (halo 1)
constexpr int kHS = 20;                   // floats per hidden point in shared memory
constexpr int kThreads = 256;
// device scalar slots used here
constexpr int kSNum = 20, kSDen = 21, kSLoss = 22;

// ---- device helpers ---------------------------------------------------------

__device__ __forceinline__ bool in_set(int N, int i, int j, int k) {
  return i >= 0 && j >= 0 && k >= 0 && i + j + k <= N;
}

__device__ __forceinline__ float wload(const float* w, int q) { return w[q]; }
__device__ __forceinline__ float wload(const __nv_bfloat16* w, int q) { return __bfloat162float(w[q]); }

// offset of tap t in a box of edge B (x fastest)
__host__ __device__ constexpr int tap_off(int t, int B) { return (t % 3 - 1) + B * ((t / 3) % 3 - 1) + B * B * (t / 9 - 1); }

// input channels at one stored node
__device__ __forceinline__ float2 features_at(const float* __restrict__ r, const float2* __restrict__ feat, long long idx) {
  const float2 f = feat[idx];
  const float a0 = r[idx] * f.x;
  return make_float2(a0, a0 * f.y);
}

// ---- forward ----------------------------------------------------------------
// One CTA per 8^3 tile of output nodes (persistent over the tile list).  The
// input channels of the tile plus a halo of 2 go to shared memory, layer 1 is
// evaluated on the tile plus a halo of 1, layer 2 on the tile.
// OUT = 0: out[idx] = ch at every node of the tile (training; interface means
//          are formed afterwards).
// OUT = 1: smoothing step, dst = src + ch at volume nodes and craw = ch at
//          nodes on macro faces/edges/vertices (finished by the interface pass).
constexpr size_t kFwdSmem = (size_t)kNW * 4 + (size_t)kBF * kBF * kBF * 8 + (size_t)kBH * kBH * kBH * kHS * 4;

template <class WT, int OUT>
__global__ void __launch_bounds__(kThreads, 2)
    conv_fwd_kernel(DepthDev D, const int4* __restrict__ tiles, int n_tiles, const WT* __restrict__ w,
                    const float* __restrict__ r, const float2* __restrict__ feat, const float* src, float* dst,
                    float* __restrict__ craw) {
  extern __shared__ __align__(16) float sm[];
  float* W1s = sm;
  float* W2s = sm + kNW1;
  float2* X = reinterpret_cast<float2*>(sm + kNW);
  float* Hs = reinterpret_cast<float*>(X + kBF * kBF * kBF);
  for (int q = threadIdx.x; q < kNW; q += blockDim.x) sm[q] = wload(w, q);
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int4 tl = tiles[tile];
    const TetDev td = D.tets[tl.x];
    const int N = td.N, i0 = tl.y, j0 = tl.z, k0 = tl.w;
    __syncthreads();  // weights loaded / previous tile finished with X and Hs
    for (int q = threadIdx.x; q < kBF * kBF * kBF; q += blockDim.x) {
      const int bi = q % kBF, bj = (q / kBF) % kBF, bk = q / (kBF * kBF);
      const int i = i0 - 2 + bi, j = j0 - 2 + bj, k = k0 - 2 + bk;
      float2 a = make_float2(0.f, 0.f);
      if (in_set(N, i, j, k)) a = features_at(r, feat, td.base + node_offset(N, i, j, k));
      X[q] = a;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kBH * kBH * kBH; q += blockDim.x) {
      const int hi = q % kBH, hj = (q / kBH) % kBH, hk = q / (kBH * kBH);
      float z[kHid];
#pragma unroll
      for (int c = 0; c < kHid; ++c) z[c] = 0.f;
      if (in_set(N, i0 - 1 + hi, j0 - 1 + hj, k0 - 1 + hk)) {
        const int xb = (hi + 1) + kBF * (hj + 1) + kBF * kBF * (hk + 1);
#pragma unroll 3
        for (int t = 0; t < kTaps; ++t) {
          const float2 a = X[xb + tap_off(t, kBF)];
          const float4* w1 = reinterpret_cast<const float4*>(W1s + t * (kIn * kHid));
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            const float4 wa = w1[c4], wb = w1[4 + c4];
            z[4 * c4 + 0] = fmaf(wb.x, a.y, fmaf(wa.x, a.x, z[4 * c4 + 0]));
            z[4 * c4 + 1] = fmaf(wb.y, a.y, fmaf(wa.y, a.x, z[4 * c4 + 1]));
            z[4 * c4 + 2] = fmaf(wb.z, a.y, fmaf(wa.z, a.x, z[4 * c4 + 2]));
            z[4 * c4 + 3] = fmaf(wb.w, a.y, fmaf(wa.w, a.x, z[4 * c4 + 3]));
          }
        }
      }
      float4* hp = reinterpret_cast<float4*>(Hs + q * kHS);
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4)
        hp[c4] = make_float4(fmaxf(z[4 * c4], 0.f), fmaxf(z[4 * c4 + 1], 0.f), fmaxf(z[4 * c4 + 2], 0.f),
                             fmaxf(z[4 * c4 + 3], 0.f));
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kT * kT * kT; q += blockDim.x) {
      const int oi = q % kT, oj = (q / kT) % kT, ok = q / (kT * kT);
      const int i = i0 + oi, j = j0 + oj, k = k0 + ok;
      if (!in_set(N, i, j, k)) continue;
      const int hb = (oi + 1) + kBH * (oj + 1) + kBH * kBH * (ok + 1);
      float acc = 0.f;
#pragma unroll 3
      for (int t = 0; t < kTaps; ++t) {
        const float4* hp = reinterpret_cast<const float4*>(Hs + (hb + tap_off(t, kBH)) * kHS);
        const float4* w2 = reinterpret_cast<const float4*>(W2s + t * kHid);
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
          const float4 hv = hp[c4], wv = w2[c4];
          acc = fmaf(hv.x, wv.x, fmaf(hv.y, wv.y, fmaf(hv.z, wv.z, fmaf(hv.w, wv.w, acc))));
        }
      }
      const long long idx = td.base + node_offset(N, i, j, k);
      if (OUT == 0) {
        dst[idx] = acc;
      } else if (face_mask(N, i, j, k)) {
        craw[idx] = acc;
      } else {
        dst[idx] = src[idx] + acc;
      }
    }
  }
}

// ---- forward on the tensor cores (BF16 weights and activations, FP32 accumulate)
// Same network and tiling as conv_fwd_kernel, evaluated with
// mma.sync.m16n8k16 (bf16 x bf16 -> f32):
//   layer 1  Z[p][c] = sum_k X[p][k] W1[k][c], k = 2 tau + a (54 used of 64):
//            rows = 16 hidden points, A fragments are single 32-bit loads of
//            the packed (a0, a1) pair at point p + tau, W1 lives in registers;
//   layer 2  P[p][tau] = sum_c h[p][c] W2[tau][c]: the FP32 accumulators of
//            layer 1 (after ReLU, rounded to BF16) are exactly the A fragment
//            of this product; 27 taps padded to 32 columns; P is kept in
//            shared memory as BF16 (54 KB instead of 109 KB), so that two
//            blocks of 8 warps share an SM and one block's contractions
//            overlap the other's gathers and input loads;
//   output   ch(x) = sum_tau P[x + tau][tau], gathered from shared memory
//            (FP32 sums, three partial sums over the tap planes).
constexpr int kHP = kBH * kBH * kBH;          // 1000 hidden points
constexpr int kMT = (kHP + 15) / 16;          // 63 row tiles
constexpr int kPS = kTaps;                    // P row stride (odd: conflict-free gather)
constexpr int kTcThreads = 256;
constexpr size_t kTcSmem = (size_t)kBF * kBF * kBF * 4 + (size_t)kMT * 16 * kPS * 2;

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int OUT>
__global__ void __launch_bounds__(kTcThreads, 2)
    conv_fwd_tc_kernel(DepthDev D, const int4* __restrict__ tiles, int n_tiles, const __nv_bfloat16* __restrict__ w,
                       const float* __restrict__ r, const float2* __restrict__ feat, const float* src, float* dst,
                       float* __restrict__ craw) {
  extern __shared__ __align__(16) unsigned char smb[];
  unsigned* X2 = reinterpret_cast<unsigned*>(smb);
  __nv_bfloat16* P = reinterpret_cast<__nv_bfloat16*>(smb + kBF * kBF * kBF * 4);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  auto wv = [&](int q) { return __bfloat162float(w[q]); };
  // B fragments: layer 1 (k-step ks, channel tile nt), layer 2 (tap tile nt)
  unsigned b1[4][2][2], b2[4][2];
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 16 * ks + 2 * t + 8 * h, c = 8 * nt + g;
        const float lo = k < kTaps * kIn ? wv(k * kHid + c) : 0.f;
        const float hi = k + 1 < kTaps * kIn ? wv((k + 1) * kHid + c) : 0.f;
        b1[ks][nt][h] = pack_bf16(lo, hi);
      }
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int tau = 8 * nt + g, c = 2 * t + 8 * h;
      b2[nt][h] = tau < kTaps ? pack_bf16(wv(kNW1 + tau * kHid + c), wv(kNW1 + tau * kHid + c + 1)) : 0u;
    }
  // tap offsets in the input box of the A-fragment columns (taps >= 27 have zero weights)
  int offA[4], offB[4];
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    offA[ks] = tap_off(min(8 * ks + t, kTaps - 1), kBF);
    offB[ks] = tap_off(min(8 * ks + 4 + t, kTaps - 1), kBF);
  }
  // the input box of the next tile is loaded into registers while the
  // current one is computed (kPre points per thread)
  constexpr int kPre = (kBF * kBF * kBF + kTcThreads - 1) / kTcThreads;
  float pr[kPre], pf[kPre], pk[kPre];
  auto prefetch = [&](int tile) {
    const int4 tl = tiles[tile];
    const TetDev td = D.tets[tl.x];
#pragma unroll
    for (int s2 = 0; s2 < kPre; ++s2) {
      const int q = threadIdx.x + s2 * kTcThreads;
      pr[s2] = 0.f;
      pf[s2] = 0.f;
      pk[s2] = 0.f;
      if (q < kBF * kBF * kBF) {
        const int bi = q % kBF, bj = (q / kBF) % kBF, bk = q / (kBF * kBF);
        const int i = tl.y - 2 + bi, j = tl.z - 2 + bj, k = tl.w - 2 + bk;
        if (in_set(td.N, i, j, k)) {
          const long long idx = td.base + node_offset(td.N, i, j, k);
          pr[s2] = r[idx];
          const float2 f = feat[idx];
          pf[s2] = f.x;
          pk[s2] = f.y;
        }
      }
    }
  };
  if (blockIdx.x < n_tiles) prefetch(blockIdx.x);
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int4 tl = tiles[tile];
    const TetDev td = D.tets[tl.x];
    const int N = td.N, i0 = tl.y, j0 = tl.z, k0 = tl.w;
    __syncthreads();  // previous tile finished with X2 and P
#pragma unroll
    for (int s2 = 0; s2 < kPre; ++s2) {
      const int q = threadIdx.x + s2 * kTcThreads;
      if (q < kBF * kBF * kBF) {
        const float a0 = pr[s2] * pf[s2];
        X2[q] = pack_bf16(a0, a0 * pk[s2]);
      }
    }
    __syncthreads();
    if (tile + (int)gridDim.x < n_tiles) prefetch(tile + gridDim.x);
    for (int mt = warp; mt < kMT; mt += nwarps) {
      int xb[2];
      bool ok[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = min(16 * mt + g + 8 * h, kHP - 1);
        const int hi = p % kBH, hj = (p / kBH) % kBH, hk = p / (kBH * kBH);
        xb[h] = (hi + 1) + kBF * (hj + 1) + kBF * kBF * (hk + 1);
        ok[h] = 16 * mt + g + 8 * h < kHP && in_set(N, i0 - 1 + hi, j0 - 1 + hj, k0 - 1 + hk);
      }
      float z[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const unsigned a0 = X2[xb[0] + offA[ks]], a1 = X2[xb[1] + offA[ks]];
        const unsigned a2 = X2[xb[0] + offB[ks]], a3 = X2[xb[1] + offB[ks]];
        mma_bf16(z[0], a0, a1, a2, a3, b1[ks][0][0], b1[ks][0][1]);
        mma_bf16(z[1], a0, a1, a2, a3, b1[ks][1][0], b1[ks][1][1]);
      }
      // h = max(z, 0) on points of the index set, as the A fragment of layer 2
      const float m0 = ok[0] ? 1.f : 0.f, m1 = ok[1] ? 1.f : 0.f;
      const unsigned h0 = pack_bf16(fmaxf(z[0][0], 0.f) * m0, fmaxf(z[0][1], 0.f) * m0);
      const unsigned h1 = pack_bf16(fmaxf(z[0][2], 0.f) * m1, fmaxf(z[0][3], 0.f) * m1);
      const unsigned h2 = pack_bf16(fmaxf(z[1][0], 0.f) * m0, fmaxf(z[1][1], 0.f) * m0);
      const unsigned h3 = pack_bf16(fmaxf(z[1][2], 0.f) * m1, fmaxf(z[1][3], 0.f) * m1);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        float pp[4] = {0.f, 0.f, 0.f, 0.f};
        mma_bf16(pp, h0, h1, h2, h3, b2[nt][0], b2[nt][1]);
        const int tau = 8 * nt + 2 * t;
        const int r0 = (16 * mt + g) * kPS, r1 = (16 * mt + g + 8) * kPS;
        if (tau < kTaps) {
          P[r0 + tau] = __float2bfloat16(pp[0]);
          P[r1 + tau] = __float2bfloat16(pp[2]);
        }
        if (tau + 1 < kTaps) {
          P[r0 + tau + 1] = __float2bfloat16(pp[1]);
          P[r1 + tau + 1] = __float2bfloat16(pp[3]);
        }
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kT * kT * kT; q += blockDim.x) {
      const int oi = q % kT, oj = (q / kT) % kT, ok = q / (kT * kT);
      const int i = i0 + oi, j = j0 + oj, k = k0 + ok;
      if (!in_set(N, i, j, k)) continue;
      const int hb = (oi + 1) + kBH * (oj + 1) + kBH * kBH * (ok + 1);
      float a3[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int tau = 0; tau < kTaps; ++tau) a3[tau / 9] += __bfloat162float(P[(hb + tap_off(tau, kBH)) * kPS + tau]);
      const float acc = a3[0] + a3[1] + a3[2];
      const long long idx = td.base + node_offset(N, i, j, k);
      if (OUT == 0) {
        dst[idx] = acc;
      } else if (face_mask(N, i, j, k)) {
        craw[idx] = acc;
      } else {
        dst[idx] = src[idx] + acc;
      }
    }
  }
}

// ---- interface / Dirichlet pass -------------------------------------------
// mode 0: x <- mean over copies of x (Dirichlet: 0)             (training forward)
// mode 1: x_dst <- x_src + mean over copies of y (Dirichlet: x_src)  (smoothing step)
// mode 2: x <- x(owner) / copies (Dirichlet: 0)                  (gradient of the mean)
// mode 3: x <- x(owner) (Dirichlet: 0)                           (consistent random vectors)
__global__ void bnode_pass_kernel(DepthDev D, int n_b, int mode, float* x, const float* y, const float* xs) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_b; b += gridDim.x * blockDim.x) {
    const int lo = D.bstart[b], hi = D.bstart[b + 1];
    const float inv = 1.f / (float)(hi - lo);
    if (D.bdir[b]) {
      for (int q = lo; q < hi; ++q) {
        const long long idx = D.bcopies[q].idx;
        x[idx] = mode == 1 ? xs[idx] : 0.f;
      }
      continue;
    }
    float v = 0.f;
    if (mode == 0 || mode == 1) {
      const float* in = mode == 0 ? x : y;
      for (int q = lo; q < hi; ++q) v += in[D.bcopies[q].idx];
      v *= inv;
    } else {
      v = x[D.bcopies[lo].idx];
      if (mode == 2) v *= inv;
    }
    for (int q = lo; q < hi; ++q) {
      const long long idx = D.bcopies[q].idx;
      x[idx] = mode == 1 ? xs[idx] + v : v;
    }
  }
}

// ---- backward ---------------------------------------------------------------
// One CTA per 8^3 tile of hidden points y.  With the gradient g of the loss
// with respect to every per-copy output ch:
//   dL/dW2[t][c]    = sum_y g(y - tau_t) h_c(y)
//   dL/dW1[t][a][c] = sum_y gz_c(y) a_a(y + tau_t),
//   gz_c(y) = [z_c(y) > 0] sum_t W2[t][c] g(y - tau_t).
// z is recomputed from the inputs.  Thread (grp = tid/16, c = tid%16) owns the
// weight entries of channel c and taps grp, grp+16; tile sums are FP32, the
// sums over tiles FP64, added into partials[block][entry].
constexpr size_t kBwdSmem = (size_t)kNW * 4 + (size_t)kBH * kBH * kBH * 8 + (size_t)kBH * kBH * kBH * 4 +
                            2 * (size_t)kT * kT * kT * 17 * 4;

template <class WT>
__global__ void __launch_bounds__(kThreads, 2)
    conv_bwd_kernel(DepthDev D, const int4* __restrict__ tiles, int n_tiles, const WT* __restrict__ w,
                    const float* __restrict__ r, const float2* __restrict__ feat, const float* __restrict__ g,
                    double* __restrict__ partials) {
  extern __shared__ __align__(16) float sm[];
  float* W1s = sm;
  float* W2s = sm + kNW1;
  float2* X = reinterpret_cast<float2*>(sm + kNW);
  float* G = reinterpret_cast<float*>(X + kBH * kBH * kBH);
  float* Hs = G + kBH * kBH * kBH;
  float* GZ = Hs + kT * kT * kT * 17;
  for (int q = threadIdx.x; q < kNW; q += blockDim.x) sm[q] = wload(w, q);
  const int c = threadIdx.x & 15, grp = threadIdx.x >> 4;
  const int t0 = grp, t1 = grp + 16;
  const bool has1 = t1 < kTaps;
  const int o0 = tap_off(t0, kBH), o1 = has1 ? tap_off(t1, kBH) : 0;
  double a2[2] = {0, 0}, a1[2][2] = {{0, 0}, {0, 0}};
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int4 tl = tiles[tile];
    const TetDev td = D.tets[tl.x];
    const int N = td.N, i0 = tl.y, j0 = tl.z, k0 = tl.w;
    __syncthreads();
    for (int q = threadIdx.x; q < kBH * kBH * kBH; q += blockDim.x) {
      const int bi = q % kBH, bj = (q / kBH) % kBH, bk = q / (kBH * kBH);
      const int i = i0 - 1 + bi, j = j0 - 1 + bj, k = k0 - 1 + bk;
      float2 a = make_float2(0.f, 0.f);
      float gv = 0.f;
      if (in_set(N, i, j, k)) {
        const long long idx = td.base + node_offset(N, i, j, k);
        a = features_at(r, feat, idx);
        gv = g[idx];
      }
      X[q] = a;
      G[q] = gv;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kT * kT * kT; q += blockDim.x) {
      const int yi = q % kT, yj = (q / kT) % kT, yk = q / (kT * kT);
      float z[kHid], gh[kHid];
#pragma unroll
      for (int cc = 0; cc < kHid; ++cc) z[cc] = gh[cc] = 0.f;
      if (in_set(N, i0 + yi, j0 + yj, k0 + yk)) {
        const int xb = (yi + 1) + kBH * (yj + 1) + kBH * kBH * (yk + 1);
#pragma unroll 3
        for (int t = 0; t < kTaps; ++t) {
          const float2 a = X[xb + tap_off(t, kBH)];
          const float gm = G[xb - tap_off(t, kBH)];
          const float4* w1 = reinterpret_cast<const float4*>(W1s + t * (kIn * kHid));
          const float4* w2 = reinterpret_cast<const float4*>(W2s + t * kHid);
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            const float4 wa = w1[c4], wb = w1[4 + c4], wv = w2[c4];
            z[4 * c4 + 0] = fmaf(wb.x, a.y, fmaf(wa.x, a.x, z[4 * c4 + 0]));
            z[4 * c4 + 1] = fmaf(wb.y, a.y, fmaf(wa.y, a.x, z[4 * c4 + 1]));
            z[4 * c4 + 2] = fmaf(wb.z, a.y, fmaf(wa.z, a.x, z[4 * c4 + 2]));
            z[4 * c4 + 3] = fmaf(wb.w, a.y, fmaf(wa.w, a.x, z[4 * c4 + 3]));
            gh[4 * c4 + 0] = fmaf(wv.x, gm, gh[4 * c4 + 0]);
            gh[4 * c4 + 1] = fmaf(wv.y, gm, gh[4 * c4 + 1]);
            gh[4 * c4 + 2] = fmaf(wv.z, gm, gh[4 * c4 + 2]);
            gh[4 * c4 + 3] = fmaf(wv.w, gm, gh[4 * c4 + 3]);
          }
        }
      }
#pragma unroll
      for (int cc = 0; cc < kHid; ++cc) {
        Hs[q * 17 + cc] = fmaxf(z[cc], 0.f);
        GZ[q * 17 + cc] = z[cc] > 0.f ? gh[cc] : 0.f;
      }
    }
    __syncthreads();
    float f2[2] = {0.f, 0.f}, f1[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int y = 0; y < kT * kT * kT; ++y) {
      const float hv = Hs[y * 17 + c], gz = GZ[y * 17 + c];
      const int yb = (y % kT + 1) + kBH * ((y / kT) % kT + 1) + kBH * kBH * (y / (kT * kT) + 1);
      f2[0] = fmaf(G[yb - o0], hv, f2[0]);
      const float2 x0 = X[yb + o0];
      f1[0][0] = fmaf(x0.x, gz, f1[0][0]);
      f1[0][1] = fmaf(x0.y, gz, f1[0][1]);
      if (has1) {
        f2[1] = fmaf(G[yb - o1], hv, f2[1]);
        const float2 x1 = X[yb + o1];
        f1[1][0] = fmaf(x1.x, gz, f1[1][0]);
        f1[1][1] = fmaf(x1.y, gz, f1[1][1]);
      }
    }
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      a2[s2] += f2[s2];
      a1[s2][0] += f1[s2][0];
      a1[s2][1] += f1[s2][1];
    }
  }
  double* P = partials + (size_t)blockIdx.x * kNW;
  const int ts[2] = {t0, t1};
  for (int s2 = 0; s2 < (has1 ? 2 : 1); ++s2) {
    const int t = ts[s2];
    P[(t * kIn + 0) * kHid + c] += a1[s2][0];
    P[(t * kIn + 1) * kHid + c] += a1[s2][1];
    P[kNW1 + t * kHid + c] += a2[s2];
  }
}

// ---- pointwise kernels --------------------------------------------------------

__host__ __device__ inline unsigned long long mix64(unsigned long long x) {  // SplitMix64 finaliser
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void noise_kernel(float* __restrict__ x, long long n, unsigned long long key) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = (float)((mix64(key ^ mix64((unsigned long long)i)) >> 40) * (1.0 / 16777216.0)) * 2.f - 1.f;
}

// one damped Jacobi sweep from zero: u1 = omega D^-1 r0, e1 = e0 - u1
__global__ void jacobi_pair_kernel(const float* __restrict__ e0, const float* __restrict__ r0,
                                   const float2* __restrict__ feat, float omega, float* __restrict__ u1,
                                   float* __restrict__ e1, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float u = omega * feat[i].x * r0[i];
    u1[i] = u;
    e1[i] = e0[i] - u;
  }
}

__global__ void sub_kernel(const float* a, const float* b, float* out, long long n) {  // out may alias a
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

// g = -2 q / (e.r)
__global__ void grad_out_kernel(const float* __restrict__ q, float* __restrict__ g, long long n, const double* S) {
  const float sc = (float)(-2.0 / S[kSDen]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    g[i] = sc * q[i];
}

__global__ void loss_acc_kernel(double* S) { S[kSLoss] += S[kSNum] / S[kSDen]; }

__global__ void feat_kernel(const double* __restrict__ diag, const double* __restrict__ k, float2* __restrict__ feat,
                            long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    feat[i] = make_float2((float)(1.0 / diag[i]), (float)log(k[i]));
}

__global__ void feat_dirichlet_kernel(DepthDev D, float2* feat) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < D.n_bnodes; b += gridDim.x * blockDim.x)
    if (D.bdir[b])
      for (int q = D.bstart[b]; q < D.bstart[b + 1]; ++q) feat[D.bcopies[q].idx].x = 0.f;
}

// gradient = sum of the per-block partials (fixed order); optional Adam step
// (Kingma & Ba, Adam: A Method for Stochastic Optimization, Alg. 1)
__global__ void adam_kernel(const double* __restrict__ partials, int nblk, double* __restrict__ grad,
                            float* __restrict__ w32, __nv_bfloat16* __restrict__ w16, float* __restrict__ am,
                            float* __restrict__ av, int t, double lr, int update) {
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kNW; e += gridDim.x * blockDim.x) {
    double gs = 0;
    for (int b = 0; b < nblk; ++b) gs += partials[(size_t)b * kNW + e];
    grad[e] = gs;
    if (!update) continue;
    const double mm = b1 * am[e] + (1 - b1) * gs;
    const double vv = b2 * av[e] + (1 - b2) * gs * gs;
    am[e] = (float)mm;
    av[e] = (float)vv;
    const double mh = mm / (1 - pow(b1, t)), vh = vv / (1 - pow(b2, t));
    const float wn = (float)(w32[e] - lr * mh / (sqrt(vh) + eps));
    w32[e] = wn;
    w16[e] = __float2bfloat16_rn(wn);
  }
}

__global__ void w16_from_w32_kernel(const float* __restrict__ w32, __nv_bfloat16* __restrict__ w16) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kNW; e += gridDim.x * blockDim.x)
    w16[e] = __float2bfloat16_rn(w32[e]);
}

inline int grid_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)std::min<long long>(b, cap);
}

// ---- host state ---------------------------------------------------------------

struct LDepth {
  float2* feat = nullptr;  // (1/D, 0 on Dirichlet nodes; log k) per stored node
  int4* tiles = nullptr;   // (slot, i0, j0, k0) of every 8^3 tile meeting an index set
  int n_tiles = 0, n_tiles_nc = 0;
  float* r = nullptr;      // residual of the smoothing step
  float* craw = nullptr;   // per-copy corrections on macro faces, edges and vertices
  // training vectors
  float *e0 = nullptr, *r0 = nullptr, *u1 = nullptr, *e1 = nullptr, *r1 = nullptr;
  float *c = nullptr, *dd = nullptr, *q = nullptr, *g = nullptr;
};

struct Learned {
  std::vector<LDepth> d;
  float* w32 = nullptr;           // FP32 master weights
  __nv_bfloat16* w16 = nullptr;   // BF16 copy read by the kernels in BF16 mode
  float* wj32 = nullptr;          // weights of the Jacobi-equivalent network (validation baseline)
  __nv_bfloat16* wj16 = nullptr;
  float *am = nullptr, *av = nullptr;
  double* partials = nullptr;     // [nblk][1296]
  double* grad = nullptr;         // [1296]
  int nblk = 0;
  bool have_weights = false, bf16 = true, feat_valid = false, accepted = false;
  bool tc = true;       // BF16 forward on the tensor cores (smoothing steps)
  bool tc_all = false;  // also for the exact forward (hhg_learned_forward, training)
  int adam_t = 0;
};

Learned& state(Mesh& m) {
  if (!m.learned) {
    Learned* L = new Learned;
    L->d.resize(m.ndepth);
    m.learned = L;
    Depth& D0 = m.depth[0];
    L->w32 = static_cast<float*>(dalloc(D0, kNW * 4));
    L->w16 = static_cast<__nv_bfloat16*>(dalloc(D0, kNW * 2));
    L->wj32 = static_cast<float*>(dalloc(D0, kNW * 4));
    L->wj16 = static_cast<__nv_bfloat16*>(dalloc(D0, kNW * 2));
    L->am = static_cast<float*>(dalloc(D0, kNW * 4));
    L->av = static_cast<float*>(dalloc(D0, kNW * 4));
    L->nblk = 2 * std::max(m.num_sms, 1);
    L->partials = static_cast<double*>(dalloc(D0, (size_t)L->nblk * kNW * 8));
    L->grad = static_cast<double*>(dalloc(D0, kNW * 8));
  }
  return *static_cast<Learned*>(m.learned);
}

void init_kernels_smem() {
  static bool done = false;
  if (done) return;
  HHG_CUDA(cudaFuncSetAttribute(conv_fwd_kernel<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem));
  HHG_CUDA(cudaFuncSetAttribute(conv_fwd_kernel<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem));
  HHG_CUDA(cudaFuncSetAttribute(conv_fwd_kernel<__nv_bfloat16, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kFwdSmem));
  HHG_CUDA(cudaFuncSetAttribute(conv_fwd_kernel<__nv_bfloat16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kFwdSmem));
  HHG_CUDA(cudaFuncSetAttribute(conv_bwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem));
  HHG_CUDA(cudaFuncSetAttribute(conv_fwd_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
  HHG_CUDA(cudaFuncSetAttribute(conv_fwd_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
  HHG_CUDA(cudaFuncSetAttribute(conv_bwd_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kBwdSmem));
  done = true;
}

void ensure_depth(Mesh& m, Learned& L, int d) {
  LDepth& X = L.d[d];
  if (X.feat) return;
  Depth& D = m.depth[d];
  const size_t n = (size_t)std::max<long long>(D.n_stored, 1);
  X.feat = static_cast<float2*>(dalloc(D, n * 8));
  X.r = static_cast<float*>(dalloc(D, n * 4));
  X.craw = static_cast<float*>(dalloc(D, n * 4));
  HHG_CUDA(cudaMemset(X.craw, 0, n * 4));
  std::vector<int4> tl;
  const int ns = (int)D.h_tets.size();
  for (int s = 0; s < ns; ++s) {
    const int N = D.h_tets[s].N;
    for (int k0 = 0; k0 <= N; k0 += kT)
      for (int j0 = 0; j0 <= N - k0; j0 += kT)
        for (int i0 = 0; i0 <= N - k0 - j0; i0 += kT) tl.push_back(make_int4(s, i0, j0, k0));
    if (s + 1 == D.n_slots_nc) X.n_tiles_nc = (int)tl.size();
  }
  X.n_tiles = (int)tl.size();
  X.tiles = static_cast<int4*>(dalloc(D, std::max<size_t>(tl.size(), 1) * sizeof(int4)));
  if (!tl.empty()) HHG_CUDA(cudaMemcpy(X.tiles, tl.data(), tl.size() * sizeof(int4), cudaMemcpyHostToDevice));
}

void ensure_train(Mesh& m, Learned& L, int d) {
  ensure_depth(m, L, d);
  LDepth& X = L.d[d];
  if (X.e0) return;
  Depth& D = m.depth[d];
  const size_t n = (size_t)std::max<long long>(D.n_stored, 1) * 4;
  float** v[] = {&X.e0, &X.r0, &X.u1, &X.e1, &X.r1, &X.c, &X.dd, &X.q, &X.g};
  for (float** p : v) {
    *p = static_cast<float*>(dalloc(D, n));
    HHG_CUDA(cudaMemset(*p, 0, n));
  }
}

void compute_features(Mesh& m, Learned& L, int d, cudaStream_t s) {
  Depth& D = m.depth[d];
  LDepth& X = L.d[d];
  if (D.n_stored == 0) return;
  double* diag = static_cast<double*>(workspace(m, d, 0, 4));
  double* zero = static_cast<double*>(workspace(m, d, 0, 5));
  HHG_CUDA(cudaMemsetAsync(zero, 0, D.n_stored * 8, s));
  OpArgs a{zero, nullptr, diag, nullptr, nullptr, 0, 0, 0, 0};
  launch_scaled_op(m, d, HHG_F64, OP_DIAG, a, s);
  feat_kernel<<<grid_for(D.n_stored, 256, 4096), 256, 0, s>>>(diag, D.k64, X.feat, D.n_stored);
  if (D.n_bnodes) feat_dirichlet_kernel<<<grid_for(D.n_bnodes, 128, 1024), 128, 0, s>>>(D.dev, X.feat);
  HHG_CUDA(cudaGetLastError());
}

bool smoothed(const Mesh& m, int d) { return d + 1 < m.ndepth && m.depth[d].n_slots_nc > 0; }

void ensure_features(Mesh& m, Learned& L, cudaStream_t s) {
  init_kernels_smem();
  for (int d = 0; d < m.ndepth; ++d)
    if (smoothed(m, d)) ensure_depth(m, L, d);
  if (L.feat_valid) return;
  for (int d = 0; d < m.ndepth; ++d)
    if (smoothed(m, d)) compute_features(m, L, d, s);
  L.feat_valid = true;
}

// ---- launches ---------------------------------------------------------------

template <int OUT>
void launch_fwd(Mesh& m, Learned& L, int d, const float* r, const float* src, float* dst, float* craw, bool nc_only,
                cudaStream_t s) {
  LDepth& X = L.d[d];
  const int nt = nc_only ? X.n_tiles_nc : X.n_tiles;
  if (nt == 0) return;
  const int g = std::min(nt, L.nblk);
  const DepthDev& DD = m.depth[d].dev;
  if (L.bf16 && (OUT == 1 ? L.tc : L.tc_all))
    conv_fwd_tc_kernel<OUT><<<std::min(nt, 2 * std::max(m.num_sms, 1)), kTcThreads, kTcSmem, s>>>(DD, X.tiles, nt, L.w16, r,
                                                                                              X.feat, src, dst, craw);
  else if (L.bf16)
    conv_fwd_kernel<__nv_bfloat16, OUT><<<g, kThreads, kFwdSmem, s>>>(DD, X.tiles, nt, L.w16, r, X.feat, src, dst, craw);
  else
    conv_fwd_kernel<float, OUT><<<g, kThreads, kFwdSmem, s>>>(DD, X.tiles, nt, L.w32, r, X.feat, src, dst, craw);
  HHG_CUDA(cudaGetLastError());
}

void bnode_pass(Mesh& m, int d, int mode, float* x, const float* y, const float* xs, bool nc_only, cudaStream_t s) {
  const Depth& D = m.depth[d];
  const int nb = nc_only ? D.n_bnodes_nc : D.n_bnodes;
  if (nb == 0) return;
  bnode_pass_kernel<<<grid_for(nb, 128, 4096), 128, 0, s>>>(D.dev, nb, mode, x, y, xs);
  HHG_CUDA(cudaGetLastError());
}

long long nvec(const Mesh& m, int d, bool nc_only) {
  return nc_only ? m.depth[d].n_stored_nc : m.depth[d].n_stored;
}

// c = N(r) (consistent, 0 on Dirichlet nodes)
void forward_consistent(Mesh& m, Learned& L, int d, const float* r, float* c, bool nc_only, cudaStream_t s) {
  launch_fwd<0>(m, L, d, r, nullptr, c, nullptr, nc_only, s);
  bnode_pass(m, d, 0, c, nullptr, nullptr, nc_only, s);
}

void apply_f32(Mesh& m, int d, const float* u, float* y, bool nc_only, cudaStream_t s) {
  OpArgs a{u, nullptr, y, nullptr, nullptr, 0, 0, 0, nc_only ? 1 : 0};
  launch_scaled_op(m, d, HHG_F32, OP_APPLY, a, s);
}

// loss of one pair (added to S[kSLoss]); with grad, its weight gradient is
// added to the partials
void pair_loss(Mesh& m, Learned& L, int d, const float* r, const float* e, bool grad, cudaStream_t s) {
  LDepth& X = L.d[d];
  const bool nc = true;
  const long long n = nvec(m, d, nc);
  const int gv = grid_for(n, 256, 8 * m.num_sms);
  forward_consistent(m, L, d, r, X.c, nc, s);
  sub_kernel<<<gv, 256, 0, s>>>(e, X.c, X.dd, n);
  HHG_CUDA(cudaGetLastError());
  apply_f32(m, d, X.dd, X.q, nc, s);
  dot(m, d, HHG_F32, X.dd, X.q, kSNum, 0, nc, s);
  dot(m, d, HHG_F32, e, r, kSDen, 0, nc, s);
  loss_acc_kernel<<<1, 1, 0, s>>>(m.d_scalars);
  HHG_CUDA(cudaGetLastError());
  if (!grad) return;
  grad_out_kernel<<<gv, 256, 0, s>>>(X.q, X.g, n, m.d_scalars);
  HHG_CUDA(cudaGetLastError());
  bnode_pass(m, d, 2, X.g, nullptr, nullptr, nc, s);
  const int nt = X.n_tiles_nc;
  const DepthDev& DD = m.depth[d].dev;
  if (L.bf16)
    conv_bwd_kernel<__nv_bfloat16><<<L.nblk, kThreads, kBwdSmem, s>>>(DD, X.tiles, nt, L.w16, r, X.feat, X.g,
                                                                       L.partials);
  else
    conv_bwd_kernel<float><<<L.nblk, kThreads, kBwdSmem, s>>>(DD, X.tiles, nt, L.w32, r, X.feat, X.g, L.partials);
  HHG_CUDA(cudaGetLastError());
}

}  // namespace

// ---- entry points used by the solver and the ABI ------------------------------

void free_learned(Mesh* m) {
  delete static_cast<Learned*>(m->learned);  // device memory belongs to the depths
  m->learned = nullptr;
}

void learned_invalidate(Mesh& m) {
  if (m.learned) static_cast<Learned*>(m.learned)->feat_valid = false;
}

void learned_prepare(Mesh& m, int dtype, cudaStream_t s) {
  HHG_REQUIRE(dtype == HHG_F32 || dtype == HHG_F32_KBF16,
              "the learned smoother runs on FP32 vectors (HHG_F32 or HHG_F32_KBF16)");
  if (!m.learned || !state(m).have_weights)
    throw Error{HHG_ERR_STATE, "learned smoother has no weights: call hhg_learned_train or hhg_learned_set_weights"};
  ensure_features(m, state(m), s);
}

// dst = src + N(f - A src) on the tetrahedra above the coarsest level (src == dst allowed)
void learned_step(Mesh& m, int d, int dtype, const void* f, const void* src, void* dst, bool nc_only, cudaStream_t s) {
  Learned& L = state(m);
  LDepth& X = L.d[d];
  residual(m, d, dtype, f, src, X.r, nc_only, s);
  launch_fwd<1>(m, L, d, X.r, static_cast<const float*>(src), static_cast<float*>(dst), X.craw, nc_only, s);
  bnode_pass(m, d, 1, static_cast<float*>(dst), X.craw, static_cast<const float*>(src), nc_only, s);
}

// consistent uniform[-1,1] vector (0 on Dirichlet nodes) at depth d
void random_vector(Mesh& m, int d, float* x, unsigned long long key, cudaStream_t s) {
  const long long n = m.depth[d].n_stored;
  if (n == 0) return;
  noise_kernel<<<grid_for(n, 256, 8 * m.num_sms), 256, 0, s>>>(x, n, key);
  HHG_CUDA(cudaGetLastError());
  bnode_pass(m, d, 3, x, nullptr, nullptr, false, s);
}

void learned_set_weights(Mesh& m, const float* w_host, int bf16, cudaStream_t s) {
  Learned& L = state(m);
  HHG_CUDA(cudaMemcpyAsync(L.w32, w_host, kNW * 4, cudaMemcpyHostToDevice, s));
  w16_from_w32_kernel<<<grid_for(kNW, 256, 8), 256, 0, s>>>(L.w32, L.w16);
  HHG_CUDA(cudaGetLastError());
  HHG_CUDA(cudaStreamSynchronize(s));
  L.bf16 = bf16 != 0;
  L.have_weights = true;
  L.accepted = true;
  L.adam_t = 0;
  drop_graphs(m);
}

void learned_get_weights(Mesh& m, float* w_host, cudaStream_t s) {
  Learned& L = state(m);
  HHG_REQUIRE(L.have_weights, "learned smoother has no weights");
  HHG_CUDA(cudaMemcpyAsync(w_host, L.w32, kNW * 4, cudaMemcpyDeviceToHost, s));
  HHG_CUDA(cudaStreamSynchronize(s));
}

// "learned_tc": BF16 smoothing steps on the tensor cores (1, default) or the
// FP32-activation kernel (0); "learned_tc_all": the same for hhg_learned_forward
// and the training forward (default 0).
bool learned_option(Mesh& m, const std::string& key, double* value, bool set) {
  if (key != "learned_tc" && key != "learned_tc_all") return false;
  if (!m.device) throw Error{HHG_ERR_STATE, "mesh was created host-only"};
  Learned& L = state(m);
  bool& f = key == "learned_tc" ? L.tc : L.tc_all;
  if (set) {
    if (*value != 0.0 && *value != 1.0) throw Error{HHG_ERR_ARG, key + " must be 0 or 1"};
    f = *value != 0.0;
    drop_graphs(m);
  } else {
    *value = f ? 1.0 : 0.0;
  }
  return true;
}

bool learned_accepted(Mesh& m) { return m.learned && state(m).have_weights && state(m).accepted; }

void learned_forward(Mesh& m, int d, const float* r, float* c, cudaStream_t s) {
  HHG_REQUIRE(smoothed(m, d), "depth is not smoothed (coarsest depth or out of range)");
  learned_prepare(m, HHG_F32, s);
  forward_consistent(m, state(m), d, r, c, true, s);
}

void learned_loss_grad(Mesh& m, int d, const float* r, const float* e, double* loss, double* grad_host,
                       cudaStream_t s) {
  HHG_REQUIRE(smoothed(m, d), "depth is not smoothed (coarsest depth or out of range)");
  learned_prepare(m, HHG_F32, s);
  Learned& L = state(m);
  ensure_train(m, L, d);
  HHG_CUDA(cudaMemsetAsync(L.partials, 0, (size_t)L.nblk * kNW * 8, s));
  HHG_CUDA(cudaMemsetAsync(m.d_scalars + kSLoss, 0, 8, s));
  pair_loss(m, L, d, r, e, true, s);
  adam_kernel<<<grid_for(kNW, 256, 8), 256, 0, s>>>(L.partials, L.nblk, L.grad, L.w32, L.w16, L.am, L.av, 1, 0.0, 0);
  HHG_CUDA(cudaGetLastError());
  HHG_CUDA(cudaMemcpyAsync(m.h_pinned, m.d_scalars + kSLoss, 8, cudaMemcpyDeviceToHost, s));
  if (grad_host) HHG_CUDA(cudaMemcpyAsync(grad_host, L.grad, kNW * 8, cudaMemcpyDeviceToHost, s));
  HHG_CUDA(cudaStreamSynchronize(s));
  if (loss) *loss = m.h_pinned[0];
}

// ---- training -------------------------------------------------------------------

namespace {

// Pair (r1, e1) at depth d: a random error e0 (or, with vc, the error left by
// one plain V-cycle applied to A e0 = b from zero), then the damped Jacobi
// sweep that precedes the learned step in the V-cycle: u1 = omega D^-1 A e0,
// e1 = e0 - u1, r1 = A e1.
void make_pair(Mesh& m, Learned& L, int d, bool vc, double omega, unsigned long long key, cudaStream_t s) {
  LDepth& X = L.d[d];
  const long long n = m.depth[d].n_stored;
  const int gv = grid_for(n, 256, 8 * m.num_sms);
  random_vector(m, d, X.e0, key, s);
  if (vc && d == 0) {
    apply_f32(m, 0, X.e0, X.r0, false, s);
    HHG_CUDA(cudaMemsetAsync(X.u1, 0, n * 4, s));
    vcycle(m, HHG_F32, 2, 2, HHG_SMOOTH_JACOBI, omega, X.r0, X.u1, s);
    sub_kernel<<<gv, 256, 0, s>>>(X.e0, X.u1, X.e0, n);
    HHG_CUDA(cudaGetLastError());
  }
  apply_f32(m, d, X.e0, X.r0, true, s);
  jacobi_pair_kernel<<<gv, 256, 0, s>>>(X.e0, X.r0, X.feat, (float)omega, X.u1, X.e1, n);
  HHG_CUDA(cudaGetLastError());
  residual(m, d, HHG_F32, X.r0, X.u1, X.r1, true, s);
}

double read_loss(Mesh& m, cudaStream_t s) {
  HHG_CUDA(cudaMemcpyAsync(m.h_pinned, m.d_scalars + kSLoss, 8, cudaMemcpyDeviceToHost, s));
  HHG_CUDA(cudaStreamSynchronize(s));
  return m.h_pinned[0];
}

}  // namespace

void learned_train(Mesh& m, const hhg_learn_params& pin, hhg_learn_stats* st, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  hhg_learn_params p = pin;
  if (p.steps <= 0) p.steps = 150;
  if (p.pairs <= 0) p.pairs = 4;
  if (p.lr <= 0) p.lr = 3e-3;
  if (p.omega <= 0) p.omega = 2.0 / 3.0;
  if (p.max_depth < 0) p.max_depth = 0;
  if (p.vcycle_pairs < 0) p.vcycle_pairs = 0;
  if (p.vcycle_pairs > p.pairs) p.vcycle_pairs = p.pairs;
  if (p.init_noise < 0) p.init_noise = 0;
  if (p.validate_its <= 0) p.validate_its = 8;
  HHG_REQUIRE(m.device && m.coef_set, "hhg_set_coefficient must be called first");
  prepare(m, HHG_F32, HHG_SMOOTH_JACOBI, s);
  Learned& L = state(m);
  std::vector<int> depths;
  for (int d = 0; d <= std::min(p.max_depth, m.ndepth - 1); ++d)
    if (smoothed(m, d)) depths.push_back(d);
  HHG_REQUIRE(!depths.empty(), "the mesh has no smoothed depth to train on");
  for (int d : depths) ensure_train(m, L, d);
  // the network equal to damped Jacobi, and the initial weights (that network
  // plus uniform noise on every other entry)
  std::vector<float> wj(kNW, 0.f), w(kNW);
  const int jac[4] = {(kCentre * kIn + 0) * kHid + 0, (kCentre * kIn + 0) * kHid + 1, kNW1 + kCentre * kHid + 0,
                      kNW1 + kCentre * kHid + 1};
  wj[jac[0]] = 1.f;
  wj[jac[1]] = -1.f;
  wj[jac[2]] = (float)p.omega;
  wj[jac[3]] = (float)-p.omega;
  for (int e = 0; e < kNW; ++e) {
    const bool fixed = e == jac[0] || e == jac[1] || e == jac[2] || e == jac[3];
    const double u = (double)(mix64(p.seed ^ mix64(0x5EED0000ull + (unsigned long long)e)) >> 11) * (1.0 / 9007199254740992.0);
    w[e] = fixed ? wj[e] : (float)(p.init_noise * (2 * u - 1));
  }
  HHG_CUDA(cudaMemcpyAsync(L.wj32, wj.data(), kNW * 4, cudaMemcpyHostToDevice, s));
  w16_from_w32_kernel<<<grid_for(kNW, 256, 8), 256, 0, s>>>(L.wj32, L.wj16);
  if (!(p.resume && L.have_weights)) {
    HHG_CUDA(cudaMemcpyAsync(L.w32, w.data(), kNW * 4, cudaMemcpyHostToDevice, s));
    w16_from_w32_kernel<<<grid_for(kNW, 256, 8), 256, 0, s>>>(L.w32, L.w16);
    HHG_CUDA(cudaMemsetAsync(L.am, 0, kNW * 4, s));
    HHG_CUDA(cudaMemsetAsync(L.av, 0, kNW * 4, s));
    L.adam_t = 0;
  }
  HHG_CUDA(cudaGetLastError());
  L.bf16 = p.weights_bf16 != 0;
  L.have_weights = true;
  drop_graphs(m);
  ensure_features(m, L, s);

  const int nval = 2 + 2 * (int)depths.size();
  auto val_loss = [&](bool jacobi_net) {
    if (jacobi_net) {
      std::swap(L.w32, L.wj32);
      std::swap(L.w16, L.wj16);
    }
    HHG_CUDA(cudaMemsetAsync(m.d_scalars + kSLoss, 0, 8, s));
    for (int v = 0; v < nval; ++v) {
      const bool vc = v < 2;
      const int d = vc ? 0 : depths[(v - 2) % depths.size()];
      make_pair(m, L, d, vc && d == 0, p.omega, mix64(p.seed ^ 0xDA7A5E7000000000ull ^ (unsigned long long)v), s);
      pair_loss(m, L, d, L.d[d].r1, L.d[d].e1, false, s);
    }
    const double l = read_loss(m, s) / nval;
    if (jacobi_net) {
      std::swap(L.w32, L.wj32);
      std::swap(L.w16, L.wj16);
    }
    return l;
  };
  const double loss_jacobi = val_loss(true);
  const double loss_init = val_loss(false);
  for (int step = 0; step < p.steps; ++step) {
    HHG_CUDA(cudaMemsetAsync(L.partials, 0, (size_t)L.nblk * kNW * 8, s));
    for (int q = 0; q < p.pairs; ++q) {
      const bool vc = q < p.vcycle_pairs;
      const int d = vc ? 0 : depths[(q - p.vcycle_pairs + step) % depths.size()];
      const unsigned long long key = mix64(p.seed ^ mix64(((unsigned long long)step << 20) | (unsigned long long)q));
      make_pair(m, L, d, vc && d == 0, p.omega, key, s);
      pair_loss(m, L, d, L.d[d].r1, L.d[d].e1, true, s);
    }
    ++L.adam_t;
    adam_kernel<<<grid_for(kNW, 256, 8), 256, 0, s>>>(L.partials, L.nblk, L.grad, L.w32, L.w16, L.am, L.av, L.adam_t,
                                                       p.lr, 1);
    HHG_CUDA(cudaGetLastError());
  }
  const double loss_final = val_loss(false);
  // the plain V-cycle judges the learned one: PCG convergence factor of both
  L.accepted = true;
  const unsigned long long vkey = mix64(p.seed ^ 0x7E57000000000000ull);
  const double rho_plain = pcg_rate(m, HHG_F32, HHG_SMOOTH_JACOBI, 2, 2, p.omega, p.validate_its, vkey, s);
  const double rho_learned = pcg_rate(m, HHG_F32, HHG_SMOOTH_LEARNED, 2, 2, p.omega, p.validate_its, vkey, s);
  L.accepted = rho_learned < rho_plain;
  drop_graphs(m);
  HHG_CUDA(cudaStreamSynchronize(s));
  if (st) {
    st->loss_jacobi = loss_jacobi;
    st->loss_init = loss_init;
    st->loss_final = loss_final;
    st->rho_plain = rho_plain;
    st->rho_learned = rho_learned;
    st->accepted = L.accepted ? 1 : 0;
    st->steps = p.steps;
    st->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
}

}  // namespace hhg
