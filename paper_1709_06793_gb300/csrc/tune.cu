// Autotuner for the volume work: every (volume kernel, kseg, korder) candidate is timed
// on the finest depth with CUDA events (median of repeated applies, the
// better of two passes, after the clocks have been brought up); the best
// is kept on the mesh and, if a cache file is given, recorded there keyed by
// the mesh shape and dtype so later runs skip the search.
#include <algorithm>
#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>

#include "hhg_internal.h"

namespace hhg {

void* workspace(Mesh& m, int depth, int prec, int w);
void apply_scaled(Mesh& m, int depth, int dtype, const void* u, void* y, cudaStream_t s);
void init_launch_configs(int dtype);
size_t elem_size(int dtype);

static std::string tune_key(const Mesh& m, int dtype) {
  std::ostringstream k;
  k << "dtype=" << dtype << ";tets=" << m.nt << ";levels=";
  for (int t = 0; t < m.nt; ++t) k << m.level[t] << (t + 1 < m.nt ? "," : "");
  return k.str();
}

// cache file: one line per entry, "<key> <kseg> <korder> <vkernel> <ms>"
static bool cache_lookup(const char* path, const std::string& key, int& kseg, int& korder, int& vkernel) {
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string k;
    int a, b, c;
    if (is >> k >> a >> b >> c && k == key) {
      kseg = a;
      korder = b;
      vkernel = c;
      return true;
    }
  }
  return false;
}

static void cache_store(const char* path, const std::string& key, int kseg, int korder, int vkernel, double ms) {
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << " " << kseg << " " << korder << " " << vkernel << " " << ms << "\n";
}

void autotune(Mesh& m, int dtype, const char* cache, int* out_kseg, int* out_korder, double* out_ms, cudaStream_t s) {
  HHG_REQUIRE(m.coef_set, "hhg_set_coefficient must be called first");
  const std::string key = tune_key(m, dtype);
  int kseg = m.kseg, korder = m.korder, vkernel = m.vkernel;
  double best_ms = -1;
  if (!cache_lookup(cache, key, kseg, korder, vkernel)) {
    init_launch_configs(dtype);
    const int pr = elem_size(dtype) == 8 ? 0 : 1;
    void* u = workspace(m, 0, pr, 0);
    void* y = workspace(m, 0, pr, 1);
    cudaEvent_t e0, e1;
    HHG_CUDA(cudaEventCreate(&e0));
    HHG_CUDA(cudaEventCreate(&e1));
    const int cand_kseg[] = {16, 32, 64};
    const int cand_order[] = {0, 1};
    auto timed_median = [&](int reps) {
      std::vector<float> t;
      for (int r = 0; r < reps; ++r) {
        HHG_CUDA(cudaEventRecord(e0, s));
        apply_scaled(m, 0, dtype, u, y, s);
        HHG_CUDA(cudaEventRecord(e1, s));
        HHG_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        HHG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        t.push_back(ms);
      }
      std::sort(t.begin(), t.end());
      return (double)t[t.size() / 2];
    };
    // bring the SM clocks up first (about 200 ms of applies): candidates
    // timed on an idle GPU's ramping clock would look slower than they are
    const double one = timed_median(3);
    const int warm = std::min(2000, std::max(10, (int)(200.0 / std::max(one, 1e-3))));
    for (int w = 0; w < warm; ++w) apply_scaled(m, 0, dtype, u, y, s);
    // two passes over the candidates (volume kernel x segmentation x order),
    // each candidate's better pass counts
    // volume kernels: tile march, column march, and for FP32 the column
    // march with two column sets per lane
    const int n_vk = elem_size(dtype) == 8 ? 2 : 3;
    double cand_ms[3][2][3];
    for (int pass = 0; pass < 2; ++pass)
      for (int vk = 0; vk < n_vk; ++vk)
        for (int oi = 0; oi < 2; ++oi)
          for (int ki = 0; ki < 3; ++ki) {
            m.vkernel = vk;
            set_kseg(m, cand_kseg[ki], cand_order[oi]);
            for (int w = 0; w < 2; ++w) apply_scaled(m, 0, dtype, u, y, s);
            const double med = timed_median(5);
            cand_ms[vk][oi][ki] = pass == 0 ? med : std::min(cand_ms[vk][oi][ki], med);
          }
    for (int vk = 0; vk < n_vk; ++vk)
      for (int oi = 0; oi < 2; ++oi)
        for (int ki = 0; ki < 3; ++ki)
          if (best_ms < 0 || cand_ms[vk][oi][ki] < best_ms) {
            best_ms = cand_ms[vk][oi][ki];
            kseg = cand_kseg[ki];
            korder = cand_order[oi];
            vkernel = vk;
          }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cache_store(cache, key, kseg, korder, vkernel, best_ms);
  }
  m.vkernel = vkernel;
  set_kseg(m, kseg, korder);
  if (out_kseg) *out_kseg = kseg;
  if (out_korder) *out_korder = korder;
  if (out_ms) *out_ms = best_ms;
}

}  // namespace hhg
