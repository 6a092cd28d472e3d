// Learned smoother (placeholder until its kernels land).
#include "hhg_internal.h"

namespace hhg {
void learned_prepare(Mesh& m, int dtype, cudaStream_t s) {
  (void)m; (void)dtype; (void)s;
  throw Error{HHG_ERR_STATE, "learned smoother not trained"};
}
void free_learned(Mesh* m) { (void)m; }
}  // namespace hhg
