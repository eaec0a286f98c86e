// J+K kernels with bra pair class 2 (all ket classes <= 2, FP64 and FP32).
#include "dispatch.cuh"
namespace eri {
cudaError_t launch_jk_bra2(int Y, int prec, const JKArgs& a, cudaStream_t s, int nsm) {
  return launch_jk_x<2>(Y, prec, a, s, nsm);
}
}  // namespace eri
