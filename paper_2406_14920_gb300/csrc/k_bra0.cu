// J+K kernels with bra pair class 0 (all ket classes <= 0, FP64 and FP32).
#include "dispatch.cuh"
namespace eri {
cudaError_t launch_jk_bra0(int Y, int prec, const JKArgs& a, cudaStream_t s, int nsm) {
  return launch_jk_x<0>(Y, prec, a, s, nsm);
}
}  // namespace eri
