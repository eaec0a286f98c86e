// J+K kernels with bra pair class 1 (all ket classes <= 1, FP64 and FP32).
#include "dispatch.cuh"
namespace eri {
cudaError_t launch_jk_bra1(int Y, int prec, const JKArgs& a, cudaStream_t s, int nsm) {
  return launch_jk_x<1>(Y, prec, a, s, nsm);
}
}  // namespace eri
