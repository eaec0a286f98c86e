// Gradient kernels with bra pair class 0 (all ket classes, FP64).
#include "dispatch.cuh"
namespace eri {
cudaError_t launch_grad_bra0(int Y, const GradArgs& a, cudaStream_t s, int nsm) {
  return launch_grad_x<0>(Y, a, s, nsm);
}
}  // namespace eri
