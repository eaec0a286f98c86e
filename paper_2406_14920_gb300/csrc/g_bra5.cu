// Gradient kernels with bra pair class 5 (all ket classes, FP64).
#include "dispatch.cuh"
namespace eri {
cudaError_t launch_grad_bra5(int Y, const GradArgs& a, cudaStream_t s, int nsm) {
  return launch_grad_x<5>(Y, a, s, nsm);
}
}  // namespace eri
