// Gradient kernels with bra pair class 8 (all ket classes, FP64).
#include "dispatch.cuh"
namespace eri {
cudaError_t launch_grad_bra8(int Y, const GradArgs& a, cudaStream_t s, int nsm) {
  return launch_grad_x<8>(Y, a, s, nsm);
}
}  // namespace eri
