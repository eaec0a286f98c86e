// J-engine kernels with bra Hermite order 4 (all ket orders 0..6, FP64 and FP32).
#include "dispatch.cuh"
namespace eri {
cudaError_t launch_j_lab4(int LCD, int prec, const JArgs& a, cudaStream_t s, int nsm) {
  return launch_j_lab<4>(LCD, prec, a, s, nsm);
}
}  // namespace eri
