// Exchange kernels with bra pair class 8 (all ket classes <= 8, FP64 and FP32).
#include "dispatch.cuh"
namespace eri {
cudaError_t launch_k_bra8(int Y, int prec, const KArgs& a, cudaStream_t s, int nsm) {
  return launch_k_x<8>(Y, prec, a, s, nsm);
}
}  // namespace eri
