// Exchange kernels with bra pair class 6 (all ket classes <= 6, FP64 and FP32).
#include "dispatch.cuh"
namespace eri {
cudaError_t launch_k_bra6(int Y, int prec, const KArgs& a, cudaStream_t s, int nsm) {
  return launch_k_x<6>(Y, prec, a, s, nsm);
}
}  // namespace eri
