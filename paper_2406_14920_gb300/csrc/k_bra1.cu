// Exchange kernels with bra pair class 1 (all ket classes <= 1, FP64 and FP32).
#include "dispatch.cuh"
namespace eri {
cudaError_t launch_k_bra1(int Y, int prec, const KArgs& a, cudaStream_t s, int nsm) {
  return launch_k_x<1>(Y, prec, a, s, nsm);
}
}  // namespace eri
