// One compilation unit of gradient kernels (see units.h): bra class
// ERI_UNIT_X, precision ERI_UNIT_P, every ket class; set on the nvcc command
// line by build.py.
#include "dispatch.cuh"

#if !defined(ERI_UNIT_X) || !defined(ERI_UNIT_P)
#error "g_unit.cu is compiled once per entry of ERI_GRAD_UNITS with -DERI_UNIT_X/_P (see build.py)"
#endif

namespace eri {
template cudaError_t launch_grad_unit<ERI_UNIT_X, ERI_UNIT_P, 0>(int, const GradArgs&, cudaStream_t, int);
}  // namespace eri
