// One compilation unit of J/K class kernels (see units.h): bra class
// ERI_UNIT_X, precision ERI_UNIT_P, ket classes ERI_UNIT_YLO..ERI_UNIT_YHI,
// set on the nvcc command line by build.py.
#include "dispatch.cuh"

#if !defined(ERI_UNIT_X) || !defined(ERI_UNIT_P) || !defined(ERI_UNIT_YLO) || !defined(ERI_UNIT_YHI)
#error "k_unit.cu is compiled once per entry of units.h with -DERI_UNIT_X/_P/_YLO/_YHI (see build.py)"
#endif

namespace eri {
template cudaError_t launch_jk_unit<ERI_UNIT_X, ERI_UNIT_P, ERI_UNIT_YLO, ERI_UNIT_YHI>(int, const JKArgs&,
                                                                                      cudaStream_t, int);
}  // namespace eri
