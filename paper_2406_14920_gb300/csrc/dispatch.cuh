// Launch helpers for the class-specialised kernels.  Each bra class gets its own
// translation unit (k_bra<X>.cu, j_lab<N>.cu) so that the build compiles them
// in parallel.
#pragma once
#include <algorithm>
#include <type_traits>
#include "kernels_g.cuh"
#include "units.h"

namespace eri {

template <int X> struct ClassL;
template <> struct ClassL<0> { static constexpr int l1 = 0, l2 = 0; };
template <> struct ClassL<1> { static constexpr int l1 = 1, l2 = 0; };
template <> struct ClassL<2> { static constexpr int l1 = 1, l2 = 1; };
template <> struct ClassL<3> { static constexpr int l1 = 2, l2 = 0; };
template <> struct ClassL<4> { static constexpr int l1 = 2, l2 = 1; };
template <> struct ClassL<5> { static constexpr int l1 = 2, l2 = 2; };
template <> struct ClassL<6> { static constexpr int l1 = 3, l2 = 0; };
template <> struct ClassL<7> { static constexpr int l1 = 3, l2 = 1; };
template <> struct ClassL<8> { static constexpr int l1 = 3, l2 = 2; };
template <> struct ClassL<9> { static constexpr int l1 = 3, l2 = 3; };

struct LaunchInfo {
  int grid, block;
  size_t smem;
};

template <typename Kern>
inline cudaError_t launch_persistent(Kern kern, size_t smem, int64_t items, int warps_per_block, int nsm,
                                     LaunchInfo* info) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * warps_per_block, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  int64_t need = (items + warps_per_block - 1) / warps_per_block;
  int64_t grid = std::min<int64_t>(need, (int64_t)nsm * occ);
  if (grid < 1) grid = 1;
  info->grid = (int)grid;
  info->block = 32 * warps_per_block;
  info->smem = smem;
  return cudaSuccess;
}

template <int LA, int LB, int LC, int LD, typename T>
cudaError_t launch_jk_t(const JKArgs& a, cudaStream_t s, int nsm) {
  if (a.k.wl.total <= 0) return cudaSuccess;
  LaunchInfo li;
  if constexpr (use_thread_kernel(LA, LB, LC, LD, sizeof(T) == 4)) {
    auto kern = jk_thread_kernel<LA, LB, LC, LD, T>;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, 0);
    if (e != cudaSuccess) return e;
    int64_t need = (a.k.wl.total + 127) / 128;
    int64_t grid = std::min<int64_t>(need, (int64_t)nsm * std::max(occ, 1));
    kern<<<(int)grid, 128, 0, s>>>(a);
  } else {
    using S = BShape<LA, LB, LC, LD, T>;
    constexpr int WPB = 4;
    static_assert(S::table_bytes() + WPB * S::smem_per_warp() <= 227 * 1024, "warp kernel block exceeds 227 KB");
    auto kern = jk_warp_kernel<LA, LB, LC, LD, T>;
    cudaError_t e = launch_persistent(kern, S::table_bytes() + WPB * S::smem_per_warp(), a.k.wl.total, WPB, nsm, &li);
    if (e != cudaSuccess) return e;
    kern<<<li.grid, li.block, li.smem, s>>>(a);
  }
  return cudaGetLastError();
}

// Launch of class pair (X, y) in precision P for y in YLO..YHI (compile-time
// chain of the ket classes of one compilation unit, see units.h)
template <int X, int P, int YLO, int YHI>
cudaError_t launch_jk_unit(int y, const JKArgs& a, cudaStream_t s, int nsm) {
  if constexpr (YLO > YHI || YLO > X) {
    return cudaErrorInvalidValue;
  } else {
    if (y == YLO) {
      constexpr int LA = ClassL<X>::l1, LB = ClassL<X>::l2, LC = ClassL<YLO>::l1, LD = ClassL<YLO>::l2;
      using T = std::conditional_t<P == 1, float, double>;
      return launch_jk_t<LA, LB, LC, LD, T>(a, s, nsm);
    }
    return launch_jk_unit<X, P, YLO + 1, YHI>(y, a, s, nsm);
  }
}

// Gradient launch of class pair (X, y) in precision P, y in 0..9 (compile-time
// chain; one compilation unit per (X, P), see units.h)
template <int X, int P, int Y = 0>
cudaError_t launch_grad_unit(int y, const GradArgs& a, cudaStream_t s, int nsm) {
  if constexpr (Y >= NPAIRCLASS) {
    return cudaErrorInvalidValue;
  } else {
    if (y == Y) {
      if (a.wl.total <= 0) return cudaSuccess;
      constexpr int LA = ClassL<X>::l1, LB = ClassL<X>::l2, LC = ClassL<Y>::l1, LD = ClassL<Y>::l2;
      using T = std::conditional_t<P == 1, float, double>;
      using S = GShape<LA, LB, LC, LD, T>;
      constexpr int WPB = 4;
      static_assert(S::table_bytes() + WPB * S::smem_per_warp() <= 227 * 1024, "gradient block exceeds 227 KB");
      LaunchInfo li;
      auto kern = grad_warp_kernel<LA, LB, LC, LD, T>;
      cudaError_t e = launch_persistent(kern, S::table_bytes() + WPB * S::smem_per_warp(), a.wl.total, WPB, nsm, &li);
      if (e != cudaSuccess) return e;
      kern<<<li.grid, li.block, li.smem, s>>>(a);
      return cudaGetLastError();
    }
    return launch_grad_unit<X, P, Y + 1>(y, a, s, nsm);
  }
}

template <int LAB, int LCD, typename T>
cudaError_t launch_j_t(const JArgs& a, cudaStream_t s, int nsm) {
  if (a.wl.total <= 0) return cudaSuccess;
  if constexpr (use_j_thread(LAB, LCD)) {
    auto kern = j_thread_kernel<LAB, LCD, T>;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, 0);
    if (e != cudaSuccess) return e;
    const int64_t need = (a.wl.total + 127) / 128;
    const int64_t grid = std::min<int64_t>(need, (int64_t)nsm * std::max(occ, 1));
    kern<<<(int)std::max<int64_t>(1, grid), 128, 0, s>>>(a);
    return cudaGetLastError();
  } else {
    using S = JShape<LAB, LCD, T>;
    constexpr int WPB = 4;
    static_assert(WPB * S::smem_per_warp() <= 227 * 1024, "J-engine block exceeds 227 KB");
    LaunchInfo li;
    auto kern = j_warp_kernel<LAB, LCD, T>;
    cudaError_t e = launch_persistent(kern, WPB * S::smem_per_warp(), a.wl.total, WPB, nsm, &li);
    if (e != cudaSuccess) return e;
    kern<<<li.grid, li.block, li.smem, s>>>(a);
    return cudaGetLastError();
  }
}

template <int LAB>
cudaError_t launch_j_lab(int LCD, int prec, const JArgs& a, cudaStream_t s, int nsm) {
#define ERI_JCASE(N) \
  case N: return prec ? launch_j_t<LAB, N, float>(a, s, nsm) : launch_j_t<LAB, N, double>(a, s, nsm);
  switch (LCD) {
    ERI_JCASE(0)
    ERI_JCASE(1)
    ERI_JCASE(2)
    ERI_JCASE(3)
    ERI_JCASE(4)
    ERI_JCASE(5)
    ERI_JCASE(6)
  }
#undef ERI_JCASE
  return cudaErrorInvalidValue;
}

// J/K entry points: explicitly instantiated once per entry of units.h in its own
// compilation unit (k_unit.cu), referenced from plan.cu
#define ERI_JK_UNIT_DECL(X, P, YLO, YHI) \
  extern template cudaError_t launch_jk_unit<X, P, YLO, YHI>(int, const JKArgs&, cudaStream_t, int);
ERI_JK_UNITS(ERI_JK_UNIT_DECL)
#undef ERI_JK_UNIT_DECL
#define ERI_GRAD_UNIT_DECL(X, P) extern template cudaError_t launch_grad_unit<X, P, 0>(int, const GradArgs&, cudaStream_t, int);
ERI_GRAD_UNITS(ERI_GRAD_UNIT_DECL)
#undef ERI_GRAD_UNIT_DECL
cudaError_t launch_j_lab0(int, int, const JArgs&, cudaStream_t, int);
cudaError_t launch_j_lab1(int, int, const JArgs&, cudaStream_t, int);
cudaError_t launch_j_lab2(int, int, const JArgs&, cudaStream_t, int);
cudaError_t launch_j_lab3(int, int, const JArgs&, cudaStream_t, int);
cudaError_t launch_j_lab4(int, int, const JArgs&, cudaStream_t, int);
cudaError_t launch_j_lab5(int, int, const JArgs&, cudaStream_t, int);
cudaError_t launch_j_lab6(int, int, const JArgs&, cudaStream_t, int);

}  // namespace eri
