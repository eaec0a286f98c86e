// Shared device code for the GB300 integral-direct J/K library.
//
// McMurchie-Davidson scheme of the paper (Wang et al., Sec. 2.1-2.4):
//   - Hermite expansion coefficients E^{ij}_t, Eq. cartesian_to_hermite and
//     its recurrence Eq. E_recursion (computed on the fly per primitive pair);
//   - Boys function F_m(T), Eq. boys_function, by tabulated Taylor expansion
//     plus downward recursion ("interpolation and downward recursion", Sec. 2.3);
//   - auxiliary integrals R^0_{tuv}, Eq. R_definition / Eq. R_recursion, built
//     level by level in shared memory by a whole warp;
//   - ERI assembly Eq. eri_formula (two transforms: ket then bra).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace eri {

constexpr int LMAX = 3;              // basis functions up to f
constexpr int LMAX_PAIR = 2 * LMAX;  // Hermite order of a pair
constexpr int LMAX_QUARTET = 4 * LMAX + 1;  // +1: gradient raises one bra index
constexpr int NPAIRCLASS = 10;       // ss ps pp ds dp dd fs fp fd ff

// Boys table: F_m(T_k) at T_k = k * BOYS_H, k = 0..BOYS_NT-1, m = 0..BOYS_MDIM-1.
constexpr double BOYS_H = 0.05;
constexpr double BOYS_INV_H = 20.0;
constexpr double BOYS_TMAX = 36.0;   // Taylor + downward recursion below, asymptote + upward above
constexpr int BOYS_NT = 722;         // covers T < 36 + h/2
constexpr int BOYS_TAYLOR64 = 8;     // |dT| <= 0.025: error ~ dT^8/8! ~ 4e-18 relative
constexpr int BOYS_TAYLOR32 = 4;     // dT^4/4! ~ 1.6e-8 relative
constexpr int BOYS_MDIM = LMAX_QUARTET + 1 + BOYS_TAYLOR64;  // 22

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
// number of Hermite triples (t,u,v) with t+u+v <= n
__host__ __device__ constexpr int nherm(int n) { return (n + 1) * (n + 2) * (n + 3) / 6; }
__host__ __device__ constexpr int pair_class(int l1, int l2) { return l1 * (l1 + 1) / 2 + l2; }  // l1 >= l2

// Cartesian components of shell l in lexicographic order (x desc, then y desc):
// xx,xy,xz,yy,yz,zz for d; xxx,xxy,...,zzz for f.  k-th component exponents.
__host__ __device__ inline void cart_xyz(int l, int k, int& x, int& y, int& z) {
  int r = 0;
  while ((r + 1) * (r + 2) / 2 <= k) ++r;  // r = y + z
  z = k - r * (r + 1) / 2;
  y = r - z;
  x = l - r;
}

// Compact Hermite index: triples grouped by n = t+u+v, inside a group ordered
// by (u+v) then v (same order as Cartesian components).
__host__ __device__ inline int herm_index(int t, int u, int v) {
  int n = t + u + v, r = u + v;
  return nherm(n - 1) + r * (r + 1) / 2 + v;
}

// One entry of the R recursion table (per compact Hermite index e):
//   R^m_e = c * (k * R^{m+1}_{dep2} + PQ_dir * R^{m+1}_{dep1}),  c = -2 rho
// (the scaled form r^m = R^m / (-2 rho)^m; see r_build below).
struct RStep {
  uint8_t t, u, v, dir;
  int16_t dep1, dep2;  // dep2 < 0: no k-term
  int16_t k, pad;
};

// Per-primitive-pair data, structure of arrays (double); float shadows for the FP32 tier.
struct PairData {
  const double* p;     // a + b
  const double* P;     // [3][n] pair centre
  const double* PA;    // [3][n] P - A (A: centre of the higher-l shell)
  const double* PB;    // [3][n]
  const double* pref;  // c_a c_b exp(-ab/p |AB|^2) sqrt(2 pi^(5/2)) / p
  const float* pf;     // float p
  const float* Pf;     // float P [3][n]
  const float* PAf;
  const float* PBf;
  const float* preff;
  int n;               // number of primitive pairs (row stride of the [3][n] arrays)
};

struct ShellPairInfo {
  const int32_t* s1;       // higher-l shell (a)
  const int32_t* s2;       // other shell (b)
  const int32_t* np;       // number of primitive pairs
  const int32_t* poff;     // first primitive pair
  const int32_t* ao1;      // AO offset of s1
  const int32_t* ao2;      // AO offset of s2
  const int32_t* hoff;     // offset of the Hermite density / Hermite J of the first primitive pair
};

// Per (bra class, ket class) work description, all device pointers.
struct WorkList {
  const int32_t* bra;      // sorted pair ids of the bra class
  const int32_t* ket;      // sorted pair ids of the ket class
  const int64_t* prefix;   // [nbra+1] inclusive prefix of kets per bra position
  int nbra;
  int64_t total;
};

// Boys F_0..F_M at T (FP64): Taylor around the nearest grid point for F_M, then
// downward recursion F_m = (2T F_{m+1} + exp(-T)) / (2m+1); above BOYS_TMAX the
// asymptote F_0 = sqrt(pi/T)/2 and upward recursion.  Own derivation from
// dF_m/dT = -F_{m+1}; CUDA's exp/sqrt are called, not reproduced.
template <int M>
__device__ __forceinline__ void boys_f64(double T, const double* __restrict__ tab, double* F) {
  if (T < BOYS_TMAX) {
    int k = __double2int_rn(T * BOYS_INV_H);
    double d = k * BOYS_H - T;  // -(T - T_k)
    const double* row = tab + k * BOYS_MDIM + M;
    double acc = __ldg(row + BOYS_TAYLOR64 - 1);
#pragma unroll
    for (int j = BOYS_TAYLOR64 - 2; j >= 0; --j) acc = fma(acc, d * (1.0 / (j + 1)), __ldg(row + j));
    F[M] = acc;
    double e = exp(-T);
    double t2 = 2.0 * T;
#pragma unroll
    for (int m = M - 1; m >= 0; --m) F[m] = fma(t2, F[m + 1], e) * (1.0 / (2 * m + 1));
  } else {
    double e = exp(-T);
    double inv2t = 0.5 / T;
    F[0] = 0.5 * sqrt(3.14159265358979323846 / T);
#pragma unroll
    for (int m = 0; m < M; ++m) F[m + 1] = fma((double)(2 * m + 1), F[m], -e) * inv2t;
  }
}

template <int M>
__device__ __forceinline__ void boys_f32(float T, const float* __restrict__ tab, float* F) {
  if (T < (float)BOYS_TMAX) {
    int k = __float2int_rn(T * (float)BOYS_INV_H);
    float d = k * (float)BOYS_H - T;
    const float* row = tab + k * BOYS_MDIM + M;
    float acc = __ldg(row + BOYS_TAYLOR32 - 1);
#pragma unroll
    for (int j = BOYS_TAYLOR32 - 2; j >= 0; --j) acc = fmaf(acc, d * (1.0f / (j + 1)), __ldg(row + j));
    F[M] = acc;
    float e = __expf(-T);
    float t2 = 2.0f * T;
#pragma unroll
    for (int m = M - 1; m >= 0; --m) F[m] = fmaf(t2, F[m + 1], e) * (1.0f / (2 * m + 1));
  } else {
    float e = __expf(-T);
    float inv2t = 0.5f / T;
    F[0] = 0.5f * sqrtf(3.14159265f / T);
#pragma unroll
    for (int m = 0; m < M; ++m) F[m + 1] = fmaf((float)(2 * m + 1), F[m], -e) * inv2t;
  }
}

template <typename T> struct Boys;
template <> struct Boys<double> {
  template <int M> __device__ static void eval(double t, const double* tab64, const float*, double* F) {
    boys_f64<M>(t, tab64, F);
  }
};
template <> struct Boys<float> {
  template <int M> __device__ static void eval(float t, const double*, const float* tab32, float* F) {
    boys_f32<M>(t, tab32, F);
  }
};

// McMurchie-Davidson E^{ij}_t for one direction, i <= LI, j <= LJ, t <= i+j
// (Eq. E_recursion with E^{00}_0 = 1; the exp(-ab/p AB^2) factor lives in the
// pair prefactor).  Layout E[(i*(LJ+1)+j)*(LI+LJ+1)+t].
template <int LI, int LJ, typename T>
__device__ __forceinline__ void md_e_1d(T PA, T PB, T o2p, T* E) {
  constexpr int NT = LI + LJ + 1;
#pragma unroll
  for (int x = 0; x < (LI + 1) * (LJ + 1) * NT; ++x) E[x] = T(0);
  E[0] = T(1);
#pragma unroll
  for (int i = 0; i < LI; ++i) {
    const T* src = E + (i * (LJ + 1)) * NT;
    T* dst = E + ((i + 1) * (LJ + 1)) * NT;
#pragma unroll
    for (int t = 0; t <= i + 1; ++t) {
      T v = PA * src[t];
      if (t > 0) v += o2p * src[t - 1];
      if (t + 1 <= i) v += T(t + 1) * src[t + 1];
      dst[t] = v;
    }
  }
#pragma unroll
  for (int i = 0; i <= LI; ++i) {
#pragma unroll
    for (int j = 0; j < LJ; ++j) {
      const T* src = E + (i * (LJ + 1) + j) * NT;
      T* dst = E + (i * (LJ + 1) + j + 1) * NT;
#pragma unroll
      for (int t = 0; t <= i + j + 1; ++t) {
        T v = PB * src[t];
        if (t > 0) v += o2p * src[t - 1];
        if (t + 1 <= i + j) v += T(t + 1) * src[t + 1];
        dst[t] = v;
      }
    }
  }
}

__device__ __forceinline__ double atomic_add_d(double* p, double v) { return atomicAdd(p, v); }

// Error codes written by device code into the plan's status word.
enum : int { DEV_OK = 0, DEV_BOUNDS = 1 };

}  // namespace eri
