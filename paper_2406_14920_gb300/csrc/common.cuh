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
#include <type_traits>
#include <utility>
#include <cuda_runtime.h>

namespace eri {

constexpr int LMAX = 3;              // basis functions up to f
constexpr int LMAX_PAIR = 2 * LMAX;  // Hermite order of a pair
constexpr int LMAX_QUARTET = 4 * LMAX + 1;  // +1: gradient raises one bra index
constexpr int NPAIRCLASS = 10;       // ss ps pp ds dp dd fs fp fd ff

// Boys tables on the grid T_k = k * BOYS_H, k = 0..BOYS_NT-1:
//   FP64: [k][m][j] = F_{m+j}(T_k) / j!, j < 8, m <= BOYS_MMAX (Taylor coefficients),
//   FP32: [k][m][j], j < 4;  plus exp(-T_k) in both precisions.
constexpr double BOYS_H = 0.05;
constexpr double BOYS_INV_H = 20.0;
constexpr double BOYS_TMAX = 36.0;   // Taylor + downward recursion below, asymptote + upward above
constexpr int BOYS_NT = 722;         // covers T < 36 + h/2
constexpr int BOYS_J64 = 8;          // |dT| <= 0.025: truncation ~ dT^8/8! ~ 4e-18 relative
constexpr int BOYS_J32 = 4;          // dT^4/4! ~ 1.6e-8 relative
constexpr int BOYS_MMAX = LMAX_QUARTET;  // 13
static_assert(BOYS_J32 == 4 && BOYS_J64 == 8, "Boys rows are read as one float4 / four double2");

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
// number of Hermite triples (t,u,v) with t+u+v <= n
__host__ __device__ constexpr int nherm(int n) { return (n + 1) * (n + 2) * (n + 3) / 6; }
__host__ __device__ constexpr int pair_class(int l1, int l2) { return l1 * (l1 + 1) / 2 + l2; }  // l1 >= l2

// Cartesian components of shell l in lexicographic order (x desc, then y desc):
// xx,xy,xz,yy,yz,zz for d; xxx,xxy,...,zzz for f.  k-th component exponents.
__host__ __device__ constexpr void cart_xyz(int l, int k, int& x, int& y, int& z) {
  int r = 0;
  while ((r + 1) * (r + 2) / 2 <= k) ++r;  // r = y + z
  z = k - r * (r + 1) / 2;
  y = r - z;
  x = l - r;
}

// position of component (l-y-z, y, z) inside shell l (loop-free)
// Compile-time loop: f(std::integral_constant<int, i>) for i = 0 .. N-1.  Every
// index is a constant expression inside f (usable in `if constexpr` and as a
// register-array index), independent of the compiler's unrolling heuristics.
template <typename F, int... I>
__device__ __forceinline__ void sfor_seq(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (N > 0) sfor_seq(f, std::make_integer_sequence<int, N>{});
}
#define ERI_CI(x) decltype(x)::value

// sum_{x <= NX, y <= NY, z <= NZ} cx[x] cy[y] cz[z] v(x, y, z), factored as
// sum_x cx[x] (sum_y cy[y] (sum_z cz[z] v)).  A direction with N = 0 has the
// single Hermite coefficient E^{00}_0 = 1 (the exponential factor lives in the
// pair prefactor), so it contributes no multiplication.  ALT: coefficient of
// index s carries (-1)^s (the ket sign of Eq. eri_formula).
template <int NX, int NY, int NZ, bool ALT, typename T, typename V>
__device__ __forceinline__ T tsum(const T* cx, const T* cy, const T* cz, V&& v) {
  T acc = T(0);
  sfor<NX + 1>([&](auto ix) {
    constexpr int x = ERI_CI(ix);
    T accy = T(0);
    sfor<NY + 1>([&](auto iy) {
      constexpr int y = ERI_CI(iy);
      T accz = T(0);
      sfor<NZ + 1>([&](auto iz) {
        constexpr int z = ERI_CI(iz);
        const T val = v(std::integral_constant<int, x>{}, std::integral_constant<int, y>{},
                        std::integral_constant<int, z>{});
        if constexpr (NZ == 0) accz = val;
        else if constexpr (ALT && (z & 1)) accz = fma(-cz[z], val, accz);
        else accz = fma(cz[z], val, accz);
      });
      if constexpr (NY == 0) accy = accz;
      else if constexpr (ALT && (y & 1)) accy = fma(-cy[y], accz, accy);
      else accy = fma(cy[y], accz, accy);
    });
    if constexpr (NX == 0) acc = accy;
    else if constexpr (ALT && (x & 1)) acc = fma(-cx[x], accy, acc);
    else acc = fma(cx[x], accy, acc);
  });
  return acc;
}

// f(x, y, z) (integral constants) for every Cartesian component of angular
// momentum L, in the lexicographic order (x descending, then y descending)
template <int L, typename F>
__device__ __forceinline__ void for_cart(F&& f) {
  sfor<L + 1>([&](auto a) {
    constexpr int x = L - ERI_CI(a);
    sfor<L - x + 1>([&](auto b) {
      constexpr int y = L - x - ERI_CI(b);
      f(std::integral_constant<int, x>{}, std::integral_constant<int, y>{}, std::integral_constant<int, L - x - y>{});
    });
  });
}

// f(t, u, v) (integral constants) for every Hermite index with t + u + v <= L
template <int L, typename F>
__device__ __forceinline__ void for_herm(F&& f) {
  sfor<L + 1>([&](auto a) {
    constexpr int t = ERI_CI(a);
    sfor<L - t + 1>([&](auto b) {
      constexpr int u = ERI_CI(b);
      sfor<L - t - u + 1>([&](auto c) {
        f(std::integral_constant<int, t>{}, std::integral_constant<int, u>{},
          std::integral_constant<int, ERI_CI(c)>{});
      });
    });
  });
}

__host__ __device__ constexpr int cidx(int l, int y, int z) {
  return (y + z) * (y + z + 1) / 2 + z + 0 * l;
}

// Compact Hermite index: triples grouped by n = t+u+v, inside a group ordered
// by (u+v) then v (same order as Cartesian components).
__host__ __device__ constexpr int herm_index(int t, int u, int v) {
  return nherm(t + u + v - 1) + (u + v) * (u + v + 1) / 2 + v;
}
// inverse of herm_index (compile-time foldable when e is a constant)
__host__ __device__ constexpr int herm_n(int e) {
  int n = 0;
  while (nherm(n) <= e) ++n;
  return n;
}
__host__ __device__ constexpr int herm_v(int e) {
  int k = e - nherm(herm_n(e) - 1), r = 0;
  while ((r + 1) * (r + 2) / 2 <= k) ++r;
  return k - r * (r + 1) / 2;
}
__host__ __device__ constexpr int herm_u(int e) {
  int k = e - nherm(herm_n(e) - 1), r = 0;
  while ((r + 1) * (r + 2) / 2 <= k) ++r;
  return r - (k - r * (r + 1) / 2);
}
__host__ __device__ constexpr int herm_t(int e) {
  int k = e - nherm(herm_n(e) - 1), r = 0;
  while ((r + 1) * (r + 2) / 2 <= k) ++r;
  return herm_n(e) - r;
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
  const double* ea;    // exponent of the s1 (higher-l shell) primitive
  const double* E;     // Hermite coefficients per primitive pair: 3 x (l1+1)(l2+1)(l1+l2+1), x then y then z
  const float* Ef;
  // FP32 shadows packed for vector loads, 3 per primitive pair i:
  //   q4[3i] = {P, p}, q4[3i+1] = {P-A, pref}, q4[3i+2] = {P-B, 0}
  const float4* q4;
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
  const int32_t* eoff;     // offset of the E tables of the first primitive pair
  // molecules (a plan may hold several independent molecules): pairs never
  // cross molecules, and D, J, K are packed one nbf_m x nbf_m block per molecule
  const int32_t* pmol;     // molecule of each pair
  const int64_t* mat_off;  // offset of each molecule's block in packed D / J / K
  const int32_t* mat_n;    // nbf of each molecule (row stride of its block)
};

// Per (bra class, ket class) work description, all device pointers.
struct WorkList {
  const int32_t* bra;      // sorted pair ids of the bra class
  const int32_t* ket;      // sorted pair ids of the ket class (molecule by molecule)
  const int32_t* kseg;     // start of each molecule's segment in `ket`, stride NPAIRCLASS
  const int64_t* prefix;   // [nbra+1] inclusive prefix of kets per bra position
  int nbra;
  int64_t total;
  int64_t first;           // items [first, total) are processed (0 except in tuning trials)
  int tile;                // consecutive items per worker tile (warp kernels: per warp; thread kernel: per lane)
  int shard, nshard;       // this launch takes the tiles t with t % nshard == shard (work split over GPUs)
};

// Boys F_0..F_M at T.  Below BOYS_TMAX: Taylor expansion of F_M around the
// nearest grid point, F_M(T) = sum_j F_{M+j}(T_k) (T_k - T)^j / j!  (from
// dF_m/dT = -F_{m+1}), exp(-T) = exp(-T_k) exp(T_k - T) with a short Taylor
// series, then the downward recursion F_m = (2T F_{m+1} + exp(-T)) / (2m+1).
// Above: F_0 = sqrt(pi/T)/2 (erf(sqrt T) = 1 to double precision) and the upward
// recursion F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T).  Our own construction
// ("interpolation and downward recursion", Sec. 2.3); CUDA's exp/rsqrt are
// called where needed, not reproduced.
struct BoysTabs {
  const double* c64;  // [BOYS_NT][BOYS_MMAX+1][BOYS_J64]
  const double* e64;  // [BOYS_NT] exp(-T_k)
  const float* c32;   // [BOYS_NT][BOYS_MMAX+1][BOYS_J32]
  const float* e32;
};

template <int M>
__device__ __forceinline__ void boys_f64(double T, const BoysTabs& bt, double* F) {
  if (T < BOYS_TMAX) {
    const int k = __double2int_rn(T * BOYS_INV_H);
    const double d = k * BOYS_H - T;
    // the 8 Taylor coefficients of (k, M) are one 64-byte row: four 16-byte loads
    const double2* c = reinterpret_cast<const double2*>(bt.c64 + ((size_t)k * (BOYS_MMAX + 1) + M) * BOYS_J64);
    const double2 c01 = __ldg(c), c23 = __ldg(c + 1), c45 = __ldg(c + 2), c67 = __ldg(c + 3);
    double f = fma(c67.y, d, c67.x);
    f = fma(f, d, c45.y);
    f = fma(f, d, c45.x);
    f = fma(f, d, c23.y);
    f = fma(f, d, c23.x);
    f = fma(f, d, c01.y);
    f = fma(f, d, c01.x);
    F[M] = f;
    if (M > 0) {
      // exp(d), |d| <= h/2, 8 Taylor terms
      double g = 1.0 / 5040.0;
      g = fma(g, d, 1.0 / 720.0);
      g = fma(g, d, 1.0 / 120.0);
      g = fma(g, d, 1.0 / 24.0);
      g = fma(g, d, 1.0 / 6.0);
      g = fma(g, d, 0.5);
      g = fma(g, d, 1.0);
      g = fma(g, d, 1.0);
      const double e = __ldg(bt.e64 + k) * g;
      const double t2 = 2.0 * T;
#pragma unroll
      for (int m = M - 1; m >= 0; --m) F[m] = fma(t2, F[m + 1], e) * (1.0 / (2 * m + 1));
    }
  } else {
    const double e = exp(-T);
    const double rt = rsqrt(T);
    F[0] = 0.88622692545275801365 * rt;  // sqrt(pi)/2
    const double inv2t = 0.5 * rt * rt;
#pragma unroll
    for (int m = 0; m < M; ++m) F[m + 1] = fma((double)(2 * m + 1), F[m], -e) * inv2t;
  }
}

template <int M>
__device__ __forceinline__ void boys_f32(float T, const BoysTabs& bt, float* F) {
  if (T < (float)BOYS_TMAX) {
    const int k = __float2int_rn(T * (float)BOYS_INV_H);
    const float d = k * (float)BOYS_H - T;
    // the 4 Taylor coefficients of (k, M) are one 16-byte row: one load
    const float4 c = __ldg(reinterpret_cast<const float4*>(bt.c32) + ((size_t)k * (BOYS_MMAX + 1) + M));
    float f = fmaf(c.w, d, c.z);
    f = fmaf(f, d, c.y);
    f = fmaf(f, d, c.x);
    F[M] = f;
    if (M > 0) {
      float g = 1.0f / 24.0f;
      g = fmaf(g, d, 1.0f / 6.0f);
      g = fmaf(g, d, 0.5f);
      g = fmaf(g, d, 1.0f);
      g = fmaf(g, d, 1.0f);
      const float e = __ldg(bt.e32 + k) * g;
      const float t2 = 2.0f * T;
#pragma unroll
      for (int m = M - 1; m >= 0; --m) F[m] = fmaf(t2, F[m + 1], e) * (1.0f / (2 * m + 1));
    }
  } else {
    const float e = __expf(-T);
    const float rt = rsqrtf(T);
    F[0] = 0.88622692545f * rt;
    const float inv2t = 0.5f * rt * rt;
#pragma unroll
    for (int m = 0; m < M; ++m) F[m + 1] = fmaf((float)(2 * m + 1), F[m], -e) * inv2t;
  }
}

template <typename T> struct Boys;
template <> struct Boys<double> {
  template <int M> __device__ static void eval(double t, const BoysTabs& bt, double* F) { boys_f64<M>(t, bt, F); }
};
template <> struct Boys<float> {
  template <int M> __device__ static void eval(float t, const BoysTabs& bt, float* F) { boys_f32<M>(t, bt, F); }
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

// Accumulation into a J / K / gradient accumulator.  det = 0: FP64 atomicAdd
// (the sum depends on the order in which the atomics land).  det = 1
// (deterministic builds): the accumulator holds a 64-bit two's-complement
// fixed-point number with scale 2^46 and v is rounded to it; integer addition
// is associative (exact modulo 2^64), so the final bits do not depend on the
// order of the additions.  Resolution 2^-46 = 1.4e-14, range |sum| < 2^17.
constexpr double kFixScale = 70368744177664.0;  // 2^46
constexpr double kFixInv = 1.0 / 70368744177664.0;
constexpr double kFixLimit = 65536.0;           // 2^16: |value| above this is reported (half the range)
__device__ __forceinline__ void acc_add(double* p, double v, int det) {
  if (det)
    atomicAdd(reinterpret_cast<unsigned long long*>(p),
              static_cast<unsigned long long>(__double2ll_rn(v * kFixScale)));
  else
    atomicAdd(p, v);
}
// value of an accumulator element (det: fixed point -> double)
__device__ __forceinline__ double acc_value(const double* p, int det) {
  if (!det) return *p;
  return (double)(*reinterpret_cast<const long long*>(p)) * kFixInv;
}

// R^0_{tuv}, t+u+v <= L, in registers (fully unrolled; every index is an
// arithmetic expression of unrolled loop counters, so it folds to a constant).
// Same scaled recursion as r_build_warp, done in place: inside a level the
// entries are updated from the highest n = t+u+v down, so the level m+1 values
// they read are still intact.
template <int L, typename T>
__device__ __forceinline__ void r_build_reg(const T* F, T pref, T X, T Y, T Z, T c, T* R) {
  const T Xc = c * X, Yc = c * Y, Zc = c * Z;
  R[0] = pref * F[L];
#pragma unroll
  for (int m = L - 1; m >= 0; --m) {
#pragma unroll
    for (int n = L - m; n >= 1; --n) {
#pragma unroll
      for (int t = n; t >= 0; --t) {
#pragma unroll
        for (int u = n - t; u >= 0; --u) {
          const int v = n - t - u;
          T val;
          if (t > 0) {
            val = Xc * R[herm_index(t - 1, u, v)];
            if (t > 1) val = fma(c * T(t - 1), R[herm_index(t - 2, u, v)], val);
          } else if (u > 0) {
            val = Yc * R[herm_index(0, u - 1, v)];
            if (u > 1) val = fma(c * T(u - 1), R[herm_index(0, u - 2, v)], val);
          } else {
            val = Zc * R[herm_index(0, 0, v - 1)];
            if (v > 1) val = fma(c * T(v - 1), R[herm_index(0, 0, v - 2)], val);
          }
          R[herm_index(t, u, v)] = val;
        }
      }
    }
    R[0] = pref * F[m];
  }
}

// Error codes written by device code into the plan's status word.
enum : int { DEV_OK = 0, DEV_BOUNDS = 1, DEV_RANGE = 2 };  // DEV_RANGE: a deterministic accumulator above 2^16

}  // namespace eri
