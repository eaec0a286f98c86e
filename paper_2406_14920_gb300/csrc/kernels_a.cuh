// Small-class J+K kernel: one thread per canonical shell quartet, everything in
// registers with compile-time indexing (the whole McMurchie-Davidson chain of
// Eq. eri_formula is unrolled per class).  Used for classes whose contracted
// ERI block and R table fit in registers.  Each lane of a warp is an
// independent quartet, so all 32 lanes issue the same FP64 instruction stream.
#pragma once
#include "kernels.cuh"

namespace eri {

struct JKArgs {
  KArgs k;     // pair data, lists, tables, D', Kh (Kh may be null: no exchange)
  double* Jh;  // half-J accumulator nbf x nbf (null: no Coulomb)
};

template <int LA, int LB, int LC, int LD>
struct AShape {
  static constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
  static constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  static constexpr int NAB = NA * NB, NCD = NC * ND, HAB = nherm(LAB), NR = nherm(L);
  static constexpr int NEB = (LA + 1) * (LB + 1) * (LAB + 1), NEK = (LC + 1) * (LD + 1) * (LCD + 1);
};

// (ab|cd) for all components of one contracted quartet, summed over primitives:
//   W_P[cd] = sum_Q E'_Q^{cd} R_{P+Q}  (E' = (-1)^|Q| E),  (ab|cd) += sum_P E_P^{ab} W_P[cd].
template <int LA, int LB, int LC, int LD, typename T>
__device__ __forceinline__ void eri_block_reg(const KArgs& a, int offb, int npb, int eb0, int offk, int npk, int ek0,
                                              T* X) {
  using S = AShape<LA, LB, LC, LD>;
  constexpr int LAB = S::LAB, LCD = S::LCD, L = S::L;
#pragma unroll
  for (int x = 0; x < S::NAB * S::NCD; ++x) X[x] = T(0);
  for (int pb = 0; pb < npb; ++pb) {
    Prim<T> bp;
    bp.load(a.pd, offb + pb);
    T eb[3][S::NEB];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int x = 0; x < S::NEB; ++x) eb[d][x] = ldE<T>(a.pd, eb0 + (pb * 3 + d) * S::NEB + x);
    for (int pk = 0; pk < npk; ++pk) {
      Prim<T> kp;
      kp.load(a.pd, offk + pk);
      T ek[3][S::NEK];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int x = 0; x < S::NEK; ++x) {
          const T v = ldE<T>(a.pd, ek0 + (pk * 3 + d) * S::NEK + x);
          ek[d][x] = ((x % (LCD + 1)) & 1) ? -v : v;  // (-1)^s folded into the ket
        }
      const T ps = bp.p + kp.p;
      const T rho = bp.p * kp.p / ps;
      const T PQx = bp.P[0] - kp.P[0], PQy = bp.P[1] - kp.P[1], PQz = bp.P[2] - kp.P[2];
      T F[L + 1];
      Boys<T>::template eval<L>(rho * (PQx * PQx + PQy * PQy + PQz * PQz), a.bt, F);
      const T pref = bp.pref * kp.pref * (T(1) / sqrt(ps));
      T R[S::NR];
      r_build_reg<L, T>(F, pref, PQx, PQy, PQz, T(-2) * rho, R);
#pragma unroll
      for (int icd = 0; icd < S::NCD; ++icd) {
        int kx = 0, ky = 0, kz = 0, lx = 0, ly = 0, lz = 0;
        cart_xyz(LC, icd / S::ND, kx, ky, kz);
        cart_xyz(LD, icd % S::ND, lx, ly, lz);
        const T* ex = ek[0] + (kx * (LD + 1) + lx) * (LCD + 1);
        const T* ey = ek[1] + (ky * (LD + 1) + ly) * (LCD + 1);
        const T* ez = ek[2] + (kz * (LD + 1) + lz) * (LCD + 1);
        T W[S::HAB];
#pragma unroll
        for (int P = 0; P < S::HAB; ++P) {
          const int t = herm_t(P), u = herm_u(P), v = herm_v(P);
          T acc = T(0);
#pragma unroll
          for (int sx = 0; sx <= kx + lx; ++sx) {
            T accy = T(0);
#pragma unroll
            for (int sy = 0; sy <= ky + ly; ++sy) {
              T accz = T(0);
#pragma unroll
              for (int sz = 0; sz <= kz + lz; ++sz) accz = fma(ez[sz], R[herm_index(t + sx, u + sy, v + sz)], accz);
              accy = fma(ey[sy], accz, accy);
            }
            acc = fma(ex[sx], accy, acc);
          }
          W[P] = acc;
        }
#pragma unroll
        for (int iab = 0; iab < S::NAB; ++iab) {
          int ix = 0, iy = 0, iz = 0, jx = 0, jy = 0, jz = 0;
          cart_xyz(LA, iab / S::NB, ix, iy, iz);
          cart_xyz(LB, iab % S::NB, jx, jy, jz);
          const T* fx = eb[0] + (ix * (LB + 1) + jx) * (LAB + 1);
          const T* fy = eb[1] + (iy * (LB + 1) + jy) * (LAB + 1);
          const T* fz = eb[2] + (iz * (LB + 1) + jz) * (LAB + 1);
          T acc = T(0);
#pragma unroll
          for (int tx = 0; tx <= ix + jx; ++tx) {
            T accy = T(0);
#pragma unroll
            for (int ty = 0; ty <= iy + jy; ++ty) {
              T accz = T(0);
#pragma unroll
              for (int tz = 0; tz <= iz + jz; ++tz) accz = fma(fz[tz], W[herm_index(tx, ty, tz)], accz);
              accy = fma(fy[ty], accz, accy);
            }
            acc = fma(fx[tx], accy, acc);
          }
          X[iab * S::NCD + icd] += acc;
        }
      }
    }
  }
}

// Contraction of one contracted ERI block into the half-J / half-K accumulators
// (Eq. j_definition, Eq. k_definition with the canonical-quartet weights; the
// transposes are added by the post kernels).
template <int LA, int LB, int LC, int LD, typename T>
__device__ __forceinline__ void contract_block(const JKArgs& A, const T* X, T w, int ao1, int ao2, int ao3, int ao4) {
  using S = AShape<LA, LB, LC, LD>;
  const int n = A.k.nbf;
  const double* Dp = A.k.Dp;
  if (A.k.Kh) {
#pragma unroll
    for (int ia = 0; ia < S::NA; ++ia) {
#pragma unroll
      for (int ic = 0; ic < S::NC; ++ic) {  // Kh_ac += w (ab|cd) D_bd
        T s = T(0);
#pragma unroll
        for (int ib = 0; ib < S::NB; ++ib)
#pragma unroll
          for (int id = 0; id < S::ND; ++id)
            s = fma(X[(ia * S::NB + ib) * S::NCD + ic * S::ND + id], ldT<T>(Dp + (size_t)(ao2 + ib) * n + ao4 + id), s);
        atomic_add_d(A.k.Kh + (size_t)(ao1 + ia) * n + ao3 + ic, (double)(w * s));
      }
#pragma unroll
      for (int id = 0; id < S::ND; ++id) {  // Kh_ad += w (ab|cd) D_bc
        T s = T(0);
#pragma unroll
        for (int ib = 0; ib < S::NB; ++ib)
#pragma unroll
          for (int ic = 0; ic < S::NC; ++ic)
            s = fma(X[(ia * S::NB + ib) * S::NCD + ic * S::ND + id], ldT<T>(Dp + (size_t)(ao2 + ib) * n + ao3 + ic), s);
        atomic_add_d(A.k.Kh + (size_t)(ao1 + ia) * n + ao4 + id, (double)(w * s));
      }
    }
#pragma unroll
    for (int ib = 0; ib < S::NB; ++ib) {
#pragma unroll
      for (int ic = 0; ic < S::NC; ++ic) {  // Kh_bc += w (ab|cd) D_ad
        T s = T(0);
#pragma unroll
        for (int ia = 0; ia < S::NA; ++ia)
#pragma unroll
          for (int id = 0; id < S::ND; ++id)
            s = fma(X[(ia * S::NB + ib) * S::NCD + ic * S::ND + id], ldT<T>(Dp + (size_t)(ao1 + ia) * n + ao4 + id), s);
        atomic_add_d(A.k.Kh + (size_t)(ao2 + ib) * n + ao3 + ic, (double)(w * s));
      }
#pragma unroll
      for (int id = 0; id < S::ND; ++id) {  // Kh_bd += w (ab|cd) D_ac
        T s = T(0);
#pragma unroll
        for (int ia = 0; ia < S::NA; ++ia)
#pragma unroll
          for (int ic = 0; ic < S::NC; ++ic)
            s = fma(X[(ia * S::NB + ib) * S::NCD + ic * S::ND + id], ldT<T>(Dp + (size_t)(ao1 + ia) * n + ao3 + ic), s);
        atomic_add_d(A.k.Kh + (size_t)(ao2 + ib) * n + ao4 + id, (double)(w * s));
      }
    }
  }
  if (A.Jh) {
    const T w2 = T(2) * w;
#pragma unroll
    for (int iab = 0; iab < S::NAB; ++iab) {  // Jh_ab += 2w (ab|cd) D_cd
      T s = T(0);
#pragma unroll
      for (int icd = 0; icd < S::NCD; ++icd)
        s = fma(X[iab * S::NCD + icd], ldT<T>(Dp + (size_t)(ao3 + icd / S::ND) * n + ao4 + icd % S::ND), s);
      atomic_add_d(A.Jh + (size_t)(ao1 + iab / S::NB) * n + ao2 + iab % S::NB, (double)(w2 * s));
    }
#pragma unroll
    for (int icd = 0; icd < S::NCD; ++icd) {  // Jh_cd += 2w (ab|cd) D_ab
      T s = T(0);
#pragma unroll
      for (int iab = 0; iab < S::NAB; ++iab)
        s = fma(X[iab * S::NCD + icd], ldT<T>(Dp + (size_t)(ao1 + iab / S::NB) * n + ao2 + iab % S::NB), s);
      atomic_add_d(A.Jh + (size_t)(ao3 + icd / S::ND) * n + ao4 + icd % S::ND, (double)(w2 * s));
    }
  }
}

template <int LA, int LB, int LC, int LD, typename T>
__global__ void __launch_bounds__(128) jk_thread_kernel(JKArgs A) {
  using S = AShape<LA, LB, LC, LD>;
  const KArgs& a = A.k;
  const int64_t total = a.wl.total;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long done = 0, doneq = 0, doneb = 0;
  for (int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; item < total; item += stride) {
    const int ib = find_bra(a.wl.prefix, a.wl.nbra, item);
    const int ik = (int)(item - __ldg(a.wl.prefix + ib));
    const int pb_id = __ldg(a.wl.bra + ib), pk_id = __ldg(a.wl.ket + ik);
    const int s1 = __ldg(a.sp.s1 + pb_id), s2 = __ldg(a.sp.s2 + pb_id);
    const int s3 = __ldg(a.sp.s1 + pk_id), s4 = __ldg(a.sp.s2 + pk_id);
    if (a.mixed && quartet_tier(a, pb_id, pk_id, s1, s2, s3, s4) != a.tier_want) continue;
    const int npb_ = __ldg(a.sp.np + pb_id), npk_ = __ldg(a.sp.np + pk_id);
    ++done;
    doneq += (unsigned long long)npb_ * npk_;
    doneb += npb_;
    T w = T(1);
    if (s1 == s2) w *= T(0.5);
    if (s3 == s4) w *= T(0.5);
    if (pb_id == pk_id) w *= T(0.5);
    T X[S::NAB * S::NCD];
    eri_block_reg<LA, LB, LC, LD, T>(a, __ldg(a.sp.poff + pb_id), __ldg(a.sp.np + pb_id), __ldg(a.sp.eoff + pb_id),
                                     __ldg(a.sp.poff + pk_id), __ldg(a.sp.np + pk_id), __ldg(a.sp.eoff + pk_id), X);
    contract_block<LA, LB, LC, LD, T>(A, X, w, __ldg(a.sp.ao1 + pb_id), __ldg(a.sp.ao2 + pb_id),
                                      __ldg(a.sp.ao1 + pk_id), __ldg(a.sp.ao2 + pk_id));
  }
  if (a.counter && done) {
    atomicAdd(a.counter, done);
    atomicAdd(a.counter + 1, doneq);
    atomicAdd(a.counter + 2, doneb);
  }
}

}  // namespace eri
