// Small-class J+K kernel: one thread per canonical shell quartet, everything in
// registers with compile-time indexing (the whole McMurchie-Davidson chain of
// Eq. eri_formula is unrolled per class).  Used for classes whose contracted
// ERI block and R table fit in registers.  Each lane of a warp is an
// independent quartet, so all 32 lanes issue the same FP64 instruction stream.
#pragma once
#include "kernels.cuh"

// 1: the register kernel sums the J_ab contributions of a warp's items over the
// warp (shuffles) when they share the bra pair, one atomic per element
#ifndef ERI_JAB_REDUCE
#define ERI_JAB_REDUCE 0
#endif
// FP64 register kernel beyond the tiny classes: largest L and footprint
// (doubles).  GB300 issues about 3.4 FP64 FMAs per clock per SM, so every warp
// instruction with idle lanes is expensive; one quartet per lane keeps all 32
// lanes busy (measured: (pp|pp) 31 -> 9.8 ms, (ds|pp) 16 -> 5.1 ms, (fp|ps)
// 12 -> 4.9 ms on workload 1; raising the limits from L 5 / 200 to L 6 / 300
// took (dp|pp) 16.5 -> 13.6 ms and (fs|fs) 2.5 -> 1.5 ms).
#ifndef ERI_THREAD64_LMAX
#define ERI_THREAD64_LMAX 6
#endif
#ifndef ERI_THREAD64_FOOT
#define ERI_THREAD64_FOOT 300
#endif

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
  // register footprint (values) of the two variants: W accumulated over the
  // ket primitives (fewer FLOPs), or the bra transform per primitive quartet
  static constexpr int REG_WACC = NCD * HAB + NAB * NCD + NR;
  static constexpr int REG_PERPQ = HAB + NAB * NCD + NR;
  // W accumulated over the ket primitives where its footprint stays near the
  // 255-register limit (a few hundred bytes of spill still beat the extra bra
  // transforms of the per-primitive-quartet variant; measured on GB300)
  static constexpr bool WACC = REG_WACC <= 260;
};

// Which classes run one quartet per thread (registers) rather than one per warp.
// FP64: classes with L <= 5 whose per-primitive-quartet footprint is at most
// 200 doubles.  FP32: every class of L <= 7 whose per-primitive-quartet register
// footprint is at most 460 values.  Measured on GB300 (workload 1, FP32 tier):
// the register kernel runs these classes 2.2x to 9.6x faster than the
// shared-memory warp kernel even where ptxas spills up to ~6 KB per thread
// (spills are lane-interleaved local memory, served by L1), because every
// index is a compile-time constant and all 32 lanes do useful work; the warp
// kernel stays for the classes with larger ERI blocks.
__host__ __device__ constexpr bool use_thread_kernel(int la, int lb, int lc, int ld, bool fp32) {
  const int L = la + lb + lc + ld;
  const int nab = ncart(la) * ncart(lb), ncd = ncart(lc) * ncart(ld);
  if (!fp32) return (L <= 3 && nab * ncd <= 27) || (L <= ERI_THREAD64_LMAX && nherm(la + lb) + nab * ncd + nherm(L) <= ERI_THREAD64_FOOT);
  const int hab = nherm(la + lb), nr = nherm(L);
  return L <= 7 && (hab + nab * ncd + nr) <= 460;
}

// (ab|cd) for all components of one contracted quartet, summed over primitives:
//   W_P[cd] = sum_{ket prims} sum_Q E'_Q^{cd} R_{P+Q}  (E' = (-1)^|Q| E),
//   (ab|cd) += sum_P E_P^{ab}(bra prim) W_P[cd]  once per bra primitive.
// E tables: FP64 loads them (memory is free next to the FP64 pipe), FP32
// rebuilds them from P-A, P-B and 1/(2p) (cheaper than scattered loads).
template <int LI, int LJ, typename T>
__device__ __forceinline__ void load_or_build_e(const PairData& pd, int e0, const Prim<T>& pr, T* e /*[3][NE]*/) {
  constexpr int NE = (LI + 1) * (LJ + 1) * (LI + LJ + 1);
  if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int x = 0; x < 3 * NE; ++x) e[x] = ldE<T>(pd, e0 + x);
  } else {
    const T o2p = T(0.5) / pr.p;
#pragma unroll
    for (int d = 0; d < 3; ++d) md_e_1d<LI, LJ, T>(pr.PA[d], pr.PB[d], o2p, e + d * NE);
  }
}

// Ket transform of one primitive quartet for one ket pair cd (compile-time
// exponents), one bra Hermite index P = (t, u, v):
//   sum_Q (-1)^|Q| E_Q^{cd} R_{P+Q}
template <int L, int KX, int KY, int KZ, int T_, int U_, int V_, typename T>
__device__ __forceinline__ T ket_term(const T* ex, const T* ey, const T* ez, const T* R) {
  return tsum<KX, KY, KZ, true>(ex, ey, ez, [&](auto sx, auto sy, auto sz) {
    return R[herm_index(T_ + ERI_CI(sx), U_ + ERI_CI(sy), V_ + ERI_CI(sz))];
  });
}

// Variant for classes whose W (all ket pairs) does not fit in registers: the
// bra transform runs per primitive quartet, one ket pair cd at a time.
template <int LA, int LB, int LC, int LD, typename T>
__device__ __forceinline__ void eri_block_reg_pq(const KArgs& a, int offb, int npb, int eb0, int offk, int npk, int ek0,
                                                 T* X) {
  using S = AShape<LA, LB, LC, LD>;
  constexpr int LAB = S::LAB, LCD = S::LCD, L = S::L;
#pragma unroll
  for (int x = 0; x < S::NAB * S::NCD; ++x) X[x] = T(0);
  for (int pb = 0; pb < npb; ++pb) {
    Prim<T> bp;
    bp.load(a.pd, offb + pb);
    T eb[3 * S::NEB];
    load_or_build_e<LA, LB, T>(a.pd, eb0 + pb * 3 * S::NEB, bp, eb);
    for (int pk = 0; pk < npk; ++pk) {
      Prim<T> kp;
      kp.load(a.pd, offk + pk);
      T ek[3 * S::NEK];
      load_or_build_e<LC, LD, T>(a.pd, ek0 + pk * 3 * S::NEK, kp, ek);
      const T ps = bp.p + kp.p;
      T rho = bp.p * kp.p / ps;
      T pref = bp.pref * kp.pref * rsqrt_t(ps);
      attenuate(om2<T>(a), rho, pref);
      const T PQx = bp.P[0] - kp.P[0], PQy = bp.P[1] - kp.P[1], PQz = bp.P[2] - kp.P[2];
      T F[L + 1];
      Boys<T>::template eval<L>(rho * (PQx * PQx + PQy * PQy + PQz * PQz), a.bt, F);
      T R[S::NR];
      r_build_reg<L, T>(F, pref, PQx, PQy, PQz, T(-2) * rho, R);
      for_cart<LC>([&](auto kx, auto ky, auto kz) {
        for_cart<LD>([&](auto lx, auto ly, auto lz) {
          constexpr int KX = ERI_CI(kx), KY = ERI_CI(ky), KZ = ERI_CI(kz);
          constexpr int LX = ERI_CI(lx), LY = ERI_CI(ly), LZ = ERI_CI(lz);
          constexpr int icd = cidx(LC, KY, KZ) * S::ND + cidx(LD, LY, LZ);
          const T* ex = ek + 0 * S::NEK + (KX * (LD + 1) + LX) * (LCD + 1);
          const T* ey = ek + 1 * S::NEK + (KY * (LD + 1) + LY) * (LCD + 1);
          const T* ez = ek + 2 * S::NEK + (KZ * (LD + 1) + LZ) * (LCD + 1);
          T W[S::HAB];
          for_herm<LAB>([&](auto t, auto u, auto v) {
            W[herm_index(ERI_CI(t), ERI_CI(u), ERI_CI(v))] =
                ket_term<L, KX + LX, KY + LY, KZ + LZ, ERI_CI(t), ERI_CI(u), ERI_CI(v)>(ex, ey, ez, R);
          });
          for_cart<LA>([&](auto ix, auto iy, auto iz) {
            for_cart<LB>([&](auto jx, auto jy, auto jz) {
              constexpr int IX = ERI_CI(ix), IY = ERI_CI(iy), IZ = ERI_CI(iz);
              constexpr int JX = ERI_CI(jx), JY = ERI_CI(jy), JZ = ERI_CI(jz);
              constexpr int iab = cidx(LA, IY, IZ) * S::NB + cidx(LB, JY, JZ);
              const T* fx = eb + 0 * S::NEB + (IX * (LB + 1) + JX) * (LAB + 1);
              const T* fy = eb + 1 * S::NEB + (IY * (LB + 1) + JY) * (LAB + 1);
              const T* fz = eb + 2 * S::NEB + (IZ * (LB + 1) + JZ) * (LAB + 1);
              X[iab * S::NCD + icd] += tsum<IX + JX, IY + JY, IZ + JZ, false>(
                  fx, fy, fz, [&](auto tx, auto ty, auto tz) { return W[herm_index(ERI_CI(tx), ERI_CI(ty), ERI_CI(tz))]; });
            });
          });
        });
      });
    }
  }
}

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
    T W[S::NCD * S::HAB];
#pragma unroll
    for (int x = 0; x < S::NCD * S::HAB; ++x) W[x] = T(0);
    for (int pk = 0; pk < npk; ++pk) {
      Prim<T> kp;
      kp.load(a.pd, offk + pk);
      T ek[3 * S::NEK];
      load_or_build_e<LC, LD, T>(a.pd, ek0 + pk * 3 * S::NEK, kp, ek);
      const T ps = bp.p + kp.p;
      T rho = bp.p * kp.p / ps;
      T pref = bp.pref * kp.pref * rsqrt_t(ps);
      attenuate(om2<T>(a), rho, pref);
      const T PQx = bp.P[0] - kp.P[0], PQy = bp.P[1] - kp.P[1], PQz = bp.P[2] - kp.P[2];
      T F[L + 1];
      Boys<T>::template eval<L>(rho * (PQx * PQx + PQy * PQy + PQz * PQz), a.bt, F);
      T R[S::NR];
      r_build_reg<L, T>(F, pref, PQx, PQy, PQz, T(-2) * rho, R);
      for_cart<LC>([&](auto kx, auto ky, auto kz) {
        for_cart<LD>([&](auto lx, auto ly, auto lz) {
          constexpr int KX = ERI_CI(kx), KY = ERI_CI(ky), KZ = ERI_CI(kz);
          constexpr int LX = ERI_CI(lx), LY = ERI_CI(ly), LZ = ERI_CI(lz);
          constexpr int icd = cidx(LC, KY, KZ) * S::ND + cidx(LD, LY, LZ);
          const T* ex = ek + 0 * S::NEK + (KX * (LD + 1) + LX) * (LCD + 1);
          const T* ey = ek + 1 * S::NEK + (KY * (LD + 1) + LY) * (LCD + 1);
          const T* ez = ek + 2 * S::NEK + (KZ * (LD + 1) + LZ) * (LCD + 1);
          for_herm<LAB>([&](auto t, auto u, auto v) {
            W[icd * S::HAB + herm_index(ERI_CI(t), ERI_CI(u), ERI_CI(v))] +=
                ket_term<L, KX + LX, KY + LY, KZ + LZ, ERI_CI(t), ERI_CI(u), ERI_CI(v)>(ex, ey, ez, R);
          });
        });
      });
    }
    T eb[3 * S::NEB];
    load_or_build_e<LA, LB, T>(a.pd, eb0 + pb * 3 * S::NEB, bp, eb);
    sfor<S::NCD>([&](auto icd_) {
      constexpr int icd = ERI_CI(icd_);
      for_cart<LA>([&](auto ix, auto iy, auto iz) {
        for_cart<LB>([&](auto jx, auto jy, auto jz) {
          constexpr int IX = ERI_CI(ix), IY = ERI_CI(iy), IZ = ERI_CI(iz);
          constexpr int JX = ERI_CI(jx), JY = ERI_CI(jy), JZ = ERI_CI(jz);
          constexpr int iab = cidx(LA, IY, IZ) * S::NB + cidx(LB, JY, JZ);
          const T* fx = eb + 0 * S::NEB + (IX * (LB + 1) + JX) * (LAB + 1);
          const T* fy = eb + 1 * S::NEB + (IY * (LB + 1) + JY) * (LAB + 1);
          const T* fz = eb + 2 * S::NEB + (IZ * (LB + 1) + JZ) * (LAB + 1);
          X[iab * S::NCD + icd] += tsum<IX + JX, IY + JY, IZ + JZ, false>(
              fx, fy, fz,
              [&](auto tx, auto ty, auto tz) { return W[icd * S::HAB + herm_index(ERI_CI(tx), ERI_CI(ty), ERI_CI(tz))]; });
        });
      });
    });
  }
}

// Contraction of one contracted ERI block into the half-J / half-K accumulators
// (Eq. j_definition, Eq. k_definition with the canonical-quartet weights; the
// transposes are added by the post kernels).
template <int LA, int LB, int LC, int LD, typename T>
__device__ __forceinline__ void contract_block(const JKArgs& A, const T* X, T w, int ao1, int ao2, int ao3, int ao4,
                                               int64_t base, int n, T* jab_out = nullptr) {
  using S = AShape<LA, LB, LC, LD>;
  const T* Dp = dens<T>(A.k) + base;
  double* Kh = A.k.Kh ? A.k.Kh + base : nullptr;
  double* Jh = A.Jh ? A.Jh + base : nullptr;
  if (Kh) {
#pragma unroll
    for (int ia = 0; ia < S::NA; ++ia) {
#pragma unroll
      for (int ic = 0; ic < S::NC; ++ic) {  // Kh_ac += w (ab|cd) D_bd
        T s = T(0);
#pragma unroll
        for (int ib = 0; ib < S::NB; ++ib)
#pragma unroll
          for (int id = 0; id < S::ND; ++id)
            s = fma(X[(ia * S::NB + ib) * S::NCD + ic * S::ND + id], __ldg(Dp + (size_t)(ao2 + ib) * n + ao4 + id), s);
        acc_add(Kh + (size_t)(ao1 + ia) * n + ao3 + ic, (double)(w * s), A.k.det);
      }
#pragma unroll
      for (int id = 0; id < S::ND; ++id) {  // Kh_ad += w (ab|cd) D_bc
        T s = T(0);
#pragma unroll
        for (int ib = 0; ib < S::NB; ++ib)
#pragma unroll
          for (int ic = 0; ic < S::NC; ++ic)
            s = fma(X[(ia * S::NB + ib) * S::NCD + ic * S::ND + id], __ldg(Dp + (size_t)(ao2 + ib) * n + ao3 + ic), s);
        acc_add(Kh + (size_t)(ao1 + ia) * n + ao4 + id, (double)(w * s), A.k.det);
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
            s = fma(X[(ia * S::NB + ib) * S::NCD + ic * S::ND + id], __ldg(Dp + (size_t)(ao1 + ia) * n + ao4 + id), s);
        acc_add(Kh + (size_t)(ao2 + ib) * n + ao3 + ic, (double)(w * s), A.k.det);
      }
#pragma unroll
      for (int id = 0; id < S::ND; ++id) {  // Kh_bd += w (ab|cd) D_ac
        T s = T(0);
#pragma unroll
        for (int ia = 0; ia < S::NA; ++ia)
#pragma unroll
          for (int ic = 0; ic < S::NC; ++ic)
            s = fma(X[(ia * S::NB + ib) * S::NCD + ic * S::ND + id], __ldg(Dp + (size_t)(ao1 + ia) * n + ao3 + ic), s);
        acc_add(Kh + (size_t)(ao2 + ib) * n + ao4 + id, (double)(w * s), A.k.det);
      }
    }
  }
  if (Jh) {
    const T w2 = T(2) * w;
#pragma unroll
    for (int iab = 0; iab < S::NAB; ++iab) {  // Jh_ab += 2w (ab|cd) D_cd
      T s = T(0);
#pragma unroll
      for (int icd = 0; icd < S::NCD; ++icd)
        s = fma(X[iab * S::NCD + icd], __ldg(Dp + (size_t)(ao3 + icd / S::ND) * n + ao4 + icd % S::ND), s);
      if (jab_out) jab_out[iab] = w2 * s;  // reduced over the warp by the caller
      else acc_add(Jh + (size_t)(ao1 + iab / S::NB) * n + ao2 + iab % S::NB, (double)(w2 * s), A.k.det);
    }
#pragma unroll
    for (int icd = 0; icd < S::NCD; ++icd) {  // Jh_cd += 2w (ab|cd) D_ab
      T s = T(0);
#pragma unroll
      for (int iab = 0; iab < S::NAB; ++iab)
        s = fma(X[iab * S::NCD + icd], __ldg(Dp + (size_t)(ao1 + iab / S::NB) * n + ao2 + iab % S::NB), s);
      acc_add(Jh + (size_t)(ao3 + icd / S::ND) * n + ao4 + icd % S::ND, (double)(w2 * s), A.k.det);
    }
  }
}

// One quartet (bra position ib, ket position ik of the work list) of a thread-kernel class.
// Where an item's J_ab contributions go when the caller reduces them over the warp.
struct JabTarget {
  int pb_id, ao1, ao2, n;
  int64_t base;
};

template <int LA, int LB, int LC, int LD, typename T>
__device__ __forceinline__ void thread_item(const JKArgs& A, int ib, int ik, unsigned long long& done,
                                            unsigned long long& doneq, unsigned long long& doneb,
                                            T* jab_out = nullptr, JabTarget* tgt = nullptr) {
  using S = AShape<LA, LB, LC, LD>;
  const KArgs& a = A.k;
  const int pb_id = __ldg(a.wl.bra + ib);
  const int mol = __ldg(a.sp.pmol + pb_id);
  const int pk_id = __ldg(a.wl.ket + __ldg(a.wl.kseg + mol * NPAIRCLASS) + ik);
  const int s1 = __ldg(a.sp.s1 + pb_id), s2 = __ldg(a.sp.s2 + pb_id);
  const int s3 = __ldg(a.sp.s1 + pk_id), s4 = __ldg(a.sp.s2 + pk_id);
  const int npb_ = __ldg(a.sp.np + pb_id), npk_ = __ldg(a.sp.np + pk_id);
  ++done;
  doneq += (unsigned long long)npb_ * npk_;
  doneb += npb_;
  T w = T(1);
  if (s1 == s2) w *= T(0.5);
  if (s3 == s4) w *= T(0.5);
  if (pb_id == pk_id) w *= T(0.5);
  T X[S::NAB * S::NCD];
  if constexpr (S::WACC)
    eri_block_reg<LA, LB, LC, LD, T>(a, __ldg(a.sp.poff + pb_id), npb_, __ldg(a.sp.eoff + pb_id),
                                     __ldg(a.sp.poff + pk_id), npk_, __ldg(a.sp.eoff + pk_id), X);
  else
    eri_block_reg_pq<LA, LB, LC, LD, T>(a, __ldg(a.sp.poff + pb_id), npb_, __ldg(a.sp.eoff + pb_id),
                                        __ldg(a.sp.poff + pk_id), npk_, __ldg(a.sp.eoff + pk_id), X);
  const int ao1 = __ldg(a.sp.ao1 + pb_id), ao2 = __ldg(a.sp.ao2 + pb_id);
  const int64_t base = __ldg(a.sp.mat_off + mol);
  const int n = __ldg(a.sp.mat_n + mol);
  if (tgt) *tgt = JabTarget{pb_id, ao1, ao2, n, base};
  contract_block<LA, LB, LC, LD, T>(A, X, w, ao1, ao2, __ldg(a.sp.ao1 + pk_id), __ldg(a.sp.ao2 + pk_id), base, n,
                                    jab_out);
}

template <int LA, int LB, int LC, int LD, typename T>
__global__ void __launch_bounds__(128) jk_thread_kernel(JKArgs A) {
  const KArgs& a = A.k;
  // items: positions in the work list, or (mixed precision) this tier's compacted list
  const bool compact = a.items != nullptr;
  const int64_t total = compact ? (int64_t)__ldg(a.nitems) : a.wl.total;
  const int64_t first = compact ? 0 : a.wl.first;
  const int nshard = compact ? 1 : a.wl.nshard, shard = compact ? 0 : a.wl.shard;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long done = 0, doneq = 0, doneb = 0;
  // a warp shares a tile of 32 * tile consecutive items, lane l takes items l, l + 32, ...
  const int64_t span = 32 * (int64_t)a.wl.tile, ntiles = (total - first + span - 1) / span;
  const int lane = threadIdx.x & 31;
  for (int64_t tl = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * nshard + shard; tl < ntiles;
       tl += (stride >> 5) * nshard) {
    const int64_t t0 = first + tl * span;
    const int64_t i1 = t0 + span < total ? t0 + span : total;
#if ERI_JAB_REDUCE
    if (A.Jh && !a.det) {
      // the list is bra-major: a warp's 32 items usually share the bra pair, so
      // their J_ab contributions are summed with shuffles (in FP64) and added
      // once; deterministic builds keep one fixed-point add per item, whose sum
      // does not depend on how items fall into warps
      using S = AShape<LA, LB, LC, LD>;
      BraCursor cur;
      if (!compact) cur.seek(a.wl, t0 + lane < i1 ? t0 + lane : t0);
      for (int64_t b0 = t0; b0 < i1; b0 += 32) {  // uniform over the warp; lane 0 always has an item
        const int64_t item = b0 + lane;
        const bool ok = item < i1;
        T jab[S::NAB];
        JabTarget tg{-1, 0, 0, 0, 0};
#pragma unroll
        for (int x = 0; x < S::NAB; ++x) jab[x] = T(0);
        if (ok) {
          int ib, ik;
          if (compact) {
            const int2 v = __ldg(a.items + item);
            ib = v.x;
            ik = v.y;
          } else {
            ik = cur.at(a.wl, item);
            ib = cur.ib;
          }
          thread_item<LA, LB, LC, LD, T>(A, ib, ik, done, doneq, doneb, jab, &tg);
        }
        const int pb0 = __shfl_sync(0xffffffffu, tg.pb_id, 0);
        if (__all_sync(0xffffffffu, !ok || tg.pb_id == pb0)) {
#pragma unroll
          for (int x = 0; x < S::NAB; ++x) {
            double v = (double)jab[x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) atomicAdd(A.Jh + tg.base + (size_t)(tg.ao1 + x / S::NB) * tg.n + tg.ao2 + x % S::NB, v);
          }
        } else if (ok) {
#pragma unroll
          for (int x = 0; x < S::NAB; ++x)
            acc_add(A.Jh + tg.base + (size_t)(tg.ao1 + x / S::NB) * tg.n + tg.ao2 + x % S::NB, (double)jab[x], a.det);
        }
      }
      continue;
    }
#endif
    const int64_t i0 = t0 + lane;
    if (i0 >= i1) continue;
    if (compact) {
      for (int64_t item = i0; item < i1; item += 32) {
        const int2 v = __ldg(a.items + item);
        thread_item<LA, LB, LC, LD, T>(A, v.x, v.y, done, doneq, doneb);
      }
    } else {
      BraCursor cur(a.wl, i0);
      for (int64_t item = i0; item < i1; item += 32) {
        const int ik = cur.at(a.wl, item);
        thread_item<LA, LB, LC, LD, T>(A, cur.ib, ik, done, doneq, doneb);
      }
    }
  }
  if (a.counter && done) {
    atomicAdd(a.counter, done);
    atomicAdd(a.counter + 1, doneq);
    atomicAdd(a.counter + 2, doneb);
  }
}

}  // namespace eri
