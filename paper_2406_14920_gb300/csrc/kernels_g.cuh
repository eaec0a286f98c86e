// Nuclear gradient of E = 1/2 tr(DJ) - 1/4 tr(DK) with D fixed (SI Sec. 1.4).
//
// Only bra derivatives are needed when the sum runs over every ordered pair
// of shell pairs (SI Eq. si_dE_J, si_dE_K).  Folding the four orderings inside
// the bra and ket pairs into one term gives, per ordered (bra pair, ket pair)
// item with shells (a b | c d),
//   dE/dR += w sum_{mu nu lam sig} G_{mu nu lam sig} d(mu nu|lam sig)/dR_bra,
//   G = 4 D_mn D_ls - D_ml D_ns - D_ms D_nl,  w = 1/2^[a=b] 1/2^[c=d].
// The bra derivative follows SI Eq. si_pair_derivative: in direction tau,
//   d/dA_tau: coefficient of Lambda_t is (a/p) E_{t-1} + E^{(1)}_t,
//   d/dB_tau: coefficient of Lambda_t is (b/p) E_{t-1} - E^{(1)}_t,
// with E^{(1)} = dE/dDelta_tau from the recurrence SI Eq. si_dE_recursion and
// base E^{00,(1)}_0 = 2a (P-A)_tau (the exp(-ab/p |AB|^2) factor of E^{00}_0
// lives in the pair prefactor).  Hermite indices run one higher than for the
// energy, so R goes to L+1 (the paper raises one bra angular momentum, SI Sec. 2).
// One warp per item, in FP64 or (mixed precision: quartets whose density-
// weighted bound is below tau, split on the device as for the energy) in FP32
// with the per-item sums added to the FP64 gradient.
#pragma once
#include "kernels_b.cuh"

#ifndef ERI_REGG
#define ERI_REGG 1
#endif

namespace eri {

struct GradArgs {
  PairData pd;
  ShellPairInfo sp;
  WorkList wl;  // ordered (J-engine) list
  BoysTabs bt;
  const RStep* rsteps;
  const double* Dp;
  const float* Dpf;    // D' in FP32 for the FP32 tier
  const double* ea;    // exponent of the s1 primitive of each primitive pair
  const int* sh_atom;
  double* grad;        // natom * 3 (all molecules' atoms)
  double cj, ck;       // weights of the Coulomb and exchange parts (1 or 0)
  double omega2;       // erf(omega r)/r: omega^2 (0 = Coulomb)
  float omega2f;
  int det;             // 1: fixed-point gradient accumulator (deterministic builds)
  unsigned long long* counter;  // items, primitive quartets, bra primitives of this launch (may be null)
  // mixed precision: this tier's compacted list (bra position, ket position) written
  // by the tier split, *nitems of them; null: items are positions in wl
  const int2* items;
  const unsigned int* nitems;
};

// E^{ij}_t and E^{ij,(1)}_t for one direction, i <= LI, j <= LJ, t <= i+j,
// stored with row length LI+LJ+2 (t = i+j+1 left zero).
template <int LI, int LJ, typename T>
__device__ __forceinline__ void md_e_deriv_1d(T PA, T PB, T o2p, T aop, T bop, T a2, T* E, T* E1) {
  constexpr int NT = LI + LJ + 2;
  for (int x = 0; x < (LI + 1) * (LJ + 1) * NT; ++x) {
    E[x] = T(0);
    E1[x] = T(0);
  }
  E[0] = T(1);
  E1[0] = a2 * PA;  // 2a (P-A)
  for (int i = 0; i < LI; ++i) {
    const T* s0 = E + (i * (LJ + 1)) * NT;
    const T* s1 = E1 + (i * (LJ + 1)) * NT;
    T* d0 = E + ((i + 1) * (LJ + 1)) * NT;
    T* d1 = E1 + ((i + 1) * (LJ + 1)) * NT;
    for (int t = 0; t <= i + 1; ++t) {
      T v = PA * s0[t], w = PA * s1[t] - bop * s0[t];
      if (t > 0) {
        v += o2p * s0[t - 1];
        w += o2p * s1[t - 1];
      }
      if (t + 1 <= i) {
        v += (t + 1) * s0[t + 1];
        w += (t + 1) * s1[t + 1];
      }
      d0[t] = v;
      d1[t] = w;
    }
  }
  for (int i = 0; i <= LI; ++i)
    for (int j = 0; j < LJ; ++j) {
      const T* s0 = E + (i * (LJ + 1) + j) * NT;
      const T* s1 = E1 + (i * (LJ + 1) + j) * NT;
      T* d0 = E + (i * (LJ + 1) + j + 1) * NT;
      T* d1 = E1 + (i * (LJ + 1) + j + 1) * NT;
      for (int t = 0; t <= i + j + 1; ++t) {
        T v = PB * s0[t], w = PB * s1[t] + aop * s0[t];
        if (t > 0) {
          v += o2p * s0[t - 1];
          w += o2p * s1[t - 1];
        }
        if (t + 1 <= i + j) {
          v += (t + 1) * s0[t + 1];
          w += (t + 1) * s1[t + 1];
        }
        d0[t] = v;
        d1[t] = w;
      }
    }
}

template <int LA, int LB, int LC, int LD, typename T = double>
struct GShape {
  static constexpr int LAB = LA + LB, LCD = LC + LD, L1 = LAB + LCD + 1;
  static constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  static constexpr int NAB = NA * NB, NCD = NC * ND, HAB1 = nherm(LAB + 1), HAB1P = HAB1 | 1;
  static constexpr int B = L1 + 1, BOX = B * B * B, NPING = nherm(L1 - 1);
  static constexpr int NTB = LAB + 2;
  static constexpr int NEB = (LA + 1) * (LB + 1) * NTB, NEK = (LC + 1) * (LD + 1) * (LCD + 1);
  static constexpr int NSC = L1 + 5;
  static constexpr int FIXED = 9 * NEB;  // E, GA, GB per direction
  static constexpr int PER_G = BOX + 2 * NPING + NSC + 3 * NEK;
  static constexpr int PER_C = HAB1P;
  // ket-primitive batch sized as for the energy kernel (BShape)
  static constexpr int BASE = sizeof(T) == 8 ? (ERI_WARP_SMEM64_KB * 1024) / 8 : (ERI_WARP_SMEM32_KB * 1024) / 4;
  static constexpr int MAXB = sizeof(T) == 8 ? (ERI_WARP_SMEM64_MAX_KB * 1024) / 8 : (ERI_WARP_SMEM32_MAX_KB * 1024) / 4;
  static constexpr int GTARGET = (LC <= 1 && LD <= 1) ? 9 : 3;
  static constexpr int fit_g(int budget) { return (budget - FIXED - NCD * PER_C) / PER_G; }
  static constexpr int GMAXB = fit_g(MAXB) < 1 ? 1 : fit_g(MAXB);
  static constexpr int NBATCH = (GTARGET + GMAXB - 1) / GMAXB;
  static constexpr int GWANT = (GTARGET + NBATCH - 1) / NBATCH;
  static constexpr int NEED = FIXED + NCD * PER_C + GWANT * PER_G;
  static constexpr int BUDGET = NEED <= BASE ? BASE : (NEED <= MAXB ? NEED : MAXB);
  static constexpr int G0 = (BUDGET - FIXED - NCD * PER_C) / PER_G;
  static constexpr int G = G0 >= 1 ? (G0 > 16 ? 16 : G0) : 1;
  static constexpr int CHMAX = (BUDGET - FIXED - G * PER_G) / PER_C;
  static constexpr int CH = CHMAX >= NCD ? NCD : (CHMAX < 1 ? 1 : CHMAX);
  // register ket transform (as in the energy kernel) where W fits
  static constexpr int NPS = (HAB1 + 31) / 32;
  static constexpr bool REGW = CH == NCD && (sizeof(T) == 4 ? NCD * NPS <= 64 : (ERI_REGW64 && NCD * NPS <= 32));
  // derivative contraction with compile-time indices: lane owns ket pair
  // cd = lane + 32 j, the bra pairs ab are an unrolled loop (coefficients
  // broadcast from shared memory, the W row at a per-lane base, the lane's
  // density values in registers); worth it when most lanes own a cd
  static constexpr int NCS = (NCD + 31) / 32;
  static constexpr bool REGG = ERI_REGG && CH == NCD && NCD >= 16;
  static constexpr int SM_BOX = 0, SM_PING = SM_BOX + G * BOX, SM_SC = SM_PING + G * 2 * NPING,
                       SM_EK = SM_SC + G * NSC, SM_EB = SM_EK + G * 3 * NEK, SM_W = SM_EB + FIXED,
                       SM_TOTAL = SM_W + CH * HAB1P;
  __host__ __device__ static constexpr size_t smem_per_warp() { return sizeof(T) * SM_TOTAL; }
  static constexpr int LEXB = (LAB + 2) * (LAB + 2);
  static constexpr int TAB_INTS = 2 * NCD + 2 * NAB + HAB1 + LEXB;
  static constexpr int TABLE_BYTES = ((4 * TAB_INTS + 15) / 16) * 16;
  __host__ __device__ static constexpr size_t table_bytes() { return TABLE_BYTES; }
};

template <int LA, int LB, int LC, int LD, typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 2 : 0) grad_warp_kernel(GradArgs a) {
  using S = GShape<LA, LB, LC, LD, T>;
  constexpr int LAB = S::LAB, LCD = S::LCD, L = S::L1, B = S::B, BOX = S::BOX, NSC = S::NSC;
  constexpr int NB = S::NB, ND = S::ND, NAB = S::NAB, NCD = S::NCD, HAB = S::HAB1, HABP = S::HAB1P, CH = S::CH,
                G = S::G, NEB = S::NEB, NEK = S::NEK, NPING = S::NPING, NTB = S::NTB;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int* tab_cd = reinterpret_cast<int*>(smraw);
  int* tab_ab = tab_cd + 2 * NCD;
  int* tab_p = tab_ab + 2 * NAB;
  int* tab_lex = tab_p + HAB;
  for (int i = threadIdx.x; i < NCD; i += blockDim.x) {
    int kx, ky, kz, lx, ly, lz;
    cart_xyz(LC, i / ND, kx, ky, kz);
    cart_xyz(LD, i % ND, lx, ly, lz);
    tab_cd[2 * i] = ((kx * (LD + 1) + lx) * (LCD + 1)) | ((NEK + (ky * (LD + 1) + ly) * (LCD + 1)) << 10) |
                    ((2 * NEK + (kz * (LD + 1) + lz) * (LCD + 1)) << 20);
    tab_cd[2 * i + 1] = (kx + lx) | ((ky + ly) << 4) | ((kz + lz) << 8);
  }
  for (int i = threadIdx.x; i < NAB; i += blockDim.x) {
    int ix, iy, iz, jx, jy, jz;
    cart_xyz(LA, i / NB, ix, iy, iz);
    cart_xyz(LB, i % NB, jx, jy, jz);
    tab_ab[2 * i] = ((ix * (LB + 1) + jx) * NTB) | ((iy * (LB + 1) + jy) * NTB << 10) | ((iz * (LB + 1) + jz) * NTB << 20);
    tab_ab[2 * i + 1] = (ix + jx) | ((iy + jy) << 4) | ((iz + jz) << 8);
  }
  for (int i = threadIdx.x; i < HAB; i += blockDim.x) {
    const int t = herm_t(i), u = herm_u(i), v = herm_v(i);
    tab_p[i] = ((t * B + u) * B + v) | ((lex_base(LAB + 1, t, u) + v) << 16);
  }
  for (int i = threadIdx.x; i < S::LEXB; i += blockDim.x) {
    const int t = i / (LAB + 2), u = i % (LAB + 2);
    tab_lex[i] = (t + u <= LAB + 1) ? lex_base(LAB + 1, t, u) : 0;
  }
  __syncthreads();
  int pslot[S::NPS];  // box offset of this lane's Hermite indices P = lane + 32 j
#pragma unroll
  for (int j = 0; j < S::NPS; ++j) pslot[j] = lane + 32 * j < HAB ? (tab_p[lane + 32 * j] & 0xffff) : 0;
  T* sm = reinterpret_cast<T*>(smraw + S::table_bytes()) + (size_t)wib * S::SM_TOTAL;
  T* boxes = sm + S::SM_BOX;
  T* pings = sm + S::SM_PING;
  T* scal = sm + S::SM_SC;
  T* Ek = sm + S::SM_EK;
  T* Eb = sm + S::SM_EB;  // [d][E | GA | GB][NEB]
  T* Ws = sm + S::SM_W;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  // items: positions in the ordered list, or (mixed precision) this tier's compacted list
  const bool compact = a.items != nullptr;
  const int64_t total = compact ? (int64_t)__ldg(a.nitems) : a.wl.total;
  const int64_t first = compact ? 0 : a.wl.first;
  const int nshard = compact ? 1 : a.wl.nshard, shard = compact ? 0 : a.wl.shard;
  unsigned long long done = 0, doneq = 0, doneb = 0;
  const int64_t tile = a.wl.tile, ntiles = (total - first + tile - 1) / tile;
  for (int64_t tl = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * nshard + shard; tl < ntiles;
       tl += nwarps * nshard) {
  const int64_t i0 = first + tl * tile, i1 = i0 + tile < total ? i0 + tile : total;
  BraCursor cur;
  if (!compact) cur.seek(a.wl, i0);
  for (int64_t item = i0; item < i1; ++item) {
    int ik, ib;
    if (compact) {
      const int2 v = __ldg(a.items + item);
      ib = v.x;
      ik = v.y;
    } else {
      ik = cur.at(a.wl, item);
      ib = cur.ib;
    }
    const int pb_id = __ldg(a.wl.bra + ib);
    const int mol = __ldg(a.sp.pmol + pb_id);
    const int pk_id = __ldg(a.wl.ket + __ldg(a.wl.kseg + mol * NPAIRCLASS) + ik);
    const int s1 = __ldg(a.sp.s1 + pb_id), s2 = __ldg(a.sp.s2 + pb_id);
    const int s3 = __ldg(a.sp.s1 + pk_id), s4 = __ldg(a.sp.s2 + pk_id);
    const int npb = __ldg(a.sp.np + pb_id), offb = __ldg(a.sp.poff + pb_id);
    const int npk = __ldg(a.sp.np + pk_id), offk = __ldg(a.sp.poff + pk_id), ek0 = __ldg(a.sp.eoff + pk_id);
    const int ao1 = __ldg(a.sp.ao1 + pb_id), ao2 = __ldg(a.sp.ao2 + pb_id);
    const int ao3 = __ldg(a.sp.ao1 + pk_id), ao4 = __ldg(a.sp.ao2 + pk_id);
    ++done;
    doneq += (unsigned long long)npb * npk;
    doneb += npb;
    T w = T(1);
    if (s1 == s2) w *= T(0.5);
    if (s3 == s4) w *= T(0.5);
    const int n = __ldg(a.sp.mat_n + mol);
    const T* Dp = (sizeof(T) == 8 ? reinterpret_cast<const T*>(a.Dp) : reinterpret_cast<const T*>(a.Dpf)) +
                  __ldg(a.sp.mat_off + mol);
    T gA[3] = {T(0), T(0), T(0)}, gB[3] = {T(0), T(0), T(0)};

    for (int c0 = 0; c0 < NCD; c0 += CH) {
      const int nci = NCD - c0 < CH ? NCD - c0 : CH;
      for (int pb = 0; pb < npb; ++pb) {
        const int ipb = offb + pb;
        const T bp_p = pdv<T>(a.pd.p, a.pd.pf, ipb), bp_pref = pdv<T>(a.pd.pref, a.pd.preff, ipb);
        if (lane < 3) {
          const T aa = (T)__ldg(a.ea + ipb);
          const T aop = aa / bp_p, bop = T(1) - aop;
          T* e = Eb + lane * 3 * NEB;
          T* ga = e + NEB;
          T* gb = e + 2 * NEB;
          md_e_deriv_1d<LA, LB, T>(pdv<T>(a.pd.PA, a.pd.PAf, lane * a.pd.n + ipb),
                                   pdv<T>(a.pd.PB, a.pd.PBf, lane * a.pd.n + ipb), T(0.5) / bp_p, aop, bop,
                                   T(2) * aa, e, ga);
          // ga currently holds E^(1); form GA, GB in place (t from high to low)
          for (int r = 0; r < (LA + 1) * (LB + 1); ++r) {
            T* er = e + r * NTB;
            T* ar = ga + r * NTB;
            T* br = gb + r * NTB;
            for (int t = NTB - 1; t >= 0; --t) {
              const T em1 = t > 0 ? er[t - 1] : T(0);
              const T e1 = ar[t];
              ar[t] = aop * em1 + e1;
              br[t] = bop * em1 - e1;
            }
          }
        }
        T wreg[S::REGW ? S::NPS * NCD : 1];
        if constexpr (S::REGW) {
#pragma unroll
          for (int x = 0; x < S::NPS * NCD; ++x) wreg[x] = T(0);
        } else {
          for (int x = lane; x < CH * HABP; x += 32) Ws[x] = T(0);
        }
        const T bPx = pdv<T>(a.pd.P, a.pd.Pf, ipb), bPy = pdv<T>(a.pd.P, a.pd.Pf, a.pd.n + ipb),
                bPz = pdv<T>(a.pd.P, a.pd.Pf, 2 * a.pd.n + ipb);
        for (int k0 = 0; k0 < npk; k0 += G) {
          const int ng = npk - k0 < G ? npk - k0 : G;
          for (int x = lane; x < ng * 3 * NEK; x += 32) {
            const int g = x / (3 * NEK), r = x - g * 3 * NEK;
            const T v = ldE<T>(a.pd, ek0 + (k0 + g) * 3 * NEK + r);
            Ek[x] = ((r % (LCD + 1)) & 1) ? -v : v;
          }
          if (lane < ng) {
            const int ipk = offk + k0 + lane;
            const T kp = pdv<T>(a.pd.p, a.pd.pf, ipk);
            const T ps = bp_p + kp;
            T rho = bp_p * kp / ps;
            T pref = bp_pref * pdv<T>(a.pd.pref, a.pd.preff, ipk) * rsqrt_t(ps);
            // s depends on exponents only: the derivative rules hold as they are
            attenuate(sizeof(T) == 8 ? T(a.omega2) : T(a.omega2f), rho, pref);
            const T X = bPx - pdv<T>(a.pd.P, a.pd.Pf, ipk), Y = bPy - pdv<T>(a.pd.P, a.pd.Pf, a.pd.n + ipk),
                    Z = bPz - pdv<T>(a.pd.P, a.pd.Pf, 2 * a.pd.n + ipk);
            T F[L + 1];
            Boys<T>::template eval<L>(rho * (X * X + Y * Y + Z * Z), a.bt, F);
            T* sc = scal + lane * NSC;
#pragma unroll
            for (int m = 0; m <= L; ++m) sc[m] = pref * F[m];
            sc[L + 1] = X;
            sc[L + 2] = Y;
            sc[L + 3] = Z;
            sc[L + 4] = T(-2) * rho;
          }
          __syncwarp();
          if (lane < ng) pings[lane * 2 * NPING] = scal[lane * NSC + L];
          __syncwarp();
          int cur = 0;
#pragma unroll
          for (int m = L - 1; m >= 0; --m) {
            const int ne = nherm(L - m);
            for (int it = lane; it < ng * ne; it += 32) {
              const int g = it / ne, e = it - g * ne;
              const T* sc = scal + g * NSC;
              const T* src = pings + g * 2 * NPING + cur * NPING;
              const RStep st = a.rsteps[e];
              T val;
              if (e == 0) {
                val = sc[m];
              } else {
                const T pq = sc[L + 1 + st.dir];
                val = pq * src[st.dep1];
                if (st.dep2 >= 0) val = fma((T)st.k, src[st.dep2], val);
                val *= sc[L + 4];
              }
              if (m == 0) boxes[g * BOX + (st.t * B + st.u) * B + st.v] = val;
              else pings[g * 2 * NPING + (1 - cur) * NPING + e] = val;
            }
            __syncwarp();
            cur = 1 - cur;
          }
          // ket transform, P over Hermite indices up to LAB+1
          if constexpr (S::REGW) {
            for (int g = 0; g < ng; ++g) {
              const T* ek = Ek + g * 3 * NEK;
              const T* rbox = boxes + g * BOX;
              for_cart<LC>([&](auto kx, auto ky, auto kz) {
                for_cart<LD>([&](auto lx, auto ly, auto lz) {
                  constexpr int KX = ERI_CI(kx), KY = ERI_CI(ky), KZ = ERI_CI(kz);
                  constexpr int LX = ERI_CI(lx), LY = ERI_CI(ly), LZ = ERI_CI(lz);
                  constexpr int icd = cidx(LC, KY, KZ) * ND + cidx(LD, LY, LZ);
                  const T* ex = ek + (KX * (LD + 1) + LX) * (LCD + 1);
                  const T* ey = ek + NEK + (KY * (LD + 1) + LY) * (LCD + 1);
                  const T* ez = ek + 2 * NEK + (KZ * (LD + 1) + LZ) * (LCD + 1);
                  sfor<S::NPS>([&](auto j_) {
                    constexpr int j = ERI_CI(j_);
                    if (j * 32 + 32 <= HAB || lane + 32 * j < HAB) {
                      const T* r = rbox + pslot[j];
                      wreg[j * NCD + icd] += tsum<KX + LX, KY + LY, KZ + LZ, false>(
                          ex, ey, ez, [&](auto sx, auto sy, auto sz) {
                            return r[(ERI_CI(sx) * B + ERI_CI(sy)) * B + ERI_CI(sz)];
                          });
                    }
                  });
                });
              });
            }
          } else {
          for (int it = lane; it < nci * HAB; it += 32) {
            const int ci = it / HAB, P = it - ci * HAB;
            const int c0w = tab_cd[2 * (c0 + ci)], c1w = tab_cd[2 * (c0 + ci) + 1];
            const int ox = c0w & 1023, oy = (c0w >> 10) & 1023, oz = c0w >> 20;
            const int nx = c1w & 15, ny = (c1w >> 4) & 15, nz = c1w >> 8;
            const int pw = tab_p[P];
            const int base = pw & 0xffff;
            T acc = T(0);
            for (int g = 0; g < ng; ++g) {
              const T* ek = Ek + g * 3 * NEK;
              const T* rb = boxes + g * BOX + base;
              for (int sx = 0; sx <= nx; ++sx) {
                T accy = T(0);
                for (int sy = 0; sy <= ny; ++sy) {
                  const T* r = rb + sx * B * B + sy * B;
                  T accz = T(0);
                  for (int sz = 0; sz <= nz; ++sz) accz = fma(ek[oz + sz], r[sz], accz);
                  accy = fma(ek[oy + sy], accz, accy);
                }
                acc = fma(ek[ox + sx], accy, acc);
              }
            }
            Ws[ci * HABP + (pw >> 16)] += acc;
          }
          }
          __syncwarp();
        }
        if constexpr (S::REGW) {
#pragma unroll
          for (int j = 0; j < S::NPS; ++j)
            if (lane + 32 * j < HAB) {
              const int slot = tab_p[lane + 32 * j] >> 16;
#pragma unroll
              for (int icd = 0; icd < NCD; ++icd) Ws[icd * HABP + slot] = wreg[j * NCD + icd];
            }
          __syncwarp();
        }
        // bra derivatives and contraction with G
        if constexpr (S::REGG) {
          sfor<S::NCS>([&](auto j_) {
            constexpr int j = ERI_CI(j_);
            const int cd = lane + 32 * j;
            if (j * 32 + 32 <= NCD || cd < NCD) {
              constexpr int NA = S::NA;
              const T* wc = Ws + cd * HABP;
              const int lam = ao3 + cd / ND, sig = ao4 + cd % ND;
              const T Dls = __ldg(Dp + (size_t)lam * n + sig);
              T Dml[NA], Dms[NA], Dnl[NB], Dns[NB];
#pragma unroll
              for (int x = 0; x < NA; ++x) {
                Dml[x] = __ldg(Dp + (size_t)(ao1 + x) * n + lam);
                Dms[x] = __ldg(Dp + (size_t)(ao1 + x) * n + sig);
              }
#pragma unroll
              for (int x = 0; x < NB; ++x) {
                Dnl[x] = __ldg(Dp + (size_t)(ao2 + x) * n + lam);
                Dns[x] = __ldg(Dp + (size_t)(ao2 + x) * n + sig);
              }
              for_cart<LA>([&](auto ix, auto iy, auto iz) {
                for_cart<LB>([&](auto jx, auto jy, auto jz) {
                  constexpr int IX = ERI_CI(ix), IY = ERI_CI(iy), IZ = ERI_CI(iz);
                  constexpr int JX = ERI_CI(jx), JY = ERI_CI(jy), JZ = ERI_CI(jz);
                  constexpr int ia = cidx(LA, IY, IZ), ib = cidx(LB, JY, JZ);
                  constexpr int NX = IX + JX, NY = IY + JY, NZ = IZ + JZ;
                  const T* ex = Eb + 0 * 3 * NEB + (IX * (LB + 1) + JX) * NTB;
                  const T* ey = Eb + 1 * 3 * NEB + (IY * (LB + 1) + JY) * NTB;
                  const T* ez = Eb + 2 * 3 * NEB + (IZ * (LB + 1) + JZ) * NTB;
                  const T Gv = T(4.0 * a.cj) * __ldg(Dp + (size_t)(ao1 + ia) * n + ao2 + ib) * Dls -
                               T(a.ck) * (Dml[ia] * Dns[ib] + Dms[ia] * Dnl[ib]);
                  auto w = [&](int tx, int ty, int tz) { return wc[lex_base(LAB + 1, tx, ty) + tz]; };
                  T dAx = T(0), dBx = T(0), dAy = T(0), dBy = T(0), dAz = T(0), dBz = T(0);
                  sfor<NX + 2>([&](auto tx_) {  // direction x open to NX + 1
                    constexpr int tx = ERI_CI(tx_);
                    T sx = T(0);
                    sfor<NY + 1>([&](auto ty_) {
                      constexpr int ty = ERI_CI(ty_);
                      T sz = T(0);
                      sfor<NZ + 1>([&](auto tz_) { sz = fma(ez[ERI_CI(tz_)], w(tx, ty, ERI_CI(tz_)), sz); });
                      sx = fma(ey[ty], sz, sx);
                    });
                    dAx = fma(ex[NEB + tx], sx, dAx);
                    dBx = fma(ex[2 * NEB + tx], sx, dBx);
                  });
                  sfor<NY + 2>([&](auto ty_) {  // direction y open
                    constexpr int ty = ERI_CI(ty_);
                    T sy = T(0);
                    sfor<NX + 1>([&](auto tx_) {
                      constexpr int tx = ERI_CI(tx_);
                      T sz = T(0);
                      sfor<NZ + 1>([&](auto tz_) { sz = fma(ez[ERI_CI(tz_)], w(tx, ty, ERI_CI(tz_)), sz); });
                      sy = fma(ex[tx], sz, sy);
                    });
                    dAy = fma(ey[NEB + ty], sy, dAy);
                    dBy = fma(ey[2 * NEB + ty], sy, dBy);
                  });
                  sfor<NZ + 2>([&](auto tz_) {  // direction z open
                    constexpr int tz = ERI_CI(tz_);
                    T sz = T(0);
                    sfor<NX + 1>([&](auto tx_) {
                      constexpr int tx = ERI_CI(tx_);
                      T sy = T(0);
                      sfor<NY + 1>([&](auto ty_) { sy = fma(ey[ERI_CI(ty_)], w(tx, ERI_CI(ty_), tz), sy); });
                      sz = fma(ex[tx], sy, sz);
                    });
                    dAz = fma(ez[NEB + tz], sz, dAz);
                    dBz = fma(ez[2 * NEB + tz], sz, dBz);
                  });
                  gA[0] = fma(Gv, dAx, gA[0]);
                  gA[1] = fma(Gv, dAy, gA[1]);
                  gA[2] = fma(Gv, dAz, gA[2]);
                  gB[0] = fma(Gv, dBx, gB[0]);
                  gB[1] = fma(Gv, dBy, gB[1]);
                  gB[2] = fma(Gv, dBz, gB[2]);
                });
              });
            }
          });
        } else {
        // items (ab, ci)
        for (int it = lane; it < NAB * nci; it += 32) {
          const int iab = it / nci, ci = it - iab * nci;
          const int cd = c0 + ci;
          const int mu = ao1 + iab / NB, nu = ao2 + iab % NB, la = ao3 + cd / ND, si = ao4 + cd % ND;
          const T Gv = T(4.0 * a.cj) * __ldg(Dp + (size_t)mu * n + nu) * __ldg(Dp + (size_t)la * n + si) -
                       T(a.ck) * (__ldg(Dp + (size_t)mu * n + la) * __ldg(Dp + (size_t)nu * n + si) +
                               __ldg(Dp + (size_t)mu * n + si) * __ldg(Dp + (size_t)nu * n + la));
          const int a0w = tab_ab[2 * iab], a1w = tab_ab[2 * iab + 1];
          const int fxo = a0w & 1023, fyo = (a0w >> 10) & 1023, fzo = a0w >> 20;
          const int nx = a1w & 15, ny = (a1w >> 4) & 15, nz = a1w >> 8;
          const T* wc = Ws + ci * HABP;
          // direction x open: Sx[tx] = sum_ty Ey sum_tz Ez W
          const T* ex = Eb + 0 * 3 * NEB + fxo;
          const T* ey = Eb + 1 * 3 * NEB + fyo;
          const T* ez = Eb + 2 * 3 * NEB + fzo;
          T dA[3] = {0, 0, 0}, dB[3] = {0, 0, 0};
          for (int tx = 0; tx <= nx + 1; ++tx) {
            T s = T(0);
            for (int ty = 0; ty <= ny; ++ty) {
              const T* wr = wc + tab_lex[tx * (LAB + 2) + ty];
              T sz = T(0);
              for (int tz = 0; tz <= nz; ++tz) sz = fma(ez[tz], wr[tz], sz);
              s = fma(ey[ty], sz, s);
            }
            dA[0] = fma(ex[NEB + tx], s, dA[0]);
            dB[0] = fma(ex[2 * NEB + tx], s, dB[0]);
          }
          for (int ty = 0; ty <= ny + 1; ++ty) {
            T s = T(0);
            for (int tx = 0; tx <= nx; ++tx) {
              const T* wr = wc + tab_lex[tx * (LAB + 2) + ty];
              T sz = T(0);
              for (int tz = 0; tz <= nz; ++tz) sz = fma(ez[tz], wr[tz], sz);
              s = fma(ex[tx], sz, s);
            }
            dA[1] = fma(ey[NEB + ty], s, dA[1]);
            dB[1] = fma(ey[2 * NEB + ty], s, dB[1]);
          }
          for (int tz = 0; tz <= nz + 1; ++tz) {
            T s = T(0);
            for (int tx = 0; tx <= nx; ++tx) {
              T sy = T(0);
              for (int ty = 0; ty <= ny; ++ty) sy = fma(ey[ty], wc[tab_lex[tx * (LAB + 2) + ty] + tz], sy);
              s = fma(ex[tx], sy, s);
            }
            dA[2] = fma(ez[NEB + tz], s, dA[2]);
            dB[2] = fma(ez[2 * NEB + tz], s, dB[2]);
          }
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            gA[d] = fma(Gv, dA[d], gA[d]);
            gB[d] = fma(Gv, dB[d], gB[d]);
          }
        }
        }
        __syncwarp();
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
      for (int o = 16; o > 0; o >>= 1) {
        gA[d] += __shfl_xor_sync(0xffffffffu, gA[d], o);
        gB[d] += __shfl_xor_sync(0xffffffffu, gB[d], o);
      }
    if (lane == 0) {
      const int atA = __ldg(a.sh_atom + s1), atB = __ldg(a.sh_atom + s2);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        acc_add(a.grad + atA * 3 + d, w * gA[d], a.det);
        acc_add(a.grad + atB * 3 + d, w * gB[d], a.det);
      }
    }
    __syncwarp();
  }
  }
  if (a.counter && lane == 0 && done) {
    atomicAdd(a.counter, done);
    atomicAdd(a.counter + 1, doneq);
    atomicAdd(a.counter + 2, doneb);
  }
}

}  // namespace eri
