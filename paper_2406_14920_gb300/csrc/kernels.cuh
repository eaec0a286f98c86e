// Class-specialised ERI kernels: exchange (K) by Cartesian ERIs and Coulomb (J)
// by the J-engine.  One specialisation per angular-momentum class, as in the
// paper (Sec. 3.3), but one warp per shell quartet instead of the paper's 8x8
// block of primitive pairs: GB300's FP64 pipe costs the same per warp
// instruction whether 1 or 32 lanes are active, so every loop below keeps its
// trip count uniform across the warp.
#pragma once
#include "common.cuh"

namespace eri {

struct KArgs {
  PairData pd;
  ShellPairInfo sp;
  WorkList wl;
  const double* boys64;
  const float* boys32;
  const RStep* rsteps;
  const double* Dp;   // density with component norms folded in, nbf x nbf
  double* Kh;         // half-K accumulator, nbf x nbf
  const uint8_t* tier;  // optional per-item precision tier (nullptr: all items)
  int tier_want;
  int nbf;
  int same_class;
};

struct JArgs {
  PairData pd;
  ShellPairInfo sp;
  WorkList wl;
  const double* boys64;
  const float* boys32;
  const RStep* rsteps;
  const double* Dherm;  // Hermite density per ket primitive pair (sign (-1)^|Q| folded in)
  double* Jherm;        // Hermite J per bra primitive pair (accumulated)
  const uint8_t* tier;
  int tier_want;
};

__device__ __forceinline__ int find_bra(const int64_t* __restrict__ prefix, int n, int64_t item) {
  int lo = 0, hi = n;  // prefix[lo] <= item < prefix[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= item) lo = mid; else hi = mid;
  }
  return lo;
}

template <typename T> __device__ __forceinline__ T ldT(const double* p) { return (T)__ldg(p); }
template <typename T> __device__ __forceinline__ T pdv(const double* d, const float* f, int i);
template <> __device__ __forceinline__ double pdv<double>(const double* d, const float*, int i) { return __ldg(d + i); }
template <> __device__ __forceinline__ float pdv<float>(const double*, const float* f, int i) { return __ldg(f + i); }

// Primitive pair scalars in precision T.
template <typename T>
struct Prim {
  T p, P[3], PA[3], PB[3], pref;
  __device__ __forceinline__ void load(const PairData& pd, int i) {
    p = pdv<T>(pd.p, pd.pf, i);
    pref = pdv<T>(pd.pref, pd.preff, i);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      P[d] = pdv<T>(pd.P, pd.Pf, d * pd.n + i);
      PA[d] = pdv<T>(pd.PA, pd.PAf, d * pd.n + i);
      PB[d] = pdv<T>(pd.PB, pd.PBf, d * pd.n + i);
    }
  }
};

// Warp-cooperative R^0_{tuv} for t+u+v <= L (Eq. R_recursion) in the scaled
// form r^m = R^m / (-2 rho)^m, which keeps intermediates near (2 rho)^(n/2)
// instead of (2 rho)^m (FP32 range):
//   r^m_000 = pref * F_m(T),  r^m_{t+1,u,v} = c (t r^{m+1}_{t-1,u,v} + X r^{m+1}_{t,u,v}), c = -2 rho.
// Level 0 is written into a (L+1)^3 box so that R_{P+Q} addressing is affine.
template <int L, typename T>
__device__ __forceinline__ void r_build_warp(const T* F, T pref, T X, T Y, T Z, T c, const RStep* __restrict__ st,
                                             T* ping0, T* ping1, T* box, int lane) {
  constexpr int B = L + 1;
  if (L == 0) {
    if (lane == 0) box[0] = pref * F[0];
    __syncwarp();
    return;
  }
  if (lane == 0) ping0[0] = pref * F[L];
  __syncwarp();
  T* cur = ping0;
  T* nxt = ping1;
#pragma unroll
  for (int m = L - 1; m >= 0; --m) {
    const int ne = nherm(L - m);
    for (int e = lane; e < ne; e += 32) {
      T val;
      RStep s = st[e];
      if (e == 0) {
        val = pref * F[m];
      } else {
        T pq = s.dir == 0 ? X : (s.dir == 1 ? Y : Z);
        val = pq * cur[s.dep1];
        if (s.dep2 >= 0) val = fma((T)s.k, cur[s.dep2], val);
        val *= c;
      }
      if (m == 0) box[(s.t * B + s.u) * B + s.v] = val;
      else nxt[e] = val;
    }
    __syncwarp();
    T* tmp = cur; cur = nxt; nxt = tmp;
  }
}

template <int LA, int LB, int LC, int LD, typename T>
struct KShape {
  static constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
  static constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  static constexpr int NCD = NC * ND, HAB = nherm(LAB), B = L + 1, BOX = B * B * B;
  static constexpr int WS = HAB | 1;
  static constexpr int NEB = (LA + 1) * (LB + 1) * (LAB + 1), NEK = (LC + 1) * (LD + 1) * (LCD + 1);
  static constexpr int NPING = L > 0 ? nherm(L - 1) : 1;
  static constexpr int NPS = (HAB + 31) / 32;
  // per-warp shared memory, in elements of T
  static constexpr int SM_BOX = 0, SM_PING = BOX, SM_W = SM_PING + 2 * NPING, SM_EB = SM_W + 32 * WS,
                       SM_EK = SM_EB + 3 * NEB, SM_KB = SM_EK + 3 * NEK, SM_TOTAL = SM_KB + 2 * NB * 32;
  static constexpr size_t smem_per_warp() { return sizeof(T) * SM_TOTAL; }
};

// Exchange over canonical shell quartets (ab|cd), bra class >= ket class.
//   phase 1 (ket transform, lanes own bra Hermite index P):
//     W_P[cd] = sum_Q E'_Q^{cd} R_{P+Q},  E' = (-1)^|Q| E      (Eq. eri_formula)
//   phase 2 (bra transform, lanes own ket pair cd):
//     (ab|cd) = sum_P E_P^{ab} W_P[cd],
//   then Kh_ac += w (ab|cd) D_bd, Kh_ad += w (ab|cd) D_bc, Kh_bc += w (ab|cd) D_ad,
//   Kh_bd += w (ab|cd) D_ac (Eq. k_definition), w = 1/2^[a=b] 1/2^[c=d] 1/2^[ab=cd];
//   K = Kh + Kh^T afterwards restores all eight permutations (Eq. 8_fold_symmetry).
template <int LA, int LB, int LC, int LD, typename T>
__global__ void __launch_bounds__(128) k_warp_kernel(KArgs a) {
  using S = KShape<LA, LB, LC, LD, T>;
  constexpr int LAB = S::LAB, LCD = S::LCD, L = S::L, B = S::B;
  constexpr int NA = S::NA, NB = S::NB, ND = S::ND, NCD = S::NCD, HAB = S::HAB, WS = S::WS;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  T* sm = reinterpret_cast<T*>(smraw) + (size_t)wib * S::SM_TOTAL;
  T* box = sm + S::SM_BOX;
  T* ping0 = sm + S::SM_PING;
  T* ping1 = ping0 + S::NPING;
  T* W = sm + S::SM_W;
  T* Eb = sm + S::SM_EB;
  T* Ek = sm + S::SM_EK;
  T* Kb = sm + S::SM_KB;

  int pbase[S::NPS];
#pragma unroll
  for (int j = 0; j < S::NPS; ++j) {
    int P = lane + 32 * j;
    pbase[j] = 0;
    if (P < HAB) {
      RStep s = a.rsteps[P];
      pbase[j] = (s.t * B + s.u) * B + s.v;
    }
  }
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t total = a.wl.total;
  const int nbf = a.nbf;
  for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; item < total; item += nwarps) {
    if (a.tier && a.tier[item] != a.tier_want) continue;
    const int ib = find_bra(a.wl.prefix, a.wl.nbra, item);
    const int ik = (int)(item - __ldg(a.wl.prefix + ib));
    const int pb_id = __ldg(a.wl.bra + ib), pk_id = __ldg(a.wl.ket + ik);
    const int s1 = __ldg(a.sp.s1 + pb_id), s2 = __ldg(a.sp.s2 + pb_id);
    const int s3 = __ldg(a.sp.s1 + pk_id), s4 = __ldg(a.sp.s2 + pk_id);
    const int npb = __ldg(a.sp.np + pb_id), offb = __ldg(a.sp.poff + pb_id);
    const int npk = __ldg(a.sp.np + pk_id), offk = __ldg(a.sp.poff + pk_id);
    const int ao1 = __ldg(a.sp.ao1 + pb_id), ao2 = __ldg(a.sp.ao2 + pb_id);
    const int ao3 = __ldg(a.sp.ao1 + pk_id), ao4 = __ldg(a.sp.ao2 + pk_id);
    T w = T(1);
    if (s1 == s2) w *= T(0.5);
    if (s3 == s4) w *= T(0.5);
    if (pb_id == pk_id) w *= T(0.5);

    for (int c0 = 0; c0 < NCD; c0 += 32) {
      const int nci = NCD - c0 < 32 ? NCD - c0 : 32;
      const int cd = c0 + lane;
      const bool cdv = lane < nci;
      const int ic = cdv ? cd / ND : 0, id = cdv ? cd % ND : 0;
      // a-indexed accumulators live in registers (the a loop is unrolled);
      // b-indexed ones in this lane's own shared-memory column (runtime b loop).
      T kac[NA], kad[NA];
#pragma unroll
      for (int x = 0; x < NA; ++x) {
        kac[x] = T(0);
        kad[x] = T(0);
      }
      T* kbc = Kb + lane;           // kbc[b * 32]
      T* kbd = Kb + NB * 32 + lane;  // kbd[b * 32]
      for (int b = 0; b < NB; ++b) {
        kbc[b * 32] = T(0);
        kbd[b * 32] = T(0);
      }
      const double* Dcol_d = a.Dp + ao4 + id;  // D'[row][d]
      const double* Dcol_c = a.Dp + ao3 + ic;  // D'[row][c]
      for (int pb = 0; pb < npb; ++pb) {
        Prim<T> bp;
        bp.load(a.pd, offb + pb);
        if (lane < 3) md_e_1d<LA, LB, T>(bp.PA[lane], bp.PB[lane], T(0.5) / bp.p, Eb + lane * S::NEB);
        for (int x = lane; x < nci * WS; x += 32) W[x] = T(0);
        __syncwarp();
        for (int pk = 0; pk < npk; ++pk) {
          Prim<T> kp;
          kp.load(a.pd, offk + pk);
          if (lane < 3) {
            T* e = Ek + lane * S::NEK;
            md_e_1d<LC, LD, T>(kp.PA[lane], kp.PB[lane], T(0.5) / kp.p, e);
            // fold (-1)^s into the ket coefficients
#pragma unroll
            for (int x = 0; x < S::NEK; ++x)
              if ((x % (LCD + 1)) & 1) e[x] = -e[x];
          }
          const T pq = bp.p * kp.p, ps = bp.p + kp.p;
          const T rho = pq / ps;
          const T X = bp.P[0] - kp.P[0], Y = bp.P[1] - kp.P[1], Z = bp.P[2] - kp.P[2];
          T F[L + 1];
          Boys<T>::template eval<L>(rho * (X * X + Y * Y + Z * Z), a.boys64, a.boys32, F);
          const T pref = bp.pref * kp.pref * (T(1) / sqrt(ps));
          r_build_warp<L, T>(F, pref, X, Y, Z, T(-2) * rho, a.rsteps, ping0, ping1, box, lane);
          // phase 1: ket transform, trip counts uniform (they depend on cd only)
#pragma unroll 1
          for (int ci = 0; ci < nci; ++ci) {
            int kx, ky, kz, lx, ly, lz;
            cart_xyz(LC, (c0 + ci) / ND, kx, ky, kz);
            cart_xyz(LD, (c0 + ci) % ND, lx, ly, lz);
            const T* ex = Ek + 0 * S::NEK + (kx * (LD + 1) + lx) * (LCD + 1);
            const T* ey = Ek + 1 * S::NEK + (ky * (LD + 1) + ly) * (LCD + 1);
            const T* ez = Ek + 2 * S::NEK + (kz * (LD + 1) + lz) * (LCD + 1);
            const int nx = kx + lx, ny = ky + ly, nz = kz + lz;
#pragma unroll
            for (int j = 0; j < S::NPS; ++j) {
              const int P = lane + 32 * j;
              if (P < HAB) {
                T acc = T(0);
#pragma unroll 1
                for (int sx = 0; sx <= nx; ++sx) {
                  T accy = T(0);
#pragma unroll 1
                  for (int sy = 0; sy <= ny; ++sy) {
                    const T* r = box + pbase[j] + sx * B * B + sy * B;
                    T accz = T(0);
#pragma unroll 1
                    for (int sz = 0; sz <= nz; ++sz) accz = fma(ez[sz], r[sz], accz);
                    accy = fma(ey[sy], accz, accy);
                  }
                  acc = fma(ex[sx], accy, acc);
                }
                W[ci * WS + P] += acc;
              }
            }
          }
          __syncwarp();
        }
        // phase 2: bra transform and contraction, lane owns column cd
        if (cdv) {
          const T* wcol = W + lane * WS;
#pragma unroll
          for (int xa = 0; xa < NA; ++xa) {
            int ix, iy, iz;
            cart_xyz(LA, xa, ix, iy, iz);
            const T dad_x = ldT<T>(a.Dp + (size_t)(ao1 + xa) * nbf + ao4 + id);
            const T dac_x = ldT<T>(a.Dp + (size_t)(ao1 + xa) * nbf + ao3 + ic);
#pragma unroll 1
            for (int xb = 0; xb < NB; ++xb) {
              int jx, jy, jz;
              cart_xyz(LB, xb, jx, jy, jz);
              const T* ex = Eb + 0 * S::NEB + (ix * (LB + 1) + jx) * (LAB + 1);
              const T* ey = Eb + 1 * S::NEB + (iy * (LB + 1) + jy) * (LAB + 1);
              const T* ez = Eb + 2 * S::NEB + (iz * (LB + 1) + jz) * (LAB + 1);
              const int nx = ix + jx, ny = iy + jy, nz = iz + jz;
              T acc = T(0);
#pragma unroll 1
              for (int tx = 0; tx <= nx; ++tx) {
                T accy = T(0);
#pragma unroll 1
                for (int ty = 0; ty <= ny; ++ty) {
                  T accz = T(0);
#pragma unroll 1
                  for (int tz = 0; tz <= nz; ++tz) {
                    // herm_index(tx,ty,tz) for fixed (tx,ty) walks groups n = tx+ty+tz
                    const int n = tx + ty + tz, r = ty + tz;
                    accz = fma(ez[tz], wcol[nherm(n - 1) + r * (r + 1) / 2 + tz], accz);
                  }
                  accy = fma(ey[ty], accz, accy);
                }
                acc = fma(ex[tx], accy, acc);
              }
              const T v = w * acc;
              const size_t rowb = (size_t)(ao2 + xb) * nbf;
              kac[xa] = fma(v, ldT<T>(Dcol_d + rowb), kac[xa]);
              kad[xa] = fma(v, ldT<T>(Dcol_c + rowb), kad[xa]);
              kbc[xb * 32] = fma(v, dad_x, kbc[xb * 32]);
              kbd[xb * 32] = fma(v, dac_x, kbd[xb * 32]);
            }
          }
        }
        __syncwarp();
      }
      if (cdv) {
#pragma unroll
        for (int x = 0; x < NA; ++x) {
          atomic_add_d(a.Kh + (size_t)(ao1 + x) * nbf + ao3 + ic, (double)kac[x]);
          atomic_add_d(a.Kh + (size_t)(ao1 + x) * nbf + ao4 + id, (double)kad[x]);
        }
        for (int b = 0; b < NB; ++b) {
          atomic_add_d(a.Kh + (size_t)(ao2 + b) * nbf + ao3 + ic, (double)kbc[b * 32]);
          atomic_add_d(a.Kh + (size_t)(ao2 + b) * nbf + ao4 + id, (double)kbd[b * 32]);
        }
      }
    }
  }
}

template <int LAB, int LCD, typename T>
struct JShape {
  static constexpr int L = LAB + LCD, B = L + 1, BOX = B * B * B, HAB = nherm(LAB), HCD = nherm(LCD);
  static constexpr int NPING = L > 0 ? nherm(L - 1) : 1, NPS = (HAB + 31) / 32;
  static constexpr int SM_BOX = 0, SM_PING = BOX, SM_TOTAL = SM_PING + 2 * NPING;
  static constexpr size_t smem_per_warp() { return sizeof(T) * SM_TOTAL; }
};

// J-engine (Eq. j_formula): for every significant ordered (bra, ket) shell-pair
// pair, J_P(bra primitive pair) += sum_Q R_{P+Q} D_Q(ket primitive pair), with
// the Hermite density D_Q = (-1)^|Q| sum_{ls} E_Q^{ls} D_ls prepared beforehand.
// Lanes own bra Hermite indices P; the Q loop is uniform across the warp.
template <int LAB, int LCD, typename T>
__global__ void __launch_bounds__(128) j_warp_kernel(JArgs a) {
  using S = JShape<LAB, LCD, T>;
  constexpr int L = S::L, B = S::B, HAB = S::HAB, HCD = S::HCD;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  T* sm = reinterpret_cast<T*>(smraw) + (size_t)wib * S::SM_TOTAL;
  T* box = sm + S::SM_BOX;
  T* ping0 = sm + S::SM_PING;
  T* ping1 = ping0 + S::NPING;
  int pbase[S::NPS];
#pragma unroll
  for (int j = 0; j < S::NPS; ++j) {
    int P = lane + 32 * j;
    pbase[j] = 0;
    if (P < HAB) {
      RStep s = a.rsteps[P];
      pbase[j] = (s.t * B + s.u) * B + s.v;
    }
  }
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t total = a.wl.total;
  for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; item < total; item += nwarps) {
    if (a.tier && a.tier[item] != a.tier_want) continue;
    const int ib = find_bra(a.wl.prefix, a.wl.nbra, item);
    const int ik = (int)(item - __ldg(a.wl.prefix + ib));
    const int pb_id = __ldg(a.wl.bra + ib), pk_id = __ldg(a.wl.ket + ik);
    const int npb = __ldg(a.sp.np + pb_id), offb = __ldg(a.sp.poff + pb_id);
    const int npk = __ldg(a.sp.np + pk_id), offk = __ldg(a.sp.poff + pk_id);
    const int hb = __ldg(a.sp.hoff + pb_id), hk = __ldg(a.sp.hoff + pk_id);
    for (int pb = 0; pb < npb; ++pb) {
      Prim<T> bp;
      bp.load(a.pd, offb + pb);
      T acc[S::NPS];
#pragma unroll
      for (int j = 0; j < S::NPS; ++j) acc[j] = T(0);
      for (int pk = 0; pk < npk; ++pk) {
        Prim<T> kp;
        kp.load(a.pd, offk + pk);
        const T pq = bp.p * kp.p, ps = bp.p + kp.p;
        const T rho = pq / ps;
        const T X = bp.P[0] - kp.P[0], Y = bp.P[1] - kp.P[1], Z = bp.P[2] - kp.P[2];
        T F[L + 1];
        Boys<T>::template eval<L>(rho * (X * X + Y * Y + Z * Z), a.boys64, a.boys32, F);
        const T pref = bp.pref * kp.pref * (T(1) / sqrt(ps));
        r_build_warp<L, T>(F, pref, X, Y, Z, T(-2) * rho, a.rsteps, ping0, ping1, box, lane);
        const double* dq = a.Dherm + hk + (size_t)pk * HCD;
#pragma unroll
        for (int j = 0; j < S::NPS; ++j) {
          const int P = lane + 32 * j;
          if (P < HAB) {
            T s = T(0);
#pragma unroll
            for (int t = 0; t <= LCD; ++t)
#pragma unroll
              for (int u = 0; u <= LCD - t; ++u) {
                const T* r = box + pbase[j] + t * B * B + u * B;
#pragma unroll
                for (int v = 0; v <= LCD - t - u; ++v) s = fma(r[v], ldT<T>(dq + herm_index(t, u, v)), s);
              }
            acc[j] += s;
          }
        }
        __syncwarp();
      }
#pragma unroll
      for (int j = 0; j < S::NPS; ++j) {
        const int P = lane + 32 * j;
        if (P < HAB) atomic_add_d(a.Jherm + hb + (size_t)pb * HAB + P, (double)acc[j]);
      }
    }
  }
}

}  // namespace eri
