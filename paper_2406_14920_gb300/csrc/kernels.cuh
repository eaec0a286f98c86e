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
  BoysTabs bt;
  const RStep* rsteps;
  const double* Dp;   // density with component norms folded in (packed per molecule)
  const float* Dpf;   // the same in FP32, read by the FP32 tier (no conversions on the FP64 pipe)
  double* Kh;         // half-K accumulator (packed per molecule)
  // precision tiers (mixed mode): a quartet is FP64 (tier 0) when
  // Q_ab Q_cd max|D'| >= tau over the six D blocks it touches, or when one of
  // its pairs has an exponent sum above pmax32; otherwise FP32 (tier 1).
  const float* Q;       // Schwarz bound per pair
  const float* dmax;    // max |D'| over the two D blocks of each shell pair (pair index)
  const float* pmaxp;   // largest primitive exponent sum per pair
  const float* prefmaxp;  // largest |primitive-pair prefactor| per pair
  const int* shloc;     // shell index inside its molecule, per (global) shell
  const int* pbase;     // first pair index of each molecule
  float tau, pmax32;
  int mixed;            // tier split only (k_tier_split): test every item
  int tier_want;        // 0 or 1: which tier this launch processes
  unsigned long long* counter;  // items processed by this launch's tier (may be null)
  unsigned long long* guard;    // tier split: quartets kept in FP64 by the range guard alone (may be null)
  unsigned long long* screened; // tier split: quartets dropped by the density screen (may be null)
  float screen;                 // density screen (Eq. kernel_upperbound): drop Q_ab Q_cd max|D'| < screen; 0 = off
  int same_class;
  // Mixed precision: the launch runs the compacted list of its tier written by
  // k_tier_split, item i = (bra position items[i].x, ket position items[i].y),
  // *nitems of them (read on the device).  Null: items are positions in wl.
  const int2* items;
  const unsigned int* nitems;
  double omega2;  // long-range operator erf(omega r)/r: omega^2 (0 = Coulomb 1/r)
  float omega2f;
  int det;        // 1: fixed-point accumulators (deterministic builds, acc_add)
};

// Long-range operator erf(omega r)/r (Sec. 2.5, Eq. eri_longrange_formula):
// the Hermite integrals keep their form with rho -> s rho and the prefactor
// times sqrt(s), s = omega^2 / (omega^2 + rho).  omega2 = 0 is the Coulomb
// operator and leaves rho and pref untouched.  omega2 is uniform over a launch.
template <typename T>
__device__ __forceinline__ void attenuate(T omega2, T& rho, T& pref) {
  if (omega2 > T(0)) {
    const T s = omega2 / (omega2 + rho);
    rho *= s;
    pref *= sqrt(s);
  }
}

// pair index of shells x, y of molecule `mol` (pairs are stored a >= b, a(a+1)/2 + b)
__device__ __forceinline__ int pair_index(const KArgs& a, int mol, int x, int y) {
  const int lx = __ldg(a.shloc + x), ly = __ldg(a.shloc + y);
  const int hi = lx > ly ? lx : ly, lo = lx > ly ? ly : lx;
  return __ldg(a.pbase + mol) + hi * (hi + 1) / 2 + lo;
}

// Tier of one quartet: 0 = FP64 (bound >= tau), 1 = FP32, 2 = FP64 because
// the FP32 range guard tripped although the bound is below tau, 3 = dropped
// by the density screen (bound below `screen`).
__device__ __forceinline__ int quartet_tier(const KArgs& a, int mol, int pb_id, int pk_id, int s1, int s2, int s3,
                                            int s4) {
  const float* dm = a.dmax;
  float d = fmaxf(fmaxf(__ldg(dm + pb_id), __ldg(dm + pk_id)),
                  fmaxf(fmaxf(__ldg(dm + pair_index(a, mol, s1, s3)), __ldg(dm + pair_index(a, mol, s1, s4))),
                        fmaxf(__ldg(dm + pair_index(a, mol, s2, s3)), __ldg(dm + pair_index(a, mol, s2, s4)))));
  const float b = __ldg(a.Q + pb_id) * __ldg(a.Q + pk_id) * d;
  if (b < a.screen) return 3;
  // FP32 range guard: tight exponents or large prefactors stay in FP64
  // (R grows like (2 rho)^(L/2) and the prefactors multiply into it)
  const bool wide = fmaxf(__ldg(a.pmaxp + pb_id), __ldg(a.pmaxp + pk_id)) > a.pmax32 ||
                    __ldg(a.prefmaxp + pb_id) * __ldg(a.prefmaxp + pk_id) > 1.0e18f;
  // 0: FP64 by the bound; 1: FP32; 2: FP64 only because of the range guard
  return b >= a.tau ? 0 : (wide ? 2 : 1);
}

// D' in the launch's precision
template <typename T> __device__ __forceinline__ const T* dens(const KArgs& a);
template <> __device__ __forceinline__ const double* dens<double>(const KArgs& a) { return a.Dp; }
template <> __device__ __forceinline__ const float* dens<float>(const KArgs& a) { return a.Dpf; }

struct JArgs {
  PairData pd;
  ShellPairInfo sp;
  WorkList wl;
  BoysTabs bt;
  const RStep* rsteps;
  const double* Dherm;  // Hermite density per ket primitive pair (sign (-1)^|Q| folded in)
  const float* Dhermf;  // the same in FP32, read by the FP32 tier (no conversions on the FP64 pipe)
  double* Jherm;        // Hermite J per bra primitive pair (accumulated in FP64 by both tiers)
  double omega2;        // erf(omega r)/r: omega^2 (0 = Coulomb)
  float omega2f;
  int det;              // 1: fixed-point Jherm (deterministic builds)
  unsigned long long* counter;  // items, primitive quartets, bra primitives of this launch (may be null)
  // mixed precision: the launch runs the compacted list of its tier, item i =
  // (bra position items[i].x, ket position items[i].y), *nitems of them.
  // Null: items are positions in wl.
  const int2* items;
  const unsigned int* nitems;
};

// Hermite density of a J-engine launch in its precision
template <typename T> __device__ __forceinline__ const T* hdens(const JArgs& a);
template <> __device__ __forceinline__ const double* hdens<double>(const JArgs& a) { return a.Dherm; }
template <> __device__ __forceinline__ const float* hdens<float>(const JArgs& a) { return a.Dhermf; }

// omega^2 of a launch in its precision
template <typename T, typename A> __device__ __forceinline__ T om2(const A& a);
template <> __device__ __forceinline__ double om2<double, KArgs>(const KArgs& a) { return a.omega2; }
template <> __device__ __forceinline__ float om2<float, KArgs>(const KArgs& a) { return a.omega2f; }
template <> __device__ __forceinline__ double om2<double, JArgs>(const JArgs& a) { return a.omega2; }
template <> __device__ __forceinline__ float om2<float, JArgs>(const JArgs& a) { return a.omega2f; }

__device__ __forceinline__ int find_bra(const int64_t* __restrict__ prefix, int n, int64_t item) {
  int lo = 0, hi = n;  // prefix[lo] <= item < prefix[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// Position in a work list: bra ib covers items [bs, be).  Workers take tiles of
// consecutive items and step through them, moving the cursor forward over the
// prefix array instead of searching it again for every item.
struct BraCursor {
  int ib;
  int64_t bs, be;
  __device__ __forceinline__ BraCursor() : ib(0), bs(0), be(0) {}
  __device__ __forceinline__ BraCursor(const WorkList& wl, int64_t item) { seek(wl, item); }
  __device__ __forceinline__ void seek(const WorkList& wl, int64_t item) {
    ib = find_bra(wl.prefix, wl.nbra, item);
    bs = __ldg(wl.prefix + ib);
    be = __ldg(wl.prefix + ib + 1);
  }
  // ket index of `item` (item >= every item seen before, < wl.total)
  __device__ __forceinline__ int at(const WorkList& wl, int64_t item) {
    while (item >= be) {
      ++ib;
      bs = be;
      be = __ldg(wl.prefix + ib + 1);
    }
    return (int)(item - bs);
  }
};

template <typename T> __device__ __forceinline__ T ldT(const double* p) { return (T)__ldg(p); }

// precision-explicit reciprocal square root (a plain overload inside this
// namespace would hide ::rsqrt(double) and silently demote FP64 to FP32)
__device__ __forceinline__ double rsqrt_t(double x) { return ::rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return ::rsqrtf(x); }
template <typename T> __device__ __forceinline__ T pdv(const double* d, const float* f, int i);
template <typename T> __device__ __forceinline__ T ldE(const PairData& pd, int i);
template <> __device__ __forceinline__ double ldE<double>(const PairData& pd, int i) { return __ldg(pd.E + i); }
template <> __device__ __forceinline__ float ldE<float>(const PairData& pd, int i) { return __ldg(pd.Ef + i); }
template <> __device__ __forceinline__ double pdv<double>(const double* d, const float*, int i) { return __ldg(d + i); }
template <> __device__ __forceinline__ float pdv<float>(const double*, const float* f, int i) { return __ldg(f + i); }

// Primitive pair scalars in precision T (FP32: three 16-byte vector loads of
// the packed shadows; unused components are dropped by the compiler).
template <typename T>
struct Prim {
  T p, P[3], PA[3], PB[3], pref;
  __device__ __forceinline__ void load(const PairData& pd, int i) {
    if constexpr (sizeof(T) == 4) {
      const float4 a = __ldg(pd.q4 + 3 * i), b = __ldg(pd.q4 + 3 * i + 1), c = __ldg(pd.q4 + 3 * i + 2);
      P[0] = a.x; P[1] = a.y; P[2] = a.z; p = a.w;
      PA[0] = b.x; PA[1] = b.y; PA[2] = b.z; pref = b.w;
      PB[0] = c.x; PB[1] = c.y; PB[2] = c.z;
    } else {
      p = pdv<T>(pd.p, pd.pf, i);
      pref = pdv<T>(pd.pref, pd.preff, i);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        P[d] = pdv<T>(pd.P, pd.Pf, d * pd.n + i);
        PA[d] = pdv<T>(pd.PA, pd.PAf, d * pd.n + i);
        PB[d] = pdv<T>(pd.PB, pd.PBf, d * pd.n + i);
      }
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
    int ib, ik;
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
    const int npb = __ldg(a.sp.np + pb_id), offb = __ldg(a.sp.poff + pb_id);
    const int npk = __ldg(a.sp.np + pk_id), offk = __ldg(a.sp.poff + pk_id);
    ++done;
    doneq += (unsigned long long)npb * npk;
    doneb += npb;
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
        T rho = pq / ps;
        T pref = bp.pref * kp.pref * (T(1) / sqrt(ps));
        attenuate(om2<T>(a), rho, pref);
        const T X = bp.P[0] - kp.P[0], Y = bp.P[1] - kp.P[1], Z = bp.P[2] - kp.P[2];
        T F[L + 1];
        Boys<T>::template eval<L>(rho * (X * X + Y * Y + Z * Z), a.bt, F);
        r_build_warp<L, T>(F, pref, X, Y, Z, T(-2) * rho, a.rsteps, ping0, ping1, box, lane);
        const T* dq = hdens<T>(a) + hk + (size_t)pk * HCD;
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
                for (int v = 0; v <= LCD - t - u; ++v) s = fma(r[v], __ldg(dq + herm_index(t, u, v)), s);
              }
            acc[j] += s;
          }
        }
        __syncwarp();
      }
#pragma unroll
      for (int j = 0; j < S::NPS; ++j) {
        const int P = lane + 32 * j;
        if (P < HAB) acc_add(a.Jherm + hb + (size_t)pb * HAB + P, (double)acc[j], a.det);
      }
    }
  }
  }
  if (a.counter && lane == 0 && done) {
    atomicAdd(a.counter, done);
    atomicAdd(a.counter + 1, doneq);
    atomicAdd(a.counter + 2, doneb);
  }
}

// Which J-engine classes run one ordered item per thread (R, the item's
// Hermite J and the ket's Hermite density in registers) instead of one per warp.
__host__ __device__ constexpr bool use_j_thread(int lab, int lcd) {
  return nherm(lab + lcd) + nherm(lab) + nherm(lcd) <= 130;
}

// J-engine (Eq. j_formula), one ordered (bra, ket) shell-pair item per lane:
// for each bra primitive pair, J_P += sum_{ket prims} sum_Q R_{P+Q} D_Q with
// every Hermite index a compile-time constant, in the launch's precision (the
// FP32 tier of a mixed build reads the FP32 pair data and Hermite density).
// The lists are bra-major, so a warp's 32 items usually share one bra pair:
// then J_P is summed over the warp with shuffles and one lane adds it to the
// bra primitive's Hermite J (one FP64 atomic per element instead of 32);
// otherwise each lane adds its own.
template <int LAB, int LCD, typename T>
__global__ void __launch_bounds__(128) j_thread_kernel(JArgs a) {
  constexpr int L = LAB + LCD, NR = nherm(L), HAB = nherm(LAB), HCD = nherm(LCD);
  const int lane = threadIdx.x & 31;
  const bool compact = a.items != nullptr;
  const int64_t total = compact ? (int64_t)__ldg(a.nitems) : a.wl.total;
  const int64_t first = compact ? 0 : a.wl.first;
  const int nshard = compact ? 1 : a.wl.nshard, shard = compact ? 0 : a.wl.shard;
  const int64_t span = 32 * (int64_t)a.wl.tile, ntiles = (total - first + span - 1) / span;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long done = 0, doneq = 0, doneb = 0;
  for (int64_t tl = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * nshard + shard;
       tl < ntiles; tl += nwarps * nshard) {
    const int64_t t0 = first + tl * span, i1 = t0 + span < total ? t0 + span : total;
    BraCursor cur;
    if (!compact) cur.seek(a.wl, t0 + lane < i1 ? t0 + lane : t0);
    for (int64_t base = t0; base < i1; base += 32) {  // uniform over the warp
      const int64_t item = base + lane;
      const bool ok = item < i1;
      int pb_id = -1, npb = 0, offb = 0, hb = 0, npk = 0, offk = 0, hk = 0;
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
        pb_id = __ldg(a.wl.bra + ib);
        const int mol = __ldg(a.sp.pmol + pb_id);
        const int pk_id = __ldg(a.wl.ket + __ldg(a.wl.kseg + mol * NPAIRCLASS) + ik);
        npb = __ldg(a.sp.np + pb_id);
        offb = __ldg(a.sp.poff + pb_id);
        hb = __ldg(a.sp.hoff + pb_id);
        npk = __ldg(a.sp.np + pk_id);
        offk = __ldg(a.sp.poff + pk_id);
        hk = __ldg(a.sp.hoff + pk_id);
        ++done;
        doneq += (unsigned long long)npb * npk;
        doneb += npb;
      }
      // lane 0's item is always valid here
      const int pb0 = __shfl_sync(0xffffffffu, pb_id, 0);
      const bool uni = __all_sync(0xffffffffu, !ok || pb_id == pb0);
      const int npb_loop = uni ? __shfl_sync(0xffffffffu, npb, 0) : npb;
      for (int pb = 0; pb < npb_loop; ++pb) {
        T acc[HAB];
#pragma unroll
        for (int x = 0; x < HAB; ++x) acc[x] = T(0);
        if (ok) {
          Prim<T> bp;
          bp.load(a.pd, offb + pb);
          for (int pk = 0; pk < npk; ++pk) {
            Prim<T> kp;
            kp.load(a.pd, offk + pk);
            const T ps = bp.p + kp.p;
            T rho = bp.p * kp.p / ps;
            T pref = bp.pref * kp.pref * rsqrt_t(ps);
            attenuate(om2<T>(a), rho, pref);
            const T X = bp.P[0] - kp.P[0], Y = bp.P[1] - kp.P[1], Z = bp.P[2] - kp.P[2];
            T F[L + 1];
            Boys<T>::template eval<L>(rho * (X * X + Y * Y + Z * Z), a.bt, F);
            T R[NR];
            r_build_reg<L, T>(F, pref, X, Y, Z, T(-2) * rho, R);
            const T* dq = hdens<T>(a) + hk + (size_t)pk * HCD;
            T Dq[HCD];
#pragma unroll
            for (int q = 0; q < HCD; ++q) Dq[q] = __ldg(dq + q);
            for_herm<LAB>([&](auto t, auto u, auto v) {
              constexpr int P = herm_index(ERI_CI(t), ERI_CI(u), ERI_CI(v));
              T s = acc[P];
              for_herm<LCD>([&](auto x, auto y, auto z) {
                s = fma(R[herm_index(ERI_CI(t) + ERI_CI(x), ERI_CI(u) + ERI_CI(y), ERI_CI(v) + ERI_CI(z))],
                        Dq[herm_index(ERI_CI(x), ERI_CI(y), ERI_CI(z))], s);
              });
              acc[P] = s;
            });
          }
        }
        if (uni) {
#pragma unroll
          for (int x = 0; x < HAB; ++x) {
            T v = acc[x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc[x] = v;
          }
          if (lane == 0)
#pragma unroll
            for (int x = 0; x < HAB; ++x) acc_add(a.Jherm + hb + (size_t)pb * HAB + x, (double)acc[x], a.det);
        } else if (ok) {
#pragma unroll
          for (int x = 0; x < HAB; ++x) acc_add(a.Jherm + hb + (size_t)pb * HAB + x, (double)acc[x], a.det);
        }
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
