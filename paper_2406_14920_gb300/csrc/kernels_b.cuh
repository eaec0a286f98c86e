// General J+K kernel: one warp per canonical shell quartet, contracted ERI block
// staged in shared memory.  Used for every class that does not fit the
// register kernel (kernels_a.cuh).
//
// Per quartet, per chunk of CH ket Cartesian pairs cd, per bra primitive pair,
// the ket primitive pairs are taken G at a time:
//   step A  (lane g): quartet scalars for ket primitive g -- rho, P-Q, prefactor,
//           Boys F_0..F_L (Eq. boys_function); all lanes: ket E tables to smem
//           with (-1)^|Q| folded in;
//   step B  items (g, e), level by level: R^0 of the G primitive quartets
//           (Eq. R_recursion);
//   step C  items (cd, P): W[cd][P] += sum_g sum_Q E'_Q^{cd}(g) R_{P+Q}(g);
// then for the bra primitive:
//   step D  items (ab, cd): X[ab][cd] += sum_P E_P^{ab} W[cd][P]        (Eq. eri_formula)
// and per chunk the contraction, one lane per output element:
//   Kh_ac, Kh_ad, Kh_bc, Kh_bd (Eq. k_definition), Jh_ab, Jh_cd (Eq. j_definition),
//   one atomic per element.
// Every per-primitive-quartet scalar is computed by one lane, not redundantly
// by the warp (GB300's FP64 pipe charges a full warp issue per instruction
// whatever the number of active lanes).
#pragma once
#include "kernels_a.cuh"

// base shared memory per warp (KB) of the warp kernel, per precision: FP64
// keeps 8 warps per SM (two resident 4-warp blocks), FP32 about 16-20
#ifndef ERI_WARP_SMEM64_KB
#define ERI_WARP_SMEM64_KB 22
#endif
#ifndef ERI_WARP_SMEM32_KB
#define ERI_WARP_SMEM32_KB 12
#endif
// upper limits when a larger ket-primitive batch saves a batch (FP64: two
// 4-warp blocks still fit in an SM's 228 KB)
#ifndef ERI_WARP_SMEM64_MAX_KB
#define ERI_WARP_SMEM64_MAX_KB 27
#endif
#ifndef ERI_WARP_SMEM32_MAX_KB
#define ERI_WARP_SMEM32_MAX_KB 16
#endif
// FP32 compile-time bra transform: largest X slice per lane, and the shared
// memory per warp a class may take to get there (measured on GB300: (fd|fp)
// 58 -> 9.9 ms with the 24 KB budget, (ff|dp) 35 -> 4.8 ms with 100-value slices)
#ifndef ERI_REGD32_MAX
#define ERI_REGD32_MAX 100
#endif
#ifndef ERI_WARP_SMEM32_FULL_KB
#define ERI_WARP_SMEM32_FULL_KB 24
#endif
// FP64 also takes the lane-owned-P ket transform where W fits in registers
#ifndef ERI_REGW64
#define ERI_REGW64 1
#endif

namespace eri {

template <int LA, int LB, int LC, int LD, typename T>
struct BShape {
  static constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
  static constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  static constexpr int NAB = NA * NB, NCD = NC * ND, HAB = nherm(LAB), HABP = HAB | 1;
  static constexpr int B = L + 1, BOX = B * B * B, NPING = L > 0 ? nherm(L - 1) : 1;
  static constexpr int NEB = (LA + 1) * (LB + 1) * (LAB + 1), NEK = (LC + 1) * (LD + 1) * (LCD + 1);
  static constexpr int NSC = L + 5;  // F'_0..F'_L, PQx, PQy, PQz, c
  // Shared memory per warp (elements of T).  Steps A and B cost the same per
  // batch of G ket primitives whatever G, so G should cover a ket pair's
  // primitives in as few batches as the memory allows: contracted s/p pairs
  // commonly have 9 (3 x 3), pairs with a d or f shell 3.  The budget starts at
  // BASE (occupancy) and grows up to MAX until that batch count is reached.
  static constexpr int FIXED = 3 * NEB;
  static constexpr int PER_G = BOX + 2 * NPING + NSC + 3 * NEK;
  static constexpr int PER_C = HABP + NAB;
  static constexpr int BASE = sizeof(T) == 8 ? (ERI_WARP_SMEM64_KB * 1024) / 8 : (ERI_WARP_SMEM32_KB * 1024) / 4;
  static constexpr int MAXB = sizeof(T) == 8 ? (ERI_WARP_SMEM64_MAX_KB * 1024) / 8 : (ERI_WARP_SMEM32_MAX_KB * 1024) / 4;
  static constexpr int GTARGET = (LC <= 1 && LD <= 1) ? 9 : 3;
  static constexpr int fit_g(int budget) { return (budget - FIXED - NCD * PER_C) / PER_G; }
  static constexpr int GMAXB = fit_g(MAXB) < 1 ? 1 : fit_g(MAXB);
  static constexpr int NBATCH = (GTARGET + GMAXB - 1) / GMAXB;
  static constexpr int GWANT = (GTARGET + NBATCH - 1) / NBATCH;
  static constexpr int NEED = FIXED + NCD * PER_C + GWANT * PER_G;
  static constexpr int BUDGET0 = NEED <= BASE ? BASE : (NEED <= MAXB ? NEED : MAXB);
  // FP32 classes with many ket components take a larger budget when that is
  // what lets the whole ket range sit in one chunk (one ket primitive per
  // batch), the condition of the compile-time bra transform below
  static constexpr int NEED_FULL = FIXED + NCD * PER_C + PER_G;
  static constexpr bool WANT_FULL = sizeof(T) == 4 && NCD >= 8 && NAB * ((NCD + 31) / 32) <= ERI_REGD32_MAX &&
                                    NEED_FULL <= (ERI_WARP_SMEM32_FULL_KB * 1024) / 4;
  static constexpr int BUDGET = (WANT_FULL && BUDGET0 < NEED_FULL) ? NEED_FULL : BUDGET0;
  static constexpr int G0 = (BUDGET - FIXED - NCD * PER_C) / PER_G;
  static constexpr int G = G0 >= 1 ? (G0 > 16 ? 16 : G0) : 1;
  static constexpr int CHMAX = (BUDGET - FIXED - G * PER_G) / PER_C;
  static constexpr int CH = CHMAX >= NCD ? NCD : (CHMAX < 1 ? 1 : CHMAX);
  // FP32 register path for step C: lane j-slot P = lane + 32 j holds W[cd][P]
  // for every ket pair cd in registers, the cd loop unrolled at compile time
  static constexpr int NPS = (HAB + 31) / 32;
  static constexpr bool REGW = CH == NCD && (sizeof(T) == 4 ? NCD * NPS <= 64 : (ERI_REGW64 && NCD * NPS <= 32));
  // step D with compile-time indices: lane owns ket pair cd = lane + 32 j, the
  // bra pairs ab are a compile-time loop (E broadcast, W row at a per-lane
  // base), X[ab][cd] stays in registers over the bra primitives.  Worth it
  // from 8 ket components up, when the X slice fits in registers (measured on
  // workload 1, FP32: (ff|pp) 17.9 -> 9.6 ms, (fd|fs) 15.8 -> 9.4 ms, against
  // the (ab, cd) item loop).
  static constexpr int NCS = (NCD + 31) / 32;
  static constexpr bool REGD = CH == NCD && NCD >= 8 && NAB * NCS <= (sizeof(T) == 4 ? ERI_REGD32_MAX : 48);
  static constexpr int SM_BOX = 0, SM_PING = SM_BOX + G * BOX, SM_SC = SM_PING + G * 2 * NPING,
                       SM_EK = SM_SC + G * NSC, SM_EB = SM_EK + G * 3 * NEK, SM_W = SM_EB + 3 * NEB,
                       SM_X = SM_W + CH * HABP, SM_TOTAL = SM_X + NAB * CH;
  __host__ __device__ static constexpr size_t smem_per_warp() { return sizeof(T) * SM_TOTAL; }
  // block-shared index tables (ints): cd table, ab table, P table, W row bases
  static constexpr int LEXB = (LAB + 1) * (LAB + 1);
  static constexpr int TAB_INTS = 2 * NCD + 2 * NAB + HAB + LEXB;
  static constexpr int TABLE_BYTES = ((4 * TAB_INTS + 15) / 16) * 16;
  __host__ __device__ static constexpr size_t table_bytes() { return TABLE_BYTES; }
};

// W is stored per cd with a "lexicographic" Hermite index (t, then u, then v)
// so that for fixed (t, u) consecutive v are consecutive: lex(t,u,v) = base(t,u) + v.
__host__ __device__ constexpr int lex_base(int lmax, int t, int u) {
  int b = 0;
  for (int x = 0; x < t; ++x) b += (lmax - x + 1) * (lmax - x + 2) / 2;
  for (int y = 0; y < u; ++y) b += lmax - t - y + 1;
  return b;
}

// FP64: two resident blocks per SM are the target (the register budget follows);
// FP32: left to the compiler
template <int LA, int LB, int LC, int LD, typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 2 : 0) jk_warp_kernel(JKArgs A) {
  using S = BShape<LA, LB, LC, LD, T>;
  constexpr int LAB = S::LAB, LCD = S::LCD, L = S::L, B = S::B, BOX = S::BOX, NSC = S::NSC;
  constexpr int NA = S::NA, NB = S::NB, ND = S::ND, NAB = S::NAB, NCD = S::NCD, HAB = S::HAB, HABP = S::HABP,
                CH = S::CH, G = S::G, NEB = S::NEB, NEK = S::NEK, NPING = S::NPING;
  const KArgs& a = A.k;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // index tables shared by the block: per ket pair cd the E offsets and term
  // counts, the same per bra pair ab, per bra Hermite index P its box offset
  // and its W slot, and the W row bases for step D
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
    tab_ab[2 * i] = ((ix * (LB + 1) + jx) * (LAB + 1)) | ((NEB + (iy * (LB + 1) + jy) * (LAB + 1)) << 10) |
                    ((2 * NEB + (iz * (LB + 1) + jz) * (LAB + 1)) << 20);
    tab_ab[2 * i + 1] = (ix + jx) | ((iy + jy) << 4) | ((iz + jz) << 8);
  }
  for (int i = threadIdx.x; i < HAB; i += blockDim.x) {
    const int t = herm_t(i), u = herm_u(i), v = herm_v(i);
    tab_p[i] = ((t * B + u) * B + v) | ((lex_base(LAB, t, u) + v) << 16);
  }
  for (int i = threadIdx.x; i < S::LEXB; i += blockDim.x) {
    const int t = i / (LAB + 1), u = i % (LAB + 1);
    tab_lex[i] = (t + u <= LAB) ? lex_base(LAB, t, u) : 0;
  }
  __syncthreads();
  int pslot[S::NPS];  // box offset of this lane's bra Hermite indices P = lane + 32 j
#pragma unroll
  for (int j = 0; j < S::NPS; ++j) pslot[j] = lane + 32 * j < HAB ? (tab_p[lane + 32 * j] & 0xffff) : 0;
  T* sm = reinterpret_cast<T*>(smraw + S::table_bytes()) + (size_t)wib * S::SM_TOTAL;
  T* boxes = sm + S::SM_BOX;
  T* pings = sm + S::SM_PING;
  T* scal = sm + S::SM_SC;
  T* Ek = sm + S::SM_EK;
  T* Eb = sm + S::SM_EB;
  T* Ws = sm + S::SM_W;
  T* Xs = sm + S::SM_X;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  // items: positions in the work list, or (mixed precision) this tier's compacted list
  const bool compact = a.items != nullptr;
  const int64_t total = compact ? (int64_t)__ldg(a.nitems) : a.wl.total;
  const int64_t first = compact ? 0 : a.wl.first;
  const int nshard = compact ? 1 : a.wl.nshard, shard = compact ? 0 : a.wl.shard;
  unsigned long long done = 0, doneq = 0, doneb = 0;
  const int64_t tile = a.wl.tile, ntiles = (total - first + tile - 1) / tile;
  for (int64_t tl = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * nshard + shard; tl < ntiles;
       tl += nwarps * nshard) {
  const int64_t t0 = first + tl * tile, i1 = t0 + tile < total ? t0 + tile : total;
  // the lanes locate 32 items at a time; the warp then runs them one by one
  BraCursor cur;
  if (!compact) cur.seek(a.wl, t0 + lane < i1 ? t0 + lane : t0);
  for (int64_t cq = t0; cq < i1; cq += 32) {
  int my_ib = 0, my_ik = 0;
  const bool ok = cq + lane < i1;
  if (ok) {
    if (compact) {
      const int2 v = __ldg(a.items + cq + lane);
      my_ib = v.x;
      my_ik = v.y;
    } else {
      my_ik = cur.at(a.wl, cq + lane);
      my_ib = cur.ib;
    }
  }
  unsigned pend = __ballot_sync(0xffffffffu, ok);
  while (pend) {
    const int src = __ffs(pend) - 1;
    pend &= pend - 1;
    const int ib = __shfl_sync(0xffffffffu, my_ib, src), ik = __shfl_sync(0xffffffffu, my_ik, src);
    const int pb_id = __ldg(a.wl.bra + ib);
    const int mol = __ldg(a.sp.pmol + pb_id);
    const int pk_id = __ldg(a.wl.ket + __ldg(a.wl.kseg + mol * NPAIRCLASS) + ik);
    const int s1 = __ldg(a.sp.s1 + pb_id), s2 = __ldg(a.sp.s2 + pb_id);
    const int s3 = __ldg(a.sp.s1 + pk_id), s4 = __ldg(a.sp.s2 + pk_id);
    const int npb = __ldg(a.sp.np + pb_id), offb = __ldg(a.sp.poff + pb_id), eb0 = __ldg(a.sp.eoff + pb_id);
    const int npk = __ldg(a.sp.np + pk_id), offk = __ldg(a.sp.poff + pk_id), ek0 = __ldg(a.sp.eoff + pk_id);
    ++done;
    doneq += (unsigned long long)npb * npk;
    doneb += npb;
    const int ao1 = __ldg(a.sp.ao1 + pb_id), ao2 = __ldg(a.sp.ao2 + pb_id);
    const int ao3 = __ldg(a.sp.ao1 + pk_id), ao4 = __ldg(a.sp.ao2 + pk_id);
    T w = T(1);
    if (s1 == s2) w *= T(0.5);
    if (s3 == s4) w *= T(0.5);
    if (pb_id == pk_id) w *= T(0.5);
    const int64_t mbase = __ldg(a.sp.mat_off + mol);
    const int n = __ldg(a.sp.mat_n + mol);
    const T* Dp = dens<T>(a) + mbase;
    double* Kh = a.Kh ? a.Kh + mbase : nullptr;
    double* Jh = A.Jh ? A.Jh + mbase : nullptr;

    for (int c0 = 0; c0 < NCD; c0 += CH) {
      const int nci = NCD - c0 < CH ? NCD - c0 : CH;
      for (int x = lane; x < NAB * CH; x += 32) Xs[x] = T(0);
      T xreg[S::REGD ? S::NCS * NAB : 1];
      if constexpr (S::REGD) {
#pragma unroll
        for (int x = 0; x < S::NCS * NAB; ++x) xreg[x] = T(0);
      }
      for (int pb = 0; pb < npb; ++pb) {
        for (int x = lane; x < 3 * NEB; x += 32) Eb[x] = ldE<T>(a.pd, eb0 + pb * 3 * NEB + x);
        T wreg[S::REGW ? S::NPS * NCD : 1];
        if constexpr (S::REGW) {
#pragma unroll
          for (int x = 0; x < S::NPS * NCD; ++x) wreg[x] = T(0);
        } else {
          for (int x = lane; x < CH * HABP; x += 32) Ws[x] = T(0);
        }
        const int ipb = offb + pb;
        const T bp_p = pdv<T>(a.pd.p, a.pd.pf, ipb), bp_pref = pdv<T>(a.pd.pref, a.pd.preff, ipb);
        const T bPx = pdv<T>(a.pd.P, a.pd.Pf, ipb), bPy = pdv<T>(a.pd.P, a.pd.Pf, a.pd.n + ipb),
                bPz = pdv<T>(a.pd.P, a.pd.Pf, 2 * a.pd.n + ipb);
        for (int k0 = 0; k0 < npk; k0 += G) {
          const int ng = npk - k0 < G ? npk - k0 : G;
          // step A: ket E tables (sign folded) and per-primitive-quartet scalars
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
            attenuate(om2<T>(a), rho, pref);
            const T X = bPx - pdv<T>(a.pd.P, a.pd.Pf, ipk);
            const T Y = bPy - pdv<T>(a.pd.P, a.pd.Pf, a.pd.n + ipk);
            const T Z = bPz - pdv<T>(a.pd.P, a.pd.Pf, 2 * a.pd.n + ipk);
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
          // step B: R^0 for the ng primitive quartets.  FP32 and L <= 6: each lane
          // builds its own quartet's table in registers (compile-time indices) and
          // stores it in its box.  Otherwise the warp builds all of them level by
          // level (scaled form, see r_build_warp).
          if constexpr (sizeof(T) == 4 && L <= 6) {
            if (lane < ng) {
              const T* sc = scal + lane * NSC;
              T Fl[L + 1];
#pragma unroll
              for (int m = 0; m <= L; ++m) Fl[m] = sc[m];
              T R[nherm(L)];
              r_build_reg<L, T>(Fl, T(1), sc[L + 1], sc[L + 2], sc[L + 3], sc[L + 4], R);
              T* bx = boxes + lane * BOX;
#pragma unroll
              for (int t = 0; t <= L; ++t)
#pragma unroll
                for (int u = 0; u <= L - t; ++u)
#pragma unroll
                  for (int v = 0; v <= L - t - u; ++v) bx[(t * B + u) * B + v] = R[herm_index(t, u, v)];
            }
          } else if (L == 0) {
            if (lane < ng) boxes[lane * BOX] = scal[lane * NSC];
          } else {
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
          }
          __syncwarp();
          // step C: ket transform
          if constexpr (S::REGW) {
            // lane-owned P, every cd unrolled: R read at a per-lane base plus
            // compile-time offsets, E' broadcast, W accumulated in registers
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
        // step D: bra transform
        if constexpr (S::REGD) {
          sfor<S::NCS>([&](auto j_) {
            constexpr int j = ERI_CI(j_);
            const int cd = lane + 32 * j;
            if (j * 32 + 32 <= NCD || cd < NCD) {
              const T* wc = Ws + cd * HABP;
              for_cart<LA>([&](auto ix, auto iy, auto iz) {
                for_cart<LB>([&](auto jx, auto jy, auto jz) {
                  constexpr int IX = ERI_CI(ix), IY = ERI_CI(iy), IZ = ERI_CI(iz);
                  constexpr int JX = ERI_CI(jx), JY = ERI_CI(jy), JZ = ERI_CI(jz);
                  constexpr int iab = cidx(LA, IY, IZ) * NB + cidx(LB, JY, JZ);
                  const T* fx = Eb + (IX * (LB + 1) + JX) * (LAB + 1);
                  const T* fy = Eb + NEB + (IY * (LB + 1) + JY) * (LAB + 1);
                  const T* fz = Eb + 2 * NEB + (IZ * (LB + 1) + JZ) * (LAB + 1);
                  xreg[j * NAB + iab] += tsum<IX + JX, IY + JY, IZ + JZ, false>(
                      fx, fy, fz, [&](auto tx, auto ty, auto tz) {
                        return wc[lex_base(LAB, ERI_CI(tx), ERI_CI(ty)) + ERI_CI(tz)];
                      });
                });
              });
            }
          });
        } else {
        // items (ab, ci)
        for (int it = lane; it < NAB * nci; it += 32) {
          const int iab = it / nci, ci = it - iab * nci;
          const int a0w = tab_ab[2 * iab], a1w = tab_ab[2 * iab + 1];
          const T* fx = Eb + (a0w & 1023);
          const T* fy = Eb + ((a0w >> 10) & 1023);
          const T* fz = Eb + (a0w >> 20);
          const int nx = a1w & 15, ny = (a1w >> 4) & 15, nz = a1w >> 8;
          const T* wc = Ws + ci * HABP;
          T acc = T(0);
          for (int tx = 0; tx <= nx; ++tx) {
            T accy = T(0);
            for (int ty = 0; ty <= ny; ++ty) {
              const T* wr = wc + tab_lex[tx * (LAB + 1) + ty];
              T accz = T(0);
              for (int tz = 0; tz <= nz; ++tz) accz = fma(fz[tz], wr[tz], accz);
              accy = fma(fy[ty], accz, accy);
            }
            acc = fma(fx[tx], accy, acc);
          }
          Xs[iab * CH + ci] += acc;
        }
        }
        __syncwarp();
      }
      if constexpr (S::REGD) {  // X to shared memory for the contraction
        sfor<S::NCS>([&](auto j_) {
          constexpr int j = ERI_CI(j_);
          const int cd = lane + 32 * j;
          if (j * 32 + 32 <= NCD || cd < NCD) {
#pragma unroll
            for (int iab = 0; iab < NAB; ++iab) Xs[iab * CH + cd] = xreg[j * NAB + iab];
          }
        });
        __syncwarp();
      }
      // contraction of the chunk; one lane per output element
      const int cfirst = c0 / ND, clast = (c0 + nci - 1) / ND;
      const int ncr = clast - cfirst + 1;
      if (Kh) {
        // Kh_ac[a][c] += w sum_{b, d: (c,d) in chunk} X D_bd ; Kh_bc[b][c] += w sum_{a,d} X D_ad
        for (int o = lane; o < (NA + NB) * ncr; o += 32) {
          const bool isA = o < NA * ncr;
          const int oo = isA ? o : o - NA * ncr;
          const int r = oo / ncr, c = cfirst + oo % ncr;
          T s = T(0);
          for (int d = 0; d < ND; ++d) {
            const int ci = c * ND + d - c0;
            if (ci < 0 || ci >= nci) continue;
            if (isA) {
              for (int b = 0; b < NB; ++b) s = fma(Xs[(r * NB + b) * CH + ci], __ldg(Dp + (size_t)(ao2 + b) * n + ao4 + d), s);
            } else {
              for (int x = 0; x < NA; ++x) s = fma(Xs[(x * NB + r) * CH + ci], __ldg(Dp + (size_t)(ao1 + x) * n + ao4 + d), s);
            }
          }
          const int row = isA ? ao1 + r : ao2 + r;
          acc_add(Kh + (size_t)row * n + ao3 + c, (double)(w * s), a.det);
        }
        // Kh_ad[a][d] += w sum_{b, c in chunk} X D_bc ; Kh_bd[b][d] += w sum_{a, c} X D_ac
        for (int o = lane; o < (NA + NB) * ND; o += 32) {
          const bool isA = o < NA * ND;
          const int oo = isA ? o : o - NA * ND;
          const int r = oo / ND, d = oo % ND;
          T s = T(0);
          for (int c = cfirst; c <= clast; ++c) {
            const int ci = c * ND + d - c0;
            if (ci < 0 || ci >= nci) continue;
            if (isA) {
              for (int b = 0; b < NB; ++b) s = fma(Xs[(r * NB + b) * CH + ci], __ldg(Dp + (size_t)(ao2 + b) * n + ao3 + c), s);
            } else {
              for (int x = 0; x < NA; ++x) s = fma(Xs[(x * NB + r) * CH + ci], __ldg(Dp + (size_t)(ao1 + x) * n + ao3 + c), s);
            }
          }
          const int row = isA ? ao1 + r : ao2 + r;
          acc_add(Kh + (size_t)row * n + ao4 + d, (double)(w * s), a.det);
        }
      }
      if (Jh) {
        const T w2 = T(2) * w;
        for (int iab = lane; iab < NAB; iab += 32) {  // Jh_ab += 2w sum_cd X D_cd (chunk part)
          T s = T(0);
          for (int ci = 0; ci < nci; ++ci) {
            const int cd = c0 + ci;
            s = fma(Xs[iab * CH + ci], __ldg(Dp + (size_t)(ao3 + cd / ND) * n + ao4 + cd % ND), s);
          }
          acc_add(Jh + (size_t)(ao1 + iab / NB) * n + ao2 + iab % NB, (double)(w2 * s), a.det);
        }
        for (int ci = lane; ci < nci; ci += 32) {  // Jh_cd += 2w sum_ab X D_ab
          T s = T(0);
          for (int iab = 0; iab < NAB; ++iab)
            s = fma(Xs[iab * CH + ci], __ldg(Dp + (size_t)(ao1 + iab / NB) * n + ao2 + iab % NB), s);
          const int cd = c0 + ci;
          acc_add(Jh + (size_t)(ao3 + cd / ND) * n + ao4 + cd % ND, (double)(w2 * s), a.det);
        }
      }
      __syncwarp();
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

}  // namespace eri
