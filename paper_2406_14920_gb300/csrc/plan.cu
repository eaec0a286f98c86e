// Plan construction, preparation kernels and the C ABI (include/eri.h).
//
// Every numerical step of the path runs in a kernel of this library:
//   normalisation (Sec. 2.1)            k_normalize, k_compfac
//   Boys table (Eq. boys_function)      k_boys_table
//   primitive pair data (Eq. pair_definition)   k_pairs
//   Schwarz bounds (Eq. cauchy_schwarz_bound)   k_schwarz
//   class-sorted lists (Sec. 3.2, Eq. kernel_upperbound)   k_sig, k_rank, k_counts, k_prefix
//   Hermite density (Eq. j_formula, first sub-step)        k_hermite_density
//   J-engine / exchange kernels (kernels.cuh)
//   Hermite J -> Cartesian J (Eq. j_formula, last sub-step) k_post_j
//   K symmetrisation (Eq. 8_fold_symmetry)                 k_post_k
//   energies (SI Eq. si_E_J_K)                             k_energy
// Host code only validates arguments, does integer bookkeeping (offsets,
// launch sizes) and launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/eri.h"
#include "dispatch.cuh"
#include "plan.cuh"

using namespace eri;

// ---------------------------------------------------------------------------
// device kernels
// ---------------------------------------------------------------------------

// Per-primitive normalised coefficient of the (l,0,0) component:
// c_k N_l(a_k) s, N_l(a) = (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2l-1)!!),
// s chosen so the contracted (l,0,0) function has unit norm; for two
// normalised (l,0,0) primitives on one centre <g_a|g_b> = (2 sqrt(ab)/(a+b))^(l+3/2).
__global__ void k_normalize(int nshell, const int* __restrict__ l, const int* __restrict__ nprim,
                            const int* __restrict__ poff, const double* __restrict__ ex,
                            const double* __restrict__ co, double* __restrict__ cn) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nshell) return;
  const int L = l[s], n = nprim[s], o = poff[s];
  double df = 1.0;
  for (int k = 2 * L - 1; k > 1; k -= 2) df *= k;
  double S = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double ai = ex[o + i], aj = ex[o + j];
      S += co[o + i] * co[o + j] * pow(2.0 * sqrt(ai * aj) / (ai + aj), L + 1.5);
    }
  const double sc = 1.0 / sqrt(S);
  for (int i = 0; i < n; ++i) {
    double a = ex[o + i];
    cn[o + i] = co[o + i] * sc * pow(2.0 * a / 3.14159265358979323846, 0.75) * pow(4.0 * a, 0.5 * L) / sqrt(df);
  }
}

// Component factor f(x,y,z) = sqrt((2l-1)!! / ((2x-1)!! (2y-1)!! (2z-1)!!)) per AO.
__global__ void k_compfac(int nshell, const int* __restrict__ l, const int* __restrict__ ao, double* __restrict__ f) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nshell) return;
  const int L = l[s];
  auto df = [](int n) {
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= k;
    return r;
  };
  for (int k = 0; k < ncart(L); ++k) {
    int x, y, z;
    cart_xyz(L, k, x, y, z);
    f[ao[s] + k] = sqrt(df(2 * L - 1) / (df(2 * x - 1) * df(2 * y - 1) * df(2 * z - 1)));
  }
}

// Boys tables: F_m(T_k), T_k = k h, from the series for a high order m_top,
// F_m(T) = exp(-T) sum_i (2T)^i / ((2m+1)(2m+3)...(2m+2i+1)), then the stable
// downward recursion F_m = (2T F_{m+1} + exp(-T)) / (2m+1).  Stored as Taylor
// coefficients c[k][m][j] = F_{m+j}(T_k) / j!  and exp(-T_k).
__global__ void k_boys_table(double* __restrict__ c64, double* __restrict__ e64, float* __restrict__ c32,
                             float* __restrict__ e32) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= BOYS_NT) return;
  const double T = k * BOYS_H;
  const int mtop = BOYS_MMAX + BOYS_J64 + 24;
  double term = 1.0 / (2 * mtop + 1), sum = term;
  for (int i = 1; i < 2000; ++i) {
    term *= 2.0 * T / (2 * mtop + 2 * i + 1);
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  const double e = exp(-T);
  double F[BOYS_MMAX + BOYS_J64 + 1];
  double f = e * sum;
  for (int m = mtop - 1; m >= 0; --m) {
    f = (2.0 * T * f + e) / (2 * m + 1);
    if (m <= BOYS_MMAX + BOYS_J64) F[m] = f;
  }
  double fact = 1.0;
  for (int j = 0; j < BOYS_J64; ++j) {
    if (j > 0) fact *= j;
    for (int m = 0; m <= BOYS_MMAX; ++m) {
      c64[((size_t)k * (BOYS_MMAX + 1) + m) * BOYS_J64 + j] = F[m + j] / fact;
      if (j < BOYS_J32) c32[((size_t)k * (BOYS_MMAX + 1) + m) * BOYS_J32 + j] = (float)(F[m + j] / fact);
    }
  }
  e64[k] = e;
  e32[k] = (float)e;
}

// Primitive-pair data for every shell pair (Eq. pair_definition):
// p = a+b, P = (aA+bB)/p, PA = P-A, PB = P-B,
// pref = c_a c_b exp(-ab/p |AB|^2) sqrt(2 pi^(5/2)) / p  (so that a quartet's
// prefactor 2 pi^(5/2)/(pq sqrt(p+q)) K_AB K_CD c c c c = pref_ab pref_cd / sqrt(p+q)).
__global__ void k_pairs(int npair, const int* __restrict__ s1, const int* __restrict__ s2,
                        const int* __restrict__ poff, const int* __restrict__ sh_atom, const int* __restrict__ sh_np,
                        const int* __restrict__ sh_po, const double* __restrict__ ex, const double* __restrict__ cn,
                        const double* __restrict__ coords, int nprimpair, double* p_, double* P_, double* PA_,
                        double* PB_, double* pref_, float* pf, float* Pf, float* PAf, float* PBf, float* preff,
                        float* pmaxp, float* prefmaxp, double* ea_, float4* q4) {
  int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= npair) return;
  const int a = s1[ip], b = s2[ip];
  const double* A = coords + 3 * sh_atom[a];
  const double* Bc = coords + 3 * sh_atom[b];
  double AB2 = 0.0;
  for (int d = 0; d < 3; ++d) AB2 += (A[d] - Bc[d]) * (A[d] - Bc[d]);
  int o = poff[ip];
  double pmx = 0.0, prmx = 0.0;
  const double s2pi52 = 5.9149671727956129;  // sqrt(2 pi^(5/2))
  for (int i = 0; i < sh_np[a]; ++i)
    for (int j = 0; j < sh_np[b]; ++j, ++o) {
      const double ea = ex[sh_po[a] + i], eb = ex[sh_po[b] + j];
      const double p = ea + eb;
      const double pr = cn[sh_po[a] + i] * cn[sh_po[b] + j] * exp(-ea * eb / p * AB2) * s2pi52 / p;
      p_[o] = p;
      ea_[o] = ea;
      pmx = fmax(pmx, p);
      prmx = fmax(prmx, fabs(pr));
      pref_[o] = pr;
      pf[o] = (float)p;
      preff[o] = (float)pr;
      float fP[3], fA[3], fB[3];
      for (int d = 0; d < 3; ++d) {
        const double P = (ea * A[d] + eb * Bc[d]) / p;
        P_[d * nprimpair + o] = P;
        PA_[d * nprimpair + o] = P - A[d];
        PB_[d * nprimpair + o] = P - Bc[d];
        fP[d] = (float)P;
        fA[d] = (float)(P - A[d]);
        fB[d] = (float)(P - Bc[d]);
        Pf[d * nprimpair + o] = fP[d];
        PAf[d * nprimpair + o] = fA[d];
        PBf[d * nprimpair + o] = fB[d];
      }
      q4[3 * (size_t)o] = make_float4(fP[0], fP[1], fP[2], (float)p);
      q4[3 * (size_t)o + 1] = make_float4(fA[0], fA[1], fA[2], (float)pr);
      q4[3 * (size_t)o + 2] = make_float4(fB[0], fB[1], fB[2], 0.0f);
    }
  pmaxp[ip] = (float)pmx;
  prefmaxp[ip] = (float)fmin(prmx, 1.0e30);
}

// Mixed-precision tier split of the items [wl.first, wl.total) of one class
// pair: one warp per chunk of 32 items (chunks t with t % nshard == shard), each
// lane locates and tests one item; the FP64-tier and FP32-tier quartets are
// appended to out0 / out1 (warp-aggregated atomics on cnt[0], cnt[1]).
__global__ void __launch_bounds__(256) k_tier_split(KArgs a, int2* __restrict__ out0, int2* __restrict__ out1,
                                                    unsigned int* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nch = (a.wl.total - a.wl.first + 31) / 32;
  for (int64_t ch = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * a.wl.nshard + a.wl.shard;
       ch < nch; ch += nwarps * a.wl.nshard) {
    const int64_t item = a.wl.first + ch * 32 + lane;
    int tier = -1, ib = 0, ik = 0;
    if (item < a.wl.total) {
      ib = find_bra(a.wl.prefix, a.wl.nbra, item);
      ik = (int)(item - __ldg(a.wl.prefix + ib));
      const int pb_id = __ldg(a.wl.bra + ib);
      const int mol = __ldg(a.sp.pmol + pb_id);
      const int pk_id = __ldg(a.wl.ket + __ldg(a.wl.kseg + mol * NPAIRCLASS) + ik);
      tier = quartet_tier(a, mol, pb_id, pk_id, __ldg(a.sp.s1 + pb_id), __ldg(a.sp.s2 + pb_id),
                          __ldg(a.sp.s1 + pk_id), __ldg(a.sp.s2 + pk_id));
    }
    const unsigned gm = __ballot_sync(0xffffffffu, tier == 2);
    if (gm && lane == 0 && a.guard) atomicAdd(a.guard, (unsigned long long)__popc(gm));
    const unsigned sm = __ballot_sync(0xffffffffu, tier == 3);
    if (sm && lane == 0 && a.screened) atomicAdd(a.screened, (unsigned long long)__popc(sm));
    if (tier == 2) tier = 0;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const unsigned m = __ballot_sync(0xffffffffu, tier == t);
      if (!m) continue;
      unsigned base = 0;
      if (lane == __ffs(m) - 1) base = atomicAdd(cnt + t, (unsigned)__popc(m));
      base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
      if (tier == t) (t == 0 ? out0 : out1)[base + __popc(m & ((1u << lane) - 1u))] = make_int2(ib, ik);
    }
  }
}

// max |D'| over the blocks (s1, s2) and (s2, s1) of every shell pair (used by
// the mixed-precision tier test)
__global__ void k_dmax(int npair, const int* __restrict__ s1, const int* __restrict__ s2, const int* __restrict__ l,
                       const int* __restrict__ pao1, const int* __restrict__ pao2, const int* __restrict__ pmol,
                       const int64_t* __restrict__ mat_off, const int* __restrict__ mat_n,
                       const double* __restrict__ Dp, float* __restrict__ dmax) {
  int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= npair) return;
  const int m = pmol[ip], n = mat_n[m];
  const double* D = Dp + mat_off[m];
  const int a = pao1[ip], b = pao2[ip], na = ncart(l[s1[ip]]), nb = ncart(l[s2[ip]]);
  double mx = 0.0;
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j)
      mx = fmax(mx, fmax(fabs(D[(size_t)(a + i) * n + b + j]), fabs(D[(size_t)(b + j) * n + a + i])));
  dmax[ip] = __double2float_ru(mx);
}


// Hermite coefficients E^{ij}_t (Eq. E_recursion) of every primitive pair, per
// direction, stored as (i*(l2+1)+j)*(l1+l2+1)+t, i <= l1, j <= l2 (x, then y, then z).
__global__ void k_etab(int npair, const int* __restrict__ s1, const int* __restrict__ s2, const int* __restrict__ np,
                       const int* __restrict__ poff, const int* __restrict__ eoff, const int* __restrict__ sh_l,
                       PairData pd, double* __restrict__ E, float* __restrict__ Ef) {
  int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= npair) return;
  const int l1 = sh_l[s1[ip]], l2 = sh_l[s2[ip]];
  const int ne = (l1 + 1) * (l2 + 1) * (l1 + l2 + 1);
  double tmp[225];
  for (int k = 0; k < np[ip]; ++k) {
    const int pi = poff[ip] + k;
    for (int d = 0; d < 3; ++d) {
      md_e_rt(l1, l2, pd.PA[d * pd.n + pi], pd.PB[d * pd.n + pi], 0.5 / pd.p[pi], tmp);
      const size_t o = (size_t)eoff[ip] + ((size_t)k * 3 + d) * ne;
      for (int i = 0; i <= l1; ++i)
        for (int j = 0; j <= l2; ++j)
          for (int t = 0; t <= l1 + l2; ++t) {
            const double v = tmp[(i * 5 + j) * 9 + t];
            E[o + (i * (l2 + 1) + j) * (l1 + l2 + 1) + t] = v;
            Ef[o + (i * (l2 + 1) + j) * (l1 + l2 + 1) + t] = (float)v;
          }
    }
  }
}

// Schwarz bound per shell pair: Q = sqrt(max_{mu,nu} |(mu nu|mu nu)|) in FP64, rounded up to float32.
__global__ void k_schwarz(int npair, const int* __restrict__ s1, const int* __restrict__ s2, const int* __restrict__ np,
                          const int* __restrict__ poff, const int* __restrict__ sh_l, const int* __restrict__ ao,
                          const double* __restrict__ f, PairData pd, BoysTabs bt,
                          const RStep* __restrict__ st, float* __restrict__ Q) {
  int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= npair) return;
  const int l1 = sh_l[s1[ip]], l2 = sh_l[s2[ip]], lp = l1 + l2, L = 2 * lp;
  const int n1 = ncart(l1), n2 = ncart(l2);
  double diag[100];
  for (int x = 0; x < n1 * n2; ++x) diag[x] = 0.0;
  double E1[3][225], E2[3][225], Ra[455], Rb[455], F[13];
  for (int i = 0; i < np[ip]; ++i) {
    const int pi = poff[ip] + i;
    for (int d = 0; d < 3; ++d) md_e_rt(l1, l2, pd.PA[d * pd.n + pi], pd.PB[d * pd.n + pi], 0.5 / pd.p[pi], E1[d]);
    for (int j = 0; j < np[ip]; ++j) {
      const int pj = poff[ip] + j;
      for (int d = 0; d < 3; ++d) md_e_rt(l1, l2, pd.PA[d * pd.n + pj], pd.PB[d * pd.n + pj], 0.5 / pd.p[pj], E2[d]);
      const double p = pd.p[pi], q = pd.p[pj], rho = p * q / (p + q);
      double X = pd.P[pi] - pd.P[pj], Y = pd.P[pd.n + pi] - pd.P[pd.n + pj], Z = pd.P[2 * pd.n + pi] - pd.P[2 * pd.n + pj];
      const double T = rho * (X * X + Y * Y + Z * Z);
      // generic Boys (runtime order): Taylor at the top order then downward
      if (T < BOYS_TMAX) {
        int k = __double2int_rn(T * BOYS_INV_H);
        const double* c = bt.c64 + ((size_t)k * (BOYS_MMAX + 1) + L) * BOYS_J64;
        double dd = k * BOYS_H - T, acc = c[BOYS_J64 - 1];
        for (int jj = BOYS_J64 - 2; jj >= 0; --jj) acc = acc * dd + c[jj];
        F[L] = acc;
        double e = exp(-T);
        for (int m = L - 1; m >= 0; --m) F[m] = (2 * T * F[m + 1] + e) / (2 * m + 1);
      } else {
        double e = exp(-T);
        F[0] = 0.5 * sqrt(3.14159265358979323846 / T);
        for (int m = 0; m < L; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) / (2 * T);
      }
      const double pref = pd.pref[pi] * pd.pref[pj] / sqrt(p + q);
      // R into Ra (ping-pong with Rb), result lands in Ra if L even else Rb
      double* cur = Ra;
      double* nxt = Rb;
      cur[0] = pref * F[L];
      for (int m = L - 1; m >= 0; --m) {
        int ne = nherm(L - m);
        for (int e = 0; e < ne; ++e) {
          if (e == 0) { nxt[0] = pref * F[m]; continue; }
          RStep s = st[e];
          double pq = s.dir == 0 ? X : (s.dir == 1 ? Y : Z);
          double v = pq * cur[s.dep1];
          if (s.dep2 >= 0) v += s.k * cur[s.dep2];
          nxt[e] = -2.0 * rho * v;
        }
        double* t = cur; cur = nxt; nxt = t;
      }
      const double* R = cur;
      for (int mu = 0; mu < n1; ++mu) {
        int ix, iy, iz;
        cart_xyz(l1, mu, ix, iy, iz);
        for (int nu = 0; nu < n2; ++nu) {
          int jx, jy, jz;
          cart_xyz(l2, nu, jx, jy, jz);
          double v = 0.0;
          for (int tx = 0; tx <= ix + jx; ++tx)
            for (int ty = 0; ty <= iy + jy; ++ty)
              for (int tz = 0; tz <= iz + jz; ++tz) {
                const double ep = E1[0][(ix * 5 + jx) * 9 + tx] * E1[1][(iy * 5 + jy) * 9 + ty] * E1[2][(iz * 5 + jz) * 9 + tz];
                for (int sx = 0; sx <= ix + jx; ++sx)
                  for (int sy = 0; sy <= iy + jy; ++sy)
                    for (int sz = 0; sz <= iz + jz; ++sz) {
                      const double eq = E2[0][(ix * 5 + jx) * 9 + sx] * E2[1][(iy * 5 + jy) * 9 + sy] *
                                        E2[2][(iz * 5 + jz) * 9 + sz];
                      const double sg = ((sx + sy + sz) & 1) ? -1.0 : 1.0;
                      v += ep * eq * sg * R[herm_index(tx + sx, ty + sy, tz + sz)];
                    }
              }
          const double fn = f[ao[s1[ip]] + mu] * f[ao[s2[ip]] + nu];
          diag[mu * n2 + nu] += v * fn * fn;
        }
      }
    }
  }
  double mx = 0.0;
  for (int x = 0; x < n1 * n2; ++x) mx = fmax(mx, fabs(diag[x]));
  (void)lp;
  Q[ip] = __double2float_ru(sqrt(mx));
}

// Per-molecule Schwarz maximum (pairs never cross molecules).  Q >= 0, so
// the unsigned order of the float bits is the float order.
__global__ void k_qmax(int n, const float* __restrict__ Q, const int* __restrict__ pmol, unsigned int* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = i < n ? pmol[i] : -1;
  unsigned int v = i < n ? __float_as_uint(Q[i]) : 0u;
  const int m0 = __shfl_sync(0xffffffffu, m, 0);
  if (__all_sync(0xffffffffu, m == m0 || m < 0)) {
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && m0 >= 0) atomicMax(out + m0, v);
  } else if (m >= 0) {
    atomicMax(out + m, v);
  }
}

// significance of each pair: (double)Q * (double)Qmax(molecule) >= thresh;
// counts per (molecule, class)
__global__ void k_sig(int npair, const float* __restrict__ Q, const int* __restrict__ pmol,
                      const unsigned int* __restrict__ qmax_bits, double thresh, const int* __restrict__ cls,
                      int* __restrict__ sig, int* __restrict__ ccm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npair) return;
  const int m = pmol[i];
  const double qmax = (double)__uint_as_float(qmax_bits[m]);
  const int s = ((double)Q[i] * qmax >= thresh) ? 1 : 0;
  sig[i] = s;
  if (s) atomicAdd(ccm + m * NPAIRCLASS + cls[i], 1);
}

// rank of each significant pair inside its (molecule, class) segment: Q
// descending, pair index ascending.  The sorted array is class-major, molecule
// by molecule inside a class: segment (X, m) starts at coff[X] + segloc[m][X].
__global__ void k_rank(int npair, const float* __restrict__ Q, const int* __restrict__ cls, const int* __restrict__ sig,
                       const int* __restrict__ pmol, const int* __restrict__ pbase, const int* __restrict__ coff,
                       const int* __restrict__ segloc, int* __restrict__ sorted, int* __restrict__ pos) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npair || !sig[i]) return;
  const float qi = Q[i];
  const int ci = cls[i], m = pmol[i];
  int r = 0;
  for (int j = pbase[m]; j < pbase[m + 1]; ++j) {
    if (!sig[j] || cls[j] != ci) continue;
    const float qj = Q[j];
    if (qj > qi || (qj == qi && j < i)) ++r;
  }
  sorted[coff[ci] + segloc[m * NPAIRCLASS + ci] + r] = i;
  pos[i] = r;
}

// counts[pair][Y] = number of kets of class Y (same molecule) with Q_i Q_k >= thresh
// (binary search on the Q-sorted segment)
__global__ void k_counts(int npair, const float* __restrict__ Q, const int* __restrict__ sig,
                         const int* __restrict__ pmol, const int* __restrict__ sorted, const int* __restrict__ coff,
                         const int* __restrict__ segloc, const int* __restrict__ ccm, double thresh,
                         int* __restrict__ counts) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npair * NPAIRCLASS) return;
  const int i = t / NPAIRCLASS, Y = t % NPAIRCLASS;
  if (!sig[i]) { counts[t] = 0; return; }
  const int m = pmol[i];
  const double qi = (double)Q[i];
  const int* lst = sorted + coff[Y] + segloc[m * NPAIRCLASS + Y];
  int lo = 0, hi = ccm[m * NPAIRCLASS + Y];  // first position with Q_i Q_k < thresh
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (qi * (double)Q[lst[mid]] >= thresh) lo = mid + 1; else hi = mid;
  }
  counts[t] = lo;
}

// Exclusive scan of one int64 per thread over the block (blockDim.x a multiple
// of 32); *total receives the block sum.  Every thread of the block must call it.
__device__ __forceinline__ int64_t block_exscan(int64_t v, int64_t* wsum, int64_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t t = lane < nw ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) wsum[lane] = t;
  }
  __syncthreads();
  const int64_t before = w > 0 ? wsum[w - 1] : 0;
  *total = wsum[nw - 1];
  __syncthreads();
  return before + x - v;
}

// cumnp[coff[Y] + Y + k] = primitive pairs of the first k entries of class Y's
// sorted list (all molecules, in list order); one block per class
__global__ void k_cumnp(const int* __restrict__ sorted, const int* __restrict__ coff, const int* __restrict__ ccount,
                        const int* __restrict__ np, int64_t* __restrict__ cumnp) {
  __shared__ int64_t wsum[32];
  const int Y = blockIdx.x;
  const int n = ccount[Y];
  const int* kl = sorted + coff[Y];
  int64_t* out = cumnp + coff[Y] + Y;  // class Y occupies ccount[Y] + 1 slots
  int64_t carry = 0;
  for (int base = 0; base < n; base += blockDim.x) {
    const int k = base + threadIdx.x;
    const int64_t v = k < n ? np[kl[k]] : 0;
    int64_t tot;
    const int64_t ex = block_exscan(v, wsum, &tot);
    if (k < n) out[k] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) out[n] = carry;
}

// Prefix arrays of the K (canonical) and J (ordered) work lists, one block per
// class pair (X, Y).  A bra of class X sees the kets of class Y of its own
// molecule; canonical lists (Y <= X) keep, for X == Y, only kets at or before
// the bra's own rank in the (molecule, class) segment.
__global__ void k_prefix(const int* __restrict__ sorted, const int* __restrict__ coff, const int* __restrict__ ccount,
                         const int* __restrict__ segloc, const int* __restrict__ pmol, const int* __restrict__ pos,
                         const int* __restrict__ counts, const int64_t* __restrict__ koff,
                         const int64_t* __restrict__ joff, int64_t* __restrict__ kpre, int64_t* __restrict__ jpre,
                         int64_t* __restrict__ ktot, int64_t* __restrict__ jtot, const int* __restrict__ np,
                         const int64_t* __restrict__ cumnp, int64_t* __restrict__ kprim) {
  __shared__ int64_t wsum[32];
  const int cp = blockIdx.x;
  const int X = cp / NPAIRCLASS, Y = cp % NPAIRCLASS;
  const bool canon = Y <= X;
  const int nb = ccount[X];
  const int* bl = sorted + coff[X];
  int64_t* jp = jpre + joff[cp];
  int64_t* kp = canon ? kpre + koff[cp] : nullptr;
  const int64_t* cy = cumnp + coff[Y] + Y;
  int64_t cj_carry = 0, ck_carry = 0, cp_carry = 0;
  for (int base = 0; base < nb; base += blockDim.x) {
    const int i = base + threadIdx.x;
    int64_t cj = 0, ck = 0, pp = 0;
    if (i < nb) {
      const int b = bl[i];
      cj = counts[b * NPAIRCLASS + Y];
      if (canon) {
        ck = cj;
        if (X == Y && ck > pos[b] + 1) ck = pos[b] + 1;
        const int s0 = segloc[pmol[b] * NPAIRCLASS + Y];
        pp = (cy[s0 + ck] - cy[s0]) * np[b];
      }
    }
    int64_t tot;
    const int64_t exj = block_exscan(cj, wsum, &tot);
    if (i < nb) jp[i] = cj_carry + exj;
    cj_carry += tot;
    if (canon) {
      const int64_t exk = block_exscan(ck, wsum, &tot);
      if (i < nb) kp[i] = ck_carry + exk;
      ck_carry += tot;
      block_exscan(pp, wsum, &tot);
      cp_carry += tot;
    }
  }
  if (threadIdx.x == 0) {
    jp[nb] = cj_carry;
    jtot[cp] = cj_carry;
    if (canon) {
      kp[nb] = ck_carry;
      ktot[cp] = ck_carry;
      kprim[cp] = cp_carry;
    }
  }
}

// Where each molecule's nbf_m x nbf_m block sits in packed D / J / K, and the
// global AO index of its first function (component factors f are global).

// D' = D f f (component norms folded in); grid (x, molecule)
__global__ void k_scale_d(MolMats mm, const double* __restrict__ D, const double* __restrict__ f,
                          double* __restrict__ Dp, float* __restrict__ Dpf) {
  const int m = blockIdx.y, n = mm.n[m];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n) return;
  const int64_t o = mm.off[m] + i;
  const int a0 = mm.aobase[m];
  const double v = D[o] * f[a0 + i / n] * f[a0 + i % n];
  Dp[o] = v;
  if (Dpf) Dpf[o] = (float)v;
}

// Hermite density per primitive pair (Eq. j_formula, first sub-step):
// D_Q = (-1)^|Q| s sum_{l in s1, s in s2} E_Q^{ls} D'_ls, s = 2 for s1 != s2
// (the pair stands for both orders), 1 for a diagonal pair.
__global__ void k_hermite_density(int npair, const int* __restrict__ s1, const int* __restrict__ s2,
                                  const int* __restrict__ np, const int* __restrict__ poff, const int* __restrict__ hoff,
                                  const int* __restrict__ sh_l, const int* __restrict__ pao1,
                                  const int* __restrict__ pao2, const int* __restrict__ pmol, MolMats mm,
                                  const int* __restrict__ sig, PairData pd, const double* __restrict__ Dp,
                                  double* __restrict__ Dh, float* __restrict__ Dhf) {
  int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= npair || !sig[ip]) return;
  const int a = s1[ip], b = s2[ip], la = sh_l[a], lb = sh_l[b], H = nherm(la + lb);
  const int m = pmol[ip], nbf = mm.n[m];
  const double* Dm = Dp + mm.off[m];
  const double sc = a == b ? 1.0 : 2.0;
  double E[3][225];
  for (int k = 0; k < np[ip]; ++k) {
    const int pi = poff[ip] + k;
    for (int d = 0; d < 3; ++d) md_e_rt(la, lb, pd.PA[d * pd.n + pi], pd.PB[d * pd.n + pi], 0.5 / pd.p[pi], E[d]);
    double* out = Dh + hoff[ip] + (size_t)k * H;
    for (int q = 0; q < H; ++q) out[q] = 0.0;
    for (int mu = 0; mu < ncart(la); ++mu) {
      int ix, iy, iz;
      cart_xyz(la, mu, ix, iy, iz);
      for (int nu = 0; nu < ncart(lb); ++nu) {
        int jx, jy, jz;
        cart_xyz(lb, nu, jx, jy, jz);
        const double dv = sc * Dm[(size_t)(pao1[ip] + mu) * nbf + pao2[ip] + nu];
        for (int tx = 0; tx <= ix + jx; ++tx)
          for (int ty = 0; ty <= iy + jy; ++ty)
            for (int tz = 0; tz <= iz + jz; ++tz) {
              const double sg = ((tx + ty + tz) & 1) ? -1.0 : 1.0;
              out[herm_index(tx, ty, tz)] +=
                  sg * dv * E[0][(ix * 5 + jx) * 9 + tx] * E[1][(iy * 5 + jy) * 9 + ty] * E[2][(iz * 5 + jz) * 9 + tz];
            }
      }
    }
    if (Dhf)  // FP32 copy for the FP32 tier of a mixed J-engine build
      for (int q = 0; q < H; ++q) Dhf[hoff[ip] + (size_t)k * H + q] = (float)out[q];
  }
}

// Cartesian J from Hermite J (Eq. j_formula, last sub-step): thread per (pair, mu, nu)
__global__ void k_post_j(int npair, const int* __restrict__ s1, const int* __restrict__ s2, const int* __restrict__ np,
                         const int* __restrict__ poff, const int* __restrict__ hoff, const int* __restrict__ sh_l,
                         const int* __restrict__ pao1, const int* __restrict__ pao2, const int* __restrict__ pmol,
                         MolMats mm, const int* __restrict__ sig, PairData pd, const double* __restrict__ Jh,
                         const double* __restrict__ f, double* __restrict__ J, int det, int* __restrict__ status) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npair * 100) return;
  const int ip = t / 100, c = t % 100;
  if (sig && !sig[ip]) return;
  const int a = s1[ip], b = s2[ip], la = sh_l[a], lb = sh_l[b];
  const int mu = c / 10, nu = c % 10;
  if (mu >= ncart(la) || nu >= ncart(lb)) return;
  int ix, iy, iz, jx, jy, jz;
  cart_xyz(la, mu, ix, iy, iz);
  cart_xyz(lb, nu, jx, jy, jz);
  const int H = nherm(la + lb);
  double E[3][225];
  double v = 0.0;
  for (int k = 0; k < np[ip]; ++k) {
    const int pi = poff[ip] + k;
    for (int d = 0; d < 3; ++d) md_e_rt(la, lb, pd.PA[d * pd.n + pi], pd.PB[d * pd.n + pi], 0.5 / pd.p[pi], E[d]);
    const double* jh = Jh + hoff[ip] + (size_t)k * H;
    for (int tx = 0; tx <= ix + jx; ++tx)
      for (int ty = 0; ty <= iy + jy; ++ty)
        for (int tz = 0; tz <= iz + jz; ++tz) {
          const double hv = acc_value(jh + herm_index(tx, ty, tz), det);
          if (det && fabs(hv) > kFixLimit) atomicOr(status, DEV_RANGE);
          v += E[0][(ix * 5 + jx) * 9 + tx] * E[1][(iy * 5 + jy) * 9 + ty] * E[2][(iz * 5 + jz) * 9 + tz] * hv;
        }
  }
  const int m = pmol[ip], nbf = mm.n[m], a0 = mm.aobase[m];
  const int r = pao1[ip] + mu, cc = pao2[ip] + nu;
  v *= f[a0 + r] * f[a0 + cc];
  double* Jm = J + mm.off[m];
  Jm[(size_t)r * nbf + cc] = v;
  if (a != b) Jm[(size_t)cc * nbf + r] = v;
}

// K = (Kh + Kh^T) f f  (Eq. 8_fold_symmetry: the transposes carry permutations 5-8); grid (x, molecule)
// (deterministic builds: Kh holds fixed point, see acc_add; an element above the
// reporting limit sets DEV_RANGE in the plan's status word)
__global__ void k_post_k(MolMats mm, const double* __restrict__ Kh, const double* __restrict__ f,
                         double* __restrict__ K, int det, int* __restrict__ status) {
  const int m = blockIdx.y, n = mm.n[m];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n) return;
  const int r = (int)(i / n), c = (int)(i % n), a0 = mm.aobase[m];
  const int64_t o = mm.off[m];
  const double x = acc_value(Kh + o + i, det), y = acc_value(Kh + o + (int64_t)c * n + r, det);
  if (det && (fabs(x) > kFixLimit || fabs(y) > kFixLimit)) atomicOr(status, DEV_RANGE);
  K[o + i] = (x + y) * f[a0 + r] * f[a0 + c];
}

// deterministic gradient: fixed-point accumulators -> doubles, in place
__global__ void k_fix_to_double(int n, double* __restrict__ x, int* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = acc_value(x + i, 1);
  if (fabs(v) > kFixLimit) atomicOr(status, DEV_RANGE);
  x[i] = v;
}

// E_J = 1/2 sum D J, E_K = -1/4 sum D K per molecule (one block each, fixed
// order: deterministic); E[2m], E[2m+1]
__global__ void k_energy(MolMats mm, const double* __restrict__ D, const double* __restrict__ J,
                         const double* __restrict__ K, double* __restrict__ E) {
  __shared__ double sj[32], sk[32];
  const int m = blockIdx.x;
  const int64_t nn = (int64_t)mm.n[m] * mm.n[m], o = mm.off[m];
  double aj = 0.0, ak = 0.0;
  for (int64_t i = threadIdx.x; i < nn; i += blockDim.x) {
    if (J) aj += D[o + i] * J[o + i];
    if (K) ak += D[o + i] * K[o + i];
  }
  for (int w = 16; w > 0; w >>= 1) {
    aj += __shfl_xor_sync(0xffffffffu, aj, w);
    ak += __shfl_xor_sync(0xffffffffu, ak, w);
  }
  if ((threadIdx.x & 31) == 0) { sj[threadIdx.x >> 5] = aj; sk[threadIdx.x >> 5] = ak; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tj = 0.0, tk = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tj += sj[w]; tk += sk[w]; }
    E[2 * m] = 0.5 * tj;
    E[2 * m + 1] = -0.25 * tk;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return eri_fail(e_); \
  } while (0)

static int eri_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return ERI_ENOMEM;
  return ERI_ECUDA;
}

template <typename T>
static cudaError_t dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc((void**)p, n * sizeof(T));
}

static int grid1(int64_t n, int b) { return (int)((n + b - 1) / b); }

static std::vector<RStep> make_rsteps() {
  std::vector<RStep> st(nherm(LMAX_QUARTET));
  for (int n = 0; n <= LMAX_QUARTET; ++n)
    for (int r = 0; r <= n; ++r)
      for (int v = 0; v <= r; ++v) {
        int u = r - v, t = n - r;
        int e = herm_index(t, u, v);
        RStep s{};
        s.t = (uint8_t)t; s.u = (uint8_t)u; s.v = (uint8_t)v;
        s.dep1 = -1; s.dep2 = -1; s.k = 0; s.dir = 0;
        int c[3] = {t, u, v};
        if (n > 0) {
          int d = t > 0 ? 0 : (u > 0 ? 1 : 2);
          s.dir = (uint8_t)d;
          int c1[3] = {c[0], c[1], c[2]};
          c1[d] -= 1;
          s.dep1 = (int16_t)herm_index(c1[0], c1[1], c1[2]);
          if (c1[d] > 0) {
            int c2[3] = {c1[0], c1[1], c1[2]};
            c2[d] -= 1;
            s.dep2 = (int16_t)herm_index(c2[0], c2[1], c2[2]);
            s.k = (int16_t)c1[d];
          }
        }
        st[e] = s;
      }
  return st;
}

int eri_plan_impl::alloc_pairs() {
  CK(dalloc(&d_p, nprimpair)); CK(dalloc(&d_P, 3 * (size_t)nprimpair)); CK(dalloc(&d_PA, 3 * (size_t)nprimpair));
  CK(dalloc(&d_PB, 3 * (size_t)nprimpair)); CK(dalloc(&d_pref, nprimpair));
  CK(dalloc(&d_pf, nprimpair)); CK(dalloc(&d_Pf, 3 * (size_t)nprimpair)); CK(dalloc(&d_PAf, 3 * (size_t)nprimpair));
  CK(dalloc(&d_PBf, 3 * (size_t)nprimpair)); CK(dalloc(&d_preff, nprimpair));
  CK(dalloc(&d_q4, 3 * (size_t)nprimpair));
  return ERI_OK;
}

PairData eri_plan_impl::pairdata() const {
  PairData pd;
  pd.p = d_p; pd.P = d_P; pd.PA = d_PA; pd.PB = d_PB; pd.pref = d_pref;
  pd.pf = d_pf; pd.Pf = d_Pf; pd.PAf = d_PAf; pd.PBf = d_PBf; pd.preff = d_preff;
  pd.E = d_E; pd.Ef = d_Ef; pd.ea = d_ea; pd.q4 = d_q4;
  pd.n = nprimpair;
  return pd;
}

BoysTabs eri_plan_impl::boystabs() const {
  BoysTabs b;
  b.c64 = d_boys64; b.e64 = d_bexp64; b.c32 = d_boys32; b.e32 = d_bexp32;
  return b;
}

ShellPairInfo eri_plan_impl::spinfo() const {
  ShellPairInfo sp;
  sp.s1 = d_ps1; sp.s2 = d_ps2; sp.np = d_pnp; sp.poff = d_ppoff; sp.ao1 = d_pao1; sp.ao2 = d_pao2; sp.hoff = d_phoff; sp.eoff = d_peoff;
  sp.pmol = d_pmol; sp.mat_off = d_mat_off; sp.mat_n = d_mat_n;
  return sp;
}

dim3 eri_plan_impl::mat_grid(int block) const {
  return dim3((unsigned)std::max<int64_t>(1, ((int64_t)max_nbf * max_nbf + block - 1) / block), (unsigned)nmol);
}

// D' = D f f into the plan's FP64 workspace (also used by nuclear.cu)
void k_scale_d_launch(const eri_plan_impl* P, const double* D, cudaStream_t s) {
  k_scale_d<<<P->mat_grid(256), 256, 0, s>>>(molmats(P), D, P->d_f, P->d_Dp, nullptr);
}

MolMats molmats(const eri_plan_impl* P) {
  MolMats m;
  m.off = P->d_mat_off; m.n = P->d_mat_n; m.aobase = P->d_aobase;
  return m;
}

// pair data + Schwarz + lists for the current device coordinates
int eri_plan_impl::geometry(cudaStream_t s, bool rebuild_q) {
  k_pairs<<<grid1(npair, 128), 128, 0, s>>>(npair, d_ps1, d_ps2, d_ppoff, d_sh_atom, d_sh_np, d_sh_po, d_exps, d_cn,
                                        d_coords, nprimpair, d_p, d_P, d_PA, d_PB, d_pref, d_pf, d_Pf, d_PAf, d_PBf,
                                        d_preff, d_pmaxp, d_prefmaxp, d_ea, d_q4);
  CK(cudaGetLastError());
  k_etab<<<grid1(npair, 64), 64, 0, s>>>(npair, d_ps1, d_ps2, d_pnp, d_ppoff, d_peoff, d_sh_l, pairdata(), d_E, d_Ef);
  CK(cudaGetLastError());
  if (rebuild_q) {
    k_schwarz<<<grid1(npair, 64), 64, 0, s>>>(npair, d_ps1, d_ps2, d_pnp, d_ppoff, d_sh_l, d_sh_ao, d_f, pairdata(), boystabs(),
                                              d_rsteps, d_Q);
    CK(cudaGetLastError());
    return build_lists(thresh, s);
  }
  return ERI_OK;
}

int eri_plan_impl::build_lists(double th, cudaStream_t s) {
  thresh = th;
  if (gexec) {  // a captured build holds the old list sizes and offsets
    CK(cudaDeviceSynchronize());
    CK(cudaGraphExecDestroy(gexec));
    gexec = nullptr;
  }
  const int nm10 = nmol * NPAIRCLASS;
  CK(cudaMemsetAsync(d_qmax, 0, sizeof(unsigned int) * nmol, s));
  CK(cudaMemsetAsync(d_ccm, 0, sizeof(int) * nm10, s));
  k_qmax<<<grid1(npair, 256), 256, 0, s>>>(npair, d_Q, d_pmol, d_qmax);
  k_sig<<<grid1(npair, 256), 256, 0, s>>>(npair, d_Q, d_pmol, d_qmax, th, d_pcls, d_sig, d_ccm);
  CK(cudaGetLastError());
  h_ccm.assign(nm10, 0);
  CK(cudaMemcpyAsync(h_ccm.data(), d_ccm, sizeof(int) * nm10, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // class-major layout, molecule by molecule inside a class
  h_segloc.assign(nm10, 0);
  int acc = 0;
  for (int X = 0; X < NPAIRCLASS; ++X) {
    h_coff[X] = acc;
    int loc = 0;
    for (int m = 0; m < nmol; ++m) {
      h_segloc[m * NPAIRCLASS + X] = loc;
      loc += h_ccm[m * NPAIRCLASS + X];
    }
    h_ccount[X] = loc;
    acc += loc;
  }
  nsig = acc;
  CK(cudaMemcpyAsync(d_coff, h_coff, sizeof(int) * NPAIRCLASS, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_ccount, h_ccount, sizeof(int) * NPAIRCLASS, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_segloc, h_segloc.data(), sizeof(int) * nm10, cudaMemcpyHostToDevice, s));
  k_rank<<<grid1(npair, 256), 256, 0, s>>>(npair, d_Q, d_pcls, d_sig, d_pmol, d_pbase, d_coff, d_segloc, d_sorted,
                                           d_pos);
  k_counts<<<grid1((int64_t)npair * NPAIRCLASS, 256), 256, 0, s>>>(npair, d_Q, d_sig, d_pmol, d_sorted, d_coff,
                                                                   d_segloc, d_ccm, th, d_counts);
  CK(cudaGetLastError());
  int64_t ko = 0, jo = 0;
  for (int X = 0; X < NPAIRCLASS; ++X)
    for (int Y = 0; Y < NPAIRCLASS; ++Y) {
      h_koff[X * NPAIRCLASS + Y] = ko;
      h_joff[X * NPAIRCLASS + Y] = jo;
      jo += h_ccount[X] + 1;
      if (Y <= X) ko += h_ccount[X] + 1;
    }
  if (ko > kpre_cap) {
    cudaFree(d_kpre);
    CK(dalloc(&d_kpre, ko));
    kpre_cap = ko;
  }
  if (jo > jpre_cap) {
    cudaFree(d_jpre);
    CK(dalloc(&d_jpre, jo));
    jpre_cap = jo;
  }
  CK(cudaMemcpyAsync(d_koff, h_koff, sizeof(h_koff), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_joff, h_joff, sizeof(h_joff), cudaMemcpyHostToDevice, s));
  k_cumnp<<<NPAIRCLASS, 1024, 0, s>>>(d_sorted, d_coff, d_ccount, d_pnp, d_cumnp);
  k_prefix<<<NPAIRCLASS * NPAIRCLASS, 1024, 0, s>>>(d_sorted, d_coff, d_ccount, d_segloc, d_pmol, d_pos, d_counts,
                                                     d_koff, d_joff, d_kpre, d_jpre, d_ktot, d_jtot, d_pnp, d_cumnp,
                                                     d_kprim);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h_ktot, d_ktot, sizeof(h_ktot), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h_jtot, d_jtot, sizeof(h_jtot), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h_kprim, d_kprim, sizeof(h_kprim), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return ERI_OK;
}

WorkList eri_plan_impl::klist(int X, int Y) const {
  WorkList w;
  w.first = 0;
  w.tile = 1;
  w.shard = shard;
  w.nshard = nshard;
  w.bra = d_sorted + h_coff[X];
  w.ket = d_sorted + h_coff[Y];
  w.kseg = d_segloc + Y;
  w.prefix = d_kpre + h_koff[X * NPAIRCLASS + Y];
  w.nbra = h_ccount[X];
  w.total = h_ktot[X * NPAIRCLASS + Y];
  return w;
}

WorkList eri_plan_impl::jlist(int X, int Y) const {
  WorkList w;
  w.first = 0;
  w.tile = 4;
  w.shard = shard;
  w.nshard = nshard;
  w.bra = d_sorted + h_coff[X];
  w.ket = d_sorted + h_coff[Y];
  w.kseg = d_segloc + Y;
  w.prefix = d_jpre + h_joff[X * NPAIRCLASS + Y];
  w.nbra = h_ccount[X];
  w.total = h_jtot[X * NPAIRCLASS + Y];
  return w;
}

void eri_plan_impl::release() {
  void* ptrs[] = {d_sh_l, d_sh_atom, d_sh_np, d_sh_po, d_sh_ao, d_exps, d_coefs, d_cn, d_f, d_coords, d_ps1, d_ps2,
                  d_pnp, d_ppoff, d_pao1, d_pao2, d_phoff, d_pcls, d_p, d_P, d_PA, d_PB, d_pref, d_pf, d_Pf, d_PAf,
                  d_PBf, d_preff, d_Q, d_qmax, d_sig, d_ccount, d_coff, d_sorted, d_pos, d_counts, d_koff, d_joff,
                  d_kpre, d_jpre, d_ktot, d_jtot, d_kprim, d_boys64, d_boys32, d_rsteps, d_Dp, d_Kh, d_Jh, d_Dherm,
                  d_Jherm, d_status, d_bexp64, d_bexp32, d_peoff, d_E, d_Ef, d_pmaxp, d_dmax, d_counters, d_cumnp, d_prefmaxp, d_ea,
                  d_mat_off, d_mat_n, d_aobase, d_pbase, d_pmol, d_shloc, d_ccm, d_segloc, d_Dpf,
                  d_nuc_list, d_nuc_goff, d_nuc_dens, d_counters2, d_q4, d_Dhermf};
  xc_release();
  for (auto& e : prof_events) cudaEventDestroy(e);
  prof_events.clear();
  if (gexec) cudaGraphExecDestroy(gexec);
  gexec = nullptr;
  for (int b = 0; b < kBranches; ++b) {
    if (branch[b]) cudaStreamDestroy(branch[b]);
    if (join_ev[b]) cudaEventDestroy(join_ev[b]);
    branch[b] = nullptr;
    join_ev[b] = nullptr;
  }
  for (int b = 0; b < kBranches; ++b) {
    if (tbuf[b]) cudaFree(tbuf[b]);
    tbuf[b] = nullptr;
  }
  if (tcnt) cudaFree(tcnt);
  tcnt = nullptr;
  if (fork_ev) cudaEventDestroy(fork_ev);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  fork_ev = nullptr;
  cap_stream = nullptr;
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// pairs with an exponent sum above this stay in FP64 in mixed mode (FP32 range)
static const double kPmax32 = 1.0e3;

static const int kClassL1[NPAIRCLASS] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3};
static const int kClassL2[NPAIRCLASS] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};

int eri_plan_impl::ensure_streams() {
  if (cap_stream) return ERI_OK;
  CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
  for (int b = 0; b < kBranches; ++b) {
    CK(cudaStreamCreateWithFlags(&branch[b], cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&join_ev[b], cudaEventDisableTiming));
  }
  return ERI_OK;
}

// Compacted tier lists of mixed-precision builds: per branch, two lists of
// tier_cap items (int2 bra / ket positions) and two counters.  tier_cap is the
// longest class-pair list, at most kTierCap; longer lists are split in windows.
static const int64_t kTierCap = 1 << 23;

int eri_plan_impl::ensure_tier_bufs(int nb) {
  int64_t mx = 1;
  for (int X = 0; X < NPAIRCLASS; ++X)
    for (int Y = 0; Y <= X; ++Y) mx = std::max(mx, h_ktot[X * NPAIRCLASS + Y]);
  const int64_t cap = std::min(mx, kTierCap);
  if (cap > tier_cap) {
    CK(cudaDeviceSynchronize());
    for (int b = 0; b < kBranches; ++b) {
      if (tbuf[b]) cudaFree(tbuf[b]);
      tbuf[b] = nullptr;
    }
    tier_nb = 0;
    tier_cap = cap;
  }
  if (!tcnt) CK(dalloc(&tcnt, 2 * kBranches));
  for (int b = tier_nb; b < nb; ++b) CK(dalloc(&tbuf[b], 2 * (size_t)tier_cap));
  tier_nb = std::max(tier_nb, nb);
  return ERI_OK;
}

cudaError_t eri_plan_impl::prof_event_pair(cudaEvent_t* a, cudaEvent_t* b) {
  while ((int)prof_events.size() < prof_ev_used + 2) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    prof_events.push_back(e);
  }
  *a = prof_events[prof_ev_used];
  *b = prof_events[prof_ev_used + 1];
  prof_ev_used += 2;
  return cudaSuccess;
}

// Algorithmic FLOPs of the McMurchie-Davidson J/K path as implemented (FMA = 2):
//   per primitive quartet: Boys 2(L+1)+20, R recursion 3 sum_{m<L} (nherm(L-m)-1),
//     ket transform 2 nherm(la+lb) sum_{cd} prod_t (k_t+l_t+1);
//   per bra primitive of a quartet: bra transform 2 ncd sum_{ab} prod_t (i_t+j_t+1);
//   per contracted quartet: K 8 nab ncd, J 4 nab ncd.
static double sum_terms(int la, int lb) {
  double s = 0.0;
  for (int x = 0; x < ncart(la); ++x)
    for (int y = 0; y < ncart(lb); ++y) {
      int ix, iy, iz, jx, jy, jz;
      cart_xyz(la, x, ix, iy, iz);
      cart_xyz(lb, y, jx, jy, jz);
      s += (double)(ix + jx + 1) * (iy + jy + 1) * (iz + jz + 1);
    }
  return s;
}
static double class_flops(int X, int Y, double nq, double npq, double nbp, bool dj, bool dk) {
  const int la = kClassL1[X], lb = kClassL2[X], lc = kClassL1[Y], ld = kClassL2[Y];
  const int L = la + lb + lc + ld;
  double rf = 0.0;
  for (int m = 0; m < L; ++m) rf += 3.0 * (nherm(L - m) - 1);
  const double nab = ncart(la) * ncart(lb), ncd = ncart(lc) * ncart(ld);
  const double per_pq = 2.0 * (L + 1) + 20.0 + rf + 2.0 * nherm(la + lb) * sum_terms(lc, ld);
  const double per_bp = 2.0 * ncd * sum_terms(la, lb);
  const double per_q = (dk ? 8.0 : 0.0) * nab * ncd + (dj ? 4.0 : 0.0) * nab * ncd;
  return npq * per_pq + nbp * per_bp + nq * per_q;
}

// J-engine (Eq. j_formula) per primitive quartet of an ordered (bra, ket) item:
// Boys 2(L+1)+20, R recursion, J_P += sum_Q R_{P+Q} D_Q: 2 nherm(lab) nherm(lcd).
static double jengine_flops(int X, int Y, double npq) {
  const int lab = kClassL1[X] + kClassL2[X], lcd = kClassL1[Y] + kClassL2[Y], L = lab + lcd;
  double rf = 0.0;
  for (int m = 0; m < L; ++m) rf += 3.0 * (nherm(L - m) - 1);
  return npq * (2.0 * (L + 1) + 20.0 + rf + 2.0 * nherm(lab) * nherm(lcd));
}

// Gradient (bra derivatives, SI Eq. si_dE_J / si_dE_K) per ordered item:
//   per primitive quartet: Boys 2(L+2)+20, R recursion to L+1, ket transform
//     2 nherm(lab+1) sum_{cd} prod_t (k_t+l_t+1);
//   per bra primitive: for every (ab, cd), direction t opened to n_t+1 (raised
//     Hermite index) and the other two closed: 2 sum_t (n_t+2) prod_{u!=t} (n_u+1)
//     plus 4 (n_t+2) for the A and B coefficients;
//   per item: the density factor, 8 FLOPs per (ab, cd).
static double grad_flops(int X, int Y, double nq, double npq, double nbp) {
  const int la = kClassL1[X], lb = kClassL2[X], lc = kClassL1[Y], ld = kClassL2[Y];
  const int L1 = la + lb + lc + ld + 1;
  double rf = 0.0;
  for (int m = 0; m < L1; ++m) rf += 3.0 * (nherm(L1 - m) - 1);
  double dab = 0.0;
  for (int x = 0; x < ncart(la); ++x)
    for (int y = 0; y < ncart(lb); ++y) {
      int ix, iy, iz, jx, jy, jz;
      cart_xyz(la, x, ix, iy, iz);
      cart_xyz(lb, y, jx, jy, jz);
      const int n[3] = {ix + jx, iy + jy, iz + jz};
      for (int t = 0; t < 3; ++t)
        dab += 2.0 * (n[t] + 2) * (n[(t + 1) % 3] + 1) * (n[(t + 2) % 3] + 1) + 4.0 * (n[t] + 2);
    }
  const double nab = ncart(la) * ncart(lb), ncd = ncart(lc) * ncart(ld);
  const double per_pq = 2.0 * (L1 + 1) + 20.0 + rf + 2.0 * nherm(la + lb + 1) * sum_terms(lc, ld);
  return npq * per_pq + nbp * ncd * dab + nq * 8.0 * nab * ncd;
}

// Default work-tile length: the thread kernel's lanes already take adjacent
// items; a warp kernel takes 4 consecutive quartets (mostly one bra) per tile.
static int default_tile(int X, int Y, int tier) {
  return use_thread_kernel(kClassL1[X], kClassL2[X], kClassL1[Y], kClassL2[Y], tier == 1) ? 1 : 4;
}

int eri_plan_impl::tile_for(int X, int Y, int tier) const {
  const int t = tile_k[(X * NPAIRCLASS + Y) * 2 + tier];
  return t > 0 ? t : default_tile(X, Y, tier);
}

static cudaError_t launch_jk_class(int X, int Y, int prec, const JKArgs& ja, cudaStream_t s, int nsm) {
#define ERI_JK_UNIT_CALL(UX, UP, YLO, YHI) \
  if (X == UX && prec == UP && Y >= YLO && Y <= YHI) return launch_jk_unit<UX, UP, YLO, YHI>(Y, ja, s, nsm);
  ERI_JK_UNITS(ERI_JK_UNIT_CALL)
#undef ERI_JK_UNIT_CALL
  return cudaErrorInvalidValue;
}

extern "C" int eri_default_opts(eri_opts_t* o) {
  if (!o) return ERI_EINVAL;
  o->thresh = 1e-12;
  o->precision = ERI_FP64;
  o->mixed_tau = 1e-5;
  o->device = -1;
  o->j_engine = 1;
  o->profile = 0;
  o->tune_cache = nullptr;
  o->deterministic = 0;
  o->density_screen = 0;
  return ERI_OK;
}

// Tile cache file (opts.tune_cache): one line per entry,
//   <key> t_0 ... t_199      key = <device name>|nbf=<n>|nmol=<m>|npair=<p>|prec=<0|1>
// with spaces in the device name replaced by '_', the tiles in eri_get_tiles order.
static std::string tune_key(const eri_plan_impl* P, int precision) {
  cudaDeviceProp prop;
  std::string name = cudaGetDeviceProperties(&prop, P->device) == cudaSuccess ? prop.name : "unknown";
  for (char& c : name)
    if (c == ' ') c = '_';
  char buf[160];
  snprintf(buf, sizeof(buf), "|nbf=%d|nmol=%d|npair=%d|prec=%d", P->nbf, P->nmol, P->npair, precision);
  return name + buf;
}

static std::vector<std::string> read_lines(const std::string& path) {
  std::vector<std::string> out;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return out;
  std::string cur;
  int ch;
  while ((ch = fgetc(f)) != EOF) {
    if (ch == '\n') {
      if (!cur.empty()) out.push_back(cur);
      cur.clear();
    } else {
      cur.push_back((char)ch);
    }
  }
  if (!cur.empty()) out.push_back(cur);
  fclose(f);
  return out;
}

// Load the entry for (this plan, precision) into tile_k; a missing file or
// entry leaves the tiles unchanged.  Malformed entries are ignored.
static void tune_cache_load(eri_plan_impl* P, int precision) {
  if (P->tune_cache.empty()) return;
  const std::string key = tune_key(P, precision) + " ";
  for (const std::string& ln : read_lines(P->tune_cache)) {
    if (ln.compare(0, key.size(), key) != 0) continue;
    int t[NPAIRCLASS * NPAIRCLASS * 2];
    const char* c = ln.c_str() + key.size();
    int k = 0;
    for (; k < NPAIRCLASS * NPAIRCLASS * 2; ++k) {
      char* e = nullptr;
      const long v = strtol(c, &e, 10);
      if (e == c || v < 0 || v > 1024) break;
      t[k] = (int)v;
      c = e;
    }
    if (k == NPAIRCLASS * NPAIRCLASS * 2) memcpy(P->tile_k, t, sizeof(t));
  }
}

// Store tile_k as the entry for (this plan, precision), replacing an older one
// (write to a temporary file, then rename).  Returns ERI_EINVAL if the file
// cannot be written.
static int tune_cache_store(const eri_plan_impl* P, int precision) {
  if (P->tune_cache.empty()) return ERI_OK;
  const std::string key = tune_key(P, precision);
  std::vector<std::string> lines;
  for (const std::string& ln : read_lines(P->tune_cache))
    if (ln.compare(0, key.size() + 1, key + " ") != 0) lines.push_back(ln);
  std::string mine = key;
  for (int X = 0; X < NPAIRCLASS; ++X)
    for (int Y = 0; Y < NPAIRCLASS; ++Y)
      for (int t = 0; t < 2; ++t) mine += " " + std::to_string(Y <= X ? P->tile_for(X, Y, t) : 0);
  lines.push_back(mine);
  const std::string tmp = P->tune_cache + ".tmp" + std::to_string((long long)(uintptr_t)P);
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return ERI_EINVAL;
  for (const std::string& ln : lines) fprintf(f, "%s\n", ln.c_str());
  const bool ok = fclose(f) == 0;
  if (!ok || rename(tmp.c_str(), P->tune_cache.c_str()) != 0) {
    remove(tmp.c_str());
    return ERI_EINVAL;
  }
  return ERI_OK;
}

static int check_basis(const eri_basis_t* basis, const double* coords, int* nprim_out) {
  if (!basis || !coords || !basis->shells || !basis->exps || !basis->coefs) return ERI_EINVAL;
  const int ns = basis->nshell, na = basis->natom;
  if (ns <= 0 || na <= 0 || ns > 100000) return ERI_EINVAL;
  int nprim_tot = 0;
  for (int s = 0; s < ns; ++s) {
    const eri_shell_t& sh = basis->shells[s];
    if (sh.l < 0 || sh.l > LMAX || sh.nprim <= 0 || sh.nprim > 64 || sh.atom < 0 || sh.atom >= na ||
        sh.prim_offset < 0)
      return sh.l > LMAX ? ERI_EUNSUPPORTED : ERI_EINVAL;
    nprim_tot = std::max(nprim_tot, sh.prim_offset + sh.nprim);
  }
  for (int i = 0; i < nprim_tot; ++i)
    if (!(basis->exps[i] > 0.0) || !std::isfinite(basis->exps[i]) || !std::isfinite(basis->coefs[i])) return ERI_EINVAL;
  for (int i = 0; i < 3 * na; ++i)
    if (!std::isfinite(coords[i])) return ERI_EINVAL;
  *nprim_out = nprim_tot;
  return ERI_OK;
}

template <typename T>
static cudaError_t upload(T* d, const std::vector<T>& h) {
  return cudaMemcpy(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
}

// One plan over nmol independent molecules.  Shells, atoms and primitives are
// numbered globally (molecule after molecule); shell pairs are formed inside
// each molecule only, pair index pairbase[m] + a(a+1)/2 + b for local shells a >= b.
static int plan_create(int nmol, const eri_basis_t* const* bases, const double* const* coords, const eri_opts_t* opts,
                       eri_plan_t** out) {
  if (!out || nmol <= 0 || nmol > 65535 || !bases || !coords) return ERI_EINVAL;
  *out = nullptr;
  std::vector<int> nprim_m(nmol);
  for (int m = 0; m < nmol; ++m) {
    const int rc = check_basis(bases[m], coords[m], &nprim_m[m]);
    if (rc != ERI_OK) return rc;
  }
  eri_opts_t o;
  eri_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.thresh >= 0.0) || !(o.mixed_tau >= 0.0) || (o.precision != ERI_FP64 && o.precision != ERI_MIXED))
    return ERI_EINVAL;

  eri_plan_impl* P = new (std::nothrow) eri_plan_impl();
  if (!P) return ERI_ENOMEM;
  P->opts = o;
  if (o.tune_cache) P->tune_cache = o.tune_cache;
  P->opts.tune_cache = nullptr;  // the caller's string is not kept
  if (o.device >= 0) {
    if (cudaSetDevice(o.device) != cudaSuccess) { delete P; return ERI_ECUDA; }
  }
  cudaGetDevice(&P->device);
  cudaDeviceGetAttribute(&P->nsm, cudaDevAttrMultiProcessorCount, P->device);
  P->nmol = nmol;
  // global numbering
  std::vector<int> l, atom, np, po, ao, aol, shloc;
  std::vector<double> ex, co, xyz;
  P->h_mat_off.assign(nmol + 1, 0);
  P->h_mat_n.assign(nmol, 0);
  P->h_aobase.assign(nmol + 1, 0);
  P->h_atombase.assign(nmol + 1, 0);
  P->h_pairbase.assign(nmol + 1, 0);
  std::vector<int> shellbase(nmol + 1, 0);
  int nbf = 0, nprim_tot = 0;
  int64_t npair64 = 0;
  for (int m = 0; m < nmol; ++m) {
    const eri_basis_t* B = bases[m];
    shellbase[m] = (int)l.size();
    P->h_atombase[m] = (int)(xyz.size() / 3);
    P->h_aobase[m] = nbf;
    P->h_pairbase[m] = (int)npair64;
    int nb = 0;
    for (int s = 0; s < B->nshell; ++s) {
      const eri_shell_t& sh = B->shells[s];
      l.push_back(sh.l);
      atom.push_back(P->h_atombase[m] + sh.atom);
      np.push_back(sh.nprim);
      po.push_back(nprim_tot + sh.prim_offset);
      ao.push_back(nbf + nb);
      aol.push_back(nb);
      shloc.push_back(s);
      nb += ncart(sh.l);
    }
    ex.insert(ex.end(), B->exps, B->exps + nprim_m[m]);
    co.insert(co.end(), B->coefs, B->coefs + nprim_m[m]);
    xyz.insert(xyz.end(), coords[m], coords[m] + 3 * B->natom);
    nprim_tot += nprim_m[m];
    nbf += nb;
    P->h_mat_n[m] = nb;
    P->h_mat_off[m + 1] = P->h_mat_off[m] + (int64_t)nb * nb;
    P->max_nbf = std::max(P->max_nbf, nb);
    npair64 += (int64_t)B->nshell * (B->nshell + 1) / 2;
  }
  const int ns = (int)l.size(), na = (int)(xyz.size() / 3);
  shellbase[nmol] = ns;
  P->h_atombase[nmol] = na;
  P->h_aobase[nmol] = nbf;
  P->h_pairbase[nmol] = (int)std::min<int64_t>(npair64, INT32_MAX);
  ao.push_back(nbf);
  if (npair64 > (1LL << 28)) { delete P; return ERI_EUNSUPPORTED; }
  P->nshell = ns;
  P->natom = na;
  P->nbf = nbf;
  P->nmat = P->h_mat_off[nmol];
  // shell pairs, molecule by molecule in pair-index order (a >= b), oriented so that s1 has the higher l
  const int npair = (int)npair64;
  P->npair = npair;
  std::vector<int> ps1(npair), ps2(npair), pnp(npair), ppoff(npair), pao1(npair), pao2(npair), phoff(npair), pcls(npair),
      peoff(npair), pmol(npair);
  int64_t nprimpair = 0, nherm_tot = 0, ne_tot = 0;
  for (int m = 0; m < nmol; ++m) {
    const int sb = shellbase[m], nsm = shellbase[m + 1] - sb;
    for (int a = 0; a < nsm; ++a)
      for (int b = 0; b <= a; ++b) {
        const int ip = P->h_pairbase[m] + a * (a + 1) / 2 + b;
        int x = sb + a, y = sb + b;
        if (l[y] > l[x]) std::swap(x, y);
        ps1[ip] = x; ps2[ip] = y;
        pnp[ip] = np[x] * np[y];
        ppoff[ip] = (int)std::min<int64_t>(nprimpair, INT32_MAX);
        pao1[ip] = aol[x]; pao2[ip] = aol[y];
        phoff[ip] = (int)std::min<int64_t>(nherm_tot, INT32_MAX);
        pcls[ip] = pair_class(l[x], l[y]);
        peoff[ip] = (int)std::min<int64_t>(ne_tot, INT32_MAX);
        pmol[ip] = m;
        nprimpair += pnp[ip];
        nherm_tot += (int64_t)pnp[ip] * nherm(l[x] + l[y]);
        ne_tot += (int64_t)pnp[ip] * 3 * (l[x] + 1) * (l[y] + 1) * (l[x] + l[y] + 1);
      }
  }
  if (nprimpair > (1LL << 30) || nherm_tot > (1LL << 31) - 1 || ne_tot > (1LL << 31) - 1) {
    delete P;
    return ERI_EUNSUPPORTED;
  }
  P->nprimpair = (int)nprimpair;
  P->nherm_tot = nherm_tot;
  int rc = ERI_OK;
#define CKP(x)                                   \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_ != cudaSuccess) { rc = eri_fail(e_); goto fail; } \
  } while (0)
  {
    cudaStream_t s = 0;
    std::vector<RStep> st = make_rsteps();
    const size_t nm10 = (size_t)nmol * NPAIRCLASS;
    CKP(dalloc(&P->d_sh_l, ns)); CKP(dalloc(&P->d_sh_atom, ns)); CKP(dalloc(&P->d_sh_np, ns));
    CKP(dalloc(&P->d_sh_po, ns)); CKP(dalloc(&P->d_sh_ao, ns + 1)); CKP(dalloc(&P->d_shloc, ns));
    CKP(dalloc(&P->d_exps, nprim_tot)); CKP(dalloc(&P->d_coefs, nprim_tot)); CKP(dalloc(&P->d_cn, nprim_tot));
    CKP(dalloc(&P->d_f, nbf)); CKP(dalloc(&P->d_coords, 3 * (size_t)na));
    CKP(dalloc(&P->d_mat_off, nmol + 1)); CKP(dalloc(&P->d_mat_n, nmol)); CKP(dalloc(&P->d_aobase, nmol + 1));
    CKP(dalloc(&P->d_pbase, nmol + 1)); CKP(dalloc(&P->d_ccm, nm10)); CKP(dalloc(&P->d_segloc, nm10));
    CKP(dalloc(&P->d_ps1, npair)); CKP(dalloc(&P->d_ps2, npair)); CKP(dalloc(&P->d_pnp, npair));
    CKP(dalloc(&P->d_ppoff, npair)); CKP(dalloc(&P->d_pao1, npair)); CKP(dalloc(&P->d_pao2, npair));
    CKP(dalloc(&P->d_phoff, npair)); CKP(dalloc(&P->d_pcls, npair)); CKP(dalloc(&P->d_pmol, npair));
    CKP(dalloc(&P->d_Q, npair)); CKP(dalloc(&P->d_qmax, nmol)); CKP(dalloc(&P->d_sig, npair));
    CKP(dalloc(&P->d_ccount, NPAIRCLASS)); CKP(dalloc(&P->d_coff, NPAIRCLASS)); CKP(dalloc(&P->d_sorted, npair));
    CKP(dalloc(&P->d_pos, npair)); CKP(dalloc(&P->d_counts, (size_t)npair * NPAIRCLASS));
    CKP(dalloc(&P->d_cumnp, (size_t)npair + NPAIRCLASS));
    CKP(dalloc(&P->d_koff, NPAIRCLASS * NPAIRCLASS)); CKP(dalloc(&P->d_joff, NPAIRCLASS * NPAIRCLASS));
    CKP(dalloc(&P->d_ktot, NPAIRCLASS * NPAIRCLASS)); CKP(dalloc(&P->d_jtot, NPAIRCLASS * NPAIRCLASS));
    CKP(dalloc(&P->d_kprim, NPAIRCLASS * NPAIRCLASS));
    CKP(dalloc(&P->d_boys64, (size_t)BOYS_NT * (BOYS_MMAX + 1) * BOYS_J64));
    CKP(dalloc(&P->d_boys32, (size_t)BOYS_NT * (BOYS_MMAX + 1) * BOYS_J32));
    CKP(dalloc(&P->d_bexp64, BOYS_NT)); CKP(dalloc(&P->d_bexp32, BOYS_NT));
    CKP(dalloc(&P->d_peoff, npair)); CKP(dalloc(&P->d_E, ne_tot)); CKP(dalloc(&P->d_Ef, ne_tot));
    CKP(dalloc(&P->d_pmaxp, npair)); CKP(dalloc(&P->d_prefmaxp, npair)); CKP(dalloc(&P->d_ea, nprimpair));
    CKP(dalloc(&P->d_dmax, npair));
    CKP(dalloc(&P->d_counters, NPAIRCLASS * NPAIRCLASS * 2 * 3 + 2));  // + range-guard and screened counts
    CKP(dalloc(&P->d_counters2, 4 * NPAIRCLASS * NPAIRCLASS * 3));
    CKP(cudaMemset(P->d_counters2, 0, sizeof(unsigned long long) * 4 * NPAIRCLASS * NPAIRCLASS * 3));
    CKP(dalloc(&P->d_rsteps, st.size()));
    CKP(dalloc(&P->d_Dp, (size_t)P->nmat)); CKP(dalloc(&P->d_Dpf, (size_t)P->nmat));
    CKP(dalloc(&P->d_Kh, (size_t)P->nmat));
    CKP(dalloc(&P->d_Jh, (size_t)P->nmat));
    CKP(dalloc(&P->d_Dherm, nherm_tot)); CKP(dalloc(&P->d_Jherm, nherm_tot)); CKP(dalloc(&P->d_Dhermf, nherm_tot));
    CKP(dalloc(&P->d_status, 1));
    if (P->alloc_pairs() != ERI_OK) { rc = ERI_ENOMEM; goto fail; }
    CKP(upload(P->d_sh_l, l)); CKP(upload(P->d_sh_atom, atom)); CKP(upload(P->d_sh_np, np));
    CKP(upload(P->d_sh_po, po)); CKP(upload(P->d_sh_ao, ao)); CKP(upload(P->d_shloc, shloc));
    CKP(upload(P->d_exps, ex)); CKP(upload(P->d_coefs, co)); CKP(upload(P->d_coords, xyz));
    CKP(upload(P->d_mat_off, P->h_mat_off)); CKP(upload(P->d_mat_n, P->h_mat_n));
    CKP(upload(P->d_aobase, P->h_aobase)); CKP(upload(P->d_pbase, P->h_pairbase));
    CKP(upload(P->d_ps1, ps1)); CKP(upload(P->d_ps2, ps2)); CKP(upload(P->d_pnp, pnp));
    CKP(upload(P->d_ppoff, ppoff)); CKP(upload(P->d_pao1, pao1)); CKP(upload(P->d_pao2, pao2));
    CKP(upload(P->d_phoff, phoff)); CKP(upload(P->d_peoff, peoff)); CKP(upload(P->d_pcls, pcls));
    CKP(upload(P->d_pmol, pmol)); CKP(upload(P->d_rsteps, st));
    CKP(cudaMemset(P->d_status, 0, sizeof(int)));
    k_normalize<<<grid1(ns, 64), 64>>>(ns, P->d_sh_l, P->d_sh_np, P->d_sh_po, P->d_exps, P->d_coefs, P->d_cn);
    k_compfac<<<grid1(ns, 64), 64>>>(ns, P->d_sh_l, P->d_sh_ao, P->d_f);
    k_boys_table<<<grid1(BOYS_NT, 128), 128>>>(P->d_boys64, P->d_bexp64, P->d_boys32, P->d_bexp32);
    CKP(cudaGetLastError());
    P->thresh = o.thresh;
    rc = P->geometry(s, true);
    if (rc != ERI_OK) goto fail;
    CKP(cudaDeviceSynchronize());
  }
#undef CKP
  tune_cache_load(P, o.precision);
  *out = reinterpret_cast<eri_plan_t*>(P);
  return ERI_OK;
fail:
  P->release();
  delete P;
  return rc;
}

extern "C" int eri_plan(const eri_basis_t* basis, const double* coords, const eri_opts_t* opts, eri_plan_t** out) {
  if (!basis || !coords || !out) return ERI_EINVAL;
  return plan_create(1, &basis, &coords, opts, out);
}

extern "C" int eri_plan_batch(int32_t nmol, const eri_basis_t* const* bases, const double* const* coords,
                              const eri_opts_t* opts, eri_plan_t** out) {
  return plan_create(nmol, bases, coords, opts, out);
}

extern "C" int eri_plan_layout(eri_plan_t* plan, int32_t* nmol, int64_t* mat_off, int32_t* nbf, int32_t* atom_off) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P) return ERI_EINVAL;
  if (nmol) *nmol = P->nmol;
  for (int m = 0; m <= P->nmol; ++m) {
    if (mat_off) mat_off[m] = P->h_mat_off[m];
    if (atom_off) atom_off[m] = P->h_atombase[m];
    if (nbf && m < P->nmol) nbf[m] = P->h_mat_n[m];
  }
  return ERI_OK;
}

extern "C" int eri_plan_set_coords(eri_plan_t* plan, const double* coords_dev, int32_t freeze_lists, void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || !coords_dev) return ERI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(P->device));
  CK(cudaMemcpyAsync(P->d_coords, coords_dev, sizeof(double) * 3 * P->natom, cudaMemcpyDeviceToDevice, s));
  ++P->geom_serial;  // an exchange-correlation grid follows the atoms at its next use
  return P->geometry(s, freeze_lists == 0);
}

// One J/K build on stream s, lists as they stand.  With `concurrent` the class
// launches are spread over the plan's side streams (fork / join by events) in
// decreasing order of estimated work; otherwise they run in order on s.
static int build_impl(eri_plan_impl* P, const double* D, double* J, double* K, int precision, cudaStream_t s,
                      int nbranch) {
  // nbranch = 0: eager build on s (profiling allowed); >= 1: graph capture,
  // class launches forked onto nbranch branch streams (least-loaded first)
  const bool concurrent = nbranch > 0;
  const int64_t nn = P->nmat;
  const MolMats mm = molmats(P);
  k_scale_d<<<P->mat_grid(256), 256, 0, s>>>(mm, D, P->d_f, P->d_Dp, P->d_Dpf);
  CK(cudaGetLastError());
  const bool jengine = J && !K && P->opts.j_engine;
  if (jengine) {
    // J alone: Hermite density -> J-engine -> Hermite J to Cartesian (Eq. j_formula).
    // Mixed precision: each ordered list is split on the device by the energy's
    // tier test (reading 5) and each tier's kernel runs its own compacted list;
    // both add into the FP64 Hermite J.
    const bool jmixed = precision == ERI_MIXED;
    CK(cudaMemsetAsync(P->d_Jherm, 0, sizeof(double) * (size_t)P->nherm_tot, s));
    k_hermite_density<<<grid1(P->npair, 64), 64, 0, s>>>(P->npair, P->d_ps1, P->d_ps2, P->d_pnp, P->d_ppoff,
                                                          P->d_phoff, P->d_sh_l, P->d_pao1, P->d_pao2, P->d_pmol, mm,
                                                          P->d_sig, P->pairdata(), P->d_Dp, P->d_Dherm,
                                                          jmixed ? P->d_Dhermf : nullptr);
    CK(cudaGetLastError());
    if (jmixed) {
      k_dmax<<<grid1(P->npair, 128), 128, 0, s>>>(P->npair, P->d_ps1, P->d_ps2, P->d_sh_l, P->d_pao1, P->d_pao2,
                                                  P->d_pmol, P->d_mat_off, P->d_mat_n, P->d_Dp, P->d_dmax);
      CK(cudaGetLastError());
      if (!concurrent) {
        const int rc = P->ensure_tier_bufs(1);
        if (rc != ERI_OK) return rc;
      }
      if (P->tier_nb < (concurrent ? nbranch : 1)) return ERI_EINVAL;
    }
    JArgs ja{};
    ja.pd = P->pairdata(); ja.sp = P->spinfo(); ja.bt = P->boystabs();
    ja.rsteps = P->d_rsteps; ja.Dherm = P->d_Dherm; ja.Dhermf = P->d_Dhermf; ja.Jherm = P->d_Jherm;
    ja.omega2 = P->omega * P->omega; ja.omega2f = (float)ja.omega2;
    ja.det = P->opts.deterministic ? 1 : 0;
    ja.items = nullptr;
    ja.nitems = nullptr;
    KArgs ka{};  // tier split of the ordered lists
    ka.pd = P->pairdata(); ka.sp = P->spinfo();
    ka.Q = P->d_Q; ka.dmax = P->d_dmax; ka.pmaxp = P->d_pmaxp; ka.prefmaxp = P->d_prefmaxp;
    ka.shloc = P->d_shloc; ka.pbase = P->d_pbase;
    ka.tau = (float)P->opts.mixed_tau; ka.pmax32 = (float)kPmax32; ka.mixed = 1;
    if (concurrent) {
      CK(cudaEventRecord(P->fork_ev, s));
      for (int b = 0; b < nbranch; ++b) CK(cudaStreamWaitEvent(P->branch[b], P->fork_ev, 0));
    }
    // counters2 kinds 0 (J-engine FP64) and 3 (J-engine FP32)
    CK(cudaMemsetAsync(P->d_counters2, 0, sizeof(unsigned long long) * NPAIRCLASS * NPAIRCLASS * 3, s));
    CK(cudaMemsetAsync(P->d_counters2 + 3 * NPAIRCLASS * NPAIRCLASS * 3, 0,
                       sizeof(unsigned long long) * NPAIRCLASS * NPAIRCLASS * 3, s));
    P->last_jmixed = jmixed;
    const bool prof = P->opts.profile && !concurrent;
    int nl = 0;
    auto jlaunch = [&](int X, int Y, int tier, cudaStream_t ls) -> int {
      const int lab = kClassL1[X] + kClassL2[X], lcd = kClassL1[Y] + kClassL2[Y];
      ja.counter = P->d_counters2 + ((tier ? 3 : 0) * NPAIRCLASS * NPAIRCLASS + X * NPAIRCLASS + Y) * 3;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (prof) {
        CK(P->prof_event_pair(&e0, &e1));
        CK(cudaEventRecord(e0, ls));
      }
      cudaError_t e = cudaErrorInvalidValue;
      switch (lab) {
        case 0: e = launch_j_lab0(lcd, tier, ja, ls, P->nsm); break;
        case 1: e = launch_j_lab1(lcd, tier, ja, ls, P->nsm); break;
        case 2: e = launch_j_lab2(lcd, tier, ja, ls, P->nsm); break;
        case 3: e = launch_j_lab3(lcd, tier, ja, ls, P->nsm); break;
        case 4: e = launch_j_lab4(lcd, tier, ja, ls, P->nsm); break;
        case 5: e = launch_j_lab5(lcd, tier, ja, ls, P->nsm); break;
        case 6: e = launch_j_lab6(lcd, tier, ja, ls, P->nsm); break;
      }
      CK(e);
      if (prof) {
        CK(cudaEventRecord(e1, ls));
        P->prof_log.push_back({X, Y, tier ? 5 : 3, P->prof_ev_used - 2});
      }
      return ERI_OK;
    };
    for (int X = 0; X < NPAIRCLASS; ++X)
      for (int Y = 0; Y < NPAIRCLASS; ++Y) {
        const WorkList full = P->jlist(X, Y);
        if (full.total == 0) continue;
        const int b = concurrent ? nl++ % nbranch : 0;
        const cudaStream_t ls = concurrent ? P->branch[b] : s;
        if (!jmixed) {
          ja.wl = full;
          const int rc = jlaunch(X, Y, 0, ls);
          if (rc != ERI_OK) return rc;
          continue;
        }
        int2* buf = P->tbuf[b];
        unsigned int* cnt = P->tcnt + 2 * b;
        for (int64_t f = 0; f < full.total; f += P->tier_cap) {
          KArgs sa = ka;
          sa.wl = full;
          sa.wl.first = f;
          sa.wl.total = std::min<int64_t>(full.total, f + P->tier_cap);
          CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned int), ls));
          const int64_t nch = (sa.wl.total - f + 31) / 32;
          k_tier_split<<<(int)std::max<int64_t>(1, std::min<int64_t>((nch + 7) / 8, (int64_t)P->nsm * 8)), 256, 0,
                         ls>>>(sa, buf, buf + P->tier_cap, cnt);
          CK(cudaGetLastError());
          for (int tier = 0; tier < 2; ++tier) {
            ja.wl = full;
            ja.wl.first = 0;
            ja.wl.total = sa.wl.total - f;  // upper bound of the tier's count (grid sizing)
            ja.items = buf + (tier ? P->tier_cap : 0);
            ja.nitems = cnt + tier;
            const int rc = jlaunch(X, Y, tier, ls);
            if (rc != ERI_OK) return rc;
          }
        }
        ja.items = nullptr;
        ja.nitems = nullptr;
      }
    if (concurrent)
      for (int b = 0; b < nbranch; ++b) {
        CK(cudaEventRecord(P->join_ev[b], P->branch[b]));
        CK(cudaStreamWaitEvent(s, P->join_ev[b], 0));
      }
    CK(cudaMemsetAsync(J, 0, sizeof(double) * nn, s));
    k_post_j<<<grid1((int64_t)P->npair * 100, 128), 128, 0, s>>>(P->npair, P->d_ps1, P->d_ps2, P->d_pnp, P->d_ppoff,
                                                                 P->d_phoff, P->d_sh_l, P->d_pao1, P->d_pao2,
                                                                 P->d_pmol, mm, P->d_sig, P->pairdata(), P->d_Jherm,
                                                                 P->d_f, J, ja.det, P->d_status);
    CK(cudaGetLastError());
  } else {
    // J and/or K from contracted Cartesian ERIs over canonical quartets
    if (K) CK(cudaMemsetAsync(P->d_Kh, 0, sizeof(double) * nn, s));
    if (J) CK(cudaMemsetAsync(P->d_Jh, 0, sizeof(double) * nn, s));
    CK(cudaMemsetAsync(P->d_counters, 0, sizeof(unsigned long long) * (NPAIRCLASS * NPAIRCLASS * 6 + 2), s));
    const bool mixed = precision == ERI_MIXED;
    // the device split pass serves the precision tiers and the density screen
    const bool split = mixed || P->opts.density_screen;
    if (split) {
      k_dmax<<<grid1(P->npair, 128), 128, 0, s>>>(P->npair, P->d_ps1, P->d_ps2, P->d_sh_l, P->d_pao1, P->d_pao2,
                                                  P->d_pmol, P->d_mat_off, P->d_mat_n, P->d_Dp, P->d_dmax);
      CK(cudaGetLastError());
    }
    JKArgs ja{};
    KArgs& ka = ja.k;
    ka.pd = P->pairdata(); ka.sp = P->spinfo(); ka.bt = P->boystabs();
    ka.rsteps = P->d_rsteps; ka.Dp = P->d_Dp; ka.Dpf = P->d_Dpf; ka.Kh = K ? P->d_Kh : nullptr;
    ka.Q = P->d_Q; ka.dmax = P->d_dmax; ka.pmaxp = P->d_pmaxp; ka.prefmaxp = P->d_prefmaxp;
    ka.shloc = P->d_shloc; ka.pbase = P->d_pbase;
    ka.tau = mixed ? (float)P->opts.mixed_tau : 0.0f; ka.pmax32 = (float)kPmax32; ka.mixed = mixed ? 1 : 0;
    ka.items = nullptr; ka.nitems = nullptr;
    ka.guard = P->d_counters + NPAIRCLASS * NPAIRCLASS * 6;
    ka.screened = P->d_counters + NPAIRCLASS * NPAIRCLASS * 6 + 1;
    ka.screen = P->opts.density_screen ? (float)P->thresh : 0.0f;
    ka.omega2 = P->omega * P->omega; ka.omega2f = (float)ka.omega2;
    ka.det = P->opts.deterministic ? 1 : 0;
    ja.Jh = J ? P->d_Jh : nullptr;
    P->last_mixed = mixed;
    P->last_do_j = J != nullptr;
    P->last_do_k = K != nullptr;
    // class pairs in decreasing order of estimated work (primitive quartets x class cost)
    struct L { int X, Y; double cost; };
    std::vector<L> order;
    for (int X = 0; X < NPAIRCLASS; ++X)
      for (int Y = 0; Y <= X; ++Y) {
        const int64_t tot = P->h_ktot[X * NPAIRCLASS + Y];
        if (tot == 0) continue;
        order.push_back({X, Y, class_flops(X, Y, (double)tot, (double)P->h_kprim[X * NPAIRCLASS + Y], 0.0,
                                           J != nullptr, K != nullptr)});
      }
    if (split && !concurrent) {
      const int rc = P->ensure_tier_bufs(1);
      if (rc != ERI_OK) return rc;
    }
    if (split && P->tier_nb < (concurrent ? nbranch : 1)) return ERI_EINVAL;
    if (concurrent) {
      std::stable_sort(order.begin(), order.end(), [](const L& a, const L& b) { return a.cost > b.cost; });
      CK(cudaEventRecord(P->fork_ev, s));
      for (int b = 0; b < nbranch; ++b) CK(cudaStreamWaitEvent(P->branch[b], P->fork_ev, 0));
    }
    const bool prof = P->opts.profile && !concurrent;
    auto launch = [&](int X, int Y, int tier, cudaStream_t ls) -> int {
      ka.tier_want = tier;
      ka.wl.tile = P->tile_for(X, Y, tier);
      ka.counter = P->d_counters + ((X * NPAIRCLASS + Y) * 2 + tier) * 3;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (prof) {
        CK(P->prof_event_pair(&e0, &e1));
        CK(cudaEventRecord(e0, ls));
      }
      CK(launch_jk_class(X, Y, tier, ja, ls, P->nsm));
      if (prof) {
        CK(cudaEventRecord(e1, ls));
        P->prof_log.push_back({X, Y, tier, P->prof_ev_used - 2});
      }
      return ERI_OK;
    };
    double load[eri_plan_impl::kBranches] = {};
    for (const L& l : order) {
      cudaStream_t ls = s;
      int b = 0;
      if (concurrent) {  // least-loaded branch
        b = (int)(std::min_element(load, load + nbranch) - load);
        load[b] += l.cost;
        ls = P->branch[b];
      }
      ka.same_class = l.X == l.Y;
      if (!split) {
        ka.wl = P->klist(l.X, l.Y);
        ka.items = nullptr;
        ka.nitems = nullptr;
        const int rc = launch(l.X, l.Y, 0, ls);
        if (rc != ERI_OK) return rc;
        continue;
      }
      // mixed precision and/or density screen: split each window of the list
      // into its two tiers, dropping screened quartets (compacted on the
      // device), then run each tier over its own list (FP64 builds: tier 0 only)
      const WorkList full = P->klist(l.X, l.Y);
      int2* buf = P->tbuf[b];
      unsigned int* cnt = P->tcnt + 2 * b;
      for (int64_t f = 0; f < full.total; f += P->tier_cap) {
        KArgs sa = ka;
        sa.wl = full;
        sa.wl.first = f;
        sa.wl.total = std::min<int64_t>(full.total, f + P->tier_cap);
        CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned int), ls));
        const int64_t nch = (sa.wl.total - f + 31) / 32;
        k_tier_split<<<(int)std::max<int64_t>(1, std::min<int64_t>((nch + 7) / 8, (int64_t)P->nsm * 8)), 256, 0,
                       ls>>>(sa, buf, buf + P->tier_cap, cnt);
        CK(cudaGetLastError());
        for (int tier = 0; tier < (mixed ? 2 : 1); ++tier) {
          ka.wl = full;
          ka.wl.first = 0;
          ka.wl.total = sa.wl.total - f;  // upper bound of the tier's count (grid sizing)
          ka.items = buf + (tier ? P->tier_cap : 0);
          ka.nitems = cnt + tier;
          const int rc = launch(l.X, l.Y, tier, ls);
          if (rc != ERI_OK) return rc;
        }
      }
      ka.items = nullptr;
      ka.nitems = nullptr;
    }
    if (concurrent)
      for (int b = 0; b < nbranch; ++b) {
        CK(cudaEventRecord(P->join_ev[b], P->branch[b]));
        CK(cudaStreamWaitEvent(s, P->join_ev[b], 0));
      }
    P->prof_builds += P->opts.profile ? 1 : 0;
    if (K) {
      k_post_k<<<P->mat_grid(256), 256, 0, s>>>(mm, P->d_Kh, P->d_f, K, ka.det, P->d_status);
      CK(cudaGetLastError());
    }
    if (J) {
      k_post_k<<<P->mat_grid(256), 256, 0, s>>>(mm, P->d_Jh, P->d_f, J, ka.det, P->d_status);
      CK(cudaGetLastError());
    }
  }
  return ERI_OK;
}

extern "C" int eri_build_jk(eri_plan_t* plan, const double* D, double* J, double* K, double thresh, int32_t precision,
                            void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || !D || (!J && !K)) return ERI_EINVAL;
  if (precision != ERI_FP64 && precision != ERI_MIXED) return ERI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(P->device));
  if (thresh >= 0.0 && thresh != P->thresh) {
    int rc = P->build_lists(thresh, s);
    if (rc != ERI_OK) return rc;
  }
  return build_impl(P, D, J, K, precision, s, 0);
}

extern "C" int eri_build_jk_graph(eri_plan_t* plan, const double* D, double* J, double* K, int32_t precision,
                                  void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || !D || (!J && !K)) return ERI_EINVAL;
  if (precision != ERI_FP64 && precision != ERI_MIXED) return ERI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(P->device));
  if (!P->gexec || P->gkey[0] != D || P->gkey[1] != J || P->gkey[2] != K || P->gprec != precision) {
    int rc = P->ensure_streams();
    if (rc != ERI_OK) return rc;
    if (precision == ERI_MIXED || P->opts.density_screen) {
      rc = P->ensure_tier_bufs(eri_plan_impl::kBranches);
      if (rc != ERI_OK) return rc;
    }
    if (P->gexec) {
      CK(cudaStreamSynchronize(s));
      CK(cudaGraphExecDestroy(P->gexec));
      P->gexec = nullptr;
    }
    // Capture the build twice: class launches in one serial chain, and forked
    // over kBranches branches (least-loaded first).  Long launches that fill
    // the GPU by themselves run best in order; many short ones (batched
    // plans, small molecules) gain from overlapping.  Each graph is replayed
    // twice on `stream` (CUDA events) and the faster one is kept.
    const int cand[2] = {1, eri_plan_impl::kBranches};
    cudaGraphExec_t ex[2] = {nullptr, nullptr};
    for (int c = 0; c < 2 && rc == ERI_OK; ++c) {
      CK(cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal));
      rc = build_impl(P, D, J, K, precision, P->cap_stream, cand[c]);
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(P->cap_stream, &g);
      if (rc == ERI_OK && ce != cudaSuccess) rc = eri_fail(ce);
      if (rc == ERI_OK) {
        const cudaError_t ie = cudaGraphInstantiate(&ex[c], g, 0);
        if (ie != cudaSuccess) {
          ex[c] = nullptr;
          rc = eri_fail(ie);
        }
      }
      if (g) cudaGraphDestroy(g);
    }
    float best[2] = {0.0f, 0.0f};
    if (rc == ERI_OK) {
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      cudaError_t te = cudaEventCreate(&e0);
      if (te == cudaSuccess) te = cudaEventCreate(&e1);
      for (int c = 0; c < 2 && te == cudaSuccess; ++c) {
        best[c] = 3.4e38f;
        for (int r = 0; r < 2 && te == cudaSuccess; ++r) {
          float ms = 0.0f;
          te = cudaEventRecord(e0, s);
          if (te == cudaSuccess) te = cudaGraphLaunch(ex[c], s);
          if (te == cudaSuccess) te = cudaEventRecord(e1, s);
          if (te == cudaSuccess) te = cudaEventSynchronize(e1);
          if (te == cudaSuccess) te = cudaEventElapsedTime(&ms, e0, e1);
          if (te == cudaSuccess && ms < best[c]) best[c] = ms;
        }
      }
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      if (te != cudaSuccess) rc = eri_fail(te);
    }
    const int keep = best[1] < best[0] ? 1 : 0;
    for (int c = 0; c < 2; ++c)
      if (ex[c] && (rc != ERI_OK || c != keep)) cudaGraphExecDestroy(ex[c]);
    if (rc != ERI_OK) {
      cudaGetLastError();
      return rc;
    }
    P->gexec = ex[keep];
    P->gbranches = cand[keep];
    P->gkey[0] = D;
    P->gkey[1] = J;
    P->gkey[2] = K;
    P->gprec = precision;
  }
  CK(cudaGraphLaunch(P->gexec, s));
  return ERI_OK;
}

// Autotuner: for every (bra class, ket class, tier) launch of this plan, time
// each candidate work-tile length on three windows of the launch's own work
// list (at 1/6, 1/2 and 5/6 of it, so that a mixed-precision tier sees its
// share of quartets) and keep the fastest.  A window is sized so that the
// default tile takes about trial_ms; each candidate is timed twice (minimum).
// The trials write into the plan's scratch accumulators only.
extern "C" int eri_autotune(eri_plan_t* plan, const double* D, int32_t precision, double trial_ms, void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || !D || !(trial_ms > 0.0)) return ERI_EINVAL;
  if (precision != ERI_FP64 && precision != ERI_MIXED) return ERI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(P->device));
  const bool mixed = precision == ERI_MIXED;
  const MolMats mm = molmats(P);
  k_scale_d<<<P->mat_grid(256), 256, 0, s>>>(mm, D, P->d_f, P->d_Dp, P->d_Dpf);
  if (mixed)
    k_dmax<<<grid1(P->npair, 128), 128, 0, s>>>(P->npair, P->d_ps1, P->d_ps2, P->d_sh_l, P->d_pao1, P->d_pao2,
                                                P->d_pmol, P->d_mat_off, P->d_mat_n, P->d_Dp, P->d_dmax);
  CK(cudaGetLastError());
  JKArgs ja{};
  KArgs& ka = ja.k;
  ka.pd = P->pairdata(); ka.sp = P->spinfo(); ka.bt = P->boystabs();
  ka.rsteps = P->d_rsteps; ka.Dp = P->d_Dp; ka.Dpf = P->d_Dpf; ka.Kh = P->d_Kh;
  ka.Q = P->d_Q; ka.dmax = P->d_dmax; ka.pmaxp = P->d_pmaxp; ka.prefmaxp = P->d_prefmaxp;
  ka.shloc = P->d_shloc; ka.pbase = P->d_pbase;
  ka.tau = (float)P->opts.mixed_tau; ka.pmax32 = (float)kPmax32; ka.mixed = mixed ? 1 : 0;
  ka.counter = nullptr;
  ka.guard = nullptr;
  ka.omega2 = P->omega * P->omega; ka.omega2f = (float)ka.omega2;
  ja.Jh = P->d_Jh;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = ERI_OK;
  if (mixed) {
    rc = P->ensure_tier_bufs(1);
    if (rc != ERI_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc;
    }
  }
  // time the three windows of `win` items each with tile t; returns ms (< 0 on
  // error).  Mixed precision: each window is first split into its tiers
  // (untimed) and the tier's compacted list is timed.
  auto trial = [&](int X, int Y, int tier, int t, int64_t win) -> double {
    const WorkList full = P->klist(X, Y);
    const int64_t tot = full.total;
    if (mixed) win = std::min<int64_t>(win, P->tier_cap);
    double best = 1e300;
    for (int rep = 0; rep < 2; ++rep) {
      double sum = 0.0;
      for (int w = 0; w < 3; ++w) {
        const int64_t c = tot * (2 * w + 1) / 6;
        const int64_t f = std::max<int64_t>(0, std::min<int64_t>(c - win / 2, tot - win));
        const int64_t last = std::min<int64_t>(tot, f + win);
        ka.wl = full;
        ka.wl.first = f;
        ka.wl.total = last;
        ka.wl.tile = t;
        ka.same_class = X == Y;
        ka.tier_want = tier;
        ka.items = nullptr;
        ka.nitems = nullptr;
        if (mixed) {
          if (cudaMemsetAsync(P->tcnt, 0, 2 * sizeof(unsigned int), s) != cudaSuccess) return -1.0;
          const int64_t nch = (last - f + 31) / 32;
          k_tier_split<<<(int)std::max<int64_t>(1, std::min<int64_t>((nch + 7) / 8, (int64_t)P->nsm * 8)), 256, 0,
                         s>>>(ka, P->tbuf[0], P->tbuf[0] + P->tier_cap, P->tcnt);
          ka.wl.first = 0;
          ka.wl.total = last - f;
          ka.items = P->tbuf[0] + (tier ? P->tier_cap : 0);
          ka.nitems = P->tcnt + tier;
        }
        if (cudaEventRecord(e0, s) != cudaSuccess) return -1.0;
        if (launch_jk_class(X, Y, tier, ja, s, P->nsm) != cudaSuccess) return -1.0;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0;
        sum += ms;
      }
      best = std::min(best, sum);
    }
    ka.items = nullptr;
    ka.nitems = nullptr;
    return best;
  };
  static const int kThreadTiles[] = {1, 2, 4, 8};
  static const int kWarpTiles[] = {1, 2, 4, 8, 16, 32};
  for (int X = 0; X < NPAIRCLASS && rc == ERI_OK; ++X)
    for (int Y = 0; Y <= X && rc == ERI_OK; ++Y) {
      const int64_t tot = P->h_ktot[X * NPAIRCLASS + Y];
      if (tot == 0) continue;
      for (int tier = 0; tier < (mixed ? 2 : 1) && rc == ERI_OK; ++tier) {
        const int def = default_tile(X, Y, tier);
        // windows long enough that every resident warp gets several tiles (a
        // short window measures the launch tail, not the tile length)
        int64_t win = std::min<int64_t>(tot, 3 * (int64_t)P->nsm * 2048);
        double t0 = trial(X, Y, tier, def, win / 3);
        if (t0 < 0.0) { rc = ERI_ECUDA; break; }
        for (int grow = 0; grow < 2 && t0 < 0.5 * trial_ms && win < tot; ++grow) {
          win = std::min<int64_t>(tot, (int64_t)((double)win * trial_ms / std::max(t0, 1e-3)));
          t0 = trial(X, Y, tier, def, win / 3 + 1);
          if (t0 < 0.0) { rc = ERI_ECUDA; break; }
        }
        if (rc != ERI_OK) break;
        const bool thr = use_thread_kernel(kClassL1[X], kClassL2[X], kClassL1[Y], kClassL2[Y], tier == 1);
        const int* cand = thr ? kThreadTiles : kWarpTiles;
        const int nc = thr ? 4 : 6;
        int best = def;
        double bt = t0;
        for (int i = 0; i < nc; ++i) {
          if (cand[i] == def) continue;
          const double t = trial(X, Y, tier, cand[i], win / 3 + 1);
          if (t < 0.0) { rc = ERI_ECUDA; break; }
          if (t < 0.95 * bt) { bt = t; best = cand[i]; }
        }
        if (rc == ERI_OK && best != def) {  // confirm against the default once more
          const double td = trial(X, Y, tier, def, win / 3 + 1), tb = trial(X, Y, tier, best, win / 3 + 1);
          if (td < 0.0 || tb < 0.0) { rc = ERI_ECUDA; break; }
          if (!(tb < 0.95 * td)) best = def;
        }
        P->tile_k[(X * NPAIRCLASS + Y) * 2 + tier] = best;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (P->gexec) {  // captured builds carry the old tiles
    cudaStreamSynchronize(s);
    cudaGraphExecDestroy(P->gexec);
    P->gexec = nullptr;
  }
  if (rc == ERI_OK) rc = tune_cache_store(P, precision);
  return rc;
}

extern "C" int eri_plan_set_shard(eri_plan_t* plan, int32_t shard, int32_t nshard) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || nshard < 1 || shard < 0 || shard >= nshard) return ERI_EINVAL;
  if (P->gexec && (shard != P->shard || nshard != P->nshard)) {  // captured builds carry the old share
    CK(cudaSetDevice(P->device));
    CK(cudaDeviceSynchronize());
    CK(cudaGraphExecDestroy(P->gexec));
    P->gexec = nullptr;
  }
  P->shard = shard;
  P->nshard = nshard;
  return ERI_OK;
}

extern "C" int eri_plan_set_omega(eri_plan_t* plan, double omega) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || !(omega >= 0.0) || !(omega < 1.0e30)) return ERI_EINVAL;
  if (P->gexec && omega != P->omega) {  // a captured graph carries the old operator
    CK(cudaSetDevice(P->device));
    CK(cudaDeviceSynchronize());
    CK(cudaGraphExecDestroy(P->gexec));
    P->gexec = nullptr;
  }
  P->omega = omega;
  return ERI_OK;
}

extern "C" int eri_plan_set_tau(eri_plan_t* plan, double mixed_tau) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || !(mixed_tau >= 0.0)) return ERI_EINVAL;
  if (P->gexec && mixed_tau != P->opts.mixed_tau) {  // the graph's launches carry the old threshold
    CK(cudaSetDevice(P->device));
    CK(cudaDeviceSynchronize());
    CK(cudaGraphExecDestroy(P->gexec));
    P->gexec = nullptr;
  }
  P->opts.mixed_tau = mixed_tau;
  return ERI_OK;
}

extern "C" int eri_get_tiles(eri_plan_t* plan, int32_t* tiles) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || !tiles) return ERI_EINVAL;
  for (int X = 0; X < NPAIRCLASS; ++X)
    for (int Y = 0; Y < NPAIRCLASS; ++Y)
      for (int t = 0; t < 2; ++t) {
        const int k = (X * NPAIRCLASS + Y) * 2 + t;
        tiles[k] = Y <= X ? P->tile_for(X, Y, t) : 0;
      }
  return ERI_OK;
}

extern "C" int eri_set_tiles(eri_plan_t* plan, const int32_t* tiles) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || !tiles) return ERI_EINVAL;
  for (int k = 0; k < NPAIRCLASS * NPAIRCLASS * 2; ++k)
    if (tiles[k] < 0 || tiles[k] > 1024) return ERI_EINVAL;
  if (P->gexec) {  // a captured graph carries the old tiles: wait for it on the plan's device, then drop it
    CK(cudaSetDevice(P->device));
    CK(cudaDeviceSynchronize());
    CK(cudaGraphExecDestroy(P->gexec));
    P->gexec = nullptr;
  }
  for (int k = 0; k < NPAIRCLASS * NPAIRCLASS * 2; ++k) P->tile_k[k] = tiles[k];
  return ERI_OK;
}

// FP64 J/K over canonical quartets with caller-provided scratch (D', half-K,
// half-J, each nbf*nbf doubles).  Serves eri_build_jk_noalloc (noalloc.cu):
// launches kernels only, allocates nothing, uses the plan's current lists.
int eri_build_jk_scratch(eri_plan_t* plan, const double* D, double* J, double* K, double* Dp, double* Kh, double* Jh,
                         cudaStream_t s) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  const int64_t nn = P->nmat;
  const MolMats mm = molmats(P);
  k_scale_d<<<P->mat_grid(256), 256, 0, s>>>(mm, D, P->d_f, Dp, nullptr);
  CK(cudaGetLastError());
  if (K) CK(cudaMemsetAsync(Kh, 0, sizeof(double) * nn, s));
  if (J) CK(cudaMemsetAsync(Jh, 0, sizeof(double) * nn, s));
  JKArgs ja{};
  KArgs& ka = ja.k;
  ka.pd = P->pairdata(); ka.sp = P->spinfo(); ka.bt = P->boystabs();
  ka.rsteps = P->d_rsteps; ka.Dp = Dp; ka.Dpf = nullptr; ka.Kh = K ? Kh : nullptr;
  ka.Q = P->d_Q; ka.dmax = P->d_dmax; ka.pmaxp = P->d_pmaxp; ka.prefmaxp = P->d_prefmaxp;
  ka.shloc = P->d_shloc; ka.pbase = P->d_pbase;
  ka.tau = 0.0f; ka.pmax32 = 0.0f; ka.mixed = 0; ka.tier_want = 0; ka.counter = nullptr; ka.guard = nullptr;
  ka.items = nullptr; ka.nitems = nullptr;
  ka.omega2 = P->omega * P->omega; ka.omega2f = (float)ka.omega2;
  ka.det = P->opts.deterministic ? 1 : 0;
  ja.Jh = J ? Jh : nullptr;
  P->last_mixed = false;
  P->last_do_j = J != nullptr;
  P->last_do_k = K != nullptr;
  for (int X = 0; X < NPAIRCLASS; ++X)
    for (int Y = 0; Y <= X; ++Y) {
      ka.wl = P->klist(X, Y);
      ka.wl.tile = P->tile_for(X, Y, 0);
      ka.same_class = X == Y;
      if (ka.wl.total == 0) continue;
      CK(launch_jk_class(X, Y, 0, ja, s, P->nsm));
    }
  if (K) {
    k_post_k<<<P->mat_grid(256), 256, 0, s>>>(mm, Kh, P->d_f, K, ka.det, P->d_status);
    CK(cudaGetLastError());
  }
  if (J) {
    k_post_k<<<P->mat_grid(256), 256, 0, s>>>(mm, Jh, P->d_f, J, ka.det, P->d_status);
    CK(cudaGetLastError());
  }
  return ERI_OK;
}

int eri_plan_nbf_device(eri_plan_t* plan, int* nbf, int* device, int* nmol) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  *nbf = P->nbf;
  *nmol = P->nmol;
  *device = P->device;
  return ERI_OK;
}

extern "C" int eri_energy(eri_plan_t* plan, const double* D, const double* J, const double* K, double* E_out,
                          void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || !D || !E_out) return ERI_EINVAL;
  CK(cudaSetDevice(P->device));
  k_energy<<<P->nmol, 1024, 0, (cudaStream_t)stream>>>(molmats(P), D, J, K, E_out);
  CK(cudaGetLastError());
  return ERI_OK;
}

static cudaError_t launch_grad_class(int X, int Y, int prec, const GradArgs& ga, cudaStream_t s, int nsm) {
#define ERI_GRAD_UNIT_CALL(UX, UP) \
  if (X == UX && prec == UP) return launch_grad_unit<UX, UP, 0>(Y, ga, s, nsm);
  ERI_GRAD_UNITS(ERI_GRAD_UNIT_CALL)
#undef ERI_GRAD_UNIT_CALL
  return cudaErrorInvalidValue;
}

extern "C" int eri_jk_grad_prec(eri_plan_t* plan, const double* D, double* dEdR, int32_t want_j, int32_t want_k,
                                int32_t precision, void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || !D || !dEdR) return ERI_EINVAL;
  if (precision != ERI_FP64 && precision != ERI_MIXED) return ERI_EINVAL;
  const bool mixed = precision == ERI_MIXED;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(P->device));
  const MolMats mm = molmats(P);
  k_scale_d<<<P->mat_grid(256), 256, 0, s>>>(mm, D, P->d_f, P->d_Dp, mixed ? P->d_Dpf : nullptr);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(dEdR, 0, sizeof(double) * 3 * P->natom, s));
  if (!want_j && !want_k) return ERI_OK;
  if (mixed) {
    k_dmax<<<grid1(P->npair, 128), 128, 0, s>>>(P->npair, P->d_ps1, P->d_ps2, P->d_sh_l, P->d_pao1, P->d_pao2,
                                                P->d_pmol, P->d_mat_off, P->d_mat_n, P->d_Dp, P->d_dmax);
    CK(cudaGetLastError());
    const int rc = P->ensure_tier_bufs(1);
    if (rc != ERI_OK) return rc;
  }
  GradArgs ga{};
  ga.pd = P->pairdata(); ga.sp = P->spinfo(); ga.bt = P->boystabs(); ga.rsteps = P->d_rsteps; ga.Dp = P->d_Dp;
  ga.Dpf = P->d_Dpf;
  ga.ea = P->d_ea; ga.sh_atom = P->d_sh_atom; ga.grad = dEdR;
  ga.cj = want_j ? 1.0 : 0.0;
  ga.ck = want_k ? 1.0 : 0.0;
  ga.omega2 = P->omega * P->omega;
  ga.omega2f = (float)ga.omega2;
  ga.det = P->opts.deterministic ? 1 : 0;
  // tier split of the ordered lists: the energy's test (reading 5) on each item
  KArgs ka{};
  ka.pd = P->pairdata(); ka.sp = P->spinfo();
  ka.Q = P->d_Q; ka.dmax = P->d_dmax; ka.pmaxp = P->d_pmaxp; ka.prefmaxp = P->d_prefmaxp;
  ka.shloc = P->d_shloc; ka.pbase = P->d_pbase;
  ka.tau = (float)P->opts.mixed_tau; ka.pmax32 = (float)kPmax32; ka.mixed = 1;
  unsigned long long* gcnt = P->d_counters2 + NPAIRCLASS * NPAIRCLASS * 3;  // kinds 1 (FP64) and 2 (FP32)
  CK(cudaMemsetAsync(gcnt, 0, sizeof(unsigned long long) * 2 * NPAIRCLASS * NPAIRCLASS * 3, s));
  auto launch = [&](int X, int Y, int tier) -> int {
    ga.counter = gcnt + ((tier * NPAIRCLASS + X) * NPAIRCLASS + Y) * 3;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (P->opts.profile) {
      CK(P->prof_event_pair(&e0, &e1));
      CK(cudaEventRecord(e0, s));
    }
    CK(launch_grad_class(X, Y, tier, ga, s, P->nsm));
    if (P->opts.profile) {
      CK(cudaEventRecord(e1, s));
      P->prof_log.push_back({X, Y, tier ? 4 : 2, P->prof_ev_used - 2});
    }
    return ERI_OK;
  };
  for (int X = 0; X < NPAIRCLASS; ++X)
    for (int Y = 0; Y < NPAIRCLASS; ++Y) {
      const WorkList full = P->jlist(X, Y);
      if (full.total == 0) continue;
      if (!mixed) {
        ga.wl = full;
        ga.items = nullptr;
        ga.nitems = nullptr;
        const int rc = launch(X, Y, 0);
        if (rc != ERI_OK) return rc;
        continue;
      }
      int2* buf = P->tbuf[0];
      unsigned int* cnt = P->tcnt;
      for (int64_t f = 0; f < full.total; f += P->tier_cap) {
        ka.wl = full;
        ka.wl.first = f;
        ka.wl.total = std::min<int64_t>(full.total, f + P->tier_cap);
        CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned int), s));
        const int64_t nch = (ka.wl.total - f + 31) / 32;
        k_tier_split<<<(int)std::max<int64_t>(1, std::min<int64_t>((nch + 7) / 8, (int64_t)P->nsm * 8)), 256, 0,
                       s>>>(ka, buf, buf + P->tier_cap, cnt);
        CK(cudaGetLastError());
        for (int tier = 0; tier < 2; ++tier) {
          ga.wl = full;
          ga.wl.first = 0;
          ga.wl.total = ka.wl.total - f;  // upper bound of the tier's count (grid sizing)
          ga.items = buf + (tier ? P->tier_cap : 0);
          ga.nitems = cnt + tier;
          const int rc = launch(X, Y, tier);
          if (rc != ERI_OK) return rc;
        }
      }
    }
  if (ga.det) {
    k_fix_to_double<<<grid1(3 * P->natom, 128), 128, 0, s>>>(3 * P->natom, dEdR, P->d_status);
    CK(cudaGetLastError());
  }
  return ERI_OK;
}

extern "C" int eri_jk_grad(eri_plan_t* plan, const double* D, double* dEdR, int32_t want_j, int32_t want_k,
                           void* stream) {
  return eri_jk_grad_prec(plan, D, dEdR, want_j, want_k, ERI_FP64, stream);
}

extern "C" int eri_get_lists(eri_plan_t* plan, float* Q, int32_t* sig, int32_t* counts, int32_t* sorted,
                             int32_t* class_count) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P) return ERI_EINVAL;
  CK(cudaSetDevice(P->device));
  CK(cudaDeviceSynchronize());
  if (Q) CK(cudaMemcpy(Q, P->d_Q, sizeof(float) * P->npair, cudaMemcpyDeviceToHost));
  if (sig) CK(cudaMemcpy(sig, P->d_sig, sizeof(int) * P->npair, cudaMemcpyDeviceToHost));
  if (counts) CK(cudaMemcpy(counts, P->d_counts, sizeof(int) * P->npair * NPAIRCLASS, cudaMemcpyDeviceToHost));
  if (sorted) CK(cudaMemcpy(sorted, P->d_sorted, sizeof(int) * P->nsig, cudaMemcpyDeviceToHost));
  if (class_count) memcpy(class_count, P->h_ccount, sizeof(int) * NPAIRCLASS);
  return ERI_OK;
}

extern "C" int eri_check(eri_plan_t* plan) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P) return ERI_EINVAL;
  CK(cudaSetDevice(P->device));
  CK(cudaDeviceSynchronize());
  int status = 0;
  CK(cudaMemcpy(&status, P->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status == 0) return ERI_OK;
  CK(cudaMemset(P->d_status, 0, sizeof(int)));
  return ERI_EDEVICE;
}

extern "C" int eri_get_stats(eri_plan_t* plan, eri_stats_t* st) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || !st) return ERI_EINVAL;
  CK(cudaSetDevice(P->device));
  memset(st, 0, sizeof(*st));
  st->nbf = P->nbf;
  st->nshell = P->nshell;
  st->npair = P->npair;
  st->nsig_pair = P->nsig;
  for (int i = 0; i < NPAIRCLASS * NPAIRCLASS; ++i) {
    st->quartets_j += P->h_jtot[i];
    int X = i / NPAIRCLASS, Y = i % NPAIRCLASS;
    if (Y <= X) {
      st->quartets_k += P->h_ktot[i];
      st->prim_quartets_k += P->h_kprim[i];
    }
  }
  {
    unsigned long long c[NPAIRCLASS * NPAIRCLASS * 6 + 2];
    CK(cudaMemcpy(c, P->d_counters, sizeof(c), cudaMemcpyDeviceToHost));
    st->quartets_k_guard = P->last_mixed ? (int64_t)c[NPAIRCLASS * NPAIRCLASS * 6] : 0;
    st->quartets_k_screened = (int64_t)c[NPAIRCLASS * NPAIRCLASS * 6 + 1];
    st->graph_branches = P->gexec ? P->gbranches : 0;
    double fl = 0.0;
    for (int X = 0; X < NPAIRCLASS; ++X)
      for (int Y = 0; Y <= X; ++Y)
        for (int t = 0; t < 2; ++t) {
          const unsigned long long* q = c + ((X * NPAIRCLASS + Y) * 2 + t) * 3;
          fl += class_flops(X, Y, (double)q[0], (double)q[1], (double)q[2], P->last_do_j, P->last_do_k);
          if (t == 1) st->quartets_k_fp32 += (int64_t)q[0];
        }
    st->flops_k = fl;
    st->flops_j = 0.0;
    unsigned long long c2[NPAIRCLASS * NPAIRCLASS * 3];
    CK(cudaMemcpy(c2, P->d_counters2 + 3 * NPAIRCLASS * NPAIRCLASS * 3, sizeof(c2), cudaMemcpyDeviceToHost));
    for (int i = 0; i < NPAIRCLASS * NPAIRCLASS; ++i) st->quartets_j_fp32 += P->last_jmixed ? (int64_t)c2[3 * i] : 0;
  }
  int status = 0;
  CK(cudaMemcpy(&status, P->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  st->device_status = status;
  return ERI_OK;
}

extern "C" int eri_get_profile(eri_plan_t* plan, eri_launch_prof_t* out, int32_t cap, int32_t* count) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P || !count || (cap > 0 && !out)) return ERI_EINVAL;
  CK(cudaSetDevice(P->device));
  CK(cudaDeviceSynchronize());
  unsigned long long c[NPAIRCLASS * NPAIRCLASS * 6], c2[4 * NPAIRCLASS * NPAIRCLASS * 3];
  CK(cudaMemcpy(c, P->d_counters, sizeof(c), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(c2, P->d_counters2, sizeof(c2), cudaMemcpyDeviceToHost));
  constexpr int NT = 6;  // tiers: 0 FP64 J/K, 1 FP32 J/K, 2 gradient FP64, 3 J-engine, 4 gradient FP32, 5 J-engine FP32
  double ms[NPAIRCLASS * NPAIRCLASS * NT] = {};
  int nl[NPAIRCLASS * NPAIRCLASS * NT] = {};
  for (const auto& r : P->prof_log) {
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, P->prof_events[r.ev], P->prof_events[r.ev + 1]));
    const int k = (r.X * NPAIRCLASS + r.Y) * NT + r.tier;
    ms[k] += t;
    nl[k] += 1;
  }
  int n = 0;
  for (int k = 0; k < NPAIRCLASS * NPAIRCLASS * NT; ++k) {
    if (!nl[k]) continue;
    if (n < cap) {
      const int X = k / (NT * NPAIRCLASS), Y = (k / NT) % NPAIRCLASS, t = k % NT;
      // counters2 kinds: J-engine FP64, gradient FP64, gradient FP32, J-engine FP32
      const int kind = t == 3 ? 0 : (t == 2 ? 1 : (t == 4 ? 2 : 3));
      const unsigned long long* q = t < 2 ? c + ((X * NPAIRCLASS + Y) * 2 + t) * 3
                                          : c2 + (kind * NPAIRCLASS * NPAIRCLASS + X * NPAIRCLASS + Y) * 3;
      eri_launch_prof_t& o = out[n];
      o.bra_class = X;
      o.ket_class = Y;
      o.tier = t;
      o.launches = nl[k];
      o.ms = ms[k];
      o.quartets = (int64_t)q[0];
      o.prim_quartets = (int64_t)q[1];
      o.flops = t < 2 ? class_flops(X, Y, (double)q[0], (double)q[1], (double)q[2], P->last_do_j, P->last_do_k)
                      : (t == 2 || t == 4) ? grad_flops(X, Y, (double)q[0], (double)q[1], (double)q[2])
                               : jengine_flops(X, Y, (double)q[1]);
    }
    ++n;
  }
  *count = n;
  P->prof_log.clear();
  P->prof_ev_used = 0;
  P->prof_builds = 0;
  return ERI_OK;
}

extern "C" int eri_plan_destroy(eri_plan_t* plan) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  if (!P) return ERI_OK;
  cudaSetDevice(P->device);
  cudaDeviceSynchronize();
  P->release();
  delete P;
  return ERI_OK;
}

extern "C" const char* eri_strerror(int code) {
  switch (code) {
    case ERI_OK: return "success";
    case ERI_EINVAL: return "invalid argument";
    case ERI_ENOMEM: return "out of memory";
    case ERI_ECUDA: return "CUDA runtime error";
    case ERI_EUNSUPPORTED: return "unsupported request";
    case ERI_ETIMEOUT: return "bounded device wait timed out";
    case ERI_EDEVICE: return "device-side check failed";
  }
  return "unknown error";
}
