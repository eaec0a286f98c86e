// Point-charge attraction matrix V and its gradient (Sec. 2.4 of Wang et al.).
//
//   V_mn = sum_C q_C (m| 1/|r - C| |n)                       Eq. v1e_definition
//        = sum_{prim pairs} (2 pi / p) C_m C_n K_AB sum_P E_P^{mn} sum_C q_C R^0_P(p, P - C)
//                                                            Eq. v1e_formula
// The sum over charges is taken in Hermite space first, exactly like the
// J-engine's ket sum (Eq. j_formula): per primitive pair of every shell pair,
//   h_P = sum_C q_C (2 pi / p) C C K R^0_P(p, P - C),
// then one Hermite-to-Cartesian pass (the J-engine's k_post_j) gives V.
//
// Gradient of E_V = sum_mn D_mn V_mn with D fixed (SI Sec. 1.3,
// Eq. si_v1e_derivative_A / _B / _C): with the Hermite densities of each
// primitive pair (sign-free, the pair counted in both orders)
//   d_P      = s sum_mn D'_mn E_P^{mn},                          P <= l1 + l2
//   dA_{t,P} = s sum_mn D'_mn [2a E_P^{(m+1_t) n} - m_t E_P^{(m-1_t) n}],  P <= l1 + l2 + 1
// (the raising/lowering rule on the centre A of the first shell), each term
// (pair, charge C) contributes
//   dE/dA_t = sum_P dA_{t,P} R_P,   dE/dC_t = -sum_P d_P R_{P+1_t}  (dR/dC = -R_{P+1_t}),
//   dE/dB_t = -(dE/dA_t + dE/dC_t)  (the term depends on A, B, C through differences only).
// One kernel runs per primitive pair over the charges (A and B), one per
// charge over the primitive pairs (C); both evaluate R up to l1 + l2 + 1 in
// registers with compile-time indices, one specialisation per l1 + l2.
#include <algorithm>
#include <vector>

#include "../../include/eri.h"
#include "dispatch.cuh"
#include "plan.cuh"

using namespace eri;

namespace {

constexpr double kVfac = 1.0622519320271968;  // (2 pi / p) / (sqrt(2 pi^(5/2)) / p): pair prefactor of V from the ERI one
constexpr int kChunk = 256;                    // charges (or primitive pairs) per block row

#define NCK(x)                                                                   \
  do {                                                                           \
    cudaError_t e_ = (x);                                                        \
    if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? ERI_ENOMEM : ERI_ECUDA; \
  } while (0)

// h_P of one list entry (primitive pair) summed over one chunk of charges
template <int L>
__global__ void __launch_bounds__(128) k_nuc_herm(const int4* __restrict__ list, int n, PairData pd, BoysTabs bt,
                                                  int nc, const double* __restrict__ q, const double* __restrict__ xyz,
                                                  double* __restrict__ Vh) {
  constexpr int NH = nherm(L);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int4 e = __ldg(list + i);
  const int pi = e.x;
  const double p = __ldg(pd.p + pi), pref = __ldg(pd.pref + pi) * kVfac;
  const double Px = __ldg(pd.P + pi), Py = __ldg(pd.P + pd.n + pi), Pz = __ldg(pd.P + 2 * pd.n + pi);
  double h[NH];
#pragma unroll
  for (int x = 0; x < NH; ++x) h[x] = 0.0;
  const int c0 = blockIdx.y * kChunk, c1 = min(nc, c0 + kChunk);
  for (int c = c0; c < c1; ++c) {
    const double X = Px - __ldg(xyz + 3 * c), Y = Py - __ldg(xyz + 3 * c + 1), Z = Pz - __ldg(xyz + 3 * c + 2);
    double F[L + 1];
    boys_f64<L>(p * (X * X + Y * Y + Z * Z), bt, F);
    double R[NH];
    r_build_reg<L, double>(F, pref * __ldg(q + c), X, Y, Z, -2.0 * p, R);
#pragma unroll
    for (int x = 0; x < NH; ++x) h[x] += R[x];
  }
#pragma unroll
  for (int x = 0; x < NH; ++x) atomicAdd(Vh + e.y + x, h[x]);
}

// Hermite densities d_P and dA_{t,P} of every primitive pair (thread per shell pair)
__global__ void k_nuc_dens(int npair, const int* __restrict__ s1, const int* __restrict__ s2,
                           const int* __restrict__ np, const int* __restrict__ poff, const int* __restrict__ goff,
                           const int* __restrict__ sh_l, const int* __restrict__ pao1, const int* __restrict__ pao2,
                           const int* __restrict__ pmol, MolMats mm, PairData pd, const double* __restrict__ Dp,
                           double* __restrict__ G) {
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= npair) return;
  const int a = s1[ip], b = s2[ip], la = sh_l[a], lb = sh_l[b], L = la + lb;
  const int H = nherm(L), H1 = nherm(L + 1), stride = H + 3 * H1;
  const int m = pmol[ip], nbf = mm.n[m];
  const double* Dm = Dp + mm.off[m];
  const double sc = a == b ? 1.0 : 2.0;
  double E[3][225];
  for (int k = 0; k < np[ip]; ++k) {
    const int pi = poff[ip] + k;
    const double a2 = 2.0 * pd.ea[pi];
    for (int d = 0; d < 3; ++d) md_e_rt(la + 1, lb, pd.PA[d * pd.n + pi], pd.PB[d * pd.n + pi], 0.5 / pd.p[pi], E[d]);
    double* out = G + goff[ip] + (size_t)k * stride;
    for (int x = 0; x < stride; ++x) out[x] = 0.0;
    for (int mu = 0; mu < ncart(la); ++mu) {
      int i3[3];
      cart_xyz(la, mu, i3[0], i3[1], i3[2]);
      for (int nu = 0; nu < ncart(lb); ++nu) {
        int j3[3];
        cart_xyz(lb, nu, j3[0], j3[1], j3[2]);
        const double dv = sc * Dm[(size_t)(pao1[ip] + mu) * nbf + pao2[ip] + nu];
        for (int tx = 0; tx <= i3[0] + j3[0]; ++tx)
          for (int ty = 0; ty <= i3[1] + j3[1]; ++ty)
            for (int tz = 0; tz <= i3[2] + j3[2]; ++tz)
              out[herm_index(tx, ty, tz)] += dv * E[0][(i3[0] * 5 + j3[0]) * 9 + tx] *
                                             E[1][(i3[1] * 5 + j3[1]) * 9 + ty] * E[2][(i3[2] * 5 + j3[2]) * 9 + tz];
        // derivative densities: direction t raised (2a) and lowered (-i_t)
        for (int t = 0; t < 3; ++t) {
          double* o = out + H + t * H1;
          for (int sgn = 0; sgn < 2; ++sgn) {
            int ii[3] = {i3[0], i3[1], i3[2]};
            double w;
            if (sgn == 0) {
              ii[t] += 1;
              w = a2 * dv;
            } else {
              if (i3[t] == 0) continue;
              ii[t] -= 1;
              w = -i3[t] * dv;
            }
            for (int tx = 0; tx <= ii[0] + j3[0]; ++tx)
              for (int ty = 0; ty <= ii[1] + j3[1]; ++ty)
                for (int tz = 0; tz <= ii[2] + j3[2]; ++tz)
                  o[herm_index(tx, ty, tz)] += w * E[0][(ii[0] * 5 + j3[0]) * 9 + tx] *
                                               E[1][(ii[1] * 5 + j3[1]) * 9 + ty] *
                                               E[2][(ii[2] * 5 + j3[2]) * 9 + tz];
          }
        }
      }
    }
  }
}

// d/dA and d/dB of one primitive pair, summed over one chunk of charges
template <int L>
__global__ void __launch_bounds__(128) k_nuc_grad_pair(const int4* __restrict__ list, int n, PairData pd,
                                                       BoysTabs bt, const int* __restrict__ s1,
                                                       const int* __restrict__ s2, const int* __restrict__ sh_atom,
                                                       const double* __restrict__ G, int nc,
                                                       const double* __restrict__ q, const double* __restrict__ xyz,
                                                       double* __restrict__ dEdR) {
  constexpr int H = nherm(L), H1 = nherm(L + 1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int4 e = __ldg(list + i);
  const int pi = e.x;
  const double p = __ldg(pd.p + pi), pref = __ldg(pd.pref + pi) * kVfac;
  const double Px = __ldg(pd.P + pi), Py = __ldg(pd.P + pd.n + pi), Pz = __ldg(pd.P + 2 * pd.n + pi);
  const double* g = G + e.z;
  double gA[3] = {0.0, 0.0, 0.0}, gC[3] = {0.0, 0.0, 0.0};
  const int c0 = blockIdx.y * kChunk, c1 = min(nc, c0 + kChunk);
  for (int c = c0; c < c1; ++c) {
    const double X = Px - __ldg(xyz + 3 * c), Y = Py - __ldg(xyz + 3 * c + 1), Z = Pz - __ldg(xyz + 3 * c + 2);
    double F[L + 2];
    boys_f64<L + 1>(p * (X * X + Y * Y + Z * Z), bt, F);
    double R[H1];
    r_build_reg<L + 1, double>(F, pref * __ldg(q + c), X, Y, Z, -2.0 * p, R);
    sfor<3>([&](auto t_) {
      constexpr int t = ERI_CI(t_);
      double sa = 0.0, sc = 0.0;
      for_herm<L + 1>([&](auto x, auto y, auto z) {
        constexpr int P = herm_index(ERI_CI(x), ERI_CI(y), ERI_CI(z));
        sa = fma(__ldg(g + H + t * H1 + P), R[P], sa);
      });
      for_herm<L>([&](auto x, auto y, auto z) {
        constexpr int P = herm_index(ERI_CI(x), ERI_CI(y), ERI_CI(z));
        constexpr int P1 = herm_index(ERI_CI(x) + (t == 0), ERI_CI(y) + (t == 1), ERI_CI(z) + (t == 2));
        sc = fma(__ldg(g + P), R[P1], sc);
      });
      gA[t] += sa;
      gC[t] -= sc;
    });
  }
  const int ip = e.w;
  const int atA = __ldg(sh_atom + __ldg(s1 + ip)), atB = __ldg(sh_atom + __ldg(s2 + ip));
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    atomicAdd(dEdR + 3 * atA + t, gA[t]);
    atomicAdd(dEdR + 3 * atB + t, -(gA[t] + gC[t]));
  }
}

// d/dC of one charge, summed over one chunk of primitive pairs of list L
template <int L>
__global__ void __launch_bounds__(128) k_nuc_grad_charge(const int4* __restrict__ list, int n, PairData pd,
                                                         BoysTabs bt, const double* __restrict__ G, int nc,
                                                         const double* __restrict__ q,
                                                         const double* __restrict__ xyz, double* __restrict__ dEdC) {
  constexpr int H = nherm(L), H1 = nherm(L + 1);
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double Cx = __ldg(xyz + 3 * c), Cy = __ldg(xyz + 3 * c + 1), Cz = __ldg(xyz + 3 * c + 2), qc = __ldg(q + c);
  double gC[3] = {0.0, 0.0, 0.0};
  const int i0 = blockIdx.y * kChunk, i1 = min(n, i0 + kChunk);
  for (int i = i0; i < i1; ++i) {  // every thread reads the same entry: broadcast loads
    const int4 e = __ldg(list + i);
    const int pi = e.x;
    const double p = __ldg(pd.p + pi), pref = __ldg(pd.pref + pi) * kVfac;
    const double X = __ldg(pd.P + pi) - Cx, Y = __ldg(pd.P + pd.n + pi) - Cy, Z = __ldg(pd.P + 2 * pd.n + pi) - Cz;
    double F[L + 2];
    boys_f64<L + 1>(p * (X * X + Y * Y + Z * Z), bt, F);
    double R[H1];
    r_build_reg<L + 1, double>(F, pref * qc, X, Y, Z, -2.0 * p, R);
    const double* g = G + e.z;
    sfor<3>([&](auto t_) {
      constexpr int t = ERI_CI(t_);
      double sc = 0.0;
      for_herm<L>([&](auto x, auto y, auto z) {
        constexpr int P = herm_index(ERI_CI(x), ERI_CI(y), ERI_CI(z));
        constexpr int P1 = herm_index(ERI_CI(x) + (t == 0), ERI_CI(y) + (t == 1), ERI_CI(z) + (t == 2));
        sc = fma(__ldg(g + P), R[P1], sc);
      });
      gC[t] -= sc;
    });
  }
#pragma unroll
  for (int t = 0; t < 3; ++t) atomicAdd(dEdC + 3 * c + t, gC[t]);
  (void)H;
}

template <int L>
cudaError_t launch_herm(const eri_plan_impl* P, int nc, const double* q, const double* xyz, cudaStream_t s) {
  const int n = P->nuc_cnt[L];
  if (n == 0 || nc == 0) return cudaSuccess;
  const dim3 grid((n + 127) / 128, (nc + kChunk - 1) / kChunk);
  k_nuc_herm<L><<<grid, 128, 0, s>>>(P->d_nuc_list + P->nuc_first[L], n, P->pairdata(), P->boystabs(), nc, q, xyz,
                                     P->d_Jherm);
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_grad(const eri_plan_impl* P, int nc, const double* q, const double* xyz, double* dEdR,
                        double* dEdC, cudaStream_t s) {
  const int n = P->nuc_cnt[L];
  if (n == 0 || nc == 0) return cudaSuccess;
  const int4* list = P->d_nuc_list + P->nuc_first[L];
  const dim3 gp((n + 127) / 128, (nc + kChunk - 1) / kChunk);
  k_nuc_grad_pair<L><<<gp, 128, 0, s>>>(list, n, P->pairdata(), P->boystabs(), P->d_ps1, P->d_ps2, P->d_sh_atom,
                                        P->d_nuc_dens, nc, q, xyz, dEdR);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !dEdC) return e;
  const dim3 gc((nc + 127) / 128, (n + kChunk - 1) / kChunk);
  k_nuc_grad_charge<L><<<gc, 128, 0, s>>>(list, n, P->pairdata(), P->boystabs(), P->d_nuc_dens, nc, q, xyz, dEdC);
  return cudaGetLastError();
}

// Per-l1+l2 lists of every primitive pair and the offsets of their Hermite
// densities (basis only: built once per plan; synchronises the device).
int ensure_nuc(eri_plan_impl* P) {
  if (P->nuc_built) return ERI_OK;
  const int npair = P->npair;
  std::vector<int> s1(npair), s2(npair), np(npair), poff(npair), hoff(npair), shl(P->nshell);
  NCK(cudaMemcpy(s1.data(), P->d_ps1, sizeof(int) * npair, cudaMemcpyDeviceToHost));
  NCK(cudaMemcpy(s2.data(), P->d_ps2, sizeof(int) * npair, cudaMemcpyDeviceToHost));
  NCK(cudaMemcpy(np.data(), P->d_pnp, sizeof(int) * npair, cudaMemcpyDeviceToHost));
  NCK(cudaMemcpy(poff.data(), P->d_ppoff, sizeof(int) * npair, cudaMemcpyDeviceToHost));
  NCK(cudaMemcpy(hoff.data(), P->d_phoff, sizeof(int) * npair, cudaMemcpyDeviceToHost));
  NCK(cudaMemcpy(shl.data(), P->d_sh_l, sizeof(int) * P->nshell, cudaMemcpyDeviceToHost));
  constexpr int NL = 2 * LMAX + 1;
  std::vector<int4> lists[NL];
  std::vector<int> goff(npair);
  int64_t g = 0;
  for (int ip = 0; ip < npair; ++ip) {
    const int L = shl[s1[ip]] + shl[s2[ip]], H = nherm(L), G = H + 3 * nherm(L + 1);
    goff[ip] = (int)g;
    for (int k = 0; k < np[ip]; ++k) lists[L].push_back(make_int4(poff[ip] + k, hoff[ip] + k * H, (int)(g + (int64_t)k * G), ip));
    g += (int64_t)np[ip] * G;
    if (g > INT32_MAX) return ERI_EUNSUPPORTED;
  }
  std::vector<int4> all;
  for (int L = 0; L < NL; ++L) {
    P->nuc_first[L] = (int)all.size();
    P->nuc_cnt[L] = (int)lists[L].size();
    all.insert(all.end(), lists[L].begin(), lists[L].end());
  }
  P->nuc_first[NL] = (int)all.size();
  NCK(cudaMalloc(&P->d_nuc_list, sizeof(int4) * std::max<size_t>(1, all.size())));
  NCK(cudaMalloc(&P->d_nuc_goff, sizeof(int) * std::max(1, npair)));
  NCK(cudaMalloc(&P->d_nuc_dens, sizeof(double) * std::max<int64_t>(1, g)));
  NCK(cudaMemcpy(P->d_nuc_list, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice));
  NCK(cudaMemcpy(P->d_nuc_goff, goff.data(), sizeof(int) * npair, cudaMemcpyHostToDevice));
  P->nuc_built = 1;
  return ERI_OK;
}

int check_charges(eri_plan_impl* P, int32_t nc, const double* q, const double* xyz) {
  if (!P || nc < 0 || (nc > 0 && (!q || !xyz))) return ERI_EINVAL;
  return ERI_OK;
}

}  // namespace

extern "C" int eri_nuclear(eri_plan_t* plan, int32_t ncharge, const double* q, const double* xyz, double* V,
                           void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  int rc = check_charges(P, ncharge, q, xyz);
  if (rc != ERI_OK || !V) return rc != ERI_OK ? rc : ERI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  NCK(cudaSetDevice(P->device));
  if ((rc = ensure_nuc(P)) != ERI_OK) return rc;
  NCK(cudaMemsetAsync(P->d_Jherm, 0, sizeof(double) * (size_t)P->nherm_tot, s));
  NCK(launch_herm<0>(P, ncharge, q, xyz, s));
  NCK(launch_herm<1>(P, ncharge, q, xyz, s));
  NCK(launch_herm<2>(P, ncharge, q, xyz, s));
  NCK(launch_herm<3>(P, ncharge, q, xyz, s));
  NCK(launch_herm<4>(P, ncharge, q, xyz, s));
  NCK(launch_herm<5>(P, ncharge, q, xyz, s));
  NCK(launch_herm<6>(P, ncharge, q, xyz, s));
  const MolMats mm = molmats(P);
  k_post_j<<<(int)(((int64_t)P->npair * 100 + 127) / 128), 128, 0, s>>>(
      P->npair, P->d_ps1, P->d_ps2, P->d_pnp, P->d_ppoff, P->d_phoff, P->d_sh_l, P->d_pao1, P->d_pao2, P->d_pmol, mm,
      nullptr, P->pairdata(), P->d_Jherm, P->d_f, V, 0, P->d_status);
  NCK(cudaGetLastError());
  return ERI_OK;
}

extern "C" int eri_nuclear_grad(eri_plan_t* plan, const double* D, int32_t ncharge, const double* q,
                                const double* xyz, double* dEdR, double* dEdC, void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  int rc = check_charges(P, ncharge, q, xyz);
  if (rc != ERI_OK || !D || !dEdR) return rc != ERI_OK ? rc : ERI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  NCK(cudaSetDevice(P->device));
  if ((rc = ensure_nuc(P)) != ERI_OK) return rc;
  const MolMats mm = molmats(P);
  k_scale_d_launch(P, D, s);
  NCK(cudaGetLastError());
  k_nuc_dens<<<(P->npair + 63) / 64, 64, 0, s>>>(P->npair, P->d_ps1, P->d_ps2, P->d_pnp, P->d_ppoff, P->d_nuc_goff,
                                                 P->d_sh_l, P->d_pao1, P->d_pao2, P->d_pmol, mm, P->pairdata(),
                                                 P->d_Dp, P->d_nuc_dens);
  NCK(cudaGetLastError());
  NCK(cudaMemsetAsync(dEdR, 0, sizeof(double) * 3 * (size_t)P->natom, s));
  if (dEdC && ncharge > 0) NCK(cudaMemsetAsync(dEdC, 0, sizeof(double) * 3 * (size_t)ncharge, s));
  NCK(launch_grad<0>(P, ncharge, q, xyz, dEdR, dEdC, s));
  NCK(launch_grad<1>(P, ncharge, q, xyz, dEdR, dEdC, s));
  NCK(launch_grad<2>(P, ncharge, q, xyz, dEdR, dEdC, s));
  NCK(launch_grad<3>(P, ncharge, q, xyz, dEdR, dEdC, s));
  NCK(launch_grad<4>(P, ncharge, q, xyz, dEdR, dEdC, s));
  NCK(launch_grad<5>(P, ncharge, q, xyz, dEdR, dEdC, s));
  NCK(launch_grad<6>(P, ncharge, q, xyz, dEdR, dEdC, s));
  return ERI_OK;
}
