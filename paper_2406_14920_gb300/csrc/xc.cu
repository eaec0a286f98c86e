// Exchange-correlation quadrature on a molecular grid (Sec. 2.6 of Wang et al.).
//
// The paper's four steps, each a device kernel here:
//  (1) grid        k_xc_nodes, k_xc_points: atom-centred products of a radial
//                  rule (Gauss-Chebyshev nodes of the second kind mapped by
//                  Becke's r = R (1+x)/(1-x)) and an angular rule
//                  (Gauss-Legendre in cos(theta) x trapezoid in phi, 2 n_theta
//                  azimuths), weighted by Becke's fuzzy cells of equal size;
//  (2) density     rho = sum_mn D_mn phi_m phi_n and grad rho
//                  (Eq. xc_density_0, Eq. xc_density_1): k_xc_ao, k_xc_rho;
//  (3) functional  Slater or Becke-88 exchange per point (k_xc_func);
//  (4) matrix      V_mn = sum_g w_g [v_rho phi_m phi_n + v_grad . grad(phi_m phi_n)]
//                  (Eq. xc_grid_sum_0 + Eq. xc_grid_sum_1): k_xc_vmat.
//
// Layout.  Points are grouped into blocks of at most 32 that are close in
// space: one atom, a group of adjacent radial shells and one thirty-second of
// the sphere (a quarter of the theta nodes x an eighth of the azimuths).  A block keeps
// the shells whose extent (the radius beyond which every component and its
// gradient stays below 1e-15) reaches its bounding sphere: the paper's grid
// boxes with pair cutoffs (Sec. 3.5), per shell instead of per pair.  The
// values phi and grad phi of every block's significant functions are computed
// once per geometry and kept in HBM ([block][component c = phi, d/dx, d/dy,
// d/dz][function][point]); above the workspace cap they are recomputed per
// chunk of blocks instead.  The density is one dense product X = D_b Phi_b per
// block (thread = grid point, rows of D_b staged in shared memory, then
// rho = sum_m phi_m X_m and grad rho = 2 sum_m grad phi_m X_m); the matrix is
// the block-sparse product V = sum_b (Z_b Phi_b^T + Phi_b Z_b^T) with
// Z = w (v_rho phi / 2 + v_grad . grad phi), computed output-stationary: a CTA
// owns a 32 x 32 tile of V and walks the blocks of its share, so V receives
// one atomic per element per share.  All arithmetic is FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/eri.h"
#include "plan.cuh"

using namespace eri;

namespace {

constexpr int kBP = 32;           // points per block (at most) = threads of the per-block kernels
constexpr int kWarps = kBP / 32;
constexpr int kRT = 16;           // rows of D_b per register tile (k_xc_rho)
constexpr int kNC = 64;           // columns of D_b per staged chunk (k_xc_rho)
constexpr int kVT = 64;           // V tile edge (basis functions), k_xc_vmat
constexpr int kVP = 16;           // points per staged chunk, k_xc_vmat
constexpr int kVThreads = 256;    // k_xc_vmat block
constexpr int kVOut = kVT * kVT / kVThreads;  // outputs per thread and block (at most)
constexpr int kSlots = 5;         // workspace rows per function: phi, d/dx, d/dy, d/dz, Z
constexpr double kAoEps = 1e-15;  // shell extent: every |phi| and |grad phi| below this beyond it
constexpr double kRhoMin = 1e-14; // points with a smaller density contribute nothing
constexpr double kPi = 3.14159265358979323846;
constexpr size_t kDefaultCap = size_t(16) << 30;  // default workspace cap for resident basis values

#define XCK(x)                                                                             \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? ERI_ENOMEM : ERI_ECUDA; \
  } while (0)

template <typename T>
cudaError_t xalloc(T** p, size_t n) {
  *p = nullptr;
  return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Radial nodes r_i, weights (pi/(n+1)) sin(theta_i) r^2 dr/dx for i = 1..nrad
// (Gauss-Chebyshev of the second kind, Becke's map); Gauss-Legendre nodes in
// cos(theta) (ascending) and weights, by Newton's method on P_n.
__global__ void k_xc_nodes(int nrad, int ntheta, double R, double* __restrict__ rad, double* __restrict__ ang) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nrad) {
    const int i = t + 1;
    const double th = i * kPi / (nrad + 1), x = cos(th);
    const double r = R * (1.0 + x) / (1.0 - x);
    rad[2 * t] = r;
    rad[2 * t + 1] = kPi / (nrad + 1) * sin(th) * r * r * 2.0 * R / ((1.0 - x) * (1.0 - x));
  }
  if (t < ntheta) {
    const int n = ntheta;
    double x = cos(kPi * (t + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (x * p1 - p0) / (x * x - 1.0);
    ang[2 * (n - 1 - t)] = x;
    ang[2 * (n - 1 - t) + 1] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

// 1/|A - B| for every atom pair (0 on the diagonal)
__global__ void k_xc_invab(int na, const double* __restrict__ xyz, double* __restrict__ inv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= na * na) return;
  const int a = i / na, b = i % na;
  if (a == b) {
    inv[i] = 0.0;
    return;
  }
  const double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1], dz = xyz[3 * a + 2] - xyz[3 * b + 2];
  inv[i] = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
}

// Step (1): point g = ((atom * nrad + i) * ntheta + j) * nphi + k, weight
// w_rad * w_ang * (Becke weight of its atom)
__global__ void k_xc_points(int64_t G, int na, int nrad, int ntheta, const double* __restrict__ xyz,
                            const double* __restrict__ rad, const double* __restrict__ ang,
                            const double* __restrict__ invab, double* __restrict__ pts, double* __restrict__ w) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int nphi = 2 * ntheta;
  int64_t q = g;
  const int k = (int)(q % nphi); q /= nphi;
  const int j = (int)(q % ntheta); q /= ntheta;
  const int i = (int)(q % nrad); q /= nrad;
  const int a = (int)q;
  const double r = rad[2 * i], wr = rad[2 * i + 1];
  const double ct = ang[2 * j], st = sqrt(1.0 - ct * ct), wa = ang[2 * j + 1] * 2.0 * kPi / nphi;
  const double ph = 2.0 * kPi * (k + 0.5) / nphi;
  const double px = xyz[3 * a] + r * st * cos(ph), py = xyz[3 * a + 1] + r * st * sin(ph), pz = xyz[3 * a + 2] + r * ct;
  pts[3 * g] = px;
  pts[3 * g + 1] = py;
  pts[3 * g + 2] = pz;
  // Becke cells: P_A = prod_{B != A} s(mu_AB), w = P_a / sum_A P_A
  double sumP = 0.0, Pown = 0.0;
  for (int A = 0; A < na; ++A) {
    const double ax = px - __ldg(xyz + 3 * A), ay = py - __ldg(xyz + 3 * A + 1), az = pz - __ldg(xyz + 3 * A + 2);
    const double dA = sqrt(ax * ax + ay * ay + az * az);
    double P = 1.0;
    for (int B = 0; B < na && P != 0.0; ++B) {
      if (B == A) continue;
      const double bx = px - __ldg(xyz + 3 * B), by = py - __ldg(xyz + 3 * B + 1), bz = pz - __ldg(xyz + 3 * B + 2);
      double mu = (dA - sqrt(bx * bx + by * by + bz * bz)) * __ldg(invab + A * na + B);
      mu = 1.5 * mu - 0.5 * mu * mu * mu;
      mu = 1.5 * mu - 0.5 * mu * mu * mu;
      mu = 1.5 * mu - 0.5 * mu * mu * mu;
      P *= 0.5 * (1.0 - mu);
    }
    sumP += P;
    if (A == a) Pown = P;
  }
  w[g] = wr * wa * (sumP > 0.0 ? Pown / sumP : 0.0);
}

// bounding sphere (centre, radius) of every block
__global__ void __launch_bounds__(kBP) k_xc_bsph(const int* __restrict__ perm, const double* __restrict__ pts,
                                                 XcSphere* __restrict__ bsph) {
  __shared__ double red[kWarps][4];
  const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, wp = t >> 5;
  const int g = perm[(int64_t)b * kBP + t];
  double x = 0.0, y = 0.0, z = 0.0, c = 0.0;
  if (g >= 0) {
    x = pts[3 * (int64_t)g];
    y = pts[3 * (int64_t)g + 1];
    z = pts[3 * (int64_t)g + 2];
    c = 1.0;
  }
  double sx = warp_sum(x), sy = warp_sum(y), sz = warp_sum(z), sc = warp_sum(c);
  if (lane == 0) { red[wp][0] = sx; red[wp][1] = sy; red[wp][2] = sz; red[wp][3] = sc; }
  __syncthreads();
  double n = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
#pragma unroll
  for (int x = 0; x < kWarps; ++x) {
    n += red[x][3];
    cx += red[x][0];
    cy += red[x][1];
    cz += red[x][2];
  }
  cx /= n;
  cy /= n;
  cz /= n;
  __syncthreads();
  double d = g >= 0 ? sqrt((x - cx) * (x - cx) + (y - cy) * (y - cy) + (z - cz) * (z - cz)) : 0.0;
  d = warp_max(d);
  if (lane == 0) red[wp][0] = d;
  __syncthreads();
  if (t == 0) {
    double rmax = 0.0;
#pragma unroll
    for (int x = 0; x < kWarps; ++x) rmax = fmax(rmax, red[x][0]);
    bsph[b] = XcSphere{cx, cy, cz, rmax};
  }
}

// extent of every shell: largest r (step 0.02 bohr, up to 80) where
// sum_k |c_k| f_max (r^l + l r^(l-1) + 2 a_k r^(l+1)) exp(-a_k r^2) >= kAoEps,
// a bound on every component and its gradient; a shell above the bound at
// 80 bohr (exponents below about 0.005) gets an unlimited extent
__global__ void k_xc_extent(int nshell, const int* __restrict__ sh_l, const int* __restrict__ sh_np,
                            const int* __restrict__ sh_po, const int* __restrict__ sh_ao,
                            const double* __restrict__ ex, const double* __restrict__ cn, const double* __restrict__ f,
                            double* __restrict__ ext) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nshell) return;
  const int L = sh_l[s], np = sh_np[s], o = sh_po[s];
  double fm = 0.0;
  for (int k = 0; k < ncart(L); ++k) fm = fmax(fm, f[sh_ao[s] + k]);
  double e = 0.0;
  for (int st = 4000; st >= 0; --st) {
    const double r = 0.02 * st;
    double b = 0.0;
    for (int k = 0; k < np; ++k) {
      const double a = ex[o + k];
      double rl = 1.0;
      for (int x = 0; x < L; ++x) rl *= r;
      const double rlm = L > 0 ? (r > 0.0 ? rl / r : (L == 1 ? 1.0 : 0.0)) : 0.0;
      b += fabs(cn[o + k]) * fm * (rl + L * rlm + 2.0 * a * rl * r) * exp(-a * r * r);
    }
    if (b >= kAoEps) {
      e = st == 4000 ? 1e300 : r + 0.02;  // still significant at 80 bohr: never screened
      break;
    }
  }
  ext[s] = e;
}

// significant shells of every block (in shell order), their local function
// offsets, and the block's function list (global AO indices, ascending)
__global__ void __launch_bounds__(kBP) k_xc_sig(int nshell, int nbf, const XcSphere* __restrict__ bsph,
                                                const int* __restrict__ sh_atom, const int* __restrict__ sh_l,
                                                const int* __restrict__ sh_ao, const double* __restrict__ xyz,
                                                const double* __restrict__ ext, int* __restrict__ nsh,
                                                int* __restrict__ shl, int* __restrict__ shoff,
                                                int* __restrict__ nbfb, int* __restrict__ bfl) {
  __shared__ int wcnt[kWarps];
  __shared__ int base;
  const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, wp = t >> 5;
  const XcSphere sp = bsph[b];
  int* myshl = shl + (int64_t)b * nshell;
  int* myoff = shoff + (int64_t)b * nshell;
  if (t == 0) base = 0;
  __syncthreads();
  for (int s0 = 0; s0 < nshell; s0 += kBP) {
    const int s = s0 + t;
    bool sig = false;
    if (s < nshell) {
      const int a = sh_atom[s];
      const double dx = sp.x - xyz[3 * a], dy = sp.y - xyz[3 * a + 1], dz = sp.z - xyz[3 * a + 2];
      sig = sqrt(dx * dx + dy * dy + dz * dz) - sp.r < ext[s];
    }
    const unsigned m = __ballot_sync(0xffffffffu, sig);
    if (lane == 0) wcnt[wp] = __popc(m);
    __syncthreads();
    int pre = base;
    for (int x = 0; x < wp; ++x) pre += wcnt[x];
    if (sig) myshl[pre + __popc(m & ((1u << lane) - 1u))] = s;
    __syncthreads();
    if (t == 0)
      for (int x = 0; x < kWarps; ++x) base += wcnt[x];
    __syncthreads();
  }
  const int n = base;
  if (t == 0) {
    int off = 0;
    for (int i = 0; i < n; ++i) {
      myoff[i] = off;
      off += ncart(sh_l[myshl[i]]);
    }
    nsh[b] = n;
    nbfb[b] = off;
  }
  __syncthreads();
  for (int i = t; i < n; i += kBP) {
    const int s = myshl[i], o = myoff[i], L = sh_l[s], ao = sh_ao[s];
    for (int k = 0; k < ncart(L); ++k) bfl[(int64_t)b * nbf + o + k] = ao + k;
  }
}

// phi and grad phi of a block's significant functions at its points
// (Eq. contracted_basis with the component norms)
__global__ void __launch_bounds__(kBP) k_xc_ao(int b0, const int* __restrict__ perm, const double* __restrict__ pts,
                                               const int* __restrict__ nsh, const int* __restrict__ shl,
                                               const int* __restrict__ shoff, const int* __restrict__ nbfb,
                                               int nshell, const int64_t* __restrict__ woff,
                                               const int* __restrict__ sh_atom, const int* __restrict__ sh_l,
                                               const int* __restrict__ sh_np, const int* __restrict__ sh_po,
                                               const int* __restrict__ sh_ao, const double* __restrict__ ex,
                                               const double* __restrict__ cn, const double* __restrict__ f,
                                               const double* __restrict__ xyz, double* __restrict__ work) {
  const int b = b0 + blockIdx.x, t = threadIdx.x;
  const int g = perm[(int64_t)b * kBP + t];
  const int n = nbfb[b], ns = nsh[b];
  double* W = work + woff[b];
  double px = 0.0, py = 0.0, pz = 0.0;
  if (g >= 0) {
    px = pts[3 * (int64_t)g];
    py = pts[3 * (int64_t)g + 1];
    pz = pts[3 * (int64_t)g + 2];
  }
  for (int i = 0; i < ns; ++i) {
    const int s = shl[(int64_t)b * nshell + i], o = shoff[(int64_t)b * nshell + i];
    const int L = sh_l[s], a = sh_atom[s], np = sh_np[s], po = sh_po[s], ao = sh_ao[s];
    const double d[3] = {px - xyz[3 * a], py - xyz[3 * a + 1], pz - xyz[3 * a + 2]};
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double e0 = 0.0, e1 = 0.0;  // sum c exp(-a r^2), sum c a exp(-a r^2)
    for (int k = 0; k < np; ++k) {
      const double al = ex[po + k], e = cn[po + k] * exp(-al * r2);
      e0 += e;
      e1 += al * e;
    }
    if (g < 0) e0 = e1 = 0.0;
    for (int k = 0; k < ncart(L); ++k) {
      int e[3];
      cart_xyz(L, k, e[0], e[1], e[2]);
      double pw[3], pl[3], pu[3];  // d^e, d^(e-1) (0 if e = 0), d^(e+1)
      for (int x = 0; x < 3; ++x) {
        double v = 1.0;
        for (int q = 0; q < e[x]; ++q) v *= d[x];
        pw[x] = v;
        pu[x] = v * d[x];
        double vl = 1.0;
        for (int q = 1; q < e[x]; ++q) vl *= d[x];
        pl[x] = e[x] > 0 ? e[x] * vl : 0.0;
      }
      const double fc = f[ao + k];
      const int row = o + k;
      W[(int64_t)row * kBP + t] = fc * pw[0] * pw[1] * pw[2] * e0;
      W[((int64_t)n + row) * kBP + t] = fc * (pl[0] * e0 - 2.0 * pu[0] * e1) * pw[1] * pw[2];
      W[((int64_t)2 * n + row) * kBP + t] = fc * (pl[1] * e0 - 2.0 * pu[1] * e1) * pw[0] * pw[2];
      W[((int64_t)3 * n + row) * kBP + t] = fc * (pl[2] * e0 - 2.0 * pu[2] * e1) * pw[0] * pw[1];
    }
  }
}

// Step (2): X_m = sum_n D_mn phi_n at every point of the block, then
// rho = sum_m phi_m X_m, grad rho = 2 sum_m grad phi_m X_m (D symmetric)
__global__ void __launch_bounds__(kBP) k_xc_rho(int b0, int nbf, const int* __restrict__ perm,
                                                const int* __restrict__ nbfb, const int* __restrict__ bfl,
                                                const int64_t* __restrict__ woff, const double* __restrict__ work,
                                                const double* __restrict__ D, double* __restrict__ rho,
                                                double* __restrict__ grad) {
  __shared__ double Ds[kRT][kNC];
  const int b = b0 + blockIdx.x, t = threadIdx.x;
  const int g = perm[(int64_t)b * kBP + t];
  const int n = nbfb[b];
  const int* L = bfl + (int64_t)b * nbf;
  const double* W = work + woff[b];
  double r = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
  for (int m0 = 0; m0 < n; m0 += kRT) {
    const int nr = min(kRT, n - m0);
    double acc[kRT];
#pragma unroll
    for (int i = 0; i < kRT; ++i) acc[i] = 0.0;
    for (int n0 = 0; n0 < n; n0 += kNC) {
      const int nc = min(kNC, n - n0);
      __syncthreads();
      for (int e = t; e < kRT * kNC; e += kBP) {
        const int i = e / kNC, c = e % kNC;
        Ds[i][c] = (i < nr && c < nc) ? __ldg(D + (int64_t)L[m0 + i] * nbf + L[n0 + c]) : 0.0;
      }
      __syncthreads();
      for (int c = 0; c < nc; ++c) {
        const double ph = W[(int64_t)(n0 + c) * kBP + t];
#pragma unroll
        for (int i = 0; i < kRT; ++i) acc[i] = fma(Ds[i][c], ph, acc[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < kRT; ++i) {
      if (i < nr) {
        const int row = m0 + i;
        r = fma(W[(int64_t)row * kBP + t], acc[i], r);
        gx = fma(W[((int64_t)n + row) * kBP + t], acc[i], gx);
        gy = fma(W[((int64_t)2 * n + row) * kBP + t], acc[i], gy);
        gz = fma(W[((int64_t)3 * n + row) * kBP + t], acc[i], gz);
      }
    }
  }
  if (g >= 0) {
    rho[g] = r;
    if (grad) {
      grad[3 * (int64_t)g] = 2.0 * gx;
      grad[3 * (int64_t)g + 1] = 2.0 * gy;
      grad[3 * (int64_t)g + 2] = 2.0 * gz;
    }
  }
}

// Step (3): energy density eps, v_rho = d eps/d rho, v_grad = d eps/d(grad rho)
// of closed-shell Slater exchange (kind 1) or Becke-88 exchange (kind 2,
// beta = 0.0042, on the spin density rho/2); E_xc += sum w eps
__global__ void k_xc_func(int64_t G, int kind, const double* __restrict__ w, const double* __restrict__ rho,
                          const double* __restrict__ grad, double* __restrict__ vrho, double* __restrict__ vgrad,
                          double* __restrict__ exc) {
  __shared__ double red[8];
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (g < G) {
    const double r = rho[g];
    double vr = 0.0, vg[3] = {0.0, 0.0, 0.0};
    if (r >= kRhoMin) {
      const double cx = 0.75 * cbrt(3.0 / kPi);
      if (kind == 1) {
        e = -cx * r * cbrt(r);
        vr = -4.0 / 3.0 * cx * cbrt(r);
      } else {
        const double cxs = 1.5 * cbrt(3.0 / (4.0 * kPi)), beta = 0.0042;
        const double rs = 0.5 * r, a = rs * cbrt(rs);
        const double g0 = grad[3 * g], g1 = grad[3 * g + 1], g2 = grad[3 * g + 2];
        const double x = 0.5 * sqrt(g0 * g0 + g1 * g1 + g2 * g2) / a, as = asinh(x);
        const double den = 1.0 + 6.0 * beta * x * as;
        const double F = beta * x * x / den;
        const double Fpx = (2.0 * beta * den - beta * x * (6.0 * beta * as + 6.0 * beta * x / sqrt(1.0 + x * x))) /
                           (den * den);  // F'(x) / x
        e = -2.0 * a * (cxs + F);
        vr = -4.0 / 3.0 * cbrt(rs) * (cxs + F - x * x * Fpx);
        const double sc = -Fpx / (2.0 * a);
        vg[0] = sc * g0;
        vg[1] = sc * g1;
        vg[2] = sc * g2;
      }
    }
    vrho[g] = vr;
    vgrad[3 * g] = vg[0];
    vgrad[3 * g + 1] = vg[1];
    vgrad[3 * g + 2] = vg[2];
    e *= w[g];
  }
  e = warp_sum(e);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    atomicAdd(exc, s);
  }
}

__device__ __forceinline__ int lower_bound_i(const int* __restrict__ a, int n, int v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Step (4a): Z_m(g) = w_g (v_rho,g phi_m(g) / 2 + v_grad,g . grad phi_m(g)) for
// every significant function of the block (workspace slot 4)
__global__ void __launch_bounds__(kBP) k_xc_z(int b0, const int* __restrict__ perm, const int* __restrict__ nbfb,
                                              const int64_t* __restrict__ woff, const double* __restrict__ w,
                                              const double* __restrict__ vrho, const double* __restrict__ vgrad,
                                              double* __restrict__ work) {
  const int b = b0 + blockIdx.x, t = threadIdx.x;
  const int g = perm[(int64_t)b * kBP + t];
  const int n = nbfb[b];
  double* W = work + woff[b];
  double pw = 0.0, pv = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
  if (g >= 0) {
    pw = w[g];
    pv = 0.5 * vrho[g];
    g0 = vgrad[3 * (int64_t)g];
    g1 = vgrad[3 * (int64_t)g + 1];
    g2 = vgrad[3 * (int64_t)g + 2];
  }
  for (int m = 0; m < n; ++m) {
    const double phi = W[(int64_t)m * kBP + t], dx = W[((int64_t)n + m) * kBP + t],
                 dy = W[((int64_t)2 * n + m) * kBP + t], dz = W[((int64_t)3 * n + m) * kBP + t];
    W[((int64_t)4 * n + m) * kBP + t] = pw * (pv * phi + g0 * dx + g1 * dy + g2 * dz);
  }
}

// Step (4b): tile (I, J), I >= J, of V over the blocks of this CTA's share:
// V_ij += sum_g Z_i(g) phi_j(g) + phi_i(g) Z_j(g).  Per block only the
// functions it holds take part: the block's rows inside the tile's function
// range (contiguous in its list) form an nI x nJ product (nI (nI+1)/2 on the
// diagonal), spread flat over the threads, so no lane works on an absent
// function.  Each product element is added to a shared-memory accumulator at
// its tile position; the tile goes to V with one atomic per element at the end.
__global__ void __launch_bounds__(kVThreads) k_xc_vmat(int b0, int b1, int nsplit, int nbf,
                                                       const int* __restrict__ nbfb, const int* __restrict__ bfl,
                                                       const int64_t* __restrict__ woff,
                                                       const double* __restrict__ work, double* __restrict__ V) {
  extern __shared__ double xs[];
  double* accs = xs;                          // [kVT][kVT + 1]
  double* zI = accs + kVT * (kVT + 1);        // [kVT][kVP + 1] each
  double* pI = zI + kVT * (kVP + 1);
  double* zJ = pI + kVT * (kVP + 1);
  double* pJ = zJ + kVT * (kVP + 1);
  int* posI = (int*)(pJ + kVT * (kVP + 1));   // [kVT]
  int* posJ = posI + kVT;
  const int tix = blockIdx.x;
  int I = (int)((sqrt(8.0 * tix + 1.0) - 1.0) * 0.5);
  while ((I + 1) * (I + 2) / 2 <= tix) ++I;
  while (I * (I + 1) / 2 > tix) --I;
  const int J = tix - I * (I + 1) / 2;
  const bool diag = I == J;
  const int t = threadIdx.x;
  for (int e = t; e < kVT * (kVT + 1); e += kVThreads) accs[e] = 0.0;
  const int nb = b1 - b0, per = (nb + nsplit - 1) / nsplit;
  const int bs = b0 + blockIdx.y * per, be = min(b1, bs + per);
  for (int b = bs; b < be; ++b) {
    const int n = nbfb[b];
    const int* L = bfl + (int64_t)b * nbf;
    const int iI0 = lower_bound_i(L, n, I * kVT), iI1 = lower_bound_i(L, n, I * kVT + kVT);
    const int iJ0 = diag ? iI0 : lower_bound_i(L, n, J * kVT), iJ1 = diag ? iI1 : lower_bound_i(L, n, J * kVT + kVT);
    const int nI = iI1 - iI0, nJ = iJ1 - iJ0;
    if (nI == 0 || nJ == 0) continue;  // uniform over the CTA
    const int nout = diag ? nI * (nI + 1) / 2 : nI * nJ;
    const double* W = work + woff[b];
    __syncthreads();  // the previous block's accumulator updates and positions are done
    if (t < nI) posI[t] = L[iI0 + t] - I * kVT;
    if (t < nJ) posJ[t] = L[iJ0 + t] - J * kVT;
    int rc[kVOut];  // row | col << 8 of each of this thread's outputs (-1: none)
    double acc[kVOut];
#pragma unroll
    for (int k = 0; k < kVOut; ++k) {
      const int o = t + k * kVThreads;
      acc[k] = 0.0;
      rc[k] = -1;
      if (o < nout) {
        int r, c;
        if (diag) {
          r = (int)((sqrtf(8.0f * o + 1.0f) - 1.0f) * 0.5f);
          while ((r + 1) * (r + 2) / 2 <= o) ++r;
          while (r * (r + 1) / 2 > o) --r;
          c = o - r * (r + 1) / 2;
        } else {
          r = o / nJ;
          c = o - r * nJ;
        }
        rc[k] = r | (c << 8);
      }
    }
    const double* zJs = diag ? zI : zJ;
    const double* pJs = diag ? pI : pJ;
    for (int p0 = 0; p0 < kBP; p0 += kVP) {
      __syncthreads();
      for (int e = t; e < kVT * kVP; e += kVThreads) {
        const int r = e / kVP, q = e - r * kVP, col = p0 + q;
        if (r < nI) {
          zI[r * (kVP + 1) + q] = W[((int64_t)4 * n + iI0 + r) * kBP + col];
          pI[r * (kVP + 1) + q] = W[(int64_t)(iI0 + r) * kBP + col];
        }
        if (!diag && r < nJ) {
          zJ[r * (kVP + 1) + q] = W[((int64_t)4 * n + iJ0 + r) * kBP + col];
          pJ[r * (kVP + 1) + q] = W[(int64_t)(iJ0 + r) * kBP + col];
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kVOut; ++k) {
        if (rc[k] < 0) continue;
        const int oi = (rc[k] & 255) * (kVP + 1), oj = (rc[k] >> 8) * (kVP + 1);
        double a = acc[k];
#pragma unroll
        for (int q = 0; q < kVP; ++q) a = fma(zI[oi + q], pJs[oj + q], fma(pI[oi + q], zJs[oj + q], a));
        acc[k] = a;
      }
    }
#pragma unroll
    for (int k = 0; k < kVOut; ++k)
      if (rc[k] >= 0) accs[posI[rc[k] & 255] * (kVT + 1) + posJ[rc[k] >> 8]] += acc[k];
  }
  __syncthreads();
  for (int e = t; e < kVT * kVT; e += kVThreads) {
    const int i = e / kVT, j = e - i * kVT;
    const int gi = I * kVT + i, gj = J * kVT + j;
    if (gi >= nbf || gj >= nbf || (diag && j > i)) continue;
    const double v = accs[i * (kVT + 1) + j];
    if (v == 0.0) continue;
    atomicAdd(V + (int64_t)gi * nbf + gj, v);
    if (gi != gj) atomicAdd(V + (int64_t)gj * nbf + gi, v);
  }
}

constexpr size_t kVmatSmem = sizeof(double) * (kVT * (kVT + 1) + 4 * kVT * (kVP + 1)) + sizeof(int) * 2 * kVT;

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

void eri_plan_impl::xc_release() {
  void* ptrs[] = {xc.d_pts, xc.d_w, xc.d_rad, xc.d_ang, xc.d_invab, xc.d_perm, xc.d_bsph, xc.d_ext, xc.d_nsh,
                  xc.d_shl, xc.d_shoff, xc.d_nbfb, xc.d_bfl, xc.d_woff, xc.d_work, xc.d_rho, xc.d_grad,
                  xc.d_vrho, xc.d_vgrad};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  xc = XcState{};
}

static int xc_build(eri_plan_impl* P, cudaStream_t s) {
  XcState& X = P->xc;
  const int na = P->natom, nrad = X.nrad, nth = X.ntheta, nphi = 2 * nth;
  // block table: (atom, group of nrb radial shells, one of kTP theta ranges, one
  // of kPP azimuth ranges), chunks of <= kBP points
  constexpr int kTP = 4, kPP = 8;
  const int patch = ((nth + kTP - 1) / kTP) * ((nphi + kPP - 1) / kPP);
  const int nrb = std::max(1, kBP / patch);
  std::vector<int> perm;
  perm.reserve((size_t)X.npts + kBP);
  std::vector<int> cur;
  auto flush = [&]() {
    for (size_t k = 0; k < cur.size(); k += kBP) {
      for (int t = 0; t < kBP; ++t) perm.push_back(k + t < cur.size() ? cur[k + t] : -1);
    }
    cur.clear();
  };
  for (int a = 0; a < na; ++a)
    for (int i0 = 0; i0 < nrad; i0 += nrb)
      for (int h = 0; h < kTP; ++h)
        for (int q = 0; q < kPP; ++q) {
          for (int i = i0; i < std::min(nrad, i0 + nrb); ++i)
            for (int j = h * nth / kTP; j < (h + 1) * nth / kTP; ++j)
              for (int k = q * nphi / kPP; k < (q + 1) * nphi / kPP; ++k)
                cur.push_back((int)(((int64_t)(a * nrad + i) * nth + j) * nphi + k));
          flush();
        }
  X.nblock = (int)(perm.size() / kBP);
  const int nb = X.nblock, ns = P->nshell, nbf = P->nbf;
  XCK(xalloc(&X.d_pts, 3 * (size_t)X.npts));
  XCK(xalloc(&X.d_w, (size_t)X.npts));
  XCK(xalloc(&X.d_rad, 2 * (size_t)nrad));
  XCK(xalloc(&X.d_ang, 2 * (size_t)nth));
  XCK(xalloc(&X.d_invab, (size_t)na * na));
  XCK(xalloc(&X.d_perm, perm.size()));
  XCK(xalloc(&X.d_bsph, (size_t)nb));
  XCK(xalloc(&X.d_ext, (size_t)ns));
  XCK(xalloc(&X.d_nsh, (size_t)nb));
  XCK(xalloc(&X.d_shl, (size_t)nb * ns));
  XCK(xalloc(&X.d_shoff, (size_t)nb * ns));
  XCK(xalloc(&X.d_nbfb, (size_t)nb));
  XCK(xalloc(&X.d_bfl, (size_t)nb * nbf));
  XCK(xalloc(&X.d_woff, (size_t)nb + 1));
  XCK(xalloc(&X.d_rho, (size_t)X.npts));
  XCK(xalloc(&X.d_grad, 3 * (size_t)X.npts));
  XCK(xalloc(&X.d_vrho, (size_t)X.npts));
  XCK(xalloc(&X.d_vgrad, 3 * (size_t)X.npts));
  XCK(cudaMemcpyAsync(X.d_perm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice, s));
  const int nt = std::max(nrad, nth);
  k_xc_nodes<<<(nt + 127) / 128, 128, 0, s>>>(nrad, nth, X.radius, X.d_rad, X.d_ang);
  k_xc_invab<<<(na * na + 127) / 128, 128, 0, s>>>(na, P->d_coords, X.d_invab);
  k_xc_points<<<(int)((X.npts + 127) / 128), 128, 0, s>>>(X.npts, na, nrad, nth, P->d_coords, X.d_rad, X.d_ang,
                                                           X.d_invab, X.d_pts, X.d_w);
  k_xc_bsph<<<nb, kBP, 0, s>>>(X.d_perm, X.d_pts, X.d_bsph);
  k_xc_extent<<<(ns + 63) / 64, 64, 0, s>>>(ns, P->d_sh_l, P->d_sh_np, P->d_sh_po, P->d_sh_ao, P->d_exps, P->d_cn,
                                            P->d_f, X.d_ext);
  k_xc_sig<<<nb, kBP, 0, s>>>(ns, nbf, X.d_bsph, P->d_sh_atom, P->d_sh_l, P->d_sh_ao, P->d_coords, X.d_ext,
                              X.d_nsh, X.d_shl, X.d_shoff, X.d_nbfb, X.d_bfl);
  XCK(cudaGetLastError());
  // workspace plan: per block kSlots x n_b x kBP doubles; chunks under the cap
  std::vector<int> nbfb(nb);
  XCK(cudaMemcpyAsync(nbfb.data(), X.d_nbfb, sizeof(int) * nb, cudaMemcpyDeviceToHost, s));
  XCK(cudaStreamSynchronize(s));
  const size_t cap = std::max<size_t>(X.cap_bytes / sizeof(double), (size_t)kSlots * nbf * kBP);
  std::vector<int64_t> woff(nb + 1);
  X.chunk.assign(1, 0);
  X.sum_nb = X.sum_nb2 = X.sum_nbp = X.sum_nb2p = 0.0;
  size_t used = 0, peak = 0;
  for (int b = 0; b < nb; ++b) {
    const size_t need = (size_t)kSlots * nbfb[b] * kBP;
    if (used + need > cap) {
      X.chunk.push_back(b);
      used = 0;
    }
    woff[b] = (int64_t)used;
    used += need;
    peak = std::max(peak, used);
    int np = 0;
    for (int t = 0; t < kBP; ++t) np += perm[(size_t)b * kBP + t] >= 0;
    X.sum_nb += nbfb[b];
    X.sum_nb2 += (double)nbfb[b] * nbfb[b];
    X.sum_nbp += (double)nbfb[b] * np;
    X.sum_nb2p += (double)nbfb[b] * nbfb[b] * np;
  }
  X.chunk.push_back(nb);
  woff[nb] = 0;
  X.work_doubles = std::max<size_t>(peak, 1);
  X.resident = X.chunk.size() == 2;
  XCK(xalloc(&X.d_work, X.work_doubles));
  XCK(cudaMemcpyAsync(X.d_woff, woff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, s));
  if (X.resident) {
    k_xc_ao<<<nb, kBP, 0, s>>>(0, X.d_perm, X.d_pts, X.d_nsh, X.d_shl, X.d_shoff, X.d_nbfb, ns, X.d_woff,
                               P->d_sh_atom, P->d_sh_l, P->d_sh_np, P->d_sh_po, P->d_sh_ao, P->d_exps, P->d_cn,
                               P->d_f, P->d_coords, X.d_work);
    XCK(cudaGetLastError());
  }
  X.built_serial = P->geom_serial;
  return ERI_OK;
}

// (re)build the grid after a change of coordinates
static int xc_ready(eri_plan_impl* P, cudaStream_t s) {
  if (P->xc.nrad == 0) return ERI_EINVAL;  // no grid requested
  if (P->xc.built_serial == P->geom_serial) return ERI_OK;
  // work queued on the old grid's buffers (any stream of this device) must end before they go
  XCK(cudaDeviceSynchronize());
  XcState keep;
  keep.nrad = P->xc.nrad;
  keep.ntheta = P->xc.ntheta;
  keep.radius = P->xc.radius;
  keep.cap_bytes = P->xc.cap_bytes;
  keep.npts = P->xc.npts;
  P->xc_release();
  P->xc.nrad = keep.nrad;
  P->xc.ntheta = keep.ntheta;
  P->xc.radius = keep.radius;
  P->xc.cap_bytes = keep.cap_bytes;
  P->xc.npts = keep.npts;
  const int rc = xc_build(P, s);
  if (rc != ERI_OK) {
    P->xc_release();
    return rc;
  }
  return ERI_OK;
}

static void xc_launch_ao(eri_plan_impl* P, int b0, int b1, cudaStream_t s) {
  XcState& X = P->xc;
  k_xc_ao<<<b1 - b0, kBP, 0, s>>>(b0, X.d_perm, X.d_pts, X.d_nsh, X.d_shl, X.d_shoff, X.d_nbfb, P->nshell, X.d_woff,
                                  P->d_sh_atom, P->d_sh_l, P->d_sh_np, P->d_sh_po, P->d_sh_ao, P->d_exps, P->d_cn,
                                  P->d_f, P->d_coords, X.d_work);
}

static int xc_density_impl(eri_plan_impl* P, const double* D, double* rho, double* grad, cudaStream_t s) {
  XcState& X = P->xc;
  for (size_t c = 0; c + 1 < X.chunk.size(); ++c) {
    const int b0 = X.chunk[c], b1 = X.chunk[c + 1];
    if (b1 <= b0) continue;
    if (!X.resident) xc_launch_ao(P, b0, b1, s);
    k_xc_rho<<<b1 - b0, kBP, 0, s>>>(b0, P->nbf, X.d_perm, X.d_nbfb, X.d_bfl, X.d_woff, X.d_work, D, rho, grad);
    XCK(cudaGetLastError());
  }
  return ERI_OK;
}

static int xc_matrix_impl(eri_plan_impl* P, const double* vrho, const double* vgrad, double* V, cudaStream_t s) {
  XcState& X = P->xc;
  const int nbf = P->nbf, T = (nbf + kVT - 1) / kVT, npairs = T * (T + 1) / 2;
  XCK(cudaMemsetAsync(V, 0, sizeof(double) * (size_t)nbf * nbf, s));
  XCK(cudaFuncSetAttribute(k_xc_vmat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVmatSmem));
  for (size_t c = 0; c + 1 < X.chunk.size(); ++c) {
    const int b0 = X.chunk[c], b1 = X.chunk[c + 1];
    if (b1 <= b0) continue;
    if (!X.resident) xc_launch_ao(P, b0, b1, s);
    k_xc_z<<<b1 - b0, kBP, 0, s>>>(b0, X.d_perm, X.d_nbfb, X.d_woff, X.d_w, vrho, vgrad, X.d_work);
    const int nsplit = std::max(1, std::min(b1 - b0, (24 * P->nsm + npairs - 1) / npairs));
    k_xc_vmat<<<dim3(npairs, nsplit), kVThreads, kVmatSmem, s>>>(b0, b1, nsplit, nbf, X.d_nbfb, X.d_bfl, X.d_woff,
                                                                 X.d_work, V);
    XCK(cudaGetLastError());
  }
  return ERI_OK;
}

static int xc_check_plan(eri_plan_impl* P) {
  if (!P) return ERI_EINVAL;
  if (P->nmol != 1) return ERI_EUNSUPPORTED;
  return ERI_OK;
}

extern "C" int eri_xc_grid(eri_plan_t* plan, int32_t nrad, int32_t ntheta, double radius, double cap_bytes,
                           int64_t* npoints, void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  int rc = xc_check_plan(P);
  if (rc != ERI_OK) return rc;
  if (nrad < 2 || nrad > 1000 || ntheta < 2 || ntheta > 64 || (ntheta & 1) || !(radius > 0.0) ||
      !(radius < 1e6) || !(cap_bytes >= 0.0))
    return ERI_EINVAL;
  const int64_t G = (int64_t)P->natom * nrad * ntheta * 2 * ntheta;
  if (G >= (int64_t)1 << 31) return ERI_EUNSUPPORTED;  // point indices are int32
  cudaStream_t s = (cudaStream_t)stream;
  XCK(cudaSetDevice(P->device));
  XCK(cudaDeviceSynchronize());  // the old grid's buffers may still be read by queued work on any stream
  P->xc_release();
  P->xc.nrad = nrad;
  P->xc.ntheta = ntheta;
  P->xc.radius = radius;
  P->xc.cap_bytes = cap_bytes > 0.0 ? (size_t)std::min(cap_bytes, 1e18) : kDefaultCap;
  P->xc.npts = G;
  P->xc.built_serial = -1;
  rc = xc_ready(P, s);
  if (rc != ERI_OK) {
    P->xc_release();
    return rc;
  }
  if (npoints) *npoints = G;
  return ERI_OK;
}

extern "C" int eri_xc_get_grid(eri_plan_t* plan, double* points, double* weights, void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  int rc = xc_check_plan(P);
  if (rc != ERI_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  XCK(cudaSetDevice(P->device));
  rc = xc_ready(P, s);
  if (rc != ERI_OK) return rc;
  if (points)
    XCK(cudaMemcpyAsync(points, P->xc.d_pts, sizeof(double) * 3 * P->xc.npts, cudaMemcpyDeviceToDevice, s));
  if (weights)
    XCK(cudaMemcpyAsync(weights, P->xc.d_w, sizeof(double) * P->xc.npts, cudaMemcpyDeviceToDevice, s));
  return ERI_OK;
}

extern "C" int eri_xc_density(eri_plan_t* plan, const double* D, double* rho, double* grad_rho, void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  int rc = xc_check_plan(P);
  if (rc != ERI_OK) return rc;
  if (!D || !rho) return ERI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  XCK(cudaSetDevice(P->device));
  rc = xc_ready(P, s);
  if (rc != ERI_OK) return rc;
  return xc_density_impl(P, D, rho, grad_rho, s);
}

extern "C" int eri_xc_matrix(eri_plan_t* plan, const double* vrho, const double* vgrad, double* V, void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  int rc = xc_check_plan(P);
  if (rc != ERI_OK) return rc;
  if (!vrho || !vgrad || !V) return ERI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  XCK(cudaSetDevice(P->device));
  rc = xc_ready(P, s);
  if (rc != ERI_OK) return rc;
  return xc_matrix_impl(P, vrho, vgrad, V, s);
}

extern "C" int eri_xc(eri_plan_t* plan, const double* D, int32_t functional, double* V, double* Exc, void* stream) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  int rc = xc_check_plan(P);
  if (rc != ERI_OK) return rc;
  if (!D || !V || !Exc || (functional != ERI_XC_SLATER && functional != ERI_XC_B88)) return ERI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  XCK(cudaSetDevice(P->device));
  rc = xc_ready(P, s);
  if (rc != ERI_OK) return rc;
  XcState& X = P->xc;
  rc = xc_density_impl(P, D, X.d_rho, X.d_grad, s);
  if (rc != ERI_OK) return rc;
  XCK(cudaMemsetAsync(Exc, 0, sizeof(double), s));
  k_xc_func<<<(int)((X.npts + 255) / 256), 256, 0, s>>>(X.npts, functional, X.d_w, X.d_rho, X.d_grad, X.d_vrho,
                                                         X.d_vgrad, Exc);
  XCK(cudaGetLastError());
  return xc_matrix_impl(P, X.d_vrho, X.d_vgrad, V, s);
}

extern "C" int eri_xc_stats(eri_plan_t* plan, eri_xc_stats_t* st) {
  eri_plan_impl* P = reinterpret_cast<eri_plan_impl*>(plan);
  int rc = xc_check_plan(P);
  if (rc != ERI_OK) return rc;
  if (!st) return ERI_EINVAL;
  const XcState& X = P->xc;
  std::memset(st, 0, sizeof(*st));
  st->npoints = X.npts;
  st->nblock = X.nblock;
  st->block_points = kBP;
  st->sum_block_functions = X.sum_nb;
  st->sum_block_functions_sq = X.sum_nb2;
  st->workspace_bytes = (double)X.work_doubles * sizeof(double);
  st->resident = X.resident;
  st->nchunk = X.chunk.empty() ? 0 : (int32_t)X.chunk.size() - 1;
  // density X = D_b Phi_b (2 n_b^2 per point) and the rho / grad rho
  // epilogue (8 n_b); matrix Z_b Phi_b^T + Phi_b Z_b^T on the lower triangle
  // (2 n_b^2 per point) and Z (8 n_b); FMA = 2 FLOP
  st->flops_density = 2.0 * X.sum_nb2p + 8.0 * X.sum_nbp;
  st->flops_matrix = 2.0 * X.sum_nb2p + 8.0 * X.sum_nbp;
  return ERI_OK;
}
