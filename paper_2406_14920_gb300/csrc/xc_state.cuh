// Exchange-correlation state of a plan (xc.cu), kept apart from plan.cuh so
// that the J/K kernels and their launch code do not depend on it.
#pragma once
#include <cstdint>
#include <vector>

// exchange-correlation grid of a plan (xc.cu): points and weights in natural
// order, blocks of at most 32 points (perm: natural index of each block slot,
// -1 for padding), per-block bounding spheres, significant shells and
// functions, and the workspace of basis values (resident when it fits the cap)
struct alignas(32) XcSphere {
  double x, y, z, r;  // centre and radius
};
struct XcState {
  int nrad = 0, ntheta = 0, nblock = 0, built_serial = -1, resident = 0;
  double radius = 1.0;
  size_t cap_bytes = 0;
  int64_t npts = 0;
  double *d_pts = nullptr, *d_w = nullptr, *d_rad = nullptr, *d_ang = nullptr, *d_invab = nullptr;
  int* d_perm = nullptr;
  XcSphere* d_bsph = nullptr;
  double* d_ext = nullptr;
  int *d_nsh = nullptr, *d_shl = nullptr, *d_shoff = nullptr, *d_nbfb = nullptr, *d_bfl = nullptr;
  int64_t* d_woff = nullptr;
  double* d_work = nullptr;
  size_t work_doubles = 0;
  std::vector<int> chunk;  // block boundaries of the workspace chunks
  double *d_rho = nullptr, *d_grad = nullptr, *d_vrho = nullptr, *d_vgrad = nullptr;
  double sum_nb = 0.0, sum_nb2 = 0.0;  // sum over blocks of n_b and n_b^2 (significant functions)
  double sum_nbp = 0.0, sum_nb2p = 0.0;  // the same weighted by each block's number of points
};
