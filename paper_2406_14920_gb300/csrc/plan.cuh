// Internal plan state behind the opaque eri_plan_t of include/eri.h.
#pragma once
#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include "common.cuh"
#include "../../include/eri.h"
#include "xc_state.cuh"

struct eri_plan_impl {
  eri_opts_t opts;
  int device = 0, nsm = 1;
  int nshell = 0, natom = 0, nbf = 0, npair = 0, nprimpair = 0, nsig = 0;
  // molecules: a plan holds nmol independent molecules; pairs never cross
  // molecules and D / J / K are packed one nbf_m x nbf_m block per molecule
  int nmol = 1, max_nbf = 0;
  int64_t nmat = 0;  // packed matrix elements, sum nbf_m^2
  std::vector<int64_t> h_mat_off;  // [nmol + 1]
  std::vector<int> h_mat_n, h_aobase, h_atombase, h_pairbase;  // h_aobase / h_atombase / h_pairbase: [nmol + 1]
  std::vector<int> h_ccm;          // significant pairs per (molecule, class)
  std::vector<int> h_segloc;       // offset of (molecule, class) segment inside the class list
  int64_t* d_mat_off = nullptr;
  int *d_mat_n = nullptr, *d_aobase = nullptr, *d_pbase = nullptr, *d_pmol = nullptr, *d_shloc = nullptr;
  int *d_ccm = nullptr, *d_segloc = nullptr;
  int64_t nherm_tot = 0;
  double thresh = 1e-12;
  double omega = 0.0;  // two-electron operator: 0 = 1/r, > 0 = erf(omega r)/r (eri_plan_set_omega)
  // shells
  int *d_sh_l = nullptr, *d_sh_atom = nullptr, *d_sh_np = nullptr, *d_sh_po = nullptr, *d_sh_ao = nullptr;
  double *d_exps = nullptr, *d_coefs = nullptr, *d_cn = nullptr, *d_f = nullptr, *d_coords = nullptr;
  // shell pairs (pair-index order)
  int *d_ps1 = nullptr, *d_ps2 = nullptr, *d_pnp = nullptr, *d_ppoff = nullptr, *d_pao1 = nullptr, *d_pao2 = nullptr;
  int *d_phoff = nullptr, *d_pcls = nullptr;
  // primitive pairs
  double *d_p = nullptr, *d_P = nullptr, *d_PA = nullptr, *d_PB = nullptr, *d_pref = nullptr;
  float *d_pf = nullptr, *d_Pf = nullptr, *d_PAf = nullptr, *d_PBf = nullptr, *d_preff = nullptr;
  float4* d_q4 = nullptr;  // packed FP32 shadows, 3 float4 per primitive pair (PairData::q4)
  // screening and lists
  float* d_Q = nullptr;
  unsigned int* d_qmax = nullptr;
  int *d_sig = nullptr, *d_ccount = nullptr, *d_coff = nullptr, *d_sorted = nullptr, *d_pos = nullptr,
      *d_counts = nullptr;
  int64_t *d_koff = nullptr, *d_joff = nullptr, *d_kpre = nullptr, *d_jpre = nullptr, *d_ktot = nullptr,
          *d_jtot = nullptr, *d_kprim = nullptr;
  int64_t kpre_cap = 0, jpre_cap = 0;
  int64_t* d_cumnp = nullptr;
  int h_ccount[eri::NPAIRCLASS] = {}, h_coff[eri::NPAIRCLASS] = {};
  int64_t h_koff[eri::NPAIRCLASS * eri::NPAIRCLASS] = {}, h_joff[eri::NPAIRCLASS * eri::NPAIRCLASS] = {};
  int64_t h_ktot[eri::NPAIRCLASS * eri::NPAIRCLASS] = {}, h_jtot[eri::NPAIRCLASS * eri::NPAIRCLASS] = {};
  int64_t h_kprim[eri::NPAIRCLASS * eri::NPAIRCLASS] = {};
  // tables
  double *d_boys64 = nullptr, *d_bexp64 = nullptr;
  float *d_boys32 = nullptr, *d_bexp32 = nullptr;
  int* d_peoff = nullptr;
  double* d_E = nullptr;
  float* d_Ef = nullptr;
  eri::RStep* d_rsteps = nullptr;
  // per-build workspace
  float* d_Dpf = nullptr;  // D' in FP32 for the FP32 tier
  double *d_Dp = nullptr, *d_Kh = nullptr, *d_Jh = nullptr, *d_Dherm = nullptr, *d_Jherm = nullptr;
  float* d_Dhermf = nullptr;  // Hermite density in FP32 (FP32 tier of a mixed J-engine build)
  int* d_status = nullptr;
  float *d_pmaxp = nullptr, *d_dmax = nullptr, *d_prefmaxp = nullptr;
  double* d_ea = nullptr;
  unsigned long long* d_counters = nullptr;  // [X*10+Y][tier][items, prim quartets, bra primitives]
  unsigned long long* d_counters2 = nullptr; // [kind][X*10+Y][same]; kinds: J-engine FP64, gradient FP64, gradient FP32, J-engine FP32
  bool last_mixed = false, last_do_j = false, last_do_k = false, last_jmixed = false;
  // optional per-launch profiling (opts.profile): events recorded around each class launch
  struct ProfRec { int X, Y, tier, ev; };
  std::vector<cudaEvent_t> prof_events;
  std::vector<ProfRec> prof_log;
  int prof_builds = 0, prof_ev_used = 0;
  cudaError_t prof_event_pair(cudaEvent_t* a, cudaEvent_t* b);

  // CUDA graph of one build (eri_build_jk_graph): captured on cap_stream, with
  // the class launches forked onto kBranches side streams so that independent
  // classes overlap (their tails, and small launches, fill idle SMs)
  static constexpr int kBranches = 4;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t branch[kBranches] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kBranches] = {};
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[3] = {};
  int gprec = -1;
  int gbranches = 0;  // branches of the kept graph (1: serial chain, kBranches: forked)
  int ensure_streams();
  // compacted tier lists of mixed builds (per branch), see ensure_tier_bufs
  int2* tbuf[kBranches] = {};
  unsigned int* tcnt = nullptr;
  int64_t tier_cap = 0;
  int tier_nb = 0;
  int ensure_tier_bufs(int nb);
  // work-tile length (items per worker tile) per (bra class, ket class, tier),
  // set by eri_autotune or eri_set_tiles; 0 = the built-in default
  int tile_k[eri::NPAIRCLASS * eri::NPAIRCLASS * 2] = {};
  std::string tune_cache;  // opts.tune_cache (copied): tile tables stored per device, plan shape and precision
  int tile_for(int X, int Y, int tier) const;
  // share of the work this plan computes (eri_plan_set_shard): tiles t of every
  // class launch with t % nshard == shard; results are this share's partial sums
  int shard = 0, nshard = 1;

  // point-charge attraction (nuclear.cu): primitive pairs of every shell pair
  // grouped by l1 + l2 (entries {prim pair, Hermite offset, density offset,
  // shell pair}), built at the first call; per-pair offsets and buffer of the
  // Hermite densities the gradient contracts
  int4* d_nuc_list = nullptr;
  int nuc_cnt[2 * eri::LMAX + 1] = {}, nuc_first[2 * eri::LMAX + 2] = {};
  int* d_nuc_goff = nullptr;
  double* d_nuc_dens = nullptr;
  int nuc_built = 0;

  // exchange-correlation grid (xc.cu); geom_serial counts coordinate changes
  // so the grid is rebuilt after one
  XcState xc;
  int geom_serial = 0;
  void xc_release();

  int alloc_pairs();
  int geometry(cudaStream_t s, bool rebuild_q);
  int build_lists(double th, cudaStream_t s);
  eri::PairData pairdata() const;
  eri::BoysTabs boystabs() const;
  eri::ShellPairInfo spinfo() const;
  eri::WorkList klist(int X, int Y) const;
  eri::WorkList jlist(int X, int Y) const;
  dim3 mat_grid(int block) const;
  void release();
};

// packed per-molecule matrices: molecule m's nbf_m x nbf_m block at off[m], AO offset aobase[m]
struct MolMats {
  const int64_t* off;
  const int* n;
  const int* aobase;
};
MolMats molmats(const eri_plan_impl* P);
void k_scale_d_launch(const eri_plan_impl* P, const double* D, cudaStream_t s);  // D' = D f f into P->d_Dp

// runtime-l E^{ij}_t (Eq. E_recursion), E[(i*5+j)*9+t], i,j <= 4
__device__ __forceinline__ void md_e_rt(int li, int lj, double PA, double PB, double o2p, double* E) {
  for (int x = 0; x < 225; ++x) E[x] = 0.0;
  E[0] = 1.0;
  for (int i = 0; i < li; ++i)
    for (int t = 0; t <= i + 1; ++t) {
      double v = PA * E[(i * 5) * 9 + t];
      if (t > 0) v += o2p * E[(i * 5) * 9 + t - 1];
      if (t + 1 <= i) v += (t + 1) * E[(i * 5) * 9 + t + 1];
      E[((i + 1) * 5) * 9 + t] = v;
    }
  for (int i = 0; i <= li; ++i)
    for (int j = 0; j < lj; ++j)
      for (int t = 0; t <= i + j + 1; ++t) {
        double v = PB * E[(i * 5 + j) * 9 + t];
        if (t > 0) v += o2p * E[(i * 5 + j) * 9 + t - 1];
        if (t + 1 <= i + j) v += (t + 1) * E[(i * 5 + j) * 9 + t + 1];
        E[(i * 5 + j + 1) * 9 + t] = v;
      }
}

// Cartesian J from Hermite J per primitive pair (plan.cu); sig == nullptr takes every pair
__global__ void k_post_j(int npair, const int* __restrict__ s1, const int* __restrict__ s2, const int* __restrict__ np,
                         const int* __restrict__ poff, const int* __restrict__ hoff, const int* __restrict__ sh_l,
                         const int* __restrict__ pao1, const int* __restrict__ pao2, const int* __restrict__ pmol,
                         MolMats mm, const int* __restrict__ sig, eri::PairData pd, const double* __restrict__ Jh,
                         const double* __restrict__ f, double* __restrict__ J, int det, int* __restrict__ status);
