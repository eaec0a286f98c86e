/*
 * eri.h -- C ABI of the GB300 integral-direct Coulomb/exchange library.
 *
 * The operations follow Wang et al., "Extending GPU-Accelerated Gaussian
 * Integrals in the TeraChem Software Package to f Type Orbitals":
 *   basis functions      Sec. 2.1, Eq. contracted_basis, Eq. primtive_basis
 *   ERIs                 Sec. 2.5, Eq. eri_definition, Eq. eri_formula
 *   long-range ERIs      Sec. 2.5, Eq. eri_longrange_definition, Eq. eri_longrange_formula
 *   point charges        Sec. 2.4, Eq. v1e_definition, Eq. v1e_formula; SI Sec. 1.3
 *   J and K              Eq. j_definition (J_mn = sum_ls (mn|ls) D_ls),
 *                        Eq. k_definition (K_ml = sum_ns (mn|ls) D_ns)
 *   screening            Eq. cauchy_schwarz_bound, Eq. kernel_upperbound
 *   energies, gradient   SI Eq. si_E_J_K, SI Eq. si_dE_J, SI Eq. si_dE_K
 *
 * Conventions (all calls):
 *   - units bohr / hartree; all floating-point arguments are FP64;
 *   - matrices are nbf x nbf, row-major, AO order = user shell order, and
 *     inside a shell the Cartesian components are lexicographic
 *     (xx,xy,xz,yy,yz,zz; xxx,xxy,xxz,xyy,xyz,xzz,yyy,yyz,yzz,zzz);
 *   - every function is normalised: each primitive component gets
 *     (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2i-1)!!(2j-1)!!(2k-1)!!) and each
 *     shell's coefficients are rescaled once so the contracted (l,0,0)
 *     function has unit norm (the paper leaves the convention open, Sec. 2.1);
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *     every call that takes a stream is ordered on it and returns before the
 *     GPU work finishes, unless stated otherwise;
 *   - D, J, K, dEdR and E pointers are DEVICE pointers on the plan's device,
 *     owned by the caller; outputs are overwritten, not accumulated;
 *   - D must be symmetric (8-fold symmetry, Eq. 8_fold_symmetry);
 *   - return value 0 on success, else a negative ERI_E* code; no call aborts
 *     the process.  eri_strerror() describes a code.
 *   - a plan must not be used from two streams at the same time.
 */
#ifndef GB300_ERI_H
#define GB300_ERI_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ERI_OK 0
#define ERI_EINVAL (-1)       /* bad argument: NULL, l > 3, nprim <= 0, exponent <= 0, NaN ... */
#define ERI_ENOMEM (-2)       /* device or host allocation failed */
#define ERI_ECUDA (-3)        /* a CUDA runtime call failed */
#define ERI_EUNSUPPORTED (-4) /* valid request this build cannot serve */
#define ERI_ETIMEOUT (-5)     /* reserved: a bounded device wait gave up (no kernel of this build waits on another) */
#define ERI_EDEVICE (-6)      /* a device-side check failed (status word set) */

#define ERI_FP64 0  /* every quartet in FP64 */
#define ERI_MIXED 1 /* quartets with bound below mixed_tau in FP32, the rest FP64 */

typedef struct eri_plan eri_plan_t;

typedef struct {
  int32_t atom;        /* index into coords */
  int32_t l;           /* 0..3 (s, p, d, f), Cartesian */
  int32_t nprim;       /* >= 1 */
  int32_t prim_offset; /* first primitive in exps / coefs */
} eri_shell_t;

typedef struct {
  int32_t nshell, natom;
  const eri_shell_t* shells; /* host, nshell entries, user order */
  const double* exps;        /* host, exponents (> 0) */
  const double* coefs;       /* host, raw contraction coefficients */
} eri_basis_t;

typedef struct {
  double thresh;      /* Schwarz quartet threshold THRECL (Eq. kernel_upperbound); default 1e-12 */
  int32_t precision;  /* ERI_FP64 (default) or ERI_MIXED */
  double mixed_tau;   /* FP64 tier: Q_ab Q_cd max|D| >= mixed_tau; default 1e-5 (paper Sec. 4.1) */
  int32_t device;     /* CUDA device ordinal; default: current device */
  int32_t j_engine;   /* J-only builds (K == NULL): 1 = Hermite J-engine of Eq. j_formula
                         (default), 0 = contraction of Cartesian ERIs */
  int32_t profile;    /* 1: record CUDA events around every class launch (see eri_get_profile) */
  const char* tune_cache; /* NULL, or a text file of autotuned tile tables: eri_plan loads the entry for
                             this device, plan shape (nbf, molecules, shell pairs) and opts.precision if
                             the file holds one, and eri_autotune stores its result there (replacing
                             the entry of the same key).  The path is copied. */
  int32_t deterministic;  /* 1: J/K builds (also the J-engine, graph and allocation-free builds) and
                             eri_jk_grad accumulate in 64-bit fixed point (scale 2^46, resolution
                             1.4e-14) with integer atomics, which are order-independent: repeated calls
                             give bit-identical results.  Accumulated magnitudes must stay below 2^17;
                             an element above 2^16 sets the device status (see eri_check).  0 (default):
                             FP64 atomics, results equal to rounding only. */
  int32_t density_screen; /* 1: J+K and K builds also drop every quartet whose density-weighted bound
                             Q_ab Q_cd max|D'| (float32; max over the six D' blocks the quartet
                             touches, D' = D with component norms) is below the threshold
                             (Eq. kernel_upperbound with the density factor; a device pass
                             compacts the kept quartets per build).  J-only J-engine builds and
                             gradients are not screened.  0 (default): lists only (Q_ab Q_cd). */
} eri_opts_t;

typedef struct {
  int32_t nbf, nshell, npair, nsig_pair;
  int64_t quartets_k;      /* canonical significant shell quartets (unique, 8-fold) */
  int64_t quartets_j;      /* ordered significant (bra, ket) shell-pair pairs of the J-engine */
  int64_t prim_quartets_k; /* primitive quartets behind quartets_k */
  int64_t quartets_k_fp32; /* of quartets_k, evaluated in FP32 by the last mixed build */
  double flops_k, flops_j; /* algorithmic FLOPs of the last build (McMurchie-Davidson count) */
  int32_t device_status;   /* device-side status word (0 = ok) */
  int64_t quartets_k_guard; /* of quartets_k, kept in FP64 by the last mixed build's FP32 range guard
                               alone (their bound was below mixed_tau, but an exponent sum above 1e3
                               or a primitive prefactor product above 1e18 would overflow FP32) */
  int64_t quartets_k_screened; /* of quartets_k, dropped by the density screen in the last build */
  int32_t graph_branches;       /* branches of the current graph build (1 serial, 4 forked; 0: none) */
  int64_t quartets_j_fp32;      /* of quartets_j, evaluated in FP32 by the last J-engine build (mixed) */
} eri_stats_t;

/* Fill opts with the defaults listed above.  Host only. */
int eri_default_opts(eri_opts_t* opts);

/*
 * Build a plan: copies the basis and coordinates (host, natom*3 doubles) to
 * the device, normalises the basis, forms every shell pair's primitive-pair
 * data, the Schwarz bounds Q_ab (Eq. cauchy_schwarz_bound, float32 rounded
 * up) and the class-sorted significant pair and quartet lists for
 * opts->thresh.  Synchronises the device.  *out owns all device memory it
 * allocates until eri_plan_destroy.  opts may be NULL (defaults).
 * Errors: ERI_EINVAL (bad basis or coords), ERI_ENOMEM, ERI_ECUDA.
 */
int eri_plan(const eri_basis_t* basis, const double* coords, const eri_opts_t* opts, eri_plan_t** out);

/*
 * One plan over nmol independent molecules (bases[m], coords[m]: host, as for
 * eri_plan), so that one eri_build_jk / eri_jk_grad covers all of them: each
 * class launch walks the quartets of every molecule (the paper's batch of many
 * systems, processed together).  Shell pairs and quartets never mix molecules;
 * thresholds apply per molecule (Q_max is each molecule's own), so molecule m
 * gets exactly the lists a single-molecule plan of it would get.
 * Packed layout of every matrix argument of the other calls (D, J, K): molecule
 * m's nbf_m x nbf_m row-major block starts at element mat_off[m]
 * (eri_plan_layout); dEdR and coordinates are natom_m x 3 per molecule, molecule
 * after molecule (atom_off).  eri_energy writes 2 doubles per molecule.
 * nmol in 1..65535; eri_plan(b, c, o, out) equals eri_plan_batch(1, &b, &c, o, out).
 * Errors as for eri_plan.
 */
int eri_plan_batch(int32_t nmol, const eri_basis_t* const* bases, const double* const* coords,
                   const eri_opts_t* opts, eri_plan_t** out);

/*
 * Layout of a plan's packed matrices (host outputs, each may be NULL):
 *   *nmol; mat_off int64 [nmol+1] (element offsets, mat_off[nmol] = total);
 *   nbf int32 [nmol]; atom_off int32 [nmol+1] (first atom of each molecule).
 * Call once with only nmol to size the arrays.
 */
int eri_plan_layout(eri_plan_t* plan, int32_t* nmol, int64_t* mat_off, int32_t* nbf, int32_t* atom_off);

/*
 * Move the atoms: coords_dev is a DEVICE pointer to natom*3 doubles.  Pair
 * data, Schwarz bounds and lists are rebuilt on `stream`, then the call waits
 * for the new list sizes (a device->host copy).  Use for finite differences
 * and for autograd.  If freeze_lists != 0 the lists and Q of the previous
 * geometry are kept (so energies are smooth functions of the coordinates).
 */
int eri_plan_set_coords(eri_plan_t* plan, const double* coords_dev, int32_t freeze_lists, void* stream);

/*
 * J_mn = sum_ls (mn|ls) D_ls and K_ml = sum_ns (mn|ls) D_ns over the quartets
 * whose Schwarz bound Q_ab Q_cd >= thresh (Eq. j_definition, Eq. k_definition,
 * Eq. kernel_upperbound).  D, J, K: device, nbf*nbf (packed per molecule for
 * a batched plan).  D must be symmetric.  J or K may be NULL to
 * skip that matrix (J alone runs only the J-engine, Eq. j_formula, unless
 * opts.j_engine = 0; with ERI_MIXED its ordered (bra, ket) items are split by
 * the same tier test and the FP32 tier reads an FP32 copy of the Hermite
 * density, both tiers adding into the FP64 Hermite J).  thresh < 0 keeps the
 * plan's threshold; another value rebuilds the lists first (with a host wait).
 * precision: ERI_FP64 or ERI_MIXED (tier split at the plan's mixed_tau: a device
 * pass writes each class pair's FP64-tier and FP32-tier quartets to two compacted
 * lists, then each tier runs over its own list; the plan holds these lists, up
 * to 2^23 quartets per tier, allocated by the first mixed build or graph capture).
 * With thresh < 0 and opts.profile = 0 the call only enqueues work on
 * `stream` (no host wait, no allocation), so it may be captured into a CUDA graph.
 */
int eri_build_jk(eri_plan_t* plan, const double* D, double* J, double* K, double thresh, int32_t precision,
                 void* stream);

/*
 * The same build as eri_build_jk(plan, D, J, K, -1, precision, stream), run as
 * one CUDA graph: the first call for a given (D, J, K, precision) captures the
 * whole build (density scaling, every class launch of every molecule, the
 * symmetrisation) on a stream of the plan and instantiates it; later calls with
 * the same pointers replay it with one cudaGraphLaunch on `stream` (the contents
 * of D may change between calls).  The first call captures two graphs, one with
 * the class launches in a serial chain and one with them forked onto four
 * branches (least-loaded first, so independent classes overlap), replays each
 * twice (host waits) and keeps the faster one.  New pointers or
 * precision re-capture (the old graph is released after a wait on `stream`);
 * a list rebuild (another threshold, new coordinates without frozen lists)
 * drops the graph.  Profiling (opts.profile) does not apply to graph builds.
 * Errors: as eri_build_jk; a failed capture returns ERI_ECUDA and leaves no graph.
 */
int eri_build_jk_graph(eri_plan_t* plan, const double* D, double* J, double* K, int32_t precision, void* stream);

/*
 * Autotuner for the work-tile length (consecutive shell quartets a warp, or for
 * the thread kernel each lane, takes before moving on; the walk steps a cursor
 * through the bra prefix array instead of searching it per quartet).  For every
 * (bra class, ket class, tier) launch of this plan and density, candidate
 * lengths (1, 2, 4, 8, and 16, 32 for warp kernels) are timed with CUDA events on
 * three windows of the launch's own list (mixed precision: of the tier's
 * compacted list), the windows sized so the current length takes about trial_ms
 * and every resident warp gets several tiles; a length replaces the default
 * only if it is more than 5 % faster twice.  Synchronises `stream` repeatedly; writes only plan scratch; J and
 * K are unchanged.  Later builds (and graphs captured after it) use the tiles.  With opts.tune_cache set,
 * the result is stored in that file under this plan's key and precision.
 * Errors: ERI_EINVAL (trial_ms <= 0, NULL, bad precision, tune_cache not writable), ERI_ECUDA.
 */
int eri_autotune(eri_plan_t* plan, const double* D, int32_t precision, double trial_ms, void* stream);

/*
 * Split the work over nshard GPUs (one plan per GPU, same basis and geometry):
 * from now on this plan's builds (eri_build_jk, eri_build_jk_graph and the
 * J-engine) and gradients take only the work tiles t of every class launch with
 * t % nshard == shard, and return the PARTIAL J, K or dE/dR of that share.  The
 * shares of shard = 0..nshard-1 cover every quartet exactly once, so a sum
 * all-reduce of the partial J / K / dEdR over the GPUs gives the full result
 * (the exchange step; the library does not communicate).  Tiles are a few
 * quartets long and interleaved, so each share gets an even mix of classes,
 * screening magnitudes and precision tiers.  A tile is `tile` consecutive items
 * of the class-pair list for the warp kernels and 32 x tile for the thread
 * kernel (eri_get_tiles); in a mixed-precision build it is 32 items, taken by
 * the tier split that compacts each tier's quartets.  (0, 1) restores the
 * whole build.
 * Errors: ERI_EINVAL (nshard < 1 or shard outside 0..nshard-1).
 */
int eri_plan_set_shard(eri_plan_t* plan, int32_t shard, int32_t nshard);

/*
 * Two-electron operator of this plan's later builds (eri_build_jk, the graph
 * build, the J-engine, eri_build_jk_noalloc) and gradients (eri_jk_grad):
 * omega = 0 (the default) is the Coulomb operator 1/r, omega > 0 the
 * long-range operator erf(omega r)/r of range-separated functionals (Sec. 2.5,
 * Eq. eri_longrange_definition).  Its ERIs follow Eq. eri_longrange_formula:
 * the same McMurchie-Davidson chain with rho -> s rho and the prefactor times
 * sqrt(s), s = omega^2 / (omega^2 + rho).  The Schwarz bounds, lists and the
 * mixed-precision tier test stay those of 1/r (a valid upper bound:
 * erfc(omega r)/r is positive definite, so (ab|erf|ab) <= (ab|ab)).  Host
 * only; a captured graph build is dropped when omega changes (after a device
 * wait).  Errors: ERI_EINVAL (NULL, omega < 0, NaN or omega >= 1e30).
 */
int eri_plan_set_omega(eri_plan_t* plan, double omega);

/*
 * Mixed-precision threshold of this plan's later ERI_MIXED builds, gradients
 * and allocation-free builds: a quartet runs in FP64 when its density-weighted
 * Schwarz bound Q_ab Q_cd max|D'| >= mixed_tau (or the FP32 range guard trips),
 * else in FP32 (Sec. 4.1).  Lowering it between builds is the dynamic-precision
 * scheme the paper cites: a loose threshold in the first SCF iterations, a
 * tighter one as the density converges.  The split is taken on the device at
 * every build, so a change costs nothing; a captured graph build is dropped when
 * the value changes (after a device wait).  Host only.
 * Errors: ERI_EINVAL (NULL, mixed_tau < 0 or NaN).
 */
int eri_plan_set_tau(eri_plan_t* plan, double mixed_tau);

/*
 * Read or set the plan's tile table (host int32 [10][10][2] indexed
 * [bra class][ket class][tier], entries with ket class > bra class unused;
 * 0 in eri_set_tiles = built-in default, valid values 0..1024).  Use them to
 * cache autotuner results across runs.
 */
int eri_get_tiles(eri_plan_t* plan, int32_t* tiles);
int eri_set_tiles(eri_plan_t* plan, const int32_t* tiles);

/*
 * E_J = 1/2 sum D_mn J_mn and E_K = -1/4 sum D_mn K_mn (SI Eq. si_E_J_K):
 * E_out is a DEVICE pointer to 2 doubles {E_J, E_K} per molecule.  J or K may be NULL
 * (its energy is written as 0).
 */
int eri_energy(eri_plan_t* plan, const double* D, const double* J, const double* K, double* E_out, void* stream);

/*
 * dE/dR for E = 1/2 tr(D J) - 1/4 tr(D K) with D held fixed (the terms in dD/dR
 * are left out, SI Eq. si_dE_J_step1): dEdR is a DEVICE pointer to natom*3
 * doubles.  Uses the bra-derivative form SI Eq. si_dE_J / si_dE_K with the
 * derivative Hermite coefficients of SI Eq. si_dE_recursion.  Lists as for
 * eri_build_jk at the plan's threshold.  want_j / want_k select the terms.
 */
int eri_jk_grad(eri_plan_t* plan, const double* D, double* dEdR, int32_t want_j, int32_t want_k, void* stream);

/*
 * eri_jk_grad with a precision: ERI_FP64 is eri_jk_grad; ERI_MIXED splits the
 * ordered items on the device with the energy's tier test (Q_ab Q_cd max|D'|
 * below the plan's mixed_tau and the FP32 range guard passed: FP32, else FP64)
 * and evaluates the FP32 tier's derivative integrals and their contraction
 * with D in FP32, adding each item's sums to the FP64 gradient.  Uses the
 * plan's tier lists (allocated by the first mixed build or gradient).
 */
int eri_jk_grad_prec(eri_plan_t* plan, const double* D, double* dEdR, int32_t want_j, int32_t want_k,
                     int32_t precision, void* stream);

/*
 * Copy the plan's lists to HOST buffers for inspection (each may be NULL):
 *   Q      float32 [npair]        Schwarz bound per shell pair, pair index a(a+1)/2+b (a >= b)
 *                                 (batched: molecule after molecule, local shell indices)
 *   sig    int32   [npair]        1 iff Q * Qmax >= thresh
 *   counts int32   [npair * 10]   kets of each pair class significant with the pair
 *   sorted int32   [npair]        significant pair indices, class by class (ss ps pp ds dp dd fs fp fd ff),
 *                                 inside a class molecule by molecule, each by Q descending then
 *                                 pair index ascending
 *   class_count int32 [10]        length of each class in `sorted`
 * Synchronises the device.
 */
int eri_get_lists(eri_plan_t* plan, float* Q, int32_t* sig, int32_t* counts, int32_t* sorted,
                  int32_t* class_count);

/* One class launch of the J/K build, as seen by eri_get_profile. */
typedef struct {
  int32_t bra_class, ket_class; /* pair classes 0..9 = ss ps pp ds dp dd fs fp fd ff */
  int32_t tier;                 /* 0 = FP64 J/K, 1 = FP32 J/K (mixed precision), 2 = gradient FP64,
                                   3 = J-engine (FP64, J-only builds), 4 = gradient FP32 tier */
  int32_t launches;             /* profiled launches summed into ms */
  double ms;                    /* total device time of those launches (CUDA events on the build stream) */
  int64_t quartets;             /* canonical shell quartets of the last build's launch */
  int64_t prim_quartets;        /* primitive quartets of the last build's launch */
  double flops;                 /* algorithmic FLOPs of the last build's launch */
} eri_launch_prof_t;

/*
 * Per-launch device times of every eri_build_jk and eri_jk_grad since the
 * previous call, for a plan created with opts.profile = 1 (eager builds; graph
 * builds are not profiled).  quartets / prim_quartets count the launch's work
 * items (ordered (bra, ket) pairs for the gradient and the J-engine); flops is
 * the algorithmic FLOP count of the implemented McMurchie-Davidson chain for
 * those items.  Fills up to cap
 * entries of out (host), sets *count to the number of (class pair, tier)
 * launches, synchronises, and resets the record.
 */
int eri_get_profile(eri_plan_t* plan, eri_launch_prof_t* out, int32_t cap, int32_t* count);

/*
 * Device-side checks: synchronises the plan's device and returns ERI_EDEVICE
 * (clearing the status word) if a kernel of this plan reported a problem
 * since the last check: in deterministic builds, an accumulated element
 * whose magnitude exceeded 2^16 (half the fixed-point range, so its value may
 * have wrapped).  ERI_OK otherwise.
 */
int eri_check(eri_plan_t* plan);

/* Statistics of the plan and of its last build (host copy; synchronises). */
int eri_get_stats(eri_plan_t* plan, eri_stats_t* stats);

/*
 * J and K in FP64 at the plan's threshold, for
 * callers that cannot allocate device memory when they build (code running
 * during CUDA graph capture, inside a device allocator, or on hosts that
 * forbid allocation after start-up).  The paper has no counterpart of this
 * call.  Its scratch (scaled density and half-J / half-K accumulators) is one
 * fixed device array inside the library, sized for at most
 * ERI_NOALLOC_MAX_NBF basis functions; a plan with more gets ERI_EUNSUPPORTED
 * and a message on stderr, and so does a batched plan.  The call allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.
 *   - The first call on a device looks up the array's device address on that
 *     device (cudaGetSymbolAddress); make that first call before any stream
 *     capture.
 *   - Every call, on every plan and stream, uses the same array, which keeps
 *     the previous call's contents (the accumulators are cleared at the start
 *     of each call).  Calls whose GPU work overlaps, on different streams or
 *     threads, race on it: order them.
 * D, J, K: device pointers as for eri_build_jk; J or K may be NULL.  J and K
 * always come from contracted Cartesian ERIs (a J-only call does not take the
 * J-engine), so they equal eri_build_jk(plan, D, J, K, -1, ERI_FP64, stream)
 * to rounding (within 1e-10, the parity tolerance), bit for bit only where
 * eri_build_jk takes the same path (J and K together, or opts.j_engine = 0).
 * eri_get_stats then describes this call as the last build.
 */
#define ERI_NOALLOC_MAX_NBF 256
int eri_build_jk_noalloc(eri_plan_t* plan, const double* D, double* J, double* K, void* stream);

/*
 * Point-charge attraction matrix (Sec. 2.4, Eq. v1e_definition and
 * Eq. v1e_summation_over_C; nuclei or QM/MM charges):
 *   V_mn = sum_C q_C (m| 1/|r - C| |n)
 * over every shell pair (no screening), by Eq. v1e_formula with the sum over
 * charges taken in Hermite space per primitive pair.  q: DEVICE, ncharge
 * doubles (the charges, signed: a nucleus of atomic number Z attracts
 * electrons with q = -Z in the electronic Hamiltonian); xyz: DEVICE,
 * ncharge x 3 doubles (bohr); V: DEVICE, nbf x nbf (packed per molecule for a
 * batched plan; every molecule sees every charge), overwritten.  ncharge = 0
 * gives V = 0.  The first call on a plan builds its primitive-pair lists (a
 * host wait); later calls only enqueue work.  Uses plan scratch, so it is
 * stream-ordered with the plan's builds.
 * Errors: ERI_EINVAL (NULL, ncharge < 0), ERI_ENOMEM, ERI_ECUDA.
 */
int eri_nuclear(eri_plan_t* plan, int32_t ncharge, const double* q, const double* xyz, double* V, void* stream);

/*
 * Gradient of E_V = sum_mn D_mn V_mn with D held fixed (SI Sec. 1.3,
 * Eq. si_v1e_derivative_A, _B and _C): dEdR (DEVICE, natom x 3) with respect to
 * the basis-function centres, dEdC (DEVICE, ncharge x 3, may be NULL) with
 * respect to the charge positions; both overwritten.  Centre A by the
 * raising/lowering rule on the Hermite coefficients, C by dR/dC = -R_{P+1},
 * B by translational invariance of each (pair, charge) term.  D as for
 * eri_build_jk.  Errors as for eri_nuclear.
 */
int eri_nuclear_grad(eri_plan_t* plan, const double* D, int32_t ncharge, const double* q, const double* xyz,
                     double* dEdR, double* dEdC, void* stream);

/*
 * Exchange-correlation quadrature on a molecular grid (Sec. 2.6; the paper's
 * four steps: grid, density, functional, matrix).  Plans of one molecule only
 * (a batched plan gets ERI_EUNSUPPORTED).  All arithmetic is FP64.
 *
 * eri_xc_grid builds the plan's grid on the device (step 1): for every atom,
 * nrad radial nodes (Gauss-Chebyshev of the second kind, x_i = cos(i pi /
 * (nrad+1)), mapped by Becke's r = radius (1+x)/(1-x), weight
 * (pi/(nrad+1)) sin(theta_i) r^2 dr/dx) times ntheta Gauss-Legendre nodes in
 * cos(theta) (ascending) times 2 ntheta azimuths phi_k = 2 pi (k+1/2)/(2 ntheta)
 * (trapezoid), each weighted by Becke's fuzzy-cell partition (equal cell sizes,
 * three iterations of p(mu) = (3 mu - mu^3)/2).  Point g = ((atom * nrad + i) *
 * ntheta + j) * 2 ntheta + k; npoints (host, may be NULL) receives
 * natom * nrad * 2 ntheta^2.  It also groups the points into blocks of at most
 * 32 (per atom: adjacent radial shells x one thirty-second of the sphere), finds the
 * shells that reach each block, and evaluates the basis functions and their
 * gradients there; when those values fit in cap_bytes (<= 0: 16 GiB) they stay
 * resident in device memory for every later call, otherwise each call
 * recomputes them in chunks of that size.  Waits for the device (a previous
 * grid's buffers are released; host bookkeeping of the block sizes).  The grid
 * follows eri_plan_set_coords: it is rebuilt, with the same parameters, at the
 * next XC call after a change (that call waits for the device too).
 * Requires 2 <= nrad <= 1000, 2 <= ntheta <= 64 with ntheta even, radius > 0,
 * and fewer than 2^31 points.
 * Errors: ERI_EINVAL, ERI_EUNSUPPORTED, ERI_ENOMEM, ERI_ECUDA.
 */
int eri_xc_grid(eri_plan_t* plan, int32_t nrad, int32_t ntheta, double radius, double cap_bytes, int64_t* npoints,
                void* stream);

/* Copy the grid out: points (DEVICE, npoints x 3, bohr) and weights (DEVICE,
 * npoints); either may be NULL.  Errors: ERI_EINVAL (no grid), ERI_ECUDA. */
int eri_xc_get_grid(eri_plan_t* plan, double* points, double* weights, void* stream);

/*
 * Step 2: rho_g = sum_mn D_mn phi_m(r_g) phi_n(r_g) (Eq. xc_density_0) and
 * grad rho_g = sum_mn D_mn grad(phi_m phi_n)(r_g) (Eq. xc_density_1) at every
 * grid point.  D: DEVICE, nbf x nbf, symmetric (AO order, unit-normalised
 * functions as for eri_build_jk); rho: DEVICE, npoints; grad_rho: DEVICE,
 * npoints x 3 or NULL; both overwritten.  Basis functions beyond their
 * extent (all components and gradients below 1e-15) are dropped per block.
 * Errors: ERI_EINVAL (NULL, no grid), ERI_EUNSUPPORTED, ERI_ECUDA.
 */
int eri_xc_density(eri_plan_t* plan, const double* D, double* rho, double* grad_rho, void* stream);

/*
 * Step 4 for given point potentials: V_mn = sum_g w_g [vrho_g phi_m phi_n +
 * vgrad_g . grad(phi_m phi_n)] (Eq. xc_grid_sum_0 + Eq. xc_grid_sum_1).
 * vrho: DEVICE, npoints (d eps/d rho); vgrad: DEVICE, npoints x 3
 * (d eps/d grad rho); V: DEVICE, nbf x nbf, overwritten (symmetric).
 * Errors: as eri_xc_density.
 */
int eri_xc_matrix(eri_plan_t* plan, const double* vrho, const double* vgrad, double* V, void* stream);

#define ERI_XC_SLATER 1 /* closed-shell Slater (Dirac) exchange, eps = -(3/4)(3/pi)^(1/3) rho^(4/3) */
#define ERI_XC_B88 2    /* Becke-88 exchange (beta = 0.0042) on the spin density rho/2 */

/*
 * Steps 2-4 with a built-in functional (step 3; the paper evaluates the
 * functional on the CPU and names none): density and gradient, eps, v_rho and
 * v_grad per point (points with rho < 1e-14 contribute nothing), then V as in
 * eri_xc_matrix.  V: DEVICE, nbf x nbf, overwritten; Exc: DEVICE, one double,
 * overwritten with E_xc = sum_g w_g eps_g (order of the partial sums not fixed).
 * Errors: ERI_EINVAL (NULL, no grid, unknown functional), ERI_EUNSUPPORTED,
 * ERI_ECUDA.
 */
int eri_xc(eri_plan_t* plan, const double* D, int32_t functional, double* V, double* Exc, void* stream);

/* Shape of the plan's grid and the work of one density / matrix pass. */
typedef struct {
  int64_t npoints;
  int32_t nblock, block_points, resident, nchunk;
  double sum_block_functions;     /* sum over blocks of the significant functions n_b */
  double sum_block_functions_sq;  /* sum over blocks of n_b^2 */
  double workspace_bytes;         /* basis-value workspace */
  double flops_density;           /* (2 n_b^2 + 8 n_b) x points, summed over blocks: X = D_b Phi_b and rho, grad rho */
  double flops_matrix;            /* the same for Z_b Phi_b^T and Z */
} eri_xc_stats_t;
int eri_xc_stats(eri_plan_t* plan, eri_xc_stats_t* stats);

/*
 * Measurement utility (not a step of the method): the FP64 (precision =
 * ERI_FP64) or FP32 (ERI_MIXED) fused multiply-add rate of the current device,
 * in TFLOP/s (FMA = 2 FLOP), from one launch of independent FMA chains over
 * every SM, `iters` iterations per chain, timed with CUDA events on `stream`.
 * These are the pipes the ERI kernels are bound by; the result is the measured
 * denominator of their roofline.  Allocates a small output buffer, waits for
 * the launch.  Errors: ERI_EINVAL, ERI_ENOMEM, ERI_ECUDA.
 */
int eri_peak_probe(int32_t precision, int32_t iters, double* tflops, void* stream);

/* Free every device and host resource of the plan (NULL is a no-op). */
int eri_plan_destroy(eri_plan_t* plan);

/* Static description of an error code. */
const char* eri_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
