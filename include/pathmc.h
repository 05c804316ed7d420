/*
 * pathmc — C ABI of a GB300 (sm_103a) library that runs many independent
 * Reversible-Jump MCMC chains over light paths, after G. H. Collin,
 * "Using path integrals for the propagation of light in a scattering
 * dominated medium" (arXiv:1811.04156).
 *
 * A path is a polyline f_0 .. f_{n-1}: f_0 is a point source, f_1 .. f_{n-2}
 * are scattering vertices, f_{n-1} lies on a spherical light sensor
 * (section "Numerical path integration").  Its density is
 *   p = p_i(f_0, f_1) * prod_k p_v(f_{k-1}, f_k, f_{k+1}) * p_f(f_{n-2}, f_{n-1})
 * (appendix, "Path probability distribution"; Eqs. emission_dist, intervtx,
 * b_depth_def, angular_scattering, detection_prob), and its integral over all
 * paths up to a vertex cap is the detected intensity per emitted photon.
 *
 * Conventions shared by every entry point:
 *  - Status: every function returns PMC_OK (0) or a PMC_ERR_* code;
 *    pmc_last_error() gives a per-thread message for the last failure.
 *  - Ownership: handles are created and destroyed by the library; descriptor
 *    structs and the host arrays they point to are copied during the call
 *    and may be freed afterwards.  Device pointers passed in (pmc_logp and
 *    friends) stay owned by the caller.
 *  - Streams: `stream` is a cudaStream_t passed as void*; NULL is the legacy
 *    default stream.  Functions marked "async" only enqueue work on it.
 *  - Units: lengths in metres, coefficients in 1/m, double precision on the
 *    host.  Device state is FP32 with FP64 estimator accumulators.
 *  - Layout of device path batches: SoA float32 [3][batch][cap] (all x, then
 *    all y, then all z), vertex k of path b at index b*cap + k; vertex
 *    counts int32 [batch].
 *  - One GPU; no CPU fallback: without a usable device the calls fail with
 *    PMC_ERR_NO_DEVICE or PMC_ERR_CUDA.
 */
#ifndef PATHMC_H
#define PATHMC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PMC_API __attribute__((visibility("default")))
#else
#define PMC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define PMC_OK 0
#define PMC_ERR_INVALID 1        /* bad argument or descriptor */
#define PMC_ERR_OOM 2            /* device allocation failed */
#define PMC_ERR_CUDA 3           /* a CUDA runtime call failed */
#define PMC_ERR_DEVICE_STATUS 4  /* a kernel reported an error word (non-finite state, bounds) */
#define PMC_ERR_ABORTED 5        /* the run was aborted through pmc_request_abort */
#define PMC_ERR_NO_DEVICE 6      /* no CUDA device available */

#define PMC_HOMOGENEOUS 0
#define PMC_LAYERED 1

#define PMC_EMIT_ISOTROPIC 0
#define PMC_EMIT_VMF 1

#define PMC_RHO_ONE 0
#define PMC_RHO_PAPER 1

#define PMC_INIT_DIRECT 0
#define PMC_INIT_STRAIGHT 1
#define PMC_INIT_USER 2

#define PMC_WITHIN_PERTURB 0
#define PMC_WITHIN_MALA 1
#define PMC_WITHIN_TREE 2
#define PMC_WITHIN_HMC 3

/* Chain layout of the kernel (pmc_run_desc.layout). */
#define PMC_LAYOUT_AUTO 0      /* autotuner's choice (warp layout when warps_per_block is given) */
#define PMC_LAYOUT_WARP 1      /* one warp per chain */
#define PMC_LAYOUT_LANE 2      /* one lane per chain: lean physics only (homogeneous medium, isotropic
                                  emission, rho = 1, pure Henyey-Greenstein) with Gaussian, MALA or
                                  tree moves */

#define PMC_FLAG_GRADIENTS 1   /* accumulate score terms for pmc_grad_estimator */
#define PMC_FLAG_NO_GRAPH 2    /* launch kernels directly instead of replaying a CUDA graph */
#define PMC_FLAG_ONE_LAUNCH 4  /* every chain in one persistent launch (one work queue, longest vertex caps
                                  first, one shared window with global spill for longer caps) instead of
                                  one launch per vertex-cap class (64, 128, 256, 512, 1024) */

#define PMC_MOVE_INTERIOR 0    /* Gaussian perturbation or MALA of an interior vertex */
#define PMC_MOVE_END 1         /* vMF step of the end vertex on the sensor sphere */
#define PMC_MOVE_BIRTH 2
#define PMC_MOVE_DEATH 3

typedef struct pmc_ctx_s* pmc_ctx_t;
typedef struct pmc_medium_s* pmc_medium_t;
typedef struct pmc_geom_s* pmc_geom_t;
typedef struct pmc_chains_s* pmc_chains_t;

/* Medium: absorption a(x) = 1/lambda_a and scattering b(x) = 1/lambda_s
 * (appendix, intermediate vertex), either constant or constant within
 * horizontal layers [z0 + l*dz, z0 + (l+1)*dz) (layer 0 and layer L-1 extend
 * to -inf / +inf).  Phase function: the mixture
 * f_sl * p_SL + (1 - f_sl) * p_HG with mean cosine g (Eq. angular_scattering).
 * Requirements: lengths > 0, |g| < 1, 0 <= f_sl <= 1 (f_sl > 0 needs g > 0),
 * dz > 0 and 1 <= n_layers <= 4096 when layered. */
typedef struct {
  int kind;                        /* PMC_HOMOGENEOUS or PMC_LAYERED */
  double lambda_s, lambda_a;       /* homogeneous lengths (m) */
  double g, f_sl;
  double z0, dz;                   /* layered geometry (m) */
  int n_layers;
  const double* lambda_s_layers;   /* host [n_layers], copied */
  const double* lambda_a_layers;   /* host [n_layers], copied */
  /* Wavelength dependence (section "Discussion"; the paper gives no model, the
   * reading here is power laws): at wavelength l the coefficients are
   * b (l / lambda0)^(-k_s) and a (l / lambda0)^(-k_a).  Used by chains that
   * sample the wavelength (pmc_run_desc.n_lambda); 0, 0, 0 = none. */
  double lambda0;                  /* reference wavelength (nm) of lambda_s, lambda_a */
  double k_s, k_a;                 /* >= 0 */
} pmc_medium_desc;

/* Point source with isotropic or von Mises-Fisher emission (Eq. emission_dist). */
typedef struct {
  double pos[3];
  int emission;                    /* PMC_EMIT_ISOTROPIC or PMC_EMIT_VMF */
  double kappa;                    /* vMF concentration (> 0 for VMF) */
  double dir[3];                   /* preferred direction (normalised internally) */
} pmc_source;

/* Spherical sensor with detection probability 1 or Eq. detection_prob. */
typedef struct {
  double centre[3];
  double radius;                   /* > 0 */
  int rho;                         /* PMC_RHO_ONE or PMC_RHO_PAPER */
  double rho_hat[3];               /* preferred direction (normalised internally) */
} pmc_sensor;

/* One source-sensor pair sampled by n_chains chains with vertex cap `cap`
 * (2 <= cap <= 1024; paths hold n in [2, cap] vertices). */
typedef struct {
  int source, sensor;
  int n_chains;
  int cap;
} pmc_pair;

typedef struct {
  int n_sources;
  const pmc_source* sources;
  int n_sensors;
  const pmc_sensor* sensors;
  int n_pairs;
  const pmc_pair* pairs;
} pmc_geometry_desc;

/* Chain settings.  Move probabilities must sum to 1 (each in [0, 1]).
 * Within-dimension moves pick one of the n-1 movable vertices uniformly:
 * the end vertex takes a vMF step of concentration kappa_end on the sensor
 * (0 -> (R/sigma)^2), an interior vertex a Gaussian step of scale sigma
 * (PMC_WITHIN_PERTURB) or a MALA step of size mala_step (PMC_WITHIN_MALA).
 * PMC_WITHIN_TREE instead moves the whole path in the paper's tree
 * coordinates (section "Path proposal distribution"; appendix "Path space
 * coordinate system"): interior vertex m = (k + l)/2 sits in the bispherical
 * system of its tree foci f_k, f_l (root: f_0, f_{n-1}) with coordinates
 * zeta = atanh(cos s), t = ln(d1/d2) and phi about the foci axis, measured
 * from the normal of the parent's triangle (inherited axes); each proposal
 * takes a vMF step of the end vertex (kappa_end; 0 -> 1/sigma^2), a normal
 * step of scale sigma/sqrt(n) (sigma dimensionless) in every node's (zeta, t,
 * phi), rebuilds the path top-down and accepts with
 * p(x') J(x') / (p(x) J(x)), J = prod over nodes (d1 d2 / (2 gamma))^3 sin^2 s.
 * PMC_WITHIN_HMC makes full-path gradient moves (section "Discussion"): when
 * the within-dimension draw picks an interior vertex, every interior vertex
 * gets a standard normal momentum and hmc_steps leapfrog steps of size
 * mala_step follow d log p / d f (zero where the density is zero) with the
 * source and the end vertex fixed, accepted with exp(H - H'), H = -log p +
 * |p|^2/2; picking the end vertex makes the vMF end move.
 * Tree and HMC moves need the whole vertex cap in shared memory (smem_window 0).
 * Births insert a vertex into a segment chosen with probability
 * tau_b(k)/sum tau_b, placed by bispherical coordinates; deaths remove an
 * interior vertex chosen uniformly (appendix, jump proposal; dimension
 * matching transformation).  States after global step index >= burn_in are
 * recorded in the estimators. */
typedef struct {
  uint64_t seed;                   /* Philox4x32-10 key */
  double p_within, p_birth, p_death;
  int within;                      /* PMC_WITHIN_PERTURB, _MALA, _TREE or _HMC */
  double sigma;                    /* Gaussian step (m); tree moves: dimensionless scale */
  double mala_step;                /* MALA epsilon, HMC leapfrog step (m) */
  double kappa_end;                /* vMF concentration of end moves; 0 -> (R/sigma)^2 (tree: 1/sigma^2) */
  uint64_t burn_in;
  uint32_t thin_bridge;            /* reference-density bridge terms every k steps; 0 = off */
  int init;                        /* PMC_INIT_DIRECT, PMC_INIT_STRAIGHT or PMC_INIT_USER */
  int init_k;                      /* STRAIGHT: interior vertices on the source-sensor line */
  double init_jitter;              /* STRAIGHT: N(0, jitter^2) per coordinate (m) */
  const float* init_xyz;           /* USER: host, [total_chains][3][init_stride], absolute (m) */
  const int* init_n;               /* USER: host, [total_chains] */
  int init_stride;                 /* USER: vertex stride of init_xyz (>= every init_n) */
  int flags;                       /* PMC_FLAG_* */
  int warps_per_block;             /* 0 = autotune (also the shared window); with smem_window set
                                      and the lane layout, 0 = the CTA size (1, 2 or 4 warps) that
                                      keeps the most 32-chain work items resident at once */
  int smem_window;                 /* vertices per chain kept in shared memory, a multiple of 32;
                                      entries beyond it live in global memory.  0 = the whole cap
                                      (or the autotuner's choice when warps_per_block = 0) */
  int hmc_steps;                   /* PMC_WITHIN_HMC: leapfrog steps per move (1..1000) */
  int layout;                      /* PMC_LAYOUT_*.  LANE: each chain on one lane of a warp, its first
                                      smem_window vertices (any value >= 2; 0 = 16 or the autotuner's
                                      choice) in shared memory; the same Markov chain and random
                                      numbers as the warp layout.  Fails with PMC_ERR_INVALID for
                                      runs that are not lean */
  /* Wavelength as a sampled coordinate (section "Discussion": a wavelength
   * parameter added to the path density, sampled along with the vertices).
   * n_lambda >= 2 (0 = off): the chains sample (path, l) from S(l) p_l(path),
   * S the emission-times-detection spectrum, piecewise linear through
   * (lambda_nm[i], spectrum[i]) (host, copied; increasing wavelengths, values
   * >= 0, any scale: normalised internally) and 0 outside, p_l the path
   * density of the medium at l.  The wavelength is one more movable
   * coordinate of the within-dimension draw (one of n: the n-1 movable
   * vertices and l); a wavelength move takes a Gaussian step of sigma_lambda
   * nm with the path held.  Initial wavelengths: the spectrum's quantile of
   * u01 of Philox counter (0, 1, chain, init purpose).  The intensity is
   * Z2 / pi(n = 2) with Z2 the spectrum-weighted direct sector.  Needs a
   * homogeneous medium, PMC_WITHIN_PERTURB, no PMC_FLAG_GRADIENTS and the
   * warp layout (PMC_ERR_INVALID otherwise); within-dimension proposal and
   * acceptance counts include the wavelength moves. */
  int n_lambda;
  const double* lambda_nm;
  const double* spectrum;
  double sigma_lambda;
  int64_t chain_lo, chain_hi;      /* chain window: this chain set holds the geometry's chains
                                      [chain_lo, chain_hi) in pair order (chains of pair p are numbered
                                      after those of pairs 0..p-1); 0, 0 = all.  A chain keeps its
                                      global index in its Philox counters and initial path, so the
                                      chains of a window evolve exactly as in the whole set (the
                                      sharded form over several GPUs, pmc_shard_range).  USER init
                                      data and pmc_set_states then cover the window's chains */
} pmc_run_desc;

/* Per-pair estimate returned by pmc_read_estimator. */
typedef struct {
  double intensity;                /* detected intensity per emitted photon */
  double std_err;                  /* standard error of `intensity` */
  double rel_err;                  /* std_err / intensity */
  double pi_direct;                /* fraction of recorded states with n == 2 */
  double z2;                       /* direct-sector integral (n == 2 part) */
  double rhat;                     /* Gelman-Rubin R-hat of the path length over chains */
  double accept[4];                /* acceptance rate per PMC_MOVE_* */
  double proposals[4];             /* proposals per PMC_MOVE_* */
  double mean_n, mean_length;      /* means over recorded states */
  double n_samples;                /* recorded states */
  double ess;                      /* effective sample size of pi_direct */
  double bridge_intensity;         /* geometric-bridge estimate (NaN when off) */
  double bridge_std_err;
} pmc_estimate;

/* ---------------------------------------------------------------------- */
/* Context, medium, geometry                                              */
/* ---------------------------------------------------------------------- */

/* Bind a context to CUDA device `device`.  Fails with PMC_ERR_NO_DEVICE when
 * the device does not exist. */
PMC_API int pmc_create_context(int device, pmc_ctx_t* out);
PMC_API int pmc_destroy_context(pmc_ctx_t ctx);

/* Copy a medium description to the device (appendix, intermediate vertex;
 * Eq. b_depth_def).  Also solves coth(k) - 1/k = g for the insertion
 * centering constant kappa_eq (appendix, dimension matching transformation). */
PMC_API int pmc_create_medium(pmc_ctx_t ctx, const pmc_medium_desc* desc, pmc_medium_t* out);
PMC_API int pmc_destroy_medium(pmc_medium_t medium);

/* Copy sources, sensors and pairs to the device (section "Implementation":
 * point source, spherical light-sensitive elements).  Rejects a source
 * inside or on its pair's sensor. */
PMC_API int pmc_create_geometry(pmc_ctx_t ctx, const pmc_geometry_desc* desc, pmc_geom_t* out);
PMC_API int pmc_destroy_geometry(pmc_geom_t geom);

/* ---------------------------------------------------------------------- */
/* Chains                                                                 */
/* ---------------------------------------------------------------------- */

/* Allocate chain state for every pair of `geom` and write the initial paths
 * (async on `stream`).  DIRECT: n = 2 with the end vertex at the sensor point
 * nearest the source.  STRAIGHT: init_k interior vertices evenly spaced on
 * the segment from the source to that point, each jittered by
 * N(0, init_jitter^2 I) from Philox.  USER: copies init_xyz / init_n.
 * The chains keep references to ctx, medium and geom, which must outlive them. */
PMC_API int pmc_init_chains(pmc_ctx_t ctx, pmc_medium_t medium, pmc_geom_t geom,
                    const pmc_run_desc* run, void* stream, pmc_chains_t* out);
PMC_API int pmc_destroy_chains(pmc_chains_t chains);

/* Re-run the initialisation of pmc_init_chains on the existing buffers
 * (async): DIRECT / STRAIGHT paths again, step counters and accumulators set
 * to zero.  Chains created with PMC_INIT_USER need pmc_set_states instead. */
PMC_API int pmc_reset_chains(pmc_chains_t chains, void* stream);

/* Replace every chain's path by host data and zero the step counters and
 * accumulators (async copy from `xyz` / `n`, which must stay valid until the
 * stream reaches it; pinned memory makes the copy asynchronous).
 * xyz: [total_chains][3][stride] absolute positions; n: [total_chains] with
 * 2 <= n <= cap of the chain's pair and n <= stride. */
PMC_API int pmc_set_states(pmc_chains_t chains, const float* xyz, const int* n, int stride, void* stream);

/* Advance every chain by n_steps RJMCMC steps (async).  One step is one
 * proposal and its accept/reject decision by Eq. acceptFact (read in Green's
 * orientation for births; deaths use the reciprocal of the reverse birth).
 * Random numbers are Philox4x32-10 keyed by the seed and indexed by
 * (global step, chain), so a run split over several calls reproduces the
 * uninterrupted trajectory exactly. */
PMC_API int pmc_run_steps(pmc_chains_t chains, uint64_t n_steps, void* stream);

/* Reduce the per-chain FP64 accumulators to one pmc_estimate per pair and
 * copy them to `out` (host, n_pairs entries, caller-owned).  Synchronises
 * `stream`.  The intensity is Z2 / pi(n=2): Z2 is the n = 2 part of the path
 * integral (2-D quadrature over the sensor as seen from the source) and
 * pi(n=2) the chains' fraction of states with n = 2; the standard error comes
 * from the across-chain variance. */
PMC_API int pmc_read_estimator(pmc_chains_t chains, pmc_estimate* out, size_t n_pairs, void* stream);

/* ---------------------------------------------------------------------- */
/* Sharded chain sets (several GPUs; section "Implementation": chains are  */
/* independent)                                                           */
/* ---------------------------------------------------------------------- */

/* Per-pair moments of the chain accumulators: PMC_MOMENT_WORDS doubles per
 * pair, each a sum over the pair's chains, so the moments of a chain set
 * split over ranks (pmc_run_desc.chain_lo/hi) add up, by one sum all-reduce,
 * to those of the whole set.  Layout (N = recorded states of a chain, n2 its
 * recorded states with n = 2, A_k its summed score of parameter k: A_0 =
 * sum_L / lambda_s^2 - (sum_n - 2 N) / lambda_s, A_1 = sum_L / lambda_a^2,
 * A_2 = sum_G; lambda = 1 for layered media): [0] chains; [1..16] the
 * PMC_ACC_WORDS accumulator words summed; [17..20] sum of the per-chain mean
 * path length, of its square, of the per-chain variance of the path length
 * and the count of chains with N > 1; [21..23] sum n2^2, N n2, N^2;
 * [24..26] sum A_k^2; [27..29] sum N A_k; [30..32] sum n2 A_k; [33..35]
 * sum A_k; the rest 0. */
#define PMC_MOMENT_WORDS 40

/* The sharded form's partition: the contiguous chain window [*chain_lo,
 * *chain_hi) of rank `rank` among `world` ranks over the chains of `pairs`
 * (pair order, as in pmc_geometry_desc), balanced by vertex cap x steps (a
 * chain costs its pair's cap; every chain runs the same steps).  Every chain
 * belongs to exactly one rank and every rank gets at least one.  Host only.
 * Errors: PMC_ERR_INVALID for rank outside [0, world), bad pairs or fewer
 * chains than ranks. */
PMC_API int pmc_shard_range(const pmc_pair* pairs, int n_pairs, int rank, int world, int64_t* chain_lo,
                            int64_t* chain_hi);

/* This chain set's per-pair moments into `out` (host, caller-owned,
 * n_pairs * PMC_MOMENT_WORDS doubles).  Synchronises `stream`; reports
 * PMC_ERR_ABORTED / PMC_ERR_DEVICE_STATUS as pmc_read_estimator does. */
PMC_API int pmc_read_moments(pmc_chains_t chains, double* out, size_t len, void* stream);

/* Direct-sector integral Z2 of every pair (host out, n_pairs doubles).
 * Synchronises `stream`. */
PMC_API int pmc_pair_z2(pmc_chains_t chains, double* z2, size_t n_pairs, void* stream);

/* Per-pair estimates from moments (host only; the reduction of
 * pmc_read_estimator, which is this function applied to the chain set's own
 * moments): intensity = Z2 / pi(n = 2) with the across-chain standard error,
 * R-hat, acceptance, means, ESS (pmc_estimate fields; bridge fields NaN) and,
 * when grad / grad_se are not NULL (3 doubles per pair each, homogeneous
 * media), intensity * E_p[score] with its delta-method standard error.
 * moments: n_pairs * PMC_MOMENT_WORDS; z2: n_pairs. */
PMC_API int pmc_estimate_from_moments(const double* moments, size_t n_pairs, const double* z2, pmc_estimate* out,
                                      double* grad, double* grad_se);

/* Host moments of stand-in accumulators: acc [n_chains][PMC_ACC_WORDS] (the
 * pmc_read_accumulators layout), chain_pair [n_chains] pair of each chain;
 * moments (n_pairs * PMC_MOMENT_WORDS) are overwritten.  The same per-chain
 * terms as the device reduction. */
PMC_API int pmc_moments_from_accumulators(const double* acc, size_t n_chains, const int* chain_pair, size_t n_pairs,
                                          double lambda_s, double lambda_a, double* moments);

/* d intensity / d theta per pair: intensity * E_p[d log p / d theta], the
 * score-function gradient (dI/dtheta = I E_p[d log p/d theta]).
 * Homogeneous media: theta = (lambda_s, lambda_a, g), with E_p over every
 * recorded state, accumulated while stepping (needs PMC_FLAG_GRADIENTS).
 * Layered media: theta = (lambda_s[0..L), lambda_a[0..L)), with E_p over the
 * chains' current states (one state per chain).  `grad` and `grad_se` are
 * host arrays of n_pairs * n_theta doubles (pair-major); grad_se may be NULL.
 * Synchronises `stream`. */
PMC_API int pmc_grad_estimator(pmc_chains_t chains, double* grad, double* grad_se, size_t len, void* stream);

/* Number of medium parameters theta (3 or 2 * n_layers). */
PMC_API int pmc_n_theta(pmc_medium_t medium);

/* Copy chain states to host buffers: xyz [total_chains][3][stride] absolute
 * positions (stride >= the largest cap), n [total_chains], steps
 * [total_chains] (may be NULL).  Synchronises `stream`. */
PMC_API int pmc_read_states(pmc_chains_t chains, float* xyz, int* n, uint64_t* steps, int stride, void* stream);

/* Raw per-chain accumulators: PMC_ACC_WORDS doubles per chain, in the order
 * n_rec, n_direct, sum_n, sum_L, sum_L2, sum_G, sum_bridge, n_bridge,
 * prop[4], acc[4] (sum_G = sum of d log sigma / d g over vertices).
 * Synchronises `stream`. */
#define PMC_ACC_WORDS 16
PMC_API int pmc_read_accumulators(pmc_chains_t chains, double* out, size_t n_doubles, void* stream);
PMC_API int pmc_total_chains(pmc_chains_t chains);

/* Launch shapes chosen for the chains (by the autotuner when
 * warps_per_block = 0): one row of 6 ints per vertex-cap class, written to
 * `out` (host): shared-memory window in vertices per chain (smaller than the
 * class's caps when entries beyond it live in global memory), first and
 * one-past-last position in the processing order, warps per block,
 * persistent grid size, and the kernel: 0 the lean and 1 the general kernel
 * with one warp per chain, 2 the general kernel with tree moves, 3 with HMC
 * moves, 4 the lean kernel with one chain per lane (32 chains per warp), 5
 * the same with MALA moves, 6 the general kernel sampling the wavelength, 7
 * the lean kernel with tree moves, 8 the lean kernel with one chain per lane
 * and tree moves (each warp's tree moves pooled over its 32 lanes).
 * Returns the number of classes in *n_classes;
 * writes at most max_rows rows. */
PMC_API int pmc_chains_launch_info(pmc_chains_t chains, int* out, int max_rows, int* n_classes);

/* Serialise / restore the complete chain state (positions, vertex counts,
 * step counters, accumulators) through a host buffer.  With buf == NULL,
 * pmc_save_state stores the needed size in *bytes.  Synchronises `stream`. */
PMC_API int pmc_save_state(pmc_chains_t chains, void* buf, size_t* bytes, void* stream);
PMC_API int pmc_load_state(pmc_chains_t chains, const void* buf, size_t bytes, void* stream);

/* The chains' current wavelengths (wavelength sampling only; PMC_ERR_INVALID
 * otherwise): out (host, caller-owned) receives total_chains floats (nm).
 * Synchronises `stream`. */
PMC_API int pmc_read_lambda(pmc_chains_t chains, float* out, size_t len, void* stream);

/* Ask running and future pmc_run_steps calls of these chains to stop at the
 * next step boundary; pmc_run_steps then reports PMC_ERR_ABORTED on the next
 * synchronising call.  flag = 0 clears the request. */
PMC_API int pmc_request_abort(pmc_chains_t chains, int flag);

/* Device status word of the chains (0 = fine); bit 0: non-finite state at
 * load, bit 1: aborted, bit 2: bad vertex count.  Synchronises `stream`. */
PMC_API int pmc_chain_status(pmc_chains_t chains, int* status, void* stream);

/* ---------------------------------------------------------------------- */
/* Density evaluation on caller-owned device batches                      */
/* ---------------------------------------------------------------------- */

/* log p of `batch` paths of pair `pair` (async).  xyz: device SoA
 * [3][batch][cap] absolute positions; n: device int32 [batch] with
 * 2 <= n <= cap; out_logp: device float32 [batch].  A path whose non-final
 * segment touches the sensor ball, whose final segment arrives from inside
 * (cos Phi <= 0) or that has a zero-length segment gets -inf. */
PMC_API int pmc_logp(pmc_ctx_t ctx, pmc_medium_t medium, pmc_geom_t geom, int pair,
             const float* xyz, const int* n, int batch, int cap, float* out_logp, void* stream);

/* log p and d log p / d(vertex positions) for every vertex (async); the
 * gradient has the layout of xyz (unused slots are written as 0).  The end
 * vertex's gradient is that of the expression with nu = (f - c)/|f - c|,
 * i.e. not projected onto the sphere. */
PMC_API int pmc_logp_grad(pmc_ctx_t ctx, pmc_medium_t medium, pmc_geom_t geom, int pair,
                  const float* xyz, const int* n, int batch, int cap,
                  float* out_logp, float* out_grad, void* stream);

/* d log p / d theta per path (async); out: device float32 [batch][n_theta]. */
PMC_API int pmc_score(pmc_ctx_t ctx, pmc_medium_t medium, pmc_geom_t geom, int pair,
              const float* xyz, const int* n, int batch, int cap, float* out, void* stream);

/* ---------------------------------------------------------------------- */
/* Normalisation by the geometric bridge                                  */
/* ---------------------------------------------------------------------- */

/* The paper's geometric estimator (section "Comparison of relative light
 * yield": B = E_0[sqrt(p_1/p_0)] / E_1[sqrt(p_0/p_1)]) with p_0 := q_ref, a
 * normalised reference density built from the paper's recursive tree of
 * bispherical coordinates (appendix, path space coordinate system): vertex
 * m = floor((k+l)/2) placed about the foci f_k, f_l by q(s) q(t) q(phi) with
 * beta from the foci (appendix, dimension matching transformation), the vertex
 * count a Poisson law in the straight-line scattering depth truncated to
 * [2, cap], the end vertex uniform over the sensor cap visible from the source.
 * Its normalisation makes the bridge an estimate of the absolute intensity. */

/* log q_ref of caller paths (async; same layout and frame as pmc_logp); -inf
 * when the end vertex lies outside the visible cap.  Synchronises `stream`. */
PMC_API int pmc_qref_logdensity(pmc_ctx_t ctx, pmc_medium_t medium, pmc_geom_t geom, int pair, const float* xyz,
                                const int* n, int batch, int cap, float* out, void* stream);

/* Draws n_draws paths of pair `pair` from q_ref (Philox counter (draw, vertex,
 * stream = pair)).  out_xyz: device [3][n_draws][stride] absolute positions,
 * out_n: device [n_draws]; stride >= cap.  Synchronises `stream`. */
PMC_API int pmc_qref_sample(pmc_ctx_t ctx, pmc_medium_t medium, pmc_geom_t geom, int pair, uint64_t seed,
                            uint64_t draw0, uint64_t n_draws, float* out_xyz, int* out_n, int stride, void* stream);

/* Bridge estimate of every pair's intensity: n_draws reference draws per pair
 * give E_q[sqrt(p/q_ref)], the chains' current states give
 * E_p[sqrt(q_ref/p)].  out (host): [n_pairs][2] = intensity, standard error
 * (delta method over both sample variances).  Synchronises `stream`. */
PMC_API int pmc_bridge(pmc_chains_t chains, uint64_t n_draws, uint64_t seed, double* out, void* stream);

/* One row of log ratios for the optimal bridge (pmc_bridge_ratio) of pair
 * `pair`'s intensity against q_ref: logr[0 .. n_draws) = log(p / q_ref) at
 * n_draws fresh reference draws numbered from draw0 (Philox key `seed`,
 * stream = pair), then logr[n_draws + i] = log(q_ref / p) at the pair's chain
 * i's current path (-inf where either density is 0).  logr: device,
 * caller-owned, n_draws + n_chains(pair) floats.  With rows stacked over
 * observations, pmc_bridge_ratio(n0 = n_draws, n1 = n_chains) returns the
 * intensity (q_ref is normalised).  Asynchronous on `stream`. */
PMC_API int pmc_bridge_observe_log(pmc_chains_t chains, int pair, uint64_t n_draws, uint64_t draw0, uint64_t seed,
                                   float* logr, void* stream);

/* ---------------------------------------------------------------------- */
/* Relative light yield of two sensors (section "Comparison of relative   */
/* light yield"; appendix "Relative light yield transformation") and      */
/* path-length distributions (section "Comparison of timing              */
/* distributions")                                                        */
/* ---------------------------------------------------------------------- */

/* The yield entry points compare two pairs that share a source: pair0's
 * paths end on sensor 0, pair1's on sensor 1.  The map T takes a path ending
 * on sensor 0 to one ending on sensor 1 by bending it along a cylinder
 * through the source whose tangent there points at sensor 0 (k = unit vector
 * to sensor 0; m in the plane of k and B = (sensor 1 - source), pointing away
 * from B; n = k x m; cos Psi = k.B/|B|; r_C = |B| / (2 sin Psi);
 * Omega = 2 Psi - R_1 / r_C; b_0 = |sensor 0 - source| - R_0; b_1 = r_C Omega):
 * interior vertex f with xb = (f - f0).m / b_0, yb = (f - f0).n / b_0,
 * w = (f - f0).k / b_0 goes to
 *   f0 - r_C m + (r_C + xb b_1)(m cos(w Omega) + k sin(w Omega)) + n yb b_1,
 * with volume ratio b_1^2 Omega (r_C + xb b_1) / b_0^3; the end vertex keeps
 * its offset direction from sensor 0's centre, rotated by Omega in the (m, k)
 * plane, on sensor 1 (area ratio (R_1/R_0)^2).  T is one-to-one where
 * r_C + xb b_1 > 0 and |w Omega| < pi; elsewhere the other density is 0.
 * Then p_1(x) = p(T x; sensor 1) |dT/dx| and the geometric estimator
 * B = E_0[sqrt(p_1/p_0)] / E_1[sqrt(p_0/p_1)] is the ratio of the light seen by
 * sensor 1 to the light seen by sensor 0.  Errors: PMC_ERR_INVALID when the
 * pairs are equal or out of range, do not share a source position, or the
 * sensors are collinear with the source. */

/* Log density ratio of caller paths (layout, frame and ownership of
 * pmc_logp).  side 0 (paths of pair0): out[b] = log p(T x; pair1) +
 * log|dT/dx| - log p(x; pair0); side 1 (paths of pair1): out[b] =
 * log p(T^-1 y; pair0) - log|dT/dx| at T^-1 y - log p(y; pair1).  -inf outside
 * T's domain or where either density is 0; NaN when n is outside [2, cap].
 * out_xyz (device, same layout as xyz, may be NULL) receives the mapped paths.
 * batch = 0 is a no-op (the buffers may then be NULL).  Asynchronous on `stream`. */
PMC_API int pmc_yield_logratio(pmc_ctx_t ctx, pmc_medium_t medium, pmc_geom_t geom, int pair0, int pair1, int side,
                               const float* xyz, const int* n, int batch, int cap, float* out, float* out_xyz,
                               void* stream);

/* One observation of every chain of pair0 and pair1 at its current path:
 * sums[i] += sqrt(p_1/p_0) for pair0's chain i (i < n0 = pair0's chain count)
 * and sums[n0 + i] += sqrt(p_0/p_1) for pair1's chain i (0 outside T's
 * domain).  sums: device, caller-owned, n0 + n1 doubles, zeroed by the caller
 * before the first observation.  Asynchronous on `stream`. */
PMC_API int pmc_yield_observe(pmc_chains_t chains, int pair0, int pair1, double* sums, void* stream);

/* Estimate from the sums of n_obs observations: out (host, 6 doubles) = B,
 * its standard error (delta method over the across-chain variances of the
 * per-chain means), E_0[sqrt(p_1/p_0)], E_1[sqrt(p_0/p_1)], and the two
 * across-chain variances.  Synchronises `stream`. */
PMC_API int pmc_yield_estimate(pmc_chains_t chains, int pair0, int pair1, const double* sums, uint64_t n_obs,
                               double* out, void* stream);

/* One observation of every chain of pair0 and pair1 as log ratios rather
 * than sums: logr[i] = log(p_1/p_0) at pair0's chain i (i < n0) and
 * logr[n0 + i] = log(p_0/p_1) at pair1's chain i (-inf outside T's domain).
 * logr: device, caller-owned, n0 + n1 floats (one row of the array that
 * pmc_bridge_ratio reads).  Asynchronous on `stream`. */
PMC_API int pmc_yield_observe_log(pmc_chains_t chains, int pair0, int pair1, float* logr, void* stream);

/* Optimal bridge estimate (Meng & Wong 1996, the iterative estimator that
 * the geometric one approximates) of r = c_1 / c_0 from stored log ratios:
 * logr (device, caller-owned) holds `rows` rows of n0 values log(q1/q0)(x),
 * x ~ p0, followed by n1 values log(q0/q1)(x), x ~ p1.  Starting from the
 * geometric estimate, r <- [mean over p0 draws of l / (s1 l + s0 r)] /
 * [mean over p1 draws of 1 / (s1 l + s0 r)], l = q1/q0, s_k = n_k/(n0 + n1),
 * until the relative change is below tol or after max_iter iterations.  The
 * standard error comes from `groups` disjoint chain groups (a chain's group
 * is its index within its side mod groups), each iterated on its own.
 * out (host, 4 doubles): r, standard error, iterations, the geometric
 * estimate.  1 <= groups <= min(n0, n1, 1024).  Synchronises `stream`. */
PMC_API int pmc_bridge_ratio(pmc_ctx_t ctx, const float* logr, uint64_t rows, int n0, int n1, int groups,
                             int max_iter, double tol, double* out, void* stream);

/* One observation of the score d log p / d theta at every chain's current
 * path, layered media only (theta = (lambda_s[0..L), lambda_a[0..L))):
 * sums[pair][j] += score_j and sums[pair][2L + j] += score_j^2, j < 2L.
 * sums: device, caller-owned, n_pairs * 4L doubles, zeroed by the caller.
 * With n_obs observations of N chains, E_p[score] = sums / (N n_obs); the
 * difference of two pairs' means is d log(I_1 / I_0) / d theta, the
 * gradient of the relative light yield (calibration of the medium from
 * detector ratios).  Homogeneous media accumulate their scores while
 * stepping (pmc_grad_estimator).  Asynchronous on `stream`. */
PMC_API int pmc_score_observe(pmc_chains_t chains, double* sums, void* stream);

/* Path-length distribution of the chains: one observation of every chain,
 * hist[pair][bin] += 1 with bin = floor((L - l_lo) / (l_hi - l_lo) * n_bins)
 * for its current path length L in [l_lo, l_hi) (others are not counted).
 * hist: device, caller-owned, n_pairs * n_bins doubles.  Asynchronous. */
PMC_API int pmc_length_hist(pmc_chains_t chains, double l_lo, double l_hi, int n_bins, double* hist, void* stream);

/* ---------------------------------------------------------------------- */
/* Comparison baseline                                                    */
/* ---------------------------------------------------------------------- */

/* Result of a forward-tracer run: the estimate of the detected intensity per
 * emitted photon, computed in the library from the run's sums. */
typedef struct {
  double intensity;                /* sum_w / emitted */
  double std_err;                  /* sqrt((sum_w2 / emitted - intensity^2) / emitted) */
  double mean_length;              /* sum_wl / sum_w: weight-averaged path length (NaN without detections) */
  double detected, emitted;        /* photon counts */
  double sum_w, sum_w2, sum_wl;    /* over detected photons: w rho, (w rho)^2, w rho x path length */
} pmc_trace_result;

/* Forward ray tracer (appendix, "Ray tracer", Algorithm 1) for pair `pair`:
 * n_photons photons numbered from photon0, free paths from b(x), absorption
 * weights from a(x), hits tallied at the first sensor intersection,
 * rejection of a photon that starts a flight beyond r_reject from the sensor
 * centre, at most max_scatter scatterings.  out: host, caller-owned.
 * Synchronises `stream`. */
PMC_API int pmc_trace(pmc_ctx_t ctx, pmc_medium_t medium, pmc_geom_t geom, int pair,
              uint64_t seed, uint64_t photon0, uint64_t n_photons, double r_reject,
              int max_scatter, pmc_trace_result* out, void* stream);

/* pmc_trace that also bins each detected photon's weight w*rho by its path
 * length L: hist (host, caller-owned, n_bins doubles) receives the summed
 * weight of bin floor((L - l_lo) / (l_hi - l_lo) * n_bins), L in [l_lo, l_hi),
 * per emitted photon (section "Comparison of timing distributions", the ray
 * tracer's side).  out as for pmc_trace.  Synchronises `stream`. */
PMC_API int pmc_trace_lengths(pmc_ctx_t ctx, pmc_medium_t medium, pmc_geom_t geom, int pair, uint64_t seed,
                              uint64_t photon0, uint64_t n_photons, double r_reject, int max_scatter, double l_lo,
                              double l_hi, int n_bins, pmc_trace_result* out, double* hist, void* stream);

/* Allocation-free forward tracer for callers that cannot allocate device
 * memory (an application whose own pool allocator has reserved the device, a
 * fixed memory budget, or a path that must not take the device-wide
 * synchronisation of cudaMalloc / cudaFree).  The paper has no counterpart:
 * it computes what pmc_trace computes, for each of the n_pairs pairs listed
 * in pair_ids (host array), with every pair traced from photon0 with the same
 * seed, and writes one pmc_trace_result per pair to `out` (host, n_pairs
 * entries).  Its accumulators live in a fixed device array of
 * PMC_NOALLOC_MAX_PAIRS * 5 doubles that every GPU loading the library holds
 * until the process exits; the call performs no device allocation.
 *  - n_pairs must be in [1, PMC_NOALLOC_MAX_PAIRS]; larger values fail with
 *    PMC_ERR_INVALID.
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any
 *    stream capture.  The address is kept for the life of the process: a
 *    cudaDeviceReset on that device after the first call is not supported.
 *  - All calls on a device share the array: calls whose work overlaps on the
 *    GPU (other streams or other host threads) race and corrupt each other's
 *    results.  Each call clears the slots it uses before tracing.
 *  - Synchronises `stream`. */
#define PMC_NOALLOC_MAX_PAIRS 128
PMC_API int pmc_trace_noalloc(pmc_ctx_t ctx, pmc_medium_t medium, pmc_geom_t geom, const int* pair_ids,
                              int n_pairs, uint64_t seed, uint64_t photon0, uint64_t n_photons,
                              double r_reject, int max_scatter, pmc_trace_result* out, void* stream);

/* Equilibrium seeds for chains (paper: chains are seeded from ray-traced
 * paths, section "Implementation"): traces n_photons photons as pmc_trace
 * does and keeps each detected photon with probability w * rho (its weight,
 * <= 1), so every kept path is an exact draw from the normalised path density
 * truncated to max_scatter + 2 vertices.  Kept paths go to out_xyz (device,
 * [3][max_paths][stride] absolute positions, stride >= max_scatter + 2) and
 * out_n (device, [max_paths]); *n_accepted (host) counts all kept paths, also
 * those beyond max_paths.  Paths take slots in the order the GPU finishes
 * them, so which kept paths fill the first slots varies between runs (each
 * is an exact draw either way).  Synchronises `stream`. */
PMC_API int pmc_trace_paths(pmc_ctx_t ctx, pmc_medium_t medium, pmc_geom_t geom, int pair, uint64_t seed,
                            uint64_t photon0, uint64_t n_photons, double r_reject, int max_scatter, int max_paths,
                            float* out_xyz, int* out_n, int stride, uint64_t* n_accepted, void* stream);

/* Equilibrium seeds for every chain of the set (the paper seeds its chains
 * with ray-traced paths, section "Implementation"): for each pair p, photons
 * 0, 1, 2, ... of the pair's tracer (pmc_trace_paths' thinning, Philox key
 * seed + p, at most cap - 2 scatterings) are traced in rounds until at least
 * as many photons were kept as the pair has chains, and chain i of the pair
 * (its index within the pair, also when a chain window holds only some of
 * the pair's chains, so sharded sets seed exactly as the whole set) takes
 * the path of the i-th kept photon in photon order (pmc_seed_select):
 * the first kept photons of a sequential tracer, i.e. independent exact draws
 * from the normalised cap-truncated path density, whatever order the GPU
 * finds them in.  Rounds trace photons_per_round photons each, at most
 * max_rounds of them; a round that keeps more photons than its index buffer
 * (twice the largest pair's chains, at least 4,096) is traced again with
 * half the photons (and later rounds keep the smaller size).  When max_rounds
 * rounds keep fewer photons than chains, the kept paths are reused
 * cyclically (chains that share a seed then differ only by their random
 * numbers until they decorrelate).  Step
 * counters, accumulators and status words restart at zero.  photons_used
 * (host, n_pairs entries, may be NULL) receives the photons traced per pair.
 * Errors: PMC_ERR_INVALID when photons_per_round == 0, max_rounds < 1,
 * r_reject <= 0 or a pair keeps no photon at all.  Synchronises `stream`. */
PMC_API int pmc_seed_from_tracer(pmc_chains_t chains, uint64_t seed, uint64_t photons_per_round, int max_rounds,
                                 double r_reject, uint64_t* photons_used, void* stream);

/* The seed selection of pmc_seed_from_tracer (host only): out[i] = the
 * (i mod count)-th smallest of the count photon indices photon_idx (the
 * accepted photons of a traced range, in any order), i < need.  Errors:
 * PMC_ERR_INVALID for NULL pointers or count == 0 with need > 0. */
PMC_API int pmc_seed_select(const uint64_t* photon_idx, size_t count, size_t need, uint64_t* out);

/* Message of the last failure on the calling thread ("" if none). */
PMC_API const char* pmc_last_error(void);

/* Library version string. */
PMC_API const char* pmc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PATHMC_H */
