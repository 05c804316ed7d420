/*
 * FP64 CPU oracle for path-integral RJMCMC light transport
 * (Collin, "Using path integrals for the propagation of light in a
 * scattering dominated medium", arXiv:1811.04156).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline / reference legs may load this library.  The CUDA
 * product path never calls, links or imports it, and it shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Everything here is plain, slow and written to be checked by eye against
 * the paper: every proposal recomputes the full log-density from scratch,
 * in double precision.
 *
 * Functions with no pin other than the paper's text are marked
 * "parity unpinned" at their definition.
 */
#ifndef PMC_ORACLE_H
#define PMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_HOMOGENEOUS = 0, OR_LAYERED = 1 };
enum { OR_EMIT_ISOTROPIC = 0, OR_EMIT_VMF = 1 };
enum { OR_RHO_ONE = 0, OR_RHO_PAPER = 1 };
enum { OR_INIT_DIRECT = 0, OR_INIT_STRAIGHT = 1, OR_INIT_USER = 2 };
enum { OR_WITHIN_PERTURB = 0, OR_WITHIN_MALA = 1, OR_WITHIN_TREE = 2, OR_WITHIN_HMC = 3 };
enum { OR_MOVE_INTERIOR = 0, OR_MOVE_END = 1, OR_MOVE_BIRTH = 2, OR_MOVE_DEATH = 3 };

typedef struct {
  int kind;                 /* OR_HOMOGENEOUS or OR_LAYERED */
  double lambda_s;          /* scattering length (m), homogeneous */
  double lambda_a;          /* absorption length (m), homogeneous */
  double g;                 /* Gamma: mean cosine of both phase components */
  double f_sl;              /* simplified-Liu weight of the mixture */
  double z0, dz;            /* layered: bottom of layer 0 and thickness */
  int n_layers;
  const double* lambda_s_layers;
  const double* lambda_a_layers;
  /* wavelength dependence (section "Discussion"): at wavelength l the
   * scattering and absorption coefficients are b (l / lambda0)^(-k_s) and
   * a (l / lambda0)^(-k_a) (homogeneous media; k = 0: none) */
  double lambda0, k_s, k_a;
} or_medium;

typedef struct {
  double pos[3];
  int emission;             /* OR_EMIT_ISOTROPIC or OR_EMIT_VMF */
  double kappa;
  double dir[3];
} or_source;

typedef struct {
  double c[3];
  double R;
  int rho;                  /* OR_RHO_ONE or OR_RHO_PAPER */
  double rho_hat[3];
} or_sensor;

typedef struct {
  uint64_t seed;
  double p_within, p_birth, p_death;
  int within;               /* OR_WITHIN_PERTURB, _MALA, _TREE or _HMC */
  double sigma;             /* Gaussian perturbation scale (m) */
  double mala_step;         /* MALA epsilon (m) */
  double kappa_end;         /* vMF concentration of end moves (> 0) */
  uint64_t burn_in;         /* global step index from which states are recorded */
  uint32_t thin_bridge;     /* record reference-density terms every k steps (0: never) */
  int gradients;            /* accumulate score terms */
  double beta_min;          /* lower clamp of the insertion concentration */
  int hmc_steps;            /* OR_WITHIN_HMC: leapfrog steps of size mala_step */
  double toy_s;             /* > 0: sample the pins' toy target instead of the path density */
  const double* toy_w;      /* toy sector weights, indexed by vertex count (cap + 1 entries) */
  /* wavelength as a sampled coordinate: n_lambda >= 2 spectrum nodes (0: off); the
   * chains sample (path, l) from S(l) p_l(path), S piecewise linear through
   * (lambda_nm[i], spectrum[i]) normalised over [lambda_nm[0], lambda_nm[n-1]] */
  int n_lambda;
  const double* lambda_nm;
  const double* spectrum;
  double sigma_lambda;      /* Gaussian step of a wavelength move (nm) */
} or_run;

/* Per-chain accumulators (FP64 sums over recorded states). */
typedef struct {
  double n_rec;             /* recorded states */
  double n_direct;          /* recorded states with n == 2 */
  double sum_n, sum_L, sum_L2;
  double sum_score[3];      /* homogeneous scores d log p / d(lambda_s, lambda_a, g) */
  double sum_bridge;        /* sum of sqrt(q_ref / p) at thinned states */
  double n_bridge;
  double prop[4], acc[4];   /* proposals / acceptances per OR_MOVE_* */
} or_acc;

/* ---- random numbers ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_u01(uint32_t x);
void or_onb(const double n[3], double e1[3], double e2[3]);

/* ---- density factors ---- */
double or_kappa_eq(double G);
double or_log_sigma(const or_medium* m, double cos_theta);       /* per steradian */
double or_log_sigma_cos(const or_medium* m, double cos_theta);   /* over cos(theta) */
double or_log_emission(const or_source* s, const double rhat[3]);
double or_log_rho(const or_sensor* d, const double nu[3]);
double or_b_at(const or_medium* m, const double x[3]);
double or_a_at(const or_medium* m, const double x[3]);
void or_segment_depths(const or_medium* m, const double P[3], const double Q[3],
                       double* tau_a, double* tau_b);
int or_segment_hits_ball(const double P[3], const double Q[3], const double c[3], double R);

/* log p of one path, xyz = n x 3 (row per vertex). */
double or_logp(const or_medium* m, const or_source* s, const or_sensor* d,
               int n, const double* xyz);
/* d log p / d xyz (n x 3).  Returns log p. */
double or_grad_logp(const or_medium* m, const or_source* s, const or_sensor* d,
                    int n, const double* xyz, double* grad);
/* Score d log p / d theta: homogeneous theta = (lambda_s, lambda_a, g) (3 values);
 * layered theta = (lambda_s[0..L), lambda_a[0..L)) (2L values).  Returns count. */
int or_score(const or_medium* m, const or_source* s, const or_sensor* d,
             int n, const double* xyz, double* score);

/* ---- birth/death geometry (appendix, dimension matching transformation) ---- */
void or_bisph_point(const double fk[3], const double fk1[3], double s, double t, double phi,
                    double out[3]);
void or_bisph_coords(const double fk[3], const double fk1[3], const double f[3],
                     double* s, double* t, double* phi);
double or_log_bisph_jacobian(double gamma, double s, double t);
double or_log_q_s(double beta, double s);
double or_log_q_t(double t);

/* ---- chains ---- */
/* Initial states: xyz is [chains][cap][3], n is [chains]. */
int or_init_chains(const or_medium* m, const or_source* s, const or_sensor* d,
                   const or_run* r, int init_kind, int init_k, double jitter,
                   int n_chains, int cap, uint32_t chain_offset,
                   double* xyz, int* n);
/* Run n_steps steps of every chain from global step index step0.
 * min_margin (optional, per chain): smallest |log A - log u| seen over finite
 * proposals, to find near-tie decisions in trajectory comparisons. */
int or_run_chains(const or_medium* m, const or_source* s, const or_sensor* d,
                  const or_run* r, int n_chains, int cap, uint32_t chain_offset,
                  uint64_t step0, uint64_t n_steps, double* xyz, int* n,
                  or_acc* acc, double* min_margin, int n_threads);
/* Same, and adds the dwell of every recorded state to n_hist[chain][n]
 * (n_hist: n_chains x (cap + 1) doubles, may be NULL). */
int or_run_chains_hist(const or_medium* m, const or_source* s, const or_sensor* d,
                       const or_run* r, int n_chains, int cap, uint32_t chain_offset,
                       uint64_t step0, uint64_t n_steps, double* xyz, int* n,
                       or_acc* acc, double* min_margin, double* n_hist, int n_threads);
/* ---- wavelength as a sampled coordinate (section "Discussion") ---- */
/* The homogeneous medium at wavelength lam (lengths scaled by (lam/lambda0)^k). */
void or_medium_at(const or_medium* m, double lam, or_medium* out);
/* log S(lam), S the run's normalised piecewise-linear spectrum (-inf outside its range). */
double or_log_spectrum(const or_run* r, double lam);
/* The wavelength at which the spectrum's CDF equals u in [0, 1]. */
double or_spectrum_quantile(const or_run* r, double u);
/* Initial wavelengths: lam[c] = quantile of u01 of Philox counter (0, 1, chain, init). */
void or_init_lambda(const or_run* r, int n_chains, uint32_t chain_offset, double* lam);
/* Chains of (path, wavelength): or_run_chains_diag with the chains' wavelengths lam
 * (n_chains, NULL when r->n_lambda == 0) updated in place. */
int or_run_chains_lam(const or_medium* m, const or_source* s, const or_sensor* d,
                      const or_run* r, int n_chains, int cap, uint32_t chain_offset,
                      uint64_t step0, uint64_t n_steps, double* xyz, int* n, double* lam,
                      or_acc* acc, double* min_margin, double* n_hist, double* min_hmc_seg, int n_threads);

/* Same, and stores in min_hmc_seg[chain] (may be NULL) the shortest segment
 * length met at any leapfrog position of the chain's HMC moves (infinity
 * without HMC moves). */
int or_run_chains_diag(const or_medium* m, const or_source* s, const or_sensor* d,
                       const or_run* r, int n_chains, int cap, uint32_t chain_offset,
                       uint64_t step0, uint64_t n_steps, double* xyz, int* n,
                       or_acc* acc, double* min_margin, double* n_hist, double* min_hmc_seg, int n_threads);

/* ---- normalisation and reference density ---- */
double or_z2(const or_medium* m, const or_source* s, const or_sensor* d, int n_v, int n_phi);
double or_qref_logdensity(const or_medium* m, const or_source* s, const or_sensor* d,
                          int cap, int n, const double* xyz);
int or_qref_sample(const or_medium* m, const or_source* s, const or_sensor* d, int cap,
                   uint64_t seed, uint32_t stream, uint64_t draw, double* xyz);
/* sums over draws of sqrt(p/q) and of p/q: out[0] = sum sqrt(p/q), out[1] = sum p/q,
 * out[2] = sum (p/q)^2, out[3] = draws. */
int or_qref_bridge_sums(const or_medium* m, const or_source* s, const or_sensor* d, int cap,
                        uint64_t seed, uint32_t stream, uint64_t n_draws, double* out,
                        int n_threads);

/* ---- forward ray tracer (appendix, Algorithm 1) ----
 * out[0] = sum of weights of detected photons, out[1] = sum of squared weights,
 * out[2] = detected photons, out[3] = emitted photons, out[4] = sum of w*L (length). */
int or_trace(const or_medium* m, const or_source* s, const or_sensor* d,
             uint64_t seed, uint64_t photon0, uint64_t n_photons, double r_reject,
             int max_scatter, double* out, int n_threads);
/* Same, and adds each detected weight to hist[scatterings] (max_scatter + 1 doubles). */
int or_trace_hist(const or_medium* m, const or_source* s, const or_sensor* d,
                  uint64_t seed, uint64_t photon0, uint64_t n_photons, double r_reject,
                  int max_scatter, double* out, double* hist, int n_threads);

/* Same as or_trace, and adds each detected weight to lhist[bin] by its path
 * length L: bin = floor((L - l_lo) / (l_hi - l_lo) * l_bins), L in [l_lo, l_hi). */
int or_trace_lhist(const or_medium* m, const or_source* s, const or_sensor* d,
                   uint64_t seed, uint64_t photon0, uint64_t n_photons, double r_reject,
                   int max_scatter, double l_lo, double l_hi, int l_bins, double* out, double* lhist,
                   int n_threads);

/* ---- relative light yield of two sensors (section "Comparison of relative
 *      light yield"; appendix, "Relative light yield transformation") ---- */
typedef struct {
  double f0[3], eta0[3], eta1[3];
  double R0, R1;
  double k[3], m[3], n[3];  /* frame: k towards sensor 0, m in the (k, B) plane away from B, n = k x m */
  double b0, b1, rC, Omega;
} or_ymap;
/* Map of source s and sensors d0 -> d1; -1 if the sensors are collinear with the source. */
int or_ymap_init(const or_source* s, const or_sensor* d0, const or_sensor* d1, or_ymap* T);
/* y = T(x) for an n-vertex path ending on sensor 0 (n x 3 rows); returns log |dT/dx|
 * (interior volume ratios and the end vertex's area ratio), -inf outside the one-to-one domain. */
double or_ymap_forward(const or_ymap* T, int n, const double* x, double* y);
/* x = T^-1(y) for a path ending on sensor 1; returns log |dT/dx| at x, -inf outside the domain. */
double or_ymap_inverse(const or_ymap* T, int n, const double* y, double* x);
/* Log of the geometric estimator's ratio at one path: side 0 (path on sensor 0):
 * log p_1(x) - log p_0(x) = log p(T x; d1) + log|dT/dx| - log p(x; d0); side 1
 * (path y on sensor 1): log p_0(x) - log p_1(x) with x = T^-1 y.  -inf where the
 * other density is zero. */
double or_ymap_logratio(const or_medium* m, const or_source* s, const or_sensor* d0, const or_sensor* d1,
                        const or_ymap* T, int side, int n, const double* path);

/* ---- tree coordinates (appendix "Path space coordinate system", Fig.
 *      tree_coords; section "Path proposal distribution") ----
 * Interior vertex m of an n-vertex path sits in the bispherical system of its
 * tree foci f_k, f_l (root: f_0, f_{n-1}; m = floor((k + l)/2)) with
 * coordinates (zeta, t, phi): cos s = tanh zeta, t = ln(d1/d2), and phi the
 * azimuth of f_m - (f_k + f_l)/2 about e = (f_l - f_k)/|f_l - f_k| in the
 * node's frame (xi, eta): eta = the unit normal e_p x (f_p - mid_p) of the
 * parent's triangle (the inherited axes rotated by the parent's phi), xi =
 * eta x e; the root's xi is v_ref projected onto the plane normal to e. */
/* Foci (k, l) and parent node (-1 for the root) of interior vertex m. */
void or_tree_node(int m, int n, int* k, int* l, int* parent);
/* coords[3 m + (0, 1, 2)] = (zeta, t, phi) of interior vertex m (1..n-2);
 * returns sum over nodes of log |d f_m / d(zeta, t, phi)| =
 * 3 log(d1 d2 / (2 gamma)) + 2 log sin s. */
double or_tree_coords(const double v_ref[3], int n, const double* path, double* coords);
/* Path from f_0 = path[0..2], f_{n-1} = path[3(n-1)..] and the coordinates of
 * the interior vertices (top-down); writes path[3..3(n-1)). */
void or_tree_path(const double v_ref[3], int n, const double* coords, double* path);
/* The HMC move's deterministic part: L leapfrog steps of size eps of the
 * interior vertices x with momenta p (both n x 3, updated in place; the
 * source and the end vertex are held), force d log p / d f (zero where
 * p = 0).  Returns log p at the end point. */
double or_hmc_leapfrog(const or_medium* m, const or_source* s, const or_sensor* d, int n, double* x, double* p,
                       double eps, int L);
/* The root frame's reference vector of a pair: the first vector of the
 * orthonormal completion of the unit source -> sensor-centre direction. */
void or_tree_vref(const or_source* s, const or_sensor* d, double v_ref[3]);

#ifdef __cplusplus
}
#endif
#endif
