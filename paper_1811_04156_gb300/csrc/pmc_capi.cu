// C ABI of libpathmc (declared in include/pathmc.h): handle management,
// validation, device buffers, CUDA-graph replay of the chain launches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <tuple>
#include <memory>
#include <string>
#include <vector>

#include "pmc_internal.h"

using namespace pmc;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      if (e_ == cudaErrorMemoryAllocation) return fail(PMC_ERR_OOM, cudaGetErrorString(e_));  \
      return fail(PMC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
    }                                                                                         \
  } while (0)

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

double norm3(const double* v) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

// Gauss-Legendre nodes and weights on [-1, 1]: Newton iteration on P_n from
// the Chebyshev guesses, P_n by the three-term recurrence.
void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int k = 1; k <= n; ++k) {
        const double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
      }
      dp = n * (z * p0 - p1) / (z * z - 1.0);
      const double dz = p0 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-15) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Inverse Langevin: coth(k) - 1/k = g (appendix, dimension matching transformation).
double kappa_eq_host(double g) {
  if (g <= 0.0) return 0.0;
  double k = 3.0 * g / (1.0 - g * g);
  for (int it = 0; it < 200; ++it) {
    const double f = 1.0 / std::tanh(k) - 1.0 / k - g;
    const double sh = std::sinh(k);
    const double df = (k > 300.0 ? 0.0 : -1.0 / (sh * sh)) + 1.0 / (k * k);
    double kn = k - f / df;
    if (kn <= 0.0) kn = 0.5 * k;
    if (std::fabs(kn - k) < 1e-14 * k) {
      k = kn;
      break;
    }
    k = kn;
  }
  return k;
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

constexpr int kClassCaps[] = {64, 128, 256, 512, 1024};
constexpr int kMaxCap = 1024;

}  // namespace

struct pmc_ctx_s {
  int device = 0;
  int n_sm = 0;
  size_t smem_per_sm = 0, smem_per_block = 0;
  // autotuned warps per block, keyed by (kernel instantiation, shared vertex cap, chain-count bucket)
  std::map<std::tuple<int, int, int>, std::tuple<int, int, int>> tuned;  // -> (warps per block, shared window, kind)
};

struct pmc_medium_s {
  pmc_ctx_s* ctx = nullptr;
  DMedium d{};
  float* d_la = nullptr;
  float* d_lb = nullptr;
  float* d_llogb = nullptr;
  double lambda_s = 0, lambda_a = 0;
  int n_theta = 3;
  double z0 = 0, dz = 1;
  std::vector<double> ls_layers, la_layers;
};

struct PairHost {
  double src[3], c[3], R;
  int emission;
  double kappa, dir[3];
  int rho;
  double rho_hat[3];
  int cap, n_chains, chain0;
};

// Pair constants in a frame: origin at the source (chains, tracer) or at the
// absolute origin (density kernels on caller batches).  The sensor centre is
// split into FP32 high and low parts.
static DPair make_dpair(const PairHost& h, bool source_frame) {
  DPair d{};
  double org[3] = {0, 0, 0};
  if (source_frame)
    for (int i = 0; i < 3; ++i) org[i] = h.src[i];
  double rel[3];
  for (int i = 0; i < 3; ++i) {
    d.org[i] = static_cast<float>(org[i]);
    d.src[i] = static_cast<float>(h.src[i] - org[i]);
    const double cc = h.c[i] - org[i];
    d.c[i] = static_cast<float>(cc);
    d.c_lo[i] = static_cast<float>(cc - static_cast<double>(d.c[i]));
    rel[i] = h.c[i] - h.src[i];
  }
  d.zoff = static_cast<float>(org[2]);
  const double D = norm3(rel);
  for (int i = 0; i < 3; ++i) d.e_near[i] = static_cast<float>(h.src[i] - org[i] + rel[i] - h.R * rel[i] / D);
  d.R = static_cast<float>(h.R);
  d.R2 = d.R * d.R;
  d.emission = h.emission;
  if (h.emission == PMC_EMIT_VMF) {
    const double nd = norm3(h.dir);
    for (int i = 0; i < 3; ++i) d.dir[i] = static_cast<float>(h.dir[i] / nd);
    d.kappa = static_cast<float>(h.kappa);
    const double k = h.kappa;
    d.vmf_lognorm = static_cast<float>(std::log(k) - std::log(2.0 * M_PI) - k - std::log(-std::expm1(-2.0 * k)));
  }
  d.rho = h.rho;
  if (h.rho == PMC_RHO_PAPER) {
    const double nr = norm3(h.rho_hat);
    for (int i = 0; i < 3; ++i) d.rho_hat[i] = static_cast<float>(h.rho_hat[i] / nr);
  }
  d.cap = h.cap;
  d.n_chains = h.n_chains;
  d.chain0 = h.chain0;
  return d;
}

struct pmc_geom_s {
  pmc_ctx_s* ctx = nullptr;
  std::vector<PairHost> host;
  std::vector<DPair> pairs;      // source frame: chains and tracer
  std::vector<DPair> abs_pairs;  // absolute frame: pmc_logp, pmc_logp_grad, pmc_score
  int total_chains = 0;
  int max_cap = 0;
};

struct ChainClass {
  int kind = 0;       // kernel kind of launch_chain (4: one lane per chain)
  bool short_paths = false;  // every pair expects <= kLaneMaxN vertices (lane layout candidate)
  int smem_cap = 0;   // shared window (vertices per chain)
  int max_cap = 0;    // largest vertex cap of the class's chains
  bool spill = false; // smem_cap < max_cap: entries beyond the window live in global memory
  int lo = 0, hi = 0;  // range into the processing order
  int warps_per_block = 4;
  int grid = 0;
};

struct pmc_chains_s {
  pmc_ctx_s* ctx = nullptr;
  pmc_medium_s* med = nullptr;
  pmc_geom_s* geom = nullptr;
  DRun run{};
  int flags = 0;
  int total = 0;
  int n_pairs = 0;
  std::vector<DPair> h_pairs;
  std::vector<long long> h_base;
  std::vector<int> h_pair_of;
  std::vector<int> h_pair_first;  // per pair: index within the pair of the window's first chain
  long long xyz_floats = 0;
  DPair* d_pairs = nullptr;
  int* d_chain_pair = nullptr;
  long long* d_chain_base = nullptr;
  int* d_order = nullptr;
  float* d_xyz = nullptr;
  int* d_n = nullptr;
  unsigned long long* d_step = nullptr;
  double* d_acc = nullptr;
  int* d_status = nullptr;
  int* d_any = nullptr;
  unsigned int* d_queue = nullptr;
  double* d_z2 = nullptr;
  std::vector<double> h_z2;        // host copy of d_z2 (filled at the first estimate)
  double* d_est = nullptr;         // per-pair moments [n_pairs][PMC_MOMENT_WORDS]
  long long chain_lo = 0;          // this set holds the geometry's chains [chain_lo, chain_lo + total)
  int* h_abort = nullptr;
  int* d_abort = nullptr;
  cudaStream_t capture_stream = nullptr;
  std::vector<ChainClass> classes;
  std::map<unsigned long long, cudaGraphExec_t> graphs;
  int general = 0;                 // chain kernel: 0 lean, 1 general, 2 with tree moves, 3 with HMC moves
  bool grad = false;               // keep d log sigma / dg per vertex
  bool autotune = false;           // warps per block chosen by timing
  int layout = PMC_LAYOUT_AUTO;    // PMC_LAYOUT_*: which chain layouts the autotuner may pick
  int lane_kind = 0;               // lane layout's kernel kind (4 Gaussian, 5 MALA, 8 tree moves); 0: not eligible
  int init_kind = 0, init_k = 0;
  float init_jitter = 0.f;
  QrefPair* d_qp = nullptr;       // reference-density tables (pmc_bridge)
  double* d_qtab = nullptr;
  double* d_bsum = nullptr;
  float* d_stage = nullptr;       // staging buffer of pmc_set_states
  int* d_stage_n = nullptr;
  size_t stage_floats = 0;
  bool lam_on = false;             // wavelength sampled with the path
  float* d_lam = nullptr;          // [total] the chains' wavelengths
  float* d_spec = nullptr;         // [2][n_spec] spectrum nodes (nm) and normalised densities
  std::vector<double> spec_x, spec_y;  // host copy (normalised densities)
};

// Scattering depth of the straight segment from the source to the sensor
// point nearest it (host, FP64): the mean of the truncated Poisson law of the
// reference density's vertex count.
static double straight_tau_b(const pmc_medium_s* m, const PairHost& h) {
  double rel[3], e[3];
  for (int i = 0; i < 3; ++i) rel[i] = h.c[i] - h.src[i];
  const double D = norm3(rel);
  for (int i = 0; i < 3; ++i) e[i] = h.src[i] + rel[i] * (D - h.R) / D;
  const double ell = D - h.R;
  if (m->d.kind == PMC_HOMOGENEOUS) return ell / m->lambda_s;
  const int L = static_cast<int>(m->ls_layers.size());
  auto layer = [&](double z) {
    double f = std::floor((z - m->z0) / m->dz);
    if (f < 0) f = 0;
    if (f > L - 1) f = L - 1;
    return static_cast<int>(f);
  };
  const double zP = h.src[2], zQ = e[2];
  const int lP = layer(zP), lQ = layer(zQ);
  if (lP == lQ) return ell / m->ls_layers[lP];
  const double zlo = std::min(zP, zQ), zhi = std::max(zP, zQ);
  double acc = 0.0;
  for (int l = std::min(lP, lQ); l <= std::max(lP, lQ); ++l) {
    const double lo = (l == std::min(lP, lQ)) ? zlo : m->z0 + l * m->dz;
    const double hi = (l == std::max(lP, lQ)) ? zhi : m->z0 + (l + 1) * m->dz;
    acc += std::max(hi - lo, 0.0) / (zhi - zlo) / m->ls_layers[l];
  }
  return ell * acc;
}

// Reference-density tables of every pair: truncated Poisson law of the vertex
// count (log P and CDF over n = 0..cap) and the visible-cap area term.
static void build_qref(const pmc_medium_s* m, const std::vector<PairHost>& host, std::vector<QrefPair>& qp,
                       std::vector<double>& tab) {
  qp.resize(host.size());
  tab.clear();
  for (size_t p = 0; p < host.size(); ++p) {
    const PairHost& h = host[p];
    const double mu = straight_tau_b(m, h);
    const int cap = h.cap;
    double norm = 0.0;
    for (int k = 0; k <= cap - 2; ++k) norm += std::exp(k * std::log(mu) - mu - std::lgamma(k + 1.0));
    qp[p].off = static_cast<long long>(tab.size());
    std::vector<double> lp(cap + 1, -std::numeric_limits<double>::infinity()), cdf(cap + 1, 0.0);
    double cum = 0.0;
    for (int n = 2; n <= cap; ++n) {
      const int k = n - 2;
      lp[n] = k * std::log(mu) - mu - std::lgamma(k + 1.0) - std::log(norm);
      cum += std::exp(lp[n]);
      cdf[n] = cum;
    }
    tab.insert(tab.end(), lp.begin(), lp.end());
    tab.insert(tab.end(), cdf.begin(), cdf.end());
    double rel[3];
    for (int i = 0; i < 3; ++i) rel[i] = h.c[i] - h.src[i];
    const double D = norm3(rel);
    qp[p].log_qend = -std::log(2.0 * M_PI * h.R * h.R * (1.0 - h.R / D));
  }
}

static DRun qref_run() {
  DRun r{};
  r.beta_min = 0.01f;
  return r;
}

namespace pmc {

// Tracer estimate from the kernel's raw sums (sum w rho, sum (w rho)^2,
// detected, emitted, sum w rho L): the mean detected weight per emitted
// photon with its standard error, and the weight-averaged path length.
pmc_trace_result trace_result(const double* raw) {
  pmc_trace_result r{};
  const double N = raw[3];
  r.sum_w = raw[0];
  r.sum_w2 = raw[1];
  r.detected = raw[2];
  r.emitted = N;
  r.sum_wl = raw[4];
  const double nan = std::numeric_limits<double>::quiet_NaN();
  r.intensity = N > 0 ? raw[0] / N : nan;
  r.std_err = N > 0 ? std::sqrt(std::max(raw[1] / N - r.intensity * r.intensity, 0.0) / N) : nan;
  r.mean_length = raw[0] > 0 ? raw[4] / raw[0] : nan;
  return r;
}

// Estimate of one pair from the sums of its chains' accumulators (pmc_moments
// layout; see add_chain_moments).  With f_c = n2_c / N_c a chain's fraction
// of direct paths and w_c = N_c / N, the across-chain variance of pi(n = 2)
// is sum w_c^2 (f_c - pi)^2 C / (C - 1) = (sum n2^2 - 2 pi sum N n2 +
// pi^2 sum N^2) / N^2 * C / (C - 1), and likewise for the score means s_c =
// A_c / N_c and their covariance with pi; I = Z2 / pi (direct-sector
// anchor), its standard error I sqrt(var pi) / pi; the gradient I * s by the
// delta method.  R-hat (Gelman-Rubin) is on the path length over chains.
void estimate_of_moments(const double* m, double z2, pmc_estimate* o, double* grad, double* grad_se) {
  const double nan = std::numeric_limits<double>::quiet_NaN();
  const double N = m[MOM_ACC + ACC_NREC];
  const double C = m[MOM_NCHAIN];
  const double pi = N > 0 ? m[MOM_ACC + ACC_NDIRECT] / N : 0.0;
  const double corr = C > 1 ? C / (C - 1.0) : 1.0;
  const double N2 = N * N;
  const double var_pi =
      N > 0 ? std::max(m[MOM_N2SQ] - 2.0 * pi * m[MOM_NN2] + pi * pi * m[MOM_NSQ], 0.0) / N2 * corr : 0.0;
  const double I = pi > 0 ? z2 / pi : nan;
  const double se = pi > 0 ? I * std::sqrt(var_pi) / pi : I;
  *o = pmc_estimate{};
  o->intensity = I;
  o->std_err = se;
  o->rel_err = se / I;
  o->pi_direct = pi;
  o->z2 = z2;
  double rhat = nan;
  const double K = m[MOM_RH_K];
  if (K > 1) {
    const double W = m[MOM_RH_VAR] / K;
    const double mbar = m[MOM_RH_M] / K;
    const double B_over_n = (m[MOM_RH_M2] / K - mbar * mbar) * K / (K - 1.0);
    const double nper = N / K;
    if (W > 0) rhat = std::sqrt(((nper - 1.0) / nper * W + B_over_n) / W);
  }
  o->rhat = rhat;
  for (int k = 0; k < 4; ++k) {
    const double pr = m[MOM_ACC + ACC_PROP + k];
    o->accept[k] = pr > 0 ? m[MOM_ACC + ACC_ACC + k] / pr : 0.0;
    o->proposals[k] = pr;
  }
  o->mean_n = N > 0 ? m[MOM_ACC + ACC_SUMN] / N : 0.0;
  o->mean_length = N > 0 ? m[MOM_ACC + ACC_SUML] / N : 0.0;
  o->n_samples = N;
  o->ess = var_pi > 0 ? pi * (1.0 - pi) / var_pi : 0.0;
  o->bridge_intensity = nan;
  o->bridge_std_err = nan;
  for (int k = 0; k < 3; ++k) {
    const double sbar = N > 0 ? m[MOM_A + k] / N : 0.0;
    const double vs = N > 0 ? std::max(m[MOM_ASQ + k] - 2.0 * sbar * m[MOM_NA + k] + sbar * sbar * m[MOM_NSQ], 0.0) /
                                  N2 * corr
                            : 0.0;
    const double cv = N > 0 ? (m[MOM_N2A + k] - sbar * m[MOM_NN2] - pi * m[MOM_NA + k] + pi * sbar * m[MOM_NSQ]) /
                                  N2 * corr
                            : 0.0;
    const double dpi = pi > 0 ? I * sbar / pi : 0.0;
    if (grad) grad[k] = I * sbar;
    if (grad_se) grad_se[k] = std::sqrt(std::max(I * I * vs + dpi * dpi * var_pi - 2.0 * I * dpi * cv, 0.0));
  }
}

}  // namespace pmc

extern "C" {

const char* pmc_last_error(void) { return g_err.c_str(); }

const char* pmc_version(void) { return "pathmc 0.1 (sm_103a)"; }

int pmc_create_context(int device, pmc_ctx_t* out) {
  if (out == nullptr) return fail(PMC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) return fail(PMC_ERR_NO_DEVICE, "no CUDA device available");
  if (device < 0 || device >= count) return fail(PMC_ERR_NO_DEVICE, "device index out of range");
  CK(cudaSetDevice(device));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, device));
  auto* c = new pmc_ctx_s;
  c->device = device;
  c->n_sm = prop.multiProcessorCount;
  c->smem_per_sm = prop.sharedMemPerMultiprocessor;
  c->smem_per_block = prop.sharedMemPerBlockOptin;
  *out = c;
  return PMC_OK;
}

int pmc_destroy_context(pmc_ctx_t ctx) {
  delete ctx;
  return PMC_OK;
}

int pmc_create_medium(pmc_ctx_t ctx, const pmc_medium_desc* desc, pmc_medium_t* out) {
  if (ctx == nullptr || desc == nullptr || out == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  *out = nullptr;
  const double g = desc->g, f = desc->f_sl;
  if (!std::isfinite(g) || std::fabs(g) >= 1.0) return fail(PMC_ERR_INVALID, "|g| must be < 1");
  if (!(f >= 0.0 && f <= 1.0)) return fail(PMC_ERR_INVALID, "f_sl must be in [0, 1]");
  if (f > 0.0 && !(g > 0.0)) return fail(PMC_ERR_INVALID, "the simplified-Liu component needs g > 0");
  CK(cudaSetDevice(ctx->device));
  auto m = std::make_unique<pmc_medium_s>();
  m->ctx = ctx;
  DMedium& d = m->d;
  d.kind = desc->kind;
  d.g = static_cast<float>(g);
  d.f_sl = static_cast<float>(f);
  d.hg_lognorm = static_cast<float>(std::log(0.5 * (1.0 - g * g)) - std::log(2.0 * M_PI));
  d.omg2 = static_cast<float>((1.0 - g) * (1.0 - g));
  d.two_g = static_cast<float>(2.0 * g);
  d.hg_dg0 = static_cast<float>(-2.0 * g / (1.0 - g * g));
  if (g > 0.0) {
    d.sl_alpha = static_cast<float>(2.0 * g / (1.0 - g));
    d.sl_lognorm = static_cast<float>(std::log(0.5 * (1.0 + g) / (1.0 - g)) - std::log(2.0 * M_PI));
  }
  d.sl_dg0 = static_cast<float>(2.0 / (1.0 - g * g));
  d.sl_dg1 = static_cast<float>(2.0 / ((1.0 - g) * (1.0 - g)));
  d.kappa_eq = static_cast<float>(kappa_eq_host(g));
  if (!(desc->k_s >= 0.0 && desc->k_a >= 0.0 && desc->lambda0 >= 0.0) || !std::isfinite(desc->k_s) ||
      !std::isfinite(desc->k_a) || !std::isfinite(desc->lambda0))
    return fail(PMC_ERR_INVALID, "wavelength law: lambda0, k_s, k_a must be finite and >= 0");
  if ((desc->k_s > 0.0 || desc->k_a > 0.0) && !(desc->lambda0 > 0.0))
    return fail(PMC_ERR_INVALID, "a wavelength-dependent medium needs lambda0 > 0");
  d.lam0 = static_cast<float>(desc->lambda0 > 0.0 ? desc->lambda0 : 1.0);
  d.ks = static_cast<float>(desc->k_s);
  d.ka = static_cast<float>(desc->k_a);
  if (desc->kind == PMC_HOMOGENEOUS) {
    if (!finite_pos(desc->lambda_s) || !finite_pos(desc->lambda_a))
      return fail(PMC_ERR_INVALID, "lambda_s and lambda_a must be finite and > 0");
    d.a = static_cast<float>(1.0 / desc->lambda_a);
    d.b = static_cast<float>(1.0 / desc->lambda_s);
    d.log_b = static_cast<float>(-std::log(desc->lambda_s));
    m->lambda_s = desc->lambda_s;
    m->lambda_a = desc->lambda_a;
    m->n_theta = 3;
  } else if (desc->kind == PMC_LAYERED) {
    const int L = desc->n_layers;
    if (L < 1 || L > 4096) return fail(PMC_ERR_INVALID, "n_layers must be in [1, 4096]");
    if (!finite_pos(desc->dz) || !std::isfinite(desc->z0)) return fail(PMC_ERR_INVALID, "bad layer geometry");
    if (desc->lambda_s_layers == nullptr || desc->lambda_a_layers == nullptr)
      return fail(PMC_ERR_INVALID, "layer tables are NULL");
    std::vector<float> la(L), lb(L), llb(L);
    for (int l = 0; l < L; ++l) {
      const double s = desc->lambda_s_layers[l], a = desc->lambda_a_layers[l];
      if (!finite_pos(s) || !finite_pos(a)) return fail(PMC_ERR_INVALID, "layer lengths must be finite and > 0");
      la[l] = static_cast<float>(1.0 / a);
      lb[l] = static_cast<float>(1.0 / s);
      llb[l] = static_cast<float>(-std::log(s));
    }
    CK(dalloc(&m->d_la, L));
    CK(dalloc(&m->d_lb, L));
    CK(dalloc(&m->d_llogb, L));
    CK(cudaMemcpy(m->d_la, la.data(), L * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d_lb, lb.data(), L * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d_llogb, llb.data(), L * sizeof(float), cudaMemcpyHostToDevice));
    m->z0 = desc->z0;
    m->dz = desc->dz;
    m->ls_layers.assign(desc->lambda_s_layers, desc->lambda_s_layers + L);
    m->la_layers.assign(desc->lambda_a_layers, desc->lambda_a_layers + L);
    d.n_layers = L;
    d.z0 = static_cast<float>(desc->z0);
    d.dz = static_cast<float>(desc->dz);
    d.inv_dz = static_cast<float>(1.0 / desc->dz);
    d.la = m->d_la;
    d.lb = m->d_lb;
    d.llogb = m->d_llogb;
    m->n_theta = 2 * L;
  } else {
    return fail(PMC_ERR_INVALID, "unknown medium kind");
  }
  *out = m.release();
  return PMC_OK;
}

int pmc_destroy_medium(pmc_medium_t m) {
  if (m == nullptr) return PMC_OK;
  cudaFree(m->d_la);
  cudaFree(m->d_lb);
  cudaFree(m->d_llogb);
  delete m;
  return PMC_OK;
}

int pmc_n_theta(pmc_medium_t m) { return m ? m->n_theta : 0; }

int pmc_create_geometry(pmc_ctx_t ctx, const pmc_geometry_desc* desc, pmc_geom_t* out) {
  if (ctx == nullptr || desc == nullptr || out == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (desc->n_pairs < 1 || desc->pairs == nullptr) return fail(PMC_ERR_INVALID, "no pairs");
  if (desc->n_sources < 1 || desc->sources == nullptr || desc->n_sensors < 1 || desc->sensors == nullptr)
    return fail(PMC_ERR_INVALID, "no sources or sensors");
  auto g = std::make_unique<pmc_geom_s>();
  g->ctx = ctx;
  long long total = 0;
  for (int p = 0; p < desc->n_pairs; ++p) {
    const pmc_pair& pr = desc->pairs[p];
    if (pr.source < 0 || pr.source >= desc->n_sources || pr.sensor < 0 || pr.sensor >= desc->n_sensors)
      return fail(PMC_ERR_INVALID, "pair refers to a missing source or sensor");
    if (pr.n_chains < 1) return fail(PMC_ERR_INVALID, "n_chains must be >= 1");
    if (pr.cap < 2 || pr.cap > kMaxCap) return fail(PMC_ERR_INVALID, "cap must be in [2, 1024]");
    const pmc_source& so = desc->sources[pr.source];
    const pmc_sensor& se = desc->sensors[pr.sensor];
    if (!finite_pos(se.radius)) return fail(PMC_ERR_INVALID, "sensor radius must be > 0");
    PairHost h{};
    double rel[3];
    for (int i = 0; i < 3; ++i) {
      if (!std::isfinite(so.pos[i]) || !std::isfinite(se.centre[i])) return fail(PMC_ERR_INVALID, "non-finite position");
      h.src[i] = so.pos[i];
      h.c[i] = se.centre[i];
      rel[i] = se.centre[i] - so.pos[i];
    }
    const double D = norm3(rel);
    if (!(D > se.radius * (1.0 + 1e-6))) return fail(PMC_ERR_INVALID, "source inside or on its sensor");
    h.R = se.radius;
    h.emission = so.emission;
    if (so.emission == PMC_EMIT_VMF) {
      if (!finite_pos(so.kappa)) return fail(PMC_ERR_INVALID, "vMF kappa must be > 0");
      if (!(norm3(so.dir) > 0)) return fail(PMC_ERR_INVALID, "zero emission direction");
      h.kappa = so.kappa;
      for (int i = 0; i < 3; ++i) h.dir[i] = so.dir[i];
    } else if (so.emission != PMC_EMIT_ISOTROPIC) {
      return fail(PMC_ERR_INVALID, "unknown emission kind");
    }
    h.rho = se.rho;
    if (se.rho == PMC_RHO_PAPER) {
      if (!(norm3(se.rho_hat) > 0)) return fail(PMC_ERR_INVALID, "zero rho_hat");
      for (int i = 0; i < 3; ++i) h.rho_hat[i] = se.rho_hat[i];
    } else if (se.rho != PMC_RHO_ONE) {
      return fail(PMC_ERR_INVALID, "unknown detection kind");
    }
    h.cap = pr.cap;
    h.n_chains = pr.n_chains;
    h.chain0 = static_cast<int>(total);
    total += pr.n_chains;
    if (total > (1ll << 30)) return fail(PMC_ERR_INVALID, "too many chains");
    g->host.push_back(h);
    g->pairs.push_back(make_dpair(h, true));
    g->abs_pairs.push_back(make_dpair(h, false));
    g->max_cap = std::max(g->max_cap, pr.cap);
  }
  g->total_chains = static_cast<int>(total);
  *out = g.release();
  return PMC_OK;
}

int pmc_destroy_geometry(pmc_geom_t g) {
  delete g;
  return PMC_OK;
}

static int class_of(int cap) {
  for (int i = 0; i < 5; ++i)
    if (cap <= kClassCaps[i]) return i;
  return 4;
}

int pmc_destroy_chains(pmc_chains_t ch) {
  if (ch == nullptr) return PMC_OK;
  cudaSetDevice(ch->ctx->device);
  for (auto& kv : ch->graphs) cudaGraphExecDestroy(kv.second);
  if (ch->capture_stream) cudaStreamDestroy(ch->capture_stream);
  cudaFree(ch->d_pairs);
  cudaFree(ch->d_chain_pair);
  cudaFree(ch->d_chain_base);
  cudaFree(ch->d_order);
  cudaFree(ch->d_xyz);
  cudaFree(ch->d_n);
  cudaFree(ch->d_step);
  cudaFree(ch->d_acc);
  cudaFree(ch->d_status);
  cudaFree(ch->d_any);
  cudaFree(ch->d_queue);
  cudaFree(ch->d_z2);
  cudaFree(ch->d_est);
  cudaFree(ch->d_stage);
  cudaFree(ch->d_stage_n);
  cudaFree(ch->d_qp);
  cudaFree(ch->d_qtab);
  cudaFree(ch->d_bsum);
  cudaFree(ch->d_lam);
  cudaFree(ch->d_spec);
  if (ch->h_abort) cudaFreeHost(ch->h_abort);
  delete ch;
  return PMC_OK;
}

// The lane layout pays for a path's length at every birth and death (its
// scans run sequentially over the lane's own path and the warp waits for its
// longest one), the warp layout spreads it over 32 lanes: the autotuner
// offers the lane layout only to classes whose pairs expect short paths,
// 2 + D b <= kLaneMaxN vertices on the straight source-sensor line (D the
// distance, b the scattering coefficient).  A short probe from the initial
// states cannot see this, since those paths have not grown yet.
constexpr double kLaneMaxN = 24.0;

// Work items of a launch: one per chain, or one per 32 chains (lane layout).
static int work_items(int kind, int chains) { return lane_kind(kind) ? (chains + 31) / 32 : chains; }

static ChainParams class_params(pmc_chains_t ch, size_t k, unsigned long long n_steps) {
  const ChainClass& cl = ch->classes[k];
  ChainParams p{};
  p.M = ch->med->d;
  p.R = ch->run;
  p.pairs = ch->d_pairs;
  p.chain_pair = ch->d_chain_pair;
  p.chain_base = ch->d_chain_base;
  p.order = ch->d_order;
  p.xyz = ch->d_xyz;
  p.n = ch->d_n;
  p.step = ch->d_step;
  p.acc = ch->d_acc;
  p.status = ch->d_status;
  p.any_status = ch->d_any;
  p.queue = ch->d_queue + k;
  p.abort_flag = ch->d_abort;
  p.chain_id0 = static_cast<uint32_t>(ch->chain_lo);
  p.lam = ch->d_lam;
  p.chain_lo = cl.lo;
  p.chain_hi = cl.hi;
  p.n_steps = n_steps;
  p.smem_cap = cl.smem_cap;
  return p;
}

// Autotuner: for every cap class, time the chain kernel over candidate launch
// shapes — 1, 2 or 4 warps per block; with one warp per chain a shared
// window of the whole cap or of 128 / 256 / 512 vertices (entries beyond it
// in global memory); with one lane per chain (lean runs with short paths) a
// per-lane window of 8 to 32 vertices — on a scratch copy of the freshly initialised
// state (256 steps, best of two probes), and keep the fastest; choices are
// cached per device, kernel, layout request and class.
static int autotune_classes(pmc_chains_t ch, cudaStream_t s) {
  const int T = ch->total;
  float* sx = nullptr;
  int* sn = nullptr;
  unsigned long long* sst = nullptr;
  double* sacc = nullptr;
  int* sstat = nullptr;
  float* slam = nullptr;  // wavelength sampling: the probes' copy of the wavelengths
  // cache key: the warp kernel instance, the layout request and which lane
  // kernel (if any) the run may use; per class also whether its paths are short
  const int kind = (((ch->general * 2 + ch->grad) * 3 + ch->layout) * 16 + ch->lane_kind) * 2;
  auto bucket_of = [](int chains) { return 31 - __builtin_clz(static_cast<unsigned>(std::max(1, chains))); };
  bool need = false;
  for (auto& cl : ch->classes)
    if (!ch->ctx->tuned.count(std::make_tuple(kind + cl.short_paths, cl.max_cap, bucket_of(cl.hi - cl.lo))))
      need = true;
  if (need) {
    CK(dalloc(&sx, static_cast<size_t>(ch->xyz_floats)));
    CK(dalloc(&sn, T));
    CK(dalloc(&sst, T));
    CK(dalloc(&sacc, static_cast<size_t>(T) * ACC_WORDS));
    CK(dalloc(&sstat, T));
    if (ch->lam_on) CK(dalloc(&slam, T));
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = PMC_OK;
  for (size_t k = 0; k < ch->classes.size() && rc == PMC_OK; ++k) {
    ChainClass& cl = ch->classes[k];
    const int chains = cl.hi - cl.lo;
    const int full = (cl.max_cap + 31) / 32 * 32;
    const auto key = std::make_tuple(kind + cl.short_paths, cl.max_cap, bucket_of(chains));
    auto it = ch->ctx->tuned.find(key);
    std::tuple<int, int, int> best(cl.warps_per_block, cl.smem_cap, cl.kind);
    if (it != ch->ctx->tuned.end()) {
      best = it->second;
    } else {
      float best_ms = 1e30f;
      struct LaneProbe {
        float ms;
        int wpb, win, kind;
        bool resident;  // the grid holds every work item at once
      };
      std::vector<LaneProbe> lane_probes;
      // candidates (kind, shared window): the warp layout with the whole cap
      // or a window with global spill (tree and HMC moves keep the whole
      // cap); the lane layout (lean runs with short paths) with per-lane
      // windows of 8 to 32 vertices
      std::vector<std::pair<int, int>> cands;
      if (ch->layout != PMC_LAYOUT_LANE) {
        cands.emplace_back(ch->general, full);
        for (int w : {128, 256, 512})
          if (w < full && ch->general < 2) cands.emplace_back(ch->general, w);
      }
      if (ch->layout == PMC_LAYOUT_LANE ||
          (ch->layout == PMC_LAYOUT_AUTO && ch->lane_kind != 0 && cl.short_paths))
        for (int w : {8, 12, 16, 20, 24, 32}) {
          cands.emplace_back(ch->lane_kind, std::min(w, cl.max_cap));
          if (w >= cl.max_cap) break;
        }
      for (const auto& cand : cands) {
        const int ckind = cand.first, win = cand.second;
        for (int wpb : {1, 2, 4}) {
          const bool spill = !lane_kind(ckind) && win < full;
          if (chain_smem_bytes(win, wpb, ckind, ch->grad) > ch->ctx->smem_per_block) continue;
          int bps = 0;
          if (chain_occupancy(ckind, ch->grad, spill, wpb, win, &bps) != cudaSuccess || bps < 1) continue;
          const int grid = std::max(1, std::min((work_items(ckind, chains) + wpb - 1) / wpb, bps * ch->ctx->n_sm));
          ChainParams p = class_params(ch, k, 256);
          p.smem_cap = win;
          p.xyz = sx;
          p.n = sn;
          p.step = sst;
          p.acc = sacc;
          p.status = sstat;
          p.lam = slam;
          p.abort_flag = nullptr;
          // two probes from the same scratch state; the faster one counts (the
          // first launch of a shape also pays its one-time set-up)
          float ms = 1e30f;
          cudaError_t e = cudaSuccess;
          for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            e = cudaMemcpyAsync(sx, ch->d_xyz, sizeof(float) * ch->xyz_floats, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(sn, ch->d_n, sizeof(int) * T, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(sst, 0, sizeof(unsigned long long) * T, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(sacc, 0, sizeof(double) * T * ACC_WORDS, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(sstat, 0, sizeof(int) * T, s);
            if (e == cudaSuccess && slam)
              e = cudaMemcpyAsync(slam, ch->d_lam, sizeof(float) * T, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(ch->d_queue + k, 0, sizeof(unsigned int), s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = launch_chain(p, ckind, ch->grad, spill, grid, wpb, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess) ms = std::min(ms, t);
          }
          if (e != cudaSuccess) {
            rc = fail(PMC_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
            break;
          }
          if (ms < best_ms) {
            best_ms = ms;
            best = std::make_tuple(wpb, win, ckind);
          }
          if (lane_kind(ckind))
            lane_probes.push_back({ms, wpb, win, ckind, (work_items(ckind, chains) + wpb - 1) / wpb <= grid});
        }
        if (rc != PMC_OK) break;
      }
      // The probes start from the initial paths, which are shorter than the
      // paths the chains grow to.  Among lane-layout probes within 5 % of the
      // fastest (a tie at the probe's path lengths) the one kept is, in this
      // order: a shape whose grid holds every work item at once (otherwise
      // the last items run after the others, a tail that grows with the
      // paths); the largest window (it keeps the most of a grown path in
      // shared memory); the fastest.
      if (rc == PMC_OK && lane_kind(std::get<2>(best))) {
        const LaneProbe* keep = nullptr;
        for (const auto& pr : lane_probes) {
          if (pr.kind != std::get<2>(best) || pr.ms > 1.05f * best_ms) continue;
          if (!keep || std::make_tuple(pr.resident, pr.win, -pr.ms) > std::make_tuple(keep->resident, keep->win, -keep->ms))
            keep = &pr;
        }
        if (keep) best = std::make_tuple(keep->wpb, keep->win, keep->kind);
      }
      if (rc == PMC_OK) ch->ctx->tuned[key] = best;
    }
    int bps = 0;
    const int bw = std::get<0>(best), bwin = std::get<1>(best), bkind = std::get<2>(best);
    const bool spill = !lane_kind(bkind) && bwin < full;
    if (rc == PMC_OK && chain_occupancy(bkind, ch->grad, spill, bw, bwin, &bps) == cudaSuccess && bps >= 1) {
      cl.kind = bkind;
      cl.warps_per_block = bw;
      cl.smem_cap = bwin;
      cl.spill = spill;
      cl.grid = std::max(1, std::min((work_items(bkind, chains) + bw - 1) / bw, bps * ch->ctx->n_sm));
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sx);
  cudaFree(sn);
  cudaFree(sst);
  cudaFree(sacc);
  cudaFree(sstat);
  cudaFree(slam);
  CK(cudaMemsetAsync(ch->d_any, 0, sizeof(int), s));
  return rc;
}

int pmc_init_chains(pmc_ctx_t ctx, pmc_medium_t med, pmc_geom_t geom, const pmc_run_desc* r, void* stream,
                    pmc_chains_t* out) {
  if (!ctx || !med || !geom || !r || !out) return fail(PMC_ERR_INVALID, "NULL argument");
  *out = nullptr;
  const double pw = r->p_within, pb = r->p_birth, pd = r->p_death;
  if (!(pw >= 0 && pb >= 0 && pd >= 0) || std::fabs(pw + pb + pd - 1.0) > 1e-9)
    return fail(PMC_ERR_INVALID, "move probabilities must be >= 0 and sum to 1");
  if (pb > 0 && !(pd > 0)) return fail(PMC_ERR_INVALID, "births need deaths (reversibility)");
  if (pd > 0 && !(pb > 0)) return fail(PMC_ERR_INVALID, "deaths need births (reversibility)");
  if (!finite_pos(r->sigma)) return fail(PMC_ERR_INVALID, "sigma must be > 0");
  if (r->within == PMC_WITHIN_MALA && !finite_pos(r->mala_step)) return fail(PMC_ERR_INVALID, "mala_step must be > 0");
  if (r->within != PMC_WITHIN_PERTURB && r->within != PMC_WITHIN_MALA && r->within != PMC_WITHIN_TREE &&
      r->within != PMC_WITHIN_HMC)
    return fail(PMC_ERR_INVALID, "bad within kind");
  if (r->within == PMC_WITHIN_HMC && !(finite_pos(r->mala_step) && r->hmc_steps >= 1 && r->hmc_steps <= 1000))
    return fail(PMC_ERR_INVALID, "HMC needs mala_step > 0 and 1 <= hmc_steps <= 1000");
  if (r->init != PMC_INIT_DIRECT && r->init != PMC_INIT_STRAIGHT && r->init != PMC_INIT_USER)
    return fail(PMC_ERR_INVALID, "bad init kind");
  if (r->init == PMC_INIT_STRAIGHT && (r->init_k < 0 || !(r->init_jitter >= 0)))
    return fail(PMC_ERR_INVALID, "bad straight init");
  if (r->init == PMC_INIT_USER && (!r->init_xyz || !r->init_n || r->init_stride < 2))
    return fail(PMC_ERR_INVALID, "USER init needs init_xyz, init_n and init_stride");
  if (r->kappa_end < 0 || !std::isfinite(r->kappa_end)) return fail(PMC_ERR_INVALID, "bad kappa_end");
  if (r->layout < PMC_LAYOUT_AUTO || r->layout > PMC_LAYOUT_LANE) return fail(PMC_ERR_INVALID, "bad layout");
  if (r->layout == PMC_LAYOUT_LANE ? (r->smem_window < 0 || r->smem_window == 1)
                                   : (r->smem_window < 0 || r->smem_window % 32 != 0))
    return fail(PMC_ERR_INVALID, "smem_window must be a multiple of 32 (lane layout: >= 2)");
  CK(cudaSetDevice(ctx->device));

  auto ch = std::unique_ptr<pmc_chains_s, int (*)(pmc_chains_t)>(new pmc_chains_s, pmc_destroy_chains);
  ch->ctx = ctx;
  ch->med = med;
  ch->geom = geom;
  ch->flags = r->flags;
  ch->init_kind = r->init;
  ch->init_k = r->init_k;
  ch->init_jitter = static_cast<float>(r->init_jitter);
  // the chain window: the geometry's chains [lo, hi) in pair order (all by default)
  const long long total_g = geom->total_chains;
  long long lo = r->chain_lo, hi = r->chain_hi;
  if (lo == 0 && hi == 0) hi = total_g;
  if (lo < 0 || hi > total_g || hi <= lo) return fail(PMC_ERR_INVALID, "chain window must satisfy 0 <= lo < hi <= total");
  ch->chain_lo = lo;
  ch->total = static_cast<int>(hi - lo);
  ch->n_pairs = static_cast<int>(geom->pairs.size());
  DRun& R = ch->run;
  R.seed = r->seed;
  R.thr_within = static_cast<uint32_t>(std::floor(pw * 8388608.0 + 0.5));
  R.thr_birth = static_cast<uint32_t>(std::floor((pw + pb) * 8388608.0 + 0.5));
  R.log_pb = pb > 0 ? static_cast<float>(std::log(pb)) : 0.f;
  R.log_pd = pd > 0 ? static_cast<float>(std::log(pd)) : 0.f;
  R.sigma = static_cast<float>(r->sigma);
  R.mala_eps = static_cast<float>(r->mala_step);
  R.within = r->within;
  R.hmc_steps = r->hmc_steps;
  R.burn_in = r->burn_in;
  R.beta_min = 0.01f;
  R.gradients = (r->flags & PMC_FLAG_GRADIENTS) ? 1 : 0;
  // wavelength sampled with the path: validate and normalise the spectrum
  ch->lam_on = r->n_lambda != 0;
  if (ch->lam_on) {
    const int K = r->n_lambda;
    if (K < 2 || K > 256 || r->lambda_nm == nullptr || r->spectrum == nullptr || !finite_pos(r->sigma_lambda))
      return fail(PMC_ERR_INVALID, "wavelength sampling needs 2..256 spectrum nodes and sigma_lambda > 0");
    if (med->d.kind != PMC_HOMOGENEOUS || r->within != PMC_WITHIN_PERTURB || (r->flags & PMC_FLAG_GRADIENTS) ||
        r->layout == PMC_LAYOUT_LANE)
      return fail(PMC_ERR_INVALID, "wavelength sampling runs in a homogeneous medium with Gaussian vertex moves, "
                                   "without gradients, in the warp layout");
    double area = 0.0;
    for (int i = 0; i < K; ++i) {
      if (!finite_pos(r->lambda_nm[i]) || !(r->spectrum[i] >= 0.0) || !std::isfinite(r->spectrum[i]) ||
          (i > 0 && !(r->lambda_nm[i] > r->lambda_nm[i - 1])))
        return fail(PMC_ERR_INVALID, "spectrum: increasing positive wavelengths, finite values >= 0");
      if (i > 0) area += 0.5 * (r->lambda_nm[i] - r->lambda_nm[i - 1]) * (r->spectrum[i] + r->spectrum[i - 1]);
    }
    if (!(area > 0.0)) return fail(PMC_ERR_INVALID, "spectrum: zero area");
    ch->spec_x.assign(r->lambda_nm, r->lambda_nm + K);
    ch->spec_y.resize(K);
    for (int i = 0; i < K; ++i) ch->spec_y[i] = r->spectrum[i] / area;
    R.n_spec = K;
    R.sigma_lam = static_cast<float>(r->sigma_lambda);
  }

  ch->h_pairs = geom->pairs;
  ch->h_pair_first.assign(ch->h_pairs.size(), 0);
  for (size_t p = 0; p < ch->h_pairs.size(); ++p) {
    DPair& d = ch->h_pairs[p];
    // the pair's chains inside the window, numbered from the window's first chain
    const long long a = std::max<long long>(d.chain0, lo), b = std::min<long long>(d.chain0 + d.n_chains, hi);
    ch->h_pair_first[p] = b > a ? static_cast<int>(a - d.chain0) : 0;
    d.chain0 = static_cast<int>(std::min<long long>(a, hi) - lo);
    d.n_chains = static_cast<int>(std::max<long long>(b - a, 0));
    if (d.chain0 < 0 || d.chain0 + d.n_chains > hi - lo) return fail(PMC_ERR_INVALID, "chain window bookkeeping");
    // tree moves: sigma is dimensionless, the default end step has angular scale sigma
    const double ke = r->kappa_end > 0 ? r->kappa_end
                      : (r->within == PMC_WITHIN_TREE ? 1.0 / (r->sigma * r->sigma) : (d.R / r->sigma) * (d.R / r->sigma));
    d.kappa_end = static_cast<float>(ke);
    d.exp_m2ke = static_cast<float>(std::exp(-2.0 * ke));
  }
  ch->grad = (r->flags & PMC_FLAG_GRADIENTS) != 0;
  ch->general = med->d.kind != PMC_HOMOGENEOUS || med->d.f_sl > 0.f || r->within == PMC_WITHIN_MALA ||
                std::any_of(ch->h_pairs.begin(), ch->h_pairs.end(),
                            [](const DPair& d) { return d.emission != PMC_EMIT_ISOTROPIC || d.rho != PMC_RHO_ONE; });
  // the lean physics: homogeneous medium, pure Henyey-Greenstein, isotropic
  // emission, rho = 1 (the lane layout runs it with Gaussian or MALA moves,
  // tree moves have a lean instantiation)
  const bool lean_physics =
      med->d.kind == PMC_HOMOGENEOUS && !(med->d.f_sl > 0.f) &&
      std::all_of(ch->h_pairs.begin(), ch->h_pairs.end(),
                  [](const DPair& d) { return d.emission == PMC_EMIT_ISOTROPIC && d.rho == PMC_RHO_ONE; });
  if (r->within == PMC_WITHIN_TREE) ch->general = lean_physics ? 7 : 2;
  if (r->within == PMC_WITHIN_HMC) ch->general = 3;
  if (ch->lam_on) ch->general = 6;
  ch->layout = r->layout;
  if (lean_physics && r->within == PMC_WITHIN_PERTURB && !ch->lam_on) ch->lane_kind = 4;
  if (lean_physics && r->within == PMC_WITHIN_MALA) ch->lane_kind = 5;
  if (lean_physics && r->within == PMC_WITHIN_TREE) ch->lane_kind = 8;
  if (r->layout == PMC_LAYOUT_LANE && ch->lane_kind == 0)
    return fail(PMC_ERR_INVALID, "the lane layout runs lean chains only (homogeneous medium, isotropic emission, "
                                 "rho = 1, Henyey-Greenstein, Gaussian, MALA or tree moves)");
  // the lane layout's tree moves keep the proposed path beyond the lane's
  // shared window in more arrays of the chain's global block
  const int n_arrays =
      chain_arrays(ch->general > 0 && ch->general != 7, ch->grad) + (ch->lane_kind == 8 ? kLaneTreeArrays : 0);
  const int T = ch->total;
  ch->h_base.resize(T);
  ch->h_pair_of.resize(T);
  long long off = 0;
  for (int p = 0; p < ch->n_pairs; ++p) {
    const DPair& d = ch->h_pairs[p];
    for (int k = 0; k < d.n_chains; ++k) {
      const int c = d.chain0 + k;
      ch->h_pair_of[c] = p;
      ch->h_base[c] = off;
      off += static_cast<long long>(n_arrays) * d.cap;
    }
  }
  ch->xyz_floats = off;
  // processing order: by cap class, longest caps first inside a class (one
  // launch: every chain in one class, longest caps first)
  const bool one_launch = (r->flags & PMC_FLAG_ONE_LAUNCH) != 0;
  auto class_key = [&](int cap) { return one_launch ? 0 : class_of(cap); };
  std::vector<int> order(T);
  for (int c = 0; c < T; ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int ca = ch->h_pairs[ch->h_pair_of[a]].cap, cb = ch->h_pairs[ch->h_pair_of[b]].cap;
    const int ka = class_key(ca), kb = class_key(cb);
    if (ka != kb) return ka < kb;
    return ca > cb;
  });
  for (int lo = 0; lo < T;) {
    const int k = class_key(ch->h_pairs[ch->h_pair_of[order[lo]]].cap);
    int hi = lo;
    int maxcap = 0;
    double max_n = 0.0;
    while (hi < T && class_key(ch->h_pairs[ch->h_pair_of[order[hi]]].cap) == k) {
      const DPair& d = ch->h_pairs[ch->h_pair_of[order[hi]]];
      maxcap = std::max(maxcap, d.cap);
      const double dx = (static_cast<double>(d.c[0]) + d.c_lo[0]) - d.src[0];
      const double dy = (static_cast<double>(d.c[1]) + d.c_lo[1]) - d.src[1];
      const double dz = (static_cast<double>(d.c[2]) + d.c_lo[2]) - d.src[2];
      max_n = std::max(max_n, 2.0 + std::sqrt(dx * dx + dy * dy + dz * dz) * med->d.b);
      ++hi;
    }
    ChainClass cl;
    cl.kind = ch->general;
    cl.short_paths = med->d.kind == PMC_HOMOGENEOUS && max_n <= kLaneMaxN;
    cl.smem_cap = (maxcap + 31) / 32 * 32;
    cl.max_cap = maxcap;
    cl.spill = false;
    if (r->layout == PMC_LAYOUT_LANE) {
      cl.kind = ch->lane_kind;
      cl.smem_cap = std::min(r->smem_window > 0 ? r->smem_window : 16, maxcap);
    } else if (r->smem_window > 0 && r->smem_window < cl.smem_cap && ch->general >= 2)
      return fail(PMC_ERR_INVALID, "tree, HMC and wavelength moves need the whole vertex cap in shared memory "
                                   "(smem_window)");
    if (r->smem_window > 0 && r->smem_window < cl.smem_cap) {
      cl.smem_cap = r->smem_window;
      cl.spill = true;
    }
    cl.lo = lo;
    cl.hi = hi;
    ch->classes.push_back(cl);
    lo = hi;
  }
  // launch shapes: warps per block from the request (0: autotune after the
  // initial paths exist), persistent grid from occupancy
  ch->autotune = r->warps_per_block <= 0 && r->smem_window <= 0;
  for (auto& cl : ch->classes) {
    int wpb = r->warps_per_block > 0 ? r->warps_per_block : 4;
    wpb = std::min(wpb, 4);
    while (wpb > 1 && chain_smem_bytes(cl.smem_cap, wpb, cl.kind, ch->grad) > ctx->smem_per_block) wpb /= 2;
    if (chain_smem_bytes(cl.smem_cap, wpb, cl.kind, ch->grad) > ctx->smem_per_block) return fail(PMC_ERR_INVALID, "vertex cap too large for shared memory");
    int bps = 0;
    CK(chain_occupancy(cl.kind, ch->grad, cl.spill, wpb, cl.smem_cap, &bps));
    if (bps < 1) return fail(PMC_ERR_INVALID, "chain kernel does not fit on an SM");
    if (lane_kind(cl.kind) && r->warps_per_block <= 0) {
      // a lane-layout window set without warps per block: the shape that
      // keeps the most work items resident at once (the larger CTA on a
      // tie), since items beyond the resident warps run after the others
      const int items = work_items(cl.kind, cl.hi - cl.lo);
      long best_res = static_cast<long>(std::min((items + wpb - 1) / wpb, bps * ctx->n_sm)) * wpb;
      for (int w2 = wpb / 2; w2 >= 1; w2 /= 2) {
        int b2 = 0;
        CK(chain_occupancy(cl.kind, ch->grad, cl.spill, w2, cl.smem_cap, &b2));
        if (b2 < 1) continue;
        const long res = static_cast<long>(std::min((items + w2 - 1) / w2, b2 * ctx->n_sm)) * w2;
        if (res > best_res) {
          best_res = res;
          wpb = w2;
          bps = b2;
        }
      }
    }
    const int want = (work_items(cl.kind, cl.hi - cl.lo) + wpb - 1) / wpb;
    cl.warps_per_block = wpb;
    cl.grid = std::max(1, std::min(want, bps * ctx->n_sm));
  }

  CK(dalloc(&ch->d_pairs, ch->n_pairs));
  CK(dalloc(&ch->d_chain_pair, T));
  CK(dalloc(&ch->d_chain_base, T));
  CK(dalloc(&ch->d_order, T));
  CK(dalloc(&ch->d_xyz, static_cast<size_t>(ch->xyz_floats)));
  CK(dalloc(&ch->d_n, T));
  CK(dalloc(&ch->d_step, T));
  CK(dalloc(&ch->d_acc, static_cast<size_t>(T) * ACC_WORDS));
  CK(dalloc(&ch->d_status, T));
  CK(dalloc(&ch->d_any, 1));
  CK(dalloc(&ch->d_queue, ch->classes.size()));
  CK(dalloc(&ch->d_z2, ch->n_pairs));
  CK(dalloc(&ch->d_est, static_cast<size_t>(ch->n_pairs) * PMC_MOMENT_WORDS));
  if (ch->lam_on) {
    const int K = R.n_spec;
    std::vector<float> spec(2 * static_cast<size_t>(K));
    for (int i = 0; i < K; ++i) {
      spec[i] = static_cast<float>(ch->spec_x[i]);
      spec[K + i] = static_cast<float>(ch->spec_y[i]);
    }
    CK(dalloc(&ch->d_lam, T));
    CK(dalloc(&ch->d_spec, 2 * static_cast<size_t>(K)));
    CK(cudaMemcpy(ch->d_spec, spec.data(), spec.size() * sizeof(float), cudaMemcpyHostToDevice));
    R.spec_x = ch->d_spec;
    R.spec_y = ch->d_spec + K;
  }
  CK(cudaHostAlloc(reinterpret_cast<void**>(&ch->h_abort), sizeof(int), cudaHostAllocMapped));
  *ch->h_abort = 0;
  CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&ch->d_abort), ch->h_abort, 0));
  CK(cudaStreamCreateWithFlags(&ch->capture_stream, cudaStreamNonBlocking));

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(ch->d_pairs, ch->h_pairs.data(), sizeof(DPair) * ch->n_pairs, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ch->d_chain_pair, ch->h_pair_of.data(), sizeof(int) * T, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ch->d_chain_base, ch->h_base.data(), sizeof(long long) * T, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ch->d_order, order.data(), sizeof(int) * T, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(ch->d_status, 0, sizeof(int) * T, s));
  CK(cudaMemsetAsync(ch->d_any, 0, sizeof(int), s));
  CK(cudaMemsetAsync(ch->d_xyz, 0, sizeof(float) * ch->xyz_floats, s));

  InitParams ip{};
  ip.R = R;
  ip.pairs = ch->d_pairs;
  ip.chain_pair = ch->d_chain_pair;
  ip.chain_base = ch->d_chain_base;
  ip.xyz = ch->d_xyz;
  ip.n = ch->d_n;
  ip.step = ch->d_step;
  ip.acc = ch->d_acc;
  ip.status = ch->d_status;
  ip.total = T;
  ip.chain_id0 = static_cast<uint32_t>(lo);
  ip.lam = ch->d_lam;
  ip.init_kind = r->init;
  ip.init_k = r->init_k;
  ip.jitter = static_cast<float>(r->init_jitter);
  float* d_user = nullptr;
  int* d_user_n = nullptr;
  if (r->init == PMC_INIT_USER) {
    const size_t nf = static_cast<size_t>(T) * 3 * r->init_stride;
    CK(dalloc(&d_user, nf));
    CK(dalloc(&d_user_n, T));
    CK(cudaMemcpyAsync(d_user, r->init_xyz, nf * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_user_n, r->init_n, T * sizeof(int), cudaMemcpyHostToDevice, s));
    ip.user_xyz = d_user;
    ip.user_n = d_user_n;
    ip.user_stride = r->init_stride;
  }
  CK(launch_init(ip, s));
  // direct-sector integral per pair (axisymmetric integrands need one azimuth)
  const bool axisym = std::all_of(ch->h_pairs.begin(), ch->h_pairs.end(),
                                  [](const DPair& d) { return d.emission == 0 && d.rho == 0; }) &&
                      med->d.kind == 0;
  if (!ch->lam_on) {
    CK(launch_z2(med->d, ch->d_pairs, ch->n_pairs, 4096, axisym ? 1 : 64, ch->d_z2, s));
  } else {
    // the direct sector of the joint density: the spectrum-weighted integral
    // over the wavelength of Z2 at the medium of each wavelength
    // (Gauss-Legendre, 8 nodes per interval of the spectrum, where S is linear)
    const int K = R.n_spec, G = 8;
    double gx[G], gw[G];
    gauss_legendre(G, gx, gw);
    std::vector<double> acc(ch->n_pairs, 0.0), z(ch->n_pairs);
    for (int i = 0; i + 1 < K; ++i) {
      const double a = ch->spec_x[i], b = ch->spec_x[i + 1];
      for (int q = 0; q < G; ++q) {
        const double lam = 0.5 * (a + b) + 0.5 * (b - a) * gx[q];
        const double sv = ch->spec_y[i] + (ch->spec_y[i + 1] - ch->spec_y[i]) * (lam - a) / (b - a);
        const double wq = 0.5 * (b - a) * gw[q] * sv;
        if (!(wq > 0.0)) continue;
        DMedium Mq = med->d;
        const double ratio = lam / med->d.lam0;
        const double bq = (1.0 / med->lambda_s) * std::pow(ratio, -static_cast<double>(med->d.ks));
        const double aq = (1.0 / med->lambda_a) * std::pow(ratio, -static_cast<double>(med->d.ka));
        Mq.b = static_cast<float>(bq);
        Mq.a = static_cast<float>(aq);
        Mq.log_b = static_cast<float>(std::log(bq));
        CK(launch_z2(Mq, ch->d_pairs, ch->n_pairs, 4096, axisym ? 1 : 64, ch->d_z2, s));
        CK(cudaMemcpyAsync(z.data(), ch->d_z2, sizeof(double) * ch->n_pairs, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int p = 0; p < ch->n_pairs; ++p) acc[p] += wq * z[p];
      }
    }
    CK(cudaMemcpyAsync(ch->d_z2, acc.data(), sizeof(double) * ch->n_pairs, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  if (d_user) {
    CK(cudaStreamSynchronize(s));
    cudaFree(d_user);
    cudaFree(d_user_n);
  }
  if (ch->autotune) {
    const int rc = autotune_classes(ch.get(), s);
    if (rc != PMC_OK) return rc;
  }
  *out = ch.release();
  return PMC_OK;
}

static InitParams init_params(pmc_chains_t ch) {
  InitParams ip{};
  ip.R = ch->run;
  ip.pairs = ch->d_pairs;
  ip.chain_pair = ch->d_chain_pair;
  ip.chain_base = ch->d_chain_base;
  ip.xyz = ch->d_xyz;
  ip.n = ch->d_n;
  ip.step = ch->d_step;
  ip.acc = ch->d_acc;
  ip.status = ch->d_status;
  ip.total = ch->total;
  ip.chain_id0 = static_cast<uint32_t>(ch->chain_lo);
  ip.lam = ch->d_lam;
  ip.init_kind = ch->init_kind;
  ip.init_k = ch->init_k;
  ip.jitter = ch->init_jitter;
  return ip;
}

int pmc_reset_chains(pmc_chains_t ch, void* stream) {
  if (ch == nullptr) return fail(PMC_ERR_INVALID, "NULL chains");
  if (ch->init_kind == PMC_INIT_USER) return fail(PMC_ERR_INVALID, "USER-initialised chains need pmc_set_states");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(ch->d_status, 0, sizeof(int) * ch->total, s));
  CK(cudaMemsetAsync(ch->d_any, 0, sizeof(int), s));
  CK(launch_init(init_params(ch), s));
  return PMC_OK;
}

int pmc_set_states(pmc_chains_t ch, const float* xyz, const int* n, int stride, void* stream) {
  if (ch == nullptr || xyz == nullptr || n == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  if (stride < 2) return fail(PMC_ERR_INVALID, "stride must be >= 2");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nf = static_cast<size_t>(ch->total) * 3 * stride;
  if (nf > ch->stage_floats) {
    cudaFree(ch->d_stage);
    cudaFree(ch->d_stage_n);
    ch->d_stage = nullptr;
    ch->d_stage_n = nullptr;
    ch->stage_floats = 0;
    CK(dalloc(&ch->d_stage, nf));
    CK(dalloc(&ch->d_stage_n, ch->total));
    ch->stage_floats = nf;
  }
  CK(cudaMemcpyAsync(ch->d_stage, xyz, nf * sizeof(float), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ch->d_stage_n, n, ch->total * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(ch->d_status, 0, sizeof(int) * ch->total, s));
  CK(cudaMemsetAsync(ch->d_any, 0, sizeof(int), s));
  InitParams ip = init_params(ch);
  ip.init_kind = PMC_INIT_USER;
  ip.user_xyz = ch->d_stage;
  ip.user_n = ch->d_stage_n;
  ip.user_stride = stride;
  CK(launch_init(ip, s));
  return PMC_OK;
}

static int enqueue_steps(pmc_chains_t ch, unsigned long long n_steps, cudaStream_t s) {
  for (size_t k = 0; k < ch->classes.size(); ++k) {
    const ChainClass& cl = ch->classes[k];
    CK(cudaMemsetAsync(ch->d_queue + k, 0, sizeof(unsigned int), s));
    CK(launch_chain(class_params(ch, k, n_steps), cl.kind, ch->grad, cl.spill, cl.grid, cl.warps_per_block, s));
  }
  return PMC_OK;
}

int pmc_run_steps(pmc_chains_t ch, uint64_t n_steps, void* stream) {
  if (ch == nullptr) return fail(PMC_ERR_INVALID, "NULL chains");
  if (n_steps == 0) return PMC_OK;
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (ch->flags & PMC_FLAG_NO_GRAPH) return enqueue_steps(ch, n_steps, s);
  auto it = ch->graphs.find(n_steps);
  if (it == ch->graphs.end()) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ch->capture_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_steps(ch, n_steps, ch->capture_stream);
    cudaError_t e = cudaStreamEndCapture(ch->capture_stream, &g);
    if (rc != PMC_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    CK(e);
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    it = ch->graphs.emplace(n_steps, ex).first;
  }
  CK(cudaGraphLaunch(it->second, s));
  return PMC_OK;
}

static int check_status(pmc_chains_t ch, cudaStream_t s) {
  int any = 0;
  CK(cudaMemcpyAsync(&any, ch->d_any, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (any & ST_ABORTED) return fail(PMC_ERR_ABORTED, "chains aborted on request");
  if (any) return fail(PMC_ERR_DEVICE_STATUS, "chain status word " + std::to_string(any));
  return PMC_OK;
}

static double moments_ls(const pmc_chains_s* ch) { return ch->med->d.kind == 0 ? ch->med->lambda_s : 1.0; }
static double moments_la(const pmc_chains_s* ch) { return ch->med->d.kind == 0 ? ch->med->lambda_a : 1.0; }

// Per-pair moments of this chain set's accumulators into host `h`.
static int read_moments(pmc_chains_t ch, std::vector<double>& h, cudaStream_t s) {
  CK(cudaSetDevice(ch->ctx->device));
  if (ch->h_z2.empty()) {
    ch->h_z2.resize(ch->n_pairs);
    CK(cudaMemcpyAsync(ch->h_z2.data(), ch->d_z2, sizeof(double) * ch->n_pairs, cudaMemcpyDeviceToHost, s));
  }
  CK(launch_moments(ch->d_acc, ch->d_pairs, ch->n_pairs, moments_ls(ch), moments_la(ch), ch->d_est, s));
  h.resize(static_cast<size_t>(ch->n_pairs) * PMC_MOMENT_WORDS);
  CK(cudaMemcpyAsync(h.data(), ch->d_est, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  return check_status(ch, s);
}

int pmc_shard_range(const pmc_pair* pairs, int n_pairs, int rank, int world, int64_t* chain_lo, int64_t* chain_hi) {
  if (pairs == nullptr || chain_lo == nullptr || chain_hi == nullptr || n_pairs < 1)
    return fail(PMC_ERR_INVALID, "NULL argument or no pairs");
  if (world < 1 || rank < 0 || rank >= world) return fail(PMC_ERR_INVALID, "need 0 <= rank < world");
  long long total = 0;
  double cost = 0.0;
  for (int p = 0; p < n_pairs; ++p) {
    if (pairs[p].n_chains < 1 || pairs[p].cap < 2) return fail(PMC_ERR_INVALID, "bad pair");
    total += pairs[p].n_chains;
    cost += static_cast<double>(pairs[p].n_chains) * pairs[p].cap;
  }
  if (total < world) return fail(PMC_ERR_INVALID, "fewer chains than ranks");
  // first chain whose cumulative cost (caps of the chains before it) reaches
  // `target`: chains of one pair cost the same, so the boundary inside a pair
  // is a division
  auto boundary = [&](double target) -> long long {
    long long c0 = 0;
    double before = 0.0;
    for (int p = 0; p < n_pairs; ++p) {
      const double per = pairs[p].cap, span = per * pairs[p].n_chains;
      if (before + span >= target) {
        const long long k = static_cast<long long>(std::ceil((target - before) / per - 1e-9));
        return c0 + std::min<long long>(std::max<long long>(k, 0), pairs[p].n_chains);
      }
      before += span;
      c0 += pairs[p].n_chains;
    }
    return total;
  };
  // edges e_0 = 0 < e_1 < ... < e_world = total: every rank keeps at least
  // one chain, and e_r <= total - (world - r) leaves one for each later rank
  long long e = 0, lo = 0;
  for (int r = 1; r <= rank + 1; ++r) {
    const long long b = r == world ? total
                                   : std::max<long long>(e + 1, std::min<long long>(boundary(cost * r / world),
                                                                                   total - (world - r)));
    if (r == rank) lo = b;
    e = b;
  }
  *chain_lo = lo;
  *chain_hi = e;
  return PMC_OK;
}

int pmc_read_moments(pmc_chains_t ch, double* out, size_t len, void* stream) {
  if (ch == nullptr || out == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  if (len < static_cast<size_t>(ch->n_pairs) * PMC_MOMENT_WORDS) return fail(PMC_ERR_INVALID, "output too short");
  std::vector<double> h;
  const int rc = read_moments(ch, h, static_cast<cudaStream_t>(stream));
  if (rc != PMC_OK) return rc;
  std::copy(h.begin(), h.end(), out);
  return PMC_OK;
}

int pmc_read_estimator(pmc_chains_t ch, pmc_estimate* out, size_t n_pairs, void* stream) {
  if (ch == nullptr || out == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  if (n_pairs < static_cast<size_t>(ch->n_pairs)) return fail(PMC_ERR_INVALID, "output has fewer entries than pairs");
  std::vector<double> h;
  const int rc = read_moments(ch, h, static_cast<cudaStream_t>(stream));
  if (rc != PMC_OK) return rc;
  for (int i = 0; i < ch->n_pairs; ++i)
    estimate_of_moments(h.data() + static_cast<size_t>(i) * PMC_MOMENT_WORDS, ch->h_z2[i], &out[i], nullptr, nullptr);
  return PMC_OK;
}

int pmc_estimate_from_moments(const double* moments, size_t n_pairs, const double* z2, pmc_estimate* out,
                              double* grad, double* grad_se) {
  if (moments == nullptr || z2 == nullptr || out == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  for (size_t i = 0; i < n_pairs; ++i)
    estimate_of_moments(moments + i * PMC_MOMENT_WORDS, z2[i], &out[i], grad ? grad + 3 * i : nullptr,
                        grad_se ? grad_se + 3 * i : nullptr);
  return PMC_OK;
}

int pmc_moments_from_accumulators(const double* acc, size_t n_chains, const int* chain_pair, size_t n_pairs,
                                  double lambda_s, double lambda_a, double* moments) {
  if (acc == nullptr || chain_pair == nullptr || moments == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  if (!(lambda_s > 0) || !(lambda_a > 0)) return fail(PMC_ERR_INVALID, "lengths must be > 0");
  std::fill(moments, moments + n_pairs * PMC_MOMENT_WORDS, 0.0);
  for (size_t c = 0; c < n_chains; ++c) {
    const int p = chain_pair[c];
    if (p < 0 || static_cast<size_t>(p) >= n_pairs) return fail(PMC_ERR_INVALID, "chain_pair out of range");
    add_chain_moments(acc + c * ACC_WORDS, lambda_s, lambda_a, moments + static_cast<size_t>(p) * PMC_MOMENT_WORDS);
  }
  return PMC_OK;
}

int pmc_pair_z2(pmc_chains_t ch, double* z2, size_t n_pairs, void* stream) {
  if (ch == nullptr || z2 == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  if (n_pairs < static_cast<size_t>(ch->n_pairs)) return fail(PMC_ERR_INVALID, "output too short");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(z2, ch->d_z2, sizeof(double) * ch->n_pairs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return PMC_OK;
}

int pmc_grad_estimator(pmc_chains_t ch, double* grad, double* grad_se, size_t len, void* stream) {
  if (ch == nullptr || grad == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  const int nt = ch->med->n_theta;
  if (len < static_cast<size_t>(ch->n_pairs) * nt) return fail(PMC_ERR_INVALID, "output too short");
  const bool layered = ch->med->d.kind != PMC_HOMOGENEOUS;
  if (!layered && !(ch->flags & PMC_FLAG_GRADIENTS))
    return fail(PMC_ERR_INVALID, "homogeneous gradients need chains created with PMC_FLAG_GRADIENTS");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<double> h;
  const int rc = read_moments(ch, h, s);
  if (rc != PMC_OK) return rc;
  std::vector<pmc_estimate> est(ch->n_pairs);
  if (!layered) {
    // accumulated over every recorded state while stepping
    for (int i = 0; i < ch->n_pairs; ++i) {
      double g[3], gs[3];
      estimate_of_moments(h.data() + static_cast<size_t>(i) * PMC_MOMENT_WORDS, ch->h_z2[i], &est[i], g, gs);
      for (int k = 0; k < 3; ++k) {
        grad[i * 3 + k] = g[k];
        if (grad_se) grad_se[i * 3 + k] = gs[k];
      }
    }
    return PMC_OK;
  }
  for (int i = 0; i < ch->n_pairs; ++i)
    estimate_of_moments(h.data() + static_cast<size_t>(i) * PMC_MOMENT_WORDS, ch->h_z2[i], &est[i], nullptr, nullptr);
  // layered: per-layer scores of the chains' current states
  const int L = ch->med->d.n_layers;
  const size_t words = static_cast<size_t>(ch->n_pairs) * 4 * L;
  double* d_sums = nullptr;
  CK(dalloc(&d_sums, words));
  cudaError_t e = cudaMemsetAsync(d_sums, 0, words * sizeof(double), s);
  if (e == cudaSuccess)
    e = launch_layer_scores(ch->med->d, ch->d_pairs, ch->d_chain_pair, ch->d_chain_base, ch->d_xyz, ch->d_n, ch->total,
                            d_sums, s);
  std::vector<double> hs(words);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), d_sums, words * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_sums);
  CK(e);
  for (int p = 0; p < ch->n_pairs; ++p) {
    const double N = static_cast<double>(ch->h_pairs[p].n_chains);
    const double I = est[p].intensity, seI = est[p].std_err;
    for (int j = 0; j < 2 * L; ++j) {
      const double m = hs[static_cast<size_t>(p) * 4 * L + j] / N;
      const double v = std::max(hs[static_cast<size_t>(p) * 4 * L + 2 * L + j] / N - m * m, 0.0);
      grad[static_cast<size_t>(p) * nt + j] = I * m;
      if (grad_se) grad_se[static_cast<size_t>(p) * nt + j] = std::sqrt(I * I * v / N + m * m * seI * seI);
    }
  }
  return PMC_OK;
}

int pmc_total_chains(pmc_chains_t ch) { return ch ? ch->total : 0; }

int pmc_chains_launch_info(pmc_chains_t ch, int* out, int max_rows, int* n_classes) {
  if (ch == nullptr || n_classes == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  *n_classes = static_cast<int>(ch->classes.size());
  for (int k = 0; k < *n_classes && k < max_rows && out != nullptr; ++k) {
    const ChainClass& cl = ch->classes[k];
    int* row = out + 6 * k;
    row[0] = cl.smem_cap;
    row[1] = cl.lo;
    row[2] = cl.hi;
    row[3] = cl.warps_per_block;
    row[4] = cl.grid;
    row[5] = cl.kind;
  }
  return PMC_OK;
}

int pmc_read_states(pmc_chains_t ch, float* xyz, int* n, uint64_t* steps, int stride, void* stream) {
  if (ch == nullptr || xyz == nullptr || n == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  if (stride < ch->geom->max_cap) return fail(PMC_ERR_INVALID, "stride smaller than the largest cap");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<float> buf(static_cast<size_t>(ch->xyz_floats));
  CK(cudaMemcpyAsync(buf.data(), ch->d_xyz, buf.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(n, ch->d_n, sizeof(int) * ch->total, cudaMemcpyDeviceToHost, s));
  if (steps) CK(cudaMemcpyAsync(steps, ch->d_step, sizeof(uint64_t) * ch->total, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int c = 0; c < ch->total; ++c) {
    const DPair& d = ch->h_pairs[ch->h_pair_of[c]];
    const float* src = buf.data() + ch->h_base[c];
    float* dst = xyz + static_cast<size_t>(c) * 3 * stride;
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < stride; ++i)
        dst[a * stride + i] = (i < n[c] && i < d.cap) ? src[a * d.cap + i] + d.org[a] : 0.f;
  }
  return PMC_OK;
}

int pmc_read_accumulators(pmc_chains_t ch, double* out, size_t n_doubles, void* stream) {
  if (ch == nullptr || out == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  const size_t need = static_cast<size_t>(ch->total) * ACC_WORDS;
  if (n_doubles < need) return fail(PMC_ERR_INVALID, "output too short");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(out, ch->d_acc, need * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return PMC_OK;
}

static size_t state_bytes(pmc_chains_t ch) {
  return 16 + sizeof(float) * static_cast<size_t>(ch->xyz_floats) + sizeof(int) * ch->total +
         sizeof(unsigned long long) * ch->total + sizeof(double) * static_cast<size_t>(ch->total) * ACC_WORDS +
         sizeof(int) * ch->total + (ch->lam_on ? sizeof(float) * ch->total : 0);
}

int pmc_save_state(pmc_chains_t ch, void* buf, size_t* bytes, void* stream) {
  if (ch == nullptr || bytes == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  const size_t need = state_bytes(ch);
  if (buf == nullptr) {
    *bytes = need;
    return PMC_OK;
  }
  if (*bytes < need) return fail(PMC_ERR_INVALID, "buffer too small");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* p = static_cast<char*>(buf);
  const long long hdr[2] = {0x504d4353544154ll, static_cast<long long>(need)};
  std::memcpy(p, hdr, 16);
  p += 16;
  CK(cudaMemcpyAsync(p, ch->d_xyz, sizeof(float) * ch->xyz_floats, cudaMemcpyDeviceToHost, s));
  p += sizeof(float) * ch->xyz_floats;
  CK(cudaMemcpyAsync(p, ch->d_n, sizeof(int) * ch->total, cudaMemcpyDeviceToHost, s));
  p += sizeof(int) * ch->total;
  CK(cudaMemcpyAsync(p, ch->d_step, sizeof(unsigned long long) * ch->total, cudaMemcpyDeviceToHost, s));
  p += sizeof(unsigned long long) * ch->total;
  CK(cudaMemcpyAsync(p, ch->d_acc, sizeof(double) * ch->total * ACC_WORDS, cudaMemcpyDeviceToHost, s));
  p += sizeof(double) * ch->total * ACC_WORDS;
  CK(cudaMemcpyAsync(p, ch->d_status, sizeof(int) * ch->total, cudaMemcpyDeviceToHost, s));
  p += sizeof(int) * ch->total;
  if (ch->lam_on) CK(cudaMemcpyAsync(p, ch->d_lam, sizeof(float) * ch->total, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *bytes = need;
  return PMC_OK;
}

int pmc_load_state(pmc_chains_t ch, const void* buf, size_t bytes, void* stream) {
  if (ch == nullptr || buf == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  const size_t need = state_bytes(ch);
  long long hdr[2];
  if (bytes < need) return fail(PMC_ERR_INVALID, "buffer too small");
  std::memcpy(hdr, buf, 16);
  if (hdr[0] != 0x504d4353544154ll || hdr[1] != static_cast<long long>(need))
    return fail(PMC_ERR_INVALID, "buffer does not hold a state of these chains");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const char* p = static_cast<const char*>(buf) + 16;
  CK(cudaMemcpyAsync(ch->d_xyz, p, sizeof(float) * ch->xyz_floats, cudaMemcpyHostToDevice, s));
  p += sizeof(float) * ch->xyz_floats;
  CK(cudaMemcpyAsync(ch->d_n, p, sizeof(int) * ch->total, cudaMemcpyHostToDevice, s));
  p += sizeof(int) * ch->total;
  CK(cudaMemcpyAsync(ch->d_step, p, sizeof(unsigned long long) * ch->total, cudaMemcpyHostToDevice, s));
  p += sizeof(unsigned long long) * ch->total;
  CK(cudaMemcpyAsync(ch->d_acc, p, sizeof(double) * ch->total * ACC_WORDS, cudaMemcpyHostToDevice, s));
  p += sizeof(double) * ch->total * ACC_WORDS;
  CK(cudaMemcpyAsync(ch->d_status, p, sizeof(int) * ch->total, cudaMemcpyHostToDevice, s));
  p += sizeof(int) * ch->total;
  if (ch->lam_on) CK(cudaMemcpyAsync(ch->d_lam, p, sizeof(float) * ch->total, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(ch->d_any, 0, sizeof(int), s));
  CK(cudaStreamSynchronize(s));
  return PMC_OK;
}

int pmc_read_lambda(pmc_chains_t ch, float* out, size_t len, void* stream) {
  if (ch == nullptr || out == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  if (!ch->lam_on) return fail(PMC_ERR_INVALID, "the chains do not sample the wavelength");
  if (len < static_cast<size_t>(ch->total)) return fail(PMC_ERR_INVALID, "output too short");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(out, ch->d_lam, sizeof(float) * ch->total, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return PMC_OK;
}

int pmc_request_abort(pmc_chains_t ch, int flag) {
  if (ch == nullptr) return fail(PMC_ERR_INVALID, "NULL chains");
  *reinterpret_cast<volatile int*>(ch->h_abort) = flag;
  return PMC_OK;
}

int pmc_chain_status(pmc_chains_t ch, int* status, void* stream) {
  if (ch == nullptr || status == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(status, ch->d_any, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return PMC_OK;
}

static const DPair* pair_of(pmc_geom_t g, int pair, bool absolute = true) {
  if (g == nullptr || pair < 0 || pair >= static_cast<int>(g->pairs.size())) return nullptr;
  return absolute ? &g->abs_pairs[pair] : &g->pairs[pair];
}

int pmc_logp(pmc_ctx_t ctx, pmc_medium_t med, pmc_geom_t geom, int pair, const float* xyz, const int* n,
             int batch, int cap, float* out_logp, void* stream) {
  const DPair* d = pair_of(geom, pair);
  if (!ctx || !med || !d || !xyz || !n || !out_logp) return fail(PMC_ERR_INVALID, "bad argument");
  if (batch < 0 || cap < 2 || cap > (1 << 20)) return fail(PMC_ERR_INVALID, "bad batch or cap");
  CK(cudaSetDevice(ctx->device));
  CK(launch_logp(med->d, *d, xyz, n, batch, cap, out_logp, nullptr, static_cast<cudaStream_t>(stream)));
  return PMC_OK;
}

int pmc_logp_grad(pmc_ctx_t ctx, pmc_medium_t med, pmc_geom_t geom, int pair, const float* xyz, const int* n,
                  int batch, int cap, float* out_logp, float* out_grad, void* stream) {
  const DPair* d = pair_of(geom, pair);
  if (!ctx || !med || !d || !xyz || !n || !out_grad) return fail(PMC_ERR_INVALID, "bad argument");
  if (batch < 0 || cap < 2 || cap > (1 << 20)) return fail(PMC_ERR_INVALID, "bad batch or cap");
  CK(cudaSetDevice(ctx->device));
  CK(launch_logp(med->d, *d, xyz, n, batch, cap, out_logp, out_grad, static_cast<cudaStream_t>(stream)));
  return PMC_OK;
}

int pmc_score(pmc_ctx_t ctx, pmc_medium_t med, pmc_geom_t geom, int pair, const float* xyz, const int* n,
              int batch, int cap, float* out, void* stream) {
  const DPair* d = pair_of(geom, pair);
  if (!ctx || !med || !d || !xyz || !n || !out) return fail(PMC_ERR_INVALID, "bad argument");
  if (batch < 0 || cap < 2) return fail(PMC_ERR_INVALID, "bad batch or cap");
  CK(cudaSetDevice(ctx->device));
  CK(launch_score(med->d, *d, xyz, n, batch, cap, out, med->n_theta, nullptr, nullptr,
                  static_cast<cudaStream_t>(stream)));
  return PMC_OK;
}

int pmc_trace(pmc_ctx_t ctx, pmc_medium_t med, pmc_geom_t geom, int pair, uint64_t seed, uint64_t photon0,
              uint64_t n_photons, double r_reject, int max_scatter, pmc_trace_result* out, void* stream) {
  const DPair* d = pair_of(geom, pair, false);
  if (!ctx || !med || !d || !out) return fail(PMC_ERR_INVALID, "bad argument");
  if (max_scatter < 0 || !(r_reject > 0)) return fail(PMC_ERR_INVALID, "bad tracer limits");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* d_out = nullptr;
  CK(dalloc(&d_out, 5));
  const float rr = std::isfinite(r_reject) ? static_cast<float>(r_reject) : std::numeric_limits<float>::infinity();
  double raw[5] = {0, 0, 0, 0, 0};
  cudaError_t e = launch_trace(med->d, *d, seed, photon0, n_photons, rr, max_scatter, d_out, ctx->n_sm, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(raw, d_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_out);
  CK(e);
  *out = trace_result(raw);
  return PMC_OK;
}

int pmc_trace_noalloc(pmc_ctx_t ctx, pmc_medium_t med, pmc_geom_t geom, const int* pair_ids, int n_pairs,
                      uint64_t seed, uint64_t photon0, uint64_t n_photons, double r_reject, int max_scatter,
                      pmc_trace_result* out, void* stream) {
  if (!ctx || !med || !geom || !pair_ids || !out) return fail(PMC_ERR_INVALID, "bad argument");
  if (n_pairs < 1 || n_pairs > PMC_NOALLOC_MAX_PAIRS)
    return fail(PMC_ERR_INVALID, "n_pairs must be in [1, PMC_NOALLOC_MAX_PAIRS]");
  if (max_scatter < 0 || !(r_reject > 0)) return fail(PMC_ERR_INVALID, "bad tracer limits");
  DPair sel[kNoAllocMaxPairs];
  for (int i = 0; i < n_pairs; ++i) {
    const DPair* d = pair_of(geom, pair_ids[i], false);
    if (d == nullptr) return fail(PMC_ERR_INVALID, "pair id out of range");
    sel[i] = *d;
  }
  CK(cudaSetDevice(ctx->device));
  const float rr = std::isfinite(r_reject) ? static_cast<float>(r_reject) : std::numeric_limits<float>::infinity();
  double raw[kNoAllocMaxPairs * 5];  // host stack: the call allocates no device memory
  CK(launch_trace_noalloc(med->d, sel, n_pairs, seed, photon0, n_photons, rr, max_scatter, raw, ctx->device,
                          ctx->n_sm, static_cast<cudaStream_t>(stream)));
  for (int i = 0; i < n_pairs; ++i) out[i] = trace_result(raw + 5 * i);
  return PMC_OK;
}

int pmc_qref_logdensity(pmc_ctx_t ctx, pmc_medium_t med, pmc_geom_t geom, int pair, const float* xyz, const int* n,
                        int batch, int cap, float* out, void* stream) {
  const DPair* d = pair_of(geom, pair);
  if (!ctx || !med || !d || !xyz || !n || !out) return fail(PMC_ERR_INVALID, "bad argument");
  if (batch < 0 || cap < 2) return fail(PMC_ERR_INVALID, "bad batch or cap");
  CK(cudaSetDevice(ctx->device));
  std::vector<QrefPair> qp;
  std::vector<double> tab;
  build_qref(med, {geom->host[pair]}, qp, tab);
  QrefPair* d_qp = nullptr;
  double* d_tab = nullptr;
  CK(dalloc(&d_qp, 1));
  cudaError_t e = dalloc(&d_tab, tab.size());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_qp, qp.data(), sizeof(QrefPair), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_qref_logdensity(med->d, qref_run(), *d, d_qp, d_tab, xyz, n, batch, cap, out, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_qp);
  cudaFree(d_tab);
  CK(e);
  return PMC_OK;
}

int pmc_qref_sample(pmc_ctx_t ctx, pmc_medium_t med, pmc_geom_t geom, int pair, uint64_t seed, uint64_t draw0,
                    uint64_t n_draws, float* out_xyz, int* out_n, int stride, void* stream) {
  const DPair* d = pair_of(geom, pair, false);
  if (!ctx || !med || !d || !out_xyz || !out_n) return fail(PMC_ERR_INVALID, "bad argument");
  if (stride < d->cap) return fail(PMC_ERR_INVALID, "stride smaller than the pair's cap");
  CK(cudaSetDevice(ctx->device));
  std::vector<QrefPair> qp;
  std::vector<double> tab;
  build_qref(med, {geom->host[pair]}, qp, tab);
  QrefPair* d_qp = nullptr;
  double* d_tab = nullptr;
  DPair* d_pair = nullptr;
  CK(dalloc(&d_qp, 1));
  cudaError_t e = dalloc(&d_tab, tab.size());
  if (e == cudaSuccess) e = dalloc(&d_pair, 1);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_qp, qp.data(), sizeof(QrefPair), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_pair, d, sizeof(DPair), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_qref_draws(med->d, qref_run(), d_pair, d_qp, d_tab, 1, pair, d->cap, seed, draw0, n_draws, nullptr,
                          out_xyz, out_n, stride, ctx->n_sm, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_qp);
  cudaFree(d_tab);
  cudaFree(d_pair);
  CK(e);
  return PMC_OK;
}

// Reference-density tables of the chains' pairs, built on first use.
static int ensure_qref(pmc_chains_t ch, cudaStream_t s) {
  if (ch->d_qp != nullptr) return PMC_OK;
  std::vector<QrefPair> qp;
  std::vector<double> tab;
  build_qref(ch->med, ch->geom->host, qp, tab);
  CK(dalloc(&ch->d_qp, qp.size()));
  CK(dalloc(&ch->d_qtab, tab.size()));
  CK(dalloc(&ch->d_bsum, 8 * static_cast<size_t>(ch->n_pairs)));
  CK(cudaMemcpyAsync(ch->d_qp, qp.data(), qp.size() * sizeof(QrefPair), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ch->d_qtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return PMC_OK;
}

int pmc_bridge_observe_log(pmc_chains_t ch, int pair, uint64_t n_draws, uint64_t draw0, uint64_t seed, float* logr,
                           void* stream) {
  if (ch == nullptr || logr == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  if (pair < 0 || pair >= ch->n_pairs) return fail(PMC_ERR_INVALID, "pair out of range");
  if (n_draws == 0) return fail(PMC_ERR_INVALID, "n_draws must be > 0");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int rc = ensure_qref(ch, s);
  if (rc != PMC_OK) return rc;
  const DPair& d = ch->h_pairs[pair];
  CK(launch_qref_draws(ch->med->d, ch->run, ch->d_pairs + pair, ch->d_qp + pair, ch->d_qtab, 1, pair, d.cap, seed,
                       draw0, n_draws, nullptr, nullptr, nullptr, 0, ch->ctx->n_sm, s, logr));
  CK(launch_qref_chain_logr(ch->med->d, ch->run, ch->d_pairs + pair, ch->d_qp + pair, ch->d_qtab, ch->d_chain_base,
                            ch->d_xyz, ch->d_n, d.chain0, d.n_chains, logr + n_draws, s));
  return PMC_OK;
}

int pmc_bridge(pmc_chains_t ch, uint64_t n_draws, uint64_t seed, double* out, void* stream) {
  if (ch == nullptr || out == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  if (n_draws == 0) return fail(PMC_ERR_INVALID, "n_draws must be > 0");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int P = ch->n_pairs;
  {
    const int rc = ensure_qref(ch, s);
    if (rc != PMC_OK) return rc;
  }
  CK(cudaMemsetAsync(ch->d_bsum, 0, 8 * sizeof(double) * P, s));
  CK(launch_qref_draws(ch->med->d, ch->run, ch->d_pairs, ch->d_qp, ch->d_qtab, P, 0, ch->geom->max_cap, seed, 0,
                       n_draws, ch->d_bsum, nullptr, nullptr, 0, ch->ctx->n_sm, s));
  CK(launch_qref_chains(ch->med->d, ch->run, ch->d_pairs, ch->d_qp, ch->d_qtab, ch->d_chain_pair, ch->d_chain_base,
                        ch->d_xyz, ch->d_n, ch->total, ch->d_bsum + 4 * P, s));
  std::vector<double> h(8 * static_cast<size_t>(P));
  CK(cudaMemcpyAsync(h.data(), ch->d_bsum, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int p = 0; p < P; ++p) {
    const double nq = static_cast<double>(n_draws);
    const double mq = h[4 * p] / nq;                      // E_q sqrt(p/q)
    const double vq = std::max(h[4 * p + 1] / nq - mq * mq, 0.0);
    const double np_ = h[4 * P + 4 * p + 2];
    const double mp = np_ > 0 ? h[4 * P + 4 * p] / np_ : 0.0;  // E_p sqrt(q/p)
    const double vp = np_ > 0 ? std::max(h[4 * P + 4 * p + 1] / np_ - mp * mp, 0.0) : 0.0;
    const double I = mq / mp;
    out[2 * p] = I;
    out[2 * p + 1] = I * std::sqrt(vq / (nq * mq * mq) + vp / (np_ * mp * mp));
  }
  return PMC_OK;
}

// Map T of paths ending on pair0's sensor to paths ending on pair1's sensor
// (FP64 constants, FP32 on the device), in the source frame of the chains or
// the absolute frame of caller batches.  Fails unless the pairs share their
// source position and the sensors are not collinear with it.
static int make_ymap(pmc_geom_t g, int pair0, int pair1, bool source_frame, DYMap* T) {
  if (g == nullptr || pair0 < 0 || pair1 < 0 || pair0 >= static_cast<int>(g->host.size()) ||
      pair1 >= static_cast<int>(g->host.size()) || pair0 == pair1)
    return fail(PMC_ERR_INVALID, "yield: pair indices out of range or equal");
  const PairHost& h0 = g->host[pair0];
  const PairHost& h1 = g->host[pair1];
  for (int i = 0; i < 3; ++i)
    if (h0.src[i] != h1.src[i]) return fail(PMC_ERR_INVALID, "yield: the two pairs must share a source position");
  double a[3], B[3], k[3], perp[3], m[3], n[3];
  for (int i = 0; i < 3; ++i) {
    a[i] = h0.c[i] - h0.src[i];
    B[i] = h1.c[i] - h1.src[i];
  }
  const double la = norm3(a), lB = norm3(B);
  if (!(la > h0.R) || !(lB > h1.R)) return fail(PMC_ERR_INVALID, "yield: source inside a sensor");
  for (int i = 0; i < 3; ++i) k[i] = a[i] / la;
  const double cpsi = (k[0] * B[0] + k[1] * B[1] + k[2] * B[2]) / lB;
  for (int i = 0; i < 3; ++i) perp[i] = B[i] / lB - cpsi * k[i];
  const double spsi = norm3(perp);
  if (!(spsi > 1e-9)) return fail(PMC_ERR_INVALID, "yield: sensors collinear with the source");
  for (int i = 0; i < 3; ++i) m[i] = -perp[i] / spsi;
  n[0] = k[1] * m[2] - k[2] * m[1];
  n[1] = k[2] * m[0] - k[0] * m[2];
  n[2] = k[0] * m[1] - k[1] * m[0];
  const double psi = std::atan2(spsi, cpsi);
  const double b0 = la - h0.R, rC = lB / (2.0 * spsi);
  const double Omega = 2.0 * psi - h1.R / rC;
  if (!(Omega > 0.0)) return fail(PMC_ERR_INVALID, "yield: sensor 1 too large for its angle to sensor 0");
  const double b1 = rC * Omega;
  *T = DYMap{};
  for (int i = 0; i < 3; ++i) {
    T->f0[i] = source_frame ? 0.0f : static_cast<float>(h0.src[i]);
    T->k[i] = static_cast<float>(k[i]);
    T->m[i] = static_cast<float>(m[i]);
    T->n[i] = static_cast<float>(n[i]);
  }
  T->rC = static_cast<float>(rC);
  T->Omega = static_cast<float>(Omega);
  T->b0 = static_cast<float>(b0);
  T->b1 = static_cast<float>(b1);
  T->inv_b0 = static_cast<float>(1.0 / b0);
  T->cosO = static_cast<float>(std::cos(Omega));
  T->sinO = static_cast<float>(std::sin(Omega));
  T->R0 = static_cast<float>(h0.R);
  T->R1 = static_cast<float>(h1.R);
  T->vol = static_cast<float>(b1 * b1 * Omega / (b0 * b0 * b0));
  T->log_area = static_cast<float>(2.0 * std::log(h1.R / h0.R));
  return PMC_OK;
}

int pmc_yield_logratio(pmc_ctx_t ctx, pmc_medium_t med, pmc_geom_t geom, int pair0, int pair1, int side,
                       const float* xyz, const int* n, int batch, int cap, float* out, float* out_xyz, void* stream) {
  if (!ctx || !med || !geom) return fail(PMC_ERR_INVALID, "bad argument");
  if (batch > 0 && (!xyz || !n || !out)) return fail(PMC_ERR_INVALID, "bad argument");
  if (side != 0 && side != 1) return fail(PMC_ERR_INVALID, "side must be 0 or 1");
  if (batch < 0 || cap < 2 || cap > (1 << 20)) return fail(PMC_ERR_INVALID, "bad batch or cap");
  DYMap T;
  const int rc = make_ymap(geom, pair0, pair1, false, &T);
  if (rc != PMC_OK) return rc;
  CK(cudaSetDevice(ctx->device));
  CK(launch_yield_logratio(med->d, geom->abs_pairs[pair0], geom->abs_pairs[pair1], T, side, xyz, n, batch, cap, out,
                           out_xyz, static_cast<cudaStream_t>(stream)));
  return PMC_OK;
}

int pmc_yield_observe(pmc_chains_t ch, int pair0, int pair1, double* sums, void* stream) {
  if (ch == nullptr || sums == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  DYMap T;
  const int rc = make_ymap(ch->geom, pair0, pair1, true, &T);
  if (rc != PMC_OK) return rc;
  CK(cudaSetDevice(ch->ctx->device));
  const DPair& p0 = ch->h_pairs[pair0];
  const DPair& p1 = ch->h_pairs[pair1];
  CK(launch_yield_chains(ch->med->d, ch->d_pairs, pair0, pair1, T, ch->d_chain_base, ch->d_xyz, ch->d_n, p0.chain0,
                         p0.n_chains, p1.chain0, p1.n_chains, sums, nullptr, static_cast<cudaStream_t>(stream)));
  return PMC_OK;
}

int pmc_yield_observe_log(pmc_chains_t ch, int pair0, int pair1, float* logr, void* stream) {
  if (ch == nullptr || logr == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  DYMap T;
  const int rc = make_ymap(ch->geom, pair0, pair1, true, &T);
  if (rc != PMC_OK) return rc;
  CK(cudaSetDevice(ch->ctx->device));
  const DPair& p0 = ch->h_pairs[pair0];
  const DPair& p1 = ch->h_pairs[pair1];
  CK(launch_yield_chains(ch->med->d, ch->d_pairs, pair0, pair1, T, ch->d_chain_base, ch->d_xyz, ch->d_n, p0.chain0,
                         p0.n_chains, p1.chain0, p1.n_chains, nullptr, logr, static_cast<cudaStream_t>(stream)));
  return PMC_OK;
}

int pmc_bridge_ratio(pmc_ctx_t ctx, const float* logr, uint64_t rows, int n0, int n1, int groups, int max_iter,
                     double tol, double* out, void* stream) {
  if (!ctx || !logr || !out) return fail(PMC_ERR_INVALID, "NULL argument");
  if (rows == 0 || n0 < 1 || n1 < 1 || groups < 1 || groups > 1024 || groups > std::min(n0, n1) || max_iter < 1 ||
      !(tol > 0))
    return fail(PMC_ERR_INVALID, "bad bridge arguments");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int G = groups;
  double* d_r = nullptr;
  double* d_acc = nullptr;
  CK(dalloc(&d_r, G + 1));
  cudaError_t e = dalloc(&d_acc, 2 * (G + 1));
  std::vector<double> r(G + 1), acc(2 * (G + 1));
  // chains per group on each side
  std::vector<double> c0(G + 1, 0.0), c1(G + 1, 0.0);
  for (int j = 0; j < n0; ++j) c0[j % G] += 1.0;
  for (int j = 0; j < n1; ++j) c1[j % G] += 1.0;
  c0[G] = n0;
  c1[G] = n1;
  const double s0 = static_cast<double>(n0) / (n0 + n1), s1 = static_cast<double>(n1) / (n0 + n1);
  auto pass = [&](int geometric) -> cudaError_t {
    cudaError_t ee = cudaMemcpyAsync(d_r, r.data(), sizeof(double) * (G + 1), cudaMemcpyHostToDevice, s);
    if (ee == cudaSuccess)
      ee = launch_bridge_sums(logr, rows, n0, n1, G, d_r, s0, s1, geometric, d_acc, ctx->n_sm, s);
    if (ee == cudaSuccess)
      ee = cudaMemcpyAsync(acc.data(), d_acc, sizeof(double) * 2 * (G + 1), cudaMemcpyDeviceToHost, s);
    if (ee == cudaSuccess) ee = cudaStreamSynchronize(s);
    return ee;
  };
  // start from the geometric estimator
  if (e == cudaSuccess) e = pass(1);
  int it = 0;
  if (e == cudaSuccess) {
    for (int g = 0; g <= G; ++g) r[g] = (acc[2 * g] / c0[g]) / (acc[2 * g + 1] / c1[g]);
    out[3] = r[G];
    for (it = 1; it <= max_iter && e == cudaSuccess; ++it) {
      e = pass(0);
      if (e != cudaSuccess) break;
      double change = 0.0;
      for (int g = 0; g <= G; ++g) {
        const double rn = (acc[2 * g] / c0[g]) / (acc[2 * g + 1] / c1[g]);
        if (std::isfinite(rn) && rn > 0) change = std::max(change, std::fabs(rn / r[g] - 1.0));
        r[g] = rn;
      }
      if (change < tol) break;
    }
  }
  cudaFree(d_r);
  cudaFree(d_acc);
  CK(e);
  double m = 0.0, v = 0.0;
  for (int g = 0; g < G; ++g) m += r[g] / G;
  for (int g = 0; g < G; ++g) v += (r[g] - m) * (r[g] - m);
  out[0] = r[G];
  out[1] = G > 1 ? std::sqrt(v / (G - 1) / G) : std::numeric_limits<double>::quiet_NaN();
  out[2] = std::min(it, max_iter);
  return PMC_OK;
}

int pmc_yield_estimate(pmc_chains_t ch, int pair0, int pair1, const double* sums, uint64_t n_obs, double* out,
                       void* stream) {
  if (ch == nullptr || sums == nullptr || out == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  if (n_obs == 0) return fail(PMC_ERR_INVALID, "n_obs must be > 0");
  if (pair0 < 0 || pair1 < 0 || pair0 >= ch->n_pairs || pair1 >= ch->n_pairs || pair0 == pair1)
    return fail(PMC_ERR_INVALID, "yield: pair indices out of range or equal");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* d_out = nullptr;
  CK(dalloc(&d_out, 6));
  cudaError_t e = launch_yield_estimate(sums, ch->h_pairs[pair0].n_chains, ch->h_pairs[pair1].n_chains,
                                        static_cast<double>(n_obs), d_out, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, 6 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_out);
  CK(e);
  return PMC_OK;
}

int pmc_score_observe(pmc_chains_t ch, double* sums, void* stream) {
  if (ch == nullptr || sums == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  if (ch->med->d.kind != PMC_LAYERED)
    return fail(PMC_ERR_INVALID, "pmc_score_observe needs a layered medium (homogeneous media: pmc_grad_estimator)");
  CK(cudaSetDevice(ch->ctx->device));
  CK(launch_layer_scores(ch->med->d, ch->d_pairs, ch->d_chain_pair, ch->d_chain_base, ch->d_xyz, ch->d_n, ch->total,
                         sums, static_cast<cudaStream_t>(stream)));
  return PMC_OK;
}

int pmc_length_hist(pmc_chains_t ch, double l_lo, double l_hi, int n_bins, double* hist, void* stream) {
  if (ch == nullptr || hist == nullptr) return fail(PMC_ERR_INVALID, "NULL argument");
  if (!(l_hi > l_lo) || !std::isfinite(l_lo) || !std::isfinite(l_hi) || n_bins < 1)
    return fail(PMC_ERR_INVALID, "bad histogram range");
  CK(cudaSetDevice(ch->ctx->device));
  CK(launch_length_hist(ch->d_pairs, ch->d_chain_pair, ch->d_chain_base, ch->d_xyz, ch->d_n, ch->total, l_lo, l_hi,
                        n_bins, hist, static_cast<cudaStream_t>(stream)));
  return PMC_OK;
}

int pmc_trace_lengths(pmc_ctx_t ctx, pmc_medium_t med, pmc_geom_t geom, int pair, uint64_t seed, uint64_t photon0,
                      uint64_t n_photons, double r_reject, int max_scatter, double l_lo, double l_hi, int n_bins,
                      pmc_trace_result* out, double* hist, void* stream) {
  const DPair* d = pair_of(geom, pair, false);
  if (!ctx || !med || !d || !out || !hist) return fail(PMC_ERR_INVALID, "bad argument");
  if (max_scatter < 0 || !(r_reject > 0)) return fail(PMC_ERR_INVALID, "bad tracer limits");
  if (!(l_hi > l_lo) || !std::isfinite(l_lo) || !std::isfinite(l_hi) || n_bins < 1)
    return fail(PMC_ERR_INVALID, "bad histogram range");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* d_out = nullptr;
  CK(dalloc(&d_out, 5 + static_cast<size_t>(n_bins)));
  const float rr = std::isfinite(r_reject) ? static_cast<float>(r_reject) : std::numeric_limits<float>::infinity();
  cudaError_t e = launch_trace_lengths(med->d, *d, seed, photon0, n_photons, rr, max_scatter, l_lo, l_hi, n_bins,
                                       d_out, d_out + 5, ctx->n_sm, s);
  double raw[5] = {0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(raw, d_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hist, d_out + 5, static_cast<size_t>(n_bins) * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_out);
  CK(e);
  *out = trace_result(raw);
  // detected weight of each length bin per emitted photon
  for (int b = 0; b < n_bins; ++b) hist[b] = raw[3] > 0 ? hist[b] / raw[3] : 0.0;
  return PMC_OK;
}

int pmc_seed_select(const uint64_t* photon_idx, size_t count, size_t need, uint64_t* out) {
  if ((count > 0 && photon_idx == nullptr) || (need > 0 && out == nullptr)) return fail(PMC_ERR_INVALID, "NULL argument");
  if (count == 0 && need > 0) return fail(PMC_ERR_INVALID, "no accepted photon to select from");
  // the accepted photons with the smallest indices: the first `need` draws of
  // a sequential tracer, whatever order the GPU found them in
  std::vector<uint64_t> v(photon_idx, photon_idx + count);
  std::sort(v.begin(), v.end());
  for (size_t i = 0; i < need; ++i) out[i] = v[i % count];
  return PMC_OK;
}

int pmc_seed_from_tracer(pmc_chains_t ch, uint64_t seed, uint64_t photons_per_round, int max_rounds, double r_reject,
                         uint64_t* photons_used, void* stream) {
  if (ch == nullptr) return fail(PMC_ERR_INVALID, "NULL chains");
  if (photons_per_round == 0 || max_rounds < 1 || !(r_reject > 0))
    return fail(PMC_ERR_INVALID, "need photons_per_round >= 1, max_rounds >= 1 and r_reject > 0");
  if (ch->lam_on) return fail(PMC_ERR_INVALID, "tracer seeds carry no wavelength: seed wavelength-sampling chains "
                                               "with pmc_set_states or their initial paths");
  CK(cudaSetDevice(ch->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float rr = std::isfinite(r_reject) ? static_cast<float>(r_reject) : std::numeric_limits<float>::infinity();
  // chain i of a pair (index within the pair, whatever chain window holds
  // it) takes the i-th accepted photon, so a sharded set seeds its chains
  // exactly as the whole set does
  int need_max = 0, local_max = 0;
  for (size_t p = 0; p < ch->h_pairs.size(); ++p) {
    need_max = std::max(need_max, ch->h_pair_first[p] + ch->h_pairs[p].n_chains);
    local_max = std::max(local_max, ch->h_pairs[p].n_chains);
  }
  // capacity of one round's accepted indices: twice the largest pair's need
  const unsigned int cap_idx = static_cast<unsigned int>(std::max(2 * need_max, 4096));
  unsigned long long* d_idx = nullptr;
  unsigned long long* d_sel = nullptr;
  unsigned int* d_count = nullptr;
  CK(dalloc(&d_idx, cap_idx));
  int rc = PMC_OK;
  cudaError_t e = cudaMalloc(&d_sel, sizeof(unsigned long long) * std::max(local_max, 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_count, sizeof(unsigned int));
  std::vector<uint64_t> got, sel;
  for (int p = 0; p < ch->n_pairs && e == cudaSuccess && rc == PMC_OK; ++p) {
    const DPair& d = ch->h_pairs[p];
    const size_t n_local = static_cast<size_t>(d.n_chains);
    const size_t first = static_cast<size_t>(ch->h_pair_first[p]);
    const size_t need = first + n_local;
    if (photons_used) photons_used[p] = 0;
    if (n_local == 0) continue;
    const unsigned long long key = seed + static_cast<unsigned long long>(p);
    got.clear();
    unsigned long long photon = 0, per_round = photons_per_round;
    int rounds = 0;
    while (rounds < max_rounds && got.size() < need) {
      unsigned int h = 0;
      e = cudaMemsetAsync(d_count, 0, sizeof(unsigned int), s);
      if (e == cudaSuccess)
        e = launch_seed_count(ch->med->d, d, key, photon, per_round, rr, d.cap - 2, d_idx, cap_idx, d_count,
                              ch->ctx->n_sm, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) break;
      if (h > cap_idx && per_round > 1) {
        per_round = std::max(1ull, per_round / 2);  // overflow: the same photons again, fewer at a time
        continue;
      }
      const size_t old = got.size();
      got.resize(old + std::min<size_t>(h, cap_idx));
      if (h > 0)
        e = cudaMemcpyAsync(got.data() + old, d_idx, sizeof(uint64_t) * (got.size() - old), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      photon += per_round;
      ++rounds;
    }
    if (e != cudaSuccess) break;
    if (got.empty()) {
      rc = fail(PMC_ERR_INVALID, "no detected photon for pair " + std::to_string(p) + " after " +
                                     std::to_string(photon) + " photons");
      break;
    }
    sel.resize(need);
    rc = pmc_seed_select(got.data(), got.size(), need, sel.data());
    if (rc != PMC_OK) break;
    e = cudaMemcpyAsync(d_sel, sel.data() + first, sizeof(uint64_t) * n_local, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = launch_seed_record(ch->med->d, d, key, rr, d_sel, d.chain0, static_cast<int>(n_local), ch->d_chain_base,
                             ch->d_xyz, ch->d_n, ch->d_status, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // sel is reused by the next pair
    if (photons_used) photons_used[p] = photon;
  }
  // the chains start afresh: step counters, accumulators, status
  if (e == cudaSuccess && rc == PMC_OK) e = cudaMemsetAsync(ch->d_step, 0, sizeof(unsigned long long) * ch->total, s);
  if (e == cudaSuccess && rc == PMC_OK)
    e = cudaMemsetAsync(ch->d_acc, 0, sizeof(double) * ACC_WORDS * static_cast<size_t>(ch->total), s);
  if (e == cudaSuccess && rc == PMC_OK) e = cudaMemsetAsync(ch->d_any, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_idx);
  cudaFree(d_sel);
  cudaFree(d_count);
  CK(e);
  return rc;
}

int pmc_trace_paths(pmc_ctx_t ctx, pmc_medium_t med, pmc_geom_t geom, int pair, uint64_t seed, uint64_t photon0,
                    uint64_t n_photons, double r_reject, int max_scatter, int max_paths, float* out_xyz, int* out_n,
                    int stride, uint64_t* n_accepted, void* stream) {
  const DPair* d = pair_of(geom, pair, false);
  if (!ctx || !med || !d || !out_xyz || !out_n || !n_accepted) return fail(PMC_ERR_INVALID, "bad argument");
  if (max_scatter < 0 || !(r_reject > 0) || max_paths < 0) return fail(PMC_ERR_INVALID, "bad tracer limits");
  if (stride < max_scatter + 2) return fail(PMC_ERR_INVALID, "stride must hold max_scatter + 2 vertices");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned int* d_count = nullptr;
  CK(dalloc(&d_count, 1));
  const float rr = std::isfinite(r_reject) ? static_cast<float>(r_reject) : std::numeric_limits<float>::infinity();
  cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess)
    e = launch_trace_paths(med->d, *d, seed, photon0, n_photons, rr, max_scatter, max_paths, stride, out_xyz, out_n,
                           d_count, ctx->n_sm, s);
  unsigned int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_count);
  CK(e);
  *n_accepted = h;
  return PMC_OK;
}

}  // extern "C"
