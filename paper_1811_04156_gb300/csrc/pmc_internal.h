// Host-side internals shared by the CUDA translation units of libpathmc.
#pragma once

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pathmc.h"
#include "pmc_device.cuh"

namespace pmc {

// Accumulator word indices (per chain, FP64), order documented in pathmc.h.
enum AccWord {
  ACC_NREC = 0,
  ACC_NDIRECT = 1,
  ACC_SUMN = 2,
  ACC_SUML = 3,
  ACC_SUML2 = 4,
  ACC_SUMG = 5,
  ACC_BRIDGE = 6,
  ACC_NBRIDGE = 7,
  ACC_PROP = 8,
  ACC_ACC = 12,
  ACC_WORDS = 16
};
static_assert(ACC_WORDS == PMC_ACC_WORDS, "accumulator layout");

// Status bits of a chain.
enum StatusBits { ST_NONFINITE = 1, ST_ABORTED = 2, ST_BAD_N = 4 };

// Random-number purposes (fourth Philox counter word).
// PUR_TREE is or-ed with (vertex << 8): the normals of one tree node.
// PUR_HMC likewise: the momentum of one interior vertex.
enum Purpose : uint32_t {
  PUR_STEP_A = 0, PUR_STEP_B = 1, PUR_INIT = 2, PUR_QREF = 3, PUR_TRACE = 4, PUR_TREE = 5, PUR_HMC = 6
};

struct ChainParams {
  DMedium M;
  DRun R;
  const DPair* pairs;
  const int* chain_pair;        // [total]
  const long long* chain_base;  // [total] float offset of x[cap], y[cap], z[cap]
  const int* order;             // processing order of chains (grouped by vertex-cap class)
  float* xyz;
  int* n;
  unsigned long long* step;
  double* acc;                  // [total][ACC_WORDS]
  int* status;                  // [total]
  int* any_status;              // OR of all status words
  unsigned int* queue;          // work counter of this launch
  const volatile int* abort_flag;
  uint32_t chain_id0;           // global index of local chain 0 (Philox counter word of a chain)
  float* lam;                   // [total] wavelength of each chain (wavelength sampling), else null
  int chain_lo, chain_hi;       // chains [lo, hi) of this launch
  unsigned long long n_steps;
  int smem_cap;                 // vertex capacity of one warp's shared arrays
};

// Kernel launchers (pmc_chain.cu)
// `general` selects the instantiation with layered media, vMF emission, the
// detection probability, the simplified-Liu mixture and MALA moves.
// `grad` selects the instantiation that keeps d log sigma / dg per vertex for
// the score of g; `spill` the one whose shared window (smem_cap vertices) is
// smaller than the chains' caps, entries beyond it living in the chain's
// global block.  The global block of a chain holds chain_arrays() arrays of
// cap floats (x, y, z first).
// `kind`: 0 the lean kernel, 1 the general one, 2 the general one with tree
// moves (3 more shared arrays per warp, no spill), 3 the general one with HMC
// moves (6 more shared arrays per warp, no spill), 4 the lean kernel with one
// chain per lane and Gaussian vertex moves, 5 the same with MALA moves
// (pmc_lane.cu; smem_cap is each lane's shared window, entries beyond it in
// the chain's global block; a work item is 32 chains), 6 the general one with
// the wavelength sampled (the medium at the chain's wavelength in the warp's
// shared slot, no spill), 7 the lean one with tree moves (3 more shared
// arrays per warp, no spill), 8 the lean one with one chain per lane and tree
// moves (the proposed paths of a warp's tree moves in a pool in its shared
// memory, or, where they do not fit, in kLaneTreeArrays more arrays of the
// chain's global block).
inline bool lane_kind(int kind) { return kind == 4 || kind == 5 || kind == 8; }
// kind 8: arrays of a proposed path that does not fit the warp's pool (x, y,
// z and the per-vertex terms of its acceptance ratio), after the lane
// layout's own in the chain's global block
constexpr int kLaneTreeArrays = 4;
int chain_arrays(bool general, bool grad);
cudaError_t launch_chain(const ChainParams& p, int kind, bool grad, bool spill, int grid, int warps_per_block,
                         cudaStream_t s);
size_t chain_smem_bytes(int smem_cap, int warps_per_block, int kind, bool grad);
cudaError_t chain_occupancy(int kind, bool grad, bool spill, int warps_per_block, int smem_cap,
                            int* blocks_per_sm);

// pmc_lane.cu (kinds 4, 5 and 8 above; `grad` adds the per-vertex d log
// sigma / dg array, `tree` the proposed path's three arrays)
size_t lane_smem_bytes(int window, int warps_per_block, bool grad, bool tree);
cudaError_t lane_occupancy(int kind, int warps_per_block, int window, bool grad, int* blocks_per_sm);
cudaError_t launch_lane_chain(const ChainParams& p, int kind, int grid, int warps_per_block, bool grad,
                              cudaStream_t s);

struct InitParams {
  DRun R;
  const DPair* pairs;
  const int* chain_pair;
  const long long* chain_base;
  float* xyz;
  int* n;
  unsigned long long* step;
  double* acc;
  int* status;
  int total;
  uint32_t chain_id0;           // global index of local chain 0
  float* lam;                   // [total] wavelengths drawn from the spectrum (R.n_spec >= 2), else null
  int init_kind, init_k;
  float jitter;
  const float* user_xyz;        // device copy, [total][3][stride] absolute
  const int* user_n;
  int user_stride;
};
cudaError_t launch_init(const InitParams& p, cudaStream_t s);

// pmc_kernels.cu
cudaError_t launch_logp(const DMedium& M, const DPair& S, const float* xyz, const int* n, int batch, int cap,
                        float* out_logp, float* out_grad, cudaStream_t s);
cudaError_t launch_score(const DMedium& M, const DPair& S, const float* xyz, const int* n, int batch, int cap,
                         float* out, int n_theta, const double* ls, const double* la, cudaStream_t s);
cudaError_t launch_z2(const DMedium& M, const DPair* pairs, int n_pairs, int n_v, int n_phi, double* out,
                      cudaStream_t s);

// Per-pair moments of the chain accumulators: sums over chains that add
// across any split of a pair's chains (layout documented at
// PMC_MOMENT_WORDS in pathmc.h).  A_k is a chain's sum of the score of
// parameter k over its recorded states: A_0 = sum_L / ls^2 - (sum_n - 2 N) / ls,
// A_1 = sum_L / la^2, A_2 = sum_G.
enum MomWord {
  MOM_NCHAIN = 0,               // chains
  MOM_ACC = 1,                  // + AccWord: the accumulator words summed over chains (16 words)
  MOM_RH_M = 17, MOM_RH_M2 = 18, MOM_RH_VAR = 19, MOM_RH_K = 20,  // R-hat on L over chains with N > 1
  MOM_N2SQ = 21, MOM_NN2 = 22, MOM_NSQ = 23,                      // sum n2^2, N n2, N^2
  MOM_ASQ = 24,                 // + k: sum A_k^2
  MOM_NA = 27,                  // + k: sum N A_k
  MOM_N2A = 30,                 // + k: sum n2 A_k
  MOM_A = 33,                   // + k: sum A_k
  MOM_USED = 36
};
static_assert(MOM_USED <= PMC_MOMENT_WORDS, "moment layout");

// Adds one chain's accumulators (acc[ACC_WORDS]) to a pair's moments
// (mom[PMC_MOMENT_WORDS]); ls, la: the homogeneous lengths (1 for layered media).
__host__ __device__ inline void add_chain_moments(const double* acc, double ls, double la, double* mom) {
  const double N = acc[ACC_NREC];
  mom[MOM_NCHAIN] += 1.0;
  for (int k = 0; k < ACC_WORDS; ++k) mom[MOM_ACC + k] += acc[k];
  if (!(N > 0.0)) return;
  if (N > 1.0) {
    const double m = acc[ACC_SUML] / N;
    const double var = (acc[ACC_SUML2] / N - m * m) * N / (N - 1.0);
    mom[MOM_RH_M] += m;
    mom[MOM_RH_M2] += m * m;
    mom[MOM_RH_VAR] += var > 0.0 ? var : 0.0;
    mom[MOM_RH_K] += 1.0;
  }
  const double n2 = acc[ACC_NDIRECT];
  mom[MOM_N2SQ] += n2 * n2;
  mom[MOM_NN2] += N * n2;
  mom[MOM_NSQ] += N * N;
  const double bs = 1.0 / ls, ba = 1.0 / la;
  const double A[3] = {acc[ACC_SUML] * bs * bs - (acc[ACC_SUMN] - 2.0 * N) * bs, acc[ACC_SUML] * ba * ba,
                       acc[ACC_SUMG]};
  for (int k = 0; k < 3; ++k) {
    mom[MOM_ASQ + k] += A[k] * A[k];
    mom[MOM_NA + k] += N * A[k];
    mom[MOM_N2A + k] += n2 * A[k];
    mom[MOM_A + k] += A[k];
  }
}

// Per-pair moments of the chains' accumulators (one block per pair, FP64):
// out[n_pairs][PMC_MOMENT_WORDS].
cudaError_t launch_moments(const double* acc, const DPair* pairs, int n_pairs, double ls, double la, double* out,
                           cudaStream_t s);
// Estimate of one pair from its moments (host; pmc_estimate_from_moments).
void estimate_of_moments(const double* mom, double z2, pmc_estimate* out, double* grad, double* grad_se);

cudaError_t launch_trace(const DMedium& M, const DPair& S, unsigned long long seed,
                         unsigned long long photon0, unsigned long long n_photons, float r_reject,
                         int max_scatter, double* out5, int n_sm, cudaStream_t s);
// Forward tracer that also adds each detected weight w*rho to hist[bin] by
// its path length L in [l_lo, l_hi) (n_bins equal bins; hist zeroed here).
cudaError_t launch_trace_lengths(const DMedium& M, const DPair& S, unsigned long long seed,
                                 unsigned long long photon0, unsigned long long n_photons, float r_reject,
                                 int max_scatter, double l_lo, double l_hi, int n_bins, double* out5, double* hist,
                                 int n_sm, cudaStream_t s);

// Per-layer score sums over the chains' current states: sums[pair][0..2L) and
// squares at sums[pair][2L..4L) (layered media, L <= 4096).
cudaError_t launch_layer_scores(const DMedium& M, const DPair* pairs, const int* chain_pair, const long long* chain_base,
                                const float* xyz, const int* n, int total, double* sums, cudaStream_t s);

// Forward tracer recording weight-thinned detected paths (exact draws from the
// normalised path density), used to seed chains at equilibrium.
cudaError_t launch_trace_paths(const DMedium& M, const DPair& S, unsigned long long seed, unsigned long long photon0,
                               unsigned long long n_photons, float r_reject, int max_scatter, int max_paths, int stride,
                               float* out_xyz, int* out_n, unsigned int* count, int n_sm, cudaStream_t s);

// Chain seeding from the tracer (pmc_seed_from_tracer): indices of the
// accepted photons of a photon range, then each chain's path from its photon.
cudaError_t launch_seed_count(const DMedium& M, const DPair& S, unsigned long long seed, unsigned long long photon0,
                              unsigned long long n_photons, float r_reject, int max_scatter, unsigned long long* idx,
                              unsigned int cap_idx, unsigned int* count, int n_sm, cudaStream_t s);
cudaError_t launch_seed_record(const DMedium& M, const DPair& S, unsigned long long seed, float r_reject,
                               const unsigned long long* sel, int chain0, int n, const long long* chain_base,
                               float* xyz, int* nv, int* status, cudaStream_t s);

// pmc_bridge.cu: reference density q_ref and the geometric bridge.
// Per pair: qtab[off + n] = log P_ref(n) (n = 0..cap, -inf below 2) and
// qtab[off + cap + 1 + n] = P_ref(N <= n); log_qend = -log(visible cap area).
struct QrefPair {
  double log_qend;
  long long off;
};
// out_logr (may be null): log(p / q_ref) of each draw (-inf where either is 0).
cudaError_t launch_qref_draws(const DMedium& M, const DRun& R, const DPair* pairs, const QrefPair* qp,
                              const double* qtab, int n_pairs, int stream_base, int max_cap, unsigned long long seed,
                              unsigned long long draw0, unsigned long long n_draws, double* sums, float* out_xyz,
                              int* out_n, int out_stride, int n_sm, cudaStream_t s, float* out_logr = nullptr);
// log(q_ref / p) at the current paths of one pair's chains [chain0, chain0 + n_chains).
cudaError_t launch_qref_chain_logr(const DMedium& M, const DRun& R, const DPair* pair, const QrefPair* qp,
                                   const double* qtab, const long long* chain_base, const float* xyz, const int* n,
                                   int chain0, int n_chains, float* out, cudaStream_t s);
cudaError_t launch_qref_chains(const DMedium& M, const DRun& R, const DPair* pairs, const QrefPair* qp,
                               const double* qtab, const int* chain_pair, const long long* chain_base,
                               const float* xyz, const int* n, int total, double* sums, cudaStream_t s);
cudaError_t launch_qref_logdensity(const DMedium& M, const DRun& R, const DPair& S, const QrefPair* qp,
                                   const double* qtab, const float* xyz, const int* n, int batch, int cap, float* out,
                                   cudaStream_t s);

// pmc_yield.cu: relative light yield of two sensors and path-length histograms.
// The map T of paths ending on sensor 0 to paths ending on sensor 1, in the
// frame of the pair structs it is used with (source frame for chain states,
// absolute frame for caller batches).
struct DYMap {
  float f0[3];                 // source position in the frame
  float k[3], m[3], n[3];      // k towards sensor 0, m in the plane of k and B away from B, n = k x m
  float rC, Omega, b0, b1, inv_b0;
  float cosO, sinO;            // rotation of the end vertex about the sensor
  float R0, R1;
  float vol;                   // b1^2 Omega / b0^3: interior volume ratio over (rC + xb b1)
  float log_area;              // 2 log(R1 / R0): end-vertex area ratio
};
// Adds exp(r/2) of every chain of pair0 (side 0) and pair1 (side 1) to sums
// [n0 + n1], r the log ratio of the other density at the mapped path to the own one.
// With logr != null each chain's log ratio is also written to logr[n0 + n1].
cudaError_t launch_yield_chains(const DMedium& M, const DPair* pairs, int pair0, int pair1, const DYMap& T,
                                const long long* chain_base, const float* xyz, const int* n, int chain0_0, int n0,
                                int chain0_1, int n1, double* sums, float* logr, cudaStream_t s);
// Sums of one optimal-bridge iteration (or of the geometric estimator) over
// stored log ratios, per chain group and overall: acc[groups + 1][2] (zeroed here).
cudaError_t launch_bridge_sums(const float* logr, unsigned long long rows, int n0, int n1, int groups,
                               const double* r, double s0, double s1, int geometric, double* acc, int n_sm,
                               cudaStream_t s);
cudaError_t launch_yield_logratio(const DMedium& M, const DPair& S0, const DPair& S1, const DYMap& T, int side,
                                  const float* xyz, const int* n, int batch, int cap, float* out,
                                  float* out_xyz, cudaStream_t s);
// out (device, 6 doubles): B, standard error, E_0, E_1, across-chain variances of the per-chain means.
cudaError_t launch_yield_estimate(const double* sums, int n0, int n1, double n_obs, double* out, cudaStream_t s);
// Adds 1 to hist[pair][bin] for each chain's current path length L in [lo, hi).
cudaError_t launch_length_hist(const DPair* pairs, const int* chain_pair, const long long* chain_base,
                               const float* xyz, const int* n, int total, double lo, double hi, int n_bins,
                               double* hist, cudaStream_t s);

// pmc_noalloc.cu: allocation-free tracer over up to kNoAllocMaxPairs pairs.
constexpr int kNoAllocMaxPairs = 128;

cudaError_t launch_trace_noalloc(const DMedium& M, const DPair* pairs, int n_pairs, unsigned long long seed,
                                 unsigned long long photon0, unsigned long long n_photons, float r_reject,
                                 int max_scatter, double* host_out, int device, int n_sm, cudaStream_t s);

}  // namespace pmc
