// Lane-per-chain RJMCMC kernel for the lean physics (homogeneous medium,
// isotropic emission, detection probability 1, Henyey-Greenstein phase
// function) with Gaussian (kMala = false) or MALA (kMala) vertex moves and
// vMF end moves, or (kTree) the paper's whole-path moves in tree coordinates
// (section "Path proposal distribution"; appendix "Path space coordinate
// system"); kGrad keeps d log sigma / dg per vertex for the score of g.
// It runs the same Markov chain as the warp-per-chain kernel in pmc_chain.cu
// (Collin, arXiv:1811.04156: section "Numerical path integration", Eq.
// acceptFact; appendix "Jump proposal" and "Dimension matching
// transformation"): the same Philox counters per step, the same proposals
// and acceptance rule, one chain per thread.
//
// Why: a perturbation changes O(1) factors, so a warp per chain leaves most
// lanes idle on the 60 % of steps that are perturbations; with a chain per
// lane every lane does useful work.  Every lane forms each move kind's
// proposal in one straight-line block and keeps its own chain's (the warp
// would issue every kind's code anyway), and the loops whose trip count
// is a path length index the shared window directly.
//
// Layout: the first W vertices of each chain (W = smem_cap) live in the
// warp's shared block as [array][vertex][lane] floats, so that every lane
// stays in its own bank whatever vertex it touches; entries W..cap-1 live in
// the chain's global block (array a at a * cap), as in the warp kernel's
// spill mode.  Tree moves add three arrays for the proposed path.  Positions are read from and written back to the global block
// at the start and end of a residency; the cached factors are rebuilt at the
// start.
#include "pmc_internal.h"
#include "pmc_tree.cuh"

namespace pmc {

namespace {

constexpr unsigned kAll = 0xffffffffu;
// x, y, z, segment factor, segment length, vertex factor (+ d log sigma / dg
// per vertex when gradients are accumulated)
__host__ __device__ constexpr int arrays_of(bool grad) { return grad ? 7 : 6; }
__host__ __device__ constexpr int row_of(bool tree) { return tree ? 33 : 32; }
constexpr int kRefresh = 256;        // recompute the path length from the caches
constexpr int kFlush = 64;           // FP32 partials -> FP64 accumulators
enum { AX = 0, AY = 1, AZ = 2, ASEG = 3, ALEN = 4, AVT = 5, AGT = 6 };
enum Move { MV_INTERIOR = 0, MV_END = 1, MV_BIRTH = 2, MV_DEATH = 3 };

// kRow: floats per vertex row of the warp's shared block (32, one per lane;
// 33 for tree moves, so that lanes working on vertices of one chain in the
// warp's pooled passes fall into different banks)
template <int kRow>
struct LanePath {
  float* sm;  // this lane's column of the warp's shared block
  float* gm;  // the chain's global block
  int W, cap;
  __device__ __forceinline__ float ld(int a, int i) const {
    return (i < W) ? sm[(a * W + i) * kRow] : gm[a * cap + i];
  }
  __device__ __forceinline__ void st(int a, int i, float v) const {
    if (i < W) sm[(a * W + i) * kRow] = v;
    else gm[a * cap + i] = v;
  }
  // entry i of every array in shared memory (i < W): array a at [a * W * kRow]
  __device__ __forceinline__ float* row(int i) const { return sm + i * kRow; }
  __device__ __forceinline__ float3 pos(int i) const { return f3(ld(AX, i), ld(AY, i), ld(AZ, i)); }
  __device__ __forceinline__ void set_pos(int i, float3 p) const {
    st(AX, i, p.x);
    st(AY, i, p.y);
    st(AZ, i, p.z);
  }
};

// Per-chain recording state: the current state's observables enter the sums
// once, weighted by the steps it stayed current (at or after burn-in).
struct LaneAcc {
  unsigned long long pn2, pn, t_a;
  float pL, pL2, pG;
  unsigned int nflush;
  unsigned int prop_w, prop_end, prop_b, prop_d;
  unsigned int acc_i, acc_e, acc_b, acc_d;
};

template <bool kGrad>
__device__ __forceinline__ void lane_close(LaneAcc& a, unsigned long long t_b, unsigned long long burn_in, int n,
                                           float L, float G) {
  const unsigned long long from = a.t_a > burn_in ? a.t_a : burn_in;
  a.t_a = t_b;
  if (t_b <= from) return;
  const unsigned long long d = t_b - from;
  const float dw = static_cast<float>(d);
  a.pn2 += (n == 2) ? d : 0ull;
  a.pn += static_cast<unsigned long long>(n) * d;
  a.pL = fmaf(L, dw, a.pL);
  a.pL2 = fmaf(L * L, dw, a.pL2);
  if constexpr (kGrad) a.pG = fmaf(G, dw, a.pG);
  a.nflush++;
}

template <bool kGrad>
__device__ __forceinline__ void lane_flush(LaneAcc& a, double* acc) {
  acc[ACC_NDIRECT] += static_cast<double>(a.pn2);
  acc[ACC_SUMN] += static_cast<double>(a.pn);
  acc[ACC_SUML] += static_cast<double>(a.pL);
  acc[ACC_SUML2] += static_cast<double>(a.pL2);
  if constexpr (kGrad) acc[ACC_SUMG] += static_cast<double>(a.pG);
  a.pn2 = a.pn = 0ull;
  a.pL = a.pL2 = a.pG = 0.f;
  a.nflush = 0;
}

// ---------------------------------------------------------------------------
// Tree moves, pooled over the warp.  A tree move updates every node of the
// path; done by each lane for its own chain alone, the warp would wait at
// every step for its longest path while the lanes whose chains drew a birth
// or a death sit idle.  Instead the lanes whose chains drew a tree move
// publish them in the warp's slot table, and each pass of the move (the
// stepped coordinates of every node; the new positions depth by depth; the
// density terms of every vertex; the commit of accepted moves) runs over the
// concatenated items of all those chains, spread over the 32 lanes.  An
// item's arithmetic is that of its chain's node or vertex, and each chain
// sums its per-vertex terms in vertex order, so a chain's results do not
// depend on the chains it shares the warp with.
// ---------------------------------------------------------------------------
struct TreeSlot {
  unsigned long long t;  // the move's step
  float* gm;             // the chain's global block
  float step;            // scale of the normal steps of the tree coordinates
  float vx, vy, vz;      // root frame reference
  int n, cap, pair;
  uint32_t cid;          // global chain index
  int off;               // first vertex of the proposal in the warp's pool; -1: the chain's global block
  int pad[3];
};
static_assert(sizeof(TreeSlot) == 16 * sizeof(float), "tree slot: 16 words");
// per warp: 32 slots, then 32 ints for the prefix sums of pooled_for
constexpr int kSlotWords = 17;
// per warp: the pool of the proposals of its tree moves, 4 arrays of kPool
// vertices (x, y, z and the per-vertex terms of the log acceptance ratio),
// each chain's vertices consecutive; a proposal that does not fit lives in
// its chain's global block, after the path's arrays
constexpr int kPool = 384;

struct Proposal {
  float* p;    // array 0 of the proposal
  int stride;  // floats between its arrays
  __device__ __forceinline__ float ld(int a, int i) const { return p[a * stride + i]; }
  __device__ __forceinline__ void st(int a, int i, float v) const { p[a * stride + i] = v; }
  __device__ __forceinline__ float3 pos(int i) const { return f3(ld(0, i), ld(1, i), ld(2, i)); }
  __device__ __forceinline__ void set_pos(int i, float3 q) const {
    st(0, i, q.x);
    st(1, i, q.y);
    st(2, i, q.z);
  }
};
constexpr int PG = 3;  // the proposal's per-vertex terms (arrays 0 - 2: its positions)

template <bool kGrad>
__device__ __forceinline__ Proposal proposal_of(const TreeSlot& T, float* pool) {
  if (T.off >= 0) return Proposal{pool + T.off, kPool};
  return Proposal{T.gm + static_cast<size_t>(arrays_of(kGrad)) * T.cap, T.cap};
}

// Every item of every lane (lane i holds `count` of them): fn(src, idx) runs
// once for item idx of lane src, item f of the warp's concatenated list on
// lane f mod 32.  All 32 lanes of the warp call it together.
template <class F>
__device__ __forceinline__ void pooled_for(TreeSlot* slots, int count, F&& fn) {
  const int lane = threadIdx.x & 31;
  int* scan = reinterpret_cast<int*>(slots + 32);
  int incl = count;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(kAll, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(kAll, incl, 31);
  scan[lane] = incl;
  __syncwarp();
  int src = 0;
  for (int f = lane; f < total; f += 32) {
    while (scan[src] <= f) ++src;
    fn(src, f - (src > 0 ? scan[src - 1] : 0));
  }
  __syncwarp();
}

// Levels of the tree of an n-vertex path: depth d has a node while its
// longest interval, ceil((n - 1) / 2^d) segments, has an interior vertex.
__device__ __forceinline__ int tree_levels(int n) {
  int d = 0;
  while ((((n - 1) + (1 << d) - 1) >> d) >= 2) ++d;
  return d;
}

// The proposals of the warp's tree moves (`mine`: this lane's chain drew
// one; its slot is filled and its proposal holds the source and the new end
// vertex).  The proposal's per-vertex terms collect the change of log J at
// each node and the log p terms of the new path.  Returns, on a lane with a
// move, log p(x') + log J(x') - log J(x) (-inf where x' has zero density).
template <bool kGrad, int kRow>
__device__ float pooled_tree_gain(const ChainParams& P, TreeSlot* slots, float* pool, float* cols, int W, bool mine,
                                  uint32_t key0, uint32_t key1) {
  const int lane = threadIdx.x & 31;
  const int n_mine = mine ? slots[lane].n : 0;
  // every interior node's stepped coordinates, and -log of its volume element at x
  pooled_for(slots, mine ? n_mine - 2 : 0, [&](int src, int idx) {
    const TreeSlot& T = slots[src];
    const LanePath<kRow> o{cols + src, T.gm, W, T.cap};
    const Proposal q = proposal_of<kGrad>(T, pool);
    const int m = idx + 1;
    float lj = 0.f;
    q.set_pos(m, tree_step_node([&](int i) { return o.pos(i); }, m, T.n, f3(T.vx, T.vy, T.vz), T.step, T.t, T.cid,
                                key0, key1, lj));
    q.st(PG, m, lj);
  });
  // the new positions, shallower nodes first (a node's frame uses its foci
  // and its parent's triangle), and +log of each volume element at x'
  const int levels = mine ? tree_levels(n_mine) : 0;
  const int depth = __reduce_max_sync(kAll, static_cast<unsigned>(levels));
  for (int d = 0; d < depth; ++d) {
    pooled_for(slots, d < levels ? (1 << d) : 0, [&](int src, int j) {
      const TreeSlot& T = slots[src];
      int k, l, kp, lp;
      if (!tree_interval(T.n, d, j, k, l, kp, lp)) return;
      const Proposal q = proposal_of<kGrad>(T, pool);
      const int m = (k + l) >> 1;
      float lj = 0.f;
      q.set_pos(m, tree_place_node([&](int i) { return q.pos(i); }, k, l, kp, lp, f3(T.vx, T.vy, T.vz), q.pos(m), lj));
      q.st(PG, m, q.ld(PG, m) + lj);
    });
  }
  // the log p terms of every vertex of the new path
  pooled_for(slots, n_mine, [&](int src, int i) {
    const TreeSlot& T = slots[src];
    const Proposal q = proposal_of<kGrad>(T, pool);
    const DPair& S = P.pairs[T.pair];
    const int n = T.n;
    const float3 Pc = q.pos(i);
    const float3 Pp = (i >= 1) ? q.pos(i - 1) : Pc;
    const float3 Pn = (i <= n - 2) ? q.pos(i + 1) : Pc;
    float vt, gt, seg, tb, len;
    vertex_and_segment<false>(P.M, S, S.zoff, Pp, Pc, Pn, i, n, vt, gt, seg, tb, len);
    const float term = vt + ((i <= n - 2) ? seg : 0.f);
    q.st(PG, i, (i == 0 || i == n - 1) ? term : q.ld(PG, i) + term);
  });
  float gain = 0.f;
  if (mine) {
    const Proposal q = proposal_of<kGrad>(slots[lane], pool);
    for (int i = 0; i < n_mine; ++i) gain += q.ld(PG, i);
  }
  return gain;
}

// The accepted proposals (`taken`: this lane's chain accepted its move)
// become their chains' paths, every cached factor rebuilt.
template <bool kGrad, int kRow>
__device__ void pooled_tree_commit(const ChainParams& P, TreeSlot* slots, float* pool, float* cols, int W,
                                   bool taken) {
  const int lane = threadIdx.x & 31;
  pooled_for(slots, taken ? slots[lane].n : 0, [&](int src, int i) {
    const TreeSlot& T = slots[src];
    const LanePath<kRow> o{cols + src, T.gm, W, T.cap};
    const Proposal q = proposal_of<kGrad>(T, pool);
    const DPair& S = P.pairs[T.pair];
    const int n = T.n;
    const float3 Pc = q.pos(i);
    const float3 Pp = (i >= 1) ? q.pos(i - 1) : Pc;
    const float3 Pn = (i <= n - 2) ? q.pos(i + 1) : Pc;
    float vt, gt, seg, tb, len;
    vertex_and_segment<false>(P.M, S, S.zoff, Pp, Pc, Pn, i, n, vt, gt, seg, tb, len);
    o.set_pos(i, Pc);
    o.st(AVT, i, vt);
    if constexpr (kGrad) o.st(AGT, i, gt);
    if (i <= n - 2) {
      o.st(ASEG, i, seg);
      o.st(ALEN, i, len);
    }
  });
}

// Path length and sum of d log sigma / dg afresh from the caches (bounds the
// drift of the running sums).
template <bool kGrad, int kRow>
__device__ __forceinline__ void lane_refresh_sums(const LanePath<kRow>& w, int n, float& L, float& G) {
  float Ls = 0.f;
  for (int q = 0; q < n - 1; ++q) Ls += w.ld(ALEN, q);
  L = Ls;
  if constexpr (kGrad) {
    float Gs = 0.f;
    for (int q = 0; q < n; ++q) Gs += w.ld(AGT, q);
    G = Gs;
  }
}

// Every step of one chain's residency, on one lane.  Mirrors the warp
// kernel's step: move draw, proposal, change of log p over the changed
// window, acceptance, commit.  The change of log p over the window is summed
// in the warp kernel's shuffle order; T_b comes from the running path length
// here (the warp kernel sums the cached tau_b afresh; the two differ by FP32
// rounding, which moves a decision only when it falls within that of the
// threshold).
template <bool kGrad, bool kMala, bool kTree>
__device__ __forceinline__ void run_chain(const ChainParams& P, int c, bool own, float* col, int W, uint32_t key0,
                                          uint32_t key1, TreeSlot* slots, float* pool) {
  constexpr int kRow = row_of(kTree);
  const DMedium& M = P.M;
  const DRun& R = P.R;
  const int lane = threadIdx.x & 31;
  // With tree moves every lane of the warp runs the step loop, for the
  // warp's pooled passes: a lane without a chain of its own (own = false; c
  // is another chain of its work item, read only) or whose chain cannot run
  // takes no step of its own.
  const DPair S = P.pairs[P.chain_pair[c]];
  const int cap = S.cap;
  int n = P.n[c];
  const unsigned long long step0 = P.step[c];
  if (n < 2 || n > cap) {
    if (own) {
      P.status[c] |= ST_BAD_N;
      atomicOr(P.any_status, ST_BAD_N);
    }
    if constexpr (!kTree) return;
    own = false;
    n = 2;
  }
  LanePath<kRow> w;
  w.sm = col;
  w.gm = P.xyz + P.chain_base[c];
  w.W = W;
  w.cap = cap;
  for (int i = 0; i < min(n, W); ++i) {
    w.sm[(AX * W + i) * kRow] = w.gm[AX * cap + i];
    w.sm[(AY * W + i) * kRow] = w.gm[AY * cap + i];
    w.sm[(AZ * W + i) * kRow] = w.gm[AZ * cap + i];
  }
  // cached factors of the whole path, with a sliding window of positions
  float lp0 = 0.f, L = 0.f, G = 0.f;
  {
    float3 Pp = w.pos(0), Pc = Pp;
    for (int i = 0; i < n; ++i) {
      const float3 Pn = (i <= n - 2) ? w.pos(i + 1) : Pc;
      float vt, gt, seg, tb, len;
      vertex_and_segment<false>(M, S, S.zoff, Pp, Pc, Pn, i, n, vt, gt, seg, tb, len);
      w.st(AVT, i, vt);
      if constexpr (kGrad) w.st(AGT, i, gt);
      lp0 += vt;
      if constexpr (kGrad) G += gt;
      if (i <= n - 2) {
        w.st(ASEG, i, seg);
        w.st(ALEN, i, len);
        lp0 += seg;
        L += len;
      }
      Pp = Pc;
      Pc = Pn;
    }
  }
  if (!isfinite(lp0)) {
    if (own) {
      P.status[c] |= ST_NONFINITE;
      atomicOr(P.any_status, ST_NONFINITE);
    }
    if constexpr (!kTree) return;
    own = false;
  }
  LaneAcc A;
  A.pn2 = A.pn = 0ull;
  A.t_a = step0;
  A.pL = A.pL2 = A.pG = 0.f;
  A.nflush = 0;
  A.prop_w = A.prop_end = A.prop_b = A.prop_d = 0;
  A.acc_i = A.acc_e = A.acc_b = A.acc_d = 0;
  double* acc = P.acc + static_cast<size_t>(c) * ACC_WORDS;
  const float3 cS = f3(S.c[0], S.c[1], S.c[2]);
  const float3 cLo = f3(S.c_lo[0], S.c_lo[1], S.c_lo[2]);
  const uint32_t cid = static_cast<uint32_t>(c) + P.chain_id0;  // global chain index
  const float3 vref = kTree ? tree_vref(S) : f3(1.f, 0.f, 0.f);  // tree moves: the root frame's reference
  float* const cols = col - lane;                                 // the warp's columns
  unsigned long long done = 0;
  bool aborted = false;
  for (unsigned long long s = 0; s < P.n_steps; ++s) {
    if ((s & 1023ull) == 0 && P.abort_flag != nullptr) {
      // with tree moves the whole warp stops together (its pooled passes need every lane)
      bool stop;
      if constexpr (kTree) stop = __any_sync(kAll, *P.abort_flag != 0);
      else stop = *P.abort_flag != 0;
      if (stop) {
        aborted = true;
        break;
      }
    }
    const unsigned long long t = step0 + s;
    bool mine = false;  // tree moves: this lane's chain drew one at this step
    float logu_mine = 0.f;
    float3 end_mine = f3(0.f, 0.f, 0.f);  // ... and its new end vertex
    if (own) {
      const uint4 ra = philox4x32_10(make_uint4(static_cast<uint32_t>(t), static_cast<uint32_t>(t >> 32), cid,
                                                PUR_STEP_A), key0, key1);
      const uint4 rb = philox4x32_10(make_uint4(static_cast<uint32_t>(t), static_cast<uint32_t>(t >> 32), cid,
                                                PUR_STEP_B), key0, key1);
      const uint32_t um = ra.x >> 9;
      const uint32_t v23 = ra.y >> 9;
      const float logu = __logf(u01(ra.z));
      const float ub0 = u01(rb.x), ub1 = u01(rb.y), ub2 = u01(rb.z), ub3 = u01(rb.w);

      // work that several move kinds share runs once, with every lane: the
      // azimuth of within-dimension moves and a second sincos (the interior
      // move's third normal, the birth's phi).  T_b, the sum of tau_b over the
      // current path (births and deaths), is b times the path length in a
      // homogeneous medium: the running length L, updated at every accepted
      // move and summed afresh from the cached lengths every kRefresh steps
      // (it differs from a fresh FP32 sum by rounding only)
      const bool within = um < R.thr_within, birth = !within && um < R.thr_birth;
      float s1, c1, sB, cB;
      sincospif(2.0f * ub1, &s1, &c1);
      sincospif(2.0f * (within ? ub3 : ub2), &sB, &cB);
      const float Tb = M.b * L;

      if constexpr (kTree) {
        if (within) {
          // whole-path move in tree coordinates, the end vertex with a vMF step
          // about its sensor normal: published in the warp's slot table; the
          // warp's pooled passes below build and weigh the proposal
          A.prop_w++;
          const float3 nu = sensor_normal(S, w.pos(n - 1));
          float3 e1, e2;
          onb(nu, e1, e2);
          const float wv = 1.0f + __fdividef(__logf(fmaf(1.0f - ub0, S.exp_m2ke, ub0)), S.kappa_end);
          const float sw = m_sqrt<true>(fmaxf(0.f, 1.0f - wv * wv));
          end_mine = cS + (cLo + S.R * (wv * nu + sw * (c1 * e1 + s1 * e2)));
          TreeSlot& T = slots[lane];
          T.t = t;
          T.gm = w.gm;
          T.step = R.sigma * rsqrtf(static_cast<float>(n));
          T.vx = vref.x;
          T.vy = vref.y;
          T.vz = vref.z;
          T.n = n;
          T.cap = cap;
          T.pair = P.chain_pair[c];
          T.cid = cid;
          mine = true;
          logu_mine = logu;
        }
      }
      if (!mine) {
        // The proposal of every kind, formed by every lane as straight-line
        // code; the lane keeps the one its chain drew.  The 32 chains of a
        // warp draw all kinds at almost every step, so the warp issues every
        // kind's code anyway; without branches between them the kinds'
        // independent arithmetic interleaves.  A kind's arithmetic is the same
        // whichever lane forms it, and only the O(n) choice of a birth's
        // segment runs on the lanes that need it.
        const bool death = !within && !birth;
        // within-dimension moves: vertex jw of 1 .. n-1 (n-1: the end vertex)
        const int jw = 1 + static_cast<int>((static_cast<unsigned long long>(v23) * (n - 1)) >> 23);
        const bool end = !kTree && within && jw == n - 1;
        // births: segment k with probability tau_b(k) / T_b (smallest k whose
        // cumulative sum exceeds u T_b); a birth at the cap is proposed and
        // rejected
        const bool born = birth && n < cap;
        const float total = Tb;
        const float target =
            __fmaf_rn(static_cast<float>(v23), 1.1920928955078125e-7f, 5.9604644775390625e-8f) * total;
        // (the cumulative sums rise with q: k counts those at or below u T_b,
        // at most n - 2; no early exit, so the loads and sums pipeline)
        int k = n - 2;
        if (born) {
          float cum = 0.f;
          int below = 0;
          const float* pl = w.sm + ALEN * W * kRow;
          const int m = min(n - 1, W);
#pragma unroll 4
          for (int q = 0; q < m; ++q) {
            cum += M.b * pl[q * kRow];
            below += (cum <= target) ? 1 : 0;
          }
          for (int q = W; q < n - 1; ++q) {
            cum += M.b * w.gm[ALEN * cap + q];
            below += (cum <= target) ? 1 : 0;
          }
          k = min(below, n - 2);
        }
        // deaths: interior vertex jd of 1 .. n-2 (a death at n = 2 is proposed and rejected)
        const int jd = 1 + static_cast<int>((static_cast<unsigned long long>(v23) * (n - 2)) >> 23);
        // wlo: the first vertex whose factor changes.  The current path about
        // it, entries wlo - 1 .. wlo + 3 clamped to the path, read once: V is
        // the moved vertex of a within-dimension move or the removed one of a
        // death, IA and IB the segment ends of a birth or about a death
        const int wlo = end ? n - 2 : (within ? jw - 1 : (birth ? k : jd - 1));
        const float3 Q0 = w.pos(max(wlo - 1, 0));
        const float3 IA = w.pos(wlo);
        const float3 V = w.pos(min(wlo + 1, n - 1));
        const float3 IB = w.pos(min(birth ? wlo + 1 : wlo + 2, n - 1));
        const float3 Y = w.pos(min(birth ? wlo + 2 : wlo + 3, n - 1));
        float3 fin = f3(0.f, 0.f, 0.f), fend = f3(0.f, 0.f, 0.f);
        float3 gx = f3(0.f, 0.f, 0.f);  // MALA: d log p / d f_j at the current path
        if constexpr (!kTree) {
          // vMF step of the end vertex about its sensor normal
          const float3 nu = sensor_normal(S, V);
          float3 e1, e2;
          onb(nu, e1, e2);
          const float wv = 1.0f + __fdividef(__logf(fmaf(1.0f - ub0, S.exp_m2ke, ub0)), S.kappa_end);
          const float sw = m_sqrt<true>(fmaxf(0.f, 1.0f - wv * wv));
          const float3 nn = wv * nu + sw * (c1 * e1 + s1 * e2);
          fend = cS + (cLo + S.R * nn);
          // Gaussian step of an interior vertex (Box-Muller)
          const float r1 = m_sqrt<true>(-2.0f * __logf(ub0));
          const float r2 = m_sqrt<true>(-2.0f * __logf(ub2));
          const float3 z = f3(r1 * c1, r1 * s1, r2 * cB);
          if constexpr (kMala) {
            // Langevin step: drift along the local gradient of log p
            if (within && !end) gx = grad_vertex(M, S, S.zoff, [&](int q) { return w.pos(q); }, n, jw);
            const float h = 0.5f * R.mala_eps * R.mala_eps;
            fin = V + h * gx + R.mala_eps * z;
          } else {
            fin = V + R.sigma * z;
          }
        }
        // bispherical insertion about segment k
        float3 fbirth;
        float extra_b;
        {
          const float3 r = IB - IA;
          const float rr = dot(r, r);
          const float irl = rsqrtf(rr);
          const float gamma = 0.5f * rr * irl;
          const float3 rh = irl * r;
          float3 xi, ze;
          onb(rh, xi, ze);
          const float beta = insertion_beta(M, R, S.zoff, IA, IB, gamma);
          float cs = -1.0f - __fdividef(__logf(fmaf(-ub0, 1.0f - __expf(-2.0f * beta), 1.0f)), beta);
          cs = fminf(fmaxf(cs, -1.0f), 1.0f);
          const float sn = m_sqrt<true>(fmaxf(0.f, (1.0f - cs) * (1.0f + cs)));
          const float et = __fdividef(ub1, 1.0f - ub1);
          const float iet = __fdividef(1.0f - ub1, ub1);
          const float sht = 0.5f * (et - iet), cht = 0.5f * (et + iet);
          const float sc = __fdividef(gamma, cht - cs);
          fbirth = 0.5f * (IA + IB) + sc * (sht * rh + sn * (cB * xi + sB * ze));
          const float tbk = M.b * w.ld(ALEN, k);
          extra_b = R.log_pd - __logf(static_cast<float>(n - 1)) - R.log_pb - __logf(__fdividef(tbk, total));
        }
        // the drawn kind's proposal
        const int move = within ? (end ? MV_END : MV_INTERIOR) : (birth ? MV_BIRTH : MV_DEATH);
        A.prop_w += within;
        A.prop_end += end;
        A.prop_b += birth;
        A.prop_d += death;
        const bool proposed = within || born || (death && n > 2);
        const int jj = within ? jw : jd, kk = k;
        const int n_new = birth ? n + 1 : (death ? n - 1 : n);
        const int inew = within ? jw : (birth ? k + 1 : -1);
        const int olo = wlo;
        const int nc = (end || death) ? 2 : 3;
        const int onc = (end || birth) ? 2 : 3;
        const float3 fnew = within ? (end ? fend : fin) : (birth ? fbirth : f3(0.f, 0.f, 0.f));
        const float3 IF = birth ? fbirth : V;
        float extra = birth ? extra_b : 0.f;
        // the insertion density at a birth's or a death's segment ends and vertex
        const float lid = log_insert_density<true>(M, R, S.zoff, IA, IB, IF);

        bool accept = false;
        float nvt[3] = {0.f, 0.f, 0.f}, nseg[2] = {0.f, 0.f}, nlen[2] = {0.f, 0.f}, ngt[3] = {0.f, 0.f, 0.f};
        float dlen = 0.f, dG = 0.f;
        if (proposed) {
          // new-path positions wlo-1 .. wlo+nc: the current path's entries, a
          // death's shifted down by one past the removed vertex, the new vertex
          // at wlo+1 (a birth's entries past it shifted up by one)
          const float3 Q[5] = {Q0, IA, death ? IB : fnew, death ? Y : IB,
                               (death || end) ? f3(0.f, 0.f, 0.f) : Y};
          // the changed vertex and segment factors against the cached ones; the
          // three per-slot differences are summed as the warp kernel's two
          // shuffle rounds sum them, (d0 + d1) + d2
          float d[3], e[3], f[3], gd[3];
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            float nv = 0.f, ns = 0.f, ntb = 0.f, nl = 0.f, ng = 0.f;
            if (v < nc) {
              float seg_, tb_, len_;
              vertex_and_segment<false>(M, S, S.zoff, Q[v], Q[v + 1], Q[v + 2], wlo + v, n_new, nv, ng, seg_, tb_,
                                        len_);
              if (v < nc - 1) {
                ns = seg_;
                ntb = tb_;
                nl = len_;
              }
            }
            float ov = 0.f, os = 0.f, otb = 0.f, ol = 0.f, og = 0.f;
            if (v < onc) {
              const int o = olo + v;
              ov = w.ld(AVT, o);
              if constexpr (kGrad) og = w.ld(AGT, o);
              if (v < onc - 1) {
                os = w.ld(ASEG, o);
                ol = w.ld(ALEN, o);
                otb = M.b * ol;
              }
            }
            nvt[v] = nv;
            ngt[v] = ng;
            if (v < 2) {
              nseg[v] = ns;
              nlen[v] = nl;
            }
            d[v] = (nv + ns) - (ov + os);
            e[v] = ntb - otb;
            f[v] = nl - ol;
            gd[v] = ng - og;
          }
          const float dlp = (d[0] + d[1]) + d[2];
          dlen = (f[0] + f[1]) + f[2];
          if constexpr (kGrad) dG = (gd[0] + gd[1]) + gd[2];
          // a death's T_b of the reduced path, from the current one; one
          // insertion density for births and deaths: a birth divides by it, a
          // death multiplies
          const float dtb = (e[0] + e[1]) + e[2];
          const float Tb_red = Tb + dtb;
          const float tb_new = M.b * nlen[0];
          const float extra_d =
              -R.log_pd + __logf(static_cast<float>(n - 2)) + R.log_pb + __logf(__fdividef(tb_new, Tb_red));
          extra = birth ? extra - lid : (death ? extra_d + lid : extra);
          if (kMala && move == MV_INTERIOR && isfinite(dlp)) {
            // MALA Hastings ratio q(x | y) / q(y | x), with the gradient at the proposal
            const float3 gy = grad_vertex(M, S, S.zoff, [&](int k) { return k == jj ? fnew : w.pos(k); }, n, jj);
            const float h = 0.5f * R.mala_eps * R.mala_eps;
            const float3 fj = w.pos(jj);
            const float3 dfw = fnew - fj - h * gx;
            const float3 dbw = fj - fnew - h * gy;
            extra = (dot(dfw, dfw) - dot(dbw, dbw)) / (2.0f * R.mala_eps * R.mala_eps);
          }
          accept = logu < dlp + extra;
        }
        if (accept) {
          A.acc_i += (move == MV_INTERIOR);
          A.acc_e += (move == MV_END);
          A.acc_b += (move == MV_BIRTH);
          A.acc_d += (move == MV_DEATH);
          lane_close<kGrad>(A, t, R.burn_in, n, L, G);
          if (move >= MV_BIRTH) {
            // a birth moves entries k+1 .. n-1 up by one (highest first), a death
            // entries j+1 .. n-1 down by one (lowest first); segment arrays only
            // below n-1.  Entries whose source and destination both lie in the
            // shared window move in one loop for both kinds; the few beyond it
            // go through the global block, before (births) or after (deaths).
            const bool up = move == MV_BIRTH;
            const int a0 = up ? kk + 1 : jj + 1;
            auto move_any = [&](int i, int j) {
              w.set_pos(j, w.pos(i));
              w.st(AVT, j, w.ld(AVT, i));
              if constexpr (kGrad) w.st(AGT, j, w.ld(AGT, i));
              if (i < n - 1) {
                w.st(ASEG, j, w.ld(ASEG, i));
                w.st(ALEN, j, w.ld(ALEN, i));
              }
            };
            if (up)
              for (int i = n - 1; i >= max(a0, W - 1); --i) move_any(i, i + 1);
            {
              const int d = up ? 1 : -1;
              const int hi = min(n - 1, up ? W - 2 : W - 1);
              const int cnt = hi - a0 + 1;
              const int WS = W * kRow;
              float* src = w.row(up ? hi : a0);
              int t = 0;
              // two entries per pass, both read before either is written (the
              // second entry's destination is the first one's source)
              for (; t + 1 < cnt; t += 2, src -= 2 * d * kRow) {
                float* src2 = src - d * kRow;
                const float x0 = src[AX * WS], y0 = src[AY * WS], z0 = src[AZ * WS], v0 = src[AVT * WS];
                const float x1 = src2[AX * WS], y1 = src2[AY * WS], z1 = src2[AZ * WS], v1 = src2[AVT * WS];
                const float q0 = kGrad ? src[AGT * WS] : 0.f, q1 = kGrad ? src2[AGT * WS] : 0.f;
                const bool s0 = (up ? hi - t : a0 + t) < n - 1, s1 = (up ? hi - t - 1 : a0 + t + 1) < n - 1;
                const float g0 = s0 ? src[ASEG * WS] : 0.f, l0 = s0 ? src[ALEN * WS] : 0.f;
                const float g1 = s1 ? src2[ASEG * WS] : 0.f, l1 = s1 ? src2[ALEN * WS] : 0.f;
                float* dst = src + d * kRow;
                dst[AX * WS] = x0;
                dst[AY * WS] = y0;
                dst[AZ * WS] = z0;
                dst[AVT * WS] = v0;
                if constexpr (kGrad) dst[AGT * WS] = q0;
                if (s0) {
                  dst[ASEG * WS] = g0;
                  dst[ALEN * WS] = l0;
                }
                src[AX * WS] = x1;
                src[AY * WS] = y1;
                src[AZ * WS] = z1;
                src[AVT * WS] = v1;
                if constexpr (kGrad) src[AGT * WS] = q1;
                if (s1) {
                  src[ASEG * WS] = g1;
                  src[ALEN * WS] = l1;
                }
              }
              if (t < cnt) {
                float* dst = src + d * kRow;
                dst[AX * WS] = src[AX * WS];
                dst[AY * WS] = src[AY * WS];
                dst[AZ * WS] = src[AZ * WS];
                dst[AVT * WS] = src[AVT * WS];
                if constexpr (kGrad) dst[AGT * WS] = src[AGT * WS];
                if ((up ? hi - t : a0 + t) < n - 1) {
                  dst[ASEG * WS] = src[ASEG * WS];
                  dst[ALEN * WS] = src[ALEN * WS];
                }
              }
            }
            if (!up)
              for (int i = max(a0, W); i <= n - 1; ++i) move_any(i, i - 1);
          }
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            if (v < nc) {
              w.st(AVT, wlo + v, nvt[v]);
              if constexpr (kGrad) w.st(AGT, wlo + v, ngt[v]);
              if (v < nc - 1 && v < 2) {
                w.st(ASEG, wlo + v, nseg[v]);
                w.st(ALEN, wlo + v, nlen[v]);
              }
            }
          }
          if (move != MV_DEATH) w.set_pos(inew, fnew);
          n = n_new;
          L += dlen;
          G += dG;
          if (A.nflush >= kFlush) lane_flush<kGrad>(A, acc);
        }
      }
    }
    if constexpr (kTree) {
      if (__any_sync(kAll, mine)) {
        // the proposals' places in the warp's pool, in lane order (a chain
        // that no longer fits uses its global block); source and end vertex
        int upto = mine ? n : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(kAll, upto, o);
          if (lane >= o) upto += v;
        }
        if (mine) {
          slots[lane].off = (upto <= kPool) ? upto - n : -1;
          const Proposal q = proposal_of<kGrad>(slots[lane], pool);
          q.set_pos(0, f3(0.f, 0.f, 0.f));
          q.set_pos(n - 1, end_mine);
        }
        __syncwarp();  // the slots and the proposals' ends, visible to the warp
        const float gain = pooled_tree_gain<kGrad, kRow>(P, slots, pool, cols, W, mine, key0, key1);
        bool taken = false;
        if (mine) {
          float lpo = 0.f;
          for (int q = 0; q < n; ++q) lpo += w.ld(AVT, q) + ((q <= n - 2) ? w.ld(ASEG, q) : 0.f);
          taken = logu_mine < gain - lpo;
          if (taken) {
            A.acc_i++;
            lane_close<kGrad>(A, t, R.burn_in, n, L, G);
          }
        }
        if (__any_sync(kAll, taken)) {
          pooled_tree_commit<kGrad, kRow>(P, slots, pool, cols, W, taken);
          if (taken) {
            lane_refresh_sums<kGrad>(w, n, L, G);
            if (A.nflush >= kFlush) lane_flush<kGrad>(A, acc);
          }
        }
      }
    }
    if (!own) continue;
    done = s + 1;
    if (((s + 1) & (kRefresh - 1)) == 0) lane_refresh_sums<kGrad>(w, n, L, G);
  }
  if (!own) return;
  lane_close<kGrad>(A, step0 + done, R.burn_in, n, L, G);
  lane_flush<kGrad>(A, acc);
  // recorded states, proposal and acceptance counts
  const unsigned long long t_end = step0 + done;
  const unsigned long long first = step0 > R.burn_in ? step0 : R.burn_in;
  acc[ACC_NREC] += t_end > first ? static_cast<double>(t_end - first) : 0.0;
  acc[ACC_PROP + 0] += static_cast<double>(A.prop_w - A.prop_end);
  acc[ACC_PROP + 1] += static_cast<double>(A.prop_end);
  acc[ACC_PROP + 2] += static_cast<double>(A.prop_b);
  acc[ACC_PROP + 3] += static_cast<double>(A.prop_d);
  acc[ACC_ACC + 0] += static_cast<double>(A.acc_i);
  acc[ACC_ACC + 1] += static_cast<double>(A.acc_e);
  acc[ACC_ACC + 2] += static_cast<double>(A.acc_b);
  acc[ACC_ACC + 3] += static_cast<double>(A.acc_d);
  for (int i = 0; i < min(n, W); ++i) {
    w.gm[AX * cap + i] = w.sm[(AX * W + i) * kRow];
    w.gm[AY * cap + i] = w.sm[(AY * W + i) * kRow];
    w.gm[AZ * cap + i] = w.sm[(AZ * W + i) * kRow];
  }
  P.n[c] = n;
  P.step[c] = t_end;
  if (aborted) {
    P.status[c] |= ST_ABORTED;
    atomicOr(P.any_status, ST_ABORTED);
  }
}

// Persistent warps; each work item is 32 consecutive chains of the
// processing order, one per lane.  Shared memory per CTA: with tree moves
// the warps' slot tables and proposal pools first, then each warp's block
// of vertex rows.  kW > 0: the per-lane window W is that compile-time
// constant (every row offset in the step loop folds to an immediate); kW = 0:
// W = P.smem_cap at run time.
template <bool kGrad, bool kMala, bool kTree, int kW>
__global__ void __launch_bounds__(128, 4) lane_chain_kernel(const ChainParams P) {
  extern __shared__ float4 lane_smem4[];
  constexpr int kRow = row_of(kTree);
  float* lane_smem = reinterpret_cast<float*>(lane_smem4);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int W = kW > 0 ? kW : P.smem_cap;
  const int n_warps = blockDim.x >> 5;
  TreeSlot* slots = kTree ? reinterpret_cast<TreeSlot*>(lane_smem + wib * 32 * kSlotWords) : nullptr;
  float* pool = kTree ? lane_smem + n_warps * 32 * kSlotWords + wib * 4 * kPool : nullptr;
  float* col = lane_smem + (kTree ? n_warps * (32 * kSlotWords + 4 * kPool) : 0) +
               static_cast<size_t>(wib) * arrays_of(kGrad) * W * kRow + lane;
  const uint32_t key0 = static_cast<uint32_t>(P.R.seed), key1 = static_cast<uint32_t>(P.R.seed >> 32);
  for (;;) {
    int item = 0;
    if (lane == 0) item = static_cast<int>(atomicAdd(P.queue, 1u));
    item = __shfl_sync(kAll, item, 0);
    const long long g = static_cast<long long>(P.chain_lo) + 32ll * item;
    if (g >= P.chain_hi) break;
    const bool own = g + lane < P.chain_hi;
    if constexpr (kTree) {
      // every lane runs (a lane past the last chain follows the item's first one, read only)
      run_chain<kGrad, kMala, kTree>(P, P.order[own ? g + lane : g], own, col, W, key0, key1, slots, pool);
    } else if (own) {
      run_chain<kGrad, kMala, kTree>(P, P.order[g + lane], true, col, W, key0, key1, nullptr, nullptr);
    }
  }
}

template <bool kGrad, bool kMala, bool kTree, int kW>
cudaError_t lane_attributes() {
  static int done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(lane_chain_kernel<kGrad, kMala, kTree, kW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(lane_chain_kernel<kGrad, kMala, kTree, kW>,
                           cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = 1;
  return e;
}

template <bool kGrad, bool kMala, bool kTree, int kW>
cudaError_t occupancy_of(int warps_per_block, int window, int* blocks_per_sm) {
  cudaError_t e = lane_attributes<kGrad, kMala, kTree, kW>();
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, lane_chain_kernel<kGrad, kMala, kTree, kW>,
                                                       warps_per_block * 32,
                                                       lane_smem_bytes(window, warps_per_block, kGrad, kTree));
}

template <bool kGrad, bool kMala, bool kTree, int kW>
cudaError_t launch_of(const ChainParams& p, int grid, int warps_per_block, cudaStream_t s) {
  cudaError_t e = lane_attributes<kGrad, kMala, kTree, kW>();
  if (e != cudaSuccess) return e;
  lane_chain_kernel<kGrad, kMala, kTree, kW>
      <<<grid, warps_per_block * 32, lane_smem_bytes(p.smem_cap, warps_per_block, kGrad, kTree), s>>>(p);
  return cudaGetLastError();
}

// Gaussian and MALA moves: an instance with a compile-time window for each
// window the autotuner offers (8, 12, 16, 20, 24, 32); other windows (a cap
// below the offered one) and tree moves take the run-time window.
template <bool kGrad, bool kMala, bool kTree>
cudaError_t occupancy_w(int warps_per_block, int window, int* blocks_per_sm) {
  if constexpr (!kTree) {
    switch (window) {
      case 8: return occupancy_of<kGrad, kMala, kTree, 8>(warps_per_block, window, blocks_per_sm);
      case 12: return occupancy_of<kGrad, kMala, kTree, 12>(warps_per_block, window, blocks_per_sm);
      case 16: return occupancy_of<kGrad, kMala, kTree, 16>(warps_per_block, window, blocks_per_sm);
      case 20: return occupancy_of<kGrad, kMala, kTree, 20>(warps_per_block, window, blocks_per_sm);
      case 24: return occupancy_of<kGrad, kMala, kTree, 24>(warps_per_block, window, blocks_per_sm);
      case 32: return occupancy_of<kGrad, kMala, kTree, 32>(warps_per_block, window, blocks_per_sm);
      default: break;
    }
  }
  return occupancy_of<kGrad, kMala, kTree, 0>(warps_per_block, window, blocks_per_sm);
}

template <bool kGrad, bool kMala, bool kTree>
cudaError_t launch_w(const ChainParams& p, int grid, int warps_per_block, cudaStream_t s) {
  if constexpr (!kTree) {
    switch (p.smem_cap) {
      case 8: return launch_of<kGrad, kMala, kTree, 8>(p, grid, warps_per_block, s);
      case 12: return launch_of<kGrad, kMala, kTree, 12>(p, grid, warps_per_block, s);
      case 16: return launch_of<kGrad, kMala, kTree, 16>(p, grid, warps_per_block, s);
      case 20: return launch_of<kGrad, kMala, kTree, 20>(p, grid, warps_per_block, s);
      case 24: return launch_of<kGrad, kMala, kTree, 24>(p, grid, warps_per_block, s);
      case 32: return launch_of<kGrad, kMala, kTree, 32>(p, grid, warps_per_block, s);
      default: break;
    }
  }
  return launch_of<kGrad, kMala, kTree, 0>(p, grid, warps_per_block, s);
}

}  // namespace

size_t lane_smem_bytes(int window, int warps_per_block, bool grad, bool tree) {
  const size_t per_warp = static_cast<size_t>(arrays_of(grad)) * window * row_of(tree) +
                          (tree ? 32u * kSlotWords + 4u * kPool : 0u);
  return static_cast<size_t>(warps_per_block) * per_warp * sizeof(float);
}

// kind 4: Gaussian vertex moves, 5: MALA vertex moves, 8: tree moves
cudaError_t lane_occupancy(int kind, int warps_per_block, int window, bool grad, int* blocks_per_sm) {
  if (kind == 8)
    return grad ? occupancy_w<true, false, true>(warps_per_block, window, blocks_per_sm)
                : occupancy_w<false, false, true>(warps_per_block, window, blocks_per_sm);
  if (kind == 5)
    return grad ? occupancy_w<true, true, false>(warps_per_block, window, blocks_per_sm)
                : occupancy_w<false, true, false>(warps_per_block, window, blocks_per_sm);
  return grad ? occupancy_w<true, false, false>(warps_per_block, window, blocks_per_sm)
              : occupancy_w<false, false, false>(warps_per_block, window, blocks_per_sm);
}

cudaError_t launch_lane_chain(const ChainParams& p, int kind, int grid, int warps_per_block, bool grad,
                              cudaStream_t s) {
  if (kind == 8)
    return grad ? launch_w<true, false, true>(p, grid, warps_per_block, s)
                : launch_w<false, false, true>(p, grid, warps_per_block, s);
  if (kind == 5)
    return grad ? launch_w<true, true, false>(p, grid, warps_per_block, s)
                : launch_w<false, true, false>(p, grid, warps_per_block, s);
  return grad ? launch_w<true, false, false>(p, grid, warps_per_block, s)
              : launch_w<false, false, false>(p, grid, warps_per_block, s);
}

}  // namespace pmc
