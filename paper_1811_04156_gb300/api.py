"""Python binding of libpathmc with the C entry points' names.

Argument marshalling only: descriptors are packed into the C structs of
include/pathmc.h, device buffers come from torch tensors, and the stream is
torch's current CUDA stream.  Every step of the path (initialisation,
stepping, estimators, density, adjoint, tracer) runs in the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import math
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from . import scenes as S
from ._lib import (Estimate, GeometryDesc, MediumDesc, PairDesc, RunDesc, SensorDesc, SourceDesc, TraceResult,
                   PMC_ACC_WORDS, PMC_FLAG_GRADIENTS, PMC_FLAG_NO_GRAPH, PMC_MOMENT_WORDS, check, load)


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _require_cuda(t: torch.Tensor, dtype, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Context:
    def __init__(self, device: int = 0):
        self.device = int(device)
        h = C.c_void_p()
        check(load().pmc_create_context(self.device, C.byref(h)), "pmc_create_context")
        self.handle = h

    def close(self):
        if self.handle:
            load().pmc_destroy_context(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def create_context(device: int = 0) -> Context:
    return Context(device)


def medium_desc(m: S.Medium):
    d = MediumDesc()
    d.kind = int(m.kind)
    d.lambda_s = float(m.lambda_s)
    d.lambda_a = float(m.lambda_a)
    d.g = float(m.g)
    d.f_sl = float(m.f_sl)
    d.z0 = float(m.z0)
    d.dz = float(m.dz)
    d.lambda0 = float(getattr(m, "lambda0", 0.0))
    d.k_s = float(getattr(m, "k_s", 0.0))
    d.k_a = float(getattr(m, "k_a", 0.0))
    keep = ()
    if m.kind == S.LAYERED:
        ls = np.ascontiguousarray(m.lambda_s_layers, dtype=np.float64)
        la = np.ascontiguousarray(m.lambda_a_layers, dtype=np.float64)
        d.n_layers = len(ls)
        d.lambda_s_layers = ls.ctypes.data_as(C.POINTER(C.c_double))
        d.lambda_a_layers = la.ctypes.data_as(C.POINTER(C.c_double))
        keep = (ls, la)
    return d, keep


class Medium:
    def __init__(self, ctx: Context, m: S.Medium):
        self.ctx = ctx
        self.scene = m
        d, keep = medium_desc(m)
        h = C.c_void_p()
        check(load().pmc_create_medium(ctx.handle, C.byref(d), C.byref(h)), "pmc_create_medium")
        self.handle = h
        self.n_theta = load().pmc_n_theta(h)

    def close(self):
        if self.handle:
            load().pmc_destroy_medium(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def create_medium(ctx: Context, m: S.Medium) -> Medium:
    return Medium(ctx, m)


class Geometry:
    def __init__(self, ctx: Context, sources: Sequence[S.Source], sensors: Sequence[S.Sensor],
                 pairs: Sequence[S.Pair]):
        self.ctx = ctx
        self.sources, self.sensors, self.pairs = list(sources), list(sensors), list(pairs)
        src = (SourceDesc * len(sources))()
        for i, s in enumerate(sources):
            src[i].pos[:] = [float(v) for v in s.pos]
            src[i].emission = int(s.emission)
            src[i].kappa = float(s.kappa)
            src[i].dir[:] = [float(v) for v in s.direction]
        sen = (SensorDesc * len(sensors))()
        for i, d in enumerate(sensors):
            sen[i].centre[:] = [float(v) for v in d.centre]
            sen[i].radius = float(d.radius)
            sen[i].rho = int(d.rho)
            sen[i].rho_hat[:] = [float(v) for v in d.rho_hat]
        prs = (PairDesc * len(pairs))()
        for i, p in enumerate(pairs):
            prs[i].source, prs[i].sensor = int(p.source), int(p.sensor)
            prs[i].n_chains, prs[i].cap = int(p.n_chains), int(p.cap)
        g = GeometryDesc(len(sources), src, len(sensors), sen, len(pairs), prs)
        h = C.c_void_p()
        check(load().pmc_create_geometry(ctx.handle, C.byref(g), C.byref(h)), "pmc_create_geometry")
        self.handle = h
        self.total_chains = int(sum(p.n_chains for p in pairs))
        self.max_cap = int(max(p.cap for p in pairs))

    def close(self):
        if self.handle:
            load().pmc_destroy_geometry(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def create_geometry(ctx: Context, sources, sensors, pairs) -> Geometry:
    return Geometry(ctx, sources, sensors, pairs)


def run_desc(r: S.Run, flags: int = 0, warps_per_block: int = 0, user_xyz: Optional[np.ndarray] = None,
             user_n: Optional[np.ndarray] = None, smem_window: int = 0, chain_window=(0, 0)):
    d = RunDesc()
    d.seed = int(r.seed)
    d.p_within, d.p_birth, d.p_death = float(r.p_within), float(r.p_birth), float(r.p_death)
    d.within = int(r.within)
    d.sigma = float(r.sigma)
    d.mala_step = float(r.mala_step)
    d.kappa_end = float(r.kappa_end)
    d.burn_in = int(r.burn_in)
    d.thin_bridge = int(r.thin_bridge)
    d.init = int(r.init)
    d.init_k = int(r.init_k)
    d.init_jitter = float(r.init_jitter)
    d.flags = int(flags) | (PMC_FLAG_GRADIENTS if r.gradients else 0)
    d.warps_per_block = int(warps_per_block)
    d.smem_window = int(smem_window)
    d.hmc_steps = int(getattr(r, "hmc_steps", 10))
    d.layout = int(getattr(r, "layout", 0))
    d.chain_lo, d.chain_hi = int(chain_window[0]), int(chain_window[1])
    keep = ()
    nm = getattr(r, "spectrum_nm", None)
    if nm is not None:
        x = np.ascontiguousarray(nm, dtype=np.float64)
        y = np.ascontiguousarray(r.spectrum, dtype=np.float64)
        d.n_lambda = len(x)
        d.lambda_nm = x.ctypes.data_as(C.POINTER(C.c_double))
        d.spectrum = y.ctypes.data_as(C.POINTER(C.c_double))
        d.sigma_lambda = float(r.sigma_lambda)
        keep = (x, y)
    if user_xyz is not None:
        ux = np.ascontiguousarray(user_xyz, dtype=np.float32)  # [chains][3][stride]
        un = np.ascontiguousarray(user_n, dtype=np.int32)
        d.init = S.INIT_USER
        d.init_xyz = ux.ctypes.data_as(C.POINTER(C.c_float))
        d.init_n = un.ctypes.data_as(C.POINTER(C.c_int))
        d.init_stride = int(ux.shape[2])
        keep = keep + (ux, un)
    return d, keep


class Chains:
    """Chains of every pair of a geometry (pmc_init_chains .. pmc_destroy_chains)."""

    def __init__(self, ctx: Context, medium: Medium, geom: Geometry, run: S.Run, flags: int = 0,
                 warps_per_block: int = 0, user_xyz=None, user_n=None, stream=None, smem_window: int = 0,
                 chain_window=(0, 0)):
        self.ctx, self.medium, self.geom, self.run = ctx, medium, geom, run
        self.chain_window = tuple(int(v) for v in chain_window)
        d, keep = run_desc(run, flags, warps_per_block, user_xyz, user_n, smem_window, chain_window)
        h = C.c_void_p()
        with torch.cuda.device(ctx.device):
            check(load().pmc_init_chains(ctx.handle, medium.handle, geom.handle, C.byref(d), _stream(stream),
                                         C.byref(h)), "pmc_init_chains")
        self.handle = h
        self.total = load().pmc_total_chains(h)
        self.n_pairs = len(geom.pairs)

    def reset(self, stream=None):
        """Re-initialise paths, step counters and accumulators (pmc_reset_chains)."""
        check(load().pmc_reset_chains(self.handle, _stream(stream)), "pmc_reset_chains")

    def set_states(self, xyz: np.ndarray, n: np.ndarray, stream=None):
        """Upload host paths [total][3][stride] and counts (pmc_set_states); arrays must outlive the copy."""
        if xyz.dtype != np.float32 or not xyz.flags.c_contiguous or xyz.ndim != 3 or xyz.shape[1] != 3:
            raise ValueError("xyz must be C-contiguous float32 of shape (total, 3, stride)")
        if n.dtype != np.int32 or not n.flags.c_contiguous:
            raise ValueError("n must be C-contiguous int32")
        check(load().pmc_set_states(self.handle, xyz.ctypes.data_as(C.POINTER(C.c_float)),
                                    n.ctypes.data_as(C.POINTER(C.c_int)), int(xyz.shape[2]), _stream(stream)),
              "pmc_set_states")

    def run_steps(self, n_steps: int, stream=None):
        check(load().pmc_run_steps(self.handle, int(n_steps), _stream(stream)), "pmc_run_steps")

    def read_estimator(self, stream=None):
        out = (Estimate * self.n_pairs)()
        check(load().pmc_read_estimator(self.handle, out, self.n_pairs, _stream(stream)), "pmc_read_estimator")
        return [e.as_dict() for e in out]

    def read_lambda(self, stream=None) -> np.ndarray:
        """The chains' current wavelengths in nm (pmc_read_lambda; wavelength sampling only)."""
        out = np.zeros(self.total, dtype=np.float32)
        check(load().pmc_read_lambda(self.handle, out.ctypes.data_as(C.POINTER(C.c_float)), self.total,
                                     _stream(stream)), "pmc_read_lambda")
        return out

    def read_moments(self, stream=None) -> np.ndarray:
        """Per-pair additive moments of this chain set (pmc_read_moments): (n_pairs, PMC_MOMENT_WORDS)."""
        out = np.zeros((self.n_pairs, PMC_MOMENT_WORDS))
        check(load().pmc_read_moments(self.handle, out.ctypes.data_as(C.POINTER(C.c_double)), out.size,
                                      _stream(stream)), "pmc_read_moments")
        return out

    def pair_z2(self, stream=None) -> np.ndarray:
        """Direct-sector integral of every pair (pmc_pair_z2)."""
        out = np.zeros(self.n_pairs)
        check(load().pmc_pair_z2(self.handle, out.ctypes.data_as(C.POINTER(C.c_double)), self.n_pairs,
                                 _stream(stream)), "pmc_pair_z2")
        return out

    def read_estimator_sharded(self, group=None, stream=None):
        """Estimates of the whole sharded chain set: this rank's moments, one
        sum all-reduce over the process group (torch.distributed), then
        pmc_estimate_from_moments.  Returns (estimates, grad, grad_se)."""
        import torch.distributed as dist
        mom = self.read_moments(stream)
        if dist.is_available() and dist.is_initialized():
            backend = dist.get_backend(group)
            dev = f"cuda:{self.ctx.device}" if backend == "nccl" else "cpu"
            t = torch.from_numpy(mom).to(dev)
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            mom = t.cpu().numpy()
        return estimate_from_moments(mom, self.pair_z2(stream))

    def grad_estimator(self, stream=None):
        nt = self.medium.n_theta
        g = np.zeros(self.n_pairs * nt)
        se = np.zeros(self.n_pairs * nt)
        check(load().pmc_grad_estimator(self.handle, g.ctypes.data_as(C.POINTER(C.c_double)),
                                        se.ctypes.data_as(C.POINTER(C.c_double)), len(g), _stream(stream)),
              "pmc_grad_estimator")
        return g.reshape(self.n_pairs, nt), se.reshape(self.n_pairs, nt)

    def bridge(self, n_draws: int, seed: int = 0, stream=None):
        """Geometric-bridge intensity per pair with the reference density (pmc_bridge): (I, SE) rows."""
        out = np.zeros((self.n_pairs, 2))
        check(load().pmc_bridge(self.handle, int(n_draws), int(seed), out.ctypes.data_as(C.POINTER(C.c_double)),
                                _stream(stream)), "pmc_bridge")
        return out

    def yield_observe(self, pair0: int, pair1: int, sums: torch.Tensor, stream=None):
        """One observation of sqrt(p_other/p_own) per chain of pair0 and pair1 (pmc_yield_observe)."""
        _require_cuda(sums, torch.float64, "sums")
        need = self.geom.pairs[pair0].n_chains + self.geom.pairs[pair1].n_chains
        if sums.numel() != need:
            raise ValueError(f"sums must hold {need} doubles")
        check(load().pmc_yield_observe(self.handle, int(pair0), int(pair1), C.c_void_p(sums.data_ptr()),
                                       _stream(stream)), "pmc_yield_observe")

    def yield_estimate(self, pair0: int, pair1: int, sums: torch.Tensor, n_obs: int, stream=None) -> dict:
        """B = light on pair1's sensor / light on pair0's sensor from the observation sums (pmc_yield_estimate)."""
        _require_cuda(sums, torch.float64, "sums")
        out = np.zeros(6)
        check(load().pmc_yield_estimate(self.handle, int(pair0), int(pair1), C.c_void_p(sums.data_ptr()),
                                        int(n_obs), out.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)),
              "pmc_yield_estimate")
        return {"B": out[0], "se": out[1], "E0": out[2], "E1": out[3], "var0": out[4], "var1": out[5]}

    def yield_observe_log(self, pair0: int, pair1: int, row: torch.Tensor, stream=None):
        """One observation of the log density ratios of pair0's and pair1's chains (pmc_yield_observe_log)."""
        _require_cuda(row, torch.float32, "row")
        need = self.geom.pairs[pair0].n_chains + self.geom.pairs[pair1].n_chains
        if row.numel() != need:
            raise ValueError(f"row must hold {need} floats")
        check(load().pmc_yield_observe_log(self.handle, int(pair0), int(pair1), C.c_void_p(row.data_ptr()),
                                           _stream(stream)), "pmc_yield_observe_log")

    def score_observe(self, sums: torch.Tensor, stream=None):
        """One observation of d log p / d theta at every chain's current path
        into sums (n_pairs, 4 L): per-layer scores then their squares
        (pmc_score_observe; layered media)."""
        _require_cuda(sums, torch.float64, "sums")
        if sums.dim() != 2 or sums.shape[0] != self.n_pairs or sums.shape[1] != 2 * self.medium.n_theta:
            raise ValueError("sums must have shape (n_pairs, 2 n_theta)")
        check(load().pmc_score_observe(self.handle, C.c_void_p(sums.data_ptr()), _stream(stream)),
              "pmc_score_observe")

    def length_hist(self, l_lo: float, l_hi: float, hist: torch.Tensor, stream=None):
        """One observation of every chain's path length into hist (n_pairs, n_bins) (pmc_length_hist)."""
        _require_cuda(hist, torch.float64, "hist")
        if hist.dim() != 2 or hist.shape[0] != self.n_pairs:
            raise ValueError("hist must have shape (n_pairs, n_bins)")
        check(load().pmc_length_hist(self.handle, float(l_lo), float(l_hi), int(hist.shape[1]),
                                     C.c_void_p(hist.data_ptr()), _stream(stream)), "pmc_length_hist")

    def bridge_observe_log(self, pair: int, n_draws: int, draw0: int, seed: int, row: torch.Tensor, stream=None):
        """One row of q_ref-bridge log ratios for `pair` (pmc_bridge_observe_log): n_draws
        reference draws' log(p/q_ref), then the pair's chains' log(q_ref/p)."""
        _require_cuda(row, torch.float32, "row")
        if row.numel() != n_draws + self.geom.pairs[pair].n_chains:
            raise ValueError("row must hold n_draws + n_chains floats")
        check(load().pmc_bridge_observe_log(self.handle, int(pair), int(n_draws), int(draw0), int(seed),
                                            C.c_void_p(row.data_ptr()), _stream(stream)), "pmc_bridge_observe_log")

    def read_states(self, stream=None):
        stride = self.geom.max_cap
        xyz = np.zeros((self.total, 3, stride), dtype=np.float32)
        n = np.zeros(self.total, dtype=np.int32)
        steps = np.zeros(self.total, dtype=np.uint64)
        check(load().pmc_read_states(self.handle, xyz.ctypes.data_as(C.POINTER(C.c_float)),
                                     n.ctypes.data_as(C.POINTER(C.c_int)),
                                     steps.ctypes.data_as(C.POINTER(C.c_uint64)), stride, _stream(stream)),
              "pmc_read_states")
        return xyz, n, steps

    def launch_info(self):
        """Per cap class: shared window, order range, warps per block, grid, general kernel (pmc_chains_launch_info)."""
        rows = np.zeros((8, 6), dtype=np.int32)
        nc = C.c_int(0)
        check(load().pmc_chains_launch_info(self.handle, rows.ctypes.data_as(C.POINTER(C.c_int)), 8, C.byref(nc)),
              "pmc_chains_launch_info")
        keys = ("smem_cap", "lo", "hi", "warps_per_block", "grid", "general")
        return [dict(zip(keys, map(int, r))) for r in rows[: nc.value]]

    def read_accumulators(self, stream=None):
        out = np.zeros((self.total, PMC_ACC_WORDS))
        check(load().pmc_read_accumulators(self.handle, out.ctypes.data_as(C.POINTER(C.c_double)), out.size,
                                           _stream(stream)), "pmc_read_accumulators")
        return out

    def save_state(self, stream=None) -> bytes:
        size = C.c_size_t(0)
        check(load().pmc_save_state(self.handle, None, C.byref(size), _stream(stream)), "pmc_save_state")
        buf = C.create_string_buffer(size.value)
        check(load().pmc_save_state(self.handle, buf, C.byref(size), _stream(stream)), "pmc_save_state")
        return buf.raw

    def load_state(self, blob: bytes, stream=None):
        buf = C.create_string_buffer(blob, len(blob))
        check(load().pmc_load_state(self.handle, buf, len(blob), _stream(stream)), "pmc_load_state")

    def request_abort(self, flag: bool = True):
        check(load().pmc_request_abort(self.handle, int(bool(flag))), "pmc_request_abort")

    def status(self, stream=None) -> int:
        st = C.c_int(0)
        check(load().pmc_chain_status(self.handle, C.byref(st), _stream(stream)), "pmc_chain_status")
        return st.value

    def close(self):
        if self.handle:
            load().pmc_destroy_chains(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shard_range(pairs: Sequence[S.Pair], rank: int, world: int):
    """Chain window (lo, hi) of `rank` among `world` ranks (pmc_shard_range)."""
    prs = (PairDesc * len(pairs))()
    for i, p in enumerate(pairs):
        prs[i].source, prs[i].sensor = int(p.source), int(p.sensor)
        prs[i].n_chains, prs[i].cap = int(p.n_chains), int(p.cap)
    lo, hi = C.c_int64(0), C.c_int64(0)
    check(load().pmc_shard_range(prs, len(pairs), int(rank), int(world), C.byref(lo), C.byref(hi)),
          "pmc_shard_range")
    return int(lo.value), int(hi.value)


def estimate_from_moments(moments: np.ndarray, z2: np.ndarray):
    """Per-pair estimates from (all-reduced) moments (pmc_estimate_from_moments):
    (list of estimate dicts, grad (n_pairs, 3), grad_se (n_pairs, 3))."""
    mom = np.ascontiguousarray(moments, dtype=np.float64)
    z = np.ascontiguousarray(z2, dtype=np.float64)
    n = len(z)
    if mom.shape != (n, PMC_MOMENT_WORDS):
        raise ValueError("moments must have shape (n_pairs, PMC_MOMENT_WORDS)")
    out = (Estimate * n)()
    g = np.zeros((n, 3))
    gs = np.zeros((n, 3))
    check(load().pmc_estimate_from_moments(mom.ctypes.data_as(C.POINTER(C.c_double)), n,
                                           z.ctypes.data_as(C.POINTER(C.c_double)), out,
                                           g.ctypes.data_as(C.POINTER(C.c_double)),
                                           gs.ctypes.data_as(C.POINTER(C.c_double))), "pmc_estimate_from_moments")
    return [e.as_dict() for e in out], g, gs


def moments_from_accumulators(acc: np.ndarray, chain_pair: np.ndarray, n_pairs: int, lambda_s: float = 1.0,
                              lambda_a: float = 1.0) -> np.ndarray:
    """Host moments of accumulator rows (pmc_moments_from_accumulators)."""
    a = np.ascontiguousarray(acc, dtype=np.float64)
    cp = np.ascontiguousarray(chain_pair, dtype=np.int32)
    if a.ndim != 2 or a.shape[1] != PMC_ACC_WORDS or len(cp) != len(a):
        raise ValueError("acc must have shape (n_chains, PMC_ACC_WORDS) and chain_pair n_chains entries")
    out = np.zeros((int(n_pairs), PMC_MOMENT_WORDS))
    check(load().pmc_moments_from_accumulators(a.ctypes.data_as(C.POINTER(C.c_double)), len(a),
                                               cp.ctypes.data_as(C.POINTER(C.c_int)), int(n_pairs),
                                               float(lambda_s), float(lambda_a),
                                               out.ctypes.data_as(C.POINTER(C.c_double))),
          "pmc_moments_from_accumulators")
    return out


def init_chains(ctx, medium, geom, run, **kw) -> Chains:
    return Chains(ctx, medium, geom, run, **kw)


def run_steps(chains: Chains, n_steps: int, stream=None):
    chains.run_steps(n_steps, stream)


def read_estimator(chains: Chains, stream=None):
    return chains.read_estimator(stream)


def grad_estimator(chains: Chains, stream=None):
    return chains.grad_estimator(stream)


def _check_batch(xyz: torch.Tensor, n: torch.Tensor):
    _require_cuda(xyz, torch.float32, "xyz")
    _require_cuda(n, torch.int32, "n")
    if xyz.dim() != 3 or xyz.shape[0] != 3:
        raise ValueError("xyz must have shape (3, batch, cap)")
    batch, cap = int(xyz.shape[1]), int(xyz.shape[2])
    if n.shape != (batch,):
        raise ValueError("n must have shape (batch,)")
    return batch, cap


def logp(ctx: Context, medium: Medium, geom: Geometry, pair: int, xyz: torch.Tensor, n: torch.Tensor,
         stream=None) -> torch.Tensor:
    """log p of a device batch (pmc_logp); xyz float32 (3, batch, cap), n int32 (batch,)."""
    batch, cap = _check_batch(xyz, n)
    out = torch.empty(batch, dtype=torch.float32, device=xyz.device)
    check(load().pmc_logp(ctx.handle, medium.handle, geom.handle, int(pair), C.c_void_p(xyz.data_ptr()),
                          C.c_void_p(n.data_ptr()), batch, cap, C.c_void_p(out.data_ptr()), _stream(stream)),
          "pmc_logp")
    return out


def logp_grad(ctx: Context, medium: Medium, geom: Geometry, pair: int, xyz: torch.Tensor, n: torch.Tensor,
              stream=None):
    """log p and d log p / d xyz (pmc_logp_grad)."""
    batch, cap = _check_batch(xyz, n)
    lp = torch.empty(batch, dtype=torch.float32, device=xyz.device)
    g = torch.empty_like(xyz)
    check(load().pmc_logp_grad(ctx.handle, medium.handle, geom.handle, int(pair), C.c_void_p(xyz.data_ptr()),
                               C.c_void_p(n.data_ptr()), batch, cap, C.c_void_p(lp.data_ptr()),
                               C.c_void_p(g.data_ptr()), _stream(stream)), "pmc_logp_grad")
    return lp, g


def score(ctx: Context, medium: Medium, geom: Geometry, pair: int, xyz: torch.Tensor, n: torch.Tensor,
          stream=None) -> torch.Tensor:
    """d log p / d theta per path (pmc_score)."""
    batch, cap = _check_batch(xyz, n)
    out = torch.empty((batch, medium.n_theta), dtype=torch.float32, device=xyz.device)
    check(load().pmc_score(ctx.handle, medium.handle, geom.handle, int(pair), C.c_void_p(xyz.data_ptr()),
                           C.c_void_p(n.data_ptr()), batch, cap, C.c_void_p(out.data_ptr()), _stream(stream)),
          "pmc_score")
    return out


def _trace_dict(r: TraceResult) -> dict:
    d = r.as_dict()
    # short names used throughout the tests and the benchmark
    d.update(I=d["intensity"], se=d["std_err"], mean_L=d["mean_length"], hits=d["detected"], photons=d["emitted"])
    return d


def trace(ctx: Context, medium: Medium, geom: Geometry, pair: int, seed: int, n_photons: int, photon0: int = 0,
          r_reject: float = math.inf, max_scatter: int = 1000, stream=None):
    """GPU forward tracer (pmc_trace): the pmc_trace_result fields as a dict,
    with the short names I, se, mean_L, hits, photons.  A photon that never
    reaches the sensor scatters until max_scatter or until it starts a flight
    beyond r_reject: with r_reject infinite the scattering limit alone ends
    it, so keep max_scatter to the path lengths of interest (the chains' cap
    - 2 for a cap-truncated comparison)."""
    out = TraceResult()
    check(load().pmc_trace(ctx.handle, medium.handle, geom.handle, int(pair), int(seed), int(photon0),
                           int(n_photons), float(r_reject), int(min(max_scatter, 2**31 - 1)), C.byref(out),
                           _stream(stream)), "pmc_trace")
    return _trace_dict(out)


def trace_lengths(ctx: Context, medium: Medium, geom: Geometry, pair: int, seed: int, n_photons: int, l_lo: float,
                  l_hi: float, n_bins: int, photon0: int = 0, r_reject: float = math.inf, max_scatter: int = 1000,
                  stream=None):
    """GPU forward tracer with the detected weight binned by path length
    (pmc_trace_lengths): (result dict as trace(), weight per bin per emitted photon)."""
    out = TraceResult()
    hist = np.zeros(int(n_bins))
    check(load().pmc_trace_lengths(ctx.handle, medium.handle, geom.handle, int(pair), int(seed), int(photon0),
                                   int(n_photons), float(r_reject), int(min(max_scatter, 2**31 - 1)), float(l_lo),
                                   float(l_hi), int(n_bins), C.byref(out), hist.ctypes.data_as(C.POINTER(C.c_double)),
                                   _stream(stream)), "pmc_trace_lengths")
    return _trace_dict(out), hist


def yield_logratio(ctx: Context, medium: Medium, geom: Geometry, pair0: int, pair1: int, side: int,
                   xyz: torch.Tensor, n: torch.Tensor, mapped: bool = False, stream=None):
    """Log density ratio of the other sensor's density (through the map T) to
    the own one for a device batch (pmc_yield_logratio); with mapped=True also
    the mapped paths (3, batch, cap)."""
    batch, cap = _check_batch(xyz, n)
    out = torch.empty(batch, dtype=torch.float32, device=xyz.device)
    oxyz = torch.zeros_like(xyz) if mapped else None
    check(load().pmc_yield_logratio(ctx.handle, medium.handle, geom.handle, int(pair0), int(pair1), int(side),
                                    C.c_void_p(xyz.data_ptr()), C.c_void_p(n.data_ptr()), batch, cap,
                                    C.c_void_p(out.data_ptr()),
                                    C.c_void_p(oxyz.data_ptr() if mapped else None), _stream(stream)),
          "pmc_yield_logratio")
    return (out, oxyz) if mapped else out


def bridge_ratio(ctx: Context, logr: torch.Tensor, n0: int, n1: int, groups: int = 16, max_iter: int = 200,
                 tol: float = 1e-10, stream=None) -> dict:
    """Optimal bridge estimate of c1/c0 from stored log ratios (pmc_bridge_ratio);
    logr: float32 (rows, n0 + n1) on the device."""
    _require_cuda(logr, torch.float32, "logr")
    if logr.dim() != 2 or logr.shape[1] != n0 + n1:
        raise ValueError("logr must have shape (rows, n0 + n1)")
    out = np.zeros(4)
    check(load().pmc_bridge_ratio(ctx.handle, C.c_void_p(logr.data_ptr()), int(logr.shape[0]), int(n0), int(n1),
                                  int(groups), int(max_iter), float(tol), out.ctypes.data_as(C.POINTER(C.c_double)),
                                  _stream(stream)), "pmc_bridge_ratio")
    return {"r": out[0], "se": out[1], "iterations": int(out[2]), "geometric": out[3]}


class YieldRatio:
    """Relative light yield B of two pairs sharing a source (pair1's sensor over
    pair0's): a device buffer of per-chain sums, filled by observe() between
    run_steps calls and reduced by estimate() (the paper's geometric
    estimator); with max_obs > 0 every observation's log ratios are also kept
    (max_obs rows) for estimate_bridge() (the optimal bridge)."""

    def __init__(self, chains: Chains, pair0: int, pair1: int, max_obs: int = 0):
        self.chains, self.pair0, self.pair1 = chains, int(pair0), int(pair1)
        self.n0 = chains.geom.pairs[pair0].n_chains
        self.n1 = chains.geom.pairs[pair1].n_chains
        dev = f"cuda:{chains.ctx.device}"
        self.sums = torch.zeros(self.n0 + self.n1, dtype=torch.float64, device=dev)
        self.logr = torch.zeros((int(max_obs), self.n0 + self.n1), dtype=torch.float32, device=dev) if max_obs else None
        self.n_obs = 0

    def observe(self, stream=None):
        self.chains.yield_observe(self.pair0, self.pair1, self.sums, stream)
        if self.logr is not None and self.n_obs < self.logr.shape[0]:
            self.chains.yield_observe_log(self.pair0, self.pair1, self.logr[self.n_obs], stream)
        self.n_obs += 1

    def estimate(self, stream=None) -> dict:
        return self.chains.yield_estimate(self.pair0, self.pair1, self.sums, self.n_obs, stream)

    def estimate_bridge(self, groups: int = 16, stream=None) -> dict:
        rows = min(self.n_obs, self.logr.shape[0])
        return bridge_ratio(self.chains.ctx, self.logr[:rows], self.n0, self.n1, groups, stream=stream)


def qref_logdensity(ctx: Context, medium: Medium, geom: Geometry, pair: int, xyz: torch.Tensor, n: torch.Tensor,
                    stream=None) -> torch.Tensor:
    """log q_ref of a device batch (pmc_qref_logdensity)."""
    batch, cap = _check_batch(xyz, n)
    out = torch.empty(batch, dtype=torch.float32, device=xyz.device)
    check(load().pmc_qref_logdensity(ctx.handle, medium.handle, geom.handle, int(pair), C.c_void_p(xyz.data_ptr()),
                                     C.c_void_p(n.data_ptr()), batch, cap, C.c_void_p(out.data_ptr()),
                                     _stream(stream)), "pmc_qref_logdensity")
    return out


def qref_sample(ctx: Context, medium: Medium, geom: Geometry, pair: int, seed: int, n_draws: int, draw0: int = 0,
                stride: Optional[int] = None, stream=None):
    """Reference-density draws (pmc_qref_sample): xyz (3, n_draws, stride) and n on the device."""
    stride = int(stride or geom.pairs[pair].cap)
    xyz = torch.zeros((3, int(n_draws), stride), dtype=torch.float32, device="cuda")
    n = torch.zeros(int(n_draws), dtype=torch.int32, device="cuda")
    check(load().pmc_qref_sample(ctx.handle, medium.handle, geom.handle, int(pair), int(seed), int(draw0),
                                 int(n_draws), C.c_void_p(xyz.data_ptr()), C.c_void_p(n.data_ptr()), stride,
                                 _stream(stream)), "pmc_qref_sample")
    return xyz, n


def trace_noalloc(ctx: Context, medium: Medium, geom: Geometry, pairs, seed: int, n_photons: int,
                  photon0: int = 0, r_reject: float = math.inf, max_scatter: int = 1000, stream=None):
    """Allocation-free GPU tracer over several pairs (pmc_trace_noalloc): one
    result dict per pair, as trace() returns."""
    ids = np.ascontiguousarray(pairs, dtype=np.int32)
    out = (TraceResult * max(len(ids), 1))()
    check(load().pmc_trace_noalloc(ctx.handle, medium.handle, geom.handle, ids.ctypes.data_as(C.POINTER(C.c_int)),
                                   len(ids), int(seed), int(photon0), int(n_photons), float(r_reject),
                                   int(min(max_scatter, 2**31 - 1)), out, _stream(stream)), "pmc_trace_noalloc")
    return [_trace_dict(out[i]) for i in range(len(ids))]


def trace_paths(ctx: Context, medium: Medium, geom: Geometry, pair: int, seed: int, n_photons: int,
                max_paths: int, photon0: int = 0, max_scatter: Optional[int] = None, r_reject: float = math.inf,
                stride: Optional[int] = None, stream=None):
    """Weight-thinned detected tracer paths (pmc_trace_paths): exact draws from
    the normalised path density; returns (xyz (3, kept, stride), n, kept)."""
    cap = geom.pairs[pair].cap
    ms = cap - 2 if max_scatter is None else int(max_scatter)
    stride = int(stride or ms + 2)
    xyz = torch.zeros((3, int(max_paths), stride), dtype=torch.float32, device="cuda")
    n = torch.zeros(int(max_paths), dtype=torch.int32, device="cuda")
    acc = C.c_uint64(0)
    check(load().pmc_trace_paths(ctx.handle, medium.handle, geom.handle, int(pair), int(seed), int(photon0),
                                 int(n_photons), float(r_reject), ms, int(max_paths), C.c_void_p(xyz.data_ptr()),
                                 C.c_void_p(n.data_ptr()), stride, C.byref(acc), _stream(stream)), "pmc_trace_paths")
    kept = min(int(acc.value), int(max_paths))
    return xyz[:, :kept], n[:kept], int(acc.value)


def seed_from_tracer(chains: "Chains", seed: int = 2024, photons_per_round: int = 1 << 26, max_rounds: int = 64,
                     r_reject: float = math.inf, stream=None):
    """Start every chain from an equilibrium path: the first weight-thinned
    tracer photons of each pair, in photon order (pmc_seed_from_tracer).
    Pair p traces with Philox key seed + p.  r_reject: photons farther than
    this from the sensor centre are dropped (a finite radius shortens the
    tracing of escaping photons; its bias is the weight of paths that leave
    the ball and return).  Returns the photons traced per pair."""
    used = np.zeros(chains.n_pairs, dtype=np.uint64)
    check(load().pmc_seed_from_tracer(chains.handle, int(seed), int(photons_per_round), int(max_rounds),
                                      float(r_reject), used.ctypes.data_as(C.POINTER(C.c_uint64)), _stream(stream)),
          "pmc_seed_from_tracer")
    return [int(u) for u in used]


def seed_select(photon_idx, need: int) -> np.ndarray:
    """The seed selection of pmc_seed_from_tracer on host data (pmc_seed_select)."""
    idx = np.ascontiguousarray(photon_idx, dtype=np.uint64)
    out = np.zeros(int(need), dtype=np.uint64)
    check(load().pmc_seed_select(idx.ctypes.data_as(C.POINTER(C.c_uint64)), len(idx), int(need),
                                 out.ctypes.data_as(C.POINTER(C.c_uint64))), "pmc_seed_select")
    return out


class LogP(torch.autograd.Function):
    """log p of a batch of paths; backward is the hand-written adjoint kernel."""

    @staticmethod
    def forward(fctx, xyz, n, handles):
        ctx_, med, geom, pair = handles
        lp, g = logp_grad(ctx_, med, geom, pair, xyz.contiguous(), n)
        fctx.save_for_backward(g)
        return lp

    @staticmethod
    def backward(fctx, grad_out):
        (g,) = fctx.saved_tensors
        return g * grad_out.view(1, -1, 1), None, None


class PathSampler:
    """Everything for one scene: context, medium, geometry and chains."""

    def __init__(self, scene: S.Scene, device: int = 0, flags: int = 0, warps_per_block: int = 0,
                 user_xyz=None, user_n=None):
        self.scene = scene
        self.ctx = Context(device)
        self.medium = Medium(self.ctx, scene.medium)
        self.geom = Geometry(self.ctx, scene.sources, scene.sensors, scene.pairs)
        self.chains = Chains(self.ctx, self.medium, self.geom, scene.run, flags, warps_per_block, user_xyz, user_n)

    def run(self, n_steps: Optional[int] = None):
        self.chains.run_steps(self.scene.run.n_steps if n_steps is None else n_steps)
        return self

    def estimate(self):
        return self.chains.read_estimator()
