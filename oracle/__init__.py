"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  The CUDA product path never
does.  The C sources in this folder are compiled with gcc into
``oracle/_build/liboracle.so`` and driven through ctypes; scene objects are
read by attribute (duck typing), so this package imports nothing from the
product package.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "oracle.c")]
_HDR = os.path.join(_HERE, "oracle.h")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, FP64, pthreads)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [_HDR])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", tmp] + _SRC + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Medium(C.Structure):
    _fields_ = [("kind", C.c_int), ("lambda_s", C.c_double), ("lambda_a", C.c_double),
                ("g", C.c_double), ("f_sl", C.c_double), ("z0", C.c_double), ("dz", C.c_double),
                ("n_layers", C.c_int), ("lambda_s_layers", C.POINTER(C.c_double)),
                ("lambda_a_layers", C.POINTER(C.c_double)), ("lambda0", C.c_double), ("k_s", C.c_double),
                ("k_a", C.c_double)]


class Source(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("emission", C.c_int), ("kappa", C.c_double),
                ("dir", C.c_double * 3)]


class Sensor(C.Structure):
    _fields_ = [("c", C.c_double * 3), ("R", C.c_double), ("rho", C.c_int),
                ("rho_hat", C.c_double * 3)]


class Run(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("p_within", C.c_double), ("p_birth", C.c_double),
                ("p_death", C.c_double), ("within", C.c_int), ("sigma", C.c_double),
                ("mala_step", C.c_double), ("kappa_end", C.c_double), ("burn_in", C.c_uint64),
                ("thin_bridge", C.c_uint32), ("gradients", C.c_int), ("beta_min", C.c_double),
                ("hmc_steps", C.c_int), ("toy_s", C.c_double), ("toy_w", C.POINTER(C.c_double)),
                ("n_lambda", C.c_int), ("lambda_nm", C.POINTER(C.c_double)), ("spectrum", C.POINTER(C.c_double)),
                ("sigma_lambda", C.c_double)]


class Acc(C.Structure):
    _fields_ = [("n_rec", C.c_double), ("n_direct", C.c_double), ("sum_n", C.c_double),
                ("sum_L", C.c_double), ("sum_L2", C.c_double), ("sum_score", C.c_double * 3),
                ("sum_bridge", C.c_double), ("n_bridge", C.c_double),
                ("prop", C.c_double * 4), ("acc", C.c_double * 4)]


class YMap(C.Structure):
    _fields_ = [("f0", C.c_double * 3), ("eta0", C.c_double * 3), ("eta1", C.c_double * 3),
                ("R0", C.c_double), ("R1", C.c_double), ("k", C.c_double * 3), ("m", C.c_double * 3),
                ("n", C.c_double * 3), ("b0", C.c_double), ("b1", C.c_double), ("rC", C.c_double),
                ("Omega", C.c_double)]


ACC_FIELDS = ["n_rec", "n_direct", "sum_n", "sum_L", "sum_L2", "sum_bridge", "n_bridge"]

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            M, S, D, R = C.POINTER(Medium), C.POINTER(Source), C.POINTER(Sensor), C.POINTER(Run)
            L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.or_u01.argtypes = [C.c_uint32]; L.or_u01.restype = C.c_double
            L.or_onb.argtypes = [_dp, _dp, _dp]
            L.or_kappa_eq.argtypes = [C.c_double]; L.or_kappa_eq.restype = C.c_double
            L.or_log_sigma.argtypes = [M, C.c_double]; L.or_log_sigma.restype = C.c_double
            L.or_log_sigma_cos.argtypes = [M, C.c_double]; L.or_log_sigma_cos.restype = C.c_double
            L.or_log_emission.argtypes = [S, _dp]; L.or_log_emission.restype = C.c_double
            L.or_log_rho.argtypes = [D, _dp]; L.or_log_rho.restype = C.c_double
            L.or_segment_depths.argtypes = [M, _dp, _dp, _dp, _dp]
            L.or_segment_hits_ball.argtypes = [_dp, _dp, _dp, C.c_double]; L.or_segment_hits_ball.restype = C.c_int
            L.or_logp.argtypes = [M, S, D, C.c_int, _dp]; L.or_logp.restype = C.c_double
            L.or_grad_logp.argtypes = [M, S, D, C.c_int, _dp, _dp]; L.or_grad_logp.restype = C.c_double
            L.or_score.argtypes = [M, S, D, C.c_int, _dp, _dp]; L.or_score.restype = C.c_int
            L.or_bisph_point.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, _dp]
            L.or_bisph_coords.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp]
            L.or_log_bisph_jacobian.argtypes = [C.c_double] * 3; L.or_log_bisph_jacobian.restype = C.c_double
            L.or_log_q_s.argtypes = [C.c_double, C.c_double]; L.or_log_q_s.restype = C.c_double
            L.or_log_q_t.argtypes = [C.c_double]; L.or_log_q_t.restype = C.c_double
            L.or_init_chains.argtypes = [M, S, D, R, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int,
                                         C.c_uint32, _dp, _ip]
            L.or_run_chains.argtypes = [M, S, D, R, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint64,
                                        _dp, _ip, C.POINTER(Acc), _dp, C.c_int]
            L.or_z2.argtypes = [M, S, D, C.c_int, C.c_int]; L.or_z2.restype = C.c_double
            L.or_qref_logdensity.argtypes = [M, S, D, C.c_int, C.c_int, _dp]
            L.or_qref_logdensity.restype = C.c_double
            L.or_qref_sample.argtypes = [M, S, D, C.c_int, C.c_uint64, C.c_uint32, C.c_uint64, _dp]
            L.or_qref_sample.restype = C.c_int
            L.or_qref_bridge_sums.argtypes = [M, S, D, C.c_int, C.c_uint64, C.c_uint32, C.c_uint64, _dp, C.c_int]
            L.or_trace.argtypes = [M, S, D, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double, C.c_int, _dp, C.c_int]
            L.or_trace_hist.argtypes = [M, S, D, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double, C.c_int, _dp, _dp,
                                        C.c_int]
            L.or_trace_lhist.argtypes = [M, S, D, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double, C.c_int,
                                         C.c_double, C.c_double, C.c_int, _dp, _dp, C.c_int]
            Y = C.POINTER(YMap)
            L.or_ymap_init.argtypes = [S, D, D, Y]
            L.or_ymap_forward.argtypes = [Y, C.c_int, _dp, _dp]; L.or_ymap_forward.restype = C.c_double
            L.or_ymap_inverse.argtypes = [Y, C.c_int, _dp, _dp]; L.or_ymap_inverse.restype = C.c_double
            L.or_ymap_logratio.argtypes = [M, S, D, D, Y, C.c_int, C.c_int, _dp]
            L.or_ymap_logratio.restype = C.c_double
            L.or_tree_node.argtypes = [C.c_int, C.c_int, _ip, _ip, _ip]
            L.or_tree_coords.argtypes = [_dp, C.c_int, _dp, _dp]; L.or_tree_coords.restype = C.c_double
            L.or_tree_path.argtypes = [_dp, C.c_int, _dp, _dp]
            L.or_tree_vref.argtypes = [S, D, _dp]
            L.or_hmc_leapfrog.argtypes = [M, S, D, C.c_int, _dp, _dp, C.c_double, C.c_int]
            L.or_hmc_leapfrog.restype = C.c_double
            L.or_run_chains_hist.argtypes = [M, S, D, R, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint64,
                                             _dp, _ip, C.POINTER(Acc), _dp, _dp, C.c_int]
            L.or_run_chains_diag.argtypes = [M, S, D, R, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint64,
                                             _dp, _ip, C.POINTER(Acc), _dp, _dp, _dp, C.c_int]
            L.or_run_chains_lam.argtypes = [M, S, D, R, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint64,
                                            _dp, _ip, _dp, C.POINTER(Acc), _dp, _dp, _dp, C.c_int]
            L.or_medium_at.argtypes = [M, C.c_double, M]
            L.or_log_spectrum.argtypes = [R, C.c_double]; L.or_log_spectrum.restype = C.c_double
            L.or_spectrum_quantile.argtypes = [R, C.c_double]; L.or_spectrum_quantile.restype = C.c_double
            L.or_init_lambda.argtypes = [R, C.c_int, C.c_uint32, _dp]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


# ---------------------------------------------------------------------------
# Scene conversion (duck-typed: any object with the scene attributes works)
# ---------------------------------------------------------------------------
class _Keep:
    """Keeps numpy arrays referenced by ctypes structs alive."""


def medium(m) -> Medium:
    out = Medium()
    out.kind = int(m.kind)
    out.lambda_s = float(m.lambda_s)
    out.lambda_a = float(m.lambda_a)
    out.g = float(m.g)
    out.f_sl = float(getattr(m, "f_sl", 0.0))
    out.z0 = float(getattr(m, "z0", 0.0))
    out.dz = float(getattr(m, "dz", 1.0))
    ls = getattr(m, "lambda_s_layers", None)
    if ls is not None:
        a = np.ascontiguousarray(ls, dtype=np.float64)
        b = np.ascontiguousarray(m.lambda_a_layers, dtype=np.float64)
        out.n_layers = len(a)
        out.lambda_s_layers = _ptr(a)
        out.lambda_a_layers = _ptr(b)
        out._keep = (a, b)
    else:
        out.n_layers = 0
    out.lambda0 = float(getattr(m, "lambda0", 0.0))
    out.k_s = float(getattr(m, "k_s", 0.0))
    out.k_a = float(getattr(m, "k_a", 0.0))
    return out


def source(s) -> Source:
    out = Source()
    out.pos[:] = [float(v) for v in s.pos]
    out.emission = int(s.emission)
    out.kappa = float(s.kappa)
    d = np.asarray(s.direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    out.dir[:] = list(d)
    return out


def sensor(d) -> Sensor:
    out = Sensor()
    out.c[:] = [float(v) for v in d.centre]
    out.R = float(d.radius)
    out.rho = int(d.rho)
    rh = np.asarray(d.rho_hat, dtype=np.float64)
    out.rho_hat[:] = list(rh / np.linalg.norm(rh))
    return out


def run(r, sensor_radius: float) -> Run:
    out = Run()
    out.seed = int(r.seed)
    out.p_within = float(r.p_within)
    out.p_birth = float(r.p_birth)
    out.p_death = float(r.p_death)
    out.within = int(r.within)
    out.sigma = float(r.sigma)
    out.mala_step = float(r.mala_step)
    ke = float(r.kappa_end)
    if ke > 0:
        out.kappa_end = ke
    elif int(r.within) == 2:
        out.kappa_end = 1.0 / float(r.sigma) ** 2  # tree moves: sigma is dimensionless
    else:
        out.kappa_end = (sensor_radius / float(r.sigma)) ** 2
    out.burn_in = int(r.burn_in)
    out.thin_bridge = int(r.thin_bridge)
    out.gradients = int(bool(r.gradients))
    out.beta_min = 0.01
    out.hmc_steps = int(getattr(r, "hmc_steps", 10))
    nm = getattr(r, "spectrum_nm", None)
    if nm is not None and len(nm) >= 2:
        x = np.ascontiguousarray(nm, dtype=np.float64)
        y = np.ascontiguousarray(r.spectrum, dtype=np.float64)
        out.n_lambda = len(x)
        out.lambda_nm = _ptr(x)
        out.spectrum = _ptr(y)
        out.sigma_lambda = float(r.sigma_lambda)
        out._keep = (x, y)
    return out


# ---------------------------------------------------------------------------
# Thin wrappers
# ---------------------------------------------------------------------------
def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def kappa_eq(G: float) -> float:
    return lib().or_kappa_eq(G)


def log_sigma(m: Medium, c: float) -> float:
    return lib().or_log_sigma(C.byref(m), c)


def log_sigma_cos(m: Medium, c: float) -> float:
    return lib().or_log_sigma_cos(C.byref(m), c)


def log_emission(s: Source, rhat) -> float:
    v = np.ascontiguousarray(rhat, dtype=np.float64)
    return lib().or_log_emission(C.byref(s), _ptr(v))


def log_rho(d: Sensor, nu) -> float:
    v = np.ascontiguousarray(nu, dtype=np.float64)
    return lib().or_log_rho(C.byref(d), _ptr(v))


def segment_depths(m: Medium, P, Q):
    P = np.ascontiguousarray(P, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    ta, tb = C.c_double(), C.c_double()
    lib().or_segment_depths(C.byref(m), _ptr(P), _ptr(Q), C.byref(ta), C.byref(tb))
    return ta.value, tb.value


def logp(m: Medium, s: Source, d: Sensor, path) -> float:
    f = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 3)
    return lib().or_logp(C.byref(m), C.byref(s), C.byref(d), len(f), _ptr(f))


def grad_logp(m: Medium, s: Source, d: Sensor, path):
    f = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 3)
    g = np.zeros_like(f)
    lp = lib().or_grad_logp(C.byref(m), C.byref(s), C.byref(d), len(f), _ptr(f), _ptr(g))
    return lp, g


def score(m: Medium, s: Source, d: Sensor, path):
    f = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(max(3, 2 * m.n_layers), dtype=np.float64)
    k = lib().or_score(C.byref(m), C.byref(s), C.byref(d), len(f), _ptr(f), _ptr(out))
    return out[:k]


def bisph_point(fk, fk1, s, t, phi):
    a = np.ascontiguousarray(fk, dtype=np.float64)
    b = np.ascontiguousarray(fk1, dtype=np.float64)
    o = np.zeros(3)
    lib().or_bisph_point(_ptr(a), _ptr(b), s, t, phi, _ptr(o))
    return o


def bisph_coords(fk, fk1, f):
    a = np.ascontiguousarray(fk, dtype=np.float64)
    b = np.ascontiguousarray(fk1, dtype=np.float64)
    c = np.ascontiguousarray(f, dtype=np.float64)
    s, t, p = C.c_double(), C.c_double(), C.c_double()
    lib().or_bisph_coords(_ptr(a), _ptr(b), _ptr(c), C.byref(s), C.byref(t), C.byref(p))
    return s.value, t.value, p.value


def z2(m: Medium, s: Source, d: Sensor, n_v: int = 4000, n_phi: int = 64) -> float:
    return lib().or_z2(C.byref(m), C.byref(s), C.byref(d), n_v, n_phi)


def qref_logdensity(m, s, d, cap, path) -> float:
    f = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 3)
    return lib().or_qref_logdensity(C.byref(m), C.byref(s), C.byref(d), cap, len(f), _ptr(f))


def qref_sample(m, s, d, cap, seed, stream, draw):
    f = np.zeros((cap, 3))
    n = lib().or_qref_sample(C.byref(m), C.byref(s), C.byref(d), cap, seed, stream, draw, _ptr(f))
    return f[:n].copy()


def qref_bridge_sums(m, s, d, cap, seed, stream, n_draws, threads=None):
    out = np.zeros(4)
    lib().or_qref_bridge_sums(C.byref(m), C.byref(s), C.byref(d), cap, seed, stream, n_draws, _ptr(out),
                              threads or os.cpu_count() or 1)
    return out


def trace(m, s, d, seed, n_photons, photon0=0, r_reject=math.inf, max_scatter=1 << 30, threads=None,
          hist=False):
    """Forward tracer (Algorithm 1).  Returns dict with intensity estimate and SE;
    with hist=True also the detected weight per number of scatterings."""
    out = np.zeros(5)
    h = np.zeros(max_scatter + 1) if hist else None
    lib().or_trace_hist(C.byref(m), C.byref(s), C.byref(d), seed, photon0, n_photons, r_reject, max_scatter,
                        _ptr(out), _ptr(h) if hist else None, threads or os.cpu_count() or 1)
    N = out[3]
    mean = out[0] / N
    var = max(out[1] / N - mean * mean, 0.0)
    res = {"I": mean, "se": math.sqrt(var / N), "hits": out[2], "photons": N,
           "mean_L": out[4] / out[0] if out[0] > 0 else float("nan"), "raw": out}
    if hist:
        res["hist"] = h / N
    return res


def trace_lengths(m, s, d, seed, n_photons, l_lo, l_hi, l_bins, photon0=0, r_reject=math.inf,
                  max_scatter=1 << 30, threads=None):
    """Forward tracer with the detected weight binned by path length:
    returns (result dict as trace(), weight per bin / emitted photons)."""
    out = np.zeros(5)
    h = np.zeros(int(l_bins))
    rc = lib().or_trace_lhist(C.byref(m), C.byref(s), C.byref(d), seed, photon0, n_photons, r_reject, max_scatter,
                              float(l_lo), float(l_hi), int(l_bins), _ptr(out), _ptr(h),
                              threads or os.cpu_count() or 1)
    if rc != 0:
        raise ValueError("bad histogram range")
    N = out[3]
    mean = out[0] / N
    var = max(out[1] / N - mean * mean, 0.0)
    return {"I": mean, "se": math.sqrt(var / N), "hits": out[2], "photons": N, "raw": out}, h / N


def ymap(s: Source, d0: Sensor, d1: Sensor) -> YMap:
    """Relative-light-yield map of paths ending on sensor d0 to paths ending on d1."""
    T = YMap()
    if lib().or_ymap_init(C.byref(s), C.byref(d0), C.byref(d1), C.byref(T)) != 0:
        raise ValueError("sensors collinear with the source, or a source inside a sensor")
    return T


def ymap_forward(T: YMap, path):
    x = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 3)
    y = np.zeros_like(x)
    lj = lib().or_ymap_forward(C.byref(T), len(x), _ptr(x), _ptr(y))
    return y, lj


def ymap_inverse(T: YMap, path):
    y = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 3)
    x = np.zeros_like(y)
    lj = lib().or_ymap_inverse(C.byref(T), len(y), _ptr(y), _ptr(x))
    return x, lj


def ymap_logratio(m: Medium, s: Source, d0: Sensor, d1: Sensor, T: YMap, side: int, path) -> float:
    f = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 3)
    return lib().or_ymap_logratio(C.byref(m), C.byref(s), C.byref(d0), C.byref(d1), C.byref(T), int(side), len(f),
                                  _ptr(f))


def tree_node(m: int, n: int):
    """(k, l, parent) of interior vertex m in the tree over an n-vertex path."""
    k, l, p = C.c_int(), C.c_int(), C.c_int()
    lib().or_tree_node(int(m), int(n), C.byref(k), C.byref(l), C.byref(p))
    return k.value, l.value, p.value


def tree_vref(s: Source, d: Sensor):
    v = np.zeros(3)
    lib().or_tree_vref(C.byref(s), C.byref(d), _ptr(v))
    return v


def hmc_leapfrog(m, s, d, path, momenta, eps, steps):
    """(x', p', log p(x')) after `steps` leapfrog steps of size eps."""
    x = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 3).copy()
    p = np.ascontiguousarray(momenta, dtype=np.float64).reshape(-1, 3).copy()
    lp = lib().or_hmc_leapfrog(C.byref(m), C.byref(s), C.byref(d), len(x), _ptr(x), _ptr(p), float(eps), int(steps))
    return x, p, lp


def tree_coords(v_ref, path):
    """Tree coordinates (zeta, t, phi) of the interior vertices, rows 1..n-2 of
    an (n, 3) array (rows 0 and n-1 unused), and the log Jacobian."""
    f = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 3)
    co = np.zeros_like(f)
    vr = np.ascontiguousarray(v_ref, dtype=np.float64)
    lj = lib().or_tree_coords(_ptr(vr), len(f), _ptr(f), _ptr(co))
    return co, lj


def tree_path(v_ref, f0, f_end, coords):
    """Path (n, 3) from its end points and the interior vertices' tree coordinates."""
    co = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 3)
    f = np.zeros_like(co)
    f[0], f[-1] = f0, f_end
    vr = np.ascontiguousarray(v_ref, dtype=np.float64)
    lib().or_tree_path(_ptr(vr), len(f), _ptr(co), _ptr(f))
    return f


def optimal_bridge(logr0, logr1, groups=16, max_iter=200, tol=1e-10):
    """Iterative optimal bridge (Meng & Wong 1996) for r = c1/c0 from draws of
    p0 (log(q1/q0) at each, array rows x n0) and of p1 (log(q0/q1) at each,
    rows x n1), started from the geometric estimate; chains (columns) are
    split into `groups` groups by index mod groups, each iterated on its own,
    and the standard error is their spread / sqrt(groups).  Returns
    (r, se, iterations, geometric estimate)."""
    L0 = np.asarray(logr0, dtype=np.float64)
    L1 = np.asarray(logr1, dtype=np.float64)
    n0, n1 = L0.shape[1], L1.shape[1]
    s0, s1 = n0 / (n0 + n1), n1 / (n0 + n1)
    l0 = np.exp(L0)          # q1/q0 at p0 draws
    l1 = np.exp(-L1)         # q1/q0 at p1 draws
    cols = [(np.arange(n0) % groups == g, np.arange(n1) % groups == g) for g in range(groups)]
    cols.append((np.ones(n0, bool), np.ones(n1, bool)))

    def geo(c0, c1):
        a = np.where(np.isfinite(L0[:, c0]), np.exp(0.5 * L0[:, c0]), 0.0).mean()
        b = np.where(np.isfinite(L1[:, c1]), np.exp(0.5 * L1[:, c1]), 0.0).mean()
        return a / b

    r = np.array([geo(c0, c1) for c0, c1 in cols])
    r_geo = r[-1]
    it = 0
    for it in range(1, max_iter + 1):
        rn = np.empty_like(r)
        for g, (c0, c1) in enumerate(cols):
            with np.errstate(divide="ignore"):
                a = (1.0 / (s1 + s0 * r[g] / l0[:, c0])).mean()
            b = (1.0 / (s1 * l1[:, c1] + s0 * r[g])).mean()
            rn[g] = a / b
        change = np.max(np.abs(rn / r - 1.0))
        r = rn
        if change < tol:
            break
    se = r[:groups].std(ddof=1) / math.sqrt(groups) if groups > 1 else float("nan")
    return r[-1], se, it, r_geo


def yield_ratio_estimate(sums0, sums1):
    """Geometric estimator B = E_0[sqrt(p_1/p_0)] / E_1[sqrt(p_0/p_1)] from
    per-chain sums of sqrt-ratios (each array: one entry per chain, equal
    observation counts); standard error by the delta method over the
    across-chain variances of the per-chain means."""
    a, b = np.asarray(sums0, float), np.asarray(sums1, float)
    m0, m1 = a.mean(), b.mean()
    v0 = a.var(ddof=1) / len(a)
    v1 = b.var(ddof=1) / len(b)
    B = m0 / m1
    return B, B * math.sqrt(v0 / m0 ** 2 + v1 / m1 ** 2)


class Chains:
    """A set of oracle chains for one source-sensor pair (state in FP64)."""

    def __init__(self, scene_medium, scene_source, scene_sensor, scene_run, n_chains, cap,
                 chain_offset=0, init=None, init_k=None, jitter=None, user_xyz=None, user_n=None):
        self.m = medium(scene_medium)
        self.s = source(scene_source)
        self.d = sensor(scene_sensor)
        self.r = run(scene_run, float(scene_sensor.radius))
        self.n_chains = int(n_chains)
        self.cap = int(cap)
        self.chain_offset = int(chain_offset)
        self.xyz = np.zeros((self.n_chains, self.cap, 3))
        self.n = np.zeros(self.n_chains, dtype=np.int32)
        self.acc = (Acc * self.n_chains)()
        self.step = 0
        # the chains' wavelengths when the run samples them (section "Discussion")
        self.lam = None
        if self.r.n_lambda >= 2:
            self.lam = np.zeros(self.n_chains)
            lib().or_init_lambda(C.byref(self.r), self.n_chains, self.chain_offset, _ptr(self.lam))
        init = scene_run.init if init is None else init
        if user_xyz is not None:
            for c in range(self.n_chains):
                k = int(user_n[c])
                self.xyz[c, :k] = user_xyz[c, :k]
                self.n[c] = k
        else:
            rc = lib().or_init_chains(C.byref(self.m), C.byref(self.s), C.byref(self.d), C.byref(self.r),
                                      int(init), int(scene_run.init_k if init_k is None else init_k),
                                      float(scene_run.init_jitter if jitter is None else jitter),
                                      self.n_chains, self.cap, self.chain_offset,
                                      _ptr(self.xyz), self.n.ctypes.data_as(_ip))
            if rc != 0:
                raise ValueError("oracle init failed")

    def run(self, n_steps, threads=None, margins=False, n_hist=None, hmc_seg=False):
        """Advance every chain; n_hist (n_chains x (cap+1) float64) collects recorded dwell per n.
        margins=True returns each chain's smallest |log A - log u|; hmc_seg=True also
        the shortest segment met at any leapfrog position of its HMC moves
        (then the return value is the pair (margins, shortest segments))."""
        mm = np.full(self.n_chains, np.inf) if (margins or hmc_seg) else None
        hs = np.full(self.n_chains, np.inf) if hmc_seg else None
        rc = lib().or_run_chains_lam(C.byref(self.m), C.byref(self.s), C.byref(self.d), C.byref(self.r),
                                     self.n_chains, self.cap, self.chain_offset, self.step, int(n_steps),
                                     _ptr(self.xyz), self.n.ctypes.data_as(_ip),
                                     _ptr(self.lam) if self.lam is not None else None, self.acc,
                                     _ptr(mm) if mm is not None else None,
                                     _ptr(n_hist) if n_hist is not None else None,
                                     _ptr(hs) if hs is not None else None, threads or os.cpu_count() or 1)
        if rc != 0:
            raise ValueError("oracle chains: wavelength sampling needs a homogeneous medium and Gaussian moves")
        self.step += int(n_steps)
        return (mm, hs) if hmc_seg else mm

    def logp(self, c):
        return logp(self.m, self.s, self.d, self.xyz[c, : self.n[c]])

    def accumulators(self):
        """Per-chain accumulators as a dict of numpy arrays."""
        out = {k: np.array([getattr(a, k) for a in self.acc]) for k in ACC_FIELDS}
        out["sum_score"] = np.array([list(a.sum_score) for a in self.acc])
        out["prop"] = np.array([list(a.prop) for a in self.acc])
        out["acc"] = np.array([list(a.acc) for a in self.acc])
        return out


def medium_at(m: Medium, lam: float) -> Medium:
    """The homogeneous medium at wavelength lam (section "Discussion")."""
    out = Medium()
    lib().or_medium_at(C.byref(m), float(lam), C.byref(out))
    return out


def log_spectrum(r: Run, lam: float) -> float:
    return lib().or_log_spectrum(C.byref(r), float(lam))


def spectrum_quantile(r: Run, u: float) -> float:
    return lib().or_spectrum_quantile(C.byref(r), float(u))


def z2_spectrum(m: Medium, s: Source, d: Sensor, r: Run, nodes: int = 8) -> float:
    """Direct-sector integral of the joint density S(l) p_l: the integral over
    the spectrum's range of S(l) Z2(medium at l), Gauss-Legendre with `nodes`
    points on every interval of the spectrum table (S is linear there)."""
    x, w = np.polynomial.legendre.leggauss(nodes)
    nm = [r.lambda_nm[i] for i in range(r.n_lambda)]
    tot = 0.0
    for i in range(r.n_lambda - 1):
        a, b = nm[i], nm[i + 1]
        for xi, wi in zip(x, w):
            lam = 0.5 * (a + b) + 0.5 * (b - a) * xi
            tot += 0.5 * (b - a) * wi * math.exp(log_spectrum(r, lam)) * z2(medium_at(m, lam), s, d)
    return tot


def direct_estimate(acc: dict, z2_value: float):
    """Intensity from the direct-sector anchor: I = Z2 / pi(n=2).

    The standard error is propagated from the across-chain variance of the
    per-chain n=2 fractions (chains are independent).
    """
    N = acc["n_rec"]
    n2 = acc["n_direct"]
    pi_hat = n2.sum() / N.sum()
    frac = n2 / np.maximum(N, 1)
    C_ = len(N)
    w = N / N.sum()
    var_pi = (w * w * (frac - pi_hat) ** 2).sum() * C_ / max(C_ - 1, 1)
    I = z2_value / pi_hat
    se = I * math.sqrt(var_pi) / pi_hat
    return I, se, pi_hat
