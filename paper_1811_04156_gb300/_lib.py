"""ctypes binding of libpathmc (include/pathmc.h): structs and prototypes.

Argument marshalling only: every computation happens in the CUDA library.
There is no CPU fallback; loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpathmc.so")

PMC_OK = 0
ERRORS = {1: "PMC_ERR_INVALID", 2: "PMC_ERR_OOM", 3: "PMC_ERR_CUDA", 4: "PMC_ERR_DEVICE_STATUS",
          5: "PMC_ERR_ABORTED", 6: "PMC_ERR_NO_DEVICE"}
PMC_FLAG_GRADIENTS = 1
PMC_FLAG_NO_GRAPH = 2
PMC_FLAG_ONE_LAUNCH = 4
PMC_LAYOUT_AUTO, PMC_LAYOUT_WARP, PMC_LAYOUT_LANE = 0, 1, 2
PMC_ACC_WORDS = 16
PMC_MOMENT_WORDS = 40
PMC_NOALLOC_MAX_PAIRS = 128


class PathmcError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


class MediumDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("lambda_s", C.c_double), ("lambda_a", C.c_double),
                ("g", C.c_double), ("f_sl", C.c_double), ("z0", C.c_double), ("dz", C.c_double),
                ("n_layers", C.c_int), ("lambda_s_layers", C.POINTER(C.c_double)),
                ("lambda_a_layers", C.POINTER(C.c_double)), ("lambda0", C.c_double), ("k_s", C.c_double),
                ("k_a", C.c_double)]


class SourceDesc(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("emission", C.c_int), ("kappa", C.c_double),
                ("dir", C.c_double * 3)]


class SensorDesc(C.Structure):
    _fields_ = [("centre", C.c_double * 3), ("radius", C.c_double), ("rho", C.c_int),
                ("rho_hat", C.c_double * 3)]


class PairDesc(C.Structure):
    _fields_ = [("source", C.c_int), ("sensor", C.c_int), ("n_chains", C.c_int), ("cap", C.c_int)]


class GeometryDesc(C.Structure):
    _fields_ = [("n_sources", C.c_int), ("sources", C.POINTER(SourceDesc)),
                ("n_sensors", C.c_int), ("sensors", C.POINTER(SensorDesc)),
                ("n_pairs", C.c_int), ("pairs", C.POINTER(PairDesc))]


class RunDesc(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("p_within", C.c_double), ("p_birth", C.c_double),
                ("p_death", C.c_double), ("within", C.c_int), ("sigma", C.c_double),
                ("mala_step", C.c_double), ("kappa_end", C.c_double), ("burn_in", C.c_uint64),
                ("thin_bridge", C.c_uint32), ("init", C.c_int), ("init_k", C.c_int),
                ("init_jitter", C.c_double), ("init_xyz", C.POINTER(C.c_float)),
                ("init_n", C.POINTER(C.c_int)), ("init_stride", C.c_int), ("flags", C.c_int),
                ("warps_per_block", C.c_int), ("smem_window", C.c_int), ("hmc_steps", C.c_int),
                ("layout", C.c_int), ("n_lambda", C.c_int), ("lambda_nm", C.POINTER(C.c_double)),
                ("spectrum", C.POINTER(C.c_double)), ("sigma_lambda", C.c_double), ("chain_lo", C.c_int64),
                ("chain_hi", C.c_int64)]


class Estimate(C.Structure):
    _fields_ = [("intensity", C.c_double), ("std_err", C.c_double), ("rel_err", C.c_double),
                ("pi_direct", C.c_double), ("z2", C.c_double), ("rhat", C.c_double),
                ("accept", C.c_double * 4), ("proposals", C.c_double * 4), ("mean_n", C.c_double),
                ("mean_length", C.c_double), ("n_samples", C.c_double), ("ess", C.c_double),
                ("bridge_intensity", C.c_double), ("bridge_std_err", C.c_double)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if not isinstance(v, (int, float)) else v
        return out


class TraceResult(C.Structure):
    _fields_ = [("intensity", C.c_double), ("std_err", C.c_double), ("mean_length", C.c_double),
                ("detected", C.c_double), ("emitted", C.c_double), ("sum_w", C.c_double), ("sum_w2", C.c_double),
                ("sum_wl", C.c_double)]

    def as_dict(self):
        return {name: float(getattr(self, name)) for name, _ in self._fields_}


# Every symbol declared in include/pathmc.h, with its ctypes prototype.
_vp = C.c_void_p
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)
_dp = C.POINTER(C.c_double)
PROTOTYPES = {
    "pmc_create_context": ([C.c_int, C.POINTER(_vp)], C.c_int),
    "pmc_destroy_context": ([_vp], C.c_int),
    "pmc_create_medium": ([_vp, C.POINTER(MediumDesc), C.POINTER(_vp)], C.c_int),
    "pmc_destroy_medium": ([_vp], C.c_int),
    "pmc_create_geometry": ([_vp, C.POINTER(GeometryDesc), C.POINTER(_vp)], C.c_int),
    "pmc_destroy_geometry": ([_vp], C.c_int),
    "pmc_init_chains": ([_vp, _vp, _vp, C.POINTER(RunDesc), _vp, C.POINTER(_vp)], C.c_int),
    "pmc_destroy_chains": ([_vp], C.c_int),
    "pmc_reset_chains": ([_vp, _vp], C.c_int),
    "pmc_set_states": ([_vp, _fp, _ip, C.c_int, _vp], C.c_int),
    "pmc_run_steps": ([_vp, C.c_uint64, _vp], C.c_int),
    "pmc_read_estimator": ([_vp, C.POINTER(Estimate), C.c_size_t, _vp], C.c_int),
    "pmc_grad_estimator": ([_vp, _dp, _dp, C.c_size_t, _vp], C.c_int),
    "pmc_shard_range": ([C.POINTER(PairDesc), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int64),
                         C.POINTER(C.c_int64)], C.c_int),
    "pmc_read_moments": ([_vp, _dp, C.c_size_t, _vp], C.c_int),
    "pmc_pair_z2": ([_vp, _dp, C.c_size_t, _vp], C.c_int),
    "pmc_estimate_from_moments": ([_dp, C.c_size_t, _dp, C.POINTER(Estimate), _dp, _dp], C.c_int),
    "pmc_moments_from_accumulators": ([_dp, C.c_size_t, _ip, C.c_size_t, C.c_double, C.c_double, _dp], C.c_int),
    "pmc_n_theta": ([_vp], C.c_int),
    "pmc_read_states": ([_vp, _fp, _ip, C.POINTER(C.c_uint64), C.c_int, _vp], C.c_int),
    "pmc_read_accumulators": ([_vp, _dp, C.c_size_t, _vp], C.c_int),
    "pmc_total_chains": ([_vp], C.c_int),
    "pmc_chains_launch_info": ([_vp, _ip, C.c_int, _ip], C.c_int),
    "pmc_save_state": ([_vp, _vp, C.POINTER(C.c_size_t), _vp], C.c_int),
    "pmc_load_state": ([_vp, _vp, C.c_size_t, _vp], C.c_int),
    "pmc_read_lambda": ([_vp, _fp, C.c_size_t, _vp], C.c_int),
    "pmc_request_abort": ([_vp, C.c_int], C.c_int),
    "pmc_chain_status": ([_vp, _ip, _vp], C.c_int),
    "pmc_logp": ([_vp, _vp, _vp, C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp], C.c_int),
    "pmc_logp_grad": ([_vp, _vp, _vp, C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp, _vp], C.c_int),
    "pmc_score": ([_vp, _vp, _vp, C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp], C.c_int),
    "pmc_trace": ([_vp, _vp, _vp, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double, C.c_int,
                   C.POINTER(TraceResult), _vp], C.c_int),
    "pmc_trace_noalloc": ([_vp, _vp, _vp, _ip, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double, C.c_int,
                           C.POINTER(TraceResult), _vp], C.c_int),
    "pmc_qref_logdensity": ([_vp, _vp, _vp, C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp], C.c_int),
    "pmc_qref_sample": ([_vp, _vp, _vp, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, _vp, _vp, C.c_int, _vp],
                        C.c_int),
    "pmc_bridge": ([_vp, C.c_uint64, C.c_uint64, _dp, _vp], C.c_int),
    "pmc_bridge_observe_log": ([_vp, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, _vp, _vp], C.c_int),
    "pmc_trace_paths": ([_vp, _vp, _vp, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double, C.c_int, C.c_int,
                         _vp, _vp, C.c_int, C.POINTER(C.c_uint64), _vp], C.c_int),
    "pmc_yield_logratio": ([_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp, _vp],
                           C.c_int),
    "pmc_yield_observe": ([_vp, C.c_int, C.c_int, _vp, _vp], C.c_int),
    "pmc_yield_estimate": ([_vp, C.c_int, C.c_int, _vp, C.c_uint64, _dp, _vp], C.c_int),
    "pmc_yield_observe_log": ([_vp, C.c_int, C.c_int, _vp, _vp], C.c_int),
    "pmc_bridge_ratio": ([_vp, _vp, C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, _dp, _vp], C.c_int),
    "pmc_length_hist": ([_vp, C.c_double, C.c_double, C.c_int, _vp, _vp], C.c_int),
    "pmc_score_observe": ([_vp, _vp, _vp], C.c_int),
    "pmc_trace_lengths": ([_vp, _vp, _vp, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double, C.c_int,
                           C.c_double, C.c_double, C.c_int, C.POINTER(TraceResult), _dp, _vp], C.c_int),
    "pmc_seed_from_tracer": ([_vp, C.c_uint64, C.c_uint64, C.c_int, C.c_double, C.POINTER(C.c_uint64), _vp],
                             C.c_int),
    "pmc_seed_select": ([C.POINTER(C.c_uint64), C.c_size_t, C.c_size_t, C.POINTER(C.c_uint64)], C.c_int),
    "pmc_last_error": ([], C.c_char_p),
    "pmc_version": ([], C.c_char_p),
}

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libpathmc.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libpathmc is not built ({path}); run paper_1811_04156_gb300/build.py")
            L = C.CDLL(path)
            for name, (args, res) in PROTOTYPES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def check(rc: int, where: str) -> None:
    if rc != PMC_OK:
        msg = load().pmc_last_error().decode(errors="replace")
        raise PathmcError(rc, where, msg)
