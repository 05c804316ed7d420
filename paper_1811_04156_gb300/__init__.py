"""GB300-native path-integral RJMCMC light transport (arXiv:1811.04156).

``scenes`` (seeded synthetic inputs) imports only numpy.  The CUDA binding
(``api``: Context, Medium, Geometry, Chains, logp, logp_grad, score, trace,
LogP, PathSampler) is imported on first use, and fails loudly when the
compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import importlib

__all__ = ["scenes", "api", "build"]

_API_NAMES = {"Context", "Medium", "Geometry", "Chains", "PathSampler", "LogP", "create_context",
              "create_medium", "create_geometry", "init_chains", "run_steps", "read_estimator",
              "grad_estimator", "logp", "logp_grad", "score", "trace"}


def __getattr__(name):
    if name in ("scenes", "api", "build", "_lib"):
        return importlib.import_module(f"{__name__}.{name}")
    if name in _API_NAMES:
        return getattr(importlib.import_module(f"{__name__}.api"), name)
    raise AttributeError(name)
