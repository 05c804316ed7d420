"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function include/pathmc.h declares, and reports the absence of
a device instead of falling back to the CPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pathmc.h")).read()
    return sorted(set(re.findall(r"^PMC_API\s+[\w\s\*]+?\b(pmc_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pmc_create_context", "pmc_create_medium", "pmc_create_geometry", "pmc_init_chains",
                     "pmc_run_steps", "pmc_read_estimator", "pmc_grad_estimator", "pmc_logp", "pmc_logp_grad",
                     "pmc_save_state", "pmc_load_state", "pmc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(pathmc_lib):
    for name in declared_symbols():
        assert hasattr(pathmc_lib, name), name
    from paper_1811_04156_gb300 import _lib
    assert set(declared_symbols()) == set(_lib.PROTOTYPES)


def test_no_device_is_an_error_not_a_fallback(pathmc_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = pathmc_lib.pmc_create_context(0, C.byref(h))
    assert rc == 6  # PMC_ERR_NO_DEVICE
    assert b"no CUDA device" in pathmc_lib.pmc_last_error()


def test_null_arguments_are_rejected(pathmc_lib):
    assert pathmc_lib.pmc_create_context(0, None) == 1
    assert pathmc_lib.pmc_run_steps(None, 10, None) == 1
    assert pathmc_lib.pmc_destroy_chains(None) == 0
