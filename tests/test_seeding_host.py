"""Host logic of the tracer seeding (pmc_seed_select in the C library; no
GPU): the seeds are the accepted photons with the smallest indices, i.e. the
first accepted draws of a sequential tracer, whatever order the GPU found
them in, reused cyclically when a pair has more chains than accepted paths.

The GPU finds accepted photons in the order their threads finish, and short
paths finish first: taking the first-found ones would favour few-scattering
paths.  The stand-in order below is exactly that biased order."""
import numpy as np
import pytest

from paper_1811_04156_gb300 import build


@pytest.fixture(scope="module")
def api():
    build.build()
    from paper_1811_04156_gb300 import api as A
    return A


def _finish_order(photons, scatterings):
    """Accepted photon indices in the order a GPU would report them: fewest
    scatterings (shortest tracing) first."""
    return photons[np.argsort(scatterings, kind="stable")]


def test_seeds_are_the_first_accepted_photons(api):
    rng = np.random.default_rng(4)
    accepted = np.sort(rng.choice(10_000_000, size=5000, replace=False)).astype(np.uint64)
    scat = rng.poisson(6.0, size=accepted.size)
    found = _finish_order(accepted, scat)
    need = 1200
    sel = api.seed_select(found, need)
    assert np.array_equal(sel, accepted[:need])
    # the first-found paths would have been the short ones; the selection is not
    first_found = scat[np.argsort(scat, kind="stable")][:need]
    chosen = scat[:need]
    assert first_found.mean() < 4.0 < chosen.mean()


def test_few_accepted_photons_are_reused_cyclically(api):
    accepted = np.array([90, 7, 55, 3], dtype=np.uint64)
    sel = api.seed_select(accepted, 10)
    assert sel.tolist() == [3, 7, 55, 90, 3, 7, 55, 90, 3, 7]


def test_selection_errors(api):
    from paper_1811_04156_gb300._lib import PathmcError
    with pytest.raises(PathmcError):
        api.seed_select(np.zeros(0, dtype=np.uint64), 3)
    assert api.seed_select(np.zeros(0, dtype=np.uint64), 0).size == 0
