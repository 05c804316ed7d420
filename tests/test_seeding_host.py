"""Host logic of the tracer seeding (api.seed_from_tracer), with a stand-in
for the GPU tracer: the seeds must be an unbiased subset of every accepted
path of the traced photon range.

The GPU buffer of pmc_trace_paths keeps the paths whose photons finish first
when a launch finds more than it holds; seeding therefore re-traces an
overflowing round with half the photons (the same photon indices), keeps every
path of each round that fits, and gives the chains a seeded random subset.
The stand-in detects photon q when q % 7 == 0 and, on overflow, keeps the
longest paths first (a deliberately biased buffer)."""
import types

import numpy as np
import pytest
import torch

from paper_1811_04156_gb300 import api


def _detected(q):
    return q % 7 == 0


def _fake_trace_paths(calls):
    def trace_paths(ctx, medium, geom, pair, seed, n_photons, max_paths, photon0=0, stride=None, r_reject=None,
                    **kw):
        qs = [q for q in range(photon0, photon0 + n_photons) if _detected(q)]
        calls.append((pair, photon0, n_photons, len(qs), max_paths))
        # biased buffer: longest paths first, truncated at max_paths
        qs_kept = sorted(qs, key=lambda q: -(q % 5))[:max_paths]
        xyz = torch.zeros((3, len(qs_kept), stride), dtype=torch.float32)
        n = torch.zeros(len(qs_kept), dtype=torch.int32)
        for i, q in enumerate(qs_kept):
            xyz[0, i, 0] = float(q)           # the photon index, read back by the test
            n[i] = 2 + q % 5
        return xyz, n, len(qs)
    return trace_paths


class _FakeChains:
    def __init__(self, n_chains, stride=8):
        pair = types.SimpleNamespace(n_chains=n_chains)
        self.geom = types.SimpleNamespace(pairs=[pair], max_cap=stride)
        self.total = n_chains
        self.ctx = self.medium = None
        self.states = None

    def set_states(self, xyz, n):
        self.states = (np.array(xyz), np.array(n))


@pytest.fixture
def fake(monkeypatch):
    calls = []
    monkeypatch.setattr(api, "trace_paths", _fake_trace_paths(calls))
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: types.SimpleNamespace(synchronize=lambda: None))
    return calls


def test_overflowing_rounds_are_retraced_with_fewer_photons(fake):
    ch = _FakeChains(50)
    used = api.seed_from_tracer(ch, seed=3, photons_per_round=1024)
    kept = [c for c in fake if c[3] <= c[4]]
    # every kept round fits the buffer, and the kept rounds tile [0, photons traced)
    start = 0
    for _, photon0, n_photons, found, cap in kept:
        assert photon0 == start and found <= cap
        start += n_photons
    assert start == used[0]
    # an overflowing round is retried from the same first photon with half the photons
    for a, b in zip(fake, fake[1:]):
        if a[3] > a[4]:
            assert b[1] == a[1] and b[2] == a[2] // 2


def test_seeds_are_a_random_subset_of_every_accepted_path(fake):
    n_chains = 50
    ch = _FakeChains(n_chains)
    used = api.seed_from_tracer(ch, seed=3, photons_per_round=1024)
    xyz, n = ch.states
    q = xyz[:, 0, 0].astype(int)
    every = [p for p in range(used[0]) if _detected(p)]
    assert len(every) >= n_chains
    assert len(set(q)) == n_chains and set(q) <= set(every)
    assert np.array_equal(n, 2 + q % 5)
    # the biased buffer would have kept only the longest paths; the subset does not favour them
    short = np.mean(q % 5 <= 1)
    assert 0.15 < short < 0.65, short
    # the subset is seeded: the same seed gives the same seeds
    ch2 = _FakeChains(n_chains)
    api.seed_from_tracer(ch2, seed=3, photons_per_round=1024)
    assert np.array_equal(ch2.states[0], xyz)


def test_few_detections_are_reused_cyclically(fake):
    ch = _FakeChains(40)
    used = api.seed_from_tracer(ch, seed=1, photons_per_round=21, max_rounds=2)
    xyz, _ = ch.states
    q = xyz[:, 0, 0].astype(int)
    every = [p for p in range(used[0]) if _detected(p)]
    assert len(every) < 40
    assert set(q) == set(every)
    assert np.array_equal(q[: len(every)], q[len(every): 2 * len(every)])
