"""Write stored expected values for the GPU tests by running the FP64 oracle.

Calls only oracle/ (and the seeded scene definitions).  Run from the repo
root:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1811_04156_gb300 import scenes as S  # noqa: E402


def plain_intensity(n_chains=4096, n_steps=10_000, burn_in=1_000):
    sc = S.plain(n_chains=n_chains, n_steps=n_steps)
    sc.run.burn_in = burn_in
    t = time.time()
    ch = O.Chains(sc.medium, sc.sources[0], sc.sensors[0], sc.run, n_chains, sc.pairs[0].cap)
    ch.run(n_steps)
    m, s, d = O.medium(sc.medium), O.source(sc.sources[0]), O.sensor(sc.sensors[0])
    acc = ch.accumulators()
    I, se, pi = O.direct_estimate(acc, O.z2(m, s, d))
    return {"scene": "plain", "n_chains": n_chains, "n_steps": n_steps, "burn_in": burn_in,
            "seed": sc.run.seed, "cap": sc.pairs[0].cap, "intensity": I, "std_err": se, "pi_direct": pi,
            "mean_n": float(acc["sum_n"].sum() / acc["n_rec"].sum()),
            "accept": (acc["acc"].sum(0) / acc["prop"].sum(0)).tolist(),
            "oracle_seconds": time.time() - t}


def batched_small_long_pairs():
    """Oracle intensities of the two long-cap pairs of the small uneven batch,
    with the batch's global chain numbering (same random streams)."""
    sc = S.batched_small()
    out = {"scene": "batched_small", "n_steps": sc.run.n_steps, "burn_in": sc.run.burn_in, "pairs": {}}
    chain0 = 0
    for i, p in enumerate(sc.pairs):
        if p.cap > 3:
            t = time.time()
            ch = O.Chains(sc.medium, sc.sources[0], sc.sensors[p.sensor], sc.run, p.n_chains, p.cap,
                          chain_offset=chain0)
            ch.run(sc.run.n_steps)
            m, s, d = O.medium(sc.medium), O.source(sc.sources[0]), O.sensor(sc.sensors[p.sensor])
            acc = ch.accumulators()
            I, se, pi = O.direct_estimate(acc, O.z2(m, s, d))
            out["pairs"][str(i)] = {"cap": p.cap, "intensity": I, "std_err": se, "pi_direct": pi,
                                    "mean_n": float(acc["sum_n"].sum() / acc["n_rec"].sum()),
                                    "oracle_seconds": time.time() - t}
        chain0 += p.n_chains
    return out


def _write(name, out):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    which = sys.argv[1:] or ["plain", "batched"]
    if "plain" in which:
        _write("plain_intensity.json", plain_intensity())
    if "batched" in which:
        _write("batched_small_intensity.json", batched_small_long_pairs())
