"""Writes bench_entries.json: FP64 oracle values of sampled estimator entries for the two
full-size workloads the benchmark checks its GPU results against (the stream of 2^26 GMSK
samples with lags 0..127 and 1024 cycle frequencies, and the 2^20-sample block with lags
0..255 and 4096 cycle frequencies), with R^0(0) for the error normalisation.  It calls
only the seeded generators and the oracle.

    python tests/golden/make_bench_entries.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth import workloads  # noqa: E402


def pick(nalpha, nlag, nent, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, nent), rng.integers(0, nalpha, nent), rng.integers(0, nlag, nent)


def record(w, nent, seed, strong):
    """`nent` random entries plus the `strong` ones (form, alpha index, lag index)."""
    x, lags, alphas = w["x"], w["lags"], w["alphas"]
    M = int(np.max(lags))
    f, ia, im = pick(len(alphas), len(lags), nent, seed)
    f, ia, im = (np.concatenate([[s[j] for s in strong], v]) for j, v in enumerate((f, ia, im)))
    R, neff = oracle.entries(x, M, f + 1, alphas[ia], lags[im])
    return {"name": w["name"], "T": int(x.size), "n_eff": neff, "r00": oracle.r00(x, M),
            "form": f.tolist(), "alpha_index": ia.tolist(), "lag_index": im.tolist(),
            "re": R.real.tolist(), "im": R.imag.tolist()}


def main():
    oracle.build()
    # strong entries: the mean power (a = 0, m = 0) and the nearest grid point to the GMSK
    # conjugate line 2 f0 + 1/(2 sps) (Sec. 3), lag 0
    c2 = workloads.config2()
    k2 = int(round(((2 * c2["f0"] + 0.125 + 0.5) % 1.0) * 4096)) % 4096
    out = {"cfg1": record(workloads.config1(), 8, 3, [(0, 512, 0), (1, 678, 0)]),
           "cfg2": record(c2, 6, 5, [(0, 2048, 0), (1, k2, 0)])}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "bench_entries.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
