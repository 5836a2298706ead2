"""The stored oracle entries the benchmark checks its GPU results against: regenerated for
the 2^20-sample block and compared, and the a = 0, m = 0 entry equals the mean power."""
import json
import os

import numpy as np

import oracle
from synth import workloads

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bench_entries.json")


def test_stored_block_entries_reproduce():
    g = json.load(open(GOLD))["cfg2"]
    w = workloads.config2()
    assert g["T"] == w["x"].size
    f = np.array(g["form"])
    R, neff = oracle.entries(w["x"], 255, f + 1, w["alphas"][g["alpha_index"]], w["lags"][g["lag_index"]])
    ref = np.array(g["re"]) + 1j * np.array(g["im"])
    assert neff == g["n_eff"]
    assert np.max(np.abs(R - ref)) / g["r00"] < 1e-9


def test_mean_power_entries():
    for key, g in json.load(open(GOLD)).items():
        j = [i for i, (f, a, m) in enumerate(zip(g["form"], g["alpha_index"], g["lag_index"]))
             if f == 0 and m == 0 and a == {"cfg1": 512, "cfg2": 2048}[key]]
        assert j and abs(g["re"][j[0]] - g["r00"]) < 1e-12 * g["r00"] and g["im"][j[0]] == 0.0
