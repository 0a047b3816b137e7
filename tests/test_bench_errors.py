"""bench.py's error_vs_oracle (host arithmetic, no GPU): a Jacobian that holds
the oracle's stored samples has zero error; a perturbation planted in one
sampled column is found in that column with its relative size, and r and f
errors are relative norms."""
import importlib.util
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_errors_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(ROOT, "tests", "golden", "full_n2048_samples.json")) as fh:
        return json.load(fh)


def outputs_from_samples(g):
    N, n = g["N"], g["n"]
    rows = np.asarray(g["rows"])
    r = np.zeros(N)
    r[rows] = g["r"]
    J = np.zeros((n + 1, N))
    for k, v in g["columns"].items():
        J[0 if k == "T" else int(k), rows] = v["values"]
    return r, J, float(g["f"])


def test_samples_themselves_have_no_error(bench, golden):
    r, J, f = outputs_from_samples(golden)
    e = bench.error_vs_oracle(bench.W.LARGE, r, J, f)
    assert e["f_rel"] == 0.0 and e["r_rel"] == 0.0 and e["J_max_col_rel"] == 0.0
    assert e["columns_compared"] == len(golden["columns"]) and e["rows_compared"] == len(golden["rows"])


def test_planted_column_error_is_found(bench, golden):
    r, J, f = outputs_from_samples(golden)
    k = sorted(golden["columns"], key=lambda s: -golden["columns"][s]["norm"])[0]   # a column well above the floor
    col = 0 if k == "T" else int(k)
    rows = np.asarray(golden["rows"])
    ref = np.asarray(golden["columns"][k]["values"])
    J[col, rows] += 1e-9 * np.linalg.norm(ref) / np.sqrt(len(rows))    # relative 1e-9 of the column
    r[rows[0]] += 1e-12 * np.linalg.norm(golden["r"])
    e = bench.error_vs_oracle(bench.W.LARGE, r, J, f * (1 + 1e-13))
    assert e["J_worst_col"] == k
    assert abs(e["J_max_col_rel"] - 1e-9) < 1e-12
    assert abs(e["r_rel"] - 1e-12) < 1e-15
    assert abs(e["f_rel"] - 1e-13) < 1e-15
    sp = golden.get("spread")
    if sp:
        assert abs(e["J_max_ratio_to_oracle_ulp_spread"] - 1e-9 / sp["columns"][k]) < 1e-6 * (1e-9 / sp["columns"][k])


def test_other_workloads_have_no_samples(bench):
    N = bench.W.SMALL.N if hasattr(bench.W, "SMALL") else 64
    assert bench.error_vs_oracle(bench.W.SEGMENTED, np.zeros(N), np.zeros((2, N)), 1.0) is None
