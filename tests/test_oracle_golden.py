"""Values the paper prints (App. A), stored as text fixtures under tests/golden/."""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_kv(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = float(v)
    return out


def test_model_parameters_are_the_papers():
    g = read_kv("raghu2_app_a.txt")
    for k in ("t1", "t2", "t3", "t4", "mu"):
        assert oracle.RAGHU2[k] == g[k]


def test_printed_filling():
    g = read_kv("raghu2_app_a.txt")
    m = oracle.make_model(mu=g["mu"])
    N = 512
    E = oracle.band_grid(m, N)
    n = 2.0 * np.count_nonzero(E < g["mu"]) / N**2
    assert abs(n - g["electrons_per_site"]) < 0.005
