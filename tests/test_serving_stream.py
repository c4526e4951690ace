"""The seeded request stream of the serving workload (the mixed-case stream):
its parameters stay within the stated distribution, both geometries occur,
the same seed gives the same stream, and the arrivals are a Poisson process
of the requested rate."""
import math

import numpy as np

from paper_2412_06546_gb300 import serving

CONFIG = dict(c_lo=1000, c_hi=40000, n_lo=16, n_hi=64, kn_lo=1e-3, kn_hi=10.0)


def test_config_stream_within_its_distribution():
    s = serving.request_stream(16, **CONFIG)
    req = [c["request"] for c in s]
    assert {r["geometry"] for r in req} == {"cavity", "cylinder"}
    for r, c in zip(req, s):
        N = math.isqrt(r["nv"])
        assert N * N == r["nv"] and 16 <= N <= 64
        assert 1e-3 <= r["Kn"] <= 10.0 and 0.1 <= r["Mach"] <= 6.0
        assert r["cells"] == len(c["mesh"]["cell_vol"])
        # a cavity is the nearest square n x n; a cylinder mesh is within 15 % of its draw
        assert 0.85 * 1000 <= r["cells"] <= 1.15 * 40000
        assert len(c["vgrid"]["w"]) == r["nv"]


def test_stream_is_seeded():
    a = [c["request"] for c in serving.request_stream(6, seed=9, **CONFIG)]
    b = [c["request"] for c in serving.request_stream(6, seed=9, **CONFIG)]
    c = [c["request"] for c in serving.request_stream(6, seed=10, **CONFIG)]
    assert a == b and a != c


def test_poisson_arrivals():
    t = serving.poisson_arrivals(4000, rate=2.5, seed=3)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 0.4) < 0.03            # mean gap 1 / rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.08   # exponential: unit coefficient of variation
