"""Seeded request streams for the serving loop (the mixed-case workload).

Each request is a 2D cavity or cylinder case with a seeded size, velocity grid,
Knudsen and Mach number, in the spirit of the mixed serving stream: geometry
50/50, cells uniform in [c_lo, c_hi], an N x N velocity grid with N uniform in
[n_lo, n_hi] spanning +-max(4, 1.5 (|U_inf| + 4)), Kn log-uniform in
[kn_lo, kn_hi], Mach uniform in [ma_lo, ma_hi].  Arrivals are Poisson.
"""
from __future__ import annotations

import math

import numpy as np

from . import cases


def request_stream(n, seed=4, c_lo=1000, c_hi=4000, n_lo=16, n_hi=32, kn_lo=1e-3, kn_hi=10.0,
                   ma_lo=0.1, ma_hi=6.0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        geom = "cavity" if rng.uniform() < 0.5 else "cylinder"
        C = int(rng.integers(c_lo, c_hi + 1))
        N = int(rng.integers(n_lo, n_hi + 1))
        Kn = float(math.exp(rng.uniform(math.log(kn_lo), math.log(kn_hi))))
        Ma = float(rng.uniform(ma_lo, ma_hi))
        U = cases.freestream_speed(Ma)
        vmax = max(4.0, 1.5 * (U + 4.0)) if geom == "cylinder" else max(4.0, 1.5 * (U + 2.0))
        if geom == "cavity":
            n = max(4, int(round(math.sqrt(C))))
            c = cases.cavity_case(n=n, nv=N, vmax=vmax, Kn=Kn, lid=U)
        else:
            c = cases.cylinder_case(n_cells=C, nvx=N, nvy=N, mach=Ma, Kn=Kn, seed=1000 + i,
                                    vx=(-vmax, vmax), vy=(-vmax, vmax))
        c["request"] = {"geometry": geom, "cells": len(c["mesh"]["cell_vol"]), "nv": N * N, "Kn": Kn, "Mach": Ma}
        out.append(c)
    return out


def poisson_arrivals(n, rate, seed=44):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
