"""Local problems for sampled checks of cases too large for a whole oracle run.

One explicit step updates a cell from data no further than two face rings
away: the limited slopes of the cell and of its face neighbours (each reads
its own neighbours' values), the interface equilibria of its faces (face
states of both sides, whose limited macroscopic gradients read the second
ring), the heat flux of both sides and, at walls, the cell's own
distribution.  A mesh made of the sample S0, S1 = S0 + face neighbours,
S2 = S1 + their face neighbours, with every face of every S1 cell, stepped
once from the same state on S2 with the same time step, therefore gives the
full-mesh step on S0.  Cells of S2 outside S1 lose faces and so get wrong
values of their own, which no S0 result reads.
"""
import numpy as np

INTERIOR, WALL, FARFIELD, PERIODIC = 0, 1, 2, 3


def _adjacency(mesh):
    fc = np.asarray(mesh["face_cells"])
    ft = np.asarray(mesh["face_type"])
    inner = (ft == INTERIOR) | (ft == PERIODIC)
    a, b = fc[inner, 0], fc[inner, 1]
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    order = np.argsort(src, kind="stable")
    C = len(mesh["cell_vol"])
    ptr = np.zeros(C + 1, np.int64)
    np.add.at(ptr, src + 1, 1)
    return np.cumsum(ptr), dst[order]


def _grow(ptr, nb, cells):
    return np.unique(np.concatenate([cells] + [nb[ptr[c]:ptr[c + 1]] for c in cells]))


def local_problem(mesh, sample, rings=2):
    """Return (sub-mesh, S2 cell ids in the full mesh, positions of the sample
    cells in S2).  Sub-mesh faces keep the full mesh's face order.  ``rings``
    < 2 builds a mesh that is too small (for the negative control)."""
    sample = np.unique(np.asarray(sample, np.int64))
    ptr, nb = _adjacency(mesh)
    s1 = sample
    for _ in range(rings - 1):
        s1 = _grow(ptr, nb, s1)
    s2 = _grow(ptr, nb, s1)
    C = len(mesh["cell_vol"])
    fc = np.asarray(mesh["face_cells"])
    own, nei = fc[:, 0], fc[:, 1]
    in1 = np.zeros(C, bool)
    in1[s1] = True
    faces = np.nonzero(in1[own] | ((nei >= 0) & in1[np.maximum(nei, 0)]))[0]
    loc = -np.ones(C, np.int64)
    loc[s2] = np.arange(len(s2))
    o, n = own[faces], nei[faces]
    sub_fc = np.stack([loc[o], np.where(n >= 0, loc[np.maximum(n, 0)], -1)], axis=1)
    assert (sub_fc[:, 0] >= 0).all() and ((n < 0) | (sub_fc[:, 1] >= 0)).all()
    sub = {"dim": mesh["dim"],
           "cell_xc": np.ascontiguousarray(np.asarray(mesh["cell_xc"])[s2]),
           "cell_vol": np.ascontiguousarray(np.asarray(mesh["cell_vol"])[s2]),
           "face_cells": np.ascontiguousarray(sub_fc)}
    for k in ("face_n", "face_S", "face_xc", "face_type", "face_tag", "face_shift"):
        sub[k] = np.ascontiguousarray(np.asarray(mesh[k])[faces])
    return sub, s2, loc[sample]


def pick_sample(mesh, n, seed):
    """Seeded sample of n cells: a quarter next to walls, a quarter next to the
    far field (where the mesh has them), the rest anywhere."""
    rng = np.random.default_rng(seed)
    fc = np.asarray(mesh["face_cells"])
    ft = np.asarray(mesh["face_type"])
    C = len(mesh["cell_vol"])
    picks = []
    for t in (WALL, FARFIELD):
        cand = np.unique(fc[ft == t, 0])
        if len(cand):
            picks.append(rng.choice(cand, size=min(len(cand), n // 4), replace=False))
    picks.append(rng.choice(C, size=n - sum(len(p) for p in picks), replace=False))
    return np.unique(np.concatenate(picks))
