"""Domain decomposition of a mesh into subdomains with a two-ring halo
(Sec. 3.3 and Algorithm 2 of the paper: physical-space partitions that
exchange the distribution of their boundary cells every step).

Host-side bookkeeping only: the partition, each subdomain's mesh (its own
cells first, then the halo), and the lists of cells the subdomains send to
and receive from each other.  The state moves through the library's halo
calls (ugks_halo_pack / ugks_halo_unpack, device buffers); between GPUs the
buffers travel by torch.distributed point-to-point messages (NCCL), within one
GPU by device copies.

One explicit step updates a cell from data at most two face rings away (the
limited slopes of its face neighbours read their own neighbours).  A subdomain
therefore holds its own cells S0, the first ring S1 \\ S0 and the second ring
S2 \\ S1, with every face of every S1 cell; a step updates S0 exactly as a
step of the whole mesh, given the same time step, and the halo's values are
replaced by their owners' before the next step.
"""
from __future__ import annotations

import numpy as np

from . import cases


def partition(mesh, nparts):
    """Recursive coordinate bisection: the cells are split along the longest
    extent of their centroids at the position that divides the parts in
    proportion, recursively, into ``nparts`` spatially compact parts whose
    sizes differ by at most one cell per level.  Returns part[C] in
    [0, nparts)."""
    x = np.asarray(mesh["cell_xc"], float)
    C = len(x)
    if not 1 <= nparts <= C:
        raise ValueError("need 1 <= nparts <= number of cells")
    part = np.empty(C, np.int64)

    def split(ids, p0, n):
        if n == 1:
            part[ids] = p0
            return
        ext = x[ids].max(axis=0) - x[ids].min(axis=0)
        d = int(np.argmax(ext))
        order = ids[np.argsort(x[ids, d], kind="stable")]
        nl = n // 2
        cut = len(ids) * nl // n
        split(order[:cut], p0, nl)
        split(order[cut:], p0 + nl, n - nl)

    split(np.arange(C, dtype=np.int64), 0, nparts)
    return part


class Subdomain:
    """Part ``p`` of a mesh: ``mesh`` lists the own cells first (ascending
    global id), then the halo (ascending global id); ``l2g`` maps local to
    global cell ids, ``n_own`` counts the own cells, ``faces`` are the global ids
    of the subdomain's faces (global face order kept)."""

    def __init__(self, mesh, part, p):
        ptr, nb = cases._adjacency(mesh)
        own = np.nonzero(np.asarray(part) == p)[0]
        s1 = cases._grow(ptr, nb, own)
        s2 = cases._grow(ptr, nb, s1)
        halo = np.setdiff1d(s2, own)
        self.p = p
        self.n_own = len(own)
        self.l2g = np.concatenate([own, halo]).astype(np.int64)
        C = len(mesh["cell_vol"])
        g2l = -np.ones(C, np.int64)
        g2l[self.l2g] = np.arange(len(self.l2g))
        self.g2l = g2l
        fc = np.asarray(mesh["face_cells"])
        own_c, nei = fc[:, 0], fc[:, 1]
        in1 = np.zeros(C, bool)
        in1[s1] = True
        faces = np.nonzero(in1[own_c] | ((nei >= 0) & in1[np.maximum(nei, 0)]))[0]
        o, n = own_c[faces], nei[faces]
        sub_fc = np.stack([g2l[o], np.where(n >= 0, g2l[np.maximum(n, 0)], -1)], axis=1)
        assert (sub_fc[:, 0] >= 0).all() and ((n < 0) | (sub_fc[:, 1] >= 0)).all()
        self.faces = faces
        m = {"dim": mesh["dim"],
             "cell_xc": np.ascontiguousarray(np.asarray(mesh["cell_xc"])[self.l2g]),
             "cell_vol": np.ascontiguousarray(np.asarray(mesh["cell_vol"])[self.l2g]),
             "face_cells": np.ascontiguousarray(sub_fc)}
        for k in ("face_n", "face_S", "face_xc", "face_type", "face_tag", "face_shift"):
            m[k] = np.ascontiguousarray(np.asarray(mesh[k])[faces])
        self.mesh = m


def halo_plan(part, subs):
    """Who sends what to whom.  Returns (send, recv): send[p][q] are the local
    ids in subdomain p of its own cells that subdomain q holds in its halo,
    recv[q][p] the local ids of the same cells in q, both in ascending global
    id, so that row i of p's buffer for q lands on q's cell recv[q][p][i].
    Only pairs with cells to exchange appear."""
    part = np.asarray(part)
    send = {s.p: {} for s in subs}
    recv = {s.p: {} for s in subs}
    for sq in subs:
        halo_g = sq.l2g[sq.n_own:]
        owner = part[halo_g]
        for p in np.unique(owner):
            g = halo_g[owner == p]                        # ascending global id
            sp = subs[int(p)]
            recv[sq.p][int(p)] = sq.g2l[g]
            send[int(p)][sq.p] = sp.g2l[g]
    return send, recv


def exchange(dist, rank, send, recv, pack, new_buffer, unpack):
    """One halo exchange of rank ``rank`` over torch.distributed: for every
    peer q in send[rank], ``pack(q)`` gives the tensor to send; for every peer
    p in recv[rank], a tensor from ``new_buffer(p)`` receives p's rows and
    ``unpack(p, tensor)`` stores them.  All messages are posted before any is
    waited for, so no ordering between ranks can deadlock."""
    reqs, bufs = [], {}
    for p in sorted(recv[rank]):
        bufs[p] = new_buffer(p)
        reqs.append(dist.irecv(bufs[p], src=p))
    out = []
    for q in sorted(send[rank]):
        t = pack(q)
        out.append(t)
        reqs.append(dist.isend(t, dst=q))
    for r in reqs:
        r.wait()
    for p in sorted(bufs):
        unpack(p, bufs[p])


def global_dt(lib, mesh_subs, vgrid, cfl):
    """The whole mesh's CFL step from its subdomains: the minimum over them of
    ugks_cfl_dt over their own cells."""
    return min(lib.cfl_dt(s.mesh, vgrid, cfl, s.n_own) for s in mesh_subs)


class DecomposedCase:
    """A case split into ``nparts`` subdomains stepped on one GPU: each step
    steps every subdomain once, then moves the halo rows by device copies
    (ugks_halo_pack into a buffer, ugks_halo_unpack from it).  All
    subdomains share one stream, so the moves are ordered after the steps.
    ``tiling`` fixes the gather tiling of every subdomain (it must match the
    undivided case's for bit-identical results)."""

    def __init__(self, case, nparts, precision, stream=None, **tiling):
        import torch
        from . import _lib
        self._lib = _lib
        mesh, vg, pr, init = case["mesh"], case["vgrid"], case["params"], case["init"]
        self.C = len(mesh["cell_vol"])
        self.D = int(mesh["dim"])
        self.part = partition(mesh, nparts)
        self.subs = [Subdomain(mesh, self.part, p) for p in range(nparts)]
        self.send, self.recv = halo_plan(self.part, self.subs)
        dt = pr.get("dt", 0.0) or global_dt(_lib, self.subs, vg, pr["cfl"])
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        init = np.asarray(init)
        self.cases = []
        for s in self.subs:
            c = _lib.Case(s.mesh, vg, dict(pr, dt=dt), init[s.l2g], precision=precision, stream=stream, **tiling)
            c.set_owned(s.n_own)
            self.cases.append(c)
        self.dt = dt
        # halo slots: slot q of subdomain p sends to q, slot nparts + p of q receives from p
        self.bufs = {}
        for p, peers in self.send.items():
            row = self.cases[p].halo_row_bytes()
            for q, ids in peers.items():
                self.cases[p].halo_set(q, ids)
                self.cases[q].halo_set(nparts + p, self.recv[q][p])
                self.bufs[(p, q)] = torch.empty(len(ids) * row, dtype=torch.uint8, device="cuda")
        self.nparts = nparts

    def exchange(self):
        for (p, q), buf in self.bufs.items():
            self.cases[p].halo_pack(q, buf.data_ptr())
            self.cases[q].halo_unpack(self.nparts + p, buf.data_ptr())

    def step(self, n=1):
        for _ in range(int(n)):
            for c in self.cases:
                c.step(1)
            self.exchange()

    def set_state(self, f=None, W=None):
        for s, c in zip(self.subs, self.cases):
            c.set_state(None if f is None else np.asarray(f)[s.l2g], None if W is None else np.asarray(W)[s.l2g])

    def state(self):
        """(f, W) of the whole mesh in global cell order, from the own cells."""
        f, W = None, np.empty((self.C, self.D + 2))
        for s, c in zip(self.subs, self.cases):
            fs, Ws = c.state()
            if f is None:
                f = np.empty((self.C,) + fs.shape[1:])
            own = s.l2g[:s.n_own]
            f[own] = fs[:s.n_own]
            W[own] = Ws[:s.n_own]
        return f, W

    def residual(self):
        tot = sum(c.residual_sums() for c in self.cases)
        M = self.D + 2
        return np.sqrt(tot[:M]) / np.sqrt(tot[M:])

    def density_range(self):
        """(min rho, max rho) over the whole mesh: each subdomain reports its
        own cells (across ranks: an all-reduce MIN and MAX of these)."""
        r = [c.density_range() for c in self.cases]
        return min(a for a, _ in r), max(b for _, b in r)

    def close(self):
        for c in self.cases:
            c.close()
        self.cases = []
