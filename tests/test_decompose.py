"""Domain decomposition on the CPU (Sec. 3.3, Algorithm 2): the partition,
the two-ring subdomains, the halo plan and the exchange, checked without a
GPU.  Subdomains are stepped by the oracle: every step of every subdomain
followed by a halo exchange reproduces the whole-mesh steps on the own cells.
Two gloo ranks run the same exchange routine the GPU path runs over NCCL."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2412_06546_gb300 import _lib, cases as cs, decompose as dc


def _cases():
    cyl = cs.cylinder_case(n_cells=700, nvx=10, nvy=8, mach=2.0)
    per = {"mesh": cs.periodic_tri_mesh(9, 7, 1.0, 0.8, jitter=0.25, seed=4),
           "vgrid": cs.cartesian_vgrid((8, 8), (-5, -5), (5, 5)), "params": cs.params(0.05)}
    per["init"] = cs.smooth_state(per["mesh"], 5, 0.15, U0=[0.3, -0.2])
    sph = cs.sphere_case(n_cells=900, nv=5, vmax=5.0, mach=1.5)
    return {"cylinder": cyl, "periodic": per, "sphere": sph}


CASES = _cases()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("nparts", [2, 3, 5])
def test_partition_subdomains_and_plan(name, nparts):
    mesh = CASES[name]["mesh"]
    C = len(mesh["cell_vol"])
    part = dc.partition(mesh, nparts)
    assert np.array_equal(part, dc.partition(mesh, nparts))                 # deterministic
    sizes = np.bincount(part, minlength=nparts)
    assert sizes.sum() == C and sizes.min() > 0 and sizes.max() - sizes.min() <= nparts
    subs = [dc.Subdomain(mesh, part, p) for p in range(nparts)]
    ptr, nb = cs._adjacency(mesh)
    for s in subs:
        own = s.l2g[:s.n_own]
        assert np.array_equal(own, np.nonzero(part == s.p)[0])
        ring2 = cs._grow(ptr, nb, cs._grow(ptr, nb, own))
        assert np.array_equal(np.sort(s.l2g), ring2)                        # own + two face rings exactly
        # every face of the own cells and of the first ring is present
        s1 = cs._grow(ptr, nb, own)
        fc = mesh["face_cells"]
        need = np.nonzero(np.isin(fc[:, 0], s1) | np.isin(fc[:, 1], s1))[0]
        assert np.array_equal(s.faces, need)
    send, recv = dc.halo_plan(part, subs)
    seen = [np.zeros(len(s.l2g) - s.n_own, int) for s in subs]
    for p in send:
        for q, ids in send[p].items():
            gp = subs[p].l2g[ids]
            gq = subs[q].l2g[recv[q][p]]
            assert np.array_equal(gp, gq) and np.all(np.diff(gp) > 0)
            assert (ids < subs[p].n_own).all() and (recv[q][p] >= subs[q].n_own).all()
            assert (part[gp] == p).all()
            seen[q][recv[q][p] - subs[q].n_own] += 1
    assert all((v == 1).all() for v in seen)                                # each halo cell from its owner, once


@pytest.mark.parametrize("name", sorted(CASES))
def test_subdomain_time_step_is_the_whole_mesh_step(name):
    """ugks_cfl_dt (host computation in the CUDA library, no GPU needed) over
    each subdomain's own cells: the minimum over the subdomains is bitwise the
    whole mesh's step."""
    c = CASES[name]
    if not c["params"]["cfl"] > 0:
        pytest.skip("fixed step")
    mesh = c["mesh"]
    full = _lib.cfl_dt(mesh, c["vgrid"], c["params"]["cfl"])
    part = dc.partition(mesh, 3)
    subs = [dc.Subdomain(mesh, part, p) for p in range(3)]
    assert dc.global_dt(_lib, subs, c["vgrid"], c["params"]["cfl"]) == full
    o = oracle.OracleCase(mesh, c["vgrid"], c["params"], c["init"])
    assert abs(o.dt - full) <= 1e-15 * full


def _exchange_serial(subs, send, recv, states):
    """The halo exchange on one process: subdomain q's halo rows take the
    values of their owners' own cells."""
    for p, peers in send.items():
        for q, ids in peers.items():
            for a in range(len(states[p])):
                states[q][a][recv[q][p]] = states[p][a][ids]


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("nparts", [2, 3])
def test_stepped_subdomains_with_exchange_match_the_whole_mesh(name, nparts):
    c = CASES[name]
    mesh, vg, pr = c["mesh"], c["vgrid"], c["params"]
    full = oracle.OracleCase(mesh, vg, pr, c["init"], n_threads=0)
    f0, W0, _ = full.state()
    f0 = f0 * cs.perturbation(f0.shape, 3, 0.1)
    full.set_state(f0, W0)
    part = dc.partition(mesh, nparts)
    subs = [dc.Subdomain(mesh, part, p) for p in range(nparts)]
    send, recv = dc.halo_plan(part, subs)
    prs = dict(pr, dt=full.dt)
    loc = [oracle.OracleCase(s.mesh, vg, prs, np.asarray(c["init"])[s.l2g], n_threads=0) for s in subs]
    for s, o in zip(subs, loc):
        o.set_state(f0[s.l2g], W0[s.l2g])
    for step in range(3):
        full.step(1)
        states = []
        for o in loc:
            o.step(1)
            f, W, _ = o.state()
            states.append([f, W])
        _exchange_serial(subs, send, recv, states)
        for o, (f, W) in zip(loc, states):
            o.set_state(f, W)
        ff, Wf, _ = full.state()
        for s, (f, W) in zip(subs, states):
            own = s.l2g[:s.n_own]
            assert np.abs(f[:s.n_own] - ff[own]).max() <= 1e-13 * np.abs(ff).max(), (name, step, s.p)
            assert np.abs(W[:s.n_own] - Wf[own]).max() <= 1e-13 * np.abs(Wf).max(), (name, step, s.p)
            # after the exchange the halo holds the owners' values too
            assert np.abs(f - ff[s.l2g]).max() <= 1e-13 * np.abs(ff).max()


# ---------------------------------------------------------------- two gloo ranks
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    c = CASES["cylinder"]
    mesh, vg, pr = c["mesh"], c["vgrid"], c["params"]
    part = dc.partition(mesh, ws)
    subs = [dc.Subdomain(mesh, part, p) for p in range(ws)]          # every rank derives the same plan
    send, recv = dc.halo_plan(part, subs)
    me = subs[rank]
    # 1) the exchange delivers each halo cell its owner's value
    vals = np.where(np.arange(len(me.l2g)) < me.n_own, me.l2g, -1).astype(np.float64)
    dc.exchange(dist, rank, send, recv,
                pack=lambda q: torch.from_numpy(vals[send[rank][q]].copy()),
                new_buffer=lambda p: torch.empty(len(recv[rank][p]), dtype=torch.float64),
                unpack=lambda p, t: vals.__setitem__(recv[rank][p], t.numpy()))
    ids_ok = bool(np.array_equal(vals, me.l2g.astype(np.float64)))
    # 2) oracle-stepped subdomain + exchange of f and W over gloo, two steps
    full = oracle.OracleCase(mesh, vg, pr, c["init"], n_threads=1)
    f0, W0, _ = full.state()
    f0 = f0 * cs.perturbation(f0.shape, 3, 0.1)
    full.set_state(f0, W0)
    o = oracle.OracleCase(me.mesh, vg, dict(pr, dt=full.dt), np.asarray(c["init"])[me.l2g], n_threads=1)
    o.set_state(f0[me.l2g], W0[me.l2g])
    row = f0.shape[1] * f0.shape[2] + W0.shape[1]
    err = 0.0
    for _ in range(2):
        full.step(1)
        o.step(1)
        f, W, _ = o.state()
        rows = np.concatenate([f.reshape(len(f), -1), W], axis=1)

        def unpack(p, t):
            r = t.numpy().reshape(-1, row)
            rows[recv[rank][p]] = r
        dc.exchange(dist, rank, send, recv,
                    pack=lambda q: torch.from_numpy(np.ascontiguousarray(rows[send[rank][q]]).ravel()),
                    new_buffer=lambda p: torch.empty(len(recv[rank][p]) * row, dtype=torch.float64),
                    unpack=unpack)
        f = rows[:, :f.shape[1] * f.shape[2]].reshape(f.shape)
        W = rows[:, f.shape[1] * f.shape[2]:]
        o.set_state(f, W)
        ff, Wf, _ = full.state()
        err = max(err, np.abs(f - ff[me.l2g]).max() / np.abs(ff).max(), np.abs(W - Wf[me.l2g]).max() / np.abs(Wf).max())
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ids_ok, err))


def test_two_gloo_ranks_exchange_and_step():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {r: (ok, e) for r, ok, e in (q.get(timeout=300) for _ in procs)}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ok, e = got[r]
        assert ok, r
        assert e <= 1e-13, (r, e)
