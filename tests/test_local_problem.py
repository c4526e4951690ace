"""The local-problem construction behind the sampled full-size checks, pinned
on the oracle alone: one step of the sub-mesh (sample cells plus two face
rings, every face of the inner ring) from the full state restricted to it
gives the full-mesh step at the sample cells."""
import numpy as np
import pytest

import oracle
from paper_2412_06546_gb300 import cases as cs


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _check(case, n_sample, seed, rings=2):
    mesh = case["mesh"]
    full = oracle.OracleCase(mesh, case["vgrid"], case["params"], case["init"], n_threads=0)
    f0, W0, _ = full.state()
    f0 = f0 * cs.perturbation(f0.shape, seed, 0.1)          # non-equilibrium state
    full.set_state(f0, W0)
    full.step(1)                                              # a developed W and q
    fn, Wn, _ = full.state()
    full.step(1)
    f1, W1, _ = full.state()

    sample = cs.pick_sample(mesh, n_sample, seed)
    sub, s2, pos = cs.local_problem(mesh, sample, rings)
    assert len(s2) < len(mesh["cell_vol"])
    params = dict(case["params"], dt=full.dt)
    loc = oracle.OracleCase(sub, case["vgrid"], params, np.asarray(case["init"])[s2], n_threads=0)
    loc.set_state(fn[s2], Wn[s2])
    loc.step(1)
    fl, Wl, _ = loc.state()
    return (np.abs(fl[pos] - f1[sample]).max() / np.abs(f1[sample]).max(),
            np.abs(Wl[pos] - W1[sample]).max() / np.abs(W1[sample]).max())


def test_local_problem_reproduces_the_step_2d():
    ef, eW = _check(cs.cylinder_case(n_cells=1500, nvx=12, nvy=10, mach=3.0), 24, 5)
    assert ef <= 1e-14 and eW <= 1e-14


def test_local_problem_reproduces_the_step_3d():
    ef, eW = _check(cs.sphere_case(n_cells=1500, nv=6, vmax=6.0, mach=2.0), 24, 6)
    assert ef <= 1e-14 and eW <= 1e-14


def test_one_ring_is_not_enough():
    """Negative control: without the second ring the sample cells' step
    differs (their neighbours' slopes and face states lose data)."""
    ef, eW = _check(cs.cylinder_case(n_cells=1500, nvx=12, nvy=10, mach=3.0), 24, 5, rings=1)
    assert ef > 1e-8


def test_local_problem_periodic_and_walls():
    mesh = cs.quad_mesh(12, 10, left="periodic", right="periodic", bottom=("wall", 0), top=("wall", 1))
    case = {"mesh": mesh, "vgrid": cs.cartesian_vgrid((12, 12), (-4, -4), (4, 4)),
            "params": cs.params(0.2, walls=[{"T": 1.0, "U": [0, 0]}, {"T": 1.2, "U": [0.3, 0]}]),
            "init": cs.uniform_state(120, 2)}
    ef, eW = _check(case, 12, 7)
    assert ef <= 1e-14 and eW <= 1e-14
