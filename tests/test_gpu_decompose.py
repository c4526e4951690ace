"""Domain decomposition on one GPU (Sec. 3.3, Algorithm 2): subdomain cases
with a two-ring halo, stepped one step at a time with a halo exchange through
ugks_halo_pack / ugks_halo_unpack and device copies, give bitwise the same f,
W and heat flux on every cell as the undivided case stepped alone (same time
step and gather tiling), and the same residual up to the order of the sums."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2412_06546_gb300 import _lib, cases as cs, decompose as dc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2412_06546_gb300 import build
    build.build()


def _case(name):
    if name == "cylinder":
        return cs.cylinder_case(n_cells=2500, nvx=24, nvy=20, mach=3.0)
    if name == "periodic":
        mesh = cs.periodic_tri_mesh(16, 12, 1.0, 0.8, jitter=0.25, seed=4)
        return {"mesh": mesh, "vgrid": cs.cartesian_vgrid((14, 12), (-5, -4.5), (5, 4.5)),
                "params": cs.params(0.05), "init": cs.smooth_state(mesh, 5, 0.15, U0=[0.3, -0.2])}
    return cs.sphere_case(n_cells=3000, nv=10, vmax=6.0, mach=2.0)


@pytest.mark.parametrize("name,precision", [("cylinder", _lib.FP64), ("cylinder", _lib.FP32),
                                            ("periodic", _lib.FP32), ("sphere", _lib.FP32),
                                            ("sphere", _lib.FP64)])
@pytest.mark.parametrize("nparts", [2, 3])
def test_decomposed_steps_are_bitwise_the_undivided_steps(name, precision, nparts):
    case = _case(name)
    mesh, vg, pr, init = case["mesh"], case["vgrid"], case["params"], case["init"]
    tiling = {"patch_cells": 32, "vtile": 32 if precision == _lib.FP64 else 64, "threads": 256, "tile_group": 1}
    dt = _lib.cfl_dt(mesh, vg, pr["cfl"])
    case = dict(case, params=dict(pr, dt=dt))
    full = _lib.Case(mesh, vg, case["params"], init, precision=precision, **tiling)
    dec = dc.DecomposedCase(case, nparts, precision, **tiling)
    assert dec.dt == dt
    f0, W0 = full.state()
    f0 = f0 * cs.perturbation(f0.shape, 7, 0.1)
    if precision == _lib.FP32:
        f0 = f0.astype(np.float32).astype(np.float64)
    full.set_state(f0, W0)
    dec.set_state(f0, W0)
    for step in range(3):
        full.step(1)
        dec.step(1)
        ff, Wf = full.state()
        fd, Wd = dec.state()
        assert np.array_equal(fd, ff), (name, step, np.abs(fd - ff).max())
        assert np.array_equal(Wd, Wf), (name, step, np.abs(Wd - Wf).max())
    qf = full.heat_flux()
    for s, c in zip(dec.subs, dec.cases):
        assert np.array_equal(c.heat_flux()[:s.n_own], qf[s.l2g[:s.n_own]])
        # the exchange left the halo with the owners' values too
        fs, Ws = c.state()
        assert np.array_equal(fs, ff[s.l2g]) and np.array_equal(Ws, Wf[s.l2g])
    assert np.allclose(dec.residual(), full.residual(), rtol=1e-12, atol=0)
    dec.close()
    full.close()


def test_halo_rows_round_trip():
    """Rows packed from one case and unpacked into another carry f, W and q
    exactly, in the listed order."""
    case = cs.cylinder_case(n_cells=900, nvx=12, nvy=10, mach=2.0)
    a = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=_lib.FP32)
    b = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=_lib.FP32)
    fa, Wa = a.state()
    fa = (fa * cs.perturbation(fa.shape, 9, 0.2)).astype(np.float32)
    a.set_state(fa, Wa * 1.01)
    src = np.array([5, 17, 3, 400, 899, 0], np.int64)
    dst = np.array([100, 2, 300, 301, 7, 899], np.int64)
    a.halo_set(0, src)
    b.halo_set(1, dst)
    buf = torch.empty(len(src) * a.halo_row_bytes(), dtype=torch.uint8, device="cuda")
    a.halo_pack(0, buf.data_ptr())
    b.halo_unpack(1, buf.data_ptr())
    fa2, Wa2 = a.state()
    fb, Wb = b.state()
    assert np.array_equal(fb[dst], fa2[src]) and np.array_equal(Wb[dst], Wa2[src])
    assert np.array_equal(b.heat_flux()[dst], a.heat_flux()[src])
    a.close()
    b.close()
