"""Batched stepping (ugks_batch_*): cases of different meshes and velocity
grids stepped together with one persistent gather launch per velocity-tile
width, captured as a CUDA graph, give bit-identical results to stepping each
case alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2412_06546_gb300 import _lib, cases as cs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2412_06546_gb300 import build
    build.build()


def _cases2d():
    return [cs.cavity_case(n=12, nv=16),
            cs.cylinder_case(n_cells=1500, nvx=20, nvy=18, mach=3.0),
            cs.cylinder_case(n_cells=800, nvx=12, nvy=10, mach=1.5, Kn=1.0),
            cs.cavity_case(n=7, nv=28, Kn=0.5, lid=0.3)]


@pytest.mark.parametrize("precision", [_lib.FP32, _lib.FP64])
def test_batch_matches_cases_stepped_alone(precision):
    specs = _cases2d()
    alone = [_lib.Case(c["mesh"], c["vgrid"], c["params"], c["init"], precision=precision) for c in specs]
    for g in alone:
        g.step(7)
    together = [_lib.Case(c["mesh"], c["vgrid"], c["params"], c["init"], precision=precision) for c in specs]
    b = _lib.Batch(together)
    b.step(3)
    b.step(4)
    for a, t in zip(alone, together):
        fa, Wa = a.state()
        ft, Wt = t.state()
        assert np.array_equal(fa, ft) and np.array_equal(Wa, Wt)
        assert a.info()["step"] == t.info()["step"] == 7
        assert np.array_equal(a.residual(), t.residual())
    b.close()


def test_batch_3d_and_interleaving_with_single_steps():
    specs = [cs.sphere_case(n_cells=1500, nv=8, vmax=7.0, mach=2.0),
             {"mesh": cs.hex_mesh(5, 4, 4), "vgrid": cs.cartesian_vgrid((8, 8, 8), (-4,) * 3, (4,) * 3),
              "params": cs.params(0.05, walls=[{"T": 1.0, "U": [0, 0, 0]}]),
              "init": cs.uniform_state(80, 3)}]
    alone = [_lib.Case(c["mesh"], c["vgrid"], c["params"], c["init"], precision=_lib.FP32) for c in specs]
    mixed = [_lib.Case(c["mesh"], c["vgrid"], c["params"], c["init"], precision=_lib.FP32) for c in specs]
    for g in alone:
        g.step(5)
    b = _lib.Batch(mixed)
    b.step(2)
    mixed[0].step(1)            # a single-case step between batch steps
    mixed[1].step(1)
    b.step(2)
    for a, t in zip(alone, mixed):
        assert np.array_equal(a.state()[0], t.state()[0])


def test_batch_with_mixed_velocity_tiles():
    """Cases tiled with 32, 64 and 128 velocities per CTA, and 256- or
    512-thread CTAs, in one batch (one persistent launch per tile width and
    block size) match the same cases stepped alone."""
    specs = _cases2d()[:3]
    tiles = [(24, 32, 256), (48, 64, 512), (16, 128, 256)]
    mk = lambda c, t: _lib.Case(c["mesh"], c["vgrid"], c["params"], c["init"], precision=_lib.FP32,
                                patch_cells=t[0], vtile=t[1], threads=t[2])
    alone = [mk(c, t) for c, t in zip(specs, tiles)]
    for g in alone:
        g.step(4)
    together = [mk(c, t) for c, t in zip(specs, tiles)]
    b = _lib.Batch(together)
    b.step(4)
    for a, t in zip(alone, together):
        assert np.array_equal(a.state()[0], t.state()[0])
        assert np.array_equal(a.residual(), t.residual())
    b.close()


def test_batch_rejects_mixed_precision():
    c = cs.cavity_case(n=4, nv=8)
    g1 = _lib.Case(c["mesh"], c["vgrid"], c["params"], c["init"], precision=_lib.FP32)
    g2 = _lib.Case(c["mesh"], c["vgrid"], c["params"], c["init"], precision=_lib.FP64)
    with pytest.raises(_lib.UGKSError) as e:
        _lib.Batch([g1, g2])
    assert e.value.code == 1


def _variant_cases():
    """2D cases that take different kernels of a step: separable face sums
    (tensor grid, walls), general face sums (unstructured velocity set),
    the analytic W0 (no first face reduction) and a periodic mesh (no walls,
    no far field)."""
    rng = np.random.default_rng(8)
    cav = cs.cavity_case(n=9, nv=14, Kn=0.2, lid=0.4)
    cyl = cs.cylinder_case(n_cells=700, nvx=12, nvy=12, mach=2.0)
    vg = cyl["vgrid"]
    perm = rng.permutation(len(vg["w"]))
    u = np.asarray(vg["u"])[perm] + rng.uniform(-0.1, 0.1, size=np.asarray(vg["u"]).shape)
    w = np.asarray(vg["w"])[perm] * rng.uniform(0.9, 1.1, size=len(perm))
    unstructured = dict(cyl, vgrid={"dim": 2, "u": u, "w": w, "cart_n": [0, 0, 0]})
    analytic = cs.cylinder_case(n_cells=500, nvx=10, nvy=11, mach=1.2, Kn=0.5)
    analytic = dict(analytic, params=dict(analytic["params"], w0_analytic=1))
    mesh = cs.periodic_tri_mesh(7, 6, 1.0, 0.8, jitter=0.2, seed=4)
    periodic = {"mesh": mesh, "vgrid": cs.cartesian_vgrid((10, 9), (-5, -4.5), (5, 4.5)),
                "params": cs.params(0.05), "init": cs.smooth_state(mesh, 5, 0.15, U0=[0.3, -0.2])}
    return [cav, unstructured, analytic, periodic]


@pytest.mark.parametrize("precision", [_lib.FP32, _lib.FP64])
def test_batch_with_cases_that_skip_kernels(precision):
    """Every kernel of a batch step is one launch over all cases; a case that
    does not run a kernel (no walls, no general sums, no first reduction)
    owns no blocks of it.  Each case still matches itself stepped alone."""
    specs = _variant_cases()
    mk = lambda c: _lib.Case(c["mesh"], c["vgrid"], c["params"], c["init"], precision=precision)
    alone = [mk(c) for c in specs]
    for g in alone:
        g.step(3)
    together = [mk(c) for c in specs]
    b = _lib.Batch(together)
    b.step(3)
    for a, t in zip(alone, together):
        assert np.array_equal(a.state()[0], t.state()[0])
        assert np.array_equal(a.state()[1], t.state()[1])
        assert np.array_equal(a.residual(), t.residual())
    b.close()
