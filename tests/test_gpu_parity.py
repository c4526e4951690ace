"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Both sides start from the same seeded, perturbed (non-equilibrium) state and
take the same steps; f, W and the heat flux are compared element by element.
FP64 path: |delta| <= 1e-12 max|x| per element (and relative L2 <= 1e-12).
FP32-storage path: relative L2 on W <= 1e-5 after 100 steps.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2412_06546_gb300 import _lib, cases as cs  # noqa: E402

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2412_06546_gb300 import build
    build.build()
    oracle.build()


def _pair(case, precision=_lib.FP64, perturb=0.1, seed=1, params=None, init=None, **kw):
    pr = params or case["params"]
    ini = case["init"] if init is None else init
    o = oracle.OracleCase(case["mesh"], case["vgrid"], pr, ini, n_threads=0)
    g = _lib.Case(case["mesh"], case["vgrid"], pr, ini, precision=precision, **kw)
    if perturb:
        f0, W0, _ = o.state()
        f0 = f0 * cs.perturbation(f0.shape, seed, perturb)
        o.set_state(f0, W0)
        g.set_state(f0, W0)
    return o, g


def _rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _compare(o, g, tol=TOL64, what=""):
    fo, Wo, qo = o.state()
    fg, Wg = g.state()
    qg = g.heat_flux()
    errs = {"f": _rel_max(fg, fo), "W": _rel_max(Wg, Wo),
            "q": np.abs(qg - qo).max() / max(np.abs(qo).max(), 1e-3),
            "f_l2": _rel_l2(fg, fo), "W_l2": _rel_l2(Wg, Wo)}
    for k, v in errs.items():
        assert v <= tol, (what, k, v, errs)
    return errs


def test_initial_state_matches():
    case = cs.cavity_case()
    o, g = _pair(case, perturb=0)
    _compare(o, g, what="init")


@pytest.mark.parametrize("steps", [1, 10])
def test_cavity_fp64(steps):
    case = cs.cavity_case()                        # 20x20 quads x 24^2, Shakhov
    o, g = _pair(case)
    o.step(steps)
    g.step(steps)
    _compare(o, g, what=f"cavity {steps}")
    assert np.allclose(g.residual(), o.residual(), rtol=1e-9, atol=1e-15)


def test_cylinder_walls_farfield_ragged_velocity_tail():
    case = cs.cylinder_case(n_cells=2000, nvx=21, nvy=17, mach=5.0)   # Nv = 357 (ragged)
    o, g = _pair(case, perturb=0.05)
    o.step(2)
    g.step(2)
    _compare(o, g, what="cylinder")


def test_periodic_shakhov_smooth_state():
    mesh = cs.periodic_tri_mesh(9, 7, 1.0, 0.8, jitter=0.25, seed=4)
    case = {"mesh": mesh, "vgrid": cs.cartesian_vgrid((12, 10), (-5, -4.5), (5, 4.5)),
            "params": cs.params(0.03), "init": cs.smooth_state(mesh, 5, 0.15, U0=[0.3, -0.2])}
    o, g = _pair(case, perturb=0.2)
    o.step(3)
    g.step(3)
    _compare(o, g, what="periodic")


def test_3d_box_moving_wall():
    mesh = cs.hex_mesh(4, 4, 3, sides={"x-": ("wall", 0), "x+": ("wall", 0), "y-": ("wall", 0),
                                       "y+": ("wall", 0), "z-": ("wall", 0), "z+": ("wall", 1)})
    vg = cs.cartesian_vgrid((9, 8, 7), (-4, -4, -4), (4, 4, 4))
    pr = cs.params(0.1, walls=[{"T": 1.0, "U": [0, 0, 0]}, {"T": 1.2, "U": [0.3, 0.1, 0]}])
    case = {"mesh": mesh, "vgrid": vg, "params": pr, "init": cs.smooth_state(mesh, 2, 0.1)}
    o, g = _pair(case, perturb=0.1)
    o.step(2)
    g.step(2)
    _compare(o, g, what="3d box")


def test_half_range_ties_on_axis_aligned_faces():
    """Odd velocity counts put a line of nodes on u.n = 0 at every face of a quad
    mesh: the half-range sums (direct and separable alike) give them half weight
    on both sides (Sec. 2.4) and their flux vanishes."""
    case = cs.cavity_case(n=8, nv=13, Kn=0.3, lid=0.3)
    o, g = _pair(case, perturb=0.1)
    o.step(3)
    g.step(3)
    _compare(o, g, what="ties 2d")


def test_descending_velocity_axis():
    """A tensor grid whose last axis descends is still a tensor grid, but takes
    the direct half-range sums (the separable ones search an ascending axis)."""
    case = cs.cavity_case(n=6, nv=11, Kn=0.3, lid=0.3)
    nx = ny = 11
    u = case["vgrid"]["u"].reshape(ny, nx, 2)[::-1].reshape(-1, 2)
    w = case["vgrid"]["w"].reshape(ny, nx)[::-1].reshape(-1)
    case = dict(case, vgrid={"dim": 2, "u": np.ascontiguousarray(u), "w": np.ascontiguousarray(w),
                             "cart_n": [nx, ny, 0]})
    o, g = _pair(case, perturb=0.1)
    o.step(2)
    g.step(2)
    _compare(o, g, what="descending axis")


@pytest.mark.parametrize("precision", [_lib.FP64, _lib.FP32])
def test_wall_surface_quantities(precision):
    """p_w, sigma_w and q_w (Sec. 2.5) of the step against the oracle: the
    cavity with a moving lid, the Mach-3 cylinder and the sphere, two steps
    from a perturbed state.  Shear and heat flux are small differences of the
    one-sided fluxes, whose size is that of the pressure, so all three are
    compared relative to the largest pressure (heat flux: or its own largest
    value, if larger)."""
    tol = 1e-12 if precision == _lib.FP64 else 1e-5
    for case in (cs.cavity_case(n=10, nv=16, Kn=0.2, lid=0.3),
                 cs.cylinder_case(n_cells=900, nvx=16, nvy=14, mach=3.0),
                 cs.sphere_case(n_cells=1200, nv=8, vmax=7.0, mach=2.0)):
        o, g = _pair(case, precision=precision, perturb=0.05)
        o.step(2)
        g.step(2)
        face, p, sg, q = g.wall_quantities()
        po, so, qo = o.wall_quantities()
        assert np.array_equal(face, np.nonzero(np.asarray(case["mesh"]["face_type"]) == 1)[0])
        ps = np.abs(po).max()
        assert np.abs(p - po).max() <= tol * ps
        assert np.abs(sg - so).max() <= tol * ps
        assert np.abs(q - qo).max() <= tol * max(np.abs(qo).max(), ps)
        g.close()


def test_near_continuum_stiff_collision():
    """Kn = 1e-4: dt / tau is far above 1, so the time integrals take their
    closed forms and stage 2 is stiff."""
    case = cs.cavity_case(n=8, nv=12, Kn=1e-4, lid=0.3)
    o, g = _pair(case, perturb=0.1)
    o.step(3)
    g.step(3)
    _compare(o, g, what="near continuum")


def test_single_cell_between_walls():
    """One cell, four walls: no least-squares neighbours (zero slopes), a patch
    of one cell with an empty ring, walls of two temperatures."""
    mesh = cs.quad_mesh(1, 1, left=("wall", 0), right=("wall", 1), bottom=("wall", 0), top=("wall", 0))
    case = {"mesh": mesh, "vgrid": cs.cartesian_vgrid((12, 12), (-5, -5), (5, 5)),
            "params": cs.params(0.5, walls=[{"T": 1.0, "U": [0, 0, 0]}, {"T": 1.5, "U": [0, 0.2, 0]}]),
            "init": cs.uniform_state(1, 2)}
    o, g = _pair(case, perturb=0.1)
    o.step(4)
    g.step(4)
    _compare(o, g, what="single cell")


def test_velocity_set_smaller_than_a_tile():
    """25 velocities in a tile of 64: 39 padding velocities (u = 0, w = 0)."""
    case = cs.cylinder_case(n_cells=700, nvx=5, nvy=5, mach=0.5, vx=(-5, 5), vy=(-5, 5))
    o, g = _pair(case, perturb=0.05, vtile=64)
    o.step(2)
    g.step(2)
    _compare(o, g, what="25 velocities")


def test_explicit_time_step():
    """A caller-given dt replaces the CFL step on both sides."""
    case = cs.cylinder_case(n_cells=900, nvx=14, nvy=12, mach=2.0)
    pr = dict(case["params"], dt=1e-3)
    o, g = _pair(case, params=pr, perturb=0.05)
    assert g.info()["dt"] == 1e-3 == o.dt
    o.step(2)
    g.step(2)
    _compare(o, g, what="explicit dt")


def test_fp32_storage_form_sphere_100_steps():
    """The FP32-storage form in 3D (one stored component), 100 steps: W within
    1e-5 (relative L2) of the FP64 oracle."""
    case = cs.sphere_case(n_cells=1200, nv=8, vmax=7.0, mach=2.0)
    o, g = _pair(case, precision=_lib.FP32, perturb=0.05)
    o.step(100)
    g.step(100)
    _, Wo, _ = o.state()
    _, Wg = g.state(with_f=False)
    assert _rel_l2(Wg, Wo) <= 1e-5


def _merge_pairs(mesh, frac, seed):
    """A mixed mesh: a seeded share of interior faces is removed and the two
    triangles on either side merged into one quadrilateral (volume-weighted
    centroid), so cells have 3 or 4 faces."""
    rng = np.random.default_rng(seed)
    fc = np.asarray(mesh["face_cells"]).copy()
    ft = np.asarray(mesh["face_type"])
    C = len(mesh["cell_vol"])
    taken = np.zeros(C, bool)
    drop = []
    for f in rng.permutation(np.nonzero(ft == 0)[0]):
        a, b = fc[f]
        if not taken[a] and not taken[b] and len(drop) < frac * C / 2:
            taken[a] = taken[b] = True
            drop.append(f)
    into = np.arange(C)
    vol = np.asarray(mesh["cell_vol"]).copy()
    xc = np.asarray(mesh["cell_xc"]).copy()
    for f in drop:
        a, b = fc[f]
        xc[a] = (vol[a] * xc[a] + vol[b] * xc[b]) / (vol[a] + vol[b])
        vol[a] += vol[b]
        into[b] = a
    keep_cells = np.nonzero(into == np.arange(C))[0]
    new_id = -np.ones(C, np.int64)
    new_id[keep_cells] = np.arange(len(keep_cells))
    keep_f = np.ones(len(ft), bool)
    keep_f[drop] = False
    nfc = fc[keep_f]
    nfc = np.stack([new_id[into[nfc[:, 0]]], np.where(nfc[:, 1] >= 0, new_id[into[np.maximum(nfc[:, 1], 0)]], -1)], 1)
    out = dict(mesh, cell_xc=xc[keep_cells], cell_vol=vol[keep_cells], face_cells=nfc)
    for k in ("face_n", "face_S", "face_xc", "face_type", "face_tag", "face_shift"):
        out[k] = np.ascontiguousarray(np.asarray(mesh[k])[keep_f])
    return out


def test_mixed_triangles_and_quadrilaterals():
    """Cells with 3 and 4 faces in one mesh (face counts vary within a patch
    and its ring)."""
    case = cs.cylinder_case(n_cells=900, nvx=14, nvy=12, mach=2.0)
    mesh = _merge_pairs(case["mesh"], 0.4, 3)
    nf = np.bincount(np.concatenate([mesh["face_cells"][:, 0], mesh["face_cells"][mesh["face_cells"][:, 1] >= 0, 1]]))
    assert set(np.unique(nf)) == {3, 4}
    case = dict(case, mesh=mesh, init=cs.blended_start(mesh, [cs.freestream_speed(2.0), 0.0]))
    for precision, tol in ((_lib.FP64, TOL64), (_lib.FP32, None)):
        o, g = _pair(case, precision=precision, perturb=0.05)
        o.step(2)
        g.step(2)
        if tol:
            _compare(o, g, what="mixed mesh")
        else:
            _, Wo, _ = o.state()
            _, Wg = g.state(with_f=False)
            assert _rel_l2(Wg, Wo) <= 1e-5


@pytest.mark.parametrize("precision", [_lib.FP64, _lib.FP32])
def test_analytic_w0_variant(precision):
    """The analytic-W0 variant (W0 from the erfc half-range moments of the
    face-state Maxwellians) against the oracle run with the same option."""
    for case in (cs.cavity_case(n=10, nv=16, Kn=0.2, lid=0.3),
                 cs.cylinder_case(n_cells=1200, nvx=16, nvy=14, mach=3.0),
                 cs.sphere_case(n_cells=1500, nv=8, vmax=7.0, mach=2.0)):
        pr = dict(case["params"], w0_analytic=1)
        o, g = _pair(case, precision=precision, params=pr, perturb=0.05)
        steps = 2 if precision == _lib.FP64 else 100
        o.step(steps)
        g.step(steps)
        if precision == _lib.FP64:
            _compare(o, g, what="analytic W0")
        else:
            _, Wo, _ = o.state()
            _, Wg = g.state(with_f=False)
            assert _rel_l2(Wg, Wo) <= 1e-5
        g.close()


def test_3d_sphere_tetrahedra():
    case = cs.sphere_case(n_cells=3000, nv=8, vmax=8.0, mach=2.0)
    o, g = _pair(case, perturb=0.05)
    o.step(1)
    g.step(1)
    _compare(o, g, what="sphere")


@pytest.mark.parametrize("variant", ["free_molecular", "no_limiter", "bgk"])
def test_limits_and_options(variant):
    case = cs.cylinder_case(n_cells=1200, nvx=16, nvy=14, mach=3.0)
    pr = dict(case["params"])
    if variant == "free_molecular":
        pr["Kn"] = float("inf")
    elif variant == "no_limiter":
        pr["limiter"] = 0
    else:
        pr["Pr"] = 1.0
    o, g = _pair(case, params=pr, perturb=0.05)
    o.step(2)
    g.step(2)
    _compare(o, g, what=variant)


@pytest.mark.parametrize("patch,vtile,group", [(4, 32, 1), (17, 64, 3), (64, 128, 1), (200, 32, 4), (24, 32, 64)])
def test_tiling_does_not_change_results(patch, vtile, group):
    """Patch size, velocity tile and the grid's tile groups (5 tiles in groups
    of 3 and 10 in groups of 4 end with a partial group; 64 is clamped to one
    group of all tiles) leave the FP64 step at the oracle's values."""
    case = cs.cylinder_case(n_cells=1500, nvx=18, nvy=15, mach=4.0)
    o, g = _pair(case, perturb=0.05, patch_cells=patch, vtile=vtile, tile_group=group)
    info = g.info()
    assert info["patch_cells"] <= patch and info["vtile"] == vtile
    assert info["gather_tile_group"] == min(group, info["nv_pad"] // vtile)
    o.step(1)
    g.step(1)
    _compare(o, g, what=f"tiling {patch}/{vtile}")


@pytest.mark.parametrize("patch,vtile,threads", [(32, 32, 512), (48, 64, 512), (40, 64, 256)])
def test_fp32_gather_block_sizes(patch, vtile, threads):
    """The FP32 gather with 256- and 512-thread CTAs (one, two or four
    velocities per lane) against the oracle: one step from an
    FP32-representable perturbed state, 1e-5 of max |f| per element."""
    case = cs.cylinder_case(n_cells=1500, nvx=18, nvy=15, mach=4.0)
    o, g = _pair(case, precision=_lib.FP32, perturb=0.05, patch_cells=patch, vtile=vtile, threads=threads)
    f0, W0, _ = o.state()
    f0 = f0.astype(np.float32).astype(np.float64)
    o.set_state(f0, W0)
    g.set_state(f0, W0)
    info = g.info()
    assert info["gather_threads"] == threads and info["vtile"] == vtile
    o.step(1)
    g.step(1)
    fo, Wo, _ = o.state()
    fg, Wg = g.state()
    assert _rel_max(fg, fo) <= 1e-5 and _rel_max(Wg, Wo) <= 1e-5, (_rel_max(fg, fo), _rel_max(Wg, Wo))


def test_runs_are_bitwise_deterministic():
    case = cs.cylinder_case(n_cells=1500, nvx=16, nvy=14)
    outs = []
    for _ in range(2):
        g = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=_lib.FP32)
        g.step(5)
        outs.append(g.state())
        g.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_fp32_storage_form_cavity_100_steps():
    case = cs.cavity_case()
    o = oracle.OracleCase(case["mesh"], case["vgrid"], case["params"], case["init"])
    g = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=_lib.FP32)
    o.step(100)
    g.step(100)
    fo, Wo, qo = o.state()
    fg, Wg = g.state()
    eW = _rel_l2(Wg, Wo)
    ef = _rel_l2(fg, fo)
    # the velocity field is what changes: its error relative to its own size
    U_o = Wo[:, 1:3] / Wo[:, :1]
    U_g = Wg[:, 1:3] / Wg[:, :1]
    eU = _rel_l2(U_g, U_o)
    print(f"fp32 cavity 100 steps: W {eW:.2e} f {ef:.2e} U {eU:.2e}")
    assert eW <= 1e-5 and ef <= 1e-5 and eU <= 1e-4


def test_fp32_storage_form_converged_cavity():
    """The lid-driven cavity (20 x 20 quadrilaterals, 24^2 velocities, Kn 0.075)
    run to its steady state: 2,400 steps bring the residual below 1e-7 (it
    falls about 3.3 times per 250 steps).  The converged fields of the
    FP32-storage form (W, the velocity and the heat flux, each against its
    own largest magnitude) match the FP64 oracle's to 1e-4."""
    case = cs.cavity_case()
    o = oracle.OracleCase(case["mesh"], case["vgrid"], case["params"], case["init"], n_threads=0)
    g = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=_lib.FP32)
    o.step(2400)
    g.step(2400)
    ro, rg = np.max(o.residual()), np.max(g.residual())
    assert ro < 1e-6 and rg < 1e-6, (ro, rg)
    _, Wo, qo = o.state()
    _, Wg = g.state(with_f=False)
    qg = g.heat_flux()
    Uo, Ug = Wo[:, 1:3] / Wo[:, :1], Wg[:, 1:3] / Wg[:, :1]
    errs = {"W": _rel_max(Wg, Wo), "U": _rel_max(Ug, Uo), "q": _rel_max(qg, qo)}
    print(f"fp32 converged cavity: residual {rg:.1e}, " + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert max(errs.values()) <= 1e-4, errs


def test_fp32_storage_form_cylinder_100_steps():
    case = cs.cylinder_case(n_cells=2000, nvx=30, nvy=25, start="impulsive")
    o = oracle.OracleCase(case["mesh"], case["vgrid"], case["params"], case["init"])
    g = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=_lib.FP32)
    o.step(100)
    g.step(100)
    _, Wo, _ = o.state()
    _, Wg = g.state()
    eW = _rel_l2(Wg, Wo)
    print(f"fp32 cylinder 100 steps: W {eW:.2e}")
    assert eW <= 1e-5


def test_numeric_failure_is_reported():
    case = cs.cavity_case(n=4, nv=8)
    g = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"])
    _, W = g.state(with_f=False)
    W[2, 3] = -1.0                                    # negative energy
    g.set_state(None, W)
    with pytest.raises(_lib.UGKSError) as e:
        g.check()
    assert e.value.code == 4


def test_full_size_cylinder_one_step_fp64():
    """The 30k-cell x 60x50 cylinder at full size, FP64, one step from a
    perturbed state: every element against the oracle."""
    case = cs.cylinder_case()
    o, g = _pair(case, perturb=0.05)
    o.step(1)
    g.step(1)
    _compare(o, g, what="cylinder full size")


def test_full_size_mach5_fp32_stays_physical():
    """The 30k-cell Mach-5 cylinder (blended start), FP32 form, 600 steps: the
    state stays finite with positive density and temperature."""
    case = cs.cylinder_case()
    g = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=_lib.FP32)
    for _ in range(6):
        g.step(100)
        g.check()
    rho, U, T, q = g.moments()
    assert rho.min() > 0 and T.min() > 0 and np.isfinite(q).all()


@pytest.mark.parametrize("D", [2, 3])
def test_unstructured_velocity_set(D, precision=_lib.FP64):
    """A non-tensor discrete velocity set (jittered points, arbitrary positive
    weights, shuffled order) takes the general per-velocity face sums."""
    rng = np.random.default_rng(21)
    if D == 2:
        vg = cs.cartesian_vgrid((17, 15), (-6, -5), (6, 5))
        case = cs.cylinder_case(n_cells=900, nvx=4, nvy=4, mach=2.0)
    else:
        vg = cs.cartesian_vgrid((9, 8, 8), (-5, -5, -5), (5, 5, 5))
        case = cs.sphere_case(n_cells=1500, nv=4, vmax=5.0, mach=1.5)
    perm = rng.permutation(len(vg["w"]))
    u = vg["u"][perm] + rng.uniform(-0.15, 0.15, size=vg["u"].shape)
    w = vg["w"][perm] * rng.uniform(0.8, 1.2, size=len(perm))
    vgu = {"dim": D, "u": u, "w": w, "cart_n": [0, 0, 0]}
    case = dict(case, vgrid=vgu)
    o, g = _pair(case, precision=precision, perturb=0.05)
    if precision == _lib.FP32:
        f0, W0, _ = o.state()
        f0 = f0.astype(np.float32).astype(np.float64)
        o.set_state(f0, W0)
        g.set_state(f0, W0)
    o.step(2)
    g.step(2)
    if precision == _lib.FP64:
        _compare(o, g, what=f"unstructured DVS {D}D")
        return
    fo, Wo, _ = o.state()
    fg, Wg = g.state()
    ef, eW = _rel_max(fg, fo), _rel_max(Wg, Wo)
    print(f"fp32 unstructured DVS {D}D, 2 steps: f {ef:.2e} W {eW:.2e}")
    assert ef <= 1e-5 and eW <= 1e-5


@pytest.mark.parametrize("D", [2, 3])
def test_unstructured_velocity_set_fp32(D):
    """The same in the FP32-storage form: FP32 monomial sums of the face
    equilibrium, FP64 assembly; 1e-5 of max |x| after two steps."""
    test_unstructured_velocity_set(D, precision=_lib.FP32)
