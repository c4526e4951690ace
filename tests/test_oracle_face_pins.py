"""Pins of the oracle's macroscopic face states (the macroscopic reconstruction
step of Algorithm 1, Sec. 2.4) and of its far-field ghost rule (Sec. 2.5).

Each check compares the oracle with a fact it does not compute itself:
linear primitive fields are reproduced exactly at face centres by a
least-squares reconstruction; on a uniform periodic grid the face states of a
field shifted by one cell are the shifted face states (translation invariance,
which holds across the periodic seam only if the seam's image shift is right);
a reconstruction that would give a non-positive density falls back to the cell
average; the ghost state is the free stream exactly on inflow faces and the
owner's state elsewhere; and in the free-molecular limit the flux of particles
entering through a far-field face is the closed-form flux of the ghost's
Maxwellian, which a velocity set of one sign isolates.
"""
import numpy as np
import pytest

import oracle
from paper_2412_06546_gb300 import cases as cs


def _cons(P, D):
    """Conserved variables of primitive states P[..., (rho, U, T)]: rho,
    rho U, rho (|U|^2/2 + 3T/2) for a monatomic gas with R = 1."""
    P = np.asarray(P, float)
    rho, U, T = P[..., 0], P[..., 1:1 + D], P[..., D + 1]
    W = np.empty(P.shape)
    W[..., 0] = rho
    W[..., 1:1 + D] = rho[..., None] * U
    W[..., D + 1] = rho * (0.5 * np.sum(U * U, axis=-1) + 1.5 * T)
    return W


def _walls_only(mesh):
    """The mesh with every boundary face made a wall (tag 0): the
    reconstruction then uses cell values only."""
    m = dict(mesh)
    ft = np.array(mesh["face_type"], copy=True)
    ft[ft == cs.FARFIELD] = cs.WALL
    m["face_type"] = ft
    m["face_tag"] = np.zeros_like(mesh["face_tag"])
    return m


def _mesh(D):
    if D == 2:
        return _walls_only(cs.cylinder_mesh(1500, seed=2))
    return _walls_only(cs.sphere_mesh(2500, seed=3))


def _vgrid(D):
    return cs.cartesian_vgrid((8,) * D, (-5.0,) * D, (5.0,) * D)


def _interior_neighbours(mesh):
    C = len(mesh["cell_vol"])
    fc, ft = mesh["face_cells"], mesh["face_type"]
    inner = ft == cs.INTERIOR
    cnt = np.zeros(C, int)
    np.add.at(cnt, fc[inner, 0], 1)
    np.add.at(cnt, fc[inner, 1], 1)
    return cnt


@pytest.mark.parametrize("D", [2, 3])
def test_face_states_reproduce_linear_primitive_fields(D):
    """Limiter off, linear rho, U, T: both face states of every interior face
    are the field's value at the face centre (a sign error in x_f - x_i, or a
    reconstruction from the other cell's centre, breaks this)."""
    mesh = _mesh(D)
    x = mesh["cell_xc"]
    rng = np.random.default_rng(5 + D)
    A = rng.uniform(-0.02, 0.02, size=(D + 2, D))
    p0 = np.array([1.0] + [0.3, -0.2, 0.1][:D] + [1.0])
    prim = p0 + x @ A.T
    assert prim[:, 0].min() > 0.5 and prim[:, D + 1].min() > 0.5
    pr = cs.params(0.1, limiter=0, walls=[{"T": 1.0, "U": [0, 0, 0]}])
    o = oracle.OracleCase(mesh, _vgrid(D), pr, prim)
    o.step(1)
    WL, WR = o.face_states()
    fc, ft = mesh["face_cells"], mesh["face_type"]
    nb = _interior_neighbours(mesh)
    sel = (ft == cs.INTERIOR) & (nb[fc[:, 0]] >= D) & (nb[np.maximum(fc[:, 1], 0)] >= D)
    assert sel.sum() > 0.9 * (ft == cs.INTERIOR).sum()
    ref = _cons(p0 + mesh["face_xc"] @ A.T, D)
    scale = np.abs(ref).max(axis=0)
    assert np.abs(WL[sel] - ref[sel]).max(axis=0).max() <= 1e-12 * scale.max()
    assert (np.abs(WL[sel] - ref[sel]) <= 1e-12 * scale).all()
    assert (np.abs(WR[sel] - ref[sel]) <= 1e-12 * scale).all()


def test_face_states_are_the_extrapolations_of_each_side():
    """Limiter off, quadratic data (gradients differ from cell to cell): W_L
    is cell i's primitive state extrapolated with cell i's least-squares
    gradient (pinned separately, test_least_squares_exact_on_linear_fields) to
    the face centre, and W_R the same from cell j, so that swapping the sides'
    gradients or centres shows."""
    D = 2
    mesh = _mesh(D)
    x = mesh["cell_xc"]
    r2 = np.sum((x - np.array([4.0, -3.0])) ** 2, axis=1)
    prim = np.stack([1.0 + 0.002 * r2, 0.2 + 0.001 * x[:, 0] * x[:, 1], -0.1 + 0.0005 * r2,
                     1.0 + 0.001 * x[:, 1] ** 2], axis=1)
    pr = cs.params(0.1, limiter=0, walls=[{"T": 1.0, "U": [0, 0, 0]}])
    o = oracle.OracleCase(mesh, _vgrid(D), pr, prim)
    grads = np.stack([o.scalar_gradient(prim[:, m], None, limited=False) for m in range(D + 2)], axis=1)
    o.step(1)
    WL, WR = o.face_states()
    fc, ft, fx = mesh["face_cells"], mesh["face_type"], mesh["face_xc"]
    sel = np.nonzero(ft == cs.INTERIOR)[0]
    i, j = fc[sel, 0], fc[sel, 1]
    PL = prim[i] + np.einsum("fmd,fd->fm", grads[i], fx[sel] - x[i])
    PR = prim[j] + np.einsum("fmd,fd->fm", grads[j], fx[sel] - x[j])
    scale = np.abs(_cons(prim, D)).max()
    assert np.abs(WL[sel] - _cons(PL, D)).max() <= 1e-12 * scale
    assert np.abs(WR[sel] - _cons(PR, D)).max() <= 1e-12 * scale
    # the two sides genuinely differ here, so a swap would be seen
    assert np.abs(_cons(PL, D) - _cons(PR, D)).max() > 1e-6 * scale


def test_face_states_are_translation_invariant_across_a_periodic_seam():
    """Uniform doubly periodic quads, smooth periodic data, limiter on: the
    face states of the data rolled by one cell along x are the face states of
    the original data one cell to the left, on the faces of the periodic seam
    as well (a wrong or missing image shift in the reconstruction breaks it)."""
    nx, ny = 8, 5
    lx, ly = 1.0, 0.7
    mesh = cs.quad_mesh(nx, ny, lx, ly, left="periodic", right="periodic", bottom="periodic", top="periodic")
    x = mesh["cell_xc"]
    D = 2
    kx, ky = 2 * np.pi / lx, 2 * np.pi / ly
    prim = np.stack([1.0 + 0.3 * np.sin(kx * x[:, 0] + 0.4) * np.cos(ky * x[:, 1]),
                     0.2 + 0.1 * np.cos(kx * x[:, 0] - 0.3),
                     -0.1 + 0.15 * np.sin(ky * x[:, 1] + kx * x[:, 0]),
                     1.0 + 0.2 * np.cos(kx * x[:, 0] + 1.1) * np.sin(ky * x[:, 1] + 0.2)], axis=1)
    ix = np.rint(x[:, 0] / (lx / nx) - 0.5).astype(int)
    iy = np.rint(x[:, 1] / (ly / ny) - 0.5).astype(int)
    cell_of = np.full((nx, ny), -1)
    cell_of[ix, iy] = np.arange(len(x))
    rolled = prim[cell_of[(ix - 1) % nx, iy]]          # value of the cell one to the left
    pr = cs.params(0.1, limiter=1, walls=[])
    states = []
    for p in (prim, rolled):
        o = oracle.OracleCase(mesh, _vgrid(D), pr, p)
        o.step(1)
        states.append(o.face_states())
    fc, fn = mesh["face_cells"], mesh["face_n"]
    # the face on the +x (resp. +y) side of each cell: owner = the cell, normal +e_d
    face_at = {}
    for f in range(len(fc)):
        d = int(np.argmax(np.abs(fn[f])))
        assert fn[f, d] == 1.0
        face_at[(d, ix[fc[f, 0]], iy[fc[f, 0]])] = f
    seam = mesh["face_type"] == cs.PERIODIC
    assert seam.sum() == nx + ny
    scale = np.abs(_cons(prim, D)).max()
    for (d, a, b), f in face_at.items():
        g = face_at[(d, (a - 1) % nx, b)]
        for side in (0, 1):
            assert np.abs(states[1][side][f] - states[0][side][g]).max() <= 1e-13 * scale, (d, a, b, side)


def test_non_positive_reconstruction_falls_back_to_the_cell_average():
    """A density spike with the limiter off: next to it the least-squares
    extrapolation gives negative densities at some faces; those face states
    are the cell's own average, all others are extrapolated."""
    D = 2
    mesh = _mesh(D)
    x = mesh["cell_xc"]
    C = len(x)
    prim = cs.uniform_state(C, D, rho=1.0, U=[0.1, 0.0], T=1.0)
    spike = int(np.argmin(np.sum((x - np.array([3.0, 2.0])) ** 2, axis=1)))
    prim[spike, 0] = 60.0
    pr = cs.params(0.1, limiter=0, walls=[{"T": 1.0, "U": [0, 0, 0]}])
    o = oracle.OracleCase(mesh, _vgrid(D), pr, prim)
    g_rho = o.scalar_gradient(prim[:, 0], None, limited=False)
    o.step(1)
    WL, _ = o.face_states()
    fc, ft, fx = mesh["face_cells"], mesh["face_type"], mesh["face_xc"]
    sel = np.nonzero(ft == cs.INTERIOR)[0]
    i = fc[sel, 0]
    rho_ext = prim[i, 0] + np.sum(g_rho[i] * (fx[sel] - x[i]), axis=1)
    neg = rho_ext <= 0.0
    assert neg.sum() >= 1
    Wc = _cons(prim, D)
    assert np.abs(WL[sel[neg]] - Wc[i[neg]]).max() <= 1e-14 * np.abs(Wc).max()
    assert np.abs(WL[sel[~neg], 0] - rho_ext[~neg]).max() <= 1e-12 * 60.0


def _farfield_box(vg, inf_U, prim, Kn=0.1, limiter=1):
    mesh = cs.quad_mesh(6, 5, 1.0, 0.8, left="farfield", right="farfield", bottom="farfield", top="farfield")
    pr = cs.params(Kn, limiter=limiter, walls=[], inf={"rho": 1.0, "U": list(inf_U) + [0.0], "T": 1.0})
    if callable(prim):
        prim = prim(mesh)
    return mesh, oracle.OracleCase(mesh, vg, pr, prim)


def test_far_field_ghost_is_the_free_stream_on_inflow_faces_only():
    """Ghost state (W_R of far-field faces) on a box with far-field faces only
    and a non-uniform interior: W_inf exactly where U_inf . n < 0, the owner's
    W^n exactly where U_inf . n > 0 and where U_inf . n = 0."""
    D = 2
    vg = _vgrid(D)
    for inf_U in ([0.7, -0.3], [0.7, 0.0], [-0.4, 0.9]):
        mesh, o = _farfield_box(vg, inf_U, lambda m: cs.smooth_state(m, 3, amp=0.2, U0=[0.1, -0.05]))
        _, Wn, _ = o.state()
        o.step(1)
        _, WR = o.face_states()
        fc, fn = mesh["face_cells"], mesh["face_n"]
        un = fn @ np.asarray(inf_U)
        W_inf = _cons(np.array([1.0] + list(inf_U) + [1.0]), D)
        far = mesh["face_type"] == cs.FARFIELD
        inflow, other = far & (un < 0), far & (un >= 0)
        assert inflow.any() and other.any()
        assert (WR[inflow] == W_inf).all()
        assert (WR[other] == Wn[fc[other, 0]]).all()


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_far_field_entering_flux_is_the_ghost_maxwellian_free_molecular(sign):
    """Kn = infinity, velocities all moving in +x (sign = 1) or all in -x
    (sign = -1), interior gas (rho 2, U 0.1, T 1.5) unlike the free stream
    (rho 1, U 0.5, T 1): at the face every particle crosses into the domain
    through (the x- faces for +x, the x+ faces for -x) the flux over the step
    is dt sum_k w_k psi_k (u_k . n) H_ghost(u_k) with H_ghost the Maxwellian of
    the free stream on the inflow x- face and of the cell on the outflow x+
    face (the two branches of the ghost rule, told apart by their states)."""
    D = 2
    ux = np.linspace(0.25, 6.0, 24) * sign
    uy = np.linspace(-5.0, 5.0, 21)
    U = np.array([[a, b] for b in uy for a in ux])
    w = np.full(len(U), abs(ux[1] - ux[0]) * (uy[1] - uy[0]))
    vg = {"dim": 2, "u": U, "w": w, "cart_n": [0, 0, 0]}
    prim_in = np.array([2.0, 0.1, 0.0, 1.5])
    mesh, o = _farfield_box(vg, [0.5, 0.0], lambda m: np.tile(prim_in, (len(m["cell_vol"]), 1)),
                            Kn=float("inf"), limiter=0)
    o.step(1)
    F = o.face_macro_flux()
    dt = o.dt
    fn = mesh["face_n"]
    ent = (fn[:, 0] == -sign) & (mesh["face_type"] == cs.FARFIELD)
    assert ent.sum() == 5
    ghost = np.array([1.0, 0.5, 0.0, 1.0]) if sign > 0 else prim_in
    rho, Ug, T = ghost[0], ghost[1:3], ghost[3]
    H = rho / (2 * np.pi * T) * np.exp(-np.sum((U - Ug) ** 2, axis=1) / (2 * T))
    B = T * H                                   # one internal translational degree of freedom in 2D
    un = U @ fn[np.nonzero(ent)[0][0]]
    assert (un < 0).all()
    Fh, Fb = dt * un * H, dt * un * B
    ref = np.array([np.sum(w * Fh), np.sum(w * U[:, 0] * Fh), np.sum(w * U[:, 1] * Fh),
                    np.sum(w * 0.5 * (np.sum(U * U, axis=1) * Fh + Fb))])
    assert np.abs(F[ent] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_uniform_free_stream_stays_stationary_in_a_far_field_box():
    """The free stream everywhere, far-field faces only, on a velocity grid
    symmetric about U_inf: every face carries the same interface distribution,
    so nothing changes."""
    D = 2
    vg = cs.cartesian_vgrid((27, 25), (0.5 - 6.5, -6.0), (0.5 + 6.5, 6.0))
    mesh, o = _farfield_box(vg, [0.5, 0.0], lambda m: cs.uniform_state(len(m["cell_vol"]), 2, U=[0.5, 0.0]))
    f0, W0, _ = o.state()
    o.step(5)
    f5, W5, _ = o.state()
    assert np.abs(W5 - W0).max() <= 1e-13 * np.abs(W0).max()
    assert np.abs(f5 - f0).max() <= 1e-13 * np.abs(f0).max()
