"""Seeded synthetic inputs: physical meshes, discrete velocity grids and case set-ups.

This module builds the *inputs* of a UGKS run and nothing else: face-list meshes
(centroids, volumes, face normals, areas, centres, boundary types), Cartesian
discrete velocity grids with trapezoid weights, and the parameter records of the
workloads.  It holds none of the scheme's arithmetic (no Maxwellians, fluxes,
slopes or collision terms), so the CPU oracle and the CUDA library can both take
their inputs from here without sharing any of the method.

Mesh convention (all arrays numpy, float64 / int64 / int32):

* ``cell_xc[C][D]``, ``cell_vol[C]``
* ``face_cells[F][2]``: owner, neighbour (``-1`` on wall / far-field faces)
* ``face_n[F][D]``: unit normal pointing from the owner to the neighbour (outward
  on boundary faces)
* ``face_S[F]``, ``face_xc[F][D]`` (the face centre as seen from the owner)
* ``face_type[F]``: ``INTERIOR``, ``WALL``, ``FARFIELD`` or ``PERIODIC``
* ``face_tag[F]``: wall index for ``WALL`` faces, else 0
* ``face_shift[F][D]``: for ``PERIODIC`` faces the vector added to the
  neighbour centroid to bring its image next to the owner (zero elsewhere).

The boundary conditions follow Sec. 2.5 of the paper (ghost far field, Maxwell
isothermal walls); periodic faces are an addition used by the conservation tests.
"""
from __future__ import annotations

import math
import numpy as np

INTERIOR, WALL, FARFIELD, PERIODIC = 0, 1, 2, 3


# ----------------------------------------------------------------------------
# discrete velocity space (Sec. 2.3: integral over velocity = sum Q_k V_k)
# ----------------------------------------------------------------------------
def cartesian_vgrid(n, lo, hi):
    """Tensor-product velocity grid with trapezoid weights.

    ``n``, ``lo``, ``hi`` are per-dimension sequences.  Velocities are ordered
    with the first axis fastest: ``k = ix + nx*(iy + ny*iz)``.  Returns a dict
    with ``u[Nv][D]``, ``w[Nv]`` (the cell volumes V_k of Sec. 2.3) and ``cart_n``.
    """
    n = [int(v) for v in n]
    D = len(n)
    axes, weights = [], []
    for d in range(D):
        x = np.linspace(lo[d], hi[d], n[d])
        h = (hi[d] - lo[d]) / (n[d] - 1)
        wd = np.full(n[d], h)
        wd[0] = wd[-1] = 0.5 * h
        axes.append(x)
        weights.append(wd)
    grids = np.meshgrid(*axes, indexing="ij")          # grids[d][i0, i1, ...]
    wgrid = np.ones_like(grids[0])
    for d in range(D):
        shape = [1] * D
        shape[d] = n[d]
        wgrid = wgrid * weights[d].reshape(shape)
    # order with axis 0 fastest -> transpose to Fortran order
    u = np.stack([g.ravel(order="F") for g in grids], axis=1)
    w = wgrid.ravel(order="F")
    cart = n + [0] * (3 - D)
    return {"dim": D, "u": np.ascontiguousarray(u), "w": np.ascontiguousarray(w),
            "cart_n": cart}


# ----------------------------------------------------------------------------
# structured meshes stored as unstructured face lists
# ----------------------------------------------------------------------------
def _bc(spec):
    if spec is None:
        return ("wall", 0)
    if isinstance(spec, str):
        return (spec, 0)
    return tuple(spec)


def quad_mesh(nx, ny, lx=1.0, ly=1.0, left="wall", right="wall", bottom="wall",
              top=("wall", 1)):
    """``nx x ny`` rectangles on ``[0,lx] x [0,ly]`` as a face list.

    Each side takes ``("wall", tag)``, ``"farfield"`` or ``"periodic"`` (periodic
    must be given on both opposite sides).
    """
    return box_mesh((nx, ny), (lx, ly), {"x-": left, "x+": right, "y-": bottom, "y+": top})


def hex_mesh(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, sides=None):
    """``nx x ny x nz`` boxes on ``[0,lx]x[0,ly]x[0,lz]``; ``sides`` maps
    ``x-, x+, y-, y+, z-, z+`` to a boundary spec (default: walls, tag 0)."""
    sides = dict(sides or {})
    return box_mesh((nx, ny, nz), (lx, ly, lz), sides)


def box_mesh(ns, ls, sides):
    D = len(ns)
    ns = [int(v) for v in ns]
    hs = [ls[d] / ns[d] for d in range(D)]
    C = int(np.prod(ns))
    idx = np.arange(C).reshape(ns[::-1]).transpose()   # idx[i0, i1, ...], axis0 fastest
    centers = np.meshgrid(*[(np.arange(ns[d]) + 0.5) * hs[d] for d in range(D)], indexing="ij")
    cell_xc = np.zeros((C, D))
    for d in range(D):
        cell_xc[idx.ravel(), d] = centers[d].ravel()
    cell_vol = np.full(C, float(np.prod(hs)))
    names = ["x", "y", "z"]
    fc, fn, fS, fx, ft, ftag, fsh = [], [], [], [], [], [], []
    for d in range(D):
        area = float(np.prod([hs[e] for e in range(D) if e != d]))
        nvec = np.zeros(D)
        nvec[d] = 1.0
        lo = _bc(sides.get(names[d] + "-"))
        hi = _bc(sides.get(names[d] + "+"))
        periodic = lo[0] == "periodic" or hi[0] == "periodic"
        if periodic and not (lo[0] == "periodic" and hi[0] == "periodic"):
            raise ValueError("periodic must be set on both sides of an axis")
        # interior faces along axis d
        sl_own = [slice(None)] * D
        sl_nb = [slice(None)] * D
        sl_own[d] = slice(0, ns[d] - 1)
        sl_nb[d] = slice(1, ns[d])
        own = idx[tuple(sl_own)].ravel()
        nb = idx[tuple(sl_nb)].ravel()
        xf = cell_xc[own].copy()
        xf[:, d] += 0.5 * hs[d]
        fc.append(np.stack([own, nb], 1)); fn.append(np.tile(nvec, (len(own), 1)))
        fS.append(np.full(len(own), area)); fx.append(xf)
        ft.append(np.full(len(own), INTERIOR)); ftag.append(np.zeros(len(own), np.int64))
        fsh.append(np.zeros((len(own), D)))
        # boundary faces
        sl_first = [slice(None)] * D
        sl_last = [slice(None)] * D
        sl_first[d] = 0
        sl_last[d] = ns[d] - 1
        first = idx[tuple(sl_first)].ravel()
        last = idx[tuple(sl_last)].ravel()
        if periodic:
            xf = cell_xc[last].copy()
            xf[:, d] += 0.5 * hs[d]
            sh = np.zeros((len(last), D))
            sh[:, d] = ls[d]
            fc.append(np.stack([last, first], 1)); fn.append(np.tile(nvec, (len(last), 1)))
            fS.append(np.full(len(last), area)); fx.append(xf)
            ft.append(np.full(len(last), PERIODIC)); ftag.append(np.zeros(len(last), np.int64))
            fsh.append(sh)
        else:
            for cells, sgn, spec in ((first, -1.0, lo), (last, 1.0, hi)):
                xf = cell_xc[cells].copy()
                xf[:, d] += sgn * 0.5 * hs[d]
                typ = {"wall": WALL, "farfield": FARFIELD}[spec[0]]
                tag = int(spec[1]) if (spec[0] == "wall" and len(spec) > 1) else 0
                fc.append(np.stack([cells, -np.ones_like(cells)], 1))
                fn.append(np.tile(sgn * nvec, (len(cells), 1)))
                fS.append(np.full(len(cells), area)); fx.append(xf)
                ft.append(np.full(len(cells), typ)); ftag.append(np.full(len(cells), tag))
                fsh.append(np.zeros((len(cells), D)))
    return _pack(D, cell_xc, cell_vol, np.concatenate(fc), np.concatenate(fn),
                 np.concatenate(fS), np.concatenate(fx), np.concatenate(ft),
                 np.concatenate(ftag), np.concatenate(fsh))


def _pack(D, cell_xc, cell_vol, face_cells, face_n, face_S, face_xc, face_type, face_tag, face_shift):
    return {
        "dim": int(D),
        "cell_xc": np.ascontiguousarray(cell_xc, dtype=np.float64),
        "cell_vol": np.ascontiguousarray(cell_vol, dtype=np.float64),
        "face_cells": np.ascontiguousarray(face_cells, dtype=np.int64),
        "face_n": np.ascontiguousarray(face_n, dtype=np.float64),
        "face_S": np.ascontiguousarray(face_S, dtype=np.float64),
        "face_xc": np.ascontiguousarray(face_xc, dtype=np.float64),
        "face_type": np.ascontiguousarray(face_type, dtype=np.int32),
        "face_tag": np.ascontiguousarray(face_tag, dtype=np.int32),
        "face_shift": np.ascontiguousarray(face_shift, dtype=np.float64),
    }


# ----------------------------------------------------------------------------
# simplex meshes (triangles / tetrahedra) from a point cloud
# ----------------------------------------------------------------------------
def _simplex_geometry(points, simp):
    D = points.shape[1]
    P = points[simp]                                   # [C, D+1, D]
    xc = P.mean(axis=1)
    E = P[:, 1:, :] - P[:, :1, :]                      # [C, D, D]
    vol = np.abs(np.linalg.det(E)) / math.factorial(D)
    return xc, vol


def simplex_mesh(points, simp, classify=None, shifts=None):
    """Face list of a simplicial mesh.

    ``classify(face_xc) -> (type, tag)`` arrays label boundary faces.  ``shifts``
    (optional, periodic meshes) maps the unwrapped vertex positions: pass
    ``points`` already unwrapped per simplex as ``points[C][D+1][D]`` together with
    ``simp`` holding the *wrapped* vertex ids used to match faces.
    """
    if points.ndim == 3:
        P = points                                      # per-simplex unwrapped vertices
        D = P.shape[2]
    else:
        P = points[simp]
        D = points.shape[1]
    C = simp.shape[0]
    xc = P.mean(axis=1)
    E = P[:, 1:, :] - P[:, :1, :]
    vol = np.abs(np.linalg.det(E)) / math.factorial(D)
    nloc = D + 1
    # faces: omit local vertex m
    fv = []      # wrapped vertex ids, sorted
    fpos = []    # unwrapped vertex positions of the face in the owning simplex
    for m in range(nloc):
        keep = [v for v in range(nloc) if v != m]
        fv.append(simp[:, keep])
        fpos.append(P[:, keep, :])
    fv = np.stack(fv, 1).reshape(C * nloc, D)
    fpos = np.stack(fpos, 1).reshape(C * nloc, D, D)
    cell_of = np.repeat(np.arange(C), nloc)
    order = np.argsort(fv, axis=1)
    fv_sorted = np.take_along_axis(fv, order, axis=1)
    keys = np.ascontiguousarray(fv_sorted).view([("", fv_sorted.dtype)] * D).ravel()
    srt = np.argsort(keys, kind="stable")
    ks = keys[srt]
    same_next = np.zeros(len(ks), bool)
    same_next[:-1] = ks[:-1] == ks[1:]
    face_own, face_nb, face_pos_own, face_pos_nb = [], [], [], []
    i = 0
    n = len(ks)
    own_l, nb_l, pos_o, pos_n = [], [], [], []
    starts = np.ones(n, bool)
    starts[1:] = ks[1:] != ks[:-1]
    gid = np.cumsum(starts) - 1
    nf = gid[-1] + 1
    first = np.full(nf, -1, np.int64)
    second = np.full(nf, -1, np.int64)
    # first / second occurrence of each key
    occ0 = srt[starts]
    first[:] = occ0
    dup = ~starts
    second[gid[dup]] = srt[dup]
    owner = cell_of[first]
    nb = np.where(second >= 0, cell_of[np.maximum(second, 0)], -1)
    pos_o = fpos[first]                                # [F, D, D]
    fx = pos_o.mean(axis=1)
    if D == 2:
        t = pos_o[:, 1, :] - pos_o[:, 0, :]
        S = np.linalg.norm(t, axis=1)
        nrm = np.stack([t[:, 1], -t[:, 0]], 1) / S[:, None]
    else:
        cr = np.cross(pos_o[:, 1, :] - pos_o[:, 0, :], pos_o[:, 2, :] - pos_o[:, 0, :])
        S = 0.5 * np.linalg.norm(cr, axis=1)
        nrm = cr / (2.0 * S[:, None])
    sign = np.sign(np.einsum("fd,fd->f", fx - xc[owner], nrm))
    sign[sign == 0] = 1.0
    nrm = nrm * sign[:, None]
    ftype = np.full(nf, INTERIOR, np.int32)
    ftag = np.zeros(nf, np.int32)
    fshift = np.zeros((nf, D))
    has_nb = nb >= 0
    if points.ndim == 3:
        pos_n = fpos[np.maximum(second, 0)]
        fx_nb = pos_n.mean(axis=1)
        sh = fx - fx_nb
        per = has_nb & (np.abs(sh).max(axis=1) > 1e-12)
        ftype[per] = PERIODIC
        fshift[per] = sh[per]
    bnd = ~has_nb
    if bnd.any():
        if classify is None:
            raise ValueError("boundary faces present but no classifier given")
        typ, tag = classify(fx[bnd])
        ftype[bnd] = typ
        ftag[bnd] = tag
    face_cells = np.stack([owner, nb], 1)
    return _pack(D, xc, vol, face_cells, nrm, S, fx, ftype, ftag, fshift)


def periodic_tri_mesh(nx, ny, lx=1.0, ly=1.0, jitter=0.2, seed=0):
    """Doubly periodic triangulation of a jittered ``nx x ny`` lattice.

    Node ``(i, j)`` is displaced by a smooth periodic field of amplitude
    ``jitter`` cell widths (seeded), and each lattice square is cut along an
    alternating diagonal, so the cells are irregular triangles while every face
    still has a periodic partner.
    """
    rng = np.random.default_rng(seed)
    dx, dy = lx / nx, ly / ny
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, size=4)
    ax = jitter * dx * (0.6 * np.sin(2 * np.pi * ii / nx + ph[0]) * np.cos(2 * np.pi * jj / ny + ph[1])
                        + 0.4 * np.sin(4 * np.pi * (ii / nx + jj / ny) + ph[2]))
    ay = jitter * dy * (0.6 * np.cos(2 * np.pi * ii / nx + ph[2]) * np.sin(2 * np.pi * jj / ny + ph[3])
                        + 0.4 * np.sin(2 * np.pi * (2 * ii / nx - jj / ny) + ph[0]))
    X = ii * dx + ax
    Y = jj * dy + ay

    def node(i, j):
        return (i % nx) * ny + (j % ny)

    def pos(i, j):
        return np.array([X[i % nx, j % ny] + (i // nx) * lx, Y[i % nx, j % ny] + (j // ny) * ly])

    simp, P = [], []
    for i in range(nx):
        for j in range(ny):
            quad = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
            if (i + j) % 2 == 0:
                tris = [(0, 1, 2), (0, 2, 3)]
            else:
                tris = [(0, 1, 3), (1, 2, 3)]
            for t in tris:
                vs = [quad[a] for a in t]
                simp.append([node(*v) for v in vs])
                P.append([pos(*v) for v in vs])
    return simplex_mesh(np.array(P), np.array(simp, np.int64))


def _geometric_layers(r0, r1, h0, ratio):
    rs = [r0]
    h = h0
    while rs[-1] + h < r1 - 0.5 * h:
        rs.append(rs[-1] + h)
        h *= ratio
    rs.append(r1)
    return np.array(rs)


def _annulus_points(h0, rng, r_in, r_out, ratio):
    rs = _geometric_layers(r_in, r_out, h0, ratio)
    pts = []
    for l, r in enumerate(rs):
        hl = rs[min(l + 1, len(rs) - 1)] - rs[max(l - 1, 0)]
        hl = 0.5 * hl if 0 < l < len(rs) - 1 else (rs[1] - rs[0] if l == 0 else rs[-1] - rs[-2])
        m = max(8, int(round(2 * np.pi * r / hl)))
        th = (np.arange(m) + rng.uniform(0, 1)) * (2 * np.pi / m)
        pts.append(np.stack([r * np.cos(th), r * np.sin(th)], 1))
    return np.concatenate(pts), rs


def cylinder_mesh(n_target=30000, seed=2, r_in=1.0, r_out=15.0, ratio=1.05, tol=0.01):
    """Seeded Delaunay triangulation around a cylinder of radius ``r_in``.

    Points sit on radial layers whose heights grow geometrically by ``ratio``
    from the wall; each layer holds as many points as its circumference divided
    by the local layer height (near-isotropic triangles).  The first height is
    bisected until the triangle count is within ``tol`` of ``n_target``.
    Boundary faces at ``r_in`` are walls (tag 0), those at ``r_out`` far field.
    """
    from scipy.spatial import Delaunay

    def build(h0):
        rng = np.random.default_rng(seed)
        pts, _ = _annulus_points(h0, rng, r_in, r_out, ratio)
        tri = Delaunay(pts)
        simp = tri.simplices
        cen = pts[simp].mean(axis=1)
        keep = np.hypot(cen[:, 0], cen[:, 1]) > r_in
        return pts, simp[keep]

    lo, hi = 1e-3, 1.0
    pts, simp = build(0.05)
    for _ in range(60):
        mid = math.sqrt(lo * hi)
        pts, simp = build(mid)
        if abs(len(simp) - n_target) <= tol * n_target:
            break
        if len(simp) > n_target:
            lo = mid
        else:
            hi = mid
    rmid = 0.5 * (r_in + r_out)

    def classify(fx):
        r = np.hypot(fx[:, 0], fx[:, 1])
        typ = np.where(r < rmid, WALL, FARFIELD).astype(np.int32)
        return typ, np.zeros(len(fx), np.int32)

    return simplex_mesh(pts, simp.astype(np.int64), classify)


def _fibonacci_sphere(m, rng):
    i = np.arange(m) + 0.5
    phi = np.arccos(1 - 2 * i / m)
    th = np.pi * (1 + 5 ** 0.5) * i + rng.uniform(0, 2 * np.pi)
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)


def sphere_mesh(n_target=150000, seed=3, r_in=1.0, r_out=12.0, ratio=1.08, tol=0.02):
    """Seeded Delaunay tetrahedralisation of a spherical shell around a sphere.

    Points sit on spherical shells (Fibonacci lattices) whose spacing grows by
    ``ratio`` from the wall; tetrahedra whose centroid falls inside the sphere
    are removed.  Boundary faces at ``r_in`` are walls, those at ``r_out`` far
    field.  The first layer height is bisected to land near ``n_target`` cells.
    """
    from scipy.spatial import Delaunay

    def build(h0):
        rng = np.random.default_rng(seed)
        rs = _geometric_layers(r_in, r_out, h0, ratio)
        pts = []
        for l, r in enumerate(rs):
            hl = rs[min(l + 1, len(rs) - 1)] - rs[max(l - 1, 0)]
            hl = 0.5 * hl if 0 < l < len(rs) - 1 else (rs[1] - rs[0] if l == 0 else rs[-1] - rs[-2])
            m = max(12, int(round(4 * np.pi * r * r / (hl * hl))))
            pts.append(r * _fibonacci_sphere(m, rng))
        pts = np.concatenate(pts)
        tri = Delaunay(pts)
        simp = tri.simplices
        cen = pts[simp].mean(axis=1)
        keep = np.linalg.norm(cen, axis=1) > r_in
        # drop flat slivers produced by co-spherical points
        P = pts[simp[keep]]
        vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6.0
        ok = vol > 1e-12 * np.max(vol)
        return pts, simp[keep][ok]

    lo, hi = 1e-3, 2.0
    pts, simp = build(0.1)
    for _ in range(50):
        mid = math.sqrt(lo * hi)
        pts, simp = build(mid)
        if abs(len(simp) - n_target) <= tol * n_target:
            break
        if len(simp) > n_target:
            lo = mid
        else:
            hi = mid
    rmid = 0.5 * (r_in + r_out)

    def classify(fx):
        r = np.linalg.norm(fx, axis=1)
        typ = np.where(r < rmid, WALL, FARFIELD).astype(np.int32)
        return typ, np.zeros(len(fx), np.int32)

    return simplex_mesh(pts, simp.astype(np.int64), classify)


# ----------------------------------------------------------------------------
# parameter records and named workloads
# ----------------------------------------------------------------------------
def params(Kn, Pr=2.0 / 3.0, omega=0.81, cfl=0.8, L_ref=1.0, dt=0.0, limiter=1,
           venkat_K=1.0, walls=None, inf=None):
    """Gas / numerical parameters.  ``walls`` is a list of ``{"T": T_w, "U": U_w}``
    (one per wall tag); ``inf`` is ``{"rho", "U", "T"}`` for far-field ghosts."""
    return {"Kn": float(Kn), "Pr": float(Pr), "omega": float(omega), "cfl": float(cfl),
            "L_ref": float(L_ref), "dt": float(dt), "limiter": int(limiter),
            "venkat_K": float(venkat_K), "walls": walls or [], "inf": inf}


def uniform_state(C, D, rho=1.0, U=None, T=1.0):
    """Primitive initial state ``[C][D+2]`` = (rho, U_1..U_D, T)."""
    s = np.zeros((C, D + 2))
    s[:, 0] = rho
    if U is not None:
        s[:, 1:1 + D] = np.asarray(U, float)[:D]
    s[:, D + 1] = T
    return s


def cavity_case(n=20, nv=24, vmax=4.0, Kn=0.075, lid=0.16):
    """2D lid-driven cavity: unit square, n x n quads, all walls at T=1; the top
    wall (tag 1) moves with speed ``lid``; nv x nv velocities on [-vmax, vmax]^2;
    Shakhov gas (Pr=2/3, omega=0.81), CFL 0.8, rest Maxwellian start."""
    mesh = quad_mesh(n, n, 1.0, 1.0, left=("wall", 0), right=("wall", 0),
                     bottom=("wall", 0), top=("wall", 1))
    vg = cartesian_vgrid((nv, nv), (-vmax, -vmax), (vmax, vmax))
    pr = params(Kn, walls=[{"T": 1.0, "U": [0.0, 0.0, 0.0]}, {"T": 1.0, "U": [lid, 0.0, 0.0]}])
    init = uniform_state(len(mesh["cell_vol"]), 2)
    return {"name": f"cavity{n}x{n}_v{nv}x{nv}", "mesh": mesh, "vgrid": vg, "params": pr, "init": init}


def freestream_speed(mach, gamma=5.0 / 3.0, T=1.0):
    return mach * math.sqrt(gamma * T)


def blended_start(mesh, U, r_body=1.0, delta=1.0):
    """Initial field for flow past a body of radius ``r_body`` centred at the
    origin: rho = T = 1 and a velocity that rises from rest at the wall to the
    free stream, U(r) = U_inf (1 - exp(-(r - r_body)/delta)).  It avoids the
    transient near-vacuum that an impulsive uniform start opens behind the
    body; the steady state does not depend on it."""
    D = mesh["dim"]
    r = np.linalg.norm(mesh["cell_xc"], axis=1)
    s = 1.0 - np.exp(-np.maximum(r - r_body, 0.0) / delta)
    init = uniform_state(len(r), D)
    init[:, 1:1 + D] = s[:, None] * np.asarray(U, float)[None, :D]
    return init


def cylinder_case(n_cells=30000, nvx=60, nvy=50, mach=5.0, Kn=0.1, seed=2,
                  vx=(-12.0, 12.0), vy=(-10.0, 10.0), start="blended"):
    """2D Mach-``mach`` argon flow past a radius-1 cylinder, far field at radius
    15; Kn defined on the diameter (L_ref = 2); isothermal wall at T_inf = 1.
    ``start``: "blended" (rest at the wall, free stream away from it) or
    "impulsive" (uniform free stream)."""
    mesh = cylinder_mesh(n_cells, seed=seed)
    vg = cartesian_vgrid((nvx, nvy), (vx[0], vy[0]), (vx[1], vy[1]))
    Uinf = freestream_speed(mach)
    pr = params(Kn, L_ref=2.0, walls=[{"T": 1.0, "U": [0.0, 0.0, 0.0]}],
                inf={"rho": 1.0, "U": [Uinf, 0.0, 0.0], "T": 1.0})
    if start == "impulsive":
        init = uniform_state(len(mesh["cell_vol"]), 2, U=[Uinf, 0.0])
    else:
        init = blended_start(mesh, [Uinf, 0.0])
    return {"name": f"cylinder_Ma{mach:g}_Kn{Kn:g}_c{len(mesh['cell_vol'])}_v{nvx}x{nvy}",
            "mesh": mesh, "vgrid": vg, "params": pr, "init": init}


def sphere_case(n_cells=150000, nv=28, vmax=10.0, mach=4.0, Kn=0.1, seed=3, start="blended"):
    """3D Mach-``mach`` argon flow past a radius-1 sphere, far field at radius
    12, Kn on the diameter; nv^3 velocities on [-vmax, vmax]^3."""
    mesh = sphere_mesh(n_cells, seed=seed)
    vg = cartesian_vgrid((nv, nv, nv), (-vmax,) * 3, (vmax,) * 3)
    Uinf = freestream_speed(mach)
    pr = params(Kn, Pr=2.0 / 3.0, L_ref=2.0, walls=[{"T": 1.0, "U": [0.0, 0.0, 0.0]}],
                inf={"rho": 1.0, "U": [Uinf, 0.0, 0.0], "T": 1.0})
    if start == "impulsive":
        init = uniform_state(len(mesh["cell_vol"]), 3, U=[Uinf, 0.0, 0.0])
    else:
        init = blended_start(mesh, [Uinf, 0.0, 0.0])
    return {"name": f"sphere_Ma{mach:g}_Kn{Kn:g}_c{len(mesh['cell_vol'])}_v{nv}^3",
            "mesh": mesh, "vgrid": vg, "params": pr, "init": init}


def perturbation(shape, seed, amp=0.1):
    """Seeded multiplicative noise factors ``1 + amp*U(-1,1)`` used to push a
    distribution away from equilibrium in tests."""
    rng = np.random.default_rng(seed)
    return 1.0 + amp * rng.uniform(-1.0, 1.0, size=shape)


def smooth_state(mesh, seed, amp=0.1, U0=None, rho0=1.0, T0=1.0):
    """Seeded smooth primitive field (rho, U, T) with sinusoidal perturbations of
    relative size ``amp`` around (rho0, U0, T0)."""
    rng = np.random.default_rng(seed)
    D = mesh["dim"]
    x = mesh["cell_xc"]
    C = len(x)
    k = rng.uniform(1.0, 3.0, size=(D + 2, D)) * 2 * np.pi
    ph = rng.uniform(0, 2 * np.pi, size=D + 2)
    s = uniform_state(C, D, rho0, U0, T0)
    for m in range(D + 2):
        wave = np.sin(x @ k[m] + ph[m])
        if m == 0:
            s[:, 0] *= 1 + amp * wave
        elif m == D + 1:
            s[:, m] *= 1 + amp * wave
        else:
            s[:, m] += amp * wave
    return s
