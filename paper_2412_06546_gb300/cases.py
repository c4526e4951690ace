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


# X38-like lifting body: a smooth convex superellipsoid of length 8 (x) and
# span 3.5 (y), F(x) = |x/a|^px + |y/b|^py + |z/c|^pz <= 1 with the exponent
# and semi-axis chosen per side: an ellipsoidal nose (x < 0) and a blunter aft
# end (x > 0), a nearly flat bottom (z < 0, exponent 6) and a rounded top.
_X38_SIDES = {"ax": (4.0, 4.0), "px": (2.0, 4.0), "b": 1.75, "py": 2.5, "cz": (0.6, 1.1), "pz": (6.0, 2.2)}


def _x38_terms(X):
    g = _X38_SIDES
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    ax = np.where(x < 0, g["ax"][0], g["ax"][1])
    px = np.where(x < 0, g["px"][0], g["px"][1])
    cz = np.where(z < 0, g["cz"][0], g["cz"][1])
    pz = np.where(z < 0, g["pz"][0], g["pz"][1])
    return (x, ax, px), (y, g["b"], g["py"]), (z, cz, pz)


def x38_body_F(X):
    """Implicit function of the X38-like body (< 1 inside, 1 on the surface)."""
    return sum(np.abs(v / a) ** q for v, a, q in _x38_terms(np.asarray(X, float)))


def _x38_normal(X):
    gr = np.stack([q * np.sign(v) * np.abs(v) ** (q - 1) / a ** q for v, a, q in _x38_terms(X)], axis=-1)
    return gr / np.linalg.norm(gr, axis=-1, keepdims=True)


def _x38_surface(m, rng):
    """m points on the body surface: directions of a Fibonacci lattice,
    stretched to the body's proportions, projected along rays from the centre."""
    d = _fibonacci_sphere(m, rng) * np.array([4.0, 1.75, 0.85])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    lo, hi = np.zeros(m), np.full(m, 8.0)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        inside = x38_body_F(mid[:, None] * d) < 1.0
        lo = np.where(inside, mid, lo)
        hi = np.where(inside, hi, mid)
    return 0.5 * (lo + hi)[:, None] * d


def _thin(X, h, rng):
    """Greedy thinning in random order: keep a point unless a kept point lies
    within its spacing h (scalar or per point)."""
    from scipy.spatial import cKDTree
    tree = cKDTree(X)
    hh = np.broadcast_to(np.asarray(h, float), (len(X),))
    gone = np.zeros(len(X), bool)
    keep = []
    for i in rng.permutation(len(X)):
        if gone[i]:
            continue
        keep.append(i)
        gone[tree.query_ball_point(X[i], hh[i])] = True
    return X[np.sort(np.asarray(keep, np.int64))]


def x38_mesh(h0=0.0449, seed=5, s_out=8.0, ratio=1.1, n_surface=400000):
    """Seeded tetrahedral mesh around the X38-like body.

    Point layers lie on offset surfaces of the (convex) body at distances
    s_k along the outward normals, with thickness h0 ratio^k; each layer is
    thinned to a spacing equal to its thickness.  Delaunay tetrahedra whose
    centroid lies inside the body are removed.  Boundary faces on the body are
    walls (tag 0), those on the outermost offset surface (at s_out) far field.
    The default h0 gives 1,051,276 cells (seed 5)."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    P0 = _x38_surface(n_surface, rng)
    N0 = _x38_normal(P0)
    pts, s, k = [], 0.0, 0
    while True:
        hk = h0 * ratio ** k
        pts.append(_thin(P0 + s * N0, hk, rng))
        if s >= s_out:
            break
        s = min(s + hk, s_out)
        k += 1
    pts = np.concatenate(pts)
    simp = Delaunay(pts).simplices
    P = pts[simp]
    keep = x38_body_F(P.mean(axis=1)) > 1.0
    vol = np.abs(np.linalg.det(P[keep][:, 1:] - P[keep][:, :1])) / 6.0
    ok = vol > 1e-12 * vol.max()
    simp = simp[keep][ok]

    def classify(fx):
        typ = np.where(x38_body_F(fx) < 4.0, WALL, FARFIELD).astype(np.int32)
        return typ, np.zeros(len(fx), np.int32)

    mesh = simplex_mesh(pts, simp.astype(np.int64), classify)
    mesh["_surface"] = P0
    return mesh


def tet_ball_vgrid(n_target=4548, R=18.9, centres=((0.0, 0.0, 0.0),), h_min=0.6, grad=0.35, seed=5,
                   tol=0.02):
    """Unstructured 3D velocity grid: a seeded Delaunay tetrahedralisation of
    the ball |u| <= R whose spacing grows from h_min at each of ``centres``
    (h = min(h_min + grad d, R/4), d the distance to the nearest centre), with
    the centroid rule (u_k = centroid, w_k = volume of cell k).  The spacing
    scale is bisected to land near ``n_target`` cells."""
    from scipy.spatial import Delaunay
    C0 = np.asarray(centres, float)

    def spacing(X, sc):
        d = np.min(np.linalg.norm(X[:, None, :] - C0[None], axis=2), axis=1)
        return sc * np.minimum(h_min + grad * d, R / 4.0)

    def build(sc):
        rng = np.random.default_rng(seed)
        cand = rng.uniform(-R, R, size=(60000, 3))
        cand = cand[np.linalg.norm(cand, axis=1) < R - 1e-9]
        inner = _thin(cand, spacing(cand, sc), rng)
        shell = R * _fibonacci_sphere(20000, rng)
        shell = _thin(shell, spacing(shell, sc), rng)
        if len(inner):
            from scipy.spatial import cKDTree
            d, _ = cKDTree(shell).query(inner)
            inner = inner[d > 0.5 * spacing(inner, sc)]
        X = np.concatenate([inner, shell])
        tet = Delaunay(X).simplices
        P = X[tet]
        w = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6.0
        ok = w > 1e-12 * w.max()
        return P[ok].mean(axis=1), w[ok]

    lo, hi = 0.2, 5.0
    u, w = build(1.0)
    for _ in range(40):
        mid = math.sqrt(lo * hi)
        u, w = build(mid)
        if abs(len(w) - n_target) <= tol * n_target:
            break
        if len(w) > n_target:
            lo = mid
        else:
            hi = mid
    return {"dim": 3, "u": np.ascontiguousarray(u), "w": np.ascontiguousarray(w), "cart_n": [0, 0, 0]}


def tri_disk_vgrid(n_target, R, centre=(0.0, 0.0), refine=(((0.0, 0.0), 3.0),), h_fine=0.5, grad=0.3,
                   seed=6):
    """Unstructured 2D velocity grid of exactly ``n_target`` triangles: a seeded
    Delaunay triangulation of the disk |u - centre| <= R, with spacing h_fine
    inside each refinement disk ``(point, radius)`` of ``refine`` and growing by
    ``grad`` per unit distance outside them (capped at R/4), with the centroid
    rule (u_k = centroid, w_k = area of triangle k).  The spacing scale is
    bisected to the largest triangulation not above the target, and the
    remaining count is made up by splitting the largest triangles that have an
    edge on the disk boundary at that edge's midpoint (each split adds one
    triangle and leaves every other triangle unchanged)."""
    from scipy.spatial import Delaunay, cKDTree
    c0 = np.asarray(centre, float)
    pts_r = [(np.asarray(p, float), float(r)) for p, r in refine]

    def spacing(X, sc):
        d = np.full(len(X), np.inf)
        for p, r in pts_r:
            d = np.minimum(d, np.maximum(np.linalg.norm(X - p, axis=1) - r, 0.0))
        return sc * np.minimum(h_fine + grad * d, R / 4.0)

    def build(sc):
        rng = np.random.default_rng(seed)
        cand = c0 + rng.uniform(-R, R, size=(40000, 2))
        cand = cand[np.linalg.norm(cand - c0, axis=1) < R - 1e-9]
        inner = _thin(cand, spacing(cand, sc), rng)
        th = np.linspace(0.0, 2 * np.pi, 4000, endpoint=False) + rng.uniform(0, 2 * np.pi / 4000)
        ring = c0 + R * np.stack([np.cos(th), np.sin(th)], axis=1)
        ring = _thin(ring, spacing(ring, sc), rng)
        d, _ = cKDTree(ring).query(inner)
        inner = inner[d > 0.5 * spacing(inner, sc)]
        X = np.concatenate([inner, ring])
        return X, Delaunay(X).simplices

    lo, hi = 0.2, 5.0
    best = None
    for _ in range(50):
        mid = math.sqrt(lo * hi)
        X, tri = build(mid)
        if len(tri) <= n_target and (best is None or len(tri) > len(best[1])):
            best = (X, tri)
        if len(tri) == n_target:
            break
        if len(tri) > n_target:
            lo = mid
        else:
            hi = mid
    X, tri = best
    X = [tuple(x) for x in X]
    tri = [list(t) for t in tri]
    on_ring = {i for i, x in enumerate(X) if abs(np.hypot(x[0] - c0[0], x[1] - c0[1]) - R) < 1e-9 * R}

    def area(t):
        a, b, c = (np.asarray(X[i]) for i in t)
        return 0.5 * abs((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))

    while len(tri) < n_target:
        # edges used by one triangle only lie on the boundary of the triangulation
        count = {}
        for t in tri:
            for e in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
                k = (min(e), max(e))
                count[k] = count.get(k, 0) + 1
        cands = [(area(t), ti, (a, b)) for ti, t in enumerate(tri)
                 for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))
                 if count[(min(a, b), max(a, b))] == 1 and a in on_ring and b in on_ring]
        _, ti, (a, b) = max(cands)
        m = len(X)
        X.append(tuple(0.5 * (np.asarray(X[a]) + np.asarray(X[b]))))
        t = tri[ti]
        o = [v for v in t if v not in (a, b)][0]
        tri[ti] = [a, m, o]
        tri.append([m, b, o])
    X = np.asarray(X)
    P = X[np.asarray(tri)]
    w = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                     - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
    return {"dim": 2, "u": np.ascontiguousarray(P.mean(axis=1)), "w": np.ascontiguousarray(w),
            "cart_n": [0, 0, 0]}


def cylinder_dvs_vgrid(mach, which="E1", n_target=None, gamma=5.0 / 3.0, T_inf=1.0, T_w=1.0):
    """The unstructured velocity meshes of the paper's hypersonic cylinder runs:
    a disk centred at 0.4 (U_inf, 0), refined around rest and around U_inf.
    E1 (Ma 5, Kn 0.1): 2,060 triangles, radius 6 sqrt(T_s), refinement radius
    3 sqrt(T) at both points; E2 (Ma 15, Kn 0.01): 3,420 triangles, radius
    5 sqrt(T_s), refinement radius 5 sqrt(T).  T_s is the stagnation
    temperature of the free stream."""
    U = freestream_speed(mach, gamma, T_inf)
    Ts = T_inf * (1.0 + 0.5 * (gamma - 1.0) * mach * mach)
    if which == "E1":
        n, R, rr = 2060, 6.0 * math.sqrt(Ts), 3.0
    else:
        n, R, rr = 3420, 5.0 * math.sqrt(Ts), 5.0
    return tri_disk_vgrid(n_target or n, R, centre=(0.4 * U, 0.0),
                          refine=(((0.0, 0.0), rr * math.sqrt(T_w)), ((U, 0.0), rr * math.sqrt(T_inf))),
                          h_fine=0.35 * math.sqrt(T_inf), grad=0.25, seed=6 if which == "E1" else 7)


# ----------------------------------------------------------------------------
# local problems: sampled checks and timings of cases too large for a whole
# oracle run.  One explicit step updates a cell from data no further than two
# face rings away: the limited slopes of the cell and of its face neighbours
# (each reads its own neighbours' values), the interface equilibria of its
# faces (face states of both sides, whose limited macroscopic gradients read
# the second ring), the heat flux of both sides and, at walls, the cell's own
# distribution.  A mesh made of the sample S0, S1 = S0 + face neighbours,
# S2 = S1 + their face neighbours, with every face of every S1 cell, stepped
# once from the same state on S2 with the same time step, therefore gives the
# full-mesh step on S0.  Cells of S2 outside S1 lose faces and so get wrong
# values of their own, which no S0 result reads.
# ----------------------------------------------------------------------------
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


def cylinder_dvs_case(which="E1", n_cells=30000, seed=2, start="blended"):
    """The paper's hypersonic cylinder setups on an unstructured velocity mesh:
    E1 is Ma 5 at Kn 0.1 with the 2,060-triangle velocity mesh, E2 is Ma 15 at
    Kn 0.01 with the 3,420-triangle one (Kn on the diameter, isothermal wall at
    T_inf), on the seeded Delaunay cylinder mesh of ``n_cells`` triangles."""
    mach, Kn = (5.0, 0.1) if which == "E1" else (15.0, 0.01)
    mesh = cylinder_mesh(n_cells, seed=seed)
    vg = cylinder_dvs_vgrid(mach, which)
    Uinf = freestream_speed(mach)
    pr = params(Kn, L_ref=2.0, walls=[{"T": 1.0, "U": [0.0, 0.0, 0.0]}],
                inf={"rho": 1.0, "U": [Uinf, 0.0, 0.0], "T": 1.0})
    if start == "impulsive":
        init = uniform_state(len(mesh["cell_vol"]), 2, U=[Uinf, 0.0])
    else:
        init = blended_start(mesh, [Uinf, 0.0])
    return {"name": f"cylinder_{which}_Ma{mach:g}_Kn{Kn:g}_c{len(mesh['cell_vol'])}_dvs{len(vg['w'])}",
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


def x38_case(h0=0.0449, nv=4548, mach=8.0, Kn=0.005, aoa_deg=20.0, T_wall=302.0 / 56.0, seed=5,
             start="blended", n_surface=400000):
    """3D Mach-8 argon flow past the X38-like body at 20 degrees angle of
    attack (the flow meets the flat bottom), Kn 0.005 on the body length 8,
    isothermal wall at T_w = 302/56 T_inf.  Velocities: ``nv`` tetrahedra in
    the ball of radius 4 sqrt(T_s), T_s = 1 + (gamma - 1)/2 Ma^2 the
    stagnation temperature, refined at rest and at U_inf (centroid rule)."""
    mesh = x38_mesh(h0, seed=seed, n_surface=n_surface)
    Uinf = freestream_speed(mach)
    a = math.radians(aoa_deg)
    Uv = [Uinf * math.cos(a), 0.0, Uinf * math.sin(a)]
    Ts = 1.0 + (5.0 / 3.0 - 1.0) / 2.0 * mach * mach
    vg = tet_ball_vgrid(nv, R=4.0 * math.sqrt(Ts), centres=((0.0, 0.0, 0.0), tuple(Uv)), seed=seed)
    pr = params(Kn, L_ref=8.0, walls=[{"T": T_wall, "U": [0.0, 0.0, 0.0]}],
                inf={"rho": 1.0, "U": Uv, "T": 1.0})
    C = len(mesh["cell_vol"])
    if start == "impulsive":
        init = uniform_state(C, 3, U=Uv)
    else:
        # U rises from rest at the wall to the free stream with the distance d
        # to the body surface: U(d) = U_inf (1 - exp(-d))
        from scipy.spatial import cKDTree
        d, _ = cKDTree(mesh["_surface"]).query(mesh["cell_xc"])
        init = uniform_state(C, 3)
        init[:, 1:4] = (1.0 - np.exp(-d))[:, None] * np.asarray(Uv)[None]
    mesh.pop("_surface")
    return {"name": f"x38_Ma{mach:g}_Kn{Kn:g}_c{C}_v{len(vg['w'])}", "mesh": mesh, "vgrid": vg,
            "params": pr, "init": init}


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
