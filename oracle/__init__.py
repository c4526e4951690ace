"""FP64 CPU oracle of one explicit UGKS step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library is plain C
(``ugks_oracle.c``), built with ``-O2 -ffp-contract=off`` and shares no code
with the CUDA library.  See ``ugks_oracle.c`` for the step (Algorithm 1 of the
paper) and the readings it takes where the paper is silent.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libugks_oracle.so")
_lib = None

D_P = ct.POINTER(ct.c_double)
I64_P = ct.POINTER(ct.c_int64)
I32_P = ct.POINTER(ct.c_int32)


def build(force=False):
    """Compile the oracle into ``oracle/_build/libugks_oracle.so``."""
    src = os.path.join(_HERE, "ugks_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src),
                                             os.path.getmtime(os.path.join(_HERE, "ugks_oracle.h")))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Mesh(ct.Structure):
    _fields_ = [("dim", ct.c_int32), ("n_cells", ct.c_int64), ("n_faces", ct.c_int64),
                ("cell_xc", D_P), ("cell_vol", D_P), ("face_cells", I64_P),
                ("face_n", D_P), ("face_S", D_P), ("face_xc", D_P),
                ("face_type", I32_P), ("face_tag", I32_P), ("face_shift", D_P)]


class _VGrid(ct.Structure):
    _fields_ = [("dim", ct.c_int32), ("nv", ct.c_int64), ("u", D_P), ("w", D_P)]


class _Params(ct.Structure):
    _fields_ = [("Kn", ct.c_double), ("L_ref", ct.c_double), ("Pr", ct.c_double),
                ("omega", ct.c_double), ("cfl", ct.c_double), ("dt", ct.c_double),
                ("limiter", ct.c_int32), ("venkat_K", ct.c_double), ("n_walls", ct.c_int32),
                ("wall_T", D_P), ("wall_U", D_P), ("inf_rho", ct.c_double),
                ("inf_U", ct.c_double * 3), ("inf_T", ct.c_double), ("n_threads", ct.c_int32),
                ("w0_analytic", ct.c_int32)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ct.CDLL(_SO)
        L.or_create.restype = ct.c_void_p
        L.or_create.argtypes = [ct.POINTER(_Mesh), ct.POINTER(_VGrid), ct.POINTER(_Params), D_P]
        L.or_destroy.argtypes = [ct.c_void_p]
        L.or_step.argtypes = [ct.c_void_p, ct.c_int32]
        L.or_dt.restype = ct.c_double
        L.or_dt.argtypes = [ct.c_void_p]
        L.or_ncomp.restype = ct.c_int32
        L.or_ncomp.argtypes = [ct.c_void_p]
        L.or_get_state.argtypes = [ct.c_void_p, D_P, D_P, D_P]
        L.or_set_state.argtypes = [ct.c_void_p, D_P, D_P]
        L.or_residual.argtypes = [ct.c_void_p, D_P]
        L.or_wall_rho.argtypes = [ct.c_void_p, D_P]
        L.or_face_macro_flux.argtypes = [ct.c_void_p, D_P]
        L.or_face_states.argtypes = [ct.c_void_p, D_P, D_P]
        L.or_wall_quantities.argtypes = [ct.c_void_p, D_P, D_P, D_P]
        L.or_time_integrals.argtypes = [ct.c_double, ct.c_double, D_P]
        L.or_maxwellian.argtypes = [ct.c_int32, ct.c_double, D_P, ct.c_double, ct.c_int64, D_P, D_P, D_P]
        L.or_shakhov.argtypes = [ct.c_int32, ct.c_double, ct.c_double, D_P, ct.c_double, D_P,
                                 ct.c_int64, D_P, D_P, D_P]
        L.or_heat_flux.argtypes = [ct.c_int32, ct.c_int64, D_P, D_P, D_P, D_P, D_P, D_P]
        L.or_venkat.restype = ct.c_double
        L.or_venkat.argtypes = [ct.c_double, ct.c_double, ct.c_double]
        L.or_face_equilibrium.argtypes = [ct.c_int32, ct.c_int64, D_P, D_P, D_P, D_P, D_P, D_P,
                                          D_P, D_P, D_P]
        L.or_face_equilibrium_ex.argtypes = [ct.c_int32, ct.c_int64, D_P, D_P, D_P, D_P, D_P, D_P,
                                             D_P, D_P, D_P, ct.c_int]
        L.or_moment_matrix.argtypes = [ct.c_int32, ct.c_int64, D_P, D_P, D_P, D_P]
        L.or_scalar_gradient.argtypes = [ct.c_void_p, D_P, D_P, ct.c_int32, D_P]
        L.or_micro_gradient.argtypes = [ct.c_void_p, D_P, D_P, D_P, D_P]
        L.or_mu_ref.restype = ct.c_double
        L.or_mu_ref.argtypes = [ct.c_void_p]
        _lib = L
    return _lib


def _p(a, typ=D_P):
    return a.ctypes.data_as(typ) if a is not None else None


def _c(a, dt=np.float64):
    return np.ascontiguousarray(a, dtype=dt)


class OracleCase:
    """One UGKS case on the CPU oracle.  ``mesh``, ``vgrid`` and ``params`` are
    the dicts of ``paper_2412_06546_gb300.cases``; ``init`` is the primitive
    state ``[C][D+2]`` (rho, U, T)."""

    def __init__(self, mesh, vgrid, params, init=None, n_threads=0):
        L = lib()
        self._keep = []
        D = mesh["dim"]
        self.D = D
        self.C = len(mesh["cell_vol"])
        self.F = len(mesh["face_S"])
        self.Nv = len(vgrid["w"])
        arrs = {k: _c(mesh[k]) for k in ("cell_xc", "cell_vol", "face_n", "face_S", "face_xc", "face_shift")}
        arrs["face_cells"] = _c(mesh["face_cells"], np.int64)
        arrs["face_type"] = _c(mesh["face_type"], np.int32)
        arrs["face_tag"] = _c(mesh["face_tag"], np.int32)
        self._keep.append(arrs)
        self.n_wall = int(np.count_nonzero(arrs["face_type"] == 1))
        m = _Mesh(D, self.C, self.F, _p(arrs["cell_xc"]), _p(arrs["cell_vol"]),
                  _p(arrs["face_cells"], I64_P), _p(arrs["face_n"]), _p(arrs["face_S"]),
                  _p(arrs["face_xc"]), _p(arrs["face_type"], I32_P), _p(arrs["face_tag"], I32_P),
                  _p(arrs["face_shift"]))
        u, w = _c(vgrid["u"]), _c(vgrid["w"])
        self.u, self.w = u, w
        self._keep += [u, w]
        v = _VGrid(D, self.Nv, _p(u), _p(w))
        walls = params.get("walls") or []
        wT = _c([wl["T"] for wl in walls] or [1.0])
        wU = _c([list(wl["U"]) + [0.0] * (3 - len(wl["U"])) for wl in walls] or [[0.0, 0.0, 0.0]])
        self._keep += [wT, wU]
        inf = params.get("inf") or {"rho": 1.0, "U": [0.0, 0.0, 0.0], "T": 1.0}
        iU = list(inf["U"]) + [0.0] * (3 - len(inf["U"]))
        p = _Params(params["Kn"], params.get("L_ref", 1.0), params["Pr"], params["omega"],
                    params["cfl"], params.get("dt", 0.0), params.get("limiter", 1),
                    params.get("venkat_K", 1.0), len(walls), _p(wT), _p(wU), inf["rho"],
                    (ct.c_double * 3)(*iU), inf["T"], n_threads, int(params.get("w0_analytic", 0)))
        init_a = _c(init) if init is not None else None
        self._h = L.or_create(ct.byref(m), ct.byref(v), ct.byref(p), _p(init_a))
        self.nc = L.or_ncomp(self._h)
        self.dt = L.or_dt(self._h)
        self.mu_ref = L.or_mu_ref(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_destroy(self._h)
            self._h = None

    def step(self, n=1):
        lib().or_step(self._h, n)

    def state(self):
        f = np.empty((self.C, self.nc, self.Nv))
        W = np.empty((self.C, self.D + 2))
        q = np.empty((self.C, self.D))
        lib().or_get_state(self._h, _p(f), _p(W), _p(q))
        return f, W, q

    def set_state(self, f=None, W=None):
        fa = _c(f) if f is not None else None
        Wa = _c(W) if W is not None else None
        lib().or_set_state(self._h, _p(fa), _p(Wa))

    def residual(self):
        r = np.empty(self.D + 2)
        lib().or_residual(self._h, _p(r))
        return r

    def wall_rho(self, n_wall):
        r = np.empty(max(n_wall, 1))
        lib().or_wall_rho(self._h, _p(r))
        return r[:n_wall]

    def wall_quantities(self):
        """p_w, sigma_w, q_w of the last step at the wall faces (face order)."""
        n = max(self.n_wall, 1)
        p, sg, q = np.empty(n), np.empty(n), np.empty(n)
        lib().or_wall_quantities(self._h, _p(p), _p(sg), _p(q))
        return p[:self.n_wall], sg[:self.n_wall], q[:self.n_wall]

    def face_states(self):
        """W_L, W_R [F][D+2] of the last step (conserved; W_R is the ghost state
        at far-field faces; zero at walls)."""
        WL = np.empty((self.F, self.D + 2))
        WR = np.empty((self.F, self.D + 2))
        lib().or_face_states(self._h, _p(WL), _p(WR))
        return WL, WR

    def face_macro_flux(self):
        F = np.empty((self.F, self.D + 2))
        lib().or_face_macro_flux(self._h, _p(F))
        return F

    def micro_gradient(self, phi, u, phi_ghost=None):
        phi, u = _c(phi), _c(u)
        g = _c(phi_ghost) if phi_ghost is not None else None
        out = np.empty((self.C, self.D))
        lib().or_micro_gradient(self._h, _p(phi), _p(g), _p(u), _p(out))
        return out

    def scalar_gradient(self, phi, phi_ghost=None, limited=False):
        phi = _c(phi)
        g = _c(phi_ghost) if phi_ghost is not None else None
        out = np.empty((self.C, self.D))
        lib().or_scalar_gradient(self._h, _p(phi), _p(g), int(limited), _p(out))
        return out


# ---- building blocks for the pin tests ----
def time_integrals(dt, tau):
    q = np.empty(5)
    lib().or_time_integrals(float(dt), float(tau), _p(q))
    return q


def maxwellian(D, rho, U, lam, u):
    u = _c(u)
    U = _c(U)
    H = np.empty(len(u))
    B = np.empty(len(u))
    lib().or_maxwellian(D, rho, _p(U), lam, len(u), _p(u), _p(H), _p(B))
    return H, B


def shakhov(D, Pr, rho, U, lam, q, u):
    u, U, q = _c(u), _c(U), _c(q)
    Hp = np.empty(len(u))
    Bp = np.empty(len(u))
    lib().or_shakhov(D, Pr, rho, _p(U), lam, _p(q), len(u), _p(u), _p(Hp), _p(Bp))
    return Hp, Bp


def heat_flux(D, u, w, h, b, U):
    u, w, h, U = _c(u), _c(w), _c(h), _c(U)
    b = _c(b) if b is not None else None
    q = np.empty(D)
    lib().or_heat_flux(D, len(w), _p(u), _p(w), _p(h), _p(b), _p(U), _p(q))
    return q


def venkat(d1, d2, eps2):
    return lib().or_venkat(float(d1), float(d2), float(eps2))


def face_equilibrium(D, u, w, n, WL, WR, gradW0, analytic=False):
    """W0, spatial slopes a and time slope A of the interface equilibrium;
    ``analytic``: W0 from the analytic half-range moments."""
    u, w, n, WL, WR, g = _c(u), _c(w), _c(n), _c(WL), _c(WR), _c(gradW0)
    W0 = np.empty(D + 2)
    a = np.empty((D, D + 2))
    A = np.empty(D + 2)
    lib().or_face_equilibrium_ex(D, len(w), _p(u), _p(w), _p(n), _p(WL), _p(WR), _p(g), _p(W0), _p(a), _p(A),
                                 1 if analytic else 0)
    return W0, a, A


def moment_matrix(D, u, w, W0):
    u, w, W0 = _c(u), _c(w), _c(W0)
    M0 = np.empty((D + 2, D + 2))
    lib().or_moment_matrix(D, len(w), _p(u), _p(w), _p(W0), _p(M0))
    return M0
