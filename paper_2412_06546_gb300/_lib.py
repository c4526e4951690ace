"""ctypes binding of the C ABI in ``include/ugks.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``_build/libugks.so``; this
module converts numpy arrays to the ABI structs, hands the library torch's
caching allocator and current stream, and turns status codes into exceptions.
There is no CPU fallback: if the library or a GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as ct
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libugks.so")

D_P = ct.POINTER(ct.c_double)
F_P = ct.POINTER(ct.c_float)
I64_P = ct.POINTER(ct.c_int64)
I32_P = ct.POINTER(ct.c_int32)

FP64, FP32 = 0, 1
STATUS = {0: "UGKS_OK", 1: "UGKS_EINVAL", 2: "UGKS_ENOMEM", 3: "UGKS_ECUDA", 4: "UGKS_ENUMERIC",
          5: "UGKS_ENOTCONVERGED", 6: "UGKS_EBUSY", 7: "UGKS_ETIMEOUT", 8: "UGKS_ENOTFOUND"}


class UGKSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Mesh(ct.Structure):
    _fields_ = [("dim", ct.c_int32), ("n_cells", ct.c_int64), ("n_faces", ct.c_int64),
                ("cell_xc", D_P), ("cell_vol", D_P), ("face_cells", I64_P), ("face_n", D_P),
                ("face_S", D_P), ("face_xc", D_P), ("face_type", I32_P), ("face_tag", I32_P),
                ("face_shift", D_P)]


class VGrid(ct.Structure):
    _fields_ = [("dim", ct.c_int32), ("nv", ct.c_int64), ("u", D_P), ("w", D_P),
                ("cart_n", ct.c_int32 * 3)]


class Params(ct.Structure):
    _fields_ = [("Kn", ct.c_double), ("L_ref", ct.c_double), ("Pr", ct.c_double),
                ("omega", ct.c_double), ("cfl", ct.c_double), ("dt", ct.c_double),
                ("limiter", ct.c_int32), ("venkat_K", ct.c_double), ("n_walls", ct.c_int32),
                ("wall_T", D_P), ("wall_U", D_P), ("inf_rho", ct.c_double),
                ("inf_U", ct.c_double * 3), ("inf_T", ct.c_double), ("precision", ct.c_int32),
                ("prim_init", D_P), ("patch_cells", ct.c_int32), ("vtile", ct.c_int32),
                ("gather_threads", ct.c_int32), ("gather_tile_group", ct.c_int32), ("w0_analytic", ct.c_int32)]


ALLOC_FN = ct.CFUNCTYPE(ct.c_void_p, ct.c_void_p, ct.c_size_t, ct.c_void_p)
FREE_FN = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_void_p, ct.c_size_t, ct.c_void_p)


class Alloc(ct.Structure):
    _fields_ = [("ctx", ct.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class Info(ct.Structure):
    _fields_ = [("dim", ct.c_int32), ("ncomp", ct.c_int32), ("precision", ct.c_int32),
                ("n_cells", ct.c_int64), ("n_faces", ct.c_int64), ("nv", ct.c_int64),
                ("nv_pad", ct.c_int64), ("dt", ct.c_double), ("step", ct.c_int64),
                ("device_bytes", ct.c_size_t), ("f_bytes", ct.c_size_t), ("n_patches", ct.c_int32),
                ("patch_cells", ct.c_int32), ("vtile", ct.c_int32),
                ("kernel_launches_per_step", ct.c_int64), ("n_wall_faces", ct.c_int64),
                ("gather_threads", ct.c_int32), ("gather_tile_group", ct.c_int32)]


class Result(ct.Structure):
    _fields_ = [("state", ct.c_int32), ("status", ct.c_int32), ("steps", ct.c_int64),
                ("residual", ct.c_double * 5), ("t_arrive", ct.c_double), ("t_admit", ct.c_double),
                ("t_done", ct.c_double), ("footprint_bytes", ct.c_size_t), ("device_bytes", ct.c_size_t),
                ("n_cells", ct.c_int64), ("nv", ct.c_int64)]


class ServerStats(ct.Structure):
    _fields_ = [("device_budget", ct.c_size_t), ("device_used", ct.c_size_t), ("n_running", ct.c_int32),
                ("n_queued", ct.c_int32), ("total_cvu", ct.c_int64), ("clock", ct.c_double)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3

EXPORTS = {
    "ugks_create": (ct.c_int, [ct.POINTER(Mesh), ct.POINTER(VGrid), ct.POINTER(Params), ct.POINTER(Alloc),
                               ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    "ugks_step": (ct.c_int, [ct.c_void_p, ct.c_int32]),
    "ugks_check": (ct.c_int, [ct.c_void_p]),
    "ugks_density_range": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "ugks_moments": (ct.c_int, [ct.c_void_p, D_P, D_P, D_P, D_P]),
    "ugks_residual": (ct.c_int, [ct.c_void_p, D_P]),
    "ugks_get_state": (ct.c_int, [ct.c_void_p, D_P, D_P]),
    "ugks_set_state": (ct.c_int, [ct.c_void_p, D_P, D_P]),
    "ugks_get_state_f32": (ct.c_int, [ct.c_void_p, F_P, D_P]),
    "ugks_set_state_f32": (ct.c_int, [ct.c_void_p, F_P, D_P]),
    "ugks_get_cells": (ct.c_int, [ct.c_void_p, I64_P, ct.c_int64, D_P, D_P]),
    "ugks_wall_quantities": (ct.c_int, [ct.c_void_p, I64_P, D_P, D_P, D_P]),
    "ugks_info": (ct.c_int, [ct.c_void_p, ct.POINTER(Info)]),
    "ugks_profile_begin": (ct.c_int, [ct.c_void_p, ct.c_int32]),
    "ugks_profile_end": (ct.c_int, [ct.c_void_p, D_P, ct.c_int32, ct.POINTER(ct.c_int32)]),
    "ugks_residual_noalloc": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_int32, ct.c_void_p,
                                         ct.c_void_p]),
    "ugks_batch_create": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int32, ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    "ugks_batch_step": (ct.c_int, [ct.c_void_p, ct.c_int32]),
    "ugks_batch_destroy": (None, [ct.c_void_p]),
    "ugks_server_create": (ct.c_int, [ct.c_size_t, ct.c_int32, ct.c_int32, ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    "ugks_server_submit": (ct.c_int, [ct.c_void_p, ct.POINTER(Mesh), ct.POINTER(VGrid), ct.POINTER(Params),
                                      ct.c_double, ct.c_int64, ct.c_double, ct.POINTER(ct.c_uint64)]),
    "ugks_server_tick": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32)]),
    "ugks_server_poll": (ct.c_int, [ct.c_void_p, ct.c_uint64, ct.POINTER(Result)]),
    "ugks_server_moments": (ct.c_int, [ct.c_void_p, ct.c_uint64, D_P, D_P, D_P, D_P]),
    "ugks_server_stats": (ct.c_int, [ct.c_void_p, ct.POINTER(ServerStats)]),
    "ugks_server_destroy": (None, [ct.c_void_p]),
    "ugks_cfl_dt": (ct.c_int, [ct.POINTER(Mesh), ct.POINTER(VGrid), ct.c_double, ct.c_int64, D_P]),
    "ugks_set_owned": (ct.c_int, [ct.c_void_p, ct.c_int64]),
    "ugks_residual_sums": (ct.c_int, [ct.c_void_p, D_P]),
    "ugks_halo_row_bytes": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_size_t)]),
    "ugks_halo_set": (ct.c_int, [ct.c_void_p, ct.c_int32, I64_P, ct.c_int64]),
    "ugks_halo_pack": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p]),
    "ugks_halo_unpack": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p]),
    "ugks_destroy": (None, [ct.c_void_p]),
    "ugks_last_error": (ct.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
        L = ct.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code != 0:
        raise UGKSError(code, load().ugks_last_error().decode())


def _c(a, dt=np.float64):
    return np.ascontiguousarray(a, dtype=dt)


def _p(a, typ=D_P):
    return a.ctypes.data_as(typ) if a is not None else None


def make_structs(mesh, vgrid, params, init=None, precision=FP64, patch_cells=0, vtile=0, threads=0, tile_group=0):
    """Marshal the dicts of ``cases`` into ABI structs; returns (structs, keepalive)."""
    keep = []
    D = int(mesh["dim"])
    arr = {k: _c(mesh[k]) for k in ("cell_xc", "cell_vol", "face_n", "face_S", "face_xc", "face_shift")}
    arr["face_cells"] = _c(mesh["face_cells"], np.int64)
    arr["face_type"] = _c(mesh["face_type"], np.int32)
    arr["face_tag"] = _c(mesh["face_tag"], np.int32)
    keep.append(arr)
    m = Mesh(D, len(arr["cell_vol"]), len(arr["face_S"]), _p(arr["cell_xc"]), _p(arr["cell_vol"]),
             _p(arr["face_cells"], I64_P), _p(arr["face_n"]), _p(arr["face_S"]), _p(arr["face_xc"]),
             _p(arr["face_type"], I32_P), _p(arr["face_tag"], I32_P), _p(arr["face_shift"]))
    u, w = _c(vgrid["u"]), _c(vgrid["w"])
    keep += [u, w]
    cart = list(vgrid.get("cart_n", [0, 0, 0])) + [0, 0, 0]
    v = VGrid(D, len(w), _p(u), _p(w), (ct.c_int32 * 3)(*cart[:3]))
    walls = params.get("walls") or []
    wT = _c([wl["T"] for wl in walls] or [1.0])
    wU = _c([list(wl["U"]) + [0.0] * (3 - len(wl["U"])) for wl in walls] or [[0.0, 0.0, 0.0]])
    keep += [wT, wU]
    inf = params.get("inf") or {"rho": 1.0, "U": [0.0, 0.0, 0.0], "T": 1.0}
    iU = list(inf["U"]) + [0.0] * (3 - len(inf["U"]))
    ini = _c(init) if init is not None else None
    keep.append(ini)
    p = Params(params["Kn"], params.get("L_ref", 1.0), params["Pr"], params["omega"], params["cfl"],
               params.get("dt", 0.0), params.get("limiter", 1), params.get("venkat_K", 1.0), len(walls),
               _p(wT), _p(wU), inf["rho"], (ct.c_double * 3)(*iU), inf["T"], int(precision), _p(ini),
               int(patch_cells), int(vtile), int(threads), int(tile_group), int(params.get("w0_analytic", 0)))
    return (m, v, p), keep


def cfl_dt(mesh, vgrid, cfl, n_cells=None):
    """ugks_cfl_dt: the CFL step over the first ``n_cells`` cells (all by default)."""
    (m, v, _), keep = make_structs(mesh, vgrid, {"Kn": 1.0, "Pr": 1.0, "omega": 0.5, "cfl": cfl})
    dt = ct.c_double()
    n = len(mesh["cell_vol"]) if n_cells is None else int(n_cells)
    check(load().ugks_cfl_dt(ct.byref(m), ct.byref(v), float(cfl), n, ct.byref(dt)))
    return dt.value


class _TorchAllocator:
    """torch's caching allocator behind the ugks_alloc callbacks."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}

        def _alloc(ctx, nbytes, stream):
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0)
            self.live[ptr] = nbytes
            return ptr

        def _free(ctx, ptr, nbytes, stream):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = Alloc(None, self._a, self._f)


class Case:
    """A UGKS case resident on the GPU (one time step = ``ugks_step``)."""

    def __init__(self, mesh, vgrid, params, init=None, precision=FP64, stream=None, torch_alloc=True,
                 patch_cells=0, vtile=0, threads=0, tile_group=0):
        L = load()
        self.D = int(mesh["dim"])
        self.C = len(mesh["cell_vol"])
        self.Nv = len(vgrid["w"])
        self.nc = 2 if self.D == 2 else 1
        (m, v, p), keep = make_structs(mesh, vgrid, params, init, precision, patch_cells, vtile, threads,
                                       tile_group)
        self._keep = keep
        self._alloc = None
        if torch_alloc:
            import torch
            dev = torch.cuda.current_device()
            self._alloc = _TorchAllocator(dev)
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
        h = ct.c_void_p()
        check(L.ugks_create(ct.byref(m), ct.byref(v), ct.byref(p),
                            ct.byref(self._alloc.struct) if self._alloc else None,
                            ct.c_void_p(stream or 0), ct.byref(h)))
        self._h = h
        self.stream = stream

    def close(self):
        if getattr(self, "_h", None):
            load().ugks_destroy(self._h)
            self._h = None

    __del__ = close

    def step(self, n=1):
        check(load().ugks_step(self._h, int(n)))

    def check(self):
        check(load().ugks_check(self._h))

    def density_range(self):
        """(min rho, max rho) over the own cells of the current state."""
        r = np.zeros(2)
        check(load().ugks_density_range(self._h, r.ctypes.data))
        return float(r[0]), float(r[1])

    def info(self):
        i = Info()
        check(load().ugks_info(self._h, ct.byref(i)))
        return {k: getattr(i, k) for k, _ in Info._fields_}

    def moments(self):
        rho = np.empty(self.C)
        U = np.empty((self.C, self.D))
        T = np.empty(self.C)
        q = np.empty((self.C, self.D))
        check(load().ugks_moments(self._h, _p(rho), _p(U), _p(T), _p(q)))
        return rho, U, T, q

    def residual(self):
        r = np.empty(self.D + 2)
        check(load().ugks_residual(self._h, _p(r)))
        return r

    def state(self, with_f=True, f_dtype=np.float64):
        """(f[C][ncomp][nv], W[C][dim+2]) in mesh order; f as FP64, or as
        FP32 with ``f_dtype=np.float32`` (exact for FP32 storage)."""
        single = np.dtype(f_dtype) == np.float32
        f = np.empty((self.C, self.nc, self.Nv), np.float32 if single else np.float64) if with_f else None
        W = np.empty((self.C, self.D + 2))
        if single:
            check(load().ugks_get_state_f32(self._h, _p(f, F_P), _p(W)))
        else:
            check(load().ugks_get_state(self._h, _p(f), _p(W)))
        return f, W

    def wall_quantities(self):
        """Face ids and p_w, sigma_w, q_w of the last step at the wall faces
        (time averages over the step, Sec. 2.5)."""
        n = self.info()["n_wall_faces"]
        face = np.empty(n, dtype=np.int64)
        p, sg, q = np.empty(n), np.empty(n), np.empty(n)
        check(load().ugks_wall_quantities(self._h, face.ctypes.data_as(I64_P), _p(p), _p(sg), _p(q)))
        return face, p, sg, q

    def cells(self, ids, with_f=True):
        """f [n][ncomp][nv] and W [n][dim+2] of the caller cells ``ids``."""
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        f = np.empty((len(ids), self.nc, self.Nv)) if with_f else None
        W = np.empty((len(ids), self.D + 2))
        check(load().ugks_get_cells(self._h, ids.ctypes.data_as(I64_P), len(ids), _p(f), _p(W)))
        return f, W

    def set_state(self, f=None, W=None):
        """Replace f and/or W; an FP32 array f goes through the FP32 upload
        (half the bytes), any other through the FP64 one.  A page-locked f
        must stay unchanged until the next synchronising call."""
        Wa = _c(W) if W is not None else None
        if f is not None and np.asarray(f).dtype == np.float32:
            check(load().ugks_set_state_f32(self._h, _p(_c(f, np.float32), F_P), _p(Wa)))
        else:
            fa = _c(f) if f is not None else None
            check(load().ugks_set_state(self._h, _p(fa), _p(Wa)))

    def heat_flux(self):
        return self.moments()[3]

    # ---- domain decomposition (subdomain cases)
    def set_owned(self, n_owned):
        check(load().ugks_set_owned(self._h, int(n_owned)))

    def residual_sums(self):
        out = np.empty(2 * (self.D + 2))
        check(load().ugks_residual_sums(self._h, _p(out)))
        return out

    def halo_row_bytes(self):
        b = ct.c_size_t()
        check(load().ugks_halo_row_bytes(self._h, ct.byref(b)))
        return b.value

    def halo_set(self, slot, cells):
        ids = np.ascontiguousarray(cells, dtype=np.int64)
        check(load().ugks_halo_set(self._h, int(slot), ids.ctypes.data_as(I64_P), len(ids)))

    def halo_pack(self, slot, device_ptr):
        check(load().ugks_halo_pack(self._h, int(slot), ct.c_void_p(int(device_ptr))))

    def halo_unpack(self, slot, device_ptr):
        check(load().ugks_halo_unpack(self._h, int(slot), ct.c_void_p(int(device_ptr))))

    GROUPS = ("prep", "face", "wall", "gather", "update_W", "collide")

    def profile_begin(self, max_steps):
        check(load().ugks_profile_begin(self._h, int(max_steps)))

    def profile_end(self):
        ms = np.zeros(len(self.GROUPS))
        n = ct.c_int32()
        check(load().ugks_profile_end(self._h, _p(ms), len(ms), ct.byref(n)))
        return dict(zip(self.GROUPS, ms)), n.value


class Batch:
    """Several cases stepped together: one persistent gather launch over a
    (case, patch, velocity tile) work list per step, the whole step captured
    once as a CUDA graph (``ugks_batch_*``)."""

    def __init__(self, cases, stream=None):
        L = load()
        self.cases = list(cases)
        arr = (ct.c_void_p * len(self.cases))(*[c._h.value for c in self.cases])
        h = ct.c_void_p()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        check(L.ugks_batch_create(arr, len(self.cases), ct.c_void_p(stream or 0), ct.byref(h)))
        self._h = h
        self.stream = stream

    def step(self, n=1):
        check(load().ugks_batch_step(self._h, int(n)))

    def close(self):
        if getattr(self, "_h", None):
            load().ugks_batch_destroy(self._h)
            self._h = None

    __del__ = close


class Server:
    """Continuous-batching serving loop (``ugks_server_*``): submit cases with
    arrival times, call ``tick`` until everything is done, poll the results."""

    def __init__(self, budget_bytes, max_slots, steps_per_tick, stream=None):
        L = load()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = ct.c_void_p()
        check(L.ugks_server_create(int(budget_bytes), int(max_slots), int(steps_per_tick), ct.c_void_p(stream or 0),
                                   ct.byref(h)))
        self._h = h
        self.shapes = {}

    def submit(self, case, tol, max_steps, t_arrive=-1.0, precision=FP32, init=None):
        (m, v, p), keep = make_structs(case["mesh"], case["vgrid"], case["params"],
                                       case.get("init") if init is None else init, precision)
        t = ct.c_uint64()
        check(load().ugks_server_submit(self._h, ct.byref(m), ct.byref(v), ct.byref(p), float(tol), int(max_steps),
                                        float(t_arrive), ct.byref(t)))
        self.shapes[t.value] = (len(case["mesh"]["cell_vol"]), int(case["mesh"]["dim"]))
        return t.value

    def tick(self):
        r, q = ct.c_int32(), ct.c_int32()
        check(load().ugks_server_tick(self._h, ct.byref(r), ct.byref(q)))
        return r.value, q.value

    def poll(self, ticket):
        res = Result()
        check(load().ugks_server_poll(self._h, int(ticket), ct.byref(res)))
        out = {k: getattr(res, k) for k, _ in Result._fields_}
        out["residual"] = list(res.residual)
        return out

    def moments(self, ticket):
        C, D = self.shapes[ticket]
        rho, U, T, q = np.empty(C), np.empty((C, D)), np.empty(C), np.empty((C, D))
        check(load().ugks_server_moments(self._h, int(ticket), _p(rho), _p(U), _p(T), _p(q)))
        return rho, U, T, q

    def stats(self):
        st = ServerStats()
        check(load().ugks_server_stats(self._h, ct.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def run(self, timeout_s=600.0, idle_sleep=0.0005):
        """Tick until no request is running or queued (or the timeout)."""
        import time
        t0 = time.time()
        while time.time() - t0 < timeout_s:
            running, queued = self.tick()
            if running == 0 and queued == 0:
                return True
            if running == 0:
                time.sleep(idle_sleep)
        return False

    def close(self):
        if getattr(self, "_h", None):
            load().ugks_server_destroy(self._h)
            self._h = None

    __del__ = close
