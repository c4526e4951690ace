"""The C ABI: the library loads, exports every entry point declared in
include/ugks.h, and the ctypes structs match the C layout (no GPU needed)."""
import ctypes as ct
import os
import re
import subprocess
import tempfile

import numpy as np

import pytest

from paper_2412_06546_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ugks.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ugks_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "ugks_create" in names and "ugks_step" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(_lib.EXPORTS), set(names) - set(_lib.EXPORTS)


def test_struct_layout_matches_header():
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "ugks.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(ugks_mesh), sizeof(ugks_vgrid), sizeof(ugks_params),
         sizeof(ugks_alloc), sizeof(ugks_info_t));
  printf("%zu %zu %zu %zu\n", offsetof(ugks_params, precision), offsetof(ugks_params, prim_init),
         offsetof(ugks_params, vtile), offsetof(ugks_info_t, kernel_launches_per_step));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    assert sizes[:5] == [ct.sizeof(_lib.Mesh), ct.sizeof(_lib.VGrid), ct.sizeof(_lib.Params),
                         ct.sizeof(_lib.Alloc), ct.sizeof(_lib.Info)]
    assert sizes[5:] == [_lib.Params.precision.offset, _lib.Params.prim_init.offset,
                         _lib.Params.vtile.offset, _lib.Info.kernel_launches_per_step.offset]


def _bad_inputs():
    from paper_2412_06546_gb300 import cases
    base = cases.cavity_case(n=3, nv=4)

    def with_mesh(**kw):
        m = {k: (v.copy() if hasattr(v, "copy") else v) for k, v in base["mesh"].items()}
        for k, f in kw.items():
            f(m)
        return m, base["vgrid"], base["params"]

    def neg_vol(m):
        m["cell_vol"][1] = -1.0

    def bad_owner(m):
        m["face_cells"][0, 0] = 99

    def bad_neighbour(m):
        i = int(np.nonzero(np.asarray(m["face_type"]) == 0)[0][0])
        m["face_cells"][i, 1] = -5

    def bad_tag(m):
        i = int(np.nonzero(np.asarray(m["face_type"]) == 1)[0][0])
        m["face_tag"][i] = 7

    vg_empty = {"dim": 2, "u": np.zeros((0, 2)), "w": np.zeros(0), "cart_n": [0, 0, 0]}
    return {
        "volume": with_mesh(v=neg_vol),
        "owner out of range": with_mesh(o=bad_owner),
        "neighbour out of range": with_mesh(n=bad_neighbour),
        "wall tag": with_mesh(t=bad_tag),
        "velocity count": (base["mesh"], vg_empty, base["params"]),
        "cfl > 0 or dt > 0": (base["mesh"], base["vgrid"], dict(base["params"], cfl=0.0, dt=0.0)),
        "Kn > 0": (base["mesh"], base["vgrid"], dict(base["params"], Kn=-1.0)),
    }


@pytest.mark.parametrize("what", list(_bad_inputs().keys()))
def test_errors_are_reported_without_a_gpu(lib, what):
    """Invalid input is rejected with UGKS_EINVAL and a message before any
    device call."""
    from paper_2412_06546_gb300 import cases
    mesh, vg, pr = _bad_inputs()[what]
    init = cases.uniform_state(len(mesh["cell_vol"]), 2)
    (m, v, p), keep = _lib.make_structs(mesh, vg, pr, init)
    h = ct.c_void_p()
    code = lib.ugks_create(ct.byref(m), ct.byref(v), ct.byref(p), None, None, ct.byref(h))
    assert code == 1 and what.encode() in lib.ugks_last_error(), lib.ugks_last_error()
    assert not h.value


def test_empty_mesh_is_rejected(lib):
    from paper_2412_06546_gb300 import cases
    case = cases.cavity_case(n=3, nv=4)
    (m, v, p), keep = _lib.make_structs(case["mesh"], case["vgrid"], case["params"], case["init"])
    m.n_cells = 0
    h = ct.c_void_p()
    assert lib.ugks_create(ct.byref(m), ct.byref(v), ct.byref(p), None, None, ct.byref(h)) == 1
    assert b"n_cells > 0" in lib.ugks_last_error() and not h.value


def test_no_cpu_fallback_without_library(tmp_path):
    with pytest.raises(RuntimeError, match="not built"):
        saved = _lib._lib
        try:
            _lib._lib = None
            _lib.load(str(tmp_path / "missing.so"))
        finally:
            _lib._lib = saved


@pytest.mark.parametrize("precision,threads,vtile,msg", [
    (_lib.FP32, 128, 0, b"gather_threads must be 0, 256 or 512"),
    (_lib.FP64, 512, 0, b"gather_threads = 512 needs UGKS_FP32"),
    (_lib.FP32, 512, 128, b"gather_threads = 512 needs UGKS_FP32"),
])
def test_gather_block_size_is_validated(lib, precision, threads, vtile, msg):
    from paper_2412_06546_gb300 import cases
    case = cases.cavity_case(n=3, nv=4)
    (m, v, p), keep = _lib.make_structs(case["mesh"], case["vgrid"], case["params"], case["init"],
                                        precision, 0, vtile, threads)
    h = ct.c_void_p()
    assert lib.ugks_create(ct.byref(m), ct.byref(v), ct.byref(p), None, None, ct.byref(h)) == 1
    assert msg in lib.ugks_last_error() and not h.value


@pytest.mark.parametrize("group", [-1, 1025])
def test_gather_tile_group_is_validated(lib, group):
    from paper_2412_06546_gb300 import cases
    case = cases.cavity_case(n=3, nv=4)
    (m, v, p), keep = _lib.make_structs(case["mesh"], case["vgrid"], case["params"], case["init"],
                                        _lib.FP32, 0, 0, 0, group)
    h = ct.c_void_p()
    assert lib.ugks_create(ct.byref(m), ct.byref(v), ct.byref(p), None, None, ct.byref(h)) == 1
    assert b"gather_tile_group must be in [0, 1024]" in lib.ugks_last_error() and not h.value
