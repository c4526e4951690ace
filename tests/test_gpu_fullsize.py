"""Sampled parity at the full workload sizes: the 30k-triangle Mach-5 cylinder
(60x50 velocities) in the benchmark's launch configuration (FP32 storage,
autotuned tiling), the 147k-tetrahedron Mach-4 sphere (28^3 velocities) and
the 1.05M-tetrahedron Mach-8 X38-like body (4,548 unstructured velocities)
in both forms.  The GPU state on two face rings around seeded sample cells is
read back with ugks_get_cells and stepped once by the oracle on the local
problem (cases.local_problem, pinned on CPU by test_local_problem.py); the
oracle's result at the sample cells is compared element by element with the
GPU's own step there.

Tolerances: FP64 path 1e-12 of max |x| per element.  FP32-storage form, one
step from the same (FP32-representable) state: the per-velocity arithmetic
is FP32 with the hardware 2^x (relative error about 2^-22), so f carries
relative errors of order 1e-6; the bound is 1e-5 of max |f| per element and
1e-5 relative L2, and W (FP64 accumulation of FP32 flux moments) 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2412_06546_gb300 import _lib, cases as cs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2412_06546_gb300 import build
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def sphere():
    return cs.sphere_case()


def _sampled(case, precision, n_sample, seed, steps_before=2, **tiling):
    mesh, vg, pr, init = case["mesh"], case["vgrid"], case["params"], case["init"]
    g = _lib.Case(mesh, vg, pr, init, precision=precision, **tiling)
    g.step(steps_before)
    sample = cs.pick_sample(mesh, n_sample, seed)
    sub, s2, pos = cs.local_problem(mesh, sample)
    fn, Wn = g.cells(s2)
    g.step(1)
    f1, W1 = g.cells(sample)
    dt = g.info()["dt"]
    g.close()
    o = oracle.OracleCase(sub, vg, dict(pr, dt=dt), np.asarray(init)[s2], n_threads=0)
    o.set_state(fn, Wn)
    o.step(1)
    fo, Wo, _ = o.state()
    fo, Wo = fo[pos], Wo[pos]
    return {"f": np.abs(f1 - fo).max() / np.abs(fo).max(),
            "f_l2": np.linalg.norm(f1 - fo) / np.linalg.norm(fo),
            "W": np.abs(W1 - Wo).max() / np.abs(Wo).max()}


def test_cylinder_full_size_fp32_bench_configuration():
    case = cs.cylinder_case(n_cells=30000, nvx=60, nvy=50, mach=5.0, Kn=0.1, seed=2)
    e = _sampled(case, _lib.FP32, 64, 11)
    assert e["f"] <= 1e-5 and e["f_l2"] <= 1e-5 and e["W"] <= 1e-5, e


def test_sphere_full_size_fp32(sphere):
    e = _sampled(sphere, _lib.FP32, 48, 12)
    assert e["f"] <= 1e-5 and e["f_l2"] <= 1e-5 and e["W"] <= 1e-5, e


def test_sphere_full_size_fp64(sphere):
    e = _sampled(sphere, _lib.FP64, 48, 13, patch_cells=16, vtile=32)
    assert max(e.values()) <= 1e-12, e


@pytest.fixture(scope="module")
def x38():
    return cs.x38_case()


def test_x38_full_size_fp32(x38):
    e = _sampled(x38, _lib.FP32, 48, 14)
    assert e["f"] <= 1e-5 and e["f_l2"] <= 1e-5 and e["W"] <= 1e-5, e


def test_x38_full_size_fp64(x38):
    e = _sampled(x38, _lib.FP64, 48, 15, patch_cells=16, vtile=32)
    assert max(e.values()) <= 1e-12, e
