"""Parity on the paper's hypersonic cylinder setups with unstructured 2D
velocity meshes (Sec. 4, the two cylinder experiments): E1, Ma 5 at Kn 0.1
with the 2,060-triangle velocity mesh, and E2, Ma 15 at Kn 0.01 with the
3,420-triangle one (cases.cylinder_dvs_case).  A triangle velocity mesh is not
a tensor grid, so the face pass takes the general per-velocity sums.

FP64 path: every element of f, W and q within 1e-12 of max |x| after two
steps from a perturbed state on a 1,500-cell mesh, and at seeded sample cells
of the full-size 30k-cell mesh.  FP32-storage form: W within 1e-5 relative L2
after 100 steps from the blended start on a 1,000-cell mesh, and one step at
full size within 1e-5 (the bounds of the other FP32 parity tests).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2412_06546_gb300 import _lib, cases as cs  # noqa: E402

from test_gpu_fullsize import _sampled  # noqa: E402
from test_gpu_parity import _compare, _pair, _rel_l2  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2412_06546_gb300 import build
    build.build()
    oracle.build()


@pytest.mark.parametrize("which", ["E1", "E2"])
def test_dvs_cylinder_fp64_two_steps(which):
    case = cs.cylinder_dvs_case(which, n_cells=1500)
    assert len(case["vgrid"]["w"]) == (2060 if which == "E1" else 3420)
    o, g = _pair(case, perturb=0.05)
    o.step(2)
    g.step(2)
    _compare(o, g, what=f"cylinder {which} fp64")
    g.close()


@pytest.mark.parametrize("which", ["E1", "E2"])
def test_dvs_cylinder_fp32_100_steps(which):
    case = cs.cylinder_dvs_case(which, n_cells=1000)
    o = oracle.OracleCase(case["mesh"], case["vgrid"], case["params"], case["init"])
    g = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=_lib.FP32)
    o.step(100)
    g.step(100)
    g.check()
    _, Wo, _ = o.state()
    _, Wg = g.state()
    eW = _rel_l2(Wg, Wo)
    print(f"fp32 cylinder {which} 100 steps: W rel L2 {eW:.2e}")
    assert eW <= 1e-5
    g.close()


@pytest.mark.parametrize("which,precision", [("E1", _lib.FP32), ("E2", _lib.FP64)])
def test_dvs_cylinder_full_size_sampled(which, precision):
    case = cs.cylinder_dvs_case(which, n_cells=30000)
    e = _sampled(case, precision, 48, 21)
    if precision == _lib.FP64:
        assert max(e.values()) <= 1e-12, e
    else:
        assert e["f"] <= 1e-5 and e["f_l2"] <= 1e-5 and e["W"] <= 1e-5, e
