"""ugks_density_range: the smallest and largest density over the own cells,
against the densities ugks_moments returns, for both storage precisions, with
and without an own-cell mask, and over a decomposed case."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2412_06546_gb300 import _lib, cases as cs, decompose as dc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2412_06546_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", [_lib.FP64, _lib.FP32])
def test_range_is_min_and_max_of_the_densities(precision):
    case = cs.cylinder_case(n_cells=1500, nvx=16, nvy=14, mach=3.0, start="impulsive")
    g = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=precision)
    g.step(20)
    rho = g.moments()[0]
    assert g.density_range() == (rho.min(), rho.max())
    n = 517
    g.set_owned(n)
    assert g.density_range() == (rho[:n].min(), rho[:n].max())
    g.set_owned(0)
    assert g.density_range() == (0.0, 0.0)
    g.close()


def test_range_of_a_decomposed_case():
    case = cs.cylinder_case(n_cells=1500, nvx=16, nvy=14, mach=3.0, start="impulsive")
    tiling = {"patch_cells": 32, "vtile": 64, "threads": 256, "tile_group": 1}
    dt = _lib.cfl_dt(case["mesh"], case["vgrid"], case["params"]["cfl"])
    case = dict(case, params=dict(case["params"], dt=dt))
    full = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=_lib.FP32, **tiling)
    dec = dc.DecomposedCase(case, 3, _lib.FP32, **tiling)
    full.step(5)
    dec.step(5)
    assert dec.density_range() == full.density_range()
    dec.close()
    full.close()
