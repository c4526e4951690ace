"""ugks_residual_noalloc: the residual of two device-resident states, computed
without allocating device memory (for callers that cannot call cudaMalloc,
e.g. code under an external memory manager that has reserved the device or a
serving loop with a fixed device budget).  Its result must match the residual
ugks_residual reports for the same step, call after call, although every call
reuses one fixed scratch array.

This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import ctypes as ct

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2412_06546_gb300 import _lib, cases as cs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2412_06546_gb300 import build
    build.build()


def _noalloc_residual(W_old, W_new, dim):
    L = _lib.load()
    a = torch.from_numpy(np.ascontiguousarray(W_old)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(W_new)).cuda()
    res = torch.full((dim + 2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    code = L.ugks_residual_noalloc(ct.c_void_p(a.data_ptr()), ct.c_void_p(b.data_ptr()), len(W_old), dim,
                                   ct.c_void_p(res.data_ptr()), ct.c_void_p(stream))
    _lib.check(code)
    torch.cuda.synchronize()
    return res.cpu().numpy()


@pytest.mark.parametrize("dim", [2, 3])
def test_matches_ugks_residual_on_consecutive_calls(dim):
    if dim == 2:
        case = cs.cylinder_case(n_cells=1500, nvx=16, nvy=14)
    else:
        case = cs.sphere_case(n_cells=2000, nv=8, vmax=8.0, mach=2.0)
    g = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=_lib.FP32)
    for _ in range(2):                                  # two calls in a row, different data
        _, W_old = g.state(with_f=False)
        g.step(1)
        _, W_new = g.state(with_f=False)
        ref = g.residual()
        got = _noalloc_residual(W_old, W_new, dim)
        assert np.all(np.isfinite(got)) and np.all(ref > 0)
        assert np.allclose(got, ref, rtol=1e-12, atol=0), (got, ref)
    g.close()


def test_rejects_sizes_beyond_the_fixed_limit():
    L = _lib.load()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ct.c_void_p(dummy.data_ptr())
    code = L.ugks_residual_noalloc(p, p, 2_097_153, 2, p, None)
    assert code == 1 and b"exceeds the fixed scratch limit" in L.ugks_last_error()


def test_exactly_the_cell_limit_uses_the_last_scratch_row():
    """At n_cells = 2,097,152 every row of the fixed scratch array holds a
    block's partial sums.  The last cell carries most of the change, so a lost
    or misplaced last block would change the result far beyond the tolerance.
    Two calls in a row (3D, then 2D) against numpy on the same device arrays."""
    n = 2_097_152
    rng = np.random.default_rng(11)
    for dim in (3, 2):
        M = dim + 2
        W_old = 1.0 + rng.random((n, M))
        W_new = W_old + 1e-6 * rng.standard_normal((n, M))
        W_new[-1] += 1.0
        got = _noalloc_residual(W_old, W_new, dim)
        d = W_new - W_old
        ref = np.sqrt((d * d).sum(axis=0)) / np.sqrt((W_old * W_old).sum(axis=0))
        assert np.allclose(got, ref, rtol=1e-10, atol=0), (dim, got, ref)
