"""The bounded wait that guards the collision pass's bulk copies: waiting on a
phase that nothing completes gives up after its limit, reports it, and leaves
the GPU usable (a case steps correctly afterwards)."""
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


def test_wait_gives_up_after_its_limit():
    limit = 20_000_000                       # 20 ms
    done, ns = _lib.selftest_wait(limit)
    assert done == 0
    assert limit <= ns < 50 * limit
    case = cs.cavity_case()
    g = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=_lib.FP32)
    g.step(3)
    g.check()
    rho = g.moments()[0]
    assert np.isfinite(rho).all() and rho.min() > 0
    g.close()
