"""State upload and download through the C ABI: the FP64 and FP32 forms of
ugks_set_state / ugks_get_state, from pageable and page-locked host memory.

The upload is staged in chunks of cells through two slots of the f_nxt
buffer, with the copies on a stream of the case overlapping the reordering of
earlier chunks.  These tests check that every cell lands in place (exact
round trips, for both the caller's cell order and the padded velocity rows),
that a step after an FP32 upload is bit-identical to a step after the FP64
upload of the same values, and that a state uploaded right after queued steps
replaces the state those steps produced (the first copy waits for them).
"""
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


def _case(precision, **kw):
    c = cs.cylinder_case(n_cells=1500, nvx=18, nvy=15, mach=3.0)
    return c, _lib.Case(c["mesh"], c["vgrid"], c["params"], c["init"], precision=precision, **kw)


def _random_state(g, seed):
    f, W = g.state()
    f = f * cs.perturbation(f.shape, seed, 0.1)
    return f, W


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("precision", [_lib.FP32, _lib.FP64])
@pytest.mark.parametrize("pinned", [False, True])
def test_fp32_round_trip_is_exact(precision, pinned):
    _, g = _case(precision)
    f, W = _random_state(g, 3)
    f32 = f.astype(np.float32)
    g.set_state(_pinned(f32) if pinned else f32, W)
    f_back32, W_back = g.state(f_dtype=np.float32)
    f_back64, _ = g.state()
    assert f_back32.dtype == np.float32
    assert np.array_equal(f_back32, f32)
    assert np.array_equal(f_back64, f32.astype(np.float64))
    assert np.array_equal(W_back, W)
    g.close()


@pytest.mark.parametrize("pinned", [False, True])
def test_fp64_round_trip_is_exact_for_the_fp64_form(pinned):
    _, g = _case(_lib.FP64)
    f, W = _random_state(g, 4)
    g.set_state(_pinned(f) if pinned else f, W)
    f_back, W_back = g.state()
    assert np.array_equal(f_back, f) and np.array_equal(W_back, W)
    f32, _ = g.state(f_dtype=np.float32)
    assert np.array_equal(f32, f.astype(np.float32))
    g.close()


def test_fp32_and_fp64_uploads_step_identically():
    _, a = _case(_lib.FP32)
    _, b = _case(_lib.FP32)
    f, W = _random_state(a, 5)
    f32 = f.astype(np.float32)
    a.set_state(f32, W)
    b.set_state(f32.astype(np.float64), W)
    a.step(3)
    b.step(3)
    fa, Wa = a.state(f_dtype=np.float32)
    fb, Wb = b.state(f_dtype=np.float32)
    assert np.array_equal(fa, fb) and np.array_equal(Wa, Wb)
    assert np.array_equal(a.residual(), b.residual())
    a.close()
    b.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_upload_after_queued_steps_replaces_their_result(dtype):
    """Steps are queued without a host wait, then the state is replaced from
    page-locked memory: the upload (on its own stream) must wait for them, so
    the result is the uploaded state stepped once, as on a fresh case."""
    _, a = _case(_lib.FP32)
    _, b = _case(_lib.FP32)
    f, W = _random_state(a, 6)
    fh = _pinned(f.astype(dtype))
    a.step(20)                          # queued, not waited for
    a.set_state(fh, W)
    a.step(1)
    b.set_state(fh, W)
    b.step(1)
    fa, Wa = a.state(f_dtype=np.float32)
    fb, Wb = b.state(f_dtype=np.float32)
    assert np.array_equal(fa, fb) and np.array_equal(Wa, Wb)
    a.close()
    b.close()


def test_small_case_with_fewer_cells_than_chunks():
    c = cs.cavity_case(n=1, nv=8)
    g = _lib.Case(c["mesh"], c["vgrid"], c["params"], c["init"], precision=_lib.FP32)
    f, W = g.state(f_dtype=np.float32)
    f2 = (f * 1.5).astype(np.float32)
    g.set_state(_pinned(f2), W * np.array([1.5, 1.5, 1.5, 1.5]))
    f_back, _ = g.state(f_dtype=np.float32)
    assert np.array_equal(f_back, f2)
    g.close()


@pytest.mark.parametrize("n", [1, 2, 3])
def test_fp64_state_io_of_tiny_fp32_cases(n):
    """One to three cells in FP32 storage through the FP64 calls.  A cell's
    FP64 row (99 velocities: 1,584 B) is larger than its FP32 row (padded
    to 128: 1,024 B), so it would not fit one FP32 copy of f (n = 1) or one
    of the two upload slots (n = 2, 3): the staging area is sized for FP64
    rows.  Round trips through ugks_set_state, ugks_get_state and
    ugks_get_cells are exact, and the case steps."""
    mesh = cs.quad_mesh(n, 1, left=("wall", 0), right=("wall", 0), bottom=("wall", 0), top=("wall", 0))
    case = {"mesh": mesh, "vgrid": cs.cartesian_vgrid((11, 9), (-5, -5), (5, 5)),
            "params": cs.params(0.5, walls=[{"T": 1.0, "U": [0, 0, 0]}]), "init": cs.uniform_state(n, 2)}
    g = _lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=_lib.FP32)
    assert g.info()["nv_pad"] == 128
    f, W = g.state()
    f2 = (f * cs.perturbation(f.shape, 7, 0.1)).astype(np.float32).astype(np.float64)
    g.set_state(f2, W)
    fb, Wb = g.state()
    assert np.array_equal(fb, f2) and np.array_equal(Wb, W)
    fc, Wc = g.cells(np.arange(n)[::-1])
    assert np.array_equal(fc, f2[::-1]) and np.array_equal(Wc, W[::-1])
    g.step(2)
    g.check()
    g.close()
