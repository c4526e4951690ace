"""Serving loop (ugks_server_*): admission by device footprint, arrival times,
step limits, and each case's result identical alone and in the mix."""
import time

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


def _mix():
    return [cs.cavity_case(n=8, nv=12, Kn=0.5),
            cs.cylinder_case(n_cells=700, nvx=14, nvy=12, mach=2.0, Kn=1.0),
            cs.cavity_case(n=10, nv=16, Kn=0.2, lid=0.3),
            cs.cylinder_case(n_cells=1200, nvx=16, nvy=14, mach=1.5, Kn=0.5)]


def test_results_identical_alone_and_in_the_mix():
    specs = _mix()
    alone = []
    for c in specs:
        srv = _lib.Server(2 << 30, 8, 10)
        t = srv.submit(c, 1e-3, 200)
        assert srv.run(300)
        alone.append((srv.poll(t), srv.moments(t)))
        srv.close()
    srv = _lib.Server(2 << 30, 8, 10)
    tickets = [srv.submit(c, 1e-3, 200) for c in specs]
    assert srv.run(300)
    for t, (ra, ma) in zip(tickets, alone):
        r = srv.poll(t)
        assert r["state"] == _lib.REQ_DONE and r["steps"] == ra["steps"]
        for x, y in zip(srv.moments(t), ma):
            assert np.array_equal(x, y)
    srv.close()


def test_admission_by_footprint_and_step_limit():
    specs = _mix()[:3]
    srv = _lib.Server(1 << 40, 8, 10)
    probe = srv.submit(specs[0], 1e-12, 10)
    assert srv.run(120)
    fp = srv.poll(probe)
    assert fp["device_bytes"] <= fp["footprint_bytes"]
    assert fp["status"] == 5 and fp["steps"] == 10            # UGKS_ENOTCONVERGED at max_steps
    srv.close()
    # room for about one of these cases at a time
    budget = int(fp["footprint_bytes"] * 1.5)
    srv = _lib.Server(budget, 8, 10)
    small = [specs[0], specs[0], specs[0]]
    ts = [srv.submit(c, 1e-12, 30) for c in small]
    peak = 0
    while True:
        running, queued = srv.tick()
        peak = max(peak, running)
        assert srv.stats()["device_used"] <= budget
        if running == 0 and queued == 0:
            break
    assert peak == 1
    rs = [srv.poll(t) for t in ts]
    assert all(r["state"] == _lib.REQ_DONE for r in rs)
    assert rs[0]["t_done"] <= rs[1]["t_admit"] <= rs[1]["t_done"] <= rs[2]["t_admit"]
    srv.close()


def test_arrival_times_are_respected():
    c = cs.cavity_case(n=6, nv=10, Kn=1.0)
    srv = _lib.Server(1 << 34, 4, 5)
    t_now = srv.stats()["clock"]
    t1 = srv.submit(c, 1e-12, 10, t_arrive=t_now + 0.5)
    r, q = srv.tick()
    assert r == 0 and q == 1 and srv.poll(t1)["state"] == _lib.REQ_QUEUED
    assert srv.run(60)
    res = srv.poll(t1)
    assert res["t_admit"] >= res["t_arrive"] >= t_now + 0.5 - 1e-9
    srv.close()
