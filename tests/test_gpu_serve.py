"""Continuous-batching service: requests that arrive while others are on the
GPU are admitted as memory frees up, and each result is the same as the
request served alone."""
import numpy as np
import pytest

from paper_2111_11866_gb300 import _lib, serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_11866_gb300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _requests(n, rate, seed=7):
    sizes = [(16, 4), (20, 5), (24, 6), (18, 4), (22, 5), (26, 6), (16, 5), (28, 7)]
    t = serve.poisson_arrivals(rate, n, seed)
    out = []
    for k in range(n):
        e, f = sizes[k % len(sizes)]
        img, seeds, _ = synth.request_window(100 + k, e, f, nsteps=3)
        out.append(serve.Request(k, float(t[k]), img, seeds, 3))
    return out


def test_served_results_equal_alone_results():
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 5.0
    reqs = _requests(8, rate=1e6)            # all present at once
    # room for about two of the largest windows: later requests must queue
    budget = int(2.2 * _lib.Batch.window_bytes((28, 28, 28, 7), 1))
    with serve.Server(budget, 16, params=p, keep_results=True) as srv:
        stats = srv.run(reqs)
    s = stats.summary()
    assert s["served"] == 8 and s["failed"] == 0
    assert s["max_resident"] >= 2            # work of different requests overlapped
    assert s["refused_admissions"] > 0       # the budget held requests back
    assert s["p99_ms"] >= s["p50_ms"] > 0
    for r in reqs:
        assert r.state == "done"
        with _lib.Batch(1 << 28, 2, params=p) as b:
            wid = b.add(r.image, r.seeds, r.nsteps)
            for _ in range(r.nsteps):
                b.advance()
            alone = b.read_u(wid)
        np.testing.assert_array_equal(r.result, alone)


def test_horizon_stops_an_overloaded_service():
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 5.0
    reqs = _requests(8, rate=1e6)
    budget = int(1.2 * _lib.Batch.window_bytes((28, 28, 28, 7), 1))
    with serve.Server(budget, 16, params=p) as srv:
        stats = srv.run(reqs, horizon_s=0.0)
    assert stats.served == 0 and stats.iterations == 0
