"""Serving loop: continuous batching across dots, admission by device footprint, eviction.

Each request's result in the mix is compared with the same request solved alone through
pp_solve_window (mixed form, residual 1e-6): same number of roots and roots within 1e-6 Ha
(the eigenvalue tolerance of the mixed form; both sides are within ~1e-7 Ha of the exact
roots).  Requests are submitted in two waves so that the second wave arrives while the
first is on the GPU and joins its batches.
"""

import time

import numpy as np
import pytest

from synth.inputs import make_inputs

pytestmark = pytest.mark.gpu

OPTS = dict(order=2, select=0, res_tol=1e-6, max_iter=300)
DOTS = [(16, 64, 192, 4), (32, 128, 384, 3)]


@pytest.fixture(scope="module")
def dots_and_requests(cuda_lib):
    pp = cuda_lib
    inps = [make_inputs(o, v, Q, seed=sd, mode="perturbative") for (o, v, Q, sd) in DOTS]
    reqs = []
    for d, inp in enumerate(inps):
        dot = pp.Dot(inp, prec=pp.PP_BF16, **OPTS)
        try:
            dA, dS = dot.diagonal()
            r = (dA / dS).ravel()
            for pct, k, width in ((15, 4, 0.08), (25, 8, 0.1), (40, 4, 0.06)):
                w0 = float(np.percentile(r, pct))
                alone = dot.solve_window(w0, width, k)
                reqs.append(dict(dot=d, omega0=w0, delta=width, k=k, alone=alone))
        finally:
            dot.close()
    return pp, inps, reqs


def _run(pp, inps, reqs, budget, slots, workers):
    srv = pp.Server(budget, slots_per_dot=slots, nworkers=workers, prec=pp.PP_BF16, **OPTS)
    try:
        ids = [srv.add_dot(inp) for inp in inps]
        first, second = reqs[::2], reqs[1::2]
        rid = {}
        for r in first:
            rid[id(r)] = srv.submit(ids[r["dot"]], r["omega0"], r["delta"], r["k"])
        time.sleep(0.3)  # the second wave arrives while the first is running
        for r in second:
            rid[id(r)] = srv.submit(ids[r["dot"]], r["omega0"], r["delta"], r["k"])
        out = {id(r): srv.wait(rid[id(r)], r["k"], timeout_ms=240_000) for r in reqs}
        stats = srv.stats()
    finally:
        srv.close()
    return out, stats


def _compare(reqs, out):
    for r in reqs:
        got, want = out[id(r)], r["alone"]
        assert got is not None
        assert len(got["omega"]) == len(want["omega"])
        np.testing.assert_allclose(got["omega"], want["omega"], atol=1e-6, rtol=0)
        assert np.all(got["resid"] <= 1e-6)
        assert got["latency_ms"] >= got["queue_ms"] >= 0.0


def test_serving_mix_matches_alone(dots_and_requests):
    pp, inps, reqs = dots_and_requests
    out, stats = _run(pp, inps, reqs, budget=64 << 30, slots=4, workers=3)
    _compare(reqs, out)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["ctx_created"] == len(inps) and stats["ctx_evicted"] == 0
    assert stats["max_windows_per_step"] >= 2  # windows of different requests shared a step


def _min_budget(pp, inp, slots, **opts):
    """Smallest budget (to 1 MiB) at which the server admits this dot (add_dot refuses a dot
    whose estimated footprint alone exceeds the budget with PP_ENOMEM)."""
    lo, hi = 1 << 20, 1 << 40
    while hi - lo > (1 << 20):
        mid = (lo + hi) // 2
        srv = pp.Server(mid, slots_per_dot=slots, nworkers=1, **opts)
        try:
            srv.add_dot(inp)
            hi = mid
        except pp.PPError as e:
            assert e.status == pp.PP_ENOMEM
            lo = mid
        finally:
            srv.close()
    return hi


def test_serving_evicts_when_over_budget(dots_and_requests):
    """A budget that holds the larger dot but not both lets one dot be resident at a time:
    every switch evicts the idle one."""
    pp, inps, reqs = dots_and_requests
    budget = max(_min_budget(pp, inp, 2, prec=pp.PP_BF16, **OPTS) for inp in inps)
    out, stats = _run(pp, inps, reqs, budget=budget, slots=2, workers=2)
    _compare(reqs, out)
    assert stats["completed"] == len(reqs)
    assert stats["ctx_evicted"] >= 1 and stats["ctx_created"] >= 2
    assert stats["max_concurrent_dots"] == 1


def test_serving_rejects_bad_requests(cuda_lib):
    pp = cuda_lib
    inp = make_inputs(8, 24, 64, seed=0, mode="literal")
    srv = pp.Server(1 << 30, prec=pp.PP_BF16, **OPTS)
    try:
        did = srv.add_dot(inp)
        with pytest.raises(pp.PPError):
            srv.submit(did + 5, 1.0, 0.1, 4)
        with pytest.raises(pp.PPError):
            srv.submit(did, 1.0, 0.1, 0)
        with pytest.raises(pp.PPError):
            srv.submit(did, 1.0, -0.1, 4)  # negative width
    finally:
        srv.close()


def test_serving_refuses_dot_beyond_budget(cuda_lib):
    """Admission by footprint: a dot that cannot fit the whole budget is refused (PP_ENOMEM)."""
    pp = cuda_lib
    inp = make_inputs(16, 64, 192, seed=4, mode="perturbative")
    srv = pp.Server(1 << 20, prec=pp.PP_BF16, **OPTS)
    try:
        with pytest.raises(pp.PPError) as ei:
            srv.add_dot(inp)
        assert ei.value.status == pp.PP_ENOMEM
        assert "exceeds the serving budget" in ei.value.args[0]
    finally:
        srv.close()
