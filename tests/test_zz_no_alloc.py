"""pp_metric_noalloc, the metric product for callers that cannot allocate device memory.

Some callers must not allocate GPU memory at the moment they need Sigma z: code that
runs inside another framework's memory pool (a raw cudaMalloc would escape the pool's
budget), or a latency-critical loop that avoids cudaMalloc/cudaFree because they can
synchronise the device.  This entry point keeps its intermediates in a fixed scratch
array compiled into the library.  Checked here, through the C ABI with device pointers:

* two calls in a row equal the CPU oracle's metric (FP64 context, 1e-12 relative) and
  pp_sigma's metric output of the same context (1e-13: same FP64 operations);
* the first-call set-up loads every kernel a call launches: in a fresh process with
  lazy module loading, on a mixed-precision context that has never run an FP64 GEMM,
  the device's free memory does not change across the first non-empty call;
* a batch beyond the scratch limit, a wrong shape and a wrong device are rejected.

This file is collected last on purpose (it is self-contained and passes alone or after
the rest of the suite).
"""

import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from synth.inputs import make_inputs, random_vectors

pytestmark = pytest.mark.gpu

O, V, Q = 32, 128, 384
TOL_SAME = 1e-13  # same FP64 operations in both entry points; only summation order may differ
TOL_ORACLE = 1e-12  # FP64 context against the FP64 CPU oracle
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("order", [2, 1])
def test_noalloc_metric_matches_oracle(cuda_lib, order):
    import torch

    from oracle import pp_oracle as po

    pp = cuda_lib
    inp = make_inputs(O, V, Q, seed=5, mode="perturbative")
    dot = pp.Dot(inp, order=order)
    try:
        nvec = 6
        Zh = random_vectors(nvec, O, V, seed=11)
        want = po.SigmaRef(inp.eps, inp.B, O, order=order).metric(Zh)
        Z = torch.from_numpy(Zh).cuda()
        _, same = pp.pp_sigma(dot.ctx, Z, pp.PP_FP64, metric=True)
        out1 = torch.full_like(Z, float("nan"))
        out2 = torch.full_like(Z, float("nan"))
        empty = torch.empty((0, 2, O, V), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()  # the library runs on its own stream
        dot.metric_noalloc(empty, empty)  # first-call set-up only
        dot.metric_noalloc(Z, out1)
        dot.metric_noalloc(Z, out2)
        torch.cuda.synchronize()
        for out in (out1, out2):
            got = out.cpu().numpy()
            assert np.isfinite(got).all()
            assert _rel(got, want) <= TOL_ORACLE
            assert _rel(got, same.cpu().numpy()) <= TOL_SAME
        if order == 1:  # Sigma = diag(1, -1) exactly
            sign = np.array([1.0, -1.0]).reshape(1, 2, 1, 1)
            np.testing.assert_array_equal(out1.cpu().numpy(), Zh * sign)
    finally:
        dot.close()


_FRESH = textwrap.dedent(
    """
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch
    import paper_2512_09811_gb300 as pp
    from oracle import pp_oracle as po
    from synth.inputs import make_inputs, random_vectors

    O, V, Q = {o}, {v}, {q}
    pp.load()
    torch.cuda.init()
    inp = make_inputs(O, V, Q, seed=5, mode="perturbative")
    dot = pp.Dot(inp, order=2, prec=pp.PP_BF16)  # mixed context: its precompute runs no FP64 GEMM
    Zh = random_vectors(4, O, V, seed=13)
    Z = torch.from_numpy(Zh).cuda()
    out1 = torch.empty_like(Z)
    out2 = torch.empty_like(Z)
    empty = torch.empty((0, 2, O, V), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    dot.metric_noalloc(empty, empty)  # set-up: address lookup and kernel loading
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    dot.metric_noalloc(Z, out1)  # first real call: must load and allocate nothing
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    dot.metric_noalloc(Z, out2)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free1 == free0 and free2 == free0, (free0, free1, free2)
    _, same = pp.pp_sigma(dot.ctx, Z, pp.PP_FP64, metric=True)
    ref = po.SigmaRef(inp.eps, inp.B, O, order=2).metric(Zh)
    for out in (out1, out2):
        got = out.cpu().numpy()
        assert np.linalg.norm(got - same.cpu().numpy()) <= 1e-13 * np.linalg.norm(got)
        # the mixed context's second-order densities carry ~1e-6 relative error
        assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)
    # a mis-shaped tensor is refused before the library sees it
    bad = torch.empty((4, 2, O, V + 1), dtype=torch.float64, device="cuda")
    try:
        dot.metric_noalloc(bad, bad)
        raise SystemExit("mis-shaped tensor accepted")
    except ValueError:
        pass
    dot.close()
    print("fresh-process no-alloc check ok")
    """
)


def test_noalloc_setup_loads_everything_fresh_process(cuda_lib):
    env = dict(os.environ, CUDA_MODULE_LOADING="LAZY")
    code = _FRESH.format(root=ROOT, o=O, v=V, q=Q)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "fresh-process no-alloc check ok" in r.stdout


def test_noalloc_rejects_batch_beyond_scratch(cuda_lib):
    import torch

    pp = cuda_lib
    inp = make_inputs(O, V, Q, seed=5, mode="perturbative")
    dot = pp.Dot(inp, order=2)
    try:
        nvec = pp.PP_METRIC_NOALLOC_MAX_ELEMS // (O * V) + 1
        Z = torch.zeros((nvec, 2, O, V), dtype=torch.float64, device="cuda")
        out = torch.full_like(Z, 7.0)
        torch.cuda.synchronize()
        with pytest.raises(pp.PPError) as ei:
            dot.metric_noalloc(Z, out)
        assert ei.value.status == pp.PP_EINVAL
        assert "exceeds" in str(ei.value)
        assert bool((out == 7.0).all())  # nothing was written
        # the largest allowed batch still runs
        n_ok = pp.PP_METRIC_NOALLOC_MAX_ELEMS // (O * V)
        Zs = torch.from_numpy(random_vectors(n_ok, O, V, seed=12)).cuda()
        o2 = torch.empty_like(Zs)
        dot.metric_noalloc(Zs, o2)
        _, want = pp.pp_sigma(dot.ctx, Zs, pp.PP_FP64, metric=True)
        torch.cuda.synchronize()
        assert _rel(o2.cpu().numpy(), want.cpu().numpy()) <= TOL_SAME
    finally:
        dot.close()
