"""pp_metric_noalloc (the allocation-free metric product) against pp_sigma's metric output.

Both compute Sigma z in FP64 through the C ABI with device pointers; the no-allocation
entry point takes its intermediates from the library's fixed scratch array.  Checked:
two calls in a row agree with pp_sigma, the device's free memory does not change across
calls once the first-call set-up has run, and a batch beyond the scratch limit is
rejected with a clear error.  Self-contained (own context), so it passes alone or after
the rest of the suite.
"""

import numpy as np
import pytest

from synth.inputs import make_inputs, random_vectors

pytestmark = pytest.mark.gpu

O, V, Q = 32, 128, 384
TOL = 1e-13  # same FP64 operations in both entry points; only summation order may differ


def _rel(a, b):
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("order", [2, 1])
def test_noalloc_metric_matches_pp_sigma(cuda_lib, order):
    import torch

    pp = cuda_lib
    inp = make_inputs(O, V, Q, seed=5, mode="perturbative")
    dot = pp.Dot(inp, order=order)
    try:
        nvec = 6
        Z = torch.from_numpy(random_vectors(nvec, O, V, seed=11)).cuda()
        _, want = pp.pp_sigma(dot.ctx, Z, pp.PP_FP64, metric=True)
        out1 = torch.full_like(Z, float("nan"))
        out2 = torch.full_like(Z, float("nan"))
        warm = torch.empty_like(Z)
        empty = torch.empty((0, 2, O, V), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()  # the library runs on its own stream
        pp.pp_metric_noalloc(dot.ctx, empty, empty)  # first-call set-up only
        pp.pp_metric_noalloc(dot.ctx, Z, warm)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        pp.pp_metric_noalloc(dot.ctx, Z, out1)
        pp.pp_metric_noalloc(dot.ctx, Z, out2)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0
        assert torch.isfinite(out1).all() and torch.isfinite(out2).all()
        assert _rel(out1, want) <= TOL
        assert _rel(out2, want) <= TOL
        if order == 1:  # Sigma = diag(1, -1) exactly
            sign = torch.tensor([1.0, -1.0], dtype=torch.float64, device="cuda").view(1, 2, 1, 1)
            assert torch.equal(out1, Z * sign)
    finally:
        dot.close()


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
            pp.pp_metric_noalloc(dot.ctx, Z, out)
        assert ei.value.status == pp.PP_EINVAL
        assert "exceeds" in str(ei.value)
        assert bool((out == 7.0).all())  # nothing was written
        # the largest allowed batch still runs
        n_ok = pp.PP_METRIC_NOALLOC_MAX_ELEMS // (O * V)
        Zs = torch.from_numpy(random_vectors(n_ok, O, V, seed=12)).cuda()
        o2 = torch.empty_like(Zs)
        pp.pp_metric_noalloc(dot.ctx, Zs, o2)
        _, want = pp.pp_sigma(dot.ctx, Zs, pp.PP_FP64, metric=True)
        assert _rel(o2, want) <= TOL
    finally:
        dot.close()
