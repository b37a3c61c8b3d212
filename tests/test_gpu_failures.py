"""Failure paths of the C ABI: each status code is produced by a real condition, on the host
side of the library or by the solver, never by faulting the GPU.

* PP_EMETRIC: at the literal width sigma_B = 0.05 the 16/64/192 dot leaves the perturbative
  regime: the second-order metric S = 1 + S(2) has negative diagonal entries (diag(S) down to
  -12.4 in the FP64 oracle), so pp_create refuses the context in either arithmetic.
* PP_ENOTCONV: a window solve capped at one iteration returns its best estimates (residuals
  above the tolerance) with PP_ENOTCONV, and the context stays usable.
* PP_ENOMEM (serving admission) is covered in test_gpu_serving.py; PP_EINVAL in
  test_capi_abi.py and here for the window arguments.
"""

import numpy as np
import pytest

from oracle import pp_oracle as po
from synth.inputs import make_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec_name", ["PP_FP64", "PP_BF16"])
def test_create_refuses_indefinite_metric(cuda_lib, prec_name):
    pp = cuda_lib
    inp = make_inputs(16, 64, 192, seed=0, mode="literal")
    dA, dS = po.SigmaRef(inp.eps, inp.B, inp.nocc, order=2).diag()
    assert dS.min() < 0  # the oracle agrees that S is not positive definite here
    with pytest.raises(pp.PPError) as ei:
        pp.Dot(inp, order=2, prec=getattr(pp, prec_name))
    assert ei.value.status == pp.PP_EMETRIC
    assert "not positive" in str(ei.value)
    # the same dot at first order (S = 1) is accepted
    d1 = pp.Dot(inp, order=1, prec=getattr(pp, prec_name))
    d1.close()


def test_solve_reports_not_converged(cuda_lib):
    pp = cuda_lib
    inp = make_inputs(32, 128, 384, seed=3, mode="perturbative")
    dot = pp.Dot(inp, prec=pp.PP_BF16, order=2, select=0, res_tol=1e-6, max_iter=1)
    try:
        dA, dS = dot.diagonal()
        w0 = float(np.percentile((dA / dS).ravel(), 20))
        with pytest.raises(pp.PPError) as ei:
            dot.solve_window(w0, 0.1, 4)
        assert ei.value.status == pp.PP_ENOTCONV
        out = dot.solve_window(w0, 0.1, 4, allow_notconv=True)
        assert out["status"] == pp.PP_ENOTCONV
        n = len(out["omega"])
        assert 0 <= n <= 4
        assert np.all(np.isfinite(out["omega"])) and np.all(np.isfinite(out["resid"]))
        assert n == 0 or out["resid"].max() > 1e-6  # best estimates, not converged roots
        st = dot.stats()
        assert 1 <= st["iterations"] <= 2  # the initial block's step and the one iteration
    finally:
        dot.close()
    # a fresh context with the default iteration cap converges on the same window
    dot = pp.Dot(inp, prec=pp.PP_BF16, order=2, select=0, res_tol=1e-6, max_iter=300)
    try:
        out = dot.solve_window(w0, 0.1, 4)
        assert out["status"] == pp.PP_OK and len(out["omega"]) == 4
        assert np.all(out["resid"] <= 1e-6)
    finally:
        dot.close()


def test_window_arguments_rejected(cuda_lib):
    pp = cuda_lib
    inp = make_inputs(8, 24, 64, seed=0, mode="literal")
    dot = pp.Dot(inp, order=2)
    try:
        for args in ((1.0, -0.1, 4), (float("nan"), 0.1, 4), (1.0, 0.1, 0)):
            with pytest.raises(pp.PPError) as ei:
                dot.solve_window(*args)
            assert ei.value.status == pp.PP_EINVAL
    finally:
        dot.close()
    dot = pp.Dot(inp, order=2, select=1)
    try:
        with pytest.raises(pp.PPError) as ei:
            dot.solve_window(1.0, 0.0, 25)  # select = 1 takes at most 24 roots
        assert ei.value.status == pp.PP_EINVAL
    finally:
        dot.close()
