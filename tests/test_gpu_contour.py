"""The contour (Riesz projector) solver of Sec. 4.4 against the dense oracle.

16/64/192 dot, second order: every root of the oracle inside a 0.02 Ha window is returned
(the filter finds all of them at once), FP64 form to 1e-8 Ha, mixed form (BF16 filter,
split-BF16 Rayleigh-Ritz) to 1e-6 Ha; oscillator strengths 1e-4 relative in the FP64 form for
roots at least 1e-5 Ha from their neighbours.  A CPU emulation of the same filter (exact
solves) finds the 17 roots of this window in one application with residuals of 1e-8.
"""

import numpy as np
import pytest

from oracle import pp_oracle as po
from synth.inputs import make_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec_name,tol", [("PP_FP64", 1e-8), ("PP_BF16", 1e-6)])
def test_contour_window_matches_dense(cuda_lib, prec_name, tol):
    pp = cuda_lib
    o, v, Q = 16, 64, 192
    inp = make_inputs(o, v, Q, seed=5, mode="perturbative")
    S, A, Bm = po.dense_blocks(inp.eps, inp.B, o, 2)
    ref = po.solve_dense(S, A, Bm, inp.mu)
    dA, dS = po.SigmaRef(inp.eps, inp.B, o, order=2).diag()
    w0 = float(np.percentile((dA / dS).ravel(), 25))
    delta = 0.02
    want = np.nonzero((ref["omega"] >= w0) & (ref["omega"] <= w0 + delta))[0]
    dot = pp.Dot(inp, order=2, prec=getattr(pp, prec_name), res_tol=tol, max_iter=60)
    try:
        got = dot.solve_window_contour(w0, delta, 64)
    finally:
        dot.close()
    assert got["status"] == pp.PP_OK
    assert len(got["omega"]) == len(want) > 8
    np.testing.assert_allclose(got["omega"], ref["omega"][want], atol=tol, rtol=0)
    assert np.all(got["resid"] <= tol)
    if prec_name == "PP_FP64":
        for i, n in enumerate(want):
            d = np.abs(ref["omega"] - ref["omega"][n])
            d[n] = np.inf
            if d.min() > 1e-5:
                f = ref["f"][n]
                assert abs(got["osc"][i] - f) <= 1e-4 * max(abs(f), 1e-3)


def test_contour_rejects_too_wide_a_window(cuda_lib):
    pp = cuda_lib
    inp = make_inputs(16, 64, 192, seed=5, mode="perturbative")
    dot = pp.Dot(inp, order=2)
    try:
        with pytest.raises(pp.PPError) as ei:
            dot.solve_window_contour(0.0, 5.0, 64)  # the whole spectrum
        assert ei.value.status == pp.PP_EINVAL
        assert "narrow the window" in str(ei.value)
    finally:
        dot.close()
