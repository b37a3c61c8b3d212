"""Tamm-Dancoff form (B = 0; the Hermitian variant of Sec. 2.2's response matrix).

sigma = (A X, A Y) against the oracle's A blocks, and window roots against the dense
oracle's solve of A X = omega S X (its Cholesky route with B = 0; pinned on the CPU to the
determinant CIS eigenvalues at first order and to scipy's generalized eigh at second).
"""

import numpy as np
import pytest

from oracle import pp_oracle as po
from synth.inputs import make_inputs, random_vectors

pytestmark = pytest.mark.gpu


def test_tda_sigma_matches_oracle(cuda_lib):
    pp = cuda_lib
    o, v, Q = 16, 64, 192
    inp = make_inputs(o, v, Q, seed=5, mode="scaled")
    ref = po.SigmaRef(inp.eps, inp.B, o, order=2)
    Z = random_vectors(3, o, v, seed=9)
    want = np.stack([np.stack([ref._A(z[0]), ref._A(z[1])]) for z in Z])
    for prec_ctx in ("PP_FP64", "PP_BF16"):
        dot = pp.Dot(inp, order=2, tda=1, prec=getattr(pp, prec_ctx))
        try:
            got, met = dot.sigma(Z, metric=True)
            if prec_ctx == "PP_FP64":
                assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
            else:  # the context's tensor-core second-order intermediates carry ~1e-6
                assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()
            np.testing.assert_allclose(met, ref.metric(Z), atol=1e-6 * np.abs(Z).max())
            for prec in (pp.PP_BF16, pp.PP_BF16X3):  # no B term: FP32-level first-order products
                g = dot.sigma(Z, prec=prec)
                assert np.abs(g - want).max() <= 1e-5 * np.abs(want).max()
        finally:
            dot.close()


@pytest.mark.parametrize("order", [1, 2])
def test_tda_window_roots_match_dense(cuda_lib, order):
    pp = cuda_lib
    o, v, Q = 16, 64, 192
    inp = make_inputs(o, v, Q, seed=5, mode="perturbative")
    S, A, Bm = po.dense_blocks(inp.eps, inp.B, o, order)
    ref = po.solve_dense(S, A, np.zeros_like(Bm), inp.mu)
    dA, dS = po.SigmaRef(inp.eps, inp.B, o, order=order).diag()
    w0 = float(np.percentile((dA / dS).ravel(), 25))
    idx = po.select_window(ref["omega"], w0, 0.1, 8, select=0)
    for prec_name, tol in (("PP_FP64", 1e-8), ("PP_BF16", 1e-6)):
        dot = pp.Dot(inp, order=order, tda=1, prec=getattr(pp, prec_name), select=0, res_tol=tol, max_iter=300)
        try:
            got = dot.solve_window(w0, 0.1, 8)
        finally:
            dot.close()
        assert len(got["omega"]) == len(idx)
        np.testing.assert_allclose(got["omega"], ref["omega"][idx], atol=tol, rtol=0)
        if prec_name == "PP_FP64":
            for i, n in enumerate(idx):
                d = np.abs(ref["omega"] - ref["omega"][n])
                d[n] = np.inf
                if d.min() > 1e-5:
                    f = ref["f"][n]
                    assert abs(got["osc"][i] - f) <= 1e-4 * max(abs(f), 1e-3)
