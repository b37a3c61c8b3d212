"""Parity at the benchmark's full size (nocc 64, nvir 256, naux 768; ph dimension 16384).

The dense oracle is out of reach here (M has 32768^2 entries and the particle ladder
needs 256^4 integrals), so parity is checked on what the oracle can compute:
its matrix-free FP64 sigma for sampled trial vectors, and the FP64 residual
|M x - theta Sigma x| of the roots the solver returns (for a symmetric-definite-
like pencil the eigenvalue error is bounded by the residual over the gap, and
theta is the oracle's own Rayleigh quotient of x).
"""

import numpy as np
import pytest

from oracle import pp_oracle as po
from synth.inputs import make_inputs, random_vectors

pytestmark = pytest.mark.gpu

O, V, Q = 64, 256, 768


@pytest.fixture(scope="module")
def dot_inputs():
    return make_inputs(O, V, Q, seed=1, mode="perturbative")


@pytest.fixture(scope="module")
def oracle_sigma(dot_inputs):
    return po.SigmaRef(dot_inputs.eps, dot_inputs.B, O, order=2)


def test_fullsize_sigma_fp64_and_bf16(cuda_lib, dot_inputs, oracle_sigma):
    pp = cuda_lib
    Z = random_vectors(1, O, V, seed=21)
    want = oracle_sigma.sigma(Z)
    want1 = po.SigmaRef(dot_inputs.eps, dot_inputs.B, O, order=1).sigma(Z)
    second = np.linalg.norm(want - want1)
    dot = pp.Dot(dot_inputs, order=2)
    try:
        got = dot.sigma(Z)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12
        got_bf = dot.sigma(Z, prec=pp.PP_BF16)
        assert np.linalg.norm(got_bf - want) <= 2.0 ** -8 * 4 * second + 1e-5 * np.linalg.norm(want)
        got_x3 = dot.sigma(Z, prec=pp.PP_BF16X3)
        assert np.linalg.norm(got_x3 - want) <= 1e-6 * np.linalg.norm(want)
    finally:
        dot.close()


def test_fullsize_window_roots_have_small_oracle_residual(cuda_lib, dot_inputs, oracle_sigma):
    """The bench's solve (BF16 sigma, FP64 Krylov, split-BF16 refinement to a residual of 1e-6):
    each returned root is an eigenpair to a few 1e-6 in the oracle's FP64 arithmetic, so the
    root lies within that distance of theta (and within |r|^2 / gap of it when isolated)."""
    pp = cuda_lib
    dot = pp.Dot(dot_inputs, prec=pp.PP_BF16, order=2, select=0, res_tol=1e-6, max_iter=300)
    try:
        dA, dS = dot.diagonal()
        w0 = float(np.percentile((dA / dS).ravel(), 20))
        out = dot.solve_window(w0, 0.1, 8, want_vectors=True)
    finally:
        dot.close()
    assert len(out["omega"]) == 8
    assert np.all(np.diff(out["omega"]) > 0)
    assert np.all(out["omega"] >= w0) and np.all(out["omega"] <= w0 + 0.1)
    for n in (0, 7):
        z = out["vectors"][n][None]
        Mz = oracle_sigma.sigma(z)[0].ravel()
        Sz = oracle_sigma.metric(z)[0].ravel()
        zz = z[0].ravel()
        norm = zz @ Sz
        assert abs(norm - 1.0) < 1e-5  # X^T S X - Y^T S Y = 1
        theta = (zz @ Mz) / norm
        assert abs(theta - out["omega"][n]) < 1e-6
        r = Mz - theta * Sz
        assert np.linalg.norm(r) / abs(norm) < 5e-6
