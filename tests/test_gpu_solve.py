"""GPU window solve against the dense CPU oracle (full diagonalisation)."""

import numpy as np
import pytest

from oracle import pp_oracle as po
from synth.inputs import make_inputs

pytestmark = pytest.mark.gpu


def dense(inp, order=2):
    S, A, Bm = po.dense_blocks(inp.eps, inp.B, inp.nocc, order)
    return po.solve_dense(S, A, Bm, inp.mu)


def window_start_diag(inp, order, pct):
    ref = po.SigmaRef(inp.eps, inp.B, inp.nocc, order=order)
    dA, dS = ref.diag()
    return float(np.percentile((dA / dS).ravel(), pct))


def osc_close(got_w, got_f, want_w, want_f, rtol=1e-4):
    """Compare f per root when isolated, else the sum over the near-degenerate cluster."""
    for i in range(len(want_w)):
        gap = min([abs(want_w[i] - want_w[j]) for j in range(len(want_w)) if j != i] + [1.0])
        if gap > 1e-5:
            assert abs(got_f[i] - want_f[i]) <= rtol * max(abs(want_f[i]), 1e-3), (i, got_f[i], want_f[i])


def test_tiny_nearest_roots(cuda_lib):
    """Tiny literal dot: the k=4 roots nearest the 3rd-lowest root, FP64, 1e-8 Ha."""
    pp = cuda_lib
    inp = make_inputs(8, 24, 64, seed=0, mode="literal")
    ref = dense(inp)
    w0 = ref["omega"][2]
    dot = pp.Dot(inp, order=2, select=1, res_tol=1e-9)
    try:
        got = dot.solve_window(w0, 0.0, 4)
    finally:
        dot.close()
    idx = po.select_window(ref["omega"], w0, 0.0, 4, select=1)
    np.testing.assert_allclose(got["omega"], ref["omega"][idx], atol=1e-8, rtol=0)
    osc_close(got["omega"], got["osc"], ref["omega"][idx], ref["f"][idx])
    assert np.all(got["resid"] <= 1e-9)


@pytest.mark.parametrize("order", [0, 1, 2])
def test_window_lowest_k(cuda_lib, order):
    pp = cuda_lib
    inp = make_inputs(16, 64, 192, seed=5, mode="perturbative")
    ref = dense(inp, order)
    w0 = window_start_diag(inp, order, 20)
    dot = pp.Dot(inp, order=order, select=0, res_tol=1e-8)
    try:
        got = dot.solve_window(w0, 0.1, 8)
    finally:
        dot.close()
    idx = po.select_window(ref["omega"], w0, 0.1, 8, select=0)
    assert len(got["omega"]) == len(idx)
    np.testing.assert_allclose(got["omega"], ref["omega"][idx], atol=1e-8, rtol=0)
    osc_close(got["omega"], got["osc"], ref["omega"][idx], ref["f"][idx])


def test_zero_integrals_bare_gaps(cuda_lib):
    pp = cuda_lib
    inp = make_inputs(8, 24, 64, seed=0, mode="zero")
    gap = np.sort((inp.eps[None, 8:] - inp.eps[:8, None]).ravel())
    dot = pp.Dot(inp, order=2, select=1, res_tol=1e-10)
    try:
        got = dot.solve_window(gap[10], 0.0, 4)
    finally:
        dot.close()
    want = gap[po.select_window(gap, gap[10], 0.0, 4, select=1)]
    np.testing.assert_allclose(got["omega"], want, atol=1e-12)


def test_several_windows_one_batch(cuda_lib):
    """Three windows solved together (one sigma batch per iteration) equal the dense roots."""
    pp = cuda_lib
    inp = make_inputs(16, 64, 192, seed=5, mode="perturbative")
    ref = dense(inp, 2)
    w0 = window_start_diag(inp, 2, 20)
    starts = np.array([w0, w0 + 0.05, w0 + 0.1])
    dot = pp.Dot(inp, order=2, select=0, res_tol=1e-8)
    try:
        res, st = dot.solve_windows(starts, np.full(3, 0.05), [4, 4, 4])
    finally:
        dot.close()
    for w in range(3):
        idx = po.select_window(ref["omega"], starts[w], 0.05, 4, select=0)
        np.testing.assert_allclose(res[w]["omega"], ref["omega"][idx], atol=1e-8, rtol=0)
