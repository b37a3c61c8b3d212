"""Window roots of the FP64 form and of the mixed-precision form against the dense oracle.

Dot 32/128/384 (ph dimension 4096, perturbative width): the dense oracle (M has 8192^2
entries) still finishes in about a minute on the host.  Five windows (k = 4, 8 and 20, widths
0.05-0.1 Ha) at different depths of the spectrum, solved one by one and all in one call.  Bars: FP64 form 1e-8 Ha, mixed form
(BF16 tensor-core sigma, FP64 Krylov, split-BF16 refinement) 1e-6 Ha.  Oscillator strengths:
1e-4 relative in the FP64 form for roots whose neighbours are at least 1e-5 Ha away.  In the
mixed form the returned vector is an eigenvector of the reduced-precision operator; it mixes
in the neighbouring root n by at most |r| / |omega - omega_n| (first-order perturbation
theory), and f, quadratic in the vector, moves by at most twice that relative to sqrt(f f_n)
per neighbour -- the test allows 1e-4 relative plus 4 |r| / gap times the larger f of the
root and its nearest neighbour, gap taken over the whole spectrum.
"""

import numpy as np
import pytest

from oracle import pp_oracle as po
from synth.inputs import make_inputs

pytestmark = pytest.mark.gpu

O, V, Q, SEED = 32, 128, 384, 3


# (percentile, width, k); k = 20 is solved in groups of 8 roots
WINDOWS = [(20, 0.1, 8), (15, 0.08, 4), (40, 0.06, 4), (30, 0.05, 8), (35, 0.1, 20)]


@pytest.fixture(scope="module")
def case():
    inp = make_inputs(O, V, Q, seed=SEED, mode="perturbative")
    S, A, Bm = po.dense_blocks(inp.eps, inp.B, O, 2)
    ref = po.solve_dense(S, A, Bm, inp.mu)
    dA, dS = po.SigmaRef(inp.eps, inp.B, O, order=2).diag()
    r = (dA / dS).ravel()
    wins = [(float(np.percentile(r, p)), w, k) for (p, w, k) in WINDOWS]
    return inp, ref, wins


def _check(got, ref, w0, width, k, tol, mixed=False):
    idx = po.select_window(ref["omega"], w0, width, k, select=0)
    assert len(got["omega"]) == len(idx)
    np.testing.assert_allclose(got["omega"], ref["omega"][idx], atol=tol, rtol=0)
    allw = ref["omega"]
    for i, n in enumerate(idx):
        d = np.abs(allw - allw[n])
        d[n] = np.inf
        nb = int(np.argmin(d))
        gap = d[nb]
        if gap <= 1e-5:
            continue
        f = ref["f"][n]
        if mixed:
            scale = max(abs(f), abs(ref["f"][nb]), 1e-3)
            assert abs(got["osc"][i] - f) <= 1e-4 * max(abs(f), 1e-3) + 4.0 * got["resid"][i] / gap * scale
        else:
            assert abs(got["osc"][i] - f) <= 1e-4 * max(abs(f), 1e-3)


def test_fp64_form_matches_dense(cuda_lib, case):
    """All windows in one pp_solve_windows call (their directions share each sigma batch)."""
    pp = cuda_lib
    inp, ref, wins = case
    dot = pp.Dot(inp, prec=pp.PP_FP64, order=2, select=0, res_tol=1e-8, max_iter=300)
    try:
        outs, st = dot.solve_windows([w[0] for w in wins], [w[1] for w in wins], [w[2] for w in wins])
    finally:
        dot.close()
    assert st == pp.PP_OK
    for (w0, width, k), got in zip(wins, outs):
        _check(got, ref, w0, width, k, 1e-8)


def test_mixed_form_matches_dense(cuda_lib, case):
    """Each window alone, then all windows in one call: the same roots either way."""
    pp = cuda_lib
    inp, ref, wins = case
    dot = pp.Dot(inp, prec=pp.PP_BF16, order=2, select=0, res_tol=1e-6, max_iter=300)
    try:
        for (w0, width, k) in wins:
            got = dot.solve_window(w0, width, k)
            assert np.all(got["resid"] <= 1e-6)
            _check(got, ref, w0, width, k, 1e-6, mixed=True)
        outs, st = dot.solve_windows([w[0] for w in wins], [w[1] for w in wins], [w[2] for w in wins])
    finally:
        dot.close()
    assert st == pp.PP_OK
    for (w0, width, k), got in zip(wins, outs):
        _check(got, ref, w0, width, k, 1e-6, mixed=True)


def test_stepped_windows_match_dense(cuda_lib, case):
    """pp_windows_begin / step / end: the batched solve driven one block iteration at a time
    reaches the same roots; collecting results while windows run is refused."""
    pp = cuda_lib
    inp, ref, wins = case
    dot = pp.Dot(inp, prec=pp.PP_BF16, order=2, select=0, res_tol=1e-6, max_iter=300)
    try:
        run = dot.windows([w[0] for w in wins], [w[1] for w in wins], [w[2] for w in wins])
        unfinished, nv, nc = run.step()
        assert unfinished == len(wins) and nv > 0 and nc >= 1
        with pytest.raises(pp.PPError) as ei:
            run.end()
        assert ei.value.status == pp.PP_EINVAL
        steps = 1
        while unfinished:
            unfinished, nv, nc = run.step()
            steps += 1
            assert steps <= 400
        assert run.step() == (0, 0, 0)  # nothing left to do
        outs, st = run.end()
        assert dot.stats()["iterations"] == steps
    finally:
        dot.close()
    assert st == pp.PP_OK
    for (w0, width, k), got in zip(wins, outs):
        assert np.all(got["resid"] <= 1e-6)
        _check(got, ref, w0, width, k, 1e-6, mixed=True)


@pytest.mark.parametrize("prec_name,tol", [("PP_FP64", 1e-8), ("PP_BF16", 1e-6)])
def test_range_spectrum_matches_dense(cuda_lib, case, prec_name, tol):
    """Absorption spectrum of a frequency range (Sec. 3) from stitched windows against the
    dense oracle's roots and strengths: every root in the range found once (5 windows, at
    most 6 roots each before a window is halved), and the broadened spectrum within 1e-4
    (FP64 form) or 2e-3 (mixed form) of its maximum.  The mixed form covers 0.02 Ha (39
    roots); the FP64 form, whose second-order sigma issues at the FP64 rate, 0.005 Ha (14)."""
    pp = cuda_lib
    inp, ref, wins = case
    w_lo = wins[0][0]
    w_hi = w_lo + (0.005 if prec_name == "PP_FP64" else 0.02)
    eta = 1e-3
    grid = np.linspace(w_lo - 0.005, w_hi + 0.005, 301)
    dot = pp.Dot(inp, prec=getattr(pp, prec_name), order=2, select=0, res_tol=tol, max_iter=300)
    try:
        got = dot.spectrum(w_lo, w_hi, 5, 6, eta, grid)
    finally:
        dot.close()
    want_idx = np.nonzero((ref["omega"] >= w_lo) & (ref["omega"] <= w_hi))[0]
    assert len(got["omega"]) == len(want_idx) and len(want_idx) >= (5 if prec_name == "PP_FP64" else 10)
    np.testing.assert_allclose(got["omega"], ref["omega"][want_idx], atol=tol, rtol=0)
    want = po.range_spectrum(ref["omega"], ref["f"], w_lo, w_hi, eta, grid)
    rel = np.abs(got["spec"] - want).max() / want.max()
    assert rel <= (1e-4 if prec_name == "PP_FP64" else 2e-3), rel
