"""Per-dot intermediates of mixed-precision contexts (tensor-core precompute) against the oracle.

A context created with prec = PP_BF16 computes the MP2 pair sums (the S(2) densities and the
A(2) weights) and the ring intermediate Gamma from split-BF16 amplitude slabs with FP32 sums.
Their error enters every sigma of that context, FP64 ones included, only through the
second-order terms.  Bars: the FP64 sigma of such a context matches the oracle to 1e-5 of the
second-order contribution (||sigma_2 - sigma_1||), and diag(S) - 1 (pure second order) to 1e-5
relative.  Cases span several tiles, ragged tails (v not a multiple of 128) and a single slab.
"""

import numpy as np
import pytest

from oracle import pp_oracle as po
from synth.inputs import make_inputs, random_vectors

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("o,v,Q,seed", [(8, 24, 64, 0), (16, 72, 150, 4), (32, 128, 384, 3)])
def test_tc_precompute_sigma_and_diagonal(cuda_lib, o, v, Q, seed):
    pp = cuda_lib
    inp = make_inputs(o, v, Q, seed=seed, mode="perturbative")
    ref2 = po.SigmaRef(inp.eps, inp.B, o, order=2)
    ref1 = po.SigmaRef(inp.eps, inp.B, o, order=1)
    Z = random_vectors(3, o, v, seed=seed + 7)
    want = ref2.sigma(Z)
    second = np.linalg.norm(want - ref1.sigma(Z))
    dot = pp.Dot(inp, prec=pp.PP_BF16, order=2)
    try:
        got = dot.sigma(Z, prec=pp.PP_FP64)
        dA, dS = dot.diagonal()
    finally:
        dot.close()
    assert np.linalg.norm(got - want) <= 1e-5 * second + 1e-12 * np.linalg.norm(want)
    wA, wS = ref2.diag()
    assert np.max(np.abs(dS - wS)) <= 1e-5 * np.max(np.abs(wS - 1.0))
    wA1, _ = ref1.diag()
    assert np.max(np.abs(dA - wA)) <= 1e-5 * np.max(np.abs(wA - wA1)) + 1e-12
