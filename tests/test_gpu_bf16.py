"""Tensor-core (tcgen05) sigma against the FP64 oracle.

The BF16 form rounds the amplitudes and C_Q(V) to BF16 (unit roundoff 2^-8
relative per element) and accumulates in FP32; the other contractions run in
FP32.  Its error is therefore bounded by a small multiple of 2^-8 times the
size of the amplitude (second-order) part of sigma, plus FP32 rounding of the
rest.  The split form (hi + lo BF16 pairs, three products) is FP32-level.
"""

import numpy as np
import pytest

from oracle import pp_oracle as po
from synth.inputs import make_inputs, random_vectors

pytestmark = pytest.mark.gpu

CASES = [
    (8, 24, 64, 0, "literal"),
    (11, 67, 75, 6, "scaled"),
    (16, 64, 192, 5, "scaled"),
    (16, 130, 70, 7, "scaled"),
]


@pytest.mark.parametrize("case", CASES)
def test_sigma_bf16_within_roundoff_bound(cuda_lib, case):
    pp = cuda_lib
    o, v, Q, seed, mode = case
    inp = make_inputs(o, v, Q, seed=seed, mode=mode)
    dot = pp.Dot(inp, order=2)
    try:
        Z = random_vectors(3, o, v, seed=seed + 7)
        ref2 = po.SigmaRef(inp.eps, inp.B, o, order=2).sigma(Z)
        ref1 = po.SigmaRef(inp.eps, inp.B, o, order=1).sigma(Z)
        second = np.linalg.norm(ref2 - ref1)
        tot = np.linalg.norm(ref2)
        got = dot.sigma(Z, prec=pp.PP_BF16)
        err = np.linalg.norm(got - ref2)
        assert err <= 2.0 ** -8 * 4 * second + 1e-5 * tot, (err, second, tot)
        got3 = dot.sigma(Z, prec=pp.PP_BF16X3)
        err3 = np.linalg.norm(got3 - ref2)
        assert err3 <= 1e-4 * second + 1e-5 * tot, (err3, second, tot)
        assert err3 < err
    finally:
        dot.close()
