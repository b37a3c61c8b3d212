"""GPU parity of the matrix-free product sigma = M z against the CPU oracle.

Element by element, FP64 path, relative Frobenius error <= 1e-12 (the FP64 bar),
on shapes that span several 64-wide tiles with ragged tails.
"""

import numpy as np
import pytest

from oracle import pp_oracle as po
from synth.inputs import make_inputs, random_vectors

pytestmark = pytest.mark.gpu

CASES = [
    # (nocc, nvir, naux, seed, mode)
    (8, 24, 64, 0, "literal"),
    (5, 13, 7, 3, "literal"),
    (3, 70, 33, 4, "literal"),
    (11, 67, 75, 6, "scaled"),
    (16, 64, 192, 5, "scaled"),
]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("case", CASES)
def test_sigma_fp64_matches_oracle(cuda_lib, case, order):
    pp = cuda_lib
    o, v, Q, seed, mode = case
    inp = make_inputs(o, v, Q, seed=seed, mode=mode)
    dot = pp.Dot(inp, order=order)
    try:
        Z = random_vectors(3, o, v, seed=seed + 100)
        sig, met = dot.sigma(Z, metric=True)
        ref = po.SigmaRef(inp.eps, inp.B, o, order=order)
        assert rel(sig, ref.sigma(Z)) < 1e-12
        assert rel(met, ref.metric(Z)) < 1e-13
        dA, dS = dot.diagonal()
        rA, rS = ref.diag()
        np.testing.assert_allclose(dA, rA, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(dS, rS, rtol=1e-12, atol=1e-14)
    finally:
        dot.close()


def test_sigma_single_and_empty_batch(cuda_lib):
    pp = cuda_lib
    inp = make_inputs(8, 24, 64, seed=0)
    dot = pp.Dot(inp)
    try:
        Z = random_vectors(1, 8, 24, seed=5)
        ref = po.SigmaRef(inp.eps, inp.B, 8, order=2)
        assert rel(dot.sigma(Z), ref.sigma(Z)) < 1e-12
        out = dot.sigma(np.zeros((0, 2, 8, 24)))
        assert out.shape == (0, 2, 8, 24)
    finally:
        dot.close()


def test_sigma_device_pointers(cuda_lib):
    import torch

    pp = cuda_lib
    inp = make_inputs(8, 24, 64, seed=0)
    dot = pp.Dot(inp)
    try:
        Z = random_vectors(4, 8, 24, seed=9)
        Zd = torch.from_numpy(Z).cuda()
        sig = dot.sigma(Zd).cpu().numpy()
        ref = po.SigmaRef(inp.eps, inp.B, 8, order=2)
        assert rel(sig, ref.sigma(Z)) < 1e-12
    finally:
        dot.close()


def test_sigma_float32_B_input(cuda_lib):
    pp = cuda_lib
    inp = make_inputs(5, 13, 7, seed=3)
    inp.B = inp.B.astype(np.float32)
    dot = pp.Dot(inp)
    try:
        Z = random_vectors(2, 5, 13, seed=1)
        ref = po.SigmaRef(inp.eps, inp.B.astype(np.float64), 5, order=2)
        assert rel(dot.sigma(Z), ref.sigma(Z)) < 1e-12
    finally:
        dot.close()
