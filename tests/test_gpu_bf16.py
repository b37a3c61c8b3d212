"""Tensor-core (tcgen05) sigma against the FP64 oracle, element by element.

The BF16 form rounds the amplitudes, C_Q(V), P_Q and the B operands of the amplitude
chain to BF16 (unit roundoff u = 2^-8) and accumulates in FP32; the other contractions run
at FP32 level.  Each element's error is therefore a few roundings of the terms of that
element's amplitude chain, which add like independent errors: bounded by kappa u times
the root of the sum of their squares (sigma_bounds.sigma_scales), plus an FP32-level floor
relative to the largest element.  The split form (hi + lo BF16 pairs, three products) has
u ~ 2^-16.  Calibration on GB300 (maximum of |error| over the bound's scale, all cases
below): 4.8 (BF16) and 8.1 (split) with a floor of 1e-7 max|sigma|; the bounds use kappa 8
and 16 with floors 1e-6 and 2e-6.  A wrong index or a dropped term makes an error of the
size of the element itself, about 30 times the BF16 bound wherever the amplitude part is
above the floor (the literal and scaled widths below).
"""

import numpy as np
import pytest

from oracle import pp_oracle as po
from sigma_bounds import sigma_scales
from synth.inputs import make_inputs, random_vectors

pytestmark = pytest.mark.gpu

CASES = [
    (8, 24, 64, 0, "literal"),
    (11, 67, 75, 6, "scaled"),
    (16, 64, 192, 5, "scaled"),
    (16, 130, 70, 7, "scaled"),
    (32, 128, 384, 3, "scaled"),
]
BOUNDS = {"PP_BF16": (8.0, 2.0 ** -8, 1e-6), "PP_BF16X3": (16.0, 2.0 ** -16, 2e-6)}


def elementwise_ok(got, want, scale, prec_name):
    kappa, u, floor = BOUNDS[prec_name]
    bound = kappa * u * scale + floor * np.abs(want).max()
    ratio = np.abs(got - want) / bound
    return float(ratio.max()), np.unravel_index(int(np.argmax(ratio)), ratio.shape)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("ctx_prec", ["PP_FP64", "PP_BF16"])
def test_sigma_bf16_elementwise(cuda_lib, case, ctx_prec):
    pp = cuda_lib
    o, v, Q, seed, mode = case
    inp = make_inputs(o, v, Q, seed=seed, mode=mode)
    dot = pp.Dot(inp, order=2, prec=getattr(pp, ctx_prec))
    try:
        Z = random_vectors(3, o, v, seed=seed + 7)
        ref = po.SigmaRef(inp.eps, inp.B, o, order=2)
        want = ref.sigma(Z)
        scale = sigma_scales(ref, Z)
        second = np.linalg.norm(want - po.SigmaRef(inp.eps, inp.B, o, order=1).sigma(Z))
        tot = np.linalg.norm(want)
        got = dot.sigma(Z, prec=pp.PP_BF16)
        r, at = elementwise_ok(got, want, scale, "PP_BF16")
        assert r <= 1.0, (r, at)
        err = np.linalg.norm(got - want)
        assert err <= 2.0 ** -8 * 4 * second + 1e-5 * tot, (err, second, tot)
        got3 = dot.sigma(Z, prec=pp.PP_BF16X3)
        r3, at3 = elementwise_ok(got3, want, scale, "PP_BF16X3")
        assert r3 <= 1.0, (r3, at3)
        assert np.linalg.norm(got3 - want) < err
    finally:
        dot.close()



def test_sigma_chunk_graphs_replay(cuda_lib):
    """The tensor-core sigma replays each chunk shape it has met before as a captured CUDA
    graph (first call kernel by kernel, second captured, third replayed): every call agrees
    with the kernel-by-kernel context to FP32-reduction noise and stays within the bounds."""
    pp = cuda_lib
    o, v, Q = 16, 130, 70
    inp = make_inputs(o, v, Q, seed=7, mode="scaled")
    ref = po.SigmaRef(inp.eps, inp.B, o, order=2)
    Z = random_vectors(3, o, v, seed=14)
    want = ref.sigma(Z)
    scale = sigma_scales(ref, Z)
    plain = pp.Dot(inp, order=2, prec=pp.PP_BF16, graphs=0)
    graph = pp.Dot(inp, order=2, prec=pp.PP_BF16, graphs=1)
    try:
        for name in ("PP_BF16", "PP_BF16X3"):
            prec = getattr(pp, name)
            base, base_m = plain.sigma(Z, prec=prec, metric=True)
            for call in range(3):
                got, met = graph.sigma(Z, prec=prec, metric=True)
                assert np.abs(got - base).max() <= 1e-6 * np.abs(base).max(), (name, call)
                # two contexts: their pair sums (FP32, split-K atomics) differ by a few FP32 ulps
                # (the metric reads them in FP64: 5.7e-8 of its largest element was measured)
                assert np.abs(met - base_m).max() <= 1e-6 * np.abs(base_m).max()
                r, at = elementwise_ok(got, want, scale, name)
                assert r <= 1.0, (name, call, r, at)
            # the same shape without the metric output is a different graph
            for call in range(2):
                got = graph.sigma(Z, prec=prec)
                assert np.abs(got - base).max() <= 1e-6 * np.abs(base).max()
    finally:
        plain.close()
        graph.close()
