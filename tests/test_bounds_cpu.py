"""The element-wise bound of the tensor-core sigma tests fails a plausible mistake (CPU only).

The mistake is planted in the oracle: the amplitudes transposed in (c, d), the slip of a
transposed operand.  Its sigma differs from the true one by more than the BF16 bound of
test_gpu_bf16.py in most elements, so a kernel making it cannot pass that test.
"""

import numpy as np

from oracle import pp_oracle as po
from sigma_bounds import sigma_scales
from synth.inputs import make_inputs, random_vectors

BF16 = (8.0, 2.0 ** -8, 1e-6)  # kappa, u, floor of test_gpu_bf16.BOUNDS["PP_BF16"]


def test_elementwise_bound_catches_a_slip():
    """The bound is tight enough to fail a plausible mistake planted in the oracle (CPU):
    the sigma of a transposed amplitude chain, t_ij^cd -> t_ij^dc, differs from the true
    one by more than the BF16 bound in most elements."""
    o, v, Q = 8, 24, 64
    inp = make_inputs(o, v, Q, seed=0, mode="literal")
    ref = po.SigmaRef(inp.eps, inp.B, o, order=2)
    Z = random_vectors(2, o, v, seed=7)
    want = ref.sigma(Z)
    scale = sigma_scales(ref, Z)
    bad = po.SigmaRef(inp.eps, inp.B, o, order=2)
    bad.t = bad.t.transpose(0, 1, 3, 2).copy()  # t_ij^cd -> t_ij^dc = -t_ij^cd
    wrong = bad.sigma(Z)
    kappa, u, floor = BF16
    bound = kappa * u * scale + floor * np.abs(want).max()
    assert np.mean(np.abs(wrong - want) > bound) > 0.5
