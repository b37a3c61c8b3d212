"""Per-element error scales for the reduced-precision sigma (test infrastructure).

The tensor-core form evaluates the amplitude part of B(2) (the ladders and the
(ki|bc)/(kj|ac) rings) as  amp = sum_Q [P_Q Bvv_Q - Boo_Q P_Q],  P_Q = T C_Q(Y),
C_Q(Y) = Y Bvv_Q - Boo_Q Y,  T[(i,c),(j,d)] = t_ij^cd,  with every operand of that
chain rounded to BF16 (u = 2^-8) in the BF16 form, or carried as a BF16 pair
(u ~ 2^-16) in the split form, and FP32 accumulation.  Each rounding perturbs one
factor of one term of the fully expanded sum by at most u relative, and the
perturbations of different terms are independent in sign, so the error of an element
scales with the root of the sum of the squared terms of that element:

    rms2[i,a] = sum_Q ( sum_c P2_Q[i,c] Bvv_Q[c,a]^2 + sum_k Boo_Q[i,k]^2 P2_Q[k,a] ),
    P2_Q = T^2 C2_Q,  C2_Q = Y^2 Bvv_Q^2 + Boo_Q^2 Y^2          (all squares elementwise).

For sums of many terms of random sign |amp| is of the size of sqrt(rms2), so a bound
kappa * u * sqrt(rms2) is a per-element test that a wrong index, a dropped term or a
transposed operand fails (their error is of the size of the element itself).  The
remaining terms (first order, the A(2) pair sums, the Gamma rings) run in FP32-level
arithmetic and get a floor relative to the largest element of sigma.

The amplitudes come from the oracle (its FP64 t); the chain is evaluated with numpy.
"""

from __future__ import annotations

import numpy as np


def amplitude_rms(t: np.ndarray, Boo: np.ndarray, Bvv: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """sqrt(rms2) above for one half-vector Y [o, v]; t is [o, o, v, v] (t[i, j, c, d])."""
    o, v = Y.shape
    Q = Bvv.shape[0]
    Y2, Boo2, Bvv2 = Y * Y, Boo * Boo, Bvv * Bvv
    C2 = np.einsum("jb,xbd->xjd", Y2, Bvv2, optimize=True) + np.einsum("xjl,ld->xjd", Boo2, Y2, optimize=True)
    T2 = (t * t).transpose(0, 2, 1, 3).reshape(o * v, o * v)  # [(i,c), (j,d)]
    P2 = (T2 @ C2.reshape(Q, o * v).T).T.reshape(Q, o, v)  # P2[x, i, c]
    rms2 = np.einsum("xic,xca->ia", P2, Bvv2, optimize=True) + np.einsum("xik,xka->ia", Boo2, P2, optimize=True)
    return np.sqrt(rms2)


def sigma_scales(ref, Z: np.ndarray) -> np.ndarray:
    """Per-element amplitude-chain scale of sigma = M z for Z [nvec, 2, o, v], using the
    oracle object ``ref`` (SigmaRef, order 2).  sigma_X takes B Y and sigma_Y takes B X."""
    out = np.empty_like(Z)
    for s in range(Z.shape[0]):
        out[s, 0] = amplitude_rms(ref.t, ref.Boo, ref.Bvv, Z[s, 1])
        out[s, 1] = amplitude_rms(ref.t, ref.Boo, ref.Bvv, Z[s, 0])
    return out
