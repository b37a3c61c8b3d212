"""The reading taken for the weighted-Jacobi step of Sec. 2.5.2, checked on the CPU.

Sec. 2.5.2 builds each new inverse-Krylov vector from one Jacobi sweep on
(M - omega Sigma) v' = v with the splitting M - omega Sigma = D + F:
    v_J = D^-1 (v - F v),   v' = v + alpha (v_J - v),
alpha minimising the folded Rayleigh quotient rho = v'^T (M - omega Sigma)^2 v' / v'^T v'.
The GPU solver instead adds the Jacobi sweep on the correction equation
(M - theta Sigma) t = -r from t = 0, i.e. t = -D^-1 r, to its basis.  This test emulates
both in plain NumPy on the dense oracle matrices of a 16/64/192 dot (one target, Rayleigh-
Ritz of the pencil on the growing basis, diagonal floored at 1e-3 Ha as in the solver):

* the correction-equation direction reaches a residual of 1e-8 within 60 iterations;
* the paper's direction v_J - v = D^-1 (v - r) in the same subspace method stalls above 1e-3
  (near convergence it tends to D^-1 v, which is dominated by the unit vectors whose diagonal
  is closest to theta, i.e. by the current vector itself);
* the literal sequence v' = v + alpha* (v_J - v) with the rational alpha* of the oracle
  (folded_alpha) at a fixed shift stalls above 1e-3 as well.
"""

import numpy as np
import pytest

from oracle import pp_oracle as po
from synth.inputs import make_inputs


@pytest.fixture(scope="module")
def system():
    o, v, Q = 16, 64, 192
    inp = make_inputs(o, v, Q, seed=5, mode="perturbative")
    M, Sig = po.assemble_M(inp.eps, inp.B, o, 2)
    S, A, Bm = po.dense_blocks(inp.eps, inp.B, o, 2)
    om = po.solve_dense(S, A, Bm)["omega"]
    dA, dS = po.SigmaRef(inp.eps, inp.B, o, 2).diag()
    w0 = om[len(om) // 5] + 1e-4
    return M, Sig, dA.ravel(), dS.ravel(), w0


def _floored(D, floor=1e-3):
    return np.where(np.abs(D) < floor, np.where(D < 0, -floor, floor), D)


def _start(dA, dS, w0):
    ratio = np.concatenate([dA / dS, -dA / dS])
    x = np.zeros(ratio.size)
    x[np.argmin(np.abs(ratio - w0))] = 1.0
    return x


def _subspace(system, mode, iters=60):
    M, Sig, dA, dS, w0 = system
    V = _start(dA, dS, w0)[:, None]
    res = []
    for _ in range(iters):
        w, C = np.linalg.eig(np.linalg.solve(V.T @ Sig @ V, V.T @ M @ V))
        c = C[:, np.argmin(np.abs(w.real - w0))].real
        x = V @ c
        x /= np.linalg.norm(x)
        theta = (x @ M @ x) / (x @ Sig @ x)
        r = M @ x - theta * (Sig @ x)
        res.append(np.linalg.norm(r) / abs(x @ Sig @ x))
        D = _floored(np.concatenate([dA - theta * dS, dA + theta * dS]))
        d = -r / D if mode == "correction" else (x - r) / D
        for _ in range(2):
            d = d - V @ (V.T @ d)
        V = np.hstack([V, (d / np.linalg.norm(d))[:, None]])
    return res


def test_correction_equation_direction_converges(system):
    res = _subspace(system, "correction")
    assert min(res) < 1e-8


def test_paper_direction_stalls_in_the_subspace_method(system):
    res = _subspace(system, "paper")
    assert min(res[20:]) > 1e-3


def test_literal_weighted_jacobi_sequence_stalls(system):
    M, Sig, dA, dS, w0 = system
    K = M - w0 * Sig
    Z = K @ K
    D = _floored(np.diag(K).copy())
    x = _start(dA, dS, w0)
    res = []
    for _ in range(200):
        x /= np.linalg.norm(x)
        rho = x @ Z @ x
        d = (x - (K @ x - D * x)) / D - x  # v_J - v with v_J = D^-1 (v - F v)
        alpha, rho_new = po.folded_alpha(rho, 2 * d @ Z @ x, d @ Z @ d, 2 * d @ x, d @ d)
        assert rho_new <= rho * (1 + 1e-12) or alpha == 1.0
        x = x + alpha * d
        xn = x / np.linalg.norm(x)
        th = (xn @ M @ xn) / (xn @ Sig @ xn)
        res.append(np.linalg.norm(M @ xn - th * (Sig @ xn)) / abs(xn @ Sig @ xn))
    assert min(res) > 1e-3
