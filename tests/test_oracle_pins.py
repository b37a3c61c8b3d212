"""Pins of the CPU oracle against things other than itself (no GPU).

* Fock-space brute force of the defining expectation values (Sec. 2.2) for
  S, A, B at orders 0, 1, 2 -- the authority for every closed form.
* CIS: the single-excitation block of H computed from determinants.
* Zero integrals: roots are exactly e_a - e_i (zeroth-order spectrum, Sec. 3).
* Structure: symmetry of M and S, +/- pairing, particle-number invariance of
  the second-order density, dense product == matrix-free product.
"""

import numpy as np
import pytest

from oracle import fock
from oracle import pp_oracle as po
from synth.inputs import make_inputs, random_vectors


def _blocks_by_order(inp):
    o = inp.nocc
    S0, A0, B0 = po.dense_blocks(inp.eps, inp.B, o, order=0)
    S1, A1, B1 = po.dense_blocks(inp.eps, inp.B, o, order=1)
    S2, A2, B2 = po.dense_blocks(inp.eps, inp.B, o, order=2)
    return dict(S0=S0, S1=S1 - S0, S2=S2 - S1, A0=A0, A1=A1 - A0, A2=A2 - A1,
                B0=B0, B1=B1 - B0, B2=B2 - B1)


@pytest.mark.parametrize("o,v,Q,seed", [(3, 4, 5, 7), (2, 5, 4, 11), (4, 4, 6, 3)])
def test_closed_forms_match_fock_bruteforce(o, v, Q, seed):
    inp = make_inputs(o, v, Q, seed=seed, sigma_b=0.15)
    bf = fock.PerturbativeElements(inp.eps, inp.B, o).matrices()
    cf = _blocks_by_order(inp)
    for key in ("S0", "S1", "S2", "A0", "A1", "A2", "B0", "B1", "B2"):
        scale = max(1.0, np.abs(bf[key]).max())
        np.testing.assert_allclose(cf[key], bf[key], atol=1e-12 * scale, rtol=0, err_msg=key)
    # every second-order block must be non-trivial, so a dropped term cannot pass
    for key in ("S2", "A2", "B2", "A1", "B1"):
        assert np.abs(bf[key]).max() > 1e-3, key


def test_mp2_energy_matches_bruteforce():
    o, v = 3, 4
    inp = make_inputs(o, v, 5, seed=2, sigma_b=0.2)
    pe = fock.PerturbativeElements(inp.eps, inp.B, o)
    t = po.mp2_amplitudes(inp.eps, inp.B, o)
    w = po.asym(inp.B, slice(0, o), slice(0, o), slice(o, o + v), slice(o, o + v))
    e2 = 0.25 * np.sum(w * t)
    assert e2 < 0
    np.testing.assert_allclose(e2, pe.mp2_energy(), rtol=1e-12)


def test_first_order_A_is_cis_hamiltonian_block():
    """A(0) + A(1) equals <Phi_i^a|H - E_HF|Phi_j^b> built from determinants."""
    o, v = 3, 4
    inp = make_inputs(o, v, 5, seed=5, sigma_b=0.2)
    pe = fock.PerturbativeElements(inp.eps, inp.B, o)
    fs = pe.fs
    H = pe.H0 + pe.W
    ref = pe.ref
    e_hf = ref @ (H @ ref)
    singles = []
    for i in range(o):
        for a in range(v):
            singles.append(fs.cre[o + a] @ (fs.ann[i] @ ref))
    Sd = np.array(singles)
    cis = Sd @ (H @ Sd.T) - e_hf * (Sd @ Sd.T)
    _, A, _ = po.dense_blocks(inp.eps, inp.B, o, order=1)
    np.testing.assert_allclose(A, cis, atol=1e-13)


def test_zero_integrals_give_bare_gaps():
    o, v, Q = 8, 24, 64
    inp = make_inputs(o, v, Q, seed=0, mode="zero")
    S, A, Bm = po.dense_blocks(inp.eps, inp.B, o, order=2)
    res = po.solve_dense(S, A, Bm, inp.mu)
    gap = (inp.eps[None, o:] - inp.eps[:o, None]).ravel()
    np.testing.assert_allclose(res["omega"], np.sort(gap), rtol=0, atol=1e-13)
    order = np.argsort(gap, kind="stable")
    mu2 = np.sum(inp.mu.reshape(3, -1) ** 2, axis=0)
    np.testing.assert_allclose(res["f"], (2.0 / 3.0) * gap[order] * mu2[order], rtol=1e-12)


@pytest.fixture(scope="module")
def tiny():
    return make_inputs(8, 24, 64, seed=0, mode="literal")


def test_symmetry_and_pairing(tiny):
    o = tiny.nocc
    S, A, Bm = po.dense_blocks(tiny.eps, tiny.B, o, order=2)
    for X in (S, A, Bm):
        np.testing.assert_allclose(X, X.T, atol=1e-14)
    M, Sig = po.assemble_M(tiny.eps, tiny.B, o, order=2)
    w = po.solve_dense_eig(M, Sig)
    res = po.solve_dense(S, A, Bm)
    np.testing.assert_allclose(w[w > 0], res["omega"], rtol=1e-10)
    np.testing.assert_allclose(-w[w < 0][::-1], res["omega"], rtol=1e-10)


def test_density_trace_invariant(tiny):
    t = po.mp2_amplitudes(tiny.eps, tiny.B, tiny.nocc)
    roo, rvv = po.densities(t)
    assert abs(np.trace(roo) + np.trace(rvv)) < 1e-14
    assert np.trace(rvv) > 0


def test_dense_product_equals_matrix_free(tiny):
    o = tiny.nocc
    M, Sig = po.assemble_M(tiny.eps, tiny.B, o, order=2)
    ref = po.SigmaRef(tiny.eps, tiny.B, o, order=2)
    Z = random_vectors(3, o, tiny.nvir, seed=1)
    flat = Z.reshape(3, -1).T
    np.testing.assert_allclose(ref.sigma(Z).reshape(3, -1).T, M @ flat, atol=1e-13)
    np.testing.assert_allclose(ref.metric(Z).reshape(3, -1).T, Sig @ flat, atol=1e-14)
    dA, dS = ref.diag()
    ov = o * tiny.nvir
    np.testing.assert_allclose(dA.ravel(), np.diag(M)[:ov], atol=1e-14)
    np.testing.assert_allclose(dS.ravel(), np.diag(Sig)[:ov], atol=1e-14)
    for order in (0, 1):
        Mo, _ = po.assemble_M(tiny.eps, tiny.B, o, order=order)
        r = po.SigmaRef(tiny.eps, tiny.B, o, order=order)
        np.testing.assert_allclose(r.sigma(Z).reshape(3, -1).T, Mo @ flat, atol=1e-13)


def test_dense_solution_is_eigenpair(tiny):
    o = tiny.nocc
    S, A, Bm = po.dense_blocks(tiny.eps, tiny.B, o, order=2)
    M, Sig = po.assemble_M(tiny.eps, tiny.B, o, order=2)
    res = po.solve_dense(S, A, Bm, tiny.mu)
    Z = np.vstack([res["X"], res["Y"]])
    R = M @ Z - (Sig @ Z) * res["omega"][None, :]
    assert np.abs(R).max() < 1e-11
    norm = np.einsum("pn,pq,qn->n", res["X"], S, res["X"]) - np.einsum("pn,pq,qn->n", res["Y"], S, res["Y"])
    np.testing.assert_allclose(norm, 1.0, atol=1e-12)
    for n in range(0, Z.shape[1], 37):
        assert po.variance(M, Sig, Z[:, n], res["omega"][n]) < 1e-20
    # the literal tiny dot is inside the perturbative regime
    assert np.linalg.eigvalsh(S).min() > 0.5


def test_alpha_minimises_rational_rayleigh():
    rng = np.random.default_rng(4)
    for _ in range(200):
        n = 12
        Z = rng.normal(size=(n, n))
        Z = Z @ Z.T
        v = rng.normal(size=n)
        v /= np.linalg.norm(v)
        d = rng.normal(size=n)
        rho_k = v @ Z @ v
        a1, a2, b1, b2 = 2 * d @ Z @ v, d @ Z @ d, 2 * d @ v, d @ d
        al, rho = po.folded_alpha(rho_k, a1, a2, b1, b2)
        grid = np.linspace(-20, 20, 40001)
        vals = (rho_k + a1 * grid + a2 * grid ** 2) / (1 + b1 * grid + b2 * grid ** 2)
        x = v + al * d
        np.testing.assert_allclose(rho, x @ Z @ x / (x @ x), rtol=1e-9)
        if rho < rho_k:
            assert rho <= vals.min() + 1e-9 * abs(vals.min())


def test_inverse_krylov_amplification(tiny):
    """(M - w Sigma)^-m x amplifies eigencomponents by (lambda - w)^-m (Sec. 2.5.1)."""
    o = tiny.nocc
    M, Sig = po.assemble_M(tiny.eps, tiny.B, o, order=2)
    lam, Vr = np.linalg.eig(np.linalg.solve(Sig, M))
    lam, Vr = lam.real, Vr.real
    pos = np.sort(lam[lam > 0])
    w = 0.5 * (pos[5] + pos[6])
    x = Vr @ np.ones(lam.size)
    R = np.linalg.inv(M - w * Sig)
    y = x.copy()
    for _ in range(2):
        y = R @ (Sig @ y)
    coef = np.linalg.solve(Vr, y)
    np.testing.assert_allclose(coef * (lam - w) ** 2, 1.0, rtol=0, atol=1e-6)
    # the two roots bracketing the shift dominate the amplified vector
    top = np.argsort(-np.abs(coef))[:2]
    assert set(np.round(lam[top], 12)) == {np.round(pos[5], 12), np.round(pos[6], 12)}


def test_window_selection_rules():
    om = np.array([0.5, 0.9, 1.0, 1.05, 1.2, 1.3])
    assert list(po.select_window(om, 1.0, 0.25, 2, 0)) == [2, 3]
    assert list(po.select_window(om, 1.0, 0.25, 5, 0)) == [2, 3, 4]
    assert list(po.select_window(om, 1.0, 0.0, 3, 1)) == [1, 2, 3]


@pytest.mark.parametrize("order", [1, 2])
def test_oscillator_strength_sum_rule(tiny, order):
    """RPA sum rule (Eq. pp_adc with F = mu): over all roots,
    sum_n omega_n (mu_c . (X_n + Y_n))^2 = mu_c^T S^-1 (A - B) S^-1 mu_c, so
    sum_n f_n = (2/3) sum_c mu_c^T S^-1 (A - B) S^-1 mu_c.

    Derived from the Cholesky-reduced form: with u_n = L^T (X_n + Y_n) and
    v_n = L^T (X_n - Y_n), (At - Bt) v_n = omega_n u_n, u_m^T v_n = delta_mn, so
    sum_n omega_n u_n u_n^T = At - Bt.  The X - Y combination would give the
    (A + B) form instead, and a wrong power of omega or a missing 2/3 changes
    the sum; B is non-zero at orders 1 and 2, so each slip fails here.
    """
    o = tiny.nocc
    S, A, Bm = po.dense_blocks(tiny.eps, tiny.B, o, order=order)
    res = po.solve_dense(S, A, Bm, tiny.mu)
    Si = np.linalg.inv(S)
    mu = tiny.mu.reshape(3, -1)
    want = (2.0 / 3.0) * sum(m @ Si @ (A - Bm) @ Si @ m for m in mu)
    np.testing.assert_allclose(res["f"].sum(), want, rtol=1e-10)
    # the X - Y slip is detectable at this size (its sum is the A + B form)
    slip = (2.0 / 3.0) * sum(m @ Si @ (A + Bm) @ Si @ m for m in mu)
    assert abs(slip - want) > 1e-3 * abs(want)
    # per root: f_n >= 0, and the zero-dipole vector gives f = 0
    assert np.all(res["f"] >= 0)
    np.testing.assert_array_equal(po.oscillator_strengths(res["omega"], res["X"], res["Y"], 0 * tiny.mu), 0.0)


def test_variance_hand_values():
    """Sec. 4.2 variance on vectors that are not eigenvectors, against hand-computed values.

    (1) M = diag(1, 3), Sigma = 1, z = (1, 1), theta = 2: r = (-1, 1), |r|^2 / |z|^2 = 1,
        which is rho_{A^2} - rho_A^2 = 5 - 4 of the paper's definition.
    (2) M = [[2, 1], [1, 2]], Sigma = diag(1, -1), z = (1, 0), theta = 1:
        M z = (2, 1), Sigma z = (1, 0), r = (1, 1), so the variance is 2.
    (3) z scaled by 3: the variance is normalised by |z|^2, so it is unchanged.
    """
    M1 = np.diag([1.0, 3.0])
    assert po.variance(M1, np.eye(2), np.array([1.0, 1.0]), 2.0) == pytest.approx(1.0, abs=1e-15)
    M2 = np.array([[2.0, 1.0], [1.0, 2.0]])
    Sg = np.diag([1.0, -1.0])
    assert po.variance(M2, Sg, np.array([1.0, 0.0]), 1.0) == pytest.approx(2.0, abs=1e-15)
    assert po.variance(M2, Sg, np.array([3.0, 0.0]), 1.0) == pytest.approx(2.0, abs=1e-14)


def test_variance_is_paper_definition_for_unit_metric():
    """With Sigma = 1 and theta the Rayleigh quotient, the variance equals
    rho_{A^2}(x) - rho_A(x)^2 (Sec. 4.2), computed here from A^2 directly."""
    rng = np.random.default_rng(9)
    A = rng.normal(size=(7, 7))
    A = A + A.T
    for _ in range(5):
        x = rng.normal(size=7)
        xn = x / np.linalg.norm(x)
        rho = xn @ A @ xn
        rho2 = xn @ (A @ A) @ xn
        assert po.variance(A, np.eye(7), x, rho) == pytest.approx(rho2 - rho * rho, rel=1e-12)
        assert rho2 - rho * rho > 1e-3  # not an eigenvector


def test_range_spectrum_closed_forms():
    """Spectrum of a frequency range (Sec. 3): each root contributes a unit-area Lorentzian
    times f_n, so over [a, b] its integral is f_n (atan((b - w_n)/eta) - atan((a - w_n)/eta))/pi
    (trapezoid sum on a fine grid against that closed form); roots outside the range do not
    contribute; an isolated root's peak height is f_n / (pi eta)."""
    omega = np.array([0.9, 1.0, 1.02, 1.3])
    f = np.array([0.7, 0.2, 0.5, 9.0])
    eta = 0.004
    a, b = 0.95, 1.1
    grid = np.linspace(0.5, 1.6, 400001)
    S = po.range_spectrum(omega, f, a, b, eta, grid)
    want = sum(fn * (np.arctan((grid[-1] - wn) / eta) - np.arctan((grid[0] - wn) / eta)) / np.pi
               for wn, fn in zip(omega[1:3], f[1:3]))
    integral = float(np.sum(0.5 * (S[1:] + S[:-1]) * np.diff(grid)))
    assert integral == pytest.approx(want, rel=1e-6)
    peak = po.range_spectrum(omega, f, a, b, eta, [1.0])[0]
    tail = 0.5 * (eta / np.pi) / (0.02 ** 2 + eta ** 2)
    assert peak == pytest.approx(0.2 / (np.pi * eta) + tail, rel=1e-12)
    assert np.all(po.range_spectrum(omega, f, 2.0, 3.0, eta, grid) == 0.0)


def test_tamm_dancoff_first_order_is_cis():
    """Tamm-Dancoff form (B = 0): at first order its roots are the eigenvalues of the CIS
    Hamiltonian built from determinants (Fock-space brute force); at second order they are
    the generalized eigenvalues of (A, S) from scipy's symmetric-definite solver."""
    import scipy.linalg as sl

    o, v = 3, 4
    inp = make_inputs(o, v, 5, seed=5, sigma_b=0.2)
    pe = fock.PerturbativeElements(inp.eps, inp.B, o)
    H = pe.H0 + pe.W
    ref = pe.ref
    e_hf = ref @ (H @ ref)
    Sd = np.array([pe.fs.cre[o + a] @ (pe.fs.ann[i] @ ref) for i in range(o) for a in range(v)])
    cis = Sd @ (H @ Sd.T) - e_hf * (Sd @ Sd.T)
    S1, A1, B1 = po.dense_blocks(inp.eps, inp.B, o, order=1)
    tda1 = po.solve_dense(S1, A1, np.zeros_like(B1))
    np.testing.assert_allclose(tda1["omega"], np.linalg.eigvalsh(cis), atol=1e-12)
    np.testing.assert_allclose(tda1["Y"], 0.0, atol=1e-14)
    S2, A2, B2 = po.dense_blocks(inp.eps, inp.B, o, order=2)
    tda2 = po.solve_dense(S2, A2, np.zeros_like(B2))
    np.testing.assert_allclose(tda2["omega"], sl.eigh(A2, S2, eigvals_only=True), atol=1e-12)


@pytest.mark.parametrize("order", [0, 1, 2])
def test_polarizability_two_routes(tiny, order):
    """Eq. (pp_adc) at real frequencies: the dense solve of (M - omega Sigma) x = F equals the
    sum over the roots, 2 omega_n (mu . u_n)^2 / (omega_n^2 - omega^2), below the first root and
    between two roots; at order 0 it is the closed form sum_ia 2 D_ia mu_ia mu_ia / (D_ia^2 - omega^2)."""
    o = tiny.nocc
    S, A, Bm = po.dense_blocks(tiny.eps, tiny.B, o, order)
    M, Sig = po.assemble_M(tiny.eps, tiny.B, o, order)
    res = po.solve_dense(S, A, Bm, tiny.mu)
    om = res["omega"]
    for w in (0.5 * om[0], 0.5 * (om[10] + om[11])):
        a = po.polarizability(M, Sig, tiny.mu, w)
        b = po.polarizability_sum_over_states(om, res["X"], res["Y"], tiny.mu, w)
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-9 * np.abs(a).max())
        np.testing.assert_allclose(a, a.T, rtol=1e-12, atol=1e-12 * np.abs(a).max())
        # the trace / 3 is sum_n f_n / (omega_n^2 - w^2)
        assert np.trace(a) / 3 == pytest.approx(np.sum(res["f"] / (om ** 2 - w ** 2)), rel=1e-9)
        if order == 0:
            gap = (tiny.eps[None, o:] - tiny.eps[:o, None]).ravel()
            m = tiny.mu.reshape(3, -1)
            c = (m * (2 * gap / (gap ** 2 - w ** 2))[None, :]) @ m.T
            np.testing.assert_allclose(a, c, rtol=1e-11, atol=1e-11 * np.abs(c).max())
