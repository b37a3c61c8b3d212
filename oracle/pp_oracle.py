"""Plain FP64 CPU oracle: the response matrix of Sec. 2.2 assembled densely.

TEST INFRASTRUCTURE ONLY -- never imported by the product path.

Conventions (spin orbitals, real integrals):
  i, j, k, l occupied; a, b, c, d virtual; n = nocc + nvir, occupied first.
  (pq|rs) = sum_Q B[Q,p,q] B[Q,r,s]                      (density fitting, Sec. 3)
  <pq||rs> = (pr|qs) - (ps|qr)                            (antisymmetrized, Sec. 2.2)
  t_ij^ab = <ab||ij> / (e_i + e_j - e_a - e_b)            (MP2, Psi1 = R0 W_N |0>, Sec. 2.2)
  q_ia = i^dagger a (de-excitation), q_ia^dagger = a^dagger i

The matrix of Eq. (m_eigen) is built from the superoperator matrix elements
of Eq. (mkk_so) over the 1p1h manifold {a^dagger i, i^dagger a} with the MP2
ground state, kept to second order in W_N.  The readings taken where the text
is ambiguous (all pinned by the Fock-space brute force in ``fock.py``):

* S = <Psi0|[q_ia, q_jb^dagger]|Psi0>/<Psi0|Psi0> (Eq. s(2) read as the
  commutator of the commented derivation, with the normalised ground state).
* A = <[q_ia, H, q_jb^dagger]>, B = -<[q_ia, H, q_jb]> with the symmetrised
  double commutator [X,H,Y] = ([X,[H,Y]] + [[X,H],Y]) / 2, normalised Psi0.
  The H0 part of A(2) is Eq. (a(2)) symmetrised; the W_N parts that the
  complete second order adds are the <0|..|Psi1> and <Psi1|..|0> terms of the
  same kind as the first two terms of Eq. (b(2)); the third (H0) term of
  Eq. (b(2)) vanishes identically because [q_ia, q_jb] = 0.
* First order A(1) = <aj||ib>, B(1) = <ab||ij>: the textbook TDHF matrices
  that Sec. 2.2 says Eqs. (a(1)) and (b(1)) reproduce.
* The property vector F of Eq. (pp_adc) is taken at zeroth order:
  transition moment sum_ia mu_ia (X + Y)_ia, eigenvectors normalised to
  X^T S X - Y^T S Y = 1, f = (2/3) omega |moment|^2.
* The absorption spectrum of a frequency range is the Lorentzian-broadened sum of
  the oscillator strengths of the roots inside the range (``range_spectrum``).
"""

from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------
# integrals and amplitudes
# ----------------------------------------------------------------------------


def _sl(nocc: int, n: int):
    return slice(0, nocc), slice(nocc, n)


def chem(B: np.ndarray, P: slice, Q: slice, R: slice, S: slice) -> np.ndarray:
    """(pq|rs) for p in P, q in Q, r in R, s in S (density-fitted, Sec. 3)."""
    return np.einsum("xpq,xrs->pqrs", B[:, P, Q], B[:, R, S], optimize=True)


def asym(B: np.ndarray, P: slice, Q: slice, R: slice, S: slice) -> np.ndarray:
    """<pq||rs> = (pr|qs) - (ps|qr), indexed [p, q, r, s] (W_N of Sec. 2.2)."""
    direct = chem(B, P, R, Q, S).transpose(0, 2, 1, 3)
    exch = chem(B, P, S, Q, R).transpose(0, 2, 3, 1)
    return direct - exch


def denominators(eps: np.ndarray, nocc: int) -> np.ndarray:
    """D[i,j,a,b] = e_i + e_j - e_a - e_b, the R0 resolvent weights (Sec. 2.2)."""
    eo, ev = eps[:nocc], eps[nocc:]
    return eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]


def mp2_amplitudes(eps: np.ndarray, B: np.ndarray, nocc: int) -> np.ndarray:
    """t[i,j,a,b] = <ab||ij>/D: Psi1 = R0 W_N|0> = 1/4 sum t a^+ b^+ j i |0> (Sec. 2.2)."""
    n = eps.size
    o, v = _sl(nocc, n)
    vabij = asym(B, v, v, o, o)
    return vabij.transpose(2, 3, 0, 1) / denominators(eps, nocc)


def densities(t: np.ndarray):
    """Second-order one-particle density corrections of the normalised MP2 state.

    rho_oo[i,j] = -1/2 sum_kcd t_ik^cd t_jk^cd,  rho_vv[a,b] = 1/2 sum_klc t_kl^ac t_kl^bc.
    S(2)_ia,jb = delta_ab rho_oo[i,j] - delta_ij rho_vv[a,b]  (Eq. s(2), commutator reading).
    """
    rho_oo = -0.5 * np.einsum("ikcd,jkcd->ij", t, t, optimize=True)
    rho_vv = 0.5 * np.einsum("klac,klbc->ab", t, t, optimize=True)
    return rho_oo, rho_vv


# ----------------------------------------------------------------------------
# dense blocks, indexed [i, a, j, b] and reshaped to (ov, ov)
# ----------------------------------------------------------------------------


def _eye_blocks(nocc: int, nvir: int):
    return np.eye(nocc), np.eye(nvir)


def dense_blocks(eps: np.ndarray, B: np.ndarray, nocc: int, order: int = 2):
    """Return S, A, B (each ov x ov, row index ia = i*nvir + a) to the given order.

    Order 0: Eqs. (a(0)), (b(0)) and S(0) = 1.  Order 1 adds Eqs. (a(1)), (b(1))
    (S(1) = 0).  Order 2 adds Eq. (s(2)), the complete A(2) and Eq. (b(2)).
    """
    n = eps.size
    nvir = n - nocc
    ov = nocc * nvir
    o, v = _sl(nocc, n)
    eo, ev = eps[:nocc], eps[nocc:]
    Io, Iv = _eye_blocks(nocc, nvir)
    gap = ev[None, :] - eo[:, None]  # Delta_ia = e_a - e_i

    S = np.einsum("ij,ab->iajb", Io, Iv)
    A = np.einsum("ia,ij,ab->iajb", gap, Io, Iv)  # Eq. (a(0))
    Bm = np.zeros_like(A)  # Eq. (b(0))
    if order >= 1:
        A = A + asym(B, v, o, o, v).transpose(2, 0, 1, 3)  # <aj||ib>, Eq. (a(1))
        vabij = asym(B, v, v, o, o)
        Bm = Bm + vabij.transpose(2, 0, 3, 1)  # <ab||ij>, Eq. (b(1))
    if order >= 2:
        t = mp2_amplitudes(eps, B, nocc)
        rho_oo, rho_vv = densities(t)
        S2 = np.einsum("ab,ij->iajb", Iv, rho_oo) - np.einsum("ij,ab->iajb", Io, rho_vv)
        S = S + S2
        # A(2), H0 part: <Psi1|[q_ia, H0, q_jb^+]|Psi1>_linked.  [q,[H0,q^+]] and
        # [[q,H0],q^+] are (e_b - e_j) and (e_a - e_i) times [q_ia, q_jb^+], so the
        # symmetrised form is (Delta_ia + Delta_jb)/2 times the S(2) element.
        A2_h0 = 0.5 * (gap[:, :, None, None] + gap[None, None, :, :]) * S2
        # A(2), W_N parts: <0|[q,W,q^+]|Psi1> + <Psi1|[q,W,q^+]|0>.
        w = asym(B, o, o, v, v)  # <jk||cd>
        x_oo = np.einsum("ikcd,jkcd->ij", t, w, optimize=True)
        x_vv = np.einsum("klac,klbc->ab", t, w, optimize=True)
        A2_w = -0.25 * np.einsum("ab,ij->iajb", Iv, x_oo + x_oo.T) \
            - 0.25 * np.einsum("ij,ab->iajb", Io, x_vv + x_vv.T)
        A = A + A2_h0 + A2_w
        # B(2) = -(<0|[q_ia,W,q_jb]|Psi1> + <Psi1|[q_ia,W,q_jb]|0>); the second is zero.
        vvvv = asym(B, v, v, v, v)  # <ab||cd>
        oooo = asym(B, o, o, o, o)  # <kl||ij>
        ovvo = asym(B, o, v, v, o)  # <kb||ci>
        ladder_pp = 0.5 * np.einsum("abcd,ijcd->iajb", vvvv, t, optimize=True)
        ladder_hh = 0.5 * np.einsum("klij,klab->iajb", oooo, t, optimize=True)
        ring_1 = -np.einsum("jkac,kbci->iajb", t, ovvo, optimize=True)
        ring_2 = -np.einsum("ikbc,kacj->iajb", t, ovvo, optimize=True)
        Bm = Bm + ladder_pp + ladder_hh + ring_1 + ring_2
    return S.reshape(ov, ov), A.reshape(ov, ov), Bm.reshape(ov, ov)


def assemble_M(eps: np.ndarray, B: np.ndarray, nocc: int, order: int = 2):
    """M = [[A, B], [B, A]] and Sigma = diag(S, -S) of Eq. (m_eigen), dense."""
    S, A, Bm = dense_blocks(eps, B, nocc, order)
    M = np.block([[A, Bm], [Bm, A]])
    Z = np.zeros_like(S)
    Sig = np.block([[S, Z], [Z, -S]])
    return M, Sig


# ----------------------------------------------------------------------------
# matrix-free sigma: the same matrix elements contracted with a vector, term by
# term, through the density-fitting factors (no 4-index integral is formed)
# ----------------------------------------------------------------------------


class SigmaRef:
    """sigma = M z and Sigma z for z = (X; Y) without assembling M.

    Every term is one matrix element of ``dense_blocks`` contracted with the
    trial vector; B_Qpq factors are contracted in the order written.
    """

    def __init__(self, eps: np.ndarray, B: np.ndarray, nocc: int, order: int = 2):
        self.nocc = nocc
        self.n = eps.size
        self.nvir = self.n - nocc
        self.order = order
        self.eps = np.asarray(eps, dtype=np.float64)
        o, v = _sl(nocc, self.n)
        B = np.asarray(B, dtype=np.float64)
        self.Boo = np.ascontiguousarray(B[:, o, o])
        self.Bov = np.ascontiguousarray(B[:, o, v])
        self.Bvv = np.ascontiguousarray(B[:, v, v])
        self.eo, self.ev = self.eps[:nocc], self.eps[nocc:]
        self.gap = self.ev[None, :] - self.eo[:, None]
        if order >= 2:
            Bov = self.Bov
            # t_ij^ab = [(ai|bj) - (aj|bi)] / D
            direct = np.einsum("xia,xjb->ijab", Bov, Bov, optimize=True)
            self.t = (direct - direct.transpose(0, 1, 3, 2)) / denominators(self.eps, nocc)
            self.rho_oo, self.rho_vv = densities(self.t)
            t = self.t
            # weighted pair sums entering A(2) (combined H0 + W_N parts):
            # A(2)_ia,jb = -1/2 d_ab sum_kcd t_ik^cd t_jk^cd (e_a + e_k - e_c - e_d)
            #              -1/2 d_ij sum_klc t_kl^ac t_kl^bc (e_k + e_l - e_c - e_i)
            eo, ev = self.eo, self.ev
            w_kcd = eo[:, None, None] - ev[None, :, None] - ev[None, None, :]
            self.p_oo = np.einsum("ikcd,jkcd->ij", t, t, optimize=True)
            self.q_oo = np.einsum("ikcd,jkcd,kcd->ij", t, t, w_kcd, optimize=True)
            w_klc = eo[:, None, None] + eo[None, :, None] - ev[None, None, :]
            self.p_vv = np.einsum("klac,klbc->ab", t, t, optimize=True)
            self.q_vv = np.einsum("klac,klbc,klc->ab", t, t, w_klc, optimize=True)

    # --- A blocks --------------------------------------------------------
    def _A(self, X: np.ndarray) -> np.ndarray:
        out = self.gap * X  # Eq. (a(0))
        if self.order >= 1:
            Boo, Bov, Bvv = self.Boo, self.Bov, self.Bvv
            # <aj||ib> X_jb = (ai|jb) X_jb - (ab|ji) X_jb
            cq = np.einsum("xjb,jb->x", Bov, X)
            out = out + np.einsum("xia,x->ia", Bov, cq)
            tmp = np.einsum("xji,jb->xib", Boo, X)
            out = out - np.einsum("xab,xib->ia", Bvv, tmp)
        if self.order >= 2:
            ea, ei = self.ev[None, :], self.eo[:, None]
            occ = -0.5 * (ea * (self.p_oo @ X) + self.q_oo @ X)
            vir = -0.5 * (X @ self.q_vv - ei * (X @ self.p_vv))
            out = out + occ + vir
        return out

    # --- B blocks --------------------------------------------------------
    def _B(self, Y: np.ndarray) -> np.ndarray:
        out = np.zeros_like(Y)
        if self.order >= 1:
            Boo, Bov, Bvv = self.Boo, self.Bov, self.Bvv
            # <ab||ij> Y_jb = (ai|bj) Y_jb - (aj|bi) Y_jb
            cq = np.einsum("xjb,jb->x", Bov, Y)
            out = out + np.einsum("xia,x->ia", Bov, cq)
            tmp = np.einsum("xib,jb->xij", Bov, Y)
            out = out - np.einsum("xja,xij->ia", Bov, tmp)
        if self.order >= 2:
            out = out + self._B2(Y)
        return out

    def _B2(self, Y: np.ndarray) -> np.ndarray:
        t, Boo, Bov, Bvv = self.t, self.Boo, self.Bov, self.Bvv
        # particle ladder 1/2 sum_cd <ab||cd> t_ij^cd Y_jb, <ab||cd> = (ac|bd) - (ad|bc)
        zy = np.einsum("xbd,jb->xjd", Bvv, Y)  # sum_b (bd| Y_jb
        h = np.einsum("ijcd,xjd->xic", t, zy, optimize=True)
        pp = np.einsum("xac,xic->ia", Bvv, h)
        zy2 = np.einsum("xbc,jb->xjc", Bvv, Y)
        h2 = np.einsum("ijcd,xjc->xid", t, zy2, optimize=True)
        pp = 0.5 * (pp - np.einsum("xad,xid->ia", Bvv, h2))
        # hole ladder 1/2 sum_kl <kl||ij> t_kl^ab Y_jb, <kl||ij> = (ki|lj) - (kj|li)
        u = np.einsum("xlj,jb->xlb", Boo, Y)
        g = np.einsum("klab,xlb->xka", t, u, optimize=True)
        hh = np.einsum("xki,xka->ia", Boo, g)
        u2 = np.einsum("xkj,jb->xkb", Boo, Y)
        g2 = np.einsum("klab,xkb->xla", t, u2, optimize=True)
        hh = 0.5 * (hh - np.einsum("xli,xla->ia", Boo, g2))
        # ring -sum_kc t_jk^ac <kb||ci> Y_jb, <kb||ci> = (kc|bi) - (ki|bc)
        gam = np.einsum("jkac,xkc->xja", t, Bov, optimize=True)  # sum_kc t_jk^ac (kc|
        e = np.einsum("xib,jb->xij", Bov, Y)  # |bi) Y_jb
        r1 = -np.einsum("xja,xij->ia", gam, e)
        zy3 = np.einsum("xbc,jb->xjc", Bvv, Y)  # (bc| Y_jb
        f = np.einsum("jkac,xjc->xka", t, zy3, optimize=True)
        r1 = r1 + np.einsum("xki,xka->ia", Boo, f)
        # ring -sum_kc t_ik^bc <ka||cj> Y_jb, <ka||cj> = (kc|aj) - (kj|ac)
        gam2 = np.einsum("ikbc,xkc->xib", t, Bov, optimize=True)
        e2 = np.einsum("xib,jb->xij", gam2, Y)
        r2 = -np.einsum("xja,xij->ia", Bov, e2)
        u3 = np.einsum("xkj,jb->xkb", Boo, Y)
        f2 = np.einsum("ikbc,xkb->xic", t, u3, optimize=True)
        r2 = r2 + np.einsum("xac,xic->ia", Bvv, f2)
        return pp + hh + r1 + r2

    # --- metric ----------------------------------------------------------
    def _S(self, X: np.ndarray) -> np.ndarray:
        if self.order >= 2:
            return X + self.rho_oo @ X - X @ self.rho_vv
        return X.copy()

    def sigma(self, Z: np.ndarray) -> np.ndarray:
        """M z for Z[..., 2, nocc, nvir]: sigma_X = A X + B Y, sigma_Y = B X + A Y."""
        Z = np.asarray(Z, dtype=np.float64)
        out = np.empty_like(Z)
        for idx in np.ndindex(Z.shape[:-3]):
            X, Y = Z[idx][0], Z[idx][1]
            out[idx][0] = self._A(X) + self._B(Y)
            out[idx][1] = self._B(X) + self._A(Y)
        return out

    def metric(self, Z: np.ndarray) -> np.ndarray:
        """Sigma z = (S X; -S Y) of Eq. (m_eigen)."""
        Z = np.asarray(Z, dtype=np.float64)
        out = np.empty_like(Z)
        for idx in np.ndindex(Z.shape[:-3]):
            out[idx][0] = self._S(Z[idx][0])
            out[idx][1] = -self._S(Z[idx][1])
        return out

    def diag(self):
        """diag(A) and diag(S) (each [nocc, nvir]): the Jacobi splitting D of Sec. 2.5.2."""
        dA = self.gap.copy()
        dS = np.ones_like(self.gap)
        if self.order >= 1:
            jj = np.einsum("xia,xia->ia", self.Bov, self.Bov)
            kk = np.einsum("xaa,xii->ia", self.Bvv, self.Boo)
            dA = dA + jj - kk
        if self.order >= 2:
            ea, ei = self.ev[None, :], self.eo[:, None]
            dA = dA - 0.5 * (ea * np.diag(self.p_oo)[:, None] + np.diag(self.q_oo)[:, None])
            dA = dA - 0.5 * (np.diag(self.q_vv)[None, :] - ei * np.diag(self.p_vv)[None, :])
            dS = dS + np.diag(self.rho_oo)[:, None] - np.diag(self.rho_vv)[None, :]
        return dA, dS


# ----------------------------------------------------------------------------
# dense generalized eigensolve M z = omega Sigma z
# ----------------------------------------------------------------------------


class MetricNotPositive(RuntimeError):
    """S is not positive definite (the ground state is outside the perturbative regime)."""


class UnstableRPA(RuntimeError):
    """A - B (in the S-orthonormal basis) is not positive definite: complex roots."""


def solve_dense(S: np.ndarray, A: np.ndarray, Bm: np.ndarray, mu: np.ndarray | None = None):
    """All positive roots of Eq. (m_eigen) by Cholesky reduction of the metric.

    S = L L^T; At = L^-1 A L^-T, Bt = L^-1 B L^-T; with u = Xt + Yt and
    v = Xt - Yt, (At - Bt)(At + Bt) u = omega^2 u.  Writing At - Bt = Lm Lm^T,
    u = Lm w turns it into the symmetric problem Lm^T (At + Bt) Lm w = omega^2 w.
    Normalising Xt^T Xt - Yt^T Yt = u^T v = 1 fixes |w|^2 = 1/omega.
    Returns omega (ascending), X, Y (columns, back-transformed), and f if mu is given.
    """
    try:
        L = np.linalg.cholesky(S)
    except np.linalg.LinAlgError as e:
        raise MetricNotPositive(str(e)) from e
    Li = np.linalg.inv(L)
    At = Li @ A @ Li.T
    Bt = Li @ Bm @ Li.T
    At = 0.5 * (At + At.T)
    Bt = 0.5 * (Bt + Bt.T)
    try:
        Lm = np.linalg.cholesky(At - Bt)
    except np.linalg.LinAlgError as e:
        raise UnstableRPA(str(e)) from e
    C = Lm.T @ (At + Bt) @ Lm
    C = 0.5 * (C + C.T)
    w2, W = np.linalg.eigh(C)
    if w2[0] <= 0:
        raise UnstableRPA("non-positive omega^2")
    omega = np.sqrt(w2)
    W = W / np.sqrt(omega)[None, :]  # |w|^2 = 1/omega
    U = Lm @ W  # Xt + Yt
    V = np.linalg.solve(Lm.T, W) * omega[None, :]  # Xt - Yt = omega Lm^-T w
    Xt, Yt = 0.5 * (U + V), 0.5 * (U - V)
    X = np.linalg.solve(L.T, Xt)
    Y = np.linalg.solve(L.T, Yt)
    out = dict(omega=omega, X=X, Y=Y)
    if mu is not None:
        out["f"] = oscillator_strengths(omega, X, Y, mu)
    return out


def solve_dense_eig(M: np.ndarray, Sig: np.ndarray) -> np.ndarray:
    """Second route: all eigenvalues of Sigma^-1 M (non-symmetric), sorted."""
    w = np.linalg.eigvals(np.linalg.solve(Sig, M))
    return np.sort(w.real)


def oscillator_strengths(omega, X, Y, mu):
    """f_n = 2/3 omega_n sum_c (mu_c . (X + Y)_n)^2, zeroth-order F (Eq. pp_adc)."""
    mom = np.einsum("cp,pn->cn", mu.reshape(3, -1), X + Y)
    return (2.0 / 3.0) * omega * np.sum(mom ** 2, axis=0)


def select_window(omega: np.ndarray, omega0: float, delta: float, k: int, select: int = 0):
    """Indices of the requested roots.

    select = 0: the k lowest roots in [omega0, omega0 + delta] (fewer if the window
    holds fewer).  select = 1: the k roots nearest omega0 (ties to the lower root).
    """
    omega = np.asarray(omega)
    if select == 0:
        idx = np.nonzero((omega >= omega0) & (omega <= omega0 + delta))[0]
        idx = idx[np.argsort(omega[idx], kind="stable")]
        return idx[:k]
    dist = np.abs(omega - omega0)
    order = np.lexsort((omega, dist))
    sel = order[:k]
    return sel[np.argsort(omega[sel], kind="stable")]


def variance(M: np.ndarray, Sig: np.ndarray, z: np.ndarray, theta: float) -> float:
    """Per-root variance |(M - theta Sigma) z|^2 / |z|^2 (Sec. 4.2, with Sigma = 1 it is
    rho_{A^2} - rho_A^2 for the Rayleigh quotient theta)."""
    r = M @ z - theta * (Sig @ z)
    return float(r @ r / (z @ z))


def folded_alpha(rho_k: float, a1: float, a2: float, b1: float, b2: float):
    """Weighting parameter of Sec. 2.5.2.

    rho(alpha) = (rho_k + a1 alpha + a2 alpha^2) / (1 + b1 alpha + b2 alpha^2);
    d rho/d alpha = 0 gives (a2 b1 - a1 b2) alpha^2 + 2 (a2 - rho_k b2) alpha
    + (a1 - rho_k b1) = 0.  Returns the stationary root with the lowest rho, or
    1 (the plain Jacobi step) if neither root lowers rho below rho_k.
    """
    def rho(al):
        return (rho_k + a1 * al + a2 * al * al) / (1.0 + b1 * al + b2 * al * al)

    c2 = a2 * b1 - a1 * b2
    c1 = 2.0 * (a2 - rho_k * b2)
    c0 = a1 - rho_k * b1
    roots = []
    if abs(c2) > 1e-300:
        disc = c1 * c1 - 4.0 * c2 * c0
        if disc >= 0:
            s = np.sqrt(disc)
            roots = [(-c1 + s) / (2 * c2), (-c1 - s) / (2 * c2)]
    elif abs(c1) > 1e-300:
        roots = [-c0 / c1]
    best, best_rho = 1.0, rho(1.0)
    for r in roots:
        den = 1.0 + b1 * r + b2 * r * r
        if den > 0 and rho(r) < best_rho:
            best, best_rho = r, rho(r)
    if best_rho >= rho_k:
        return 1.0, rho(1.0)
    return best, best_rho


# ----------------------------------------------------------------------------
# absorption spectrum of the roots in a frequency range
# ----------------------------------------------------------------------------


def lorentzian(x, eta: float):
    """Unit-area Lorentzian of half width eta: (eta / pi) / (x^2 + eta^2)."""
    return (eta / np.pi) / (np.asarray(x) ** 2 + eta * eta)


def range_spectrum(omega, f, w_lo: float, w_hi: float, eta: float, grid):
    """Absorption-like spectrum of the roots inside [w_lo, w_hi] (Sec. 3): the oscillator
    strengths broadened by a Lorentzian of half width eta,
        S(w) = sum_{n : w_lo <= omega_n <= w_hi} f_n (eta / pi) / ((w - omega_n)^2 + eta^2),
    i.e. -Im of the pole sum of Eq. (pp_adc) at w + i eta divided by pi, restricted to the poles
    in the range (the frequency windows of Sec. 2.5 supply exactly those)."""
    omega = np.asarray(omega)
    f = np.asarray(f)
    sel = (omega >= w_lo) & (omega <= w_hi)
    grid = np.asarray(grid, dtype=np.float64)
    out = np.zeros_like(grid)
    for w_n, f_n in zip(omega[sel], f[sel]):
        out += f_n * lorentzian(grid - w_n, eta)
    return out


# ----------------------------------------------------------------------------
# frequency-dependent linear response
# ----------------------------------------------------------------------------


def polarizability(M: np.ndarray, Sig: np.ndarray, mu: np.ndarray, omega: float) -> np.ndarray:
    """Dipole polarizability at a real frequency, Eq. (pp_adc) with F_c = (mu_c; mu_c):
    alpha[c, c'] = F_c^T (M - omega Sigma)^-1 F_c', by a dense linear solve."""
    m = mu.reshape(3, -1)
    F = np.concatenate([m, m], axis=1).T  # [2 ov, 3]
    X = np.linalg.solve(M - omega * Sig, F)
    return F.T @ X


def polarizability_sum_over_states(omega_n, X, Y, mu, omega: float) -> np.ndarray:
    """The same tensor from the roots: sum_n 2 omega_n (mu_c . u_n)(mu_c' . u_n) / (omega_n^2 - omega^2),
    u_n = X_n + Y_n (eigenvectors normalised to X^T S X - Y^T S Y = 1)."""
    mom = mu.reshape(3, -1) @ (X + Y)  # [3, n]
    wts = 2.0 * omega_n / (omega_n ** 2 - omega ** 2)
    return (mom * wts[None, :]) @ mom.T
