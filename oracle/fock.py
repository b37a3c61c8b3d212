"""Jordan-Wigner Fock-space brute force for the matrix elements of Sec. 2.2.

TEST INFRASTRUCTURE ONLY.  Used to pin the closed forms of ``pp_oracle`` on
systems of at most ~12 spin orbitals.  Nothing here uses Wick's theorem or a
diagram: the operators are sparse matrices on the full 2^n Fock space and the
matrix elements are the defining expectation values.

* H = sum_pq h_pq p^+ q + 1/4 sum <pq||rs> p^+ q^+ s r with
  h = diag(eps) - sum_i <p i||q i>, so that the Fock matrix is diag(eps).
* H0 = sum_p eps_p p^+ p and W_N = H - H0 - <0|H - H0|0> (Sec. 2.2).
* Psi1 = R0 W_N |0> with R0 = sum_{Phi != 0} |Phi>(E0 - E_Phi)^-1 <Phi|.
* For X(lam) = <Psi0|O(lam)|Psi0> / <Psi0|Psi0>, Psi0 = |0> + lam Psi1 and
  H = H0 + lam W_N, the coefficient of lam^m is returned (m = 0, 1, 2).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class FockSpace:
    def __init__(self, nmodes: int):
        if nmodes > 14:
            raise ValueError("brute force limited to 14 spin orbitals")
        self.n = nmodes
        self.dim = 1 << nmodes
        states = np.arange(self.dim)
        self.ann = []
        for p in range(nmodes):
            occ = (states >> p) & 1
            src = states[occ == 1]
            dst = src ^ (1 << p)
            # Jordan-Wigner sign: parity of occupied modes below p
            below = src & ((1 << p) - 1)
            par = np.array([bin(x).count("1") & 1 for x in below], dtype=np.int64)
            sign = 1.0 - 2.0 * par
            a = sp.csr_matrix((sign, (dst, src)), shape=(self.dim, self.dim))
            self.ann.append(a)
        self.cre = [a.T.tocsr() for a in self.ann]

    def det(self, occupied) -> np.ndarray:
        v = np.zeros(self.dim)
        idx = 0
        for p in occupied:
            idx |= 1 << p
        v[idx] = 1.0
        return v

    def one_body(self, h: np.ndarray) -> sp.csr_matrix:
        n = self.n
        op = sp.csr_matrix((self.dim, self.dim))
        for p in range(n):
            for q in range(n):
                if h[p, q] != 0.0:
                    op = op + h[p, q] * (self.cre[p] @ self.ann[q])
        return op

    def two_body(self, v: np.ndarray) -> sp.csr_matrix:
        """1/4 sum_pqrs v[p,q,r,s] p^+ q^+ s r."""
        n = self.n
        op = sp.csr_matrix((self.dim, self.dim))
        for p in range(n):
            for q in range(n):
                if p == q:
                    continue
                pq = self.cre[p] @ self.cre[q]
                for r in range(n):
                    for s in range(n):
                        if r == s or v[p, q, r, s] == 0.0:
                            continue
                        op = op + (0.25 * v[p, q, r, s]) * (pq @ self.ann[s] @ self.ann[r])
        return op


def _antisym_integrals(B: np.ndarray) -> np.ndarray:
    """<pq||rs> = (pr|qs) - (ps|qr) with (pq|rs) = sum_Q B[Q,p,q] B[Q,r,s]."""
    chem = np.einsum("xpq,xrs->pqrs", B, B)
    return chem.transpose(0, 2, 1, 3) - chem.transpose(0, 2, 3, 1)


class PerturbativeElements:
    """Second-order expansion of the metric and superoperator matrices, by brute force."""

    def __init__(self, eps: np.ndarray, B: np.ndarray, nocc: int):
        self.eps = np.asarray(eps, dtype=np.float64)
        n = self.eps.size
        self.nocc, self.nvir = nocc, n - nocc
        self.fs = fs = FockSpace(n)
        v = _antisym_integrals(np.asarray(B, dtype=np.float64))
        h = np.diag(self.eps) - np.einsum("piqi->pq", v[:, :nocc, :, :nocc])
        H = fs.one_body(h) + fs.two_body(v)
        self.H0 = fs.one_body(np.diag(self.eps))
        self.ref = fs.det(range(nocc))
        W = H - self.H0
        e_shift = self.ref @ (W @ self.ref)
        self.W = (W - e_shift * sp.identity(fs.dim, format="csr")).tocsr()
        # R0 W_N |0>: divide each determinant by E0 - E_det (zeroth-order energies)
        e_det = np.zeros(fs.dim)
        for p in range(n):
            e_det += self.eps[p] * ((np.arange(fs.dim) >> p) & 1)
        e0 = float(self.ref @ e_det)
        w0 = self.W @ self.ref
        denom = e0 - e_det
        psi1 = np.zeros(fs.dim)
        mask = np.abs(w0) > 0
        mask[np.argmax(self.ref)] = False
        psi1[mask] = w0[mask] / denom[mask]
        self.psi1 = psi1
        self.norm1 = float(psi1 @ psi1)

    # q_ia = i^+ a,  q_ia^+ = a^+ i
    def _q(self, i, a):
        fs = self.fs
        return fs.cre[i] @ fs.ann[self.nocc + a]

    def _qd(self, i, a):
        fs = self.fs
        return fs.cre[self.nocc + a] @ fs.ann[i]

    @staticmethod
    def _sym_dc(X, Hm, Y):
        """[X, H, Y] = ([X,[H,Y]] + [[X,H],Y]) / 2."""
        HY = Hm @ Y - Y @ Hm
        XH = X @ Hm - Hm @ X
        return 0.5 * ((X @ HY - HY @ X) + (XH @ Y - Y @ XH))

    def _expand(self, C0, C1):
        """lambda^0, lambda^1, lambda^2 coefficients of <Psi0|C0 + lam C1|Psi0>/<Psi0|Psi0>."""
        r, p = self.ref, self.psi1
        n0 = r @ (C0 @ r)
        n1 = r @ (C1 @ r) + p @ (C0 @ r) + r @ (C0 @ p)
        n2 = p @ (C0 @ p) + p @ (C1 @ r) + r @ (C1 @ p)
        return n0, n1, n2 - self.norm1 * n0

    def matrices(self):
        """Return dict of S0,S1,S2, A0,A1,A2, B0,B1,B2 as (ov, ov) arrays."""
        o, vn = self.nocc, self.nvir
        ov = o * vn
        out = {k: np.zeros((ov, ov)) for k in ("S0", "S1", "S2", "A0", "A1", "A2", "B0", "B1", "B2")}
        zero = sp.csr_matrix((self.fs.dim, self.fs.dim))
        pairs = [(i, a) for i in range(o) for a in range(vn)]
        for I, (i, a) in enumerate(pairs):
            q = self._q(i, a)
            for J, (j, b) in enumerate(pairs):
                qd = self._qd(j, b)
                qj = self._q(j, b)
                # metric
                s = q @ qd - qd @ q
                s0, s1, s2 = self._expand(s, zero)
                out["S0"][I, J], out["S1"][I, J], out["S2"][I, J] = s0, s1, s2
                # A = <[q_ia, H, q_jb^+]>
                a0, a1, a2 = self._expand(self._sym_dc(q, self.H0, qd), self._sym_dc(q, self.W, qd))
                out["A0"][I, J], out["A1"][I, J], out["A2"][I, J] = a0, a1, a2
                # B = -<[q_ia, H, q_jb]>
                b0, b1, b2 = self._expand(self._sym_dc(q, self.H0, qj), self._sym_dc(q, self.W, qj))
                out["B0"][I, J], out["B1"][I, J], out["B2"][I, J] = -b0, -b1, -b2
        return out

    def mp2_energy(self) -> float:
        """<0|W_N|Psi1>, the second-order energy."""
        return float(self.ref @ (self.W @ self.psi1))
