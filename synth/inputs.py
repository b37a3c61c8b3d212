"""Seeded generator for quantum-dot-shaped synthetic inputs.

The paper's real inputs (Hartree-Fock orbitals of PbS/CdS dots and their
density-fitted integrals, Sec. 3) are not available, so every run draws
synthetic ones with the shapes of Table 1's particle-hole spaces:

* orbital energies: occupied uniform in [-1.0, -0.3] Ha, virtual uniform in
  [0.05, 2.0] Ha, each block sorted ascending (occupied first);
* density-fitting tensor B[Q, p, q], symmetric in (p, q): for every Q the
  upper triangle p <= q is drawn row-major from N(0, sigma_B^2) and mirrored,
  so that (pq|rs) = sum_Q B[Q,p,q] B[Q,r,s];
* dipole integrals mu[c, i, a] ~ N(0, 1) for c = x, y, z.

Draw order is eps_occ, eps_vir, B, mu from ``numpy.random.default_rng(seed)``.

Three widths of B are offered.  ``literal`` uses sigma_B = 0.05 at every size.
``scaled`` shrinks sigma_B with the dot so that the second-order density
correction and the first-order coupling stay at the level of the 8/24/64
case: sigma_B = 0.05 * (8 * 24**2 * 64 / (o * v**2 * Q)) ** 0.25.  With the
literal width the perturbation grows with the dot until the metric S stops
being positive definite.  ``perturbative`` keeps instead the first-order
coupling per matrix element, sigma_B^2 sqrt(Q), in a fixed ratio to the mean
level spacing of the ov gaps: sigma_B = 0.82 / sqrt(o v sqrt(Q)).  There the
second-order metric stays within a few per cent of 1 and each interior root
mixes a handful of particle-hole states, the regime in which a diagonal Jacobi
splitting is a useful preconditioner; root finding above the tiny case uses it.
Sigma products and FLOP counts do not depend on the width.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SIGMA_B_LITERAL = 0.05

# (name, nocc, nvir, naux, seed) of the workloads; the names say what they are.
CONFIGS = {
    "tiny-8x24x64": dict(nocc=8, nvir=24, naux=64, seed=0),
    "dot-64x256x768": dict(nocc=64, nvir=256, naux=768, seed=1),
    "dot-128x512x1536": dict(nocc=128, nvir=512, naux=1536, seed=2),
    "dot-256x1024x3072": dict(nocc=256, nvir=1024, naux=3072, seed=4),
    # serving sizes (nocc, nvir, naux)
    "serve-32x128x384": dict(nocc=32, nvir=128, naux=384, seed=3),
}


@dataclass
class DotInputs:
    nocc: int
    nvir: int
    naux: int
    eps: np.ndarray  # [nocc + nvir] float64, occupied first
    B: np.ndarray  # [naux, n, n] float64 (or float32), symmetric in the last two
    mu: np.ndarray  # [3, nocc, nvir] float64
    sigma_b: float
    seed: int

    @property
    def n(self) -> int:
        return self.nocc + self.nvir


def scaled_sigma_b(nocc: int, nvir: int, naux: int) -> float:
    return SIGMA_B_LITERAL * (8 * 24 ** 2 * 64 / (nocc * nvir ** 2 * naux)) ** 0.25


def perturbative_sigma_b(nocc: int, nvir: int, naux: int) -> float:
    return 0.82 / float(np.sqrt(nocc * nvir * np.sqrt(max(naux, 1))))


def make_inputs(nocc: int, nvir: int, naux: int, seed: int, mode: str = "literal",
                sigma_b: float | None = None, b_dtype=np.float64) -> DotInputs:
    """Draw one synthetic dot.  ``mode`` is 'literal', 'scaled' or 'zero' (B = 0)."""
    if nocc < 1 or nvir < 1 or naux < 0:
        raise ValueError("need nocc >= 1, nvir >= 1, naux >= 0")
    if sigma_b is None:
        if mode == "literal" or mode == "zero":
            sigma_b = SIGMA_B_LITERAL
        elif mode == "scaled":
            sigma_b = scaled_sigma_b(nocc, nvir, naux)
        elif mode == "perturbative":
            sigma_b = perturbative_sigma_b(nocc, nvir, naux)
        else:
            raise ValueError(f"unknown mode {mode!r}")
    rng = np.random.default_rng(seed)
    eps_o = np.sort(rng.uniform(-1.0, -0.3, nocc))
    eps_v = np.sort(rng.uniform(0.05, 2.0, nvir))
    eps = np.concatenate([eps_o, eps_v])
    n = nocc + nvir
    iu, ju = np.triu_indices(n)
    B = np.empty((naux, n, n), dtype=b_dtype)
    for Q in range(naux):
        g = rng.normal(0.0, sigma_b, iu.size)
        blk = np.empty((n, n))
        blk[iu, ju] = g
        blk[ju, iu] = g
        B[Q] = blk
    mu = rng.normal(0.0, 1.0, (3, nocc, nvir))
    if mode == "zero":
        B[...] = 0.0
    return DotInputs(nocc, nvir, naux, eps, B, mu, float(sigma_b), seed)


def window_start(eps: np.ndarray, nocc: int, pct: float) -> float:
    """Percentile of the zeroth-order gaps eps_a - eps_i, used to place windows."""
    d = (eps[None, nocc:] - eps[:nocc, None]).ravel()
    return float(np.percentile(d, pct))


def random_vectors(nvec: int, nocc: int, nvir: int, seed: int) -> np.ndarray:
    """Trial supervectors Z[nvec, 2, nocc, nvir] (X block, then Y block)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.0, (nvec, 2, nocc, nvir))
