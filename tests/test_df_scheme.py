"""The double-FP32 arithmetic of the Krylov-space kernels, emulated on the CPU.

`k_gram2d`, `k_combine_ts` and `k_jacobi_eig` hold FP64 data as pairs of floats (hi + lo,
48 significant bits), form products with the exact FMA residual of hi * hi plus the cross
terms, keep sums with an error-free two-sum, and rotate with (c, s) renormalised so that
c^2 + s^2 = 1 to about 2^-46.  These tests run the same formulas in numpy float32 (every
operation rounded to float32; an FMA is a float64 product-sum rounded once, exact for the
operand sizes used) and pin the scheme's accuracy against exact rational arithmetic and
`numpy.linalg.eigh`:
  * the split reproduces x to 2^-47 relative and drops |x| < 2^-100;
  * a 256-term dot product (the chunk length of one Gram block) is within 1e-13 of the sum of
    |a_i b_i| (worst seen 5e-14: the float correction term's own rounding sets the floor;
    FP64 summation of the same terms is at about 1e-16, and the solver needs errors far below
    the 1e-12 relative scale of the folded Grams' smallest eigenvalues);
  * the Jacobi on small symmetric matrices returns eigenvalues within 1e-12 of ||A||, residuals
    below 1e-12 ||A|| and eigenvectors orthonormal to 1e-13.
"""

import struct
from fractions import Fraction

import numpy as np
import pytest

F = np.float32


def _fma(a, b, c):
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def split_df(x):
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    sgn = (b >> 32) & 0x80000000
    e = ((b >> 52) & 0x7FF) - 1023
    if e < -100:
        return F(0), F(0)
    if e > 100:
        h = F(x)
        return h, F(x - float(h))
    mant = b & 0xFFFFFFFFFFFFF
    hi = struct.unpack("<f", struct.pack("<I", sgn | ((e + 127) << 23) | (mant >> 29)))[0]
    lo = F(0)
    if e >= -70:
        scale = struct.unpack("<f", struct.pack("<I", (e - 52 + 127) << 23))[0]
        mag = F(F(mant & 0x1FFFFFFF) * F(scale))
        lo = -mag if sgn else mag
    return F(hi), F(lo)


def df_fma(s, c, a, b):
    p = F(a[0] * b[0])
    e = _fma(a[0], b[0], -p)
    e = _fma(a[0], b[1], e)
    e = _fma(a[1], b[0], e)
    t = F(s + p)
    z = F(t - s)
    w = F(F(s - F(t - z)) + F(p - z))
    return t, F(c + F(w + e))


def df_mul(a, b):
    p = F(a[0] * b[0])
    e = _fma(a[0], b[0], -p)
    e = _fma(a[0], b[1], e)
    e = _fma(a[1], b[0], e)
    s = F(p + e)
    return s, F(e - F(s - p))


def df_add(a, b):
    s = F(a[0] + b[0])
    z = F(s - a[0])
    e = F(F(a[0] - F(s - z)) + F(b[0] - z))
    e = F(e + F(a[1] + b[1]))
    t = F(s + e)
    return t, F(e - F(t - s))


def unit_rotation(c, s):
    c2 = F(c * c)
    c2e = _fma(c, c, -c2)
    s2 = F(s * s)
    s2e = _fma(s, s, -s2)
    n = df_add((c2, c2e), (s2, s2e))
    d = F(F(n[0] - F(1)) + n[1])
    eps = _fma(F(0.375) * d, d, F(-0.5) * d)
    return (c, F(c * eps)), (s, F(s * eps))


def jacobi_df(G, max_sweeps=16):
    m = G.shape[0]
    mp = (m + 1) & ~1
    A = [[split_df(0.5 * (G[i, j] + G[j, i])) if i < m and j < m else (F(0), F(0)) for j in range(mp)]
         for i in range(mp)]
    V = [[(F(1.0 if i == j else 0.0), F(0)) for j in range(mp)] for i in range(mp)]
    if mp != m:
        A[mp - 1][mp - 1] = (F(1 + 2 * sum(abs(float(A[i][j][0])) for i in range(m) for j in range(m))), F(0))
    half = mp // 2
    for _ in range(max_sweeps):
        off = sum(float(A[i][j][0]) ** 2 for i in range(mp) for j in range(mp) if i != j)
        tot = sum(float(A[i][j][0]) ** 2 for i in range(mp) for j in range(mp))
        if off <= 1e-22 * tot or off == 0:
            break
        for r in range(mp - 1):
            rots = []
            for k in range(half):
                if k == 0:
                    a, b = 0, (r % (mp - 1)) + 1
                else:
                    a, b = ((r + k) % (mp - 1)) + 1, ((r - k + (mp - 1)) % (mp - 1)) + 1
                p, q = min(a, b), max(a, b)
                apq = A[p][q]
                cd, sd = (F(1), F(0)), (F(0), F(0))
                if apq[0] != 0:
                    app, aqq = A[p][p], A[q][q]
                    diff = F(F(aqq[0] - app[0]) + F(aqq[1] - app[1]))
                    with np.errstate(over="ignore"):
                        theta = F(diff / F(F(2) * F(apq[0] + apq[1])))
                        t = F(F(1 if theta >= 0 else -1) / F(abs(theta) + F(np.sqrt(_fma(theta, theta, F(1))))))
                    c = F(1 / np.sqrt(np.float64(_fma(t, t, F(1)))))
                    cd, sd = unit_rotation(c, F(t * c))
                rots.append((p, q, cd, sd))
            for p, q, c, s in rots:
                ms = (-s[0], -s[1])
                for j in range(mp):
                    ap, aq = A[p][j], A[q][j]
                    A[p][j] = df_add(df_mul(c, ap), df_mul(ms, aq))
                    A[q][j] = df_add(df_mul(s, ap), df_mul(c, aq))
            for p, q, c, s in rots:
                ms = (-s[0], -s[1])
                for i in range(mp):
                    ap, aq = A[i][p], A[i][q]
                    A[i][p] = df_add(df_mul(c, ap), df_mul(ms, aq))
                    A[i][q] = df_add(df_mul(s, ap), df_mul(c, aq))
                    vp, vq = V[i][p], V[i][q]
                    V[i][p] = df_add(df_mul(c, vp), df_mul(ms, vq))
                    V[i][q] = df_add(df_mul(s, vp), df_mul(c, vq))
    lam = np.array([float(A[i][i][0]) + float(A[i][i][1]) for i in range(m)])
    vec = np.array([[float(V[i][j][0]) + float(V[i][j][1]) for j in range(m)] for i in range(m)])
    return lam, vec


def test_split_is_exact_to_48_bits():
    rng = np.random.default_rng(0)
    xs = rng.standard_normal(400) * np.exp(rng.uniform(-40, 40, 400))
    for x in xs:
        h, l = split_df(float(x))
        assert abs(float(h) + float(l) - x) <= 2.0 ** -47 * abs(x)
        # hi is x truncated to 24 significant bits: same sign, no larger in magnitude
        assert abs(float(h)) <= abs(x) and (float(h) == 0 or np.sign(float(h)) == np.sign(x))
    assert split_df(3e-31) == (0.0, 0.0)
    assert split_df(0.0) == (0.0, 0.0)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dot_product_of_one_gram_chunk(seed):
    rng = np.random.default_rng(seed)
    n = 256
    x = rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))
    y = rng.standard_normal(n)
    s, c = F(0), F(0)
    for a, b in zip(x, y):
        s, c = df_fma(s, c, split_df(float(a)), split_df(float(b)))
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y))
    err = abs(Fraction(float(s)) + Fraction(float(c)) - exact)
    assert float(err) <= 1e-13 * float(np.sum(np.abs(x * y)))


@pytest.mark.parametrize("m,seed", [(7, 4), (10, 5)])
def test_jacobi_eigenpairs(m, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, m))
    G = X + X.T
    G[0, 1] = G[1, 0] = 1e-9  # a nearly decoupled pair
    lam, vec = jacobi_df(G)
    scale = np.linalg.norm(G, 2)
    assert np.max(np.abs(np.sort(lam) - np.linalg.eigvalsh(G))) <= 1e-12 * scale
    assert np.max(np.linalg.norm(G @ vec - vec * lam, axis=0)) <= 1e-12 * scale
    assert np.max(np.abs(vec.T @ vec - np.eye(m))) <= 1e-13


def test_rotation_renormalisation():
    rng = np.random.default_rng(6)
    for t in rng.standard_normal(200) * 10:
        t = F(t)
        c = F(1 / np.sqrt(np.float64(_fma(t, t, F(1)))))
        (ch, cl), (sh, sl) = unit_rotation(c, F(t * c))
        cc = Fraction(float(ch)) + Fraction(float(cl))
        ss = Fraction(float(sh)) + Fraction(float(sl))
        assert abs(float(cc * cc + ss * ss - 1)) <= 2.0 ** -45
