"""Brute-force quadrature of Gaussian integrals, independent of the oracle.

Used only to pin the oracle.  Every integral is evaluated straight from its
definition with numerical quadrature:
  * 1-D moments of a Gaussian by Gauss-Hermite (exact for polynomials);
  * 1/r = (2/sqrt(pi)) int_0^inf exp(-t^2 r^2) dt, the t-integral by
    Gauss-Legendre after t = s/(1-s);
  * per Cartesian axis the two-electron factor is a 2-D Gaussian integral,
    done by Gauss-Hermite after a Cholesky change of variables.
Functions are single normalised Cartesian primitives (x-A)^i (y-A)^j (z-A)^k
exp(-a |r-A|^2) with N = (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2i-1)!!(2j-1)!!(2k-1)!!).
"""
from __future__ import annotations

import math

import numpy as np

GH_X, GH_W = np.polynomial.hermite.hermgauss(12)


def dfact(n):
    r = 1
    for k in range(n, 0, -2):
        r *= k
    return r


def norm(a, ijk):
    l = sum(ijk)
    return (2 * a / math.pi) ** 0.75 * (4 * a) ** (l / 2) / math.sqrt(
        dfact(2 * ijk[0] - 1) * dfact(2 * ijk[1] - 1) * dfact(2 * ijk[2] - 1))


def cart(l):
    return [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]


def _t_rule(n=600):
    s, w = np.polynomial.legendre.leggauss(n)
    s = 0.5 * (s + 1.0)
    w = 0.5 * w
    t = s / (1.0 - s)
    return t, w / (1.0 - s) ** 2


T_NODES, T_WEIGHTS = _t_rule()


def overlap1d(i, a, A, j, b, B):
    """int (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2) dx by Gauss-Hermite."""
    p = a + b
    P = (a * A + b * B) / p
    K = math.exp(-a * b / p * (A - B) ** 2)
    x = P + GH_X / math.sqrt(p)
    return K / math.sqrt(p) * np.sum(GH_W * (x - A) ** i * (x - B) ** j)


def overlap(f1, f2):
    (a, A, c1), (b, B, c2) = f1, f2
    return norm(a, c1) * norm(b, c2) * np.prod(
        [overlap1d(c1[x], a, A[x], c2[x], b, B[x]) for x in range(3)])


def _dpoly1d(i, a, A, x):
    """d/dx of (x-A)^i exp(-a(x-A)^2), without the exponential."""
    d = x - A
    v = -2.0 * a * d ** (i + 1)
    if i > 0:
        v = v + i * d ** (i - 1)
    return v


def kinetic(f1, f2):
    """T = 1/2 int grad f1 . grad f2 (integration by parts of -1/2 lapl)."""
    (a, A, c1), (b, B, c2) = f1, f2
    p = a + b
    tot = 0.0
    for ax in range(3):
        prod = 1.0
        for x in range(3):
            P = (a * A[x] + b * B[x]) / p
            K = math.exp(-a * b / p * (A[x] - B[x]) ** 2)
            xs = P + GH_X / math.sqrt(p)
            if x == ax:
                g = _dpoly1d(c1[x], a, A[x], xs) * _dpoly1d(c2[x], b, B[x], xs)
            else:
                g = (xs - A[x]) ** c1[x] * (xs - B[x]) ** c2[x]
            prod *= K / math.sqrt(p) * np.sum(GH_W * g)
        tot += prod
    return 0.5 * norm(a, c1) * norm(b, c2) * tot


def nuclear(f1, f2, C, Z=1.0):
    """-Z int f1 f2 / |r - C| via the Gaussian transform of 1/r."""
    (a, A, c1), (b, B, c2) = f1, f2
    vals = np.ones_like(T_NODES)
    for x in range(3):
        p = a + b
        P = (a * A[x] + b * B[x]) / p
        K = math.exp(-a * b / p * (A[x] - B[x]) ** 2)
        t2 = T_NODES ** 2
        q = p + t2
        Pc = (p * P + t2 * C[x]) / q
        Kc = np.exp(-p * t2 / q * (P - C[x]) ** 2)
        xs = Pc[:, None] + GH_X[None, :] / np.sqrt(q)[:, None]
        g = (xs - A[x]) ** c1[x] * (xs - B[x]) ** c2[x]
        vals = vals * K * Kc / np.sqrt(q) * np.sum(GH_W[None, :] * g, axis=1)
    return -Z * norm(a, c1) * norm(b, c2) * 2.0 / math.sqrt(math.pi) * np.sum(T_WEIGHTS * vals)


def _pair_axis(fa, fb, x):
    """Exponent, centre, prefactor and polynomial factors of a product on one axis."""
    if fb is None:
        a, A, c = fa
        return a, A[x], 1.0, [(A[x], c[x])]
    (a, A, c1), (b, B, c2) = fa, fb
    p = a + b
    P = (a * A[x] + b * B[x]) / p
    return p, P, math.exp(-a * b / p * (A[x] - B[x]) ** 2), [(A[x], c1[x]), (B[x], c2[x])]


def eri(fa, fb, fc, fd):
    """(ab|cd) with b and/or d None for 3- and 2-centre integrals."""
    L = np.linalg.cholesky
    vals = np.ones_like(T_NODES)
    Y1, Y2 = np.meshgrid(GH_X, GH_X, indexing="ij")
    W = np.outer(GH_W, GH_W)
    for x in range(3):
        p, P, K1, pol1 = _pair_axis(fa, fb, x)
        q, Q, K2, pol2 = _pair_axis(fc, fd, x)
        acc = np.empty_like(T_NODES)
        for it, t in enumerate(T_NODES):
            t2 = t * t
            M = np.array([[p + t2, -t2], [-t2, q + t2]])
            mu = np.linalg.solve(M, np.array([p * P, q * Q]))
            const = -(p * P * P + q * Q * Q) + mu @ M @ mu
            R = L(M)                              # M = R R^T
            Rinv_T = np.linalg.inv(R).T
            x1 = mu[0] + Rinv_T[0, 0] * Y1 + Rinv_T[0, 1] * Y2
            x2 = mu[1] + Rinv_T[1, 0] * Y1 + Rinv_T[1, 1] * Y2
            g = np.ones_like(x1)
            for (c, e) in pol1:
                g = g * (x1 - c) ** e
            for (c, e) in pol2:
                g = g * (x2 - c) ** e
            acc[it] = math.exp(const) / np.prod(np.diag(R)) * np.sum(W * g)
        vals = vals * K1 * K2 * acc
    n = norm(fa[0], fa[2]) * norm(fc[0], fc[2])
    if fb is not None:
        n *= norm(fb[0], fb[2])
    if fd is not None:
        n *= norm(fd[0], fd[2])
    return n * 2.0 / math.sqrt(math.pi) * np.sum(T_WEIGHTS * vals)
