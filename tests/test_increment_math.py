"""Host-side pins of the arithmetic behind two GPU paths (no GPU needed).

1. The rank-2k exchange increment of the incremental FP64 stage: the current
   occupied orbitals C_k are rotated onto the anchor's C_a by the orthogonal
   polar factor R of M = C_k^T S C_a, computed as M (M^T M)^(-1/2) from the
   eigen-decomposition of M^T M (the library's route), which must equal U V^T
   of M's SVD (orthogonal Procrustes in the S metric).  Then with
   C_t = C_k R, C_d = C_t - C_a and C_w = (C_a + C_t) / 2:
   C_t C_t^T = C_k C_k^T, D_k - D_a = C_w C_d^T + C_d C_w^T exactly, and
   |C_d| shrinks with the change of the occupied space (not with the
   arbitrary rotation inside it), and K[dD] built from W = B C_w and
   Y = B C_d as sum_P W_P Y_P^T + Y_P W_P^T equals K[D_k] - K[D_a].
2. Float-float accumulation as the J pass does it on the FP32 pipe: terms
   w_P B_P with w and B held as float pairs (hi = fl(x), lo = fl(x - hi)),
   the exact product of the hi parts from one FMA, the two cross terms, and a
   two-sum into the running pair; the result must match the exact sum within
   a few 2^-46 of sum |terms| (48-bit pairs), while a plain FP32 sum is
   ~2^-24 off.  The emulation uses numpy float32 scalars, whose
   multiply-add is rounded separately, so the FMA is written as the exact
   FP64 product of two floats plus the addend, rounded to FP32 (a fused
   multiply-add's value up to the rare double rounding of that FP64 sum).
"""
from fractions import Fraction

import numpy as np
import pytest


def _spd(n, rng):
    A = rng.standard_normal((n, n))
    return A @ A.T / n + np.eye(n)


def _s_orthonormal(C, S):
    G = C.T @ S @ C
    w, V = np.linalg.eigh(G)
    return C @ (V @ np.diag(w ** -0.5) @ V.T)


def _polar_by_eigh(M):
    lam, V = np.linalg.eigh(M.T @ M)
    return M @ (V @ np.diag(lam ** -0.5) @ V.T)


@pytest.mark.parametrize("n,no,eps", [(30, 6, 1e-3), (60, 12, 1e-5), (40, 15, 1e-7)])
def test_procrustes_rank2k_identity(n, no, eps):
    rng = np.random.default_rng(n * 100 + no)
    S = _spd(n, rng)
    Ca = _s_orthonormal(rng.standard_normal((n, no)), S)
    # the same occupied space rotated arbitrarily, then changed by eps
    Q, _ = np.linalg.qr(rng.standard_normal((no, no)))
    Ck = _s_orthonormal(Ca @ Q + eps * rng.standard_normal((n, no)), S)
    M = Ck.T @ S @ Ca
    R = _polar_by_eigh(M)
    U, _, Vt = np.linalg.svd(M)
    np.testing.assert_allclose(R, U @ Vt, atol=1e-10)
    np.testing.assert_allclose(R.T @ R, np.eye(no), atol=1e-12)
    Ct = Ck @ R
    Dk, Da = Ck @ Ck.T, Ca @ Ca.T
    np.testing.assert_allclose(Ct @ Ct.T, Dk, atol=1e-12)
    Cd = Ct - Ca
    Cw = 0.5 * (Ca + Ct)
    np.testing.assert_allclose(Cw @ Cd.T + Cd @ Cw.T, Dk - Da, atol=1e-12)
    # the rotation Q does not enter C_d: it is of the order of the change eps
    assert np.abs(Cd).max() < 50 * eps * max(1.0, np.abs(Ca).max())
    # without the alignment the difference is of order one
    assert np.abs(Ck - Ca).max() > 100 * np.abs(Cd).max()


def test_rank2k_exchange_equals_difference_of_K():
    rng = np.random.default_rng(7)
    n, no, naux = 20, 5, 30
    S = _spd(n, rng)
    B = rng.standard_normal((naux, n, n))
    B = B + B.transpose(0, 2, 1)
    Ca = _s_orthonormal(rng.standard_normal((n, no)), S)
    Ck = _s_orthonormal(Ca + 1e-3 * rng.standard_normal((n, no)), S)
    R = _polar_by_eigh(Ck.T @ S @ Ca)
    Ct = Ck @ R
    Cd, Cw = Ct - Ca, 0.5 * (Ct + Ca)
    W = np.einsum("pmn,ni->pmi", B, Cw)
    Y = np.einsum("pmn,ni->pmi", B, Cd)
    Kinc = np.einsum("pmi,pni->mn", W, Y) + np.einsum("pmi,pni->mn", Y, W)

    def K(C):
        X = np.einsum("pmn,ni->pmi", B, C)
        return np.einsum("pmi,pni->mn", X, X)

    np.testing.assert_allclose(Kinc, K(Ck) - K(Ca), atol=1e-11)


f32 = np.float32


def _pair(x):
    h = f32(x)
    return h, f32(x - float(h))


def _fma(a, b, c):
    """fl(a b + c) with one rounding (exact FP64 product of two floats)."""
    return f32(float(a) * float(b) + float(c))


def _ff_acc(sh, sl, wh, wl, bh, bl):
    p = f32(wh * bh)
    e = _fma(wh, bh, -p)
    e = _fma(wh, bl, e)
    e = _fma(wl, bh, e)
    t = f32(sh + p)
    bp = f32(t - sh)
    err = f32(f32(sh - f32(t - bp)) + f32(p - bp))
    return t, f32(sl + f32(err + e))


@pytest.mark.parametrize("seed,cancel", [(1, 1.0), (2, 1e3)])
def test_float_float_accumulation(seed, cancel):
    rng = np.random.default_rng(seed)
    m = 2000
    w = rng.standard_normal(m) * cancel
    b = rng.standard_normal(m)
    # make the sum cancel: subtract the mean contribution through the last term
    w[-1] -= float(np.dot(w, b)) / b[-1]
    # exact reference: rational arithmetic on the FP64 inputs
    exact = float(sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(w, b)))
    absum = float(np.sum(np.abs(w * b)))
    sh, sl = f32(0), f32(0)
    plain = f32(0)
    for x, y in zip(w, b):
        wh, wl = _pair(x)
        bh, bl = _pair(y)
        sh, sl = _ff_acc(sh, sl, wh, wl, bh, bl)
        plain = f32(plain + f32(f32(x) * f32(y)))
    ff = float(sh) + float(sl)
    assert abs(ff - exact) <= 4 * 2.0 ** -46 * absum
    # a plain FP32 sum is orders of magnitude worse
    assert abs(float(plain) - exact) > 100 * abs(ff - exact)
