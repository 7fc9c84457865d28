"""Pins of the oracle integrals: closed forms, brute-force quadrature, symmetry."""
import math

import numpy as np
import pytest

import bruteforce as bf
import oracle
from oracle.ints import OracleBasis
from workload import Shell


def _basis(specs):
    """specs: list of (l, exponent, centre) -> (OracleBasis, list of bf functions per fn)."""
    xyz = np.array([c for (_, _, c) in specs], dtype=float)
    shells = [Shell(i, l, [a], [1.0]) for i, (l, a, _) in enumerate(specs)]
    ob = OracleBasis(shells, xyz)
    fns = []
    for (l, a, c) in specs:
        for ijk in bf.cart(l):
            fns.append((a, np.array(c, dtype=float), ijk))
    return ob, fns


CEN = [np.array([0.0, 0.0, 0.0]), np.array([0.4, -0.3, 0.9]), np.array([-0.7, 0.5, 0.2]),
       np.array([1.1, 0.8, -0.6])]


def test_s_overlap_closed_form():
    ob, fns = _basis([(0, 0.7, CEN[0]), (0, 0.25, CEN[1])])
    S = oracle.one_electron("S", ob)
    a, b = 0.7, 0.25
    p = a + b
    ref = (4 * a * b / p ** 2) ** 0.75 * math.exp(-a * b / p * np.sum((CEN[0] - CEN[1]) ** 2))
    assert abs(S[0, 1] - ref) < 1e-15
    assert abs(S[0, 0] - 1.0) < 1e-15


def test_ssss_and_3c_2c_closed_forms():
    a, b, c, d = 0.9, 0.35, 0.6, 1.4
    A, B, C, D = CEN
    ob, _ = _basis([(0, a, A), (0, b, B), (0, c, C), (0, d, D)])
    eri = oracle.int4c(ob)

    def F0(T):
        return 1.0 if T < 1e-14 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))

    def g(e1, X1, e2, X2, e3, X3, e4, X4):
        p, q = e1 + e2, e3 + e4
        P, Q = (e1 * X1 + e2 * X2) / p, (e3 * X3 + e4 * X4) / q
        K = math.exp(-e1 * e2 / p * np.sum((X1 - X2) ** 2) - e3 * e4 / q * np.sum((X3 - X4) ** 2))
        n = np.prod([(2 * e / math.pi) ** 0.75 for e in (e1, e2, e3, e4)])
        return n * 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * K * F0(p * q / (p + q) * np.sum((P - Q) ** 2))

    assert abs(eri[0, 1, 2, 3] - g(a, A, b, B, c, C, d, D)) < 1e-14
    # 3-centre (P|mu nu): aux s on C; 2-centre (P|Q)
    aux, _ = _basis([(0, c, C), (0, d, D)])
    orb, _ = _basis([(0, a, A), (0, b, B)])
    t3 = oracle.int3c(aux, orb)
    p = a + b
    P = (a * A + b * B) / p
    K = math.exp(-a * b / p * np.sum((A - B) ** 2))
    T = p * c / (p + c) * np.sum((P - C) ** 2)
    n3 = np.prod([(2 * e / math.pi) ** 0.75 for e in (a, b, c)])
    ref3 = n3 * 2 * math.pi ** 2.5 / (p * c * math.sqrt(p + c)) * K * F0(T)
    assert abs(t3[0, 0, 1] - ref3) < 1e-14
    V = oracle.int2c(aux)
    T2 = c * d / (c + d) * np.sum((C - D) ** 2)
    n2 = np.prod([(2 * e / math.pi) ** 0.75 for e in (c, d)])
    ref2 = n2 * 2 * math.pi ** 2.5 / (c * d * math.sqrt(c + d)) * F0(T2)
    assert abs(V[0, 1] - ref2) < 1e-14


def test_long_range_charge_limit():
    """(a|c) -> q_a q_c / R for well separated s functions (q = int phi)."""
    a, c = 1.3, 0.8
    R = 40.0
    aux, _ = _basis([(0, a, np.zeros(3)), (0, c, np.array([0.0, 0.0, R]))])
    V = oracle.int2c(aux)
    q = lambda e: (2 * e / math.pi) ** 0.75 * (math.pi / e) ** 1.5
    assert abs(V[0, 1] - q(a) * q(c) / R) < 1e-13


SPECS = [(1, 0.55, CEN[0]), (2, 0.8, CEN[1]), (3, 0.45, CEN[2]), (0, 1.7, CEN[3])]


@pytest.mark.parametrize("la,lb", [(1, 2), (2, 2), (0, 1)])
def test_one_electron_vs_quadrature(la, lb):
    specs = [(la, 0.55, CEN[0]), (lb, 0.8, CEN[1])]
    ob, fns = _basis(specs)
    S = oracle.one_electron("S", ob)
    T = oracle.one_electron("T", ob)
    Zs = np.array([1, 8], dtype=np.int32)
    Cs = np.array([CEN[2], CEN[3]])
    V = oracle.one_electron("V", ob, Zs, Cs)
    rng = np.random.default_rng(0)
    n = len(fns)
    for _ in range(6):
        i, j = rng.integers(0, n, 2)
        assert abs(S[i, j] - bf.overlap(fns[i], fns[j])) < 1e-13
        assert abs(T[i, j] - bf.kinetic(fns[i], fns[j])) < 1e-12
        v = sum(bf.nuclear(fns[i], fns[j], Cs[k], Zs[k]) for k in range(2))
        assert abs(V[i, j] - v) < 2e-11, (i, j, V[i, j], v)


def test_3c_high_l_vs_quadrature():
    """(f|dd), (d|pd), (p|ps) components against the Gaussian-transform quadrature."""
    aux, afn = _basis([(3, 0.45, CEN[2]), (2, 0.3, CEN[3]), (1, 1.2, CEN[0])])
    orb, ofn = _basis([(2, 0.8, CEN[1]), (1, 0.55, CEN[0]), (2, 0.2, CEN[3]), (0, 0.15, CEN[2])])
    t3 = oracle.int3c(aux, orb)
    rng = np.random.default_rng(1)
    for _ in range(8):
        P = rng.integers(0, len(afn))
        m, n = rng.integers(0, len(ofn), 2)
        ref = bf.eri(afn[P], None, ofn[m], ofn[n])
        assert abs(t3[P, m, n] - ref) < 1e-11, (P, m, n, t3[P, m, n], ref)


def test_2c_4c_high_l_vs_quadrature():
    aux, afn = _basis([(3, 0.45, CEN[2]), (2, 0.3, CEN[3])])
    V = oracle.int2c(aux)
    for (P, Q) in [(0, 11), (3, 15), (9, 12), (5, 5)]:
        assert abs(V[P, Q] - bf.eri(afn[P], None, afn[Q], None)) < 1e-11
    orb, ofn = _basis([(1, 0.55, CEN[0]), (2, 0.8, CEN[1])])
    eri = oracle.int4c(orb)
    for idx in [(0, 4, 7, 2), (3, 5, 8, 6), (1, 1, 2, 0)]:
        ref = bf.eri(ofn[idx[0]], ofn[idx[1]], ofn[idx[2]], ofn[idx[3]])
        assert abs(eri[idx] - ref) < 1e-11


def test_permutational_symmetry():
    orb, _ = _basis([(1, 0.55, CEN[0]), (2, 0.8, CEN[1]), (0, 0.3, CEN[2])])
    eri = oracle.int4c(orb)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.abs(eri - eri.transpose(perm)).max() < 1e-14
    aux, _ = _basis([(3, 0.45, CEN[2]), (2, 0.3, CEN[3]), (0, 0.9, CEN[0])])
    t3 = oracle.int3c(aux, orb)
    assert np.abs(t3 - t3.transpose(0, 2, 1)).max() < 1e-14
    V = oracle.int2c(aux)
    assert np.abs(V - V.T).max() < 1e-14
    assert np.linalg.eigvalsh(V).min() > 0


def test_derivative_relation_p_from_s():
    """(s|p_x) = (1/2a) d/dA_x (s|s) at centre A (unnormalised p), 5-point stencil."""
    a, c = 0.7, 0.4
    A = np.array([0.3, -0.2, 0.5])
    C = np.array([-0.6, 0.4, 0.1])

    def ss(Ax):
        Ap = A.copy()
        Ap[0] = Ax
        aux, _ = _basis([(0, c, C), (0, a, Ap)])
        return oracle.int2c(aux)[0, 1]

    h = 1e-3
    d = (-ss(A[0] + 2 * h) + 8 * ss(A[0] + h) - 8 * ss(A[0] - h) + ss(A[0] - 2 * h)) / (12 * h)
    aux, _ = _basis([(0, c, C), (1, a, A)])
    V = oracle.int2c(aux)
    # normalised p_x = N_p (x-A) e; N_p / N_s = sqrt(4a); (x-A)e = (1/2a) d/dA_x e
    pred = d / (2 * a) * math.sqrt(4 * a)
    assert abs(V[0, 1] - pred) < 1e-10
