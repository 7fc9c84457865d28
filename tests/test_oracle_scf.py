"""Pins of the oracle SCF: textbook H2/STO-3G, He HF limit, DF exactness,
rigid-motion invariance and the properties of a converged closed-shell SCF."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle.ints import OracleBasis
from workload import Molecule, Shell, single_water, water_cluster

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_h2_sto3g_szabo_ostlund():
    g = _load("h2_sto3g.json")
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, g["R_bohr"]]])
    shells = [Shell(i, 0, g["sto3g_exponents"], g["sto3g_coefficients"]) for i in range(2)]
    ob = OracleBasis(shells, xyz)
    Z = np.array([1, 1], dtype=np.int32)
    S = oracle.one_electron("S", ob)
    T = oracle.one_electron("T", ob)
    V = oracle.one_electron("V", ob, Z, xyz)
    H = T + V
    eri = oracle.int4c(ob)
    tol = g["tolerance"]
    assert abs(S[0, 1] - g["S12"]) < tol
    assert abs(T[0, 0] - g["T11"]) < tol and abs(T[0, 1] - g["T12"]) < tol
    assert abs(H[0, 0] - g["H11"]) < tol and abs(H[0, 1] - g["H12"]) < tol
    assert abs(eri[0, 0, 0, 0] - g["eri_1111"]) < tol
    assert abs(eri[0, 0, 1, 1] - g["eri_1122"]) < tol
    assert abs(eri[1, 0, 0, 0] - g["eri_2111"]) < tol
    assert abs(eri[1, 0, 1, 0] - g["eri_2121"]) < tol
    enuc = oracle.nuclear_repulsion(Z, xyz)
    r = oracle.rhf(S, H, lambda C: oracle.jk_4c(eri, C), 1, enuc)
    assert r.converged
    assert np.allclose(r.eps, g["eps"], atol=tol)
    assert abs(r.energy - g["E_total"]) < tol


def _he(exps_orb, exps_aux):
    xyz = np.zeros((1, 3))
    m = Molecule(np.array([2], dtype=np.int32), xyz,
                 [Shell(0, 0, [e], [1.0]) for e in exps_orb],
                 [Shell(0, 0, [e], [1.0]) for e in exps_aux], "He")
    return m


def test_he_hf_limit_four_centre():
    g = _load("he_hf_limit.json")
    exps = [0.08 * 2.6 ** k for k in range(12)]
    m = _he(exps, exps)
    I = oracle.system_integrals(m)
    eri = oracle.int4c(I["orb"])
    r = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_4c(eri, C), 1, 0.0)
    assert r.converged
    assert r.energy > g["E_hf_limit"] - 1e-9       # variational
    assert r.energy - g["E_hf_limit"] < 2e-5


def test_df_exact_when_aux_spans_products():
    """Same-centre s products are s Gaussians with summed exponents; with that
    auxiliary set DF reproduces the four-centre integrals and energy."""
    exps = [0.3 * 3.0 ** k for k in range(4)]
    aux = sorted({a + b for a in exps for b in exps})
    m = _he(exps, aux)
    I = oracle.system_integrals(m)
    eri = oracle.int4c(I["orb"])
    B, L = oracle.df_tensor(I["aux"], I["orb"])
    eri_df = np.einsum("pmn,pls->mnls", B, B)
    assert np.abs(eri_df - eri).max() < 1e-10
    r4 = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_4c(eri, C), 1, 0.0)
    rdf = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), 1, 0.0)
    assert abs(r4.energy - rdf.energy) < 1e-10


def test_df_jk_matches_four_centre_contraction_of_fitted_eri():
    """J/K from B equal the 4-index contraction of sum_P B_P B_P (transposed-operand check)."""
    m = water_cluster(2)
    I = oracle.system_integrals(m)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    rng = np.random.default_rng(3)
    C = rng.standard_normal((I["orb"].nfn, m.nocc)) * 0.3
    J, K = oracle.jk_df(B, C)
    eri = np.einsum("pmn,pls->mnls", B, B)
    J4, K4 = oracle.jk_4c(eri, C)
    assert np.abs(J - J4).max() < 1e-11
    assert np.abs(K - K4).max() < 1e-11
    assert np.abs(K - K.T).max() < 1e-12


def _scf(m):
    I = oracle.system_integrals(m)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    return I, oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), m.nocc, I["enuc"])


def test_converged_scf_properties():
    m = single_water()
    I, r = _scf(m)
    assert r.converged and r.diis_err < 1e-8
    S = I["S"]
    assert np.abs(r.D @ S @ r.D - r.D).max() < 1e-9          # idempotent (in the S metric)
    assert abs(np.trace(r.D @ S) - m.nocc) < 1e-10
    assert r.eps[m.nocc] - r.eps[m.nocc - 1] > 0.05          # aufbau gap
    C = r.C
    assert np.abs(C.T @ S @ C - np.eye(C.shape[1])).max() < 1e-9


def _rotate(m, R, shift):
    m2 = Molecule(m.Z.copy(), m.xyz @ R.T + shift, m.orb, m.aux, m.name)
    return m2


def test_energy_invariant_under_rigid_motion():
    m = single_water()
    _, r0 = _scf(m)
    th = 0.7
    R1 = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    ph = -1.1
    R2 = np.array([[1, 0, 0], [0, math.cos(ph), -math.sin(ph)], [0, math.sin(ph), math.cos(ph)]])
    _, r1 = _scf(_rotate(m, R2 @ R1, np.array([0.3, -2.0, 1.7])))
    assert abs(r0.energy - r1.energy) < 1e-10


def test_dimer_energy_invariance_with_d_and_f_shells():
    """Cluster basis has Cartesian d (orbital) and f (aux) shells: still rotation invariant."""
    m = water_cluster(2)
    _, r0 = _scf(m)
    th = 0.9
    R = np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])
    _, r1 = _scf(_rotate(m, R, np.array([-1.0, 0.5, 3.0])))
    assert r0.converged and r1.converged
    assert abs(r0.energy - r1.energy) < 1e-9


def test_packed_aux_blocked_path_equals_plain_path():
    """The aux-blocked oracle (packed B solved in column blocks, J/K summed
    over P blocks) used at cluster sizes whose full-square B does not fit the
    host: the same B, J and K as the plain definitions, on (H2O)_2 with odd
    block sizes so that every block boundary is ragged; and its absolute
    contractions bound the element magnitudes."""
    mol = water_cluster(2)
    I = oracle.system_integrals(mol)
    B, L = oracle.df_tensor(I["aux"], I["orb"])
    Bp, L2 = oracle.df_tensor_packed(I["aux"], I["orb"], col_block=97)
    N = I["orb"].nfn
    assert np.array_equal(L, L2)
    assert np.abs(oracle.unpack_rows(Bp, N) - B).max() < 1e-14
    rng = np.random.default_rng(5)
    C = rng.standard_normal((N, mol.nocc)) * 0.3
    J, K = oracle.jk_df(B, C)
    J2, K2, JA, KA = oracle.jk_df_packed(Bp, N, C, block=13, bounds=True)
    assert np.abs(J - J2).max() < 1e-12 * np.abs(J).max()
    assert np.abs(K - K2).max() < 1e-12 * np.abs(K).max()
    assert (np.abs(J) <= JA * (1 + 1e-12)).all() and (np.abs(K) <= KA * (1 + 1e-12)).all()
    # the packed column of (mu, nu) is mu(mu+1)/2 + nu: spot-check one entry
    mu, nu = 37, 11
    assert Bp[5, mu * (mu + 1) // 2 + nu] == B[5, mu, nu] == B[5, nu, mu]
