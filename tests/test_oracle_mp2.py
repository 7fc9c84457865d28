"""Pins of the oracle MP2 energy (closed shell, canonical orbitals).

  * textbook H2/STO-3G: the molecular-orbital integrals J11, J12, J22, K12 and
    the second-order energy as printed by Szabo & Ostlund;
  * the closed-shell spatial-orbital formula equals the spin-orbital one
    (1/4 sum |<IJ||AB>|^2 / D), a separate route that a wrong factor, a
    swapped exchange index or a wrong denominator sign fails;
  * DF-MP2 equals 4-centre MP2 when the auxiliary set spans every orbital
    product (He, even-tempered s; aux = pairwise exponent sums);
  * invariance under rigid rotation and translation (water dimer with
    Cartesian d shells), and E2 < 0.
"""
import json
import os

import numpy as np

import oracle
from oracle.ints import OracleBasis
from workload import Molecule, Shell, water_cluster

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _scf_4c(mol):
    I = oracle.system_integrals(mol)
    eri = oracle.int4c(I["orb"])
    r = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_4c(eri, C), mol.nocc, I["enuc"])
    assert r.converged
    return I, eri, r


def test_h2_sto3g_mp2_szabo_ostlund():
    g0 = json.load(open(os.path.join(GOLD, "h2_sto3g.json")))
    g = json.load(open(os.path.join(GOLD, "h2_sto3g_mp2.json")))
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, g0["R_bohr"]]])
    sh = [Shell(i, 0, g0["sto3g_exponents"], g0["sto3g_coefficients"]) for i in range(2)]
    mol = Molecule(np.array([1, 1], dtype=np.int32), xyz, sh, sh, "H2")
    I, eri, r = _scf_4c(mol)
    C = r.C
    mo = np.einsum("mnls,mp,nq,lr,st->pqrt", eri, C, C, C, C, optimize=True)
    tol = g["tolerance"]
    assert abs(mo[0, 0, 0, 0] - g["J11"]) < tol
    assert abs(mo[0, 0, 1, 1] - g["J12"]) < tol
    assert abs(mo[1, 1, 1, 1] - g["J22"]) < tol
    assert abs(mo[0, 1, 0, 1] - g["K12"]) < tol
    ovov = oracle.ovov_4c(eri, C, 1)
    assert abs(ovov[0, 0, 0, 0] - g["K12"]) < tol
    e2 = oracle.mp2_energy(ovov, r.eps, 1)
    assert abs(e2 - g["E2"]) < tol


def test_closed_shell_formula_equals_spin_orbital_form():
    mol = water_cluster(1)
    I = oracle.system_integrals(mol)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    r = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), mol.nocc, I["enuc"])
    ovov = oracle.ovov_df(B, r.C, mol.nocc)
    e_cs = oracle.mp2_energy(ovov, r.eps, mol.nocc)
    e_so = oracle.mp2_energy_spin_orbital(ovov, r.eps, mol.nocc)
    assert e_cs < 0.0
    assert abs(e_cs - e_so) < 1e-12 * abs(e_cs)


def test_df_mp2_exact_when_aux_spans_products():
    exps = [0.3 * 3.0 ** k for k in range(4)]
    aux = sorted({a + b for a in exps for b in exps})
    mol = Molecule(np.array([2], dtype=np.int32), np.zeros((1, 3)),
                   [Shell(0, 0, [e], [1.0]) for e in exps],
                   [Shell(0, 0, [e], [1.0]) for e in aux], "He")
    I, eri, r = _scf_4c(mol)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    e4 = oracle.mp2_energy(oracle.ovov_4c(eri, r.C, 1), r.eps, 1)
    edf = oracle.mp2_energy(oracle.ovov_df(B, r.C, 1), r.eps, 1)
    assert e4 < 0.0
    assert abs(e4 - edf) < 1e-10


def _rotated(mol, R, t):
    return Molecule(mol.Z.copy(), mol.xyz @ R.T + t, mol.orb, mol.aux, mol.name)


def test_mp2_invariant_under_rigid_motion():
    mol = water_cluster(2)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0, 0, 1.0]])
    R = R @ np.array([[1, 0, 0], [0, np.cos(0.4), -np.sin(0.4)], [0, np.sin(0.4), np.cos(0.4)]])
    es = []
    for m in (mol, _rotated(mol, R, np.array([1.3, -0.7, 2.1]))):
        I = oracle.system_integrals(m)
        B, _ = oracle.df_tensor(I["aux"], I["orb"])
        r = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), m.nocc, I["enuc"])
        es.append(oracle.mp2_energy(oracle.ovov_df(B, r.C, m.nocc), r.eps, m.nocc))
    assert es[0] < 0.0
    assert abs(es[0] - es[1]) < 1e-9
