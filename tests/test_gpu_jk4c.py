"""Conventional (non-DF) direct J/K from four-centre integrals (DF mode NONE).

  * J and K against the oracle's full four-centre contraction
    (oracle.jk_4c over its own McMurchie-Davidson (mu nu|lambda sigma)) for
    seeded occupied orbitals, element by element to 1e-10, with screening off
    and at 1e-12 (single water, (H2O)_2 and (H2O)_3: every pair class from
    (ss|ss) to (dd|dd), shells that coincide in bra, ket and across);
  * the SCF on these J/K (bqc_scf_run, FP64) against the oracle's 4-centre
    RHF to 1e-8 Eh, and the textbook H2/STO-3G energy;
  * the quartet screening keeps fewer quartets than it considers for two
    waters far apart, with the energy unchanged; mixed precisions are
    refused.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workload
from workload import Molecule, Shell

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(__file__)


@pytest.fixture(scope="module")
def bqc():
    import paper_2502_17963_gb300 as m
    return m


@pytest.mark.parametrize("name", ["h2o", "w2", "w3"])
@pytest.mark.parametrize("tau", [0.0, 1e-12])
def test_jk4c_against_oracle(gpu_ctx, bqc, name, tau):
    import torch
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, mode=bqc.DF_NONE, schwarz=tau)
    I = oracle.system_integrals(mol)
    eri = oracle.int4c(I["orb"])
    rng = np.random.default_rng(41)
    C = rng.standard_normal((basis.nbf, basis.nocc)) * 0.3
    J, K = df.jk(torch.tensor(C, device="cuda"), bqc.PREC_FP64)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    Jo, Ko = oracle.jk_4c(eri, C)
    dJ, dK = np.abs(J - Jo).max(), np.abs(K - Ko).max()
    cand, kept = df.screening()
    print(f"{name} tau {tau:g}: max|dJ| {dJ:.2e} max|dK| {dK:.2e} (max|J| {np.abs(Jo).max():.2e}),"
          f" quartets kept {kept}/{cand}")
    assert (J == J.T).all() and (K == K.T).all()
    assert dJ < 1e-10 and dK < 1e-10


@pytest.mark.parametrize("name", ["h2o", "w2"])
def test_scf_4c_against_oracle(gpu_ctx, bqc, name):
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, mode=bqc.DF_NONE)
    r = bqc.scf_run(gpu_ctx, df)
    I = oracle.system_integrals(mol)
    eri = oracle.int4c(I["orb"])
    ro = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_4c(eri, C), mol.nocc, I["enuc"])
    print(f"{name}: 4c SCF gpu {r['energy']:.10f} oracle {ro.energy:.10f}")
    assert r["converged"] and abs(r["energy"] - ro.energy) < 1e-8
    with pytest.raises(bqc.BqcError) as e:
        bqc.scf_run(gpu_ctx, df, prec=bqc.PREC_MIXED_TF32X3)
    assert e.value.status == -9


def test_h2_sto3g_textbook_energy_4c(gpu_ctx, bqc):
    g = json.load(open(os.path.join(HERE, "golden", "h2_sto3g.json")))
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, g["R_bohr"]]])
    orb = [Shell(i, 0, g["sto3g_exponents"], g["sto3g_coefficients"]) for i in range(2)]
    mol = Molecule(np.array([1, 1], dtype=np.int32), xyz, orb, orb, "H2")
    basis = bqc.Basis(gpu_ctx, mol)
    r = bqc.scf_run(gpu_ctx, bqc.DF(gpu_ctx, basis, mode=bqc.DF_NONE))
    assert r["converged"] and abs(r["energy"] - g["E_total"]) < g["tolerance"]


def test_far_apart_dimer_quartet_screening(gpu_ctx, bqc):
    w = workload.single_water()
    shift = np.array([60.0, 0.0, 0.0])
    n1 = len(w.Z)
    mol = Molecule(np.concatenate([w.Z, w.Z]), np.vstack([w.xyz, w.xyz + shift]),
                   w.orb + [Shell(s.atom + n1, s.l, s.exps, s.coefs) for s in w.orb],
                   w.aux + [Shell(s.atom + n1, s.l, s.exps, s.coefs) for s in w.aux], "far")
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, mode=bqc.DF_NONE, schwarz=1e-12)
    cand, kept = df.screening()
    assert kept < 0.5 * cand
    r = bqc.scf_run(gpu_ctx, df)
    rm = bqc.scf_run(gpu_ctx, bqc.DF(gpu_ctx, bqc.Basis(gpu_ctx, w), mode=bqc.DF_NONE))
    assert r["converged"] and abs(r["energy"] - 2 * rm["energy"]) < 1e-4
