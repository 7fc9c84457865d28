"""DF-MP2 on the GPU (bqc_mp2) against the oracle.

  * arithmetic: the oracle's canonical orbitals and energies handed to both
    sides, E2 equal to 1e-10 Eh (single water, (H2O)_3, and (H2O)_8 whose 40
    occupied orbitals run as ragged blocks of 16, 16 and 8);
  * end to end: the GPU's own SCF orbitals (bqc_scf_run) into bqc_mp2 against
    the oracle's SCF + MP2, to 1e-8 Eh;
  * the degenerate case of no virtual orbitals (nmo = nocc) gives E2 = 0, and
    a direct-mode handle is refused.
"""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bqc():
    import paper_2502_17963_gb300 as m
    return m


def _oracle_scf(mol):
    I = oracle.system_integrals(mol)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    r = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), mol.nocc, I["enuc"])
    assert r.converged
    return B, r


@pytest.mark.parametrize("name", ["h2o", "w3", "w8"])
def test_mp2_arithmetic_against_oracle(gpu_ctx, bqc, name):
    import torch
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=False)
    B, r = _oracle_scf(mol)
    e_o = oracle.mp2_energy(oracle.ovov_df(B, r.C, mol.nocc), r.eps, mol.nocc)
    e_g = bqc.mp2(df, torch.tensor(r.C, device="cuda"), torch.tensor(r.eps, device="cuda"))
    print(f"{name}: E2 gpu {e_g:.12f} oracle {e_o:.12f} diff {e_g - e_o:.2e}")
    assert e_o < 0.0
    assert abs(e_g - e_o) < 1e-10


@pytest.mark.parametrize("name", ["h2o", "w4"])
def test_mp2_end_to_end(gpu_ctx, bqc, name):
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=False)
    rg = bqc.scf_run(gpu_ctx, df, keep_arrays=True)
    assert rg["converged"]
    e_g = bqc.mp2(df, rg["C"], rg["eps"])
    B, r = _oracle_scf(mol)
    e_o = oracle.mp2_energy(oracle.ovov_df(B, r.C, mol.nocc), r.eps, mol.nocc)
    print(f"{name}: SCF+MP2 gpu {rg['energy'] + e_g:.10f} oracle {r.energy + e_o:.10f}")
    assert abs(e_g - e_o) < 1e-8


def test_mp2_edge_cases(gpu_ctx, bqc):
    import torch
    mol = workload.single_water()
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=False)
    _, r = _oracle_scf(mol)
    C = torch.tensor(r.C[:, :mol.nocc].copy(), device="cuda")
    eps = torch.tensor(r.eps[:mol.nocc].copy(), device="cuda")
    assert bqc.mp2(df, C, eps) == 0.0  # no virtual orbitals
    dd = bqc.DF(gpu_ctx, basis, mode=bqc.DF_DIRECT, keep_fp32=False)
    with pytest.raises(bqc.BqcError) as e:
        bqc.mp2(dd, torch.tensor(r.C, device="cuda"), torch.tensor(r.eps, device="cuda"))
    assert e.value.status == -1
