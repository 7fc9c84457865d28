"""DF-MP2 on the GPU (bqc_mp2) against the oracle.

  * arithmetic: the oracle's canonical orbitals and energies handed to both
    sides, E2 equal to 1e-10 Eh (single water, (H2O)_3, and (H2O)_8 whose 40
    occupied orbitals run as ragged blocks of 16, 16 and 8);
  * end to end: the GPU's own SCF orbitals (bqc_scf_run) into bqc_mp2 against
    the oracle's SCF + MP2, to 1e-8 Eh;
  * the degenerate case of no virtual orbitals (nmo = nocc) gives E2 = 0, and
    a direct-mode handle is refused;
  * MIXED_F16X3 (pair blocks on the tensor cores, split FP16): within 2^-18
    of the absolute sum of the MP2 terms, sum |(ia|jb)[2(ia|jb) - (ib|ja)] /
    (e_i + e_j - e_a - e_b)| (the integrals carry ~2^-22 relative rounding and
    the energy is linear in each of them to first order).
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


@pytest.mark.parametrize("name", ["h2o", "w3", "w8"])
def test_mp2_f16x3_against_oracle(gpu_ctx, bqc, name):
    import torch
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=False)
    B, r = _oracle_scf(mol)
    no = mol.nocc
    ovov = oracle.ovov_df(B, r.C, no)
    e_o = oracle.mp2_energy(ovov, r.eps, no)
    eo, ev = r.eps[:no], r.eps[no:]
    den = eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] \
        - ev[None, None, None, :]
    absum = float(np.sum(np.abs(ovov * (2.0 * ovov - ovov.transpose(0, 3, 2, 1)) / den)))
    Cg, eg = torch.tensor(r.C, device="cuda"), torch.tensor(r.eps, device="cuda")
    e_g = bqc.mp2(df, Cg, eg, prec=bqc.PREC_MIXED_F16X3)
    e_g2 = bqc.mp2(df, Cg, eg, prec=bqc.PREC_MIXED_F16X3)
    ratio = abs(e_g - e_o) / absum
    print(f"{name}: F16X3 E2 {e_g:.12f} oracle {e_o:.12f} diff {e_g - e_o:.2e} "
          f"(ratio to the absolute term sum {ratio:.2e})")
    assert e_g == e_g2  # deterministic: fixed-order reductions, no atomics
    assert ratio < 2.0 ** -18
