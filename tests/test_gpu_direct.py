"""Direct (on-the-fly) DF: integrals regenerated in aux blocks at each build.

Pins: FP64 direct J/K equal the oracle's DF J/K and the stored-mode J/K (same
method, different evaluation order: gamma/c and Y = L^{-1} X instead of a
stored B; the metric conditioning bounds the difference, see the L/B tests);
mixed direct against FP64 direct at the 3xTF32 level; blocks of 64 and 100
aux functions with ragged last blocks.
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


def _orbitals(mol):
    I = oracle.system_integrals(mol)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    r = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), mol.nocc, I["enuc"], max_iter=2)
    return I, B, r.Cocc


@pytest.mark.parametrize("name,block", [("w3", 64), ("w4", 100)])
def test_direct_fp64_matches_oracle_and_stored(gpu_ctx, bqc, name, block):
    import torch
    mol = workload.molecule_for(name)
    I, B, C = _orbitals(mol)
    basis = bqc.Basis(gpu_ctx, mol)
    dd = bqc.DF(gpu_ctx, basis, mode=bqc.DF_DIRECT, schwarz=0.0, aux_block=block)
    assert dd.mode == bqc.DF_DIRECT
    Cg = torch.tensor(C, device="cuda")
    J, K = [x.cpu().numpy() for x in dd.jk(Cg, bqc.PREC_FP64)]
    Jr, Kr = oracle.jk_df(B, C)
    assert np.abs(J - Jr).max() < 1e-9
    assert np.abs(K - Kr).max() < 1e-9
    ds = bqc.DF(gpu_ctx, basis, schwarz=0.0, keep_fp32=False)
    Js, Ks = [x.cpu().numpy() for x in ds.jk(Cg, bqc.PREC_FP64)]
    assert np.abs(J - Js).max() < 1e-9 and np.abs(K - Ks).max() < 1e-9
    # a second build reuses every buffer
    J2, K2 = [x.cpu().numpy() for x in dd.jk(Cg, bqc.PREC_FP64)]
    assert np.abs(J2 - J).max() < 1e-12 and np.abs(K2 - K).max() < 1e-12


@pytest.mark.parametrize("name,block", [("w4", 64), ("w8", 256), ("w16", 1024)])
def test_direct_mixed_against_fp64(gpu_ctx, bqc, name, block):
    import torch
    mol = workload.molecule_for(name)
    _, _, C = _orbitals(mol)
    basis = bqc.Basis(gpu_ctx, mol)
    dd = bqc.DF(gpu_ctx, basis, mode=bqc.DF_DIRECT, schwarz=0.0, aux_block=block)
    Cg = torch.tensor(C, device="cuda")
    J64, K64 = dd.jk(Cg, bqc.PREC_FP64)
    J, K = dd.jk(Cg, bqc.PREC_MIXED_TF32X3)
    dF = (2 * (J - J64) - (K - K64)).abs().max().item()
    print(name, "direct 3xTF32 max|dF| vs FP64", dF)
    assert (K - K.T).abs().max().item() == 0.0
    assert dF < 1e-4


def test_direct_staged_scf_energy(gpu_ctx, bqc):
    mol = workload.water_cluster(4)
    basis = bqc.Basis(gpu_ctx, mol)
    dd = bqc.DF(gpu_ctx, basis, mode=bqc.DF_DIRECT, schwarz=1e-12, aux_block=128)
    r = bqc.scf_run(gpu_ctx, dd, prec=bqc.PREC_MIXED_TF32X3)
    I = oracle.system_integrals(mol)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    ro = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), mol.nocc, I["enuc"])
    assert r["converged"]
    assert abs(r["energy"] - ro.energy) < 1e-8


def test_auto_mode_picks_stored_when_it_fits(gpu_ctx, bqc):
    basis = bqc.Basis(gpu_ctx, workload.single_water())
    d = bqc.DF(gpu_ctx, basis, mode=bqc.DF_AUTO)
    assert d.mode == bqc.DF_STORED
    d2 = bqc.DF(gpu_ctx, basis, mode=bqc.DF_AUTO, hbm_limit=1024)
    assert d2.mode == bqc.DF_DIRECT
