"""DF tensor B, its Cholesky factor, and J/K (FP64) against the oracle."""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bqc():
    import paper_2502_17963_gb300 as m
    return m


def _oracle_df(mol):
    I = oracle.system_integrals(mol)
    B, L = oracle.df_tensor(I["aux"], I["orb"])
    return I, B, L


@pytest.mark.parametrize("name", ["h2o", "w2", "w4"])
def test_B_and_L(gpu_ctx, bqc, name):
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, schwarz=0.0, keep_fp32=False)
    I, B, L = _oracle_df(mol)
    Lg = df.copy(1).cpu().numpy()
    V = oracle.int2c(I["aux"])
    # backward error of the factorisation, then the forward error: the metric
    # has cond ~1e8, so one rounding-level change of V moves L by ~2e-10 and
    # B by ~4e-11 (measured on these molecules); the bounds are 5x that.
    assert np.abs(Lg @ Lg.T - V).max() < 1e-12 * np.abs(V).max()
    assert np.abs(np.triu(Lg, 1)).max() == 0.0
    assert np.abs(Lg - L).max() < 1e-9
    Bg = df.copy(0).cpu().numpy()
    r, c = np.tril_indices(basis.nbf)
    Bo = B[:, r, c]
    assert np.abs(Bg - Bo).max() < 5e-10
    # the fitted integrals sum_P B_P,mn B_P,ls are well conditioned
    assert np.abs(Bg.T @ Bg - Bo.T @ Bo).max() < 1e-10


@pytest.mark.parametrize("name", ["h2o", "w3"])
def test_jk_fp64(gpu_ctx, bqc, name):
    import torch
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, schwarz=0.0, keep_fp32=False)
    I, B, _ = _oracle_df(mol)
    rng = np.random.default_rng(5)
    C = rng.standard_normal((basis.nbf, basis.nocc)) * 0.3
    J, K = df.jk(torch.tensor(C, device="cuda"), bqc.PREC_FP64)
    Jr, Kr = oracle.jk_df(B, C)
    assert np.abs(J.cpu().numpy() - Jr).max() < 1e-10
    assert np.abs(K.cpu().numpy() - Kr).max() < 1e-10
    # host entry point gives the same
    Jh, Kh = df.jk_host(C, bqc.PREC_FP64)
    assert np.abs(Jh - Jr).max() < 1e-10 and np.abs(Kh - Kr).max() < 1e-10


def test_jk_rejects_wrong_nocc(gpu_ctx, bqc):
    import torch
    mol = workload.single_water()
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=False)
    with pytest.raises(bqc.BqcError):
        df.jk(torch.zeros((basis.nbf, basis.nocc + 1), dtype=torch.float64, device="cuda"))
