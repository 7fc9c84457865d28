"""The Coulomb matrix by the two passes over the stored CD-ERIs (Sec. 2.2):
w = B.D, then J = sum_P w_P B_P, with FP64 FMAs or in float-float arithmetic
on the FP32 pipe over the float-pair copy of B.

Checks: the FP64 variant against the oracle's J (1e-10 absolute) for
D = C C^T; the float-float variant against the FP64 one within 1e-12 of
max|J| (float-float carries ~2^-46 per term), for a physical density and for
an indefinite symmetric matrix (the density differences of the incremental
SCF stage); an odd number of packed elements (the single water, Npair = 351)
takes the scalar tail; a TF32 handle has no float-pair B.
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


@pytest.mark.parametrize("name", ["h2o", "w3", "w8"])
def test_coulomb_variants(gpu_ctx, bqc, name):
    import torch
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=bqc.SHADOW_F16)
    n, no = basis.nbf, basis.nocc
    rng = np.random.default_rng(11)
    C = rng.standard_normal((n, no)) / np.sqrt(n)
    D = C @ C.T
    Jd = df.coulomb(torch.tensor(D, device="cuda"), bqc.COULOMB_FP64)
    Jf = df.coulomb(torch.tensor(D, device="cuda"), bqc.COULOMB_FF)
    I = oracle.system_integrals(mol)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    Jo, _ = oracle.jk_df(B, C)
    Jd_h, Jf_h = Jd.cpu().numpy(), Jf.cpu().numpy()
    assert np.abs(Jd_h - Jo).max() < 1e-10
    scale = np.abs(Jd_h).max()
    assert np.abs(Jf_h - Jd_h).max() <= 1e-12 * scale
    # the same J as the FP64 Fock build
    J64, _ = df.jk(torch.tensor(C, device="cuda"), bqc.PREC_FP64)
    assert np.abs(J64.cpu().numpy() - Jd_h).max() <= 1e-12 * scale
    # an indefinite symmetric matrix (a density difference)
    E = rng.standard_normal((n, n)) * 1e-3
    E = E + E.T
    Jd2 = df.coulomb(torch.tensor(E, device="cuda"), bqc.COULOMB_FP64).cpu().numpy()
    Jf2 = df.coulomb(torch.tensor(E, device="cuda"), bqc.COULOMB_FF).cpu().numpy()
    Jo2 = np.einsum("pmn,p->mn", B, np.einsum("pmn,mn->p", B, E))
    assert np.abs(Jd2 - Jo2).max() < 1e-12 + 1e-10 * np.abs(Jo2).max()
    assert np.abs(Jf2 - Jd2).max() <= 1e-12 * np.abs(Jd2).max()
    df.close()


def test_coulomb_needs_float_pairs(gpu_ctx, bqc):
    import torch
    basis = bqc.Basis(gpu_ctx, workload.molecule_for("w2"))
    df = bqc.DF(gpu_ctx, basis, keep_fp32=bqc.SHADOW_TF32)
    D = torch.zeros((basis.nbf, basis.nbf), dtype=torch.float64, device="cuda")
    J = df.coulomb(D, bqc.COULOMB_FP64)
    assert float(J.abs().max()) == 0.0
    with pytest.raises(bqc.BqcError) as e:
        df.coulomb(D, bqc.COULOMB_FF)
    assert e.value.status == bqc.BQC_E_UNSUPPORTED
    with pytest.raises(bqc.BqcError) as e:
        df.coulomb(D, 7)
    assert e.value.status == bqc.BQC_E_INVALID
    df.close()
