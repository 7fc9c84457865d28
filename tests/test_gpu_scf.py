"""FP64 SCF energies on the GPU against the oracle (bar: 1e-8 Eh)."""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bqc():
    import paper_2502_17963_gb300 as m
    return m


@pytest.mark.parametrize("name", ["h2o", "w2", "w4"])
def test_scf_energy_fp64(gpu_ctx, bqc, name):
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=False)
    r = bqc.scf_run(gpu_ctx, df, keep_arrays=True)
    I = oracle.system_integrals(mol)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    ro = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), mol.nocc, I["enuc"])
    assert r["converged"] and ro.converged
    assert abs(r["energy"] - ro.energy) < 1e-8, (r["energy"], ro.energy)
    assert r["diis_err"] < 1e-8
    # same density
    C = r["C"].cpu().numpy()[:, : mol.nocc]
    D = C @ C.T
    assert np.abs(D - ro.D).max() < 1e-6


@pytest.mark.parametrize("prec", [0, 2])
def test_scf_on_own_stream_graph_replay(gpu_ctx, bqc, prec):
    """On a non-default stream the per-iteration Fock build is captured into a
    CUDA graph and replayed; the energy must not change."""
    import torch
    mol = workload.water_cluster(3)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=True)
    st = torch.cuda.Stream()
    r = bqc.scf_run(gpu_ctx, df, prec=prec, stream=st)
    torch.cuda.synchronize()
    r0 = bqc.scf_run(gpu_ctx, df, prec=prec)  # default stream: direct launches
    assert r["converged"] and r0["converged"]
    assert abs(r["energy"] - r0["energy"]) < 1e-10
    assert r["iterations"] == r0["iterations"]


def test_scf_resume_from_checkpoint(gpu_ctx, bqc):
    """Checkpoint / resume: an SCF stopped after a few iterations restarts
    from its occupied orbitals (bqc_scf_opts.guess_C) and reaches the
    uninterrupted energy; restarting from converged orbitals converges at
    once."""
    mol = workload.molecule_for("w4")
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis)
    no = basis.nocc
    full = bqc.scf_run(gpu_ctx, df, prec=bqc.PREC_FP64)
    part = bqc.scf_run(gpu_ctx, df, prec=bqc.PREC_FP64, max_iter=4, keep_arrays=True)
    assert full["converged"] and not part["converged"]
    res = bqc.scf_run(gpu_ctx, df, prec=bqc.PREC_FP64, keep_arrays=True,
                      guess=part["C"][:, :no].contiguous())
    assert res["converged"] and abs(res["energy"] - full["energy"]) < 1e-8
    again = bqc.scf_run(gpu_ctx, df, prec=bqc.PREC_FP64, guess=res["C"][:, :no].contiguous())
    assert again["converged"] and again["iterations"] <= 3, again
    assert abs(again["energy"] - full["energy"]) < 1e-8
