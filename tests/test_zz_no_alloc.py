"""The allocation-free FP64 Fock build (bqc_jk_fp64_noalloc).

It serves callers that cannot allocate device memory when they need a Fock
build (a framework that already owns the GPU's memory pool, or a loop that
cannot afford cudaMalloc's device-wide synchronisation); its scratch is a
fixed array inside the library.  Checked here through the C ABI against the
regular entry point (bqc_jk, FP64) at the FP64 tolerance of the other J/K
tests, on two calls in a row, since every call reuses the same array.
This file sorts last so that a run stopping at the first failure has run
every other test before it.
"""
import ctypes

import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu


def test_noalloc_matches_bqc_jk(gpu_ctx):
    import torch
    import paper_2502_17963_gb300 as bqc
    L = bqc.lib()
    for name in ("h2o", "w3"):
        mol = workload.molecule_for(name)
        basis = bqc.Basis(gpu_ctx, mol)
        df = bqc.DF(gpu_ctx, basis, keep_fp32=False)
        B = df.copy(0)
        n, naux, no = basis.nbf, basis.naux, basis.nocc
        stream = torch.cuda.current_stream().cuda_stream
        rng = np.random.default_rng(17)
        for call in range(2):  # two calls in a row share the scratch array
            C = torch.tensor(rng.standard_normal((n, no)) * 0.3, device="cuda")
            J0, K0 = df.jk(C, bqc.PREC_FP64)
            J = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
            K = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
            st = L.bqc_jk_fp64_noalloc(B.data_ptr(), naux, n, C.data_ptr(), no, J.data_ptr(),
                                       K.data_ptr(), stream)
            assert st == 0, L.bqc_last_error()
            torch.cuda.synchronize()
            assert (J - J0).abs().max().item() < 1e-10, (name, call)
            assert (K - K0).abs().max().item() < 1e-10, (name, call)


def test_noalloc_matches_oracle_w3(gpu_ctx):
    """The same entry point against the oracle directly ((H2O)_3, the
    oracle's own B, J = sum_P w_P B_P and K = sum_P X_P X_P^T), two calls in
    a row, at the 1e-10 bar of the FP64 J/K tests."""
    import torch
    import oracle
    import paper_2502_17963_gb300 as bqc
    L = bqc.lib()
    mol = workload.molecule_for("w3")
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=False)
    B = df.copy(0)
    n, naux, no = basis.nbf, basis.naux, basis.nocc
    I = oracle.system_integrals(mol)
    Bo, _ = oracle.df_tensor(I["aux"], I["orb"])
    rng = np.random.default_rng(23)
    for call in range(2):
        C = rng.standard_normal((n, no)) * 0.3
        Cg = torch.tensor(C, device="cuda")
        J = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        K = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        st = L.bqc_jk_fp64_noalloc(B.data_ptr(), naux, n, Cg.data_ptr(), no, J.data_ptr(),
                                   K.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert st == 0, L.bqc_last_error()
        torch.cuda.synchronize()
        Jo, Ko = oracle.jk_df(Bo, C)
        assert np.abs(J.cpu().numpy() - Jo).max() < 1e-10, call
        assert np.abs(K.cpu().numpy() - Ko).max() < 1e-10, call


def test_noalloc_rejects_oversized(gpu_ctx):
    import paper_2502_17963_gb300 as bqc
    L = bqc.lib()
    # (H2O)_8 needs 600*200*40 doubles of scratch, beyond the 32 MiB array;
    # the size check runs before any pointer is touched
    dummy = ctypes.c_void_p(1)
    st = L.bqc_jk_fp64_noalloc(dummy, 600, 200, dummy, 40, dummy, dummy, None)
    assert st == -1
    assert b"limit" in L.bqc_last_error()
