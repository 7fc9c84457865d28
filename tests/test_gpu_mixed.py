"""Mixed-precision (TF32 tcgen05) Fock build.

Two checks per molecule:
  * kernel exactness: against an FP64 evaluation of the same TF32-rounded
    operands (B and C rounded to nearest TF32, X rounded to TF32 before the
    SYRK), which removes the precision choice and leaves only FP32
    accumulation order, so indexing or pipeline mistakes show as O(1) errors;
  * method error: against the plain FP64 oracle J and K, bounded by the
    TF32 input rounding (unit roundoff 2^-11).
Sizes span several 128-row tiles with ragged tails (N = 75, 125, 200, 400).
"""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


def tf32(x):
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def bqc():
    import paper_2502_17963_gb300 as m
    return m


@pytest.mark.parametrize("name", ["w3", "w5", "w8", "w16"])
def test_jk_mixed(gpu_ctx, bqc, name):
    import torch
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, schwarz=0.0, keep_fp32=True)
    N, no = basis.nbf, basis.nocc
    Bp = df.copy(0).cpu().numpy()                     # GPU FP64 B (checked elsewhere)
    r, c = np.tril_indices(N)
    B = np.zeros((basis.naux, N, N))
    B[:, r, c] = Bp
    B[:, c, r] = Bp
    rng = np.random.default_rng(9)
    C = rng.standard_normal((N, no)) * 0.3
    J, K = df.jk(torch.tensor(C, device="cuda"), bqc.PREC_MIXED_TF32)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    # emulated-rounding reference
    Bt, Ct = tf32(B), tf32(C)
    X = np.einsum("pmn,ni->pmi", Bt, Ct, optimize=True)
    w = np.einsum("pmi,mi->p", X, C.astype(np.float32).astype(np.float64), optimize=True)
    Xr = tf32(X)
    Ke = np.einsum("pmi,pni->mn", Xr, Xr, optimize=True)
    Je = np.einsum("p,pmn->mn", w, Bt, optimize=True)
    assert np.abs(K - K.T).max() == 0.0 and np.abs(J - J.T).max() == 0.0
    assert np.abs(K - Ke).max() < 2e-5 * np.abs(Ke).max(), np.abs(K - Ke).max()
    assert np.abs(J - Je).max() < 2e-6 * np.abs(Je).max(), np.abs(J - Je).max()
    # method error against FP64
    J64, K64 = df.jk(torch.tensor(C, device="cuda"), bqc.PREC_FP64)
    J64, K64 = J64.cpu().numpy(), K64.cpu().numpy()
    assert np.abs(K - K64).max() < 3e-3 * np.abs(K64).max()
    assert np.abs(J - J64).max() < 3e-3 * np.abs(J64).max()
