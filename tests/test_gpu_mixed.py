"""Mixed-precision (TF32 tcgen05) Fock build.

Per molecule and precision two checks:
  * kernel exactness: against an FP64 evaluation of the same split operands
    (TF32X3: X = Bh Ch + Bh Cl + Bl Ch with hi/lo TF32 parts; TF32: X = Bh Ch).
    The J pass reads the FP64 B for TF32X3 (w from the split X either way).
    The remaining differences are the FP32
    accumulation of X (relative to XA = |B| |C|, which exceeds |X| by the
    cancellation in B C) and, for
    TF32, the rounding of X before the SYRK.  They are bounded elementwise by
    a constant times the absolute-value contractions
    KA = sum_{P,i} (|X| XA^T + XA |X|^T) for K and JA = sum_P |w|_P |B_P| for
    J (the standard form of a rounding-error bound), so a wrong index or a
    dropped block shows up as an O(1) violation;
  * method error: against the plain FP64 build with the same orbitals.
Sizes span several 128-row tiles with ragged tails (N = 75, 125, 200, 400).
"""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


def split(x):
    """FP32 value -> (hi, lo) TF32 parts, round to nearest (ties away)."""
    def rna(a):
        f = np.asarray(a, dtype=np.float32)
        b = f.view(np.uint32).astype(np.uint64)
        b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
        return b.view(np.float32)
    f = np.asarray(x, dtype=np.float32)
    h = rna(f)
    l = rna(f - h)
    return h.astype(np.float64), l.astype(np.float64)


@pytest.fixture(scope="module")
def bqc():
    import paper_2502_17963_gb300 as m
    return m


# ratio bounds: |K_gpu - K_ref| <= c * (|X||X|^T); measured ratios are printed
BOUND = {1: (2.0 ** -9, 2.0 ** -9), 2: (2.0 ** -14, 2.0 ** -14)}


@pytest.mark.parametrize("name", ["w3", "w5", "w8", "w16"])
@pytest.mark.parametrize("prec", [1, 2])
def test_jk_mixed(gpu_ctx, bqc, name, prec):
    import torch
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, schwarz=0.0, keep_fp32=True)
    N, no = basis.nbf, basis.nocc
    Bp = df.copy(0).cpu().numpy()                     # GPU FP64 B (pinned elsewhere)
    r, c = np.tril_indices(N)
    B = np.zeros((basis.naux, N, N))
    B[:, r, c] = Bp
    B[:, c, r] = Bp
    I = oracle.system_integrals(mol)
    Bo, _ = oracle.df_tensor(I["aux"], I["orb"])
    ro = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(Bo, C), mol.nocc, I["enuc"], max_iter=2)
    C = ro.Cocc                                       # physical orbitals (cancellation-prone)
    J, K = df.jk(torch.tensor(C, device="cuda"), prec)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    Bh, Bl = split(B)
    Ch, Cl = split(C)
    if prec == 2:
        X = np.einsum("pmn,ni->pmi", Bh, Ch + Cl, optimize=True) + \
            np.einsum("pmn,ni->pmi", Bl, Ch, optimize=True)
        Bs = Bh + Bl
    else:
        X = np.einsum("pmn,ni->pmi", Bh, Ch, optimize=True)
        Bs = Bh
    Cf = C.astype(np.float32).astype(np.float64)
    Ke = np.einsum("pmi,pni->mn", X, X, optimize=True)
    w = np.einsum("pmi,mi->p", X, Cf, optimize=True)
    # TF32X3's J pass reads the FP64 B, single-pass TF32's the TF32 shadow
    Je = np.einsum("p,pmn->mn", w, B if prec == 2 else Bs, optimize=True)
    Xa = np.abs(X)
    XA = np.einsum("pmn,ni->pmi", np.abs(B), np.abs(C), optimize=True)
    KA = np.einsum("pmi,pni->mn", Xa, XA, optimize=True)
    KA = KA + KA.T
    wa = np.einsum("pmi,mi->p", XA, np.abs(Cf), optimize=True)
    JA = np.einsum("p,pmn->mn", wa, np.abs(B), optimize=True)
    assert np.abs(K - K.T).max() == 0.0 and np.abs(J - J.T).max() == 0.0
    # entries whose scale underflows in FP32 (|B| ~ 1e-40) carry no information
    mk, mj = KA > 1e-30, JA > 1e-30
    rk = (np.abs(K - Ke)[mk] / KA[mk]).max()
    rj = (np.abs(J - Je)[mj] / JA[mj]).max()
    print(f"{name} prec={prec}: K ratio {rk:.3e}  J ratio {rj:.3e}")
    cK, cJ = BOUND[prec]
    assert rk < cK, rk
    assert rj < cJ, rj
    J64, K64 = df.jk(torch.tensor(C, device="cuda"), bqc.PREC_FP64)
    J64, K64 = J64.cpu().numpy(), K64.cpu().numpy()
    dF = np.abs(2 * (J - J64) - (K - K64)).max()
    print(f"{name} prec={prec}: max|dF| vs FP64 = {dF:.3e}")
    if prec == 2:
        assert dF < 1e-4


@pytest.mark.parametrize("name", ["w4", "w8"])
def test_staged_scf_energy(gpu_ctx, bqc, name):
    """Mixed first stage (TF32X3), FP64 second stage: same energy as the oracle."""
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=True)
    r = bqc.scf_run(gpu_ctx, df, prec=bqc.PREC_MIXED_TF32X3)
    I = oracle.system_integrals(mol)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    ro = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), mol.nocc, I["enuc"])
    print(name, {k: v for k, v in r.items() if k != "history"})
    assert r["converged"] and r["iterations_mixed"] > 0
    assert abs(r["energy"] - ro.energy) < 1e-8
    # one history entry per Fock build: the mixed ones (the last of them is
    # redone in FP64 at the switch), then FP64 to convergence
    h, m = r["history"], r["iterations_mixed"]
    assert len(h) == r["iterations"] + 1
    assert all(p == bqc.PREC_MIXED_TF32X3 for p, _, _ in h[:m])
    assert all(p == bqc.PREC_FP64 for p, _, _ in h[m:])
    assert h[-1][1] == r["diis_err"] < 1e-8 and h[-1][2] == r["energy"]
