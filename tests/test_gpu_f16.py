"""Mixed-precision Fock build with split FP16 operands (MIXED_F16X3).

B, C_occ and X are scaled by powers of two (largest magnitude at most 2^14)
and split into FP16 hi + lo parts; K and the B.D products take three
products per term (hi*hi + hi*lo + lo*hi) on kind::f16 tensor cores with FP32
accumulation.  Checks, as for the TF32 split (test_gpu_mixed.py):
  * kernel exactness against an FP64 evaluation of the same split operands
    (the scales recomputed here from max|B| and max|C| by the documented
    rule; the split of X before the SYRK is inside the bound), elementwise
    within 2^-14 of the absolute contractions KA, JA;
  * method error against the plain FP64 build at the same orbitals;
  * the staged SCF (F16X3 first stage, FP64 second) against the oracle's
    energy to 1e-8 Eh.
Sizes span several 128-row tiles with ragged tails (N = 75 .. 400).
"""
import math

import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


def pow2_scale(maxabs):
    """2^(14 - e) with maxabs <= 2^e (maxabs taken in FP32, as on the device)."""
    m = float(np.float32(maxabs))
    if m <= 0.0:
        return 2.0 ** 14
    mt, e = math.frexp(m)
    if mt == 0.5:
        e -= 1
    return 2.0 ** (14 - e)


def split16(x, scale):
    """(hi, lo) FP16 parts of fp32(x * scale), each rounded to nearest."""
    f = np.asarray(np.asarray(x, dtype=np.float64) * scale, dtype=np.float32)
    h = f.astype(np.float16)
    lo = (f - h.astype(np.float32)).astype(np.float16)
    return h.astype(np.float64), lo.astype(np.float64)


@pytest.fixture(scope="module")
def bqc():
    import paper_2502_17963_gb300 as m
    return m


@pytest.mark.parametrize("name", ["w3", "w5", "w8", "w16"])
def test_jk_f16x3(gpu_ctx, bqc, name):
    import torch
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, schwarz=0.0, keep_fp32=bqc.SHADOW_F16)
    N = basis.nbf
    Bp = df.copy(0).cpu().numpy()
    r, c = np.tril_indices(N)
    B = np.zeros((basis.naux, N, N))
    B[:, r, c] = Bp
    B[:, c, r] = Bp
    I = oracle.system_integrals(mol)
    Bo, _ = oracle.df_tensor(I["aux"], I["orb"])
    ro = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(Bo, C), mol.nocc, I["enuc"], max_iter=2)
    C = ro.Cocc
    J, K = df.jk(torch.tensor(C, device="cuda"), bqc.PREC_MIXED_F16X3)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    sB, sC = pow2_scale(np.abs(B).max()), pow2_scale(np.abs(C).max())
    Bh, Bl = split16(B, sB)
    Ch, Cl = split16(C, sC)
    X = (np.einsum("pmn,ni->pmi", Bh, Ch + Cl, optimize=True) +
         np.einsum("pmn,ni->pmi", Bl, Ch, optimize=True)) / (sB * sC)
    Cf = C.astype(np.float32).astype(np.float64)
    Ke = np.einsum("pmi,pni->mn", X, X, optimize=True)
    w = np.einsum("pmi,mi->p", X, Cf, optimize=True)
    Je = np.einsum("p,pmn->mn", w, B, optimize=True)   # the J pass reads the FP64 B
    XA = np.einsum("pmn,ni->pmi", np.abs(B), np.abs(C), optimize=True)
    KA = np.einsum("pmi,pni->mn", np.abs(X), XA, optimize=True)
    KA = KA + KA.T
    wa = np.einsum("pmi,mi->p", XA, np.abs(Cf), optimize=True)
    JA = np.einsum("p,pmn->mn", wa, np.abs(B), optimize=True)
    assert np.abs(K - K.T).max() == 0.0 and np.abs(J - J.T).max() == 0.0
    mk, mj = KA > 1e-30, JA > 1e-30
    rk = (np.abs(K - Ke)[mk] / KA[mk]).max()
    rj = (np.abs(J - Je)[mj] / JA[mj]).max()
    J64, K64 = df.jk(torch.tensor(C, device="cuda"), bqc.PREC_FP64)
    J64, K64 = J64.cpu().numpy(), K64.cpu().numpy()
    dF = np.abs(2 * (J - J64) - (K - K64)).max()
    print(f"{name} F16X3: K ratio {rk:.3e}  J ratio {rj:.3e}  max|dF| vs FP64 {dF:.3e}  "
          f"scales sB=2^{math.log2(sB):.0f} sC=2^{math.log2(sC):.0f}")
    assert rk < 2.0 ** -14, rk
    assert rj < 2.0 ** -14, rj
    assert dF < 1e-4


def test_f16x3_needs_f16_shadows(gpu_ctx, bqc):
    """F16X3 on a handle with TF32 shadows (and the reverse) is refused with
    BQC_E_INVALID; direct mode refuses F16X3 with BQC_E_UNSUPPORTED."""
    import torch
    mol = workload.single_water()
    basis = bqc.Basis(gpu_ctx, mol)
    C = torch.zeros((basis.nbf, basis.nocc), dtype=torch.float64, device="cuda")
    df = bqc.DF(gpu_ctx, basis, keep_fp32=True)
    with pytest.raises(bqc.BqcError) as e:
        df.jk(C, bqc.PREC_MIXED_F16X3)
    assert e.value.status == -1
    d16 = bqc.DF(gpu_ctx, basis, keep_fp32=bqc.SHADOW_F16)
    with pytest.raises(bqc.BqcError) as e:
        d16.jk(C, bqc.PREC_MIXED_TF32X3)
    assert e.value.status == -1
    dd = bqc.DF(gpu_ctx, basis, mode=bqc.DF_DIRECT, keep_fp32=True)
    with pytest.raises(bqc.BqcError) as e:
        dd.jk(C, bqc.PREC_MIXED_F16X3)
    assert e.value.status == -9
    # a zero C_occ is a valid input: J = K = 0 exactly (the scales fall back to 2^14)
    J, K = d16.jk(C, bqc.PREC_MIXED_F16X3)
    assert J.abs().max().item() == 0.0 and K.abs().max().item() == 0.0


@pytest.mark.parametrize("name", ["w4", "w8"])
def test_staged_scf_energy_f16x3(gpu_ctx, bqc, name):
    """F16X3 first stage, FP64 second stage: the oracle's energy to 1e-8 Eh."""
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=bqc.SHADOW_F16)
    r = bqc.scf_run(gpu_ctx, df, prec=bqc.PREC_MIXED_F16X3)
    I = oracle.system_integrals(mol)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    ro = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), mol.nocc, I["enuc"])
    print(name, {k: v for k, v in r.items() if k != "history"})
    assert r["converged"] and r["iterations_mixed"] > 0
    assert abs(r["energy"] - ro.energy) < 1e-8
    h, m = r["history"], r["iterations_mixed"]
    assert all(p == bqc.PREC_MIXED_F16X3 for p, _, _ in h[:m])
    assert all(p == bqc.PREC_FP64 for p, _, _ in h[m:])


@pytest.mark.parametrize("name", ["w4", "w8"])
@pytest.mark.parametrize("prec", [2, 3])
def test_staged_scf_incremental(gpu_ctx, bqc, name, prec):
    """Anchored incremental FP64 stage: the FP64-stage Fock matrices are
    F_(k-1) plus mixed-precision J and K of the density change (factored
    into its positive and negative parts), with full FP64 anchors; the run
    converges on a full FP64 build, to the oracle's energy within 1e-8 Eh,
    with fewer full FP64 builds than the plain staged SCF."""
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=bqc.SHADOW_F16 if prec == 3 else bqc.SHADOW_TF32)
    r = bqc.scf_run(gpu_ctx, df, prec=prec, incremental=True)
    rp = bqc.scf_run(gpu_ctx, df, prec=prec)
    I = oracle.system_integrals(mol)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    ro = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), mol.nocc, I["enuc"])
    print(name, prec, "incremental:", r["builds"], r["iterations"], "plain staged:", rp["builds"],
          f"dE {r['energy'] - ro.energy:.2e}")
    assert r["converged"] and abs(r["energy"] - ro.energy) < 1e-8
    h = r["history"]
    assert h[-1][0] == bqc.PREC_FP64 and h[-1][1] == r["diis_err"] < 1e-8
    assert r["builds"]["incremental"] == sum(1 for p, _, _ in h if p == -1) > 0
    assert r["builds"]["fp64"] == sum(1 for p, _, _ in h if p == bqc.PREC_FP64)
    assert r["builds"]["fp64"] <= rp["builds"]["fp64"]
