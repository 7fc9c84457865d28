"""Edge and degenerate cases of the C ABI on the GPU, against the oracle.

  * a single atom with s functions only (He, DF exact: the auxiliary set spans
    every orbital product) - the smallest shell classes, one tile, ragged
    everywhere; energy equals the oracle's 4-centre RHF;
  * contracted shells (H2 in STO-3G, three primitives per shell, with an
    even-tempered s/p auxiliary basis): the textbook H2 case through the GPU
    path, DF-RHF energy equal to the oracle's;
  * two waters 60 bohr apart: the shell pairs across the gap screened out,
    energy still the oracle's, and the same interaction energy;
  * invalid input: odd electron count, orbital f shell, no shells, bad
    primitive count, wrong nocc: the documented status, no device work.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workload
from workload import Molecule, Shell

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(__file__)


@pytest.fixture(scope="module")
def bqc():
    import paper_2502_17963_gb300 as m
    return m


def _oracle_df_energy(mol):
    I = oracle.system_integrals(mol)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    return oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), mol.nocc, I["enuc"])


def test_single_atom_s_only(gpu_ctx, bqc):
    exps = [0.3 * 3.0 ** k for k in range(4)]
    aux = sorted({a + b for a in exps for b in exps})
    mol = Molecule(np.array([2], dtype=np.int32), np.zeros((1, 3)),
                   [Shell(0, 0, [e], [1.0]) for e in exps],
                   [Shell(0, 0, [e], [1.0]) for e in aux], "He")
    basis = bqc.Basis(gpu_ctx, mol)
    assert (basis.nbf, basis.naux, basis.nocc) == (4, len(aux), 1)
    for prec in (bqc.PREC_FP64, bqc.PREC_MIXED_TF32X3):
        df = bqc.DF(gpu_ctx, basis, keep_fp32=True)
        r = bqc.scf_run(gpu_ctx, df, prec=prec)
        I = oracle.system_integrals(mol)
        eri = oracle.int4c(I["orb"])
        r4 = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_4c(eri, C), 1, 0.0)
        assert r["converged"]
        assert abs(r["energy"] - r4.energy) < 1e-8, (prec, r["energy"], r4.energy)
        df.close()


def test_contracted_h2_sto3g(gpu_ctx, bqc):
    g = json.load(open(os.path.join(HERE, "golden", "h2_sto3g.json")))
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, g["R_bohr"]]])
    orb = [Shell(i, 0, g["sto3g_exponents"], g["sto3g_coefficients"]) for i in range(2)]
    aux = [Shell(i, l, [0.2 * 3.0 ** k], [1.0]) for i in range(2) for l in (0, 1)
           for k in range(4)]
    mol = Molecule(np.array([1, 1], dtype=np.int32), xyz, orb, aux, "H2")
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=False)
    r = bqc.scf_run(gpu_ctx, df)
    ro = _oracle_df_energy(mol)
    assert r["converged"]
    assert abs(r["energy"] - ro.energy) < 1e-8
    # and it reproduces the textbook 4-centre value to its printed digits
    # (the fitting error of this auxiliary set is 2.4e-5 Eh in the oracle)
    assert abs(r["energy"] - g["E_total"]) < g["tolerance"]


def test_far_apart_dimer_screened(gpu_ctx, bqc):
    w = workload.single_water()
    shift = np.array([60.0, 0.0, 0.0])
    n1 = len(w.Z)
    mol = Molecule(np.concatenate([w.Z, w.Z]), np.vstack([w.xyz, w.xyz + shift]),
                   w.orb + [Shell(s.atom + n1, s.l, s.exps, s.coefs) for s in w.orb],
                   w.aux + [Shell(s.atom + n1, s.l, s.exps, s.coefs) for s in w.aux], "far")
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, schwarz=1e-12, keep_fp32=False)
    cand, kept = df.screening()
    assert kept < 0.7 * cand  # pairs across the gap are screened out
    r = bqc.scf_run(gpu_ctx, df)
    ro = _oracle_df_energy(mol)
    assert r["converged"] and abs(r["energy"] - ro.energy) < 1e-8
    bm = bqc.Basis(gpu_ctx, w)
    rm = bqc.scf_run(gpu_ctx, bqc.DF(gpu_ctx, bm, keep_fp32=False))
    # the interaction left at 60 bohr is the dipole-dipole tail (5.7e-6 Eh in
    # the oracle); the GPU gets the same number
    e_int = r["energy"] - 2 * rm["energy"]
    e_int_o = ro.energy - 2 * _oracle_df_energy(w).energy
    assert abs(e_int - e_int_o) < 3e-8, (e_int, e_int_o)


def _status(bqc, mol, gpu_ctx):
    with pytest.raises(bqc.BqcError) as e:
        bqc.Basis(gpu_ctx, mol)
    return e.value.status


def test_invalid_inputs(gpu_ctx, bqc):
    import torch
    w = workload.single_water()
    # odd electron count (one H removed)
    keep = [s for s in w.orb if s.atom != 2]
    keepa = [s for s in w.aux if s.atom != 2]
    oh = Molecule(w.Z[:2].copy(), w.xyz[:2].copy(), keep, keepa, "OH")
    assert _status(bqc, oh, gpu_ctx) == -1
    # an f shell in the orbital basis
    f = Molecule(w.Z, w.xyz, w.orb + [Shell(0, 3, [0.5], [1.0])], w.aux, "f")
    assert _status(bqc, f, gpu_ctx) == -9
    # no auxiliary shells
    na = Molecule(w.Z, w.xyz, w.orb, [], "noaux")
    assert _status(bqc, na, gpu_ctx) == -1
    # a shell without primitives
    np0 = Molecule(w.Z, w.xyz, w.orb + [Shell(0, 0, [], [])], w.aux, "np0")
    assert _status(bqc, np0, gpu_ctx) == -1
    # the context still works, and a wrong nocc is rejected by bqc_jk
    basis = bqc.Basis(gpu_ctx, w)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=False)
    with pytest.raises(bqc.BqcError) as e:
        df.jk(torch.zeros((basis.nbf, basis.nocc - 1), dtype=torch.float64, device="cuda"))
    assert e.value.status == -1
    r = bqc.scf_run(gpu_ctx, df)
    assert r["converged"]


def test_nonfinite_host_orbitals_rejected(gpu_ctx, bqc):
    """Failure detection on the host: a NaN or an infinity in C_occ handed to
    the end-to-end entry point is refused before any copy or launch, with the
    offending index named, and the handle keeps working."""
    w = workload.single_water()
    basis = bqc.Basis(gpu_ctx, w)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=True)
    rng = np.random.default_rng(3)
    C = rng.standard_normal((basis.nbf, basis.nocc)) * 0.2
    J0, K0 = df.jk_host(C, bqc.PREC_FP64)
    for bad in (np.nan, np.inf, -np.inf):
        Cb = C.copy()
        Cb[7, 2] = bad
        J = np.full((basis.nbf, basis.nbf), 123.0)
        with pytest.raises(bqc.BqcError) as e:
            df.jk_host(Cb, bqc.PREC_MIXED_TF32X3, J, J.copy())
        assert e.value.status == -1
        assert f"C_occ[{7 * basis.nocc + 2}]" in str(e.value)
        assert (J == 123.0).all()  # nothing was written back
    J1, K1 = df.jk_host(C, bqc.PREC_FP64)
    assert np.array_equal(J0, J1) and np.array_equal(K0, K1)


def test_bounded_device_wait_reports_flag(gpu_ctx, bqc):
    """Failure detection on the device without a fault: a wait on a barrier
    that nothing completes gives up after its clock limit (2e6 cycles, about
    a millisecond), the kernel returns, the call reports BQC_E_DEVICE_FLAG,
    and the context stays usable (a Fock build afterwards matches the oracle)."""
    import torch
    L = bqc.lib()
    st = L.bqc_wait_selftest(gpu_ctx.h, 2_000_000, None)
    assert st == -7, L.bqc_last_error()
    assert b"code 99" in L.bqc_last_error()
    assert L.bqc_wait_selftest(gpu_ctx.h, 0, None) == -1
    w = workload.single_water()
    basis = bqc.Basis(gpu_ctx, w)
    df = bqc.DF(gpu_ctx, basis, keep_fp32=False)
    rng = np.random.default_rng(11)
    C = rng.standard_normal((basis.nbf, basis.nocc)) * 0.2
    J, K = df.jk(torch.tensor(C, device="cuda"), bqc.PREC_FP64)
    I = oracle.system_integrals(w)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    Jr, Kr = oracle.jk_df(B, C)
    assert np.abs(J.cpu().numpy() - Jr).max() < 1e-10
    assert np.abs(K.cpu().numpy() - Kr).max() < 1e-10
