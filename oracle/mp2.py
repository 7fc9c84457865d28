"""Oracle closed-shell MP2 (second-order Moller-Plesset) correlation energy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's DF-MP2 (Sec. 2.3) reuses the three-index tensor of the mean-field
stage: in the basis of canonical SCF orbitals,
    B_P,ia = sum_{mu,nu} C_mu,i B_P,mu nu C_nu,a          (i occupied, a virtual)
    (ia|jb) = sum_P B_P,ia B_P,jb
and the closed-shell second-order energy in spatial orbitals (Szabo & Ostlund
Eq. 6.74, written in chemists' notation, (ia|jb) = <ij|ab>) is
    E2 = sum_{i,j,a,b} (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b).
"""
from __future__ import annotations

import numpy as np


def ovov_4c(eri: np.ndarray, C: np.ndarray, nocc: int) -> np.ndarray:
    """(ia|jb) from the full AO integrals (mu nu|lambda sigma): (nocc, nvir, nocc, nvir)."""
    Co, Cv = C[:, :nocc], C[:, nocc:]
    return np.einsum("mnls,mi,na,lj,sb->iajb", eri, Co, Cv, Co, Cv, optimize=True)


def b_mo(B: np.ndarray, C: np.ndarray, nocc: int) -> np.ndarray:
    """B_P,ia = C_occ^T B_P C_vir: (Naux, nocc, nvir)."""
    return np.einsum("pmn,mi,na->pia", B, C[:, :nocc], C[:, nocc:], optimize=True)


def ovov_df(B: np.ndarray, C: np.ndarray, nocc: int) -> np.ndarray:
    """(ia|jb) = sum_P B_P,ia B_P,jb (density-fitted): (nocc, nvir, nocc, nvir)."""
    Bia = b_mo(B, C, nocc)
    return np.einsum("pia,pjb->iajb", Bia, Bia, optimize=True)


def mp2_energy(ovov: np.ndarray, eps: np.ndarray, nocc: int) -> float:
    """Closed-shell E2 from (ia|jb) and the canonical orbital energies."""
    eo, ev = eps[:nocc], eps[nocc:]
    den = eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] \
        - ev[None, None, None, :]
    exch = ovov.transpose(0, 3, 2, 1)  # (ib|ja) at index (i, a, j, b)
    return float(np.sum(ovov * (2.0 * ovov - exch) / den))


def mp2_energy_spin_orbital(ovov: np.ndarray, eps: np.ndarray, nocc: int) -> float:
    """The same energy from the spin-orbital form (Szabo & Ostlund Eq. 6.72):
    E2 = 1/4 sum_{IJAB} |<IJ||AB>|^2 / (e_I + e_J - e_A - e_B) over spin
    orbitals, with <IJ|AB> = (ia|jb) when I, A and J, B share spins and
    <IJ||AB> = <IJ|AB> - <IJ|BA>.  A separate route to E2 (no closed-shell
    spin summation), used to pin mp2_energy."""
    nv = ovov.shape[1]
    so, sv = 2 * nocc, 2 * nv
    g = np.zeros((so, so, sv, sv))
    for si in range(2):
        for sj in range(2):
            # spin orbital 2p + s: spatial p, spin s
            g[si::2, sj::2, si::2, sj::2] = ovov.transpose(0, 2, 1, 3)
    anti = g - g.transpose(0, 1, 3, 2)
    eo = np.repeat(eps[:nocc], 2)
    ev = np.repeat(eps[nocc:], 2)
    den = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] \
        - ev[None, None, None, :]
    return float(0.25 * np.sum(anti ** 2 / den))
