"""Oracle: a plain, slow FP64 CPU reference of the density-fitted RHF method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2502_17963_gb300`` and never imports it.

What it computes (the paper names these techniques in Sec. 2.2 without
equations; the formulas are textbook, cited per function):
  * Gaussian integrals by McMurchie-Davidson (``md_ints.c``);
  * the density-fitting tensor B = L^{-1} (Q|mu nu) with V = L L^T, the
    Cholesky-decomposed ERIs (CD-ERIs) of Sec. 2.2;
  * J and K from B and the occupied orbitals, F = H + 2J - K;
  * the closed-shell SCF with canonical orthogonalisation, core guess and
    Pulay DIIS (Szabo & Ostlund, Sec. 3.4; Pulay 1982);
  * the closed-shell MP2 energy from (ia|jb), density-fitted or from the
    full AO integrals (Sec. 2.3 of the paper; Szabo & Ostlund Eq. 6.74).

Pins: see tests/test_oracle_*.py.  Parity of the cluster energies against the
GPU is pinned through these, not through a published number (the paper prints
none for this path).
"""
from .ints import OracleBasis, boys, one_electron, int2c, int3c, int4c, nuclear_repulsion  # noqa: F401
from .mp2 import b_mo, mp2_energy, mp2_energy_spin_orbital, ovov_4c, ovov_df  # noqa: F401
from .scf import (  # noqa: F401
    df_tensor,
    df_tensor_packed,
    jk_df,
    jk_df_packed,
    raw_3c_packed,
    unpack_rows,
    jk_4c,
    rhf,
    RhfResult,
    system_integrals,
)
