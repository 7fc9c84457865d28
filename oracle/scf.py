"""Oracle DF-RHF: density-fitting tensor, J/K, and the closed-shell SCF.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper (Sec. 2.2) builds the mean field from Cholesky-decomposed ERIs:
with the Coulomb metric V = (P|Q) = L L^T, B_P,mu nu = sum_Q (L^{-1})_PQ (Q|mu nu)
so that (mu nu|lambda sigma) ~ sum_P B_P,mu nu B_P,lambda sigma.  With
D = C_occ C_occ^T (no factor 2), J = sum_P B_P (B_P : D) and
K = sum_P B_P D B_P; F = H + 2J - K; E = sum D (H + F) + E_nn
(Szabo & Ostlund, Eq. 3.154 and 3.184 with P = 2D).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional, Tuple

import numpy as np
import scipy.linalg as sla

from .ints import OracleBasis, int2c, int3c, nuclear_repulsion, one_electron


def system_integrals(mol) -> dict:
    """One-electron matrices and nuclear repulsion of a workload.Molecule."""
    orb = OracleBasis(mol.orb, mol.xyz)
    aux = OracleBasis(mol.aux, mol.xyz)
    S = one_electron("S", orb)
    T = one_electron("T", orb)
    V = one_electron("V", orb, mol.Z, mol.xyz)
    return dict(orb=orb, aux=aux, S=S, T=T, Vne=V, H=T + V,
                enuc=nuclear_repulsion(mol.Z, mol.xyz), nocc=mol.nocc)


def raw_3c(aux: OracleBasis, orb: OracleBasis) -> np.ndarray:
    """(P|mu nu) as (Naux, N, N): shell pairs a >= b computed, the rest mirrored."""
    pairs = [(a, b) for a in range(orb.nshell) for b in range(a + 1)]
    blk = int3c(aux, orb, pairs=pairs)
    N = orb.nfn
    out = np.zeros((aux.nfn, N, N))
    col = 0
    for a, b in pairs:
        na, nb = orb.ncart[a], orb.ncart[b]
        t = blk[:, col:col + na * nb].reshape(-1, na, nb)
        out[:, orb.off[a]:orb.off[a] + na, orb.off[b]:orb.off[b] + nb] = t
        out[:, orb.off[b]:orb.off[b] + nb, orb.off[a]:orb.off[a] + na] = t.transpose(0, 2, 1)
        col += na * nb
    return out


def df_tensor(aux: OracleBasis, orb: OracleBasis, metric=None) -> Tuple[np.ndarray, np.ndarray]:
    """B = L^{-1} (Q|mu nu) with V = L L^T (lower Cholesky factor, positive diagonal).

    Returns (B as (Naux, N, N), L).
    """
    V = int2c(aux) if metric is None else metric
    L = np.linalg.cholesky(V)
    raw = raw_3c(aux, orb)
    N = orb.nfn
    B = sla.solve_triangular(L, raw.reshape(aux.nfn, N * N), lower=True)
    return B.reshape(aux.nfn, N, N), L


def jk_df(B: np.ndarray, Cocc: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """J and K from B and C_occ through X_P = B_P C_occ (textbook DF contraction).

    w_P = sum_mu,i X_P,mu i C_mu i = B_P : D;  J = sum_P w_P B_P;
    K = sum_P X_P X_P^T.
    """
    X = np.einsum("pmn,ni->pmi", B, Cocc, optimize=True)
    w = np.einsum("pmi,mi->p", X, Cocc, optimize=True)
    J = np.einsum("p,pmn->mn", w, B, optimize=True)
    K = np.einsum("pmi,pni->mn", X, X, optimize=True)
    return J, K


def raw_3c_packed(aux: OracleBasis, orb: OracleBasis) -> np.ndarray:
    """(P|mu nu) on the packed lower triangle, (Naux, N(N+1)/2) with column
    mu(mu+1)/2 + nu for mu >= nu; computed one orbital shell a at a time (all
    its pairs (a, b <= a) against every aux shell), so the full square is
    never held."""
    N = orb.nfn
    out = np.zeros((aux.nfn, N * (N + 1) // 2))
    for a in range(orb.nshell):
        pairs = [(a, b) for b in range(a + 1)]
        blk = int3c(aux, orb, pairs=pairs)
        na = orb.ncart[a]
        col = 0
        for _, b in pairs:
            nb = orb.ncart[b]
            t = blk[:, col:col + na * nb].reshape(-1, na, nb)
            for i in range(na):
                mu = orb.off[a] + i
                for j in range(nb):
                    nu = orb.off[b] + j
                    if nu <= mu:
                        out[:, mu * (mu + 1) // 2 + nu] = t[:, i, j]
            col += na * nb
    return out


def df_tensor_packed(aux: OracleBasis, orb: OracleBasis, col_block: int = 32768):
    """B = L^{-1} (Q|mu nu) on the packed lower triangle (Naux, Npair), V = L L^T.

    The definition of df_tensor; B's column for one orbital pair depends only
    on that pair's column of (Q|mu nu), so the triangular solve runs over
    blocks of columns (the aux-blocked CPU form that large clusters need).
    Returns (B packed, L).
    """
    V = int2c(aux)
    L = np.linalg.cholesky(V)
    B = raw_3c_packed(aux, orb)
    for c0 in range(0, B.shape[1], col_block):
        c1 = min(B.shape[1], c0 + col_block)
        B[:, c0:c1] = sla.solve_triangular(L, B[:, c0:c1], lower=True)
    return B, L


def unpack_rows(Bp: np.ndarray, N: int) -> np.ndarray:
    """Packed lower triangles (rows, Npair) -> symmetric full squares (rows, N, N)."""
    out = np.zeros((Bp.shape[0], N, N))
    il = np.tril_indices(N)
    out[:, il[0], il[1]] = Bp
    out[:, il[1], il[0]] = Bp
    return out


def jk_df_packed(Bp: np.ndarray, N: int, Cocc: np.ndarray, block: int = 64, bounds=False):
    """jk_df over a packed B, summing the aux index P in blocks of `block`
    (J and K are sums over P of per-P terms).  With bounds=True also returns
    the absolute contractions JA = sum_P |w_P| |B_P| and
    KA = sum_P |X_P| (|B_P| |C|)^T + (|B_P| |C|) |X_P|^T, the scale of the
    rounding error of any evaluation order."""
    J = np.zeros((N, N))
    K = np.zeros((N, N))
    JA = np.zeros((N, N)) if bounds else None
    KA = np.zeros((N, N)) if bounds else None
    Ca = np.abs(Cocc)
    for P0 in range(0, Bp.shape[0], block):
        Bf = unpack_rows(Bp[P0:P0 + block], N)
        X = np.einsum("pmn,ni->pmi", Bf, Cocc, optimize=True)
        w = np.einsum("pmi,mi->p", X, Cocc, optimize=True)
        J += np.einsum("p,pmn->mn", w, Bf, optimize=True)
        K += np.einsum("pmi,pni->mn", X, X, optimize=True)
        if bounds:
            Ba = np.abs(Bf)
            XA = np.einsum("pmn,ni->pmi", Ba, Ca, optimize=True)
            JA += np.einsum("p,pmn->mn", np.abs(w), Ba, optimize=True)
            t = np.einsum("pmi,pni->mn", np.abs(X), XA, optimize=True)
            KA += t + t.T
    if bounds:
        return J, K, JA, KA
    return J, K


def jk_4c(eri: np.ndarray, Cocc: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """J_mn = sum (mn|ls) D_ls, K_mn = sum (ml|ns) D_ls with D = C_occ C_occ^T."""
    D = Cocc @ Cocc.T
    J = np.einsum("mnls,ls->mn", eri, D, optimize=True)
    K = np.einsum("mlns,ls->mn", eri, D, optimize=True)
    return J, K


@dataclass
class RhfResult:
    energy: float
    converged: bool
    iterations: int
    C: np.ndarray
    eps: np.ndarray
    Cocc: np.ndarray
    D: np.ndarray
    F: np.ndarray
    diis_err: float
    history: List[Tuple[float, float]] = field(default_factory=list)


def canonical_orthogonaliser(S: np.ndarray, thresh: float = 1e-8) -> np.ndarray:
    """X = U s^{-1/2} over eigenvalues of S above thresh (Szabo & Ostlund Eq. 3.169)."""
    s, U = np.linalg.eigh(S)
    keep = s > thresh
    return U[:, keep] / np.sqrt(s[keep])


def diis_coefficients(errs: List[np.ndarray]) -> np.ndarray:
    """Pulay (1982): minimise |sum c_i e_i| subject to sum c_i = 1."""
    m = len(errs)
    Bm = np.zeros((m + 1, m + 1))
    for i in range(m):
        for j in range(m):
            Bm[i, j] = float(np.sum(errs[i] * errs[j]))
    Bm[m, :m] = -1.0
    Bm[:m, m] = -1.0
    rhs = np.zeros(m + 1)
    rhs[m] = -1.0
    return np.linalg.solve(Bm, rhs)[:m]


def rhf(S: np.ndarray, H: np.ndarray, jk: Callable[[np.ndarray], Tuple[np.ndarray, np.ndarray]],
        nocc: int, enuc: float, tol: float = 1e-8, etol: float = 1e-10, max_iter: int = 100,
        diis_space: int = 8, orth_thresh: float = 1e-8) -> RhfResult:
    """Closed-shell SCF: canonical orthogonalisation, core guess, Pulay DIIS.

    Each iteration: J, K from the current C_occ; F = H + 2J - K;
    E = sum D (H + F) + E_nn; e = X^T (F D S - S D F) X; converged when
    max|e| < tol and |E - E_prev| < max(etol, eps * N * |E|) (the energy's own
    rounding noise, a sum over N^2 products); else DIIS over the last diis_space
    (F, e) pairs once two are stored, then diagonalise X^T F X.
    """
    X = canonical_orthogonaliser(S, orth_thresh)

    def diag(F):
        eps, Cp = np.linalg.eigh(X.T @ F @ X)
        C = X @ Cp
        return eps, C

    eps, C = diag(H)
    Cocc = C[:, :nocc]
    Fs: List[np.ndarray] = []
    Es: List[np.ndarray] = []
    E_prev: Optional[float] = None
    hist: List[Tuple[float, float]] = []
    converged = False
    F = H
    emax = np.inf
    E = 0.0
    it = 0
    for it in range(1, max_iter + 1):
        J, K = jk(Cocc)
        F = H + 2.0 * J - K
        D = Cocc @ Cocc.T
        E = float(np.sum(D * (H + F)) + enuc)
        err = X.T @ (F @ D @ S - S @ D @ F) @ X
        emax = float(np.max(np.abs(err)))
        hist.append((E, emax))
        enoise = np.finfo(np.float64).eps * S.shape[0] * abs(E)
        if emax < tol and E_prev is not None and abs(E - E_prev) < max(etol, enoise):
            converged = True
            break
        E_prev = E
        Fs.append(F)
        Es.append(err)
        if len(Fs) > diis_space:
            Fs.pop(0)
            Es.pop(0)
        Fx = F
        if len(Fs) >= 2:
            c = diis_coefficients(Es)
            Fx = sum(ci * Fi for ci, Fi in zip(c, Fs))
        eps, C = diag(Fx)
        Cocc = C[:, :nocc]
    D = Cocc @ Cocc.T
    return RhfResult(E, converged, it, C, eps, Cocc, D, F, emax, hist)
