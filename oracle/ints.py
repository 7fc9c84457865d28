"""ctypes wrapper over the oracle's McMurchie-Davidson integrals (md_ints.c).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from . import _build

_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        d, i = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        _lib.orc_boys.argtypes = [ctypes.c_int, ctypes.c_double, d]
        _lib.orc_one_electron.argtypes = [ctypes.c_int, ctypes.c_int, i, i, i, d, d, d,
                                          ctypes.c_int, i, d, d]
        _lib.orc_int2c.argtypes = [ctypes.c_int, i, i, i, d, d, d, d]
        _lib.orc_int3c.argtypes = ([ctypes.c_int, i, i, i, d, d, d] * 2
                                   + [ctypes.c_int, i, ctypes.c_int, i, i, d])
        _lib.orc_int4c.argtypes = [ctypes.c_int, i, i, i, d, d, d, d]
        _lib.orc_nuclear_repulsion.argtypes = [ctypes.c_int, i, d]
        _lib.orc_nuclear_repulsion.restype = ctypes.c_double
    return _lib


def _p(a):
    if a.dtype == np.float64:
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class OracleBasis:
    """Flattened shells: l, nprim, primitive offsets, centres, exponents, coefs."""

    def __init__(self, shells: Sequence, xyz: np.ndarray):
        self.l = np.array([s.l for s in shells], dtype=np.int32)
        self.nprim = np.array([len(s.exps) for s in shells], dtype=np.int32)
        self.poff = np.concatenate([[0], np.cumsum(self.nprim)[:-1]]).astype(np.int32)
        self.xyz = np.ascontiguousarray(np.array([xyz[s.atom] for s in shells],
                                                 dtype=np.float64).reshape(-1, 3))
        self.exps = np.array([e for s in shells for e in s.exps], dtype=np.float64)
        self.coefs = np.array([c for s in shells for c in s.coefs], dtype=np.float64)
        self.ncart = (self.l + 1) * (self.l + 2) // 2
        self.off = np.concatenate([[0], np.cumsum(self.ncart)]).astype(np.int64)
        self.nfn = int(self.off[-1])
        self.nshell = len(shells)

    def args(self):
        return (self.nshell, _p(self.l), _p(self.nprim), _p(self.poff), _p(self.xyz),
                _p(self.exps), _p(self.coefs))


def boys(mmax: int, T: float) -> np.ndarray:
    """F_m(T), m = 0..mmax (HJO Sec. 9.8)."""
    out = np.zeros(mmax + 1)
    _L().orc_boys(mmax, float(T), _p(out))
    return out


def one_electron(kind: str, basis: OracleBasis, Z=None, xyz=None) -> np.ndarray:
    """'S' overlap, 'T' kinetic, 'V' nuclear attraction (HJO Sec. 9.3, 9.9)."""
    which = {"S": 0, "T": 1, "V": 2}[kind]
    N = basis.nfn
    out = np.zeros((N, N))
    if Z is None:
        Zc = np.zeros(1, dtype=np.int32)
        C = np.zeros(3)
        nat = 0
    else:
        Zc = np.ascontiguousarray(Z, dtype=np.int32)
        C = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
        nat = len(Zc)
    _L().orc_one_electron(which, *basis.args(), nat, _p(Zc), _p(C), _p(out))
    return out


def int2c(aux: OracleBasis) -> np.ndarray:
    """Coulomb metric V_PQ = (P|Q)."""
    out = np.zeros((aux.nfn, aux.nfn))
    _L().orc_int2c(*aux.args(), _p(out))
    return out


def int3c(aux: OracleBasis, orb: OracleBasis, pshells=None, pairs=None) -> np.ndarray:
    """(P|mu nu).  Default: all aux shells, full square -> array (Naux, N, N).

    With ``pshells`` (aux shell indices) and ``pairs`` (list of orbital shell
    index pairs (a, b)) returns a (sum of aux components, sum of na*nb) matrix
    in the order given, each pair block laid out a-major.
    """
    full = pairs is None
    ps = np.arange(aux.nshell, dtype=np.int32) if pshells is None else \
        np.ascontiguousarray(pshells, dtype=np.int32)
    if full:
        a = np.repeat(np.arange(orb.nshell, dtype=np.int32), orb.nshell)
        b = np.tile(np.arange(orb.nshell, dtype=np.int32), orb.nshell)
    else:
        a = np.ascontiguousarray([p[0] for p in pairs], dtype=np.int32)
        b = np.ascontiguousarray([p[1] for p in pairs], dtype=np.int32)
    nrow = int(aux.ncart[ps].sum())
    ncol = int((orb.ncart[a] * orb.ncart[b]).sum())
    out = np.zeros((nrow, ncol))
    _L().orc_int3c(*aux.args(), *orb.args(), len(ps), _p(ps), len(a), _p(a), _p(b), _p(out))
    if not full:
        return out
    # scatter pair blocks into the full square
    N = orb.nfn
    res = np.zeros((nrow, N, N))
    col = 0
    for sa, sb in zip(a, b):
        na, nb = orb.ncart[sa], orb.ncart[sb]
        blk = out[:, col:col + na * nb].reshape(nrow, na, nb)
        res[:, orb.off[sa]:orb.off[sa] + na, orb.off[sb]:orb.off[sb] + nb] = blk
        col += na * nb
    return res


def int4c(orb: OracleBasis) -> np.ndarray:
    """Full (mu nu|lambda sigma), chemists' notation (HJO 9.9.33)."""
    N = orb.nfn
    out = np.zeros((N, N, N, N))
    _L().orc_int4c(*orb.args(), _p(out))
    return out


def nuclear_repulsion(Z, xyz) -> float:
    Zc = np.ascontiguousarray(Z, dtype=np.int32)
    C = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    return float(_L().orc_nuclear_repulsion(len(Zc), _p(Zc), _p(C)))
