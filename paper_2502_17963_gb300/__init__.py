"""GB300-native density-fitted RHF Fock build (arXiv 2502.17963, Sec. 2.2).

A thin ctypes binding over ``libbqc.so`` (the C ABI declared in
``include/bqc.h``).  The functions named ``bqc_*`` mirror the C entry points
one to one; the small classes below only marshal arguments (molecule ->
shell arrays, torch tensors -> device pointers).  Every step of the method
runs in the library's CUDA kernels; there is no Python or CPU fallback: if
the shared library is missing or fails to load, importing the binding's
entry points raises.

PyTorch supplies device memory (through the caching allocator, passed to the
library as callbacks) and streams.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

from . import _build

BQC_OK = 0
BQC_E_INVALID = -1
BQC_E_NOT_CONVERGED = -4
BQC_E_NOT_READY = -8
BQC_E_UNSUPPORTED = -9
BQC_E_CANCELLED = -10
PREC_FP64 = 0
PREC_MIXED_TF32 = 1
PREC_MIXED_TF32X3 = 2
PREC_MIXED_F16X3 = 3
SHADOW_NONE, SHADOW_TF32, SHADOW_F16 = 0, 1, 2
COULOMB_FP64, COULOMB_FF = 0, 1
SERVE_BACKFILL, SERVE_FIFO = 0, 1
DF_STORED, DF_DIRECT, DF_AUTO, DF_NONE = 0, 1, 2, 3


class BqcError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().bqc_strerror(status).decode()
        detail = lib().bqc_last_error().decode()
        super().__init__(f"{where}: {msg} [{status}] {detail}")


class bqc_shell(ctypes.Structure):
    _fields_ = [("atom", ctypes.c_int), ("l", ctypes.c_int), ("nprim", ctypes.c_int),
                ("exps", ctypes.POINTER(ctypes.c_double)),
                ("coefs", ctypes.POINTER(ctypes.c_double))]


class bqc_df_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("schwarz", ctypes.c_double),
                ("aux_block", ctypes.c_int), ("keep_fp32", ctypes.c_int),
                ("hbm_limit", ctypes.c_size_t), ("aux_begin", ctypes.c_int),
                ("aux_end", ctypes.c_int)]


class bqc_scf_opts(ctypes.Structure):
    _fields_ = [("diis_tol", ctypes.c_double), ("energy_tol", ctypes.c_double),
                ("stage_tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("diis_space", ctypes.c_int), ("prec", ctypes.c_int),
                ("orth_thresh", ctypes.c_double), ("incremental", ctypes.c_int),
                ("guess_C", ctypes.c_void_p)]


class bqc_scf_result(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("e_nuc", ctypes.c_double),
                ("diis_err", ctypes.c_double), ("iterations", ctypes.c_int),
                ("converged", ctypes.c_int), ("iterations_mixed", ctypes.c_int),
                ("nmo", ctypes.c_int), ("C_dev", ctypes.c_void_p), ("eps_dev", ctypes.c_void_p),
                ("F_dev", ctypes.c_void_p), ("history", ctypes.POINTER(ctypes.c_double)),
                ("history_cap", ctypes.c_int), ("history_len", ctypes.c_int),
                ("switch_rule", ctypes.c_int), ("switch_err", ctypes.c_double),
                ("builds_fp64", ctypes.c_int), ("builds_mixed", ctypes.c_int),
                ("builds_incremental", ctypes.c_int)]


class bqc_serve_opts(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("hbm_budget", ctypes.c_size_t),
                ("prec", ctypes.c_int), ("scf", bqc_scf_opts), ("policy", ctypes.c_int),
                ("max_skips", ctypes.c_int), ("grouped", ctypes.c_int),
                ("group_window_us", ctypes.c_double)]


class bqc_request(ctypes.Structure):
    _fields_ = [("natom", ctypes.c_int), ("Z", ctypes.POINTER(ctypes.c_int)),
                ("xyz_bohr", ctypes.POINTER(ctypes.c_double)),
                ("orb", ctypes.POINTER(bqc_shell)), ("norb_shell", ctypes.c_int),
                ("aux", ctypes.POINTER(bqc_shell)), ("naux_shell", ctypes.c_int)]


class bqc_serve_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("energy", ctypes.c_double),
                ("diis_err", ctypes.c_double), ("iterations", ctypes.c_int),
                ("nbf", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("iterations_mixed", ctypes.c_int), ("priority", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
vp, ip, dp, i64p = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64

# C signatures: name -> (restype, argtypes)
_SIGS = {
    "bqc_strerror": (ctypes.c_char_p, [ip]),
    "bqc_last_error": (ctypes.c_char_p, []),
    "bqc_ctx_create": (ip, [ip, ctypes.c_size_t, ALLOC_FN, FREE_FN, vp, ctypes.POINTER(vp)]),
    "bqc_ctx_destroy": (ip, [vp]),
    "bqc_basis_load": (ip, [vp, ip, ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(bqc_shell), ip,
                            ctypes.POINTER(bqc_shell), ip, ctypes.POINTER(vp)]),
    "bqc_basis_destroy": (ip, [vp]),
    "bqc_basis_info": (ip, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)]),
    "bqc_basis_enuc": (ip, [vp, ctypes.POINTER(ctypes.c_double)]),
    "bqc_one_electron": (ip, [vp, vp, vp, vp, vp]),
    "bqc_boys": (ip, [vp, ip, vp, ip, vp, vp]),
    "bqc_int2c": (ip, [vp, vp, vp]),
    "bqc_int3c": (ip, [vp, dp, vp, vp]),
    "bqc_df_build": (ip, [vp, vp, ctypes.POINTER(bqc_df_opts), vp, ctypes.POINTER(vp)]),
    "bqc_df_destroy": (ip, [vp]),
    "bqc_df_info": (ip, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)]),
    "bqc_df_shard": (ip, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "bqc_df_screening": (ip, [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "bqc_df_copy": (ip, [vp, ip, vp, vp]),
    "bqc_int3c_screened": (ip, [vp, ip, ip, ip, vp, vp]),
    "bqc_jk": (ip, [vp, vp, ip, ip, vp, vp, vp]),
    "bqc_jk_host": (ip, [vp, vp, ip, ip, vp, vp, vp]),
    "bqc_jk_fp64_noalloc": (ip, [vp, ip, ip, vp, ip, vp, vp, vp]),
    "bqc_df_timing": (ip, [vp, ip]),
    "bqc_df_phase_ms": (ip, [vp, ctypes.POINTER(ctypes.c_float), ip]),
    "bqc_scf_run": (ip, [vp, vp, ctypes.POINTER(bqc_scf_opts), vp,
                         ctypes.POINTER(bqc_scf_result)]),
    "bqc_serve_create": (ip, [vp, ctypes.POINTER(bqc_serve_opts), ctypes.POINTER(vp)]),
    "bqc_serve_submit": (ip, [vp, ctypes.POINTER(bqc_request), ctypes.POINTER(ctypes.c_uint64)]),
    "bqc_serve_poll": (ip, [vp, ctypes.c_uint64, ctypes.POINTER(bqc_serve_result)]),
    "bqc_serve_drain": (ip, [vp, dp]),
    "bqc_serve_cancel": (ip, [vp, ctypes.c_uint64]),
    "bqc_serve_destroy": (ip, [vp]),
    "bqc_serve_footprint": (ctypes.c_size_t, [ip, ip, ip, ip]),
    "bqc_serve_group_stats": (ip, [vp, ctypes.POINTER(ctypes.c_uint64),
                                   ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int)]),
    "bqc_jk_grouped": (ip, [ip, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                            ctypes.POINTER(vp), vp]),
    "bqc_df_coulomb": (ip, [vp, vp, vp, ip, vp]),
    "bqc_wait_selftest": (ip, [vp, ctypes.c_longlong, vp]),
    "bqc_mp2": (ip, [vp, vp, vp, ip, ip, ctypes.POINTER(ctypes.c_double), vp]),
}


def exported_symbols():
    """Names of the C entry points this binding expects from libbqc.so."""
    return sorted(_SIGS)


def lib(path: Optional[str] = None):
    """Loads libbqc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    so = path or _build.LIB
    if not os.path.exists(so):
        raise ImportError(f"libbqc.so not found at {so}: run __graft_entry__.build() "
                          "(the CUDA library is required; there is no fallback)")
    L = ctypes.CDLL(so)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(status: int, where: str) -> int:
    if status not in (BQC_OK,):
        raise BqcError(status, where)
    return status


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def _ptr(t) -> int:
    return int(t.data_ptr())


class Context:
    """bqc_ctx with the torch caching allocator as device-memory provider."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, torch_allocator: bool = True):
        import torch
        self.device = device
        self._blocks = {}
        L = lib()
        if torch_allocator:
            def _alloc(nbytes, _ud):
                try:
                    with torch.cuda.device(device):
                        p = torch.cuda.caching_allocator_alloc(int(nbytes), device)
                    return p
                except Exception:
                    return None

            def _free(ptr, _ud):
                torch.cuda.caching_allocator_delete(ptr)

            self._afn, self._ffn = ALLOC_FN(_alloc), FREE_FN(_free)
        else:
            self._afn, self._ffn = ALLOC_FN(), FREE_FN()
        h = vp()
        check(L.bqc_ctx_create(device, hbm_budget, self._afn, self._ffn, None,
                               ctypes.byref(h)), "bqc_ctx_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().bqc_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _ShellArrays:
    """Keeps the ctypes arrays of a shell list alive."""

    def __init__(self, shells):
        self.keep = []
        arr = (bqc_shell * len(shells))()
        for i, s in enumerate(shells):
            e = (ctypes.c_double * len(s.exps))(*s.exps)
            c = (ctypes.c_double * len(s.coefs))(*s.coefs)
            self.keep += [e, c]
            arr[i] = bqc_shell(int(s.atom), int(s.l), len(s.exps),
                               ctypes.cast(e, ctypes.POINTER(ctypes.c_double)),
                               ctypes.cast(c, ctypes.POINTER(ctypes.c_double)))
        self.arr = arr
        self.n = len(shells)


def molecule_request(mol):
    """bqc_request (and the arrays it points to) for a workload.Molecule."""
    Z = (ctypes.c_int * len(mol.Z))(*[int(z) for z in mol.Z])
    xyz = (ctypes.c_double * (3 * len(mol.Z)))(*[float(v) for v in mol.xyz.reshape(-1)])
    orb, aux = _ShellArrays(mol.orb), _ShellArrays(mol.aux)
    req = bqc_request(len(mol.Z), Z, xyz, orb.arr, orb.n, aux.arr, aux.n)
    return req, (Z, xyz, orb, aux)


class Basis:
    """bqc_basis of a molecule (workload.Molecule or anything with Z, xyz, orb, aux)."""

    def __init__(self, ctx: Context, mol):
        self.ctx = ctx
        req, self._keep = molecule_request(mol)
        h = vp()
        check(lib().bqc_basis_load(ctx.h, req.natom, req.Z, req.xyz_bohr, req.orb,
                                   req.norb_shell, req.aux, req.naux_shell, ctypes.byref(h)),
              "bqc_basis_load")
        self.h = h
        n, na, no = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        npr = ctypes.c_int64()
        check(lib().bqc_basis_info(h, ctypes.byref(n), ctypes.byref(na), ctypes.byref(no),
                                   ctypes.byref(npr)), "bqc_basis_info")
        self.nbf, self.naux, self.nocc, self.nshell_pair = n.value, na.value, no.value, npr.value
        e = ctypes.c_double()
        check(lib().bqc_basis_enuc(h, ctypes.byref(e)), "bqc_basis_enuc")
        self.enuc = e.value

    @property
    def npair(self) -> int:
        return self.nbf * (self.nbf + 1) // 2

    def close(self):
        if getattr(self, "h", None):
            lib().bqc_basis_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _empty(shape, dtype=None):
    import torch
    return torch.empty(shape, dtype=dtype or torch.float64, device="cuda")


def one_electron(basis: Basis, stream=None):
    """(S, T, Vne) as N x N device tensors."""
    n = basis.nbf
    S, T, V = _empty((n, n)), _empty((n, n)), _empty((n, n))
    check(lib().bqc_one_electron(basis.h, _ptr(S), _ptr(T), _ptr(V), _stream_ptr(stream)),
          "bqc_one_electron")
    return S, T, V


def boys(ctx: Context, T, mmax: int, stream=None):
    """Device Boys function values, (len(T), mmax+1)."""
    out = _empty((T.numel(), mmax + 1))
    check(lib().bqc_boys(ctx.h, T.numel(), _ptr(T), mmax, _ptr(out), _stream_ptr(stream)),
          "bqc_boys")
    return out


def int2c(basis: Basis, stream=None):
    V = _empty((basis.naux, basis.naux))
    check(lib().bqc_int2c(basis.h, _ptr(V), _stream_ptr(stream)), "bqc_int2c")
    return V


def int3c(basis: Basis, schwarz: float = 0.0, stream=None):
    """Raw (P|mu nu), (Naux, Npair) packed lower triangle."""
    out = _empty((basis.naux, basis.npair))
    check(lib().bqc_int3c(basis.h, schwarz, _ptr(out), _stream_ptr(stream)), "bqc_int3c")
    return out


class DF:
    """bqc_df: the density-fitting tensor (stored) or its on-the-fly machinery (direct)."""

    def __init__(self, ctx: Context, basis: Basis, mode: int = DF_STORED, schwarz: float = -1.0,
                 aux_block: int = 1024, keep_fp32=True, hbm_limit: int = 0, stream=None,
                 aux_range=None):
        """keep_fp32: True / SHADOW_TF32 (split TF32 shadows), SHADOW_F16 (split
        FP16 shadows, for PREC_MIXED_F16X3), False / SHADOW_NONE (FP64 only).
        aux_range: (P0, P1) to hold only that aux shard of B (stored mode)."""
        self.ctx, self.basis = ctx, basis
        shadow = SHADOW_TF32 if keep_fp32 is True else (SHADOW_NONE if keep_fp32 is False
                                                          else int(keep_fp32))
        p0, p1 = aux_range if aux_range is not None else (0, 0)
        o = bqc_df_opts(mode, schwarz, aux_block, shadow, hbm_limit, p0, p1)
        h = vp()
        check(lib().bqc_df_build(ctx.h, basis.h, ctypes.byref(o), _stream_ptr(stream),
                                 ctypes.byref(h)), "bqc_df_build")
        self.h = h
        m, b = ctypes.c_int(), ctypes.c_size_t()
        check(lib().bqc_df_info(h, ctypes.byref(m), ctypes.byref(b)), "bqc_df_info")
        self.mode, self.device_bytes = m.value, b.value
        a0, a1 = ctypes.c_int(), ctypes.c_int()
        check(lib().bqc_df_shard(h, ctypes.byref(a0), ctypes.byref(a1)), "bqc_df_shard")
        self.aux_range = (a0.value, a1.value)

    def screening(self):
        """(shell triplets considered, kept) by the Schwarz screening."""
        c, k = ctypes.c_int64(), ctypes.c_int64()
        check(lib().bqc_df_screening(self.h, ctypes.byref(c), ctypes.byref(k)), "bqc_df_screening")
        return c.value, k.value

    def int3c_screened(self, p0: int, p1: int, variant: int = 0, out=None, stream=None):
        """(P|mu nu) for aux functions [p0, p1) with this handle's screening and
        the chosen survivor compaction (0 sorted prefix, 1 loop buffer, 2 list)."""
        import torch
        if out is None:
            out = torch.zeros((p1 - p0, self.basis.npair), dtype=torch.float64, device="cuda")
        check(lib().bqc_int3c_screened(self.h, p0, p1, variant, _ptr(out), _stream_ptr(stream)),
              "bqc_int3c_screened")
        return out

    def copy(self, which: int = 0, stream=None):
        """B (Naux, Npair) for which=0, the Cholesky factor L (Naux, Naux) for which=1."""
        shape = (self.aux_range[1] - self.aux_range[0], self.basis.npair) if which == 0 else \
            (self.basis.naux, self.basis.naux)
        out = _empty(shape)
        check(lib().bqc_df_copy(self.h, which, _ptr(out), _stream_ptr(stream)), "bqc_df_copy")
        return out

    def jk(self, Cocc, prec: int = PREC_FP64, J=None, K=None, stream=None):
        """J, K (N x N device tensors) from C_occ (N x nocc device tensor)."""
        n = self.basis.nbf
        J = _empty((n, n)) if J is None else J
        K = _empty((n, n)) if K is None else K
        check(lib().bqc_jk(self.h, _ptr(Cocc), Cocc.shape[1], prec, _ptr(J), _ptr(K),
                           _stream_ptr(stream)), "bqc_jk")
        return J, K

    def jk_host(self, Cocc_host, prec: int = PREC_FP64, J=None, K=None, stream=None):
        """J, K into host (numpy, preferably pinned) arrays from a host C_occ."""
        import numpy as np
        n = self.basis.nbf
        J = np.empty((n, n)) if J is None else J
        K = np.empty((n, n)) if K is None else K
        C = np.ascontiguousarray(Cocc_host, dtype=np.float64)
        check(lib().bqc_jk_host(self.h, C.ctypes.data, C.shape[1], prec, J.ctypes.data,
                                K.ctypes.data, _stream_ptr(stream)), "bqc_jk_host")
        return J, K

    def coulomb(self, D, variant: int = 0, J=None, stream=None):
        """J[D] (N x N device tensor) of a symmetric density by the two passes
        over B: variant COULOMB_FP64 (FP64 FMAs) or COULOMB_FF (float-float)."""
        n = self.basis.nbf
        J = _empty((n, n)) if J is None else J
        check(lib().bqc_df_coulomb(self.h, _ptr(D), _ptr(J), variant, _stream_ptr(stream)),
              "bqc_df_coulomb")
        return J

    def timing(self, enable: bool = True):
        check(lib().bqc_df_timing(self.h, 1 if enable else 0), "bqc_df_timing")

    def phase_ms(self):
        """[X pass, J pass, K, prep] ms of the last timed bqc_jk."""
        out = (ctypes.c_float * 4)()
        check(lib().bqc_df_phase_ms(self.h, out, 4), "bqc_df_phase_ms")
        return list(out)

    def close(self):
        if getattr(self, "h", None):
            lib().bqc_df_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mp2(df: DF, C, eps, prec: int = PREC_FP64, stream=None) -> float:
    """DF-MP2 correlation energy from canonical orbitals C (N x nmo device
    tensor, occupied first) and orbital energies eps (nmo device tensor)."""
    e2 = ctypes.c_double()
    C = C.contiguous()
    eps = eps.contiguous()
    check(lib().bqc_mp2(df.h, _ptr(C), _ptr(eps), C.shape[1], prec, ctypes.byref(e2),
                        _stream_ptr(stream)), "bqc_mp2")
    return e2.value


def scf_run(ctx: Context, df: DF, prec: int = PREC_FP64, diis_tol: float = 1e-8,
            energy_tol: float = 1e-10, stage_tol: float = 1e-5, max_iter: int = 100,
            diis_space: int = 8, orth_thresh: float = 1e-8, stream=None, keep_arrays=False,
            incremental: bool = False, guess=None):
    """Runs bqc_scf_run; returns a dict (energy, iterations, converged, ...,
    history = [(prec, DIIS error, energy)] per Fock build).

    With keep_arrays the MO coefficients (N x nmo), orbital energies and the
    last Fock matrix come back as device tensors.  guess: a contiguous
    N x nocc device tensor of occupied orbitals to start from (resume from a
    checkpoint, e.g. result["C"][:, :nocc].contiguous()).
    """
    o = bqc_scf_opts(diis_tol, energy_tol, stage_tol, max_iter, diis_space, prec, orth_thresh,
                     1 if incremental else 0, _ptr(guess) if guess is not None else None)
    r = bqc_scf_result()
    n = df.basis.nbf
    cap = 2 * max_iter + 2
    hist = (ctypes.c_double * (3 * cap))()
    r.history, r.history_cap = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)), cap
    if keep_arrays:
        Cbuf, eps, F = _empty((n * n,)), _empty((n,)), _empty((n, n))
        r.C_dev, r.eps_dev, r.F_dev = _ptr(Cbuf), _ptr(eps), _ptr(F)
    st = lib().bqc_scf_run(ctx.h, df.h, ctypes.byref(o), _stream_ptr(stream), ctypes.byref(r))
    if st not in (BQC_OK, BQC_E_NOT_CONVERGED):
        raise BqcError(st, "bqc_scf_run")
    out = dict(energy=r.energy, e_nuc=r.e_nuc, diis_err=r.diis_err, iterations=r.iterations,
               converged=bool(r.converged), iterations_mixed=r.iterations_mixed, nmo=r.nmo,
               switch_rule={0: None, 1: "stage_tol", 2: "floor"}.get(r.switch_rule),
               switch_err=r.switch_err if r.switch_rule else None,
               builds={"fp64": r.builds_fp64, "mixed": r.builds_mixed,
                       "incremental": r.builds_incremental},
               history=[(int(hist[3 * i]), hist[3 * i + 1], hist[3 * i + 2])
                        for i in range(r.history_len)])
    if keep_arrays:
        out.update(C=Cbuf[: n * r.nmo].view(n, r.nmo), eps=eps[: r.nmo], F=F)
    return out


class Server:
    """bqc_server: continuous batching of SCF solves (see bqc_serve_create)."""

    def __init__(self, ctx: Context, max_slots: int = 4, hbm_budget: int = 0,
                 prec: int = PREC_MIXED_F16X3, diis_tol: float = 1e-8, energy_tol: float = 1e-10,
                 stage_tol: float = 1e-5, max_iter: int = 100, diis_space: int = 8,
                 orth_thresh: float = 1e-8, policy: int = 0, max_skips: int = 8,
                 incremental: bool = False, grouped: bool = False,
                 group_window_us: float = 1000.0):
        self.ctx = ctx
        o = bqc_serve_opts(max_slots, hbm_budget, prec,
                           bqc_scf_opts(diis_tol, energy_tol, stage_tol, max_iter, diis_space,
                                        prec, orth_thresh, 1 if incremental else 0),
                           policy, max_skips, 1 if grouped else 0, group_window_us)
        h = vp()
        check(lib().bqc_serve_create(ctx.h, ctypes.byref(o), ctypes.byref(h)), "bqc_serve_create")
        self.h = h

    def submit(self, mol) -> int:
        """Queues a solve of a workload.Molecule; returns its ticket."""
        req, keep = molecule_request(mol)
        t = ctypes.c_uint64()
        check(lib().bqc_serve_submit(self.h, ctypes.byref(req), ctypes.byref(t)), "bqc_serve_submit")
        del keep  # the server copied the request
        return t.value

    def poll(self, ticket: int):
        """Result dict once done, else None."""
        r = bqc_serve_result()
        st = lib().bqc_serve_poll(self.h, ticket, ctypes.byref(r))
        if st == BQC_E_NOT_READY:
            return None
        check(st, "bqc_serve_poll")
        return dict(status=r.status, energy=r.energy, diis_err=r.diis_err,
                    iterations=r.iterations, nbf=r.nbf, t_submit=r.t_submit, t_admit=r.t_admit,
                    t_done=r.t_done, iterations_mixed=r.iterations_mixed, priority=r.priority)

    def cancel(self, ticket: int):
        """Cancels a queued or running request (bqc_serve_cancel)."""
        check(lib().bqc_serve_cancel(self.h, ticket), "bqc_serve_cancel")

    def drain(self, timeout_s: float = 0.0):
        check(lib().bqc_serve_drain(self.h, timeout_s), "bqc_serve_drain")

    def group_stats(self):
        """Grouped-build counters: batches, builds, largest batch."""
        b, j, m = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int()
        check(lib().bqc_serve_group_stats(self.h, ctypes.byref(b), ctypes.byref(j),
                                          ctypes.byref(m)), "bqc_serve_group_stats")
        return dict(batches=b.value, builds=j.value, max_batch=m.value)

    def close(self):
        if getattr(self, "h", None):
            lib().bqc_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def jk_grouped(dfs, Cs, Js=None, Ks=None, stream=None):
    """bqc_jk_grouped: split-FP16 J, K of several independent handles in
    grouped launches; returns the lists (Js, Ks) of N_k x N_k device tensors."""
    n = len(dfs)
    if len(Cs) != n:
        raise ValueError("one C per handle")
    Js = [_empty((d.basis.nbf, d.basis.nbf)) for d in dfs] if Js is None else Js
    Ks = [_empty((d.basis.nbf, d.basis.nbf)) for d in dfs] if Ks is None else Ks
    arr = ctypes.c_void_p * max(1, n)
    h = arr(*[d.h for d in dfs])
    c = arr(*[_ptr(x) for x in Cs])
    j = arr(*[_ptr(x) for x in Js])
    k = arr(*[_ptr(x) for x in Ks])
    check(lib().bqc_jk_grouped(n, h, c, j, k, _stream_ptr(stream)), "bqc_jk_grouped")
    return Js, Ks


def serve_footprint(nbf: int, naux: int, nocc: int, prec: int = PREC_MIXED_F16X3) -> int:
    return int(lib().bqc_serve_footprint(nbf, naux, nocc, prec))
