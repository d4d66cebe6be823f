"""GB300 (sm_103a) density-fitted Hartree-Fock: thin Python binding of libdfscf.so.

Every function here only marshals torch CUDA tensors into the C ABI declared in
include/dfscf.h; all computation happens in the library's CUDA kernels.  There is no
CPU fallback: if the library is missing or no GPU is present, calls raise.

Method: density fitting as stated in arXiv 2506.06661, Section "Density fitting"
(M = L L^T, B = L^-1 (Q|mn)), the DF Coulomb and exchange builds
J = sum_P B_P (B_P . D), K = sum_P (B_P C)(B_P C)^T, and an RHF SCF with DIIS.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

DF_OK = 0
DF_ERR_ARG = 1
DF_ERR_CUDA = 2
DF_ERR_NOT_SPD = 3
DF_ERR_NOCONV = 4
DF_ERR_TIMEOUT = 5
DF_ERR_NOMEM = 6
DF_ERR_NUMERIC = 7
DF_FP64 = 0
DF_MIXED = 1
_PREC = {"fp64": DF_FP64, "mixed": DF_MIXED, DF_FP64: DF_FP64, DF_MIXED: DF_MIXED}


class DFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code
        self.msg = msg


class DFMolecule(ctypes.Structure):
    _fields_ = [("natm", ctypes.c_int), ("xyz", ctypes.c_void_p), ("charges", ctypes.c_void_p),
                ("nao", ctypes.c_int), ("ao_xyz", ctypes.c_void_p), ("ao_exp", ctypes.c_void_p),
                ("naux", ctypes.c_int), ("aux_xyz", ctypes.c_void_p), ("aux_exp", ctypes.c_void_p),
                ("nelec", ctypes.c_int)]


class ScfOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("diis_space", ctypes.c_int), ("max_cycle", ctypes.c_int),
                ("n_fp64_final", ctypes.c_int), ("conv_tol", ctypes.c_double), ("conv_err", ctypes.c_double),
                ("lindep", ctypes.c_double), ("switch_tol", ctypes.c_double), ("switch_err", ctypes.c_double),
                ("verbose", ctypes.c_int), ("guess_params", ctypes.c_void_p)]


class ScfResultC(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("e_nuc", ctypes.c_double), ("homo", ctypes.c_double),
                ("lumo", ctypes.c_double), ("last_de", ctypes.c_double), ("last_err", ctypes.c_double),
                ("iterations", ctypes.c_int), ("fp64_iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("guess", ctypes.c_int), ("nmo", ctypes.c_int), ("hess_min", ctypes.c_double),
                ("stability_restarts", ctypes.c_int)]


_lib = None
_VP = ctypes.c_void_p
_SZ = ctypes.c_size_t
_I = ctypes.c_int
_L = ctypes.c_long
_D = ctypes.c_double

_SIGS = {
    "df_last_error": (ctypes.c_char_p, []),
    "df_version": (_I, []),
    "df_boys_f0": (_I, [_VP, _L, _VP, _VP]),
    "df_int1e": (_I, [_VP, _VP, _I, _VP, _VP, _I, _VP, _VP, _VP, _VP]),
    "df_nuclear_repulsion": (_I, [_VP, _VP, _I, _VP, _VP]),
    "df_metric_chol_work_bytes": (_SZ, [_I]),
    "df_metric_chol": (_I, [_VP, _VP, _I, _VP, _VP, ctypes.POINTER(_I), _VP, _SZ, _VP]),
    "df_B_ld": (_L, [_I]),
    "df_nao_pad": (_I, [_I]),
    "df_B_bytes": (_SZ, [_I, _I, _I]),
    "df_build_B_work_bytes": (_SZ, [_I, _I]),
    "df_build_B": (_I, [_VP, _VP, _I, _VP, _VP, _I, _VP, _I, _VP, _SZ, _VP, _SZ, _VP]),
    "df_B_get_packed": (_I, [_VP, _I, _I, _I, _VP, _VP]),
    "df_jk_work_bytes": (_SZ, [_I, _I, _I, _I]),
    "df_jk": (_I, [_VP, _I, _I, _I, _VP, _VP, _I, _VP, _VP, _VP, _SZ, _VP]),
    "df_eigh_work_bytes": (_SZ, [_I]),
    "df_eigh": (_I, [_VP, _I, _VP, _VP, _VP, _SZ, _VP]),
    "df_tune_set": (_I, [ctypes.c_char_p, _I]),
    "df_tune_get": (_I, [ctypes.c_char_p]),
    "df_tune_reset": (None, []),
    "df_eigh_lowest_work_bytes": (_SZ, [_I, _I]),
    "df_eigh_lowest": (_I, [_VP, _I, _I, _VP, _VP, _VP, _SZ, _VP]),
    "scf_default_opts": (None, [ctypes.POINTER(ScfOpts)]),
    "df_core_guess_work_bytes": (_SZ, [_I, _I]),
    "df_core_guess": (_I, [ctypes.POINTER(DFMolecule), _D, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(_I), _VP, _SZ,
                           _VP]),
    "df_profile_enable": (None, [_I]),
    "df_profile_reset": (None, []),
    "df_profile_count": (_I, []),
    "df_profile_name": (ctypes.c_char_p, [_I]),
    "df_profile_ms": (_D, [_I]),
    "df_profile_calls": (_L, [_I]),
    "scf_work_bytes": (_SZ, [_I, _I, _I, _I]),
    "scf_run": (_I, [ctypes.POINTER(DFMolecule), ctypes.POINTER(ScfOpts), _VP, _VP, _VP, _VP,
                     ctypes.POINTER(ScfResultC), _VP, _SZ, _VP]),
    "guess_mlp_param_count": (_SZ, []),
    "guess_mlp_work_bytes": (_SZ, [_I]),
    "guess_features": (_I, [_VP, _I, _VP, _VP, _VP, _SZ, _VP]),
    "guess_targets": (_I, [_VP, _I, _VP, _VP]),
    "guess_mlp_forward": (_I, [_VP, _VP, _I, _VP, _I, _VP, _SZ, _VP]),
    "guess_mlp_loss_grad": (_I, [_VP, _VP, _VP, _VP, _I, ctypes.c_float, _VP, _VP, _VP, _SZ, _VP]),
    "guess_mlp_train_step": (_I, [_VP, _VP, _VP, _I, ctypes.c_float, _VP, _VP, _VP, _I, ctypes.c_float, _VP, _VP,
                                  _SZ, _VP]),
    "guess_mlp_create": (_I, [ctypes.c_ulonglong, _VP, _VP, _VP, _VP]),
    "guess_mlp_blob_bytes": (_SZ, [_I]),
    "guess_mlp_save": (_I, [_VP, _VP, _VP, _I, _VP, _SZ, _VP]),
    "guess_mlp_load": (_I, [_VP, _SZ, _VP, _VP, _VP, ctypes.POINTER(_I), _VP]),
    "guess_density_work_bytes": (_SZ, [_I]),
    "guess_density": (_I, [_VP, _VP, _I, _I, _VP, _VP, _VP, _SZ, _VP]),
    "df_lowdin_work_bytes": (_SZ, [_I]),
    "df_lowdin_factors": (_I, [_VP, _VP, _I, _D, _VP, _VP, _VP, _SZ, _VP]),
    "df_congruence_work_bytes": (_SZ, [_I]),
    "df_congruence": (_I, [_VP, _VP, _I, _VP, _VP, _SZ, _VP]),
    "df_fit_residual_work_bytes": (_SZ, [_I, _I, _I]),
    "df_fit_residual": (_I, [_VP, _VP, _I, _VP, _VP, _I, _VP, _I, _VP, _VP, ctypes.POINTER(_D), _VP, _SZ, _VP]),
    "df_lrdf_build_work_bytes": (_SZ, [_I, _I]),
    "df_lrdf_build": (_I, [_VP, _VP, _I, _VP, _VP, _I, _D, _VP, _SZ, _VP, _SZ, _VP]),
    "df_lrdf_jk_work_bytes": (_SZ, [_I, _I, _I]),
    "df_lrdf_jk": (_I, [_VP, _VP, _VP, _I, _I, _D, _VP, _VP, _I, _VP, _VP, _VP, _SZ, _VP]),
    "df_bounds_checked": (_I, []),
    "df_bounds_violations": (_I, [ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_char_p, _SZ]),
    "df_j_noalloc_capacity": (_SZ, []),
    "df_j_noalloc": (_I, [_VP, _I, _I, _VP, _VP, _VP]),
    "scf_batch_work_bytes": (_SZ, [ctypes.POINTER(DFMolecule), _I, _I, _I]),
    "scf_run_batch": (_I, [ctypes.POINTER(DFMolecule), _I, ctypes.POINTER(ScfOpts), ctypes.POINTER(_VP),
                           ctypes.POINTER(_VP), ctypes.POINTER(ScfResultC), _I, _VP, _SZ, _VP]),
}


def lib():
    """Load libdfscf.so (building it with nvcc first if it is missing or stale); with the
    environment variable DFSCF_VARIANT=bounds, the bounds-checking build instead."""
    global _lib
    if _lib is None:
        path = _build.build(variant=os.environ.get("DFSCF_VARIANT", ""))
        if not os.path.exists(path):
            raise RuntimeError("libdfscf.so is missing and could not be built")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def library_path() -> str:
    return _build.variant_path(os.environ.get("DFSCF_VARIANT", ""))


def bounds_violations():
    """(count, first location) of out-of-range indices since the last call (checking build)."""
    n = ctypes.c_ulonglong(0)
    where = ctypes.create_string_buffer(256)
    _check(lib().df_bounds_violations(ctypes.byref(n), where, 256))
    return int(n.value), where.value.decode()


def _check(rc: int):
    if rc != DF_OK:
        raise DFError(rc, lib().df_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise TypeError("tensors passed to the library must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _dev(x, dtype=torch.float64):
    if isinstance(x, torch.Tensor):
        return x.to(device="cuda", dtype=dtype).contiguous()
    return torch.as_tensor(x, dtype=dtype).to("cuda").contiguous()


def _work(nbytes: int) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device="cuda")


def boys_f0(t) -> torch.Tensor:
    t = _dev(t)
    out = torch.empty_like(t)
    _check(lib().df_boys_f0(_ptr(t), t.numel(), _ptr(out), _stream()))
    return out


def int1e(ao_xyz, ao_exp, nuc_xyz, nuc_z):
    ao_xyz, ao_exp, nuc_xyz, nuc_z = map(_dev, (ao_xyz, ao_exp, nuc_xyz, nuc_z))
    n = ao_exp.numel()
    S, T, V = (torch.empty(n, n, dtype=torch.float64, device="cuda") for _ in range(3))
    _check(lib().df_int1e(_ptr(ao_xyz), _ptr(ao_exp), n, _ptr(nuc_xyz), _ptr(nuc_z), nuc_z.numel(),
                          _ptr(S), _ptr(T), _ptr(V), _stream()))
    return S, T, V


def nuclear_repulsion(xyz, z) -> float:
    xyz, z = _dev(xyz), _dev(z)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    _check(lib().df_nuclear_repulsion(_ptr(xyz), _ptr(z), z.numel(), _ptr(out), _stream()))
    return float(out.item())


def metric_chol(aux_xyz, aux_exp, return_metric: bool = False):
    """(L, pivot) or (L, M, pivot); raises DFError(DF_ERR_NOT_SPD) on a bad pivot."""
    aux_xyz, aux_exp = _dev(aux_xyz), _dev(aux_exp)
    n = aux_exp.numel()
    L = torch.empty(n, n, dtype=torch.float64, device="cuda")
    M = torch.empty(n, n, dtype=torch.float64, device="cuda") if return_metric else None
    piv = ctypes.c_int(-1)
    w = _work(lib().df_metric_chol_work_bytes(n))
    rc = lib().df_metric_chol(_ptr(aux_xyz), _ptr(aux_exp), n, _ptr(L), _ptr(M), ctypes.byref(piv), _ptr(w),
                              w.numel(), _stream())
    if rc != DF_OK:
        err = DFError(rc, lib().df_last_error().decode())
        err.pivot = piv.value
        raise err
    return (L, M) if return_metric else L


@dataclass
class DFTensor:
    """Caller-owned whitened tensor B (layout documented in include/dfscf.h)."""
    buf: torch.Tensor
    nao: int
    naux: int
    precision: int

    @property
    def ld(self) -> int:
        return int(lib().df_B_ld(self.nao))


def B_bytes(nao: int, naux: int, precision="fp64") -> int:
    return int(lib().df_B_bytes(nao, naux, _PREC[precision]))


def build_B(ao_xyz, ao_exp, aux_xyz, aux_exp, L, precision="fp64") -> DFTensor:
    ao_xyz, ao_exp, aux_xyz, aux_exp, L = map(_dev, (ao_xyz, ao_exp, aux_xyz, aux_exp, L))
    nao, naux = ao_exp.numel(), aux_exp.numel()
    p = _PREC[precision]
    nb = B_bytes(nao, naux, p)
    buf = torch.empty(nb, dtype=torch.uint8, device="cuda")
    w = _work(lib().df_build_B_work_bytes(nao, naux))
    _check(lib().df_build_B(_ptr(ao_xyz), _ptr(ao_exp), nao, _ptr(aux_xyz), _ptr(aux_exp), naux, _ptr(L), p,
                            _ptr(buf), nb, _ptr(w), w.numel(), _stream()))
    return DFTensor(buf, nao, naux, p)


def B_get_packed(B: DFTensor, P: int) -> torch.Tensor:
    row = torch.empty(B.nao * (B.nao + 1) // 2, dtype=torch.float64, device="cuda")
    _check(lib().df_B_get_packed(_ptr(B.buf), B.nao, B.naux, P, _ptr(row), _stream()))
    return row


class JKWorkspace:
    """Reusable df_jk workspace for one (nao, naux, nocc, precision)."""

    def __init__(self, nao, naux, nocc, precision="fp64"):
        self.key = (nao, naux, nocc, _PREC[precision])
        self.buf = _work(lib().df_jk_work_bytes(nao, naux, nocc, _PREC[precision]))


def jk(B: DFTensor, D=None, C=None, precision=None, want_j=True, want_k=True, work: JKWorkspace | None = None,
       out_j=None, out_k=None):
    p = B.precision if precision is None else _PREC[precision]
    nao = B.nao
    D = _dev(D) if (D is not None and want_j) else None
    C = _dev(C) if (C is not None and want_k) else None
    nocc = C.shape[1] if C is not None else 0
    J = (out_j if out_j is not None else torch.empty(nao, nao, dtype=torch.float64, device="cuda")) if D is not None else None
    K = (out_k if out_k is not None else torch.empty(nao, nao, dtype=torch.float64, device="cuda")) if C is not None else None
    if work is None or work.key != (nao, B.naux, nocc, p):
        work = JKWorkspace(nao, B.naux, nocc, p)
    _check(lib().df_jk(_ptr(B.buf), nao, B.naux, p, _ptr(D), _ptr(C), nocc, _ptr(J), _ptr(K), _ptr(work.buf),
                       work.buf.numel(), _stream()))
    return J, K


def lrdf_build(ao_xyz, ao_exp, aux_xyz, aux_exp, omega: float) -> DFTensor:
    """Long-range whitened tensor T (FP64 B layout) of the LRDF scheme (df_lrdf_build)."""
    ao_xyz, ao_exp, aux_xyz, aux_exp = map(_dev, (ao_xyz, ao_exp, aux_xyz, aux_exp))
    nao, naux = ao_exp.numel(), aux_exp.numel()
    nb = B_bytes(nao, naux, "fp64")
    buf = torch.empty(nb, dtype=torch.uint8, device="cuda")
    w = _work(lib().df_lrdf_build_work_bytes(nao, naux))
    _check(lib().df_lrdf_build(_ptr(ao_xyz), _ptr(ao_exp), nao, _ptr(aux_xyz), _ptr(aux_exp), naux, float(omega),
                               _ptr(buf), nb, _ptr(w), w.numel(), _stream()))
    return DFTensor(buf, nao, naux, DF_FP64)


def lrdf_jk(T: DFTensor, ao_xyz, ao_exp, omega: float, D=None, C=None):
    """J[D] and K[C C^T] with long-range DF plus exact short-range four-centre terms."""
    ao_xyz, ao_exp = _dev(ao_xyz), _dev(ao_exp)
    nao = T.nao
    D = _dev(D) if D is not None else None
    C = _dev(C) if C is not None else None
    nocc = C.shape[1] if C is not None else 0
    J = torch.empty(nao, nao, dtype=torch.float64, device="cuda") if D is not None else None
    K = torch.empty(nao, nao, dtype=torch.float64, device="cuda") if C is not None else None
    w = _work(lib().df_lrdf_jk_work_bytes(nao, T.naux, nocc))
    _check(lib().df_lrdf_jk(_ptr(T.buf), _ptr(ao_xyz), _ptr(ao_exp), nao, T.naux, float(omega), _ptr(D), _ptr(C), nocc,
                            _ptr(J), _ptr(K), _ptr(w), w.numel(), _stream()))
    return J, K


def fit_residual(ao_xyz, ao_exp, aux_xyz, aux_exp, dalpha=None):
    """(sigma [npair], jac [npair][ntheta] or None, Delta) of the density fit (df_fit_residual)."""
    ao_xyz, ao_exp, aux_xyz, aux_exp = map(_dev, (ao_xyz, ao_exp, aux_xyz, aux_exp))
    nao, naux = ao_exp.numel(), aux_exp.numel()
    sigma = torch.empty(nao * (nao + 1) // 2, dtype=torch.float64, device="cuda")
    jac, nt, da = None, 0, None
    if dalpha is not None:
        da = _dev(dalpha)
        if da.dim() == 1:
            da = da.reshape(-1, 1).contiguous()
        nt = da.shape[1]
        jac = torch.empty(sigma.numel(), nt, dtype=torch.float64, device="cuda")
    w = _work(lib().df_fit_residual_work_bytes(nao, naux, 1 if jac is not None else 0))
    delta = ctypes.c_double(0.0)
    _check(lib().df_fit_residual(_ptr(ao_xyz), _ptr(ao_exp), nao, _ptr(aux_xyz), _ptr(aux_exp), naux, _ptr(da), nt,
                                 _ptr(sigma), _ptr(jac), ctypes.byref(delta), _ptr(w), w.numel(), _stream()))
    return sigma, jac, delta.value


def eigh(A):
    A = _dev(A).clone()
    n = A.shape[0]
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    Z = torch.empty(n, n, dtype=torch.float64, device="cuda")
    work = _work(lib().df_eigh_work_bytes(n))
    _check(lib().df_eigh(_ptr(A), n, _ptr(w), _ptr(Z), _ptr(work), work.numel(), _stream()))
    return w, Z


def eigh_lowest(A, k: int):
    """k lowest eigenpairs (w [k], Z [n][k]) of a symmetric matrix."""
    A = _dev(A).clone()
    n = A.shape[0]
    w = torch.empty(k, dtype=torch.float64, device="cuda")
    Z = torch.empty(n, k, dtype=torch.float64, device="cuda")
    work = _work(lib().df_eigh_lowest_work_bytes(n, k))
    _check(lib().df_eigh_lowest(_ptr(A), n, k, _ptr(w), _ptr(Z), _ptr(work), work.numel(), _stream()))
    return w, Z


def default_opts(**kw) -> ScfOpts:
    o = ScfOpts()
    lib().scf_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision":
            v = _PREC[v]
        elif k == "guess_params" and isinstance(v, torch.Tensor):
            # the learned guess's parameters (float32, on the device); the caller keeps them alive
            if not (v.dtype == torch.float32 and v.is_cuda and v.is_contiguous()):
                raise TypeError("guess_params must be a contiguous float32 CUDA tensor")
            v = v.data_ptr()
        setattr(o, k, v)
    return o


@dataclass
class SCFResult:
    energy: float
    e_nuc: float
    homo: float
    lumo: float
    last_de: float
    last_err: float
    iterations: int
    fp64_iterations: int
    converged: bool
    guess: int
    nmo: int
    D: torch.Tensor
    C: torch.Tensor
    mo_energy: torch.Tensor
    hess_min: float = float("nan")
    stability_restarts: int = 0


class MoleculeOnDevice:
    """Device copies of a gen.Molecule's arrays, kept alive for the C struct."""

    def __init__(self, mol):
        self.xyz = _dev(mol.xyz)
        self.charges = _dev(mol.charges)
        self.ao_xyz = _dev(mol.ao_xyz)
        self.ao_exp = _dev(mol.ao_exp)
        self.aux_xyz = _dev(mol.aux_xyz)
        self.aux_exp = _dev(mol.aux_exp)
        self.nao, self.naux, self.natm, self.nelec = mol.nao, mol.naux, mol.natm, mol.nelec
        self.c = DFMolecule(self.natm, self.xyz.data_ptr(), self.charges.data_ptr(), self.nao,
                            self.ao_xyz.data_ptr(), self.ao_exp.data_ptr(), self.naux, self.aux_xyz.data_ptr(),
                            self.aux_exp.data_ptr(), self.nelec)


def scf_work_bytes(nao, naux, nocc, precision="fp64") -> int:
    return int(lib().scf_work_bytes(nao, naux, nocc, _PREC[precision]))


def scf_run(mol, opts: ScfOpts | None = None, dm0=None, work: torch.Tensor | None = None,
            raise_on_noconv: bool = True, **kw) -> SCFResult:
    md = mol if isinstance(mol, MoleculeOnDevice) else MoleculeOnDevice(mol)
    o = opts if opts is not None else default_opts(**kw)
    nocc = md.nelec // 2
    nb = scf_work_bytes(md.nao, md.naux, nocc, o.precision)
    if work is None or work.numel() < nb:
        work = _work(nb)
    D = torch.empty(md.nao, md.nao, dtype=torch.float64, device="cuda")
    C = torch.empty(md.nao, nocc, dtype=torch.float64, device="cuda")
    eps = torch.zeros(nocc + 1, dtype=torch.float64, device="cuda")
    dm0 = _dev(dm0) if dm0 is not None else None
    r = ScfResultC()
    rc = lib().scf_run(ctypes.byref(md.c), ctypes.byref(o), _ptr(dm0), _ptr(D), _ptr(C), _ptr(eps), ctypes.byref(r),
                       _ptr(work), work.numel(), _stream())
    if rc != DF_OK and not (rc == DF_ERR_NOCONV and not raise_on_noconv):
        raise DFError(rc, lib().df_last_error().decode())
    return SCFResult(r.energy, r.e_nuc, r.homo, r.lumo, r.last_de, r.last_err, r.iterations, r.fp64_iterations,
                     bool(r.converged), r.guess, r.nmo, D, C, eps, r.hess_min, r.stability_restarts)


def core_guess(mol, lindep: float = 1e-8):
    """Core-Hamiltonian guess on the GPU: returns (C_occ, D, S, h, mo_energy, nmo)."""
    md = mol if isinstance(mol, MoleculeOnDevice) else MoleculeOnDevice(mol)
    nao, nocc = md.nao, md.nelec // 2
    S = torch.empty(nao, nao, dtype=torch.float64, device="cuda")
    h = torch.empty_like(S)
    D = torch.empty_like(S)
    C = torch.empty(nao, nocc, dtype=torch.float64, device="cuda")
    eps = torch.zeros(nocc + 1, dtype=torch.float64, device="cuda")
    nmo = ctypes.c_int(0)
    w = _work(lib().df_core_guess_work_bytes(nao, nocc))
    _check(lib().df_core_guess(ctypes.byref(md.c), lindep, _ptr(S), _ptr(h), _ptr(C), _ptr(D), _ptr(eps),
                               ctypes.byref(nmo), _ptr(w), w.numel(), _stream()))
    return C, D, S, h, eps, nmo.value


def profile_enable(on: bool = True) -> None:
    lib().df_profile_enable(1 if on else 0)


def profile_reset() -> None:
    lib().df_profile_reset()


def profile_read() -> dict:
    """{phase name: (total ms, launches)} since the last reset (synchronises)."""
    L = lib()
    n = L.df_profile_count()
    return {L.df_profile_name(i).decode(): (L.df_profile_ms(i), L.df_profile_calls(i)) for i in range(n)}


@dataclass
class BatchResult:
    results: list
    D: list | None


def scf_run_batch(mols, opts: ScfOpts | None = None, dm0s=None, slots: int = 16, want_D: bool = False,
                  work: torch.Tensor | None = None, raise_on_noconv: bool = True, **kw) -> BatchResult:
    """Batched DF-RHF over molecules of uneven size (scf_run_batch in the C ABI)."""
    devs = [m if isinstance(m, MoleculeOnDevice) else MoleculeOnDevice(m) for m in mols]
    n = len(devs)
    arr = (DFMolecule * n)(*[d.c for d in devs])
    o = opts if opts is not None else default_opts(**kw)
    slots = max(1, min(slots, n))
    if work is None:
        # molecules take regions of their own size: give the library up to `slots` copies of
        # the largest molecule, capped at 85% of the free device memory (it needs one)
        nb = int(lib().scf_batch_work_bytes(arr, n, o.precision, slots))
        largest = int(lib().scf_batch_work_bytes(arr, n, o.precision, 1))
        # blocks torch still caches (an earlier batch's workspace) count as free
        torch.cuda.empty_cache()
        free = torch.cuda.mem_get_info()[0]
        work = _work(max(largest, min(nb, int(0.85 * free))))
    dm0_t = None
    dm0_arr = None
    if dm0s is not None:
        dm0_t = [(_dev(d) if d is not None else None) for d in dm0s]
        dm0_arr = (_VP * n)(*[(t.data_ptr() if t is not None else None) for t in dm0_t])
    Ds = None
    D_arr = None
    if want_D:
        Ds = [torch.empty(d.nao, d.nao, dtype=torch.float64, device="cuda") for d in devs]
        D_arr = (_VP * n)(*[t.data_ptr() for t in Ds])
    res = (ScfResultC * n)()
    rc = lib().scf_run_batch(arr, n, ctypes.byref(o), dm0_arr, D_arr, res, slots, _ptr(work), work.numel(),
                             _stream())
    if rc != DF_OK and not (rc == DF_ERR_NOCONV and not raise_on_noconv):
        raise DFError(rc, lib().df_last_error().decode())
    out = [SCFResult(r.energy, r.e_nuc, r.homo, r.lumo, r.last_de, r.last_err, r.iterations, r.fp64_iterations,
                     bool(r.converged), r.guess, r.nmo, None, None, None, r.hess_min, r.stability_restarts)
           for r in res]
    return BatchResult(out, Ds)
