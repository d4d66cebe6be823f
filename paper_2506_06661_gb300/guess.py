"""Learned initial guess: data from converged SCFs, GPU training, evaluation.

Thin orchestration over the library's guess_* entry points (features, targets, MLP
forward / backward / Adam, density assembly) and scf_run_batch.  The paper lets the SCF
start from any density (Section "Initial Guess for Mean-field Methods"); the model here
predicts one from geometry, and scf_run falls back to the core-Hamiltonian guess when
the prediction fails the trace or idempotency check.

Random numbers (weight initialisation, mini-batch order) are drawn on the host with
numpy's PCG64 and passed to the GPU.
"""
from __future__ import annotations

import ctypes
import json
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import (DF_OK, DFError, MoleculeOnDevice, _check, _dev, _ptr, _stream, _work, lib, scf_run_batch)

NIN, NHID, NOUT, NRBF = 65, 256, 15, 32
LAYERS = [(NIN, NHID), (NHID, NHID), (NHID, NHID), (NHID, NOUT)]


def param_count() -> int:
    return int(lib().guess_mlp_param_count())


def init_params(seed: int = 0) -> np.ndarray:
    """Uniform(-sqrt(3/fan_in), +sqrt(3/fan_in)) weights, zero biases, flattened per layer
    as W [out][in] then b [out] (the library's parameter layout)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in LAYERS:
        bound = np.sqrt(3.0 / fan_in)
        parts.append(rng.uniform(-bound, bound, size=(fan_out, fan_in)).ravel())
        parts.append(np.zeros(fan_out))
    flat = np.concatenate(parts)
    if flat.size != param_count():
        raise RuntimeError(f"initial parameters: {flat.size} values, the library expects {param_count()}")
    return flat


@dataclass
class GuessModel:
    params: torch.Tensor                     # float32 [param_count] on the GPU
    m: torch.Tensor | None = None            # Adam first moment
    v: torch.Tensor | None = None            # Adam second moment
    step: int = 0
    history: list = field(default_factory=list)

    @classmethod
    def create(cls, seed: int = 0) -> "GuessModel":
        p = torch.tensor(init_params(seed), dtype=torch.float32, device="cuda")
        return cls(p, torch.zeros_like(p), torch.zeros_like(p), 0)

    @classmethod
    def create_on_device(cls, seed: int = 0) -> "GuessModel":
        """Initialise through the library's guess_mlp_create (counter-based generator on the
        GPU) instead of the host generator of create()."""
        p = torch.empty(param_count(), dtype=torch.float32, device="cuda")
        m, v = torch.empty_like(p), torch.empty_like(p)
        _check(lib().guess_mlp_create(ctypes.c_ulonglong(seed), _ptr(p), _ptr(m), _ptr(v), _stream()))
        return cls(p, m, v, 0)

    def to_blob(self, with_moments: bool = True) -> bytes:
        """The library's self-describing model blob (guess_mlp_save)."""
        n = int(lib().guess_mlp_blob_bytes(1 if with_moments else 0))
        buf = ctypes.create_string_buffer(n)
        _check(lib().guess_mlp_save(_ptr(self.params), _ptr(self.m) if with_moments else None,
                                    _ptr(self.v) if with_moments else None, self.step, buf, n, _stream()))
        return buf.raw

    @classmethod
    def from_blob(cls, blob: bytes) -> "GuessModel":
        p = torch.empty(param_count(), dtype=torch.float32, device="cuda")
        m, v = torch.empty_like(p), torch.empty_like(p)
        step = ctypes.c_int(0)
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        _check(lib().guess_mlp_load(buf, len(blob), _ptr(p), _ptr(m), _ptr(v), ctypes.byref(step), _stream()))
        return cls(p, m, v, step.value)

    def save(self, path: str) -> None:
        """Write the model blob (parameters, Adam moments and step) to a file."""
        with open(path, "wb") as fh:
            fh.write(self.to_blob(True))

    @classmethod
    def load(cls, path: str) -> "GuessModel":
        with open(path, "rb") as fh:
            return cls.from_blob(fh.read())


def features(xyz):
    """(feat [npairs, 65] float32, mask [npairs]) for one geometry (pairs A >= B, packed)."""
    x = _dev(xyz)
    natm = x.shape[0]
    npairs = natm * (natm + 1) // 2
    feat = torch.empty(npairs, NIN, dtype=torch.float32, device="cuda")
    mask = torch.empty(npairs, dtype=torch.float32, device="cuda")
    w = _work(128 * natm)
    _check(lib().guess_features(_ptr(x), natm, _ptr(feat), _ptr(mask), _ptr(w), w.numel(), _stream()))
    return feat, mask


def lowdin_factors(mol, lindep: float = 1e-8):
    """(S^1/2, S^-1/2) of the molecule's orbital overlap, on the GPU."""
    ao_xyz, ao_exp = _dev(mol.ao_xyz), _dev(mol.ao_exp)
    n = ao_exp.numel()
    Sh = torch.empty(n, n, dtype=torch.float64, device="cuda")
    Sih = torch.empty_like(Sh)
    w = _work(lib().df_lowdin_work_bytes(n))
    _check(lib().df_lowdin_factors(_ptr(ao_xyz), _ptr(ao_exp), n, ctypes.c_double(lindep), _ptr(Sh), _ptr(Sih),
                                   _ptr(w), w.numel(), _stream()))
    return Sh, Sih


def congruence(M: torch.Tensor, A) -> torch.Tensor:
    """M A M on the GPU."""
    A = _dev(A)
    n = A.shape[0]
    out = torch.empty_like(A)
    w = _work(lib().df_congruence_work_bytes(n))
    _check(lib().df_congruence(_ptr(M), _ptr(A), n, _ptr(out), _ptr(w), w.numel(), _stream()))
    return out


def targets(D, mol) -> torch.Tensor:
    """Blocks of the Loewdin density S^1/2 D S^1/2 for every centre pair."""
    Sh, _ = lowdin_factors(mol)
    Dt = congruence(Sh, D)
    natm = mol.natm
    Y = torch.empty(natm * (natm + 1) // 2, NOUT, dtype=torch.float32, device="cuda")
    _check(lib().guess_targets(_ptr(Dt), natm, _ptr(Y), _stream()))
    return Y


def forward(params: torch.Tensor, X: torch.Tensor, bf16: bool = False) -> torch.Tensor:
    n = X.shape[0]
    out = torch.empty(n, NOUT, dtype=torch.float32, device="cuda")
    w = _work(lib().guess_mlp_work_bytes(n))
    _check(lib().guess_mlp_forward(_ptr(params), _ptr(X.contiguous()), n, _ptr(out), 1 if bf16 else 0, _ptr(w),
                                   w.numel(), _stream()))
    return out


def loss_grad(params: torch.Tensor, X, Y, mask=None):
    n = X.shape[0]
    nvalid = float(mask.sum().item()) if mask is not None else float(n)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(params)
    w = _work(lib().guess_mlp_work_bytes(n))
    _check(lib().guess_mlp_loss_grad(_ptr(params), _ptr(X), _ptr(Y), _ptr(mask), n, ctypes.c_float(nvalid), _ptr(loss),
                                     _ptr(grad), _ptr(w), w.numel(), _stream()))
    return float(loss.item()), grad


def predict_density(model_or_params, mol, normalise: bool = True) -> torch.Tensor:
    """Starting density dm0 = S^-1/2 Dt S^-1/2 from the network's Loewdin-basis blocks, with
    Dt scaled to tr(Dt) = nelec unless normalise is False."""
    params = model_or_params.params if isinstance(model_or_params, GuessModel) else model_or_params
    _, Sih = lowdin_factors(mol)
    x = _dev(mol.xyz)
    natm = x.shape[0]
    D0 = torch.empty(5 * natm, 5 * natm, dtype=torch.float64, device="cuda")
    w = _work(lib().guess_density_work_bytes(natm))
    _check(lib().guess_density(_ptr(params), _ptr(x), natm, int(mol.nelec) if normalise else 0, _ptr(Sih), _ptr(D0), _ptr(w), w.numel(), _stream()))
    return D0


def build_dataset(mols, Ds):
    """Concatenated (X, Y, mask) over molecules with converged densities Ds."""
    Xs, Ys, Ms = [], [], []
    for mol, D in zip(mols, Ds):
        f, m = features(mol.xyz)
        Xs.append(f)
        Ms.append(m)
        Ys.append(targets(D, mol))
    return torch.cat(Xs), torch.cat(Ys), torch.cat(Ms)


def train(model: GuessModel, X, Y, mask, epochs: int = 10, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
          log=None):
    """Mini-batch Adam over valid pair samples; the permutation is drawn on the host."""
    keep = torch.nonzero(mask > 0).squeeze(1)
    X, Y = X[keep].contiguous(), Y[keep].contiguous()
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    w = _work(lib().guess_mlp_work_bytes(batch))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for ep in range(epochs):
        perm = torch.tensor(rng.permutation(n), device="cuda")
        tot, cnt = 0.0, 0
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            xb, yb = X[idx].contiguous(), Y[idx].contiguous()
            nb = xb.shape[0]
            model.step += 1
            _check(lib().guess_mlp_train_step(_ptr(model.params), _ptr(model.m), _ptr(model.v), model.step,
                                              ctypes.c_float(lr), _ptr(xb), _ptr(yb), None, nb, ctypes.c_float(nb),
                                              _ptr(loss), _ptr(w), w.numel(), _stream()))
            tot += float(loss.item()) * nb
            cnt += nb
        model.history.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep + 1}/{epochs}: mse {model.history[-1]:.3e}")
    return model.history


def converged_densities(mols, slots: int = 32, precision: str = "fp64", chunk: int = 512):
    """Run the batched SCF and return (results, densities) for training data."""
    res, Ds = [], []
    for i in range(0, len(mols), chunk):
        out = scf_run_batch(mols[i:i + chunk], slots=slots, precision=precision, want_D=True,
                            raise_on_noconv=False)
        res += out.results
        Ds += out.D
    return res, Ds


def evaluate(model: GuessModel, mols, slots: int = 32, precision: str = "mixed", want_D: bool = False,
             core_run=None, in_library: bool = True):
    """Batched SCF from the core guess and from the learned guess on the same molecules.
    With want_D the converged densities of both runs are returned too (keys D_core,
    D_learned), and per-molecule energies and iterations always are.  core_run = (batch
    result, seconds) of an earlier core-guess run on the same molecules skips that run.
    in_library: the batched SCF predicts each starting density itself (scf_opts.guess_params,
    from the overlap eigen-decomposition it computes anyway); else dm0 comes from
    predict_density, one molecule after another, before the batch."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if core_run is None:
        out_core = scf_run_batch(mols, slots=slots, precision=precision, raise_on_noconv=False, want_D=want_D)
        torch.cuda.synchronize()
        t_core = time.perf_counter() - t0
    else:
        out_core, t_core = core_run
    core = out_core.results
    t0 = time.perf_counter()
    if in_library:
        t_predict = 0.0
        out_learned = scf_run_batch(mols, slots=slots, precision=precision, guess_params=model.params,
                                    raise_on_noconv=False, want_D=want_D)
    else:
        dm0 = [predict_density(model, m) for m in mols]
        torch.cuda.synchronize()
        t_predict = time.perf_counter() - t0
        out_learned = scf_run_batch(mols, slots=slots, precision=precision, dm0s=dm0, raise_on_noconv=False,
                                    want_D=want_D)
    learned = out_learned.results
    torch.cuda.synchronize()
    t_learned = time.perf_counter() - t0
    both = [i for i in range(len(mols)) if core[i].converged and learned[i].converged]
    # SCF equations of these clusters can have several solutions: compare iteration counts
    # over the molecules where both starts reach the same state (|dE| <= 1e-6 Eh)
    same = [i for i in both if abs(core[i].energy - learned[i].energy) <= 1e-6]
    other = [learned[i].energy - core[i].energy for i in both if i not in same]
    it_core = np.array([core[i].iterations for i in same], dtype=float)
    it_learn = np.array([learned[i].iterations for i in same], dtype=float)
    de = np.array([abs(core[i].energy - learned[i].energy) for i in same])
    ev = {"molecules": len(mols), "both_converged": len(both), "same_state": len(same),
            "other_state": [i for i in both if i not in same],
            "energy_core": [r.energy for r in core], "energy_learned": [r.energy for r in learned],
            "iterations_core": [r.iterations for r in core], "iterations_learned": [r.iterations for r in learned],
            "other_state_dE_learned_minus_core": other,
            "mean_iter_core": float(it_core.mean()) if same else None,
            "mean_iter_learned": float(it_learn.mean()) if same else None,
            "wall_s_core": t_core, "wall_s_learned": t_learned, "wall_s_predict": t_predict,
            "guess_used": int(sum(r.guess == 1 for r in learned)), "guess_rejected": int(sum(r.guess == 2 for r in learned)),
            "max_abs_dE_same_state": float(de.max()) if same else None, "converged_core": int(sum(r.converged for r in core)),
            "converged_learned": int(sum(r.converged for r in learned))}
    if want_D:
        ev["D_core"], ev["D_learned"] = out_core.D, out_learned.D
    ev["_core_run"] = (out_core, t_core)
    return ev
