"""Learned initial guess: features, MLP forward/backward and Adam (oracle, FP64, numpy).

TEST INFRASTRUCTURE ONLY.  The paper allows any density matrix as an SCF starting
point, idempotent or not and with any electron count (Section "Initial Guess for
Mean-field Methods"); this module is the plain reference for the learned guess that
produces such a density from geometry:

* radial basis: 32 Gaussians exp(-gamma (R - r_k)^2), r_k = 12 k / 31 bohr,
  gamma = 1 / (12/31)^2, pairs beyond 12 bohr are dropped;
* environment of centre A: env_A = (1/8) sum_{C != A, R_AC <= 12} rbf(R_AC);
* features of an off-diagonal pair (A > B): [rbf(R_AB), env_A + env_B, 0];
  of a diagonal pair (A, A): [0, 2 env_A, 1]   (65 inputs, symmetric in A and B);
* network 65 -> 256 -> 256 -> 256 -> 15 with SiLU after each hidden layer;
* the 15 outputs are the upper triangle (row-major, a <= b) of a symmetric 5x5 block of
  the Loewdin-orthogonalised density Dt = S^1/2 D S^1/2 (eigenvalues 0 or 2 at
  convergence; the blocks of D itself are ill-conditioned in this strongly
  non-orthogonal basis); the starting density is D0 = S^-1/2 Dt S^-1/2;
* loss: mean squared error over all pairs and outputs; optimiser: Adam.
"""
from __future__ import annotations

import numpy as np

NRBF = 32
RCUT = 12.0
ENV_SCALE = 1.0 / 8.0
NIN = 2 * NRBF + 1
NHID = 256
NOUT = 15
NBF = 5  # orbital functions per centre
LAYERS = [(NIN, NHID), (NHID, NHID), (NHID, NHID), (NHID, NOUT)]

_RK = RCUT * np.arange(NRBF) / (NRBF - 1)
_GAMMA = 1.0 / (RCUT / (NRBF - 1)) ** 2
# (a, b) positions of the 15 unique entries, row-major upper triangle
TRIU = [(a, b) for a in range(NBF) for b in range(a, NBF)]


def rbf(r):
    r = np.asarray(r, dtype=np.float64)[..., None]
    return np.exp(-_GAMMA * (r - _RK) ** 2)


def pair_features(xyz: np.ndarray):
    """Returns (pairs [npairs, 2] with A >= B, features [npairs, 65])."""
    xyz = np.asarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    R = np.sqrt(((xyz[:, None, :] - xyz[None, :, :]) ** 2).sum(-1))
    env = np.zeros((n, NRBF))
    for a in range(n):
        for c in range(n):
            if c != a and R[a, c] <= RCUT:
                env[a] += rbf(R[a, c])
    env *= ENV_SCALE
    pairs, feats = [], []
    for a in range(n):
        for b in range(a + 1):
            if a == b:
                f = np.concatenate([np.zeros(NRBF), 2.0 * env[a], [1.0]])
            elif R[a, b] <= RCUT:
                f = np.concatenate([rbf(R[a, b]), env[a] + env[b], [0.0]])
            else:
                continue
            pairs.append((a, b))
            feats.append(f)
    return np.array(pairs, dtype=np.int64).reshape(-1, 2), np.array(feats).reshape(-1, NIN)


def init_params(seed: int = 0):
    """He-style uniform init; weights [out][in], biases [out]."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in LAYERS:
        bound = np.sqrt(3.0 / fan_in)
        params.append(rng.uniform(-bound, bound, size=(fan_out, fan_in)))
        params.append(np.zeros(fan_out))
    return params


def silu(z):
    return z / (1.0 + np.exp(-z))


def forward(params, X):
    """Returns (output [N, 15], cache of pre-activations and activations)."""
    acts = [X]
    pres = []
    h = X
    nl = len(LAYERS)
    for l in range(nl):
        W, b = params[2 * l], params[2 * l + 1]
        z = h @ W.T + b
        pres.append(z)
        h = silu(z) if l < nl - 1 else z
        acts.append(h)
    return h, (pres, acts)


def bf16_round(x):
    """Round to the nearest BF16 value (8 significant bits, ties to even), returned as float64:
    the top 16 bits of the IEEE single, rounded on the 16 bits dropped.  Finite inputs only."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(params, X):
    """BF16 inference: the inputs, every weight matrix and every hidden activation rounded to
    BF16; products and sums, bias and SiLU exact (FP64); the output layer's result unrounded."""
    h = bf16_round(X)
    nl = len(LAYERS)
    for l in range(nl):
        W, b = bf16_round(params[2 * l]), np.asarray(params[2 * l + 1], dtype=np.float64)
        z = h @ W.T + b
        h = bf16_round(silu(z)) if l < nl - 1 else z
    return h


def loss_and_grad(params, X, Y):
    """MSE loss (mean over N*15 entries) and its gradient w.r.t. every parameter."""
    out, (pres, acts) = forward(params, X)
    N = X.shape[0]
    diff = out - Y
    loss = float(np.mean(diff ** 2))
    g = 2.0 * diff / diff.size
    grads = [None] * len(params)
    nl = len(LAYERS)
    for l in reversed(range(nl)):
        if l < nl - 1:
            z = pres[l]
            sig = 1.0 / (1.0 + np.exp(-z))
            g = g * (sig * (1.0 + z * (1.0 - sig)))
        grads[2 * l] = g.T @ acts[l]
        grads[2 * l + 1] = g.sum(axis=0)
        g = g @ params[2 * l]
    del N
    return loss, grads


class Adam:
    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        for i, (p, g) in enumerate(zip(params, grads)):
            self.m[i] = self.b1 * self.m[i] + (1 - self.b1) * g
            self.v[i] = self.b2 * self.v[i] + (1 - self.b2) * g * g
            mhat = self.m[i] / (1 - self.b1 ** self.t)
            vhat = self.v[i] / (1 - self.b2 ** self.t)
            p -= self.lr * mhat / (np.sqrt(vhat) + self.eps)


def block_targets(D: np.ndarray, pairs: np.ndarray) -> np.ndarray:
    """15 unique entries of the symmetrised 5x5 block of D for every pair."""
    out = np.empty((len(pairs), NOUT))
    for k, (a, b) in enumerate(pairs):
        blk = D[NBF * a:NBF * a + NBF, NBF * b:NBF * b + NBF]
        blk = 0.5 * (blk + blk.T)
        out[k] = [blk[i, j] for i, j in TRIU]
    return out


def assemble_density(pred: np.ndarray, pairs: np.ndarray, natm: int) -> np.ndarray:
    """Symmetric nao x nao density from predicted blocks (absent pairs stay zero)."""
    nao = NBF * natm
    D = np.zeros((nao, nao))
    for k, (a, b) in enumerate(pairs):
        blk = np.zeros((NBF, NBF))
        for v, (i, j) in zip(pred[k], TRIU):
            blk[i, j] = blk[j, i] = v
        D[NBF * a:NBF * a + NBF, NBF * b:NBF * b + NBF] = blk
        D[NBF * b:NBF * b + NBF, NBF * a:NBF * a + NBF] = blk.T
    return D


def normalise_trace(Dt: np.ndarray, nelec: int) -> np.ndarray:
    """Orthonormal-basis density scaled to tr(Dt) = nelec; a non-positive trace is left as it
    is.  The starting density may carry any electron count (Section "Initial Guess for
    Mean-field Methods"); the scaling removes the network's systematic overshoot."""
    t = float(np.trace(Dt))
    return Dt * (nelec / t) if t > 0.0 else Dt.copy()


def lowdin_factors(S: np.ndarray, lindep: float = 1e-8):
    """(S^1/2, S^-1/2) from the eigen-decomposition of S, dropping eigenvalues <= lindep."""
    s, U = np.linalg.eigh(S)
    keep = s > lindep
    U, s = U[:, keep], s[keep]
    return (U * np.sqrt(s)) @ U.T, (U / np.sqrt(s)) @ U.T


def guess_is_valid(D: np.ndarray, S: np.ndarray, nelec: int, tr_tol: float = 0.05, idem_tol: float = 1.0) -> bool:
    """Electron count tr(DS) within 5% of nelec, and the idempotency error of D measured in
    an orthonormal basis, ||Dt Dt - 2 Dt||_F / ||Dt||_F with Dt = S^1/2 D S^1/2 (the same for
    every orthonormal basis), below 1."""
    ne = float(np.sum(D * S))
    if not np.isfinite(ne) or abs(ne - nelec) / nelec >= tr_tol:
        return False
    Sh, _ = lowdin_factors(S)
    Dt = Sh @ D @ Sh
    nd = np.linalg.norm(Dt)
    return bool(nd > 0 and np.linalg.norm(Dt @ Dt - 2.0 * Dt) / nd < idem_tol)
