"""Pins for the learned-guess oracle: central finite differences of the loss, the Adam
first-step property (bias correction makes the first update lr*g/(|g|+eps)), block
round trips and the validity checks on a converged density."""
import numpy as np
import pytest

from oracle import mlp


def small_problem(seed=0, n=24):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, mlp.NIN))
    Y = 0.2 * rng.standard_normal((n, mlp.NOUT))
    return X, Y


def test_backward_matches_central_differences():
    params = mlp.init_params(1)
    X, Y = small_problem()
    loss, grads = mlp.loss_and_grad(params, X, Y)
    rng = np.random.default_rng(9)
    h = 1e-6
    for li, p in enumerate(params):
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in p.shape)
            old = p[idx]
            p[idx] = old + h
            lp, _ = mlp.loss_and_grad(params, X, Y)
            p[idx] = old - h
            lm, _ = mlp.loss_and_grad(params, X, Y)
            p[idx] = old
            fd = (lp - lm) / (2 * h)
            assert grads[li][idx] == pytest.approx(fd, rel=1e-5, abs=1e-10), (li, idx)


def test_adam_first_step_is_sign_step():
    params = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -4.0, 1e-3])]
    opt = mlp.Adam(params, lr=1e-2)
    before = params[0].copy()
    opt.step(params, g)
    expect = before - 1e-2 * g[0] / (np.abs(g[0]) + 1e-8)
    assert np.allclose(params[0], expect, rtol=1e-12)


def test_adam_minimises_quadratic():
    p = [np.array([3.0, -1.0])]
    opt = mlp.Adam(p, lr=0.05)
    for _ in range(2000):
        opt.step(p, [2 * p[0]])
    assert np.max(np.abs(p[0])) < 1e-2


def test_training_reduces_loss():
    params = mlp.init_params(2)
    X, Y = small_problem(3, 64)
    opt = mlp.Adam(params, lr=1e-3)
    l0, _ = mlp.loss_and_grad(params, X, Y)
    for _ in range(200):
        _, g = mlp.loss_and_grad(params, X, Y)
        opt.step(params, g)
    l1, _ = mlp.loss_and_grad(params, X, Y)
    assert l1 < 0.2 * l0


def test_features_symmetric_and_cutoff():
    xyz = np.array([[0, 0, 0], [1.5, 0, 0], [0, 13.0, 0]], dtype=float)
    pairs, f = mlp.pair_features(xyz)
    got = {tuple(p) for p in pairs}
    # centre 2 is more than 12 bohr from both others: only its diagonal block remains
    assert got == {(0, 0), (1, 0), (1, 1), (2, 2)}
    # distance 1.5 peaks in the bin nearest 1.5 bohr
    k = list(map(tuple, pairs)).index((1, 0))
    assert np.argmax(f[k, :mlp.NRBF]) == int(round(1.5 / (12 / 31)))
    assert f[k, -1] == 0.0
    d = list(map(tuple, pairs)).index((0, 0))
    assert f[d, -1] == 1.0 and np.all(f[d, :mlp.NRBF] == 0)


def test_block_round_trip(c0, c0_scf):
    pairs, _ = mlp.pair_features(c0.xyz)
    t = mlp.block_targets(c0_scf.D, pairs)
    D = mlp.assemble_density(t, pairs, c0.natm)
    # all pairs of the 6 bohr cube are within the cutoff, and converged blocks of a
    # symmetric D need not be symmetric, so compare the symmetrised blocks
    for (a, b) in pairs[:50]:
        blk = c0_scf.D[5 * a:5 * a + 5, 5 * b:5 * b + 5]
        assert np.allclose(D[5 * a:5 * a + 5, 5 * b:5 * b + 5], 0.5 * (blk + blk.T))


def test_lowdin_factors_invert_each_other(c0_system):
    Sh, Sih = mlp.lowdin_factors(c0_system.S)
    assert np.allclose(Sh @ Sh, c0_system.S, atol=1e-10)
    assert np.allclose(Sh @ Sih, np.eye(len(Sh)), atol=1e-8)


def test_validity_checks(c0_system, c0_scf):
    assert mlp.guess_is_valid(c0_scf.D, c0_system.S, c0_system.nelec)
    # the orthonormal-basis idempotency of a converged density vanishes
    Sh, _ = mlp.lowdin_factors(c0_system.S)
    Dt = Sh @ c0_scf.D @ Sh
    assert np.linalg.norm(Dt @ Dt - 2 * Dt) <= 1e-9 * np.linalg.norm(Dt)
    assert not mlp.guess_is_valid(1.3 * c0_scf.D, c0_system.S, c0_system.nelec)
    # right electron count, wrong occupations: 1.5 x the density of half the electrons...
    Sh, Sih = mlp.lowdin_factors(c0_system.S)
    Dt = Sh @ c0_scf.D @ Sh
    w, U = np.linalg.eigh(Dt)
    occ = np.where(w > 1.0)[0]
    w2 = w.copy()
    w2[occ] = 0.0
    w2[occ[: len(occ) // 2]] = 4.0   # same trace, far from idempotent
    bad = Sih @ (U * w2) @ U.T @ Sih
    assert abs(np.sum(bad * c0_system.S) - c0_system.nelec) < 1e-6
    assert not mlp.guess_is_valid(bad, c0_system.S, c0_system.nelec)


def test_trace_normalisation_restores_electron_count(c0_system, c0_scf):
    # a converged density scaled by 1.3 fails the electron-count gate; scaling its
    # orthonormal-basis form back to tr = nelec recovers the converged density exactly,
    # and tr(dm0 S) = tr(Dt) under dm0 = S^-1/2 Dt S^-1/2 for a full-rank S
    S, ne = c0_system.S, c0_system.nelec
    Sh, Sih = mlp.lowdin_factors(S)
    Dt = Sh @ c0_scf.D @ Sh
    fixed = mlp.normalise_trace(1.3 * Dt, ne)
    assert abs(np.trace(fixed) - ne) <= 1e-10 * ne
    assert np.allclose(fixed, Dt, rtol=0, atol=1e-12 * np.max(np.abs(Dt)))
    dm0 = Sih @ fixed @ Sih
    assert abs(np.sum(dm0 * S) - ne) <= 1e-8 * ne
    assert not mlp.guess_is_valid(Sih @ (1.3 * Dt) @ Sih, S, ne)
    assert mlp.guess_is_valid(dm0, S, ne)
    # a density with non-positive trace is returned unchanged (the gate rejects it)
    neg = -0.5 * Dt
    assert np.array_equal(mlp.normalise_trace(neg, ne), neg)


def test_bf16_round_pins():
    """The oracle's BF16 rounding: representable values are kept, halfway cases go to the
    even significand, the relative error is at most 2^-8 (8 significant bits), and it agrees with torch's CPU
    float32 -> bfloat16 cast (round to nearest even)."""
    import torch
    from oracle import mlp as om
    keep = np.array([0.0, 1.0, -2.5, 0.5 + 2.0 ** -8, 3.0 * 2.0 ** -100, 65280.0])
    assert np.array_equal(om.bf16_round(keep), keep)
    one = 1.0
    assert om.bf16_round(one + 2.0 ** -8) == one                        # tie, even neighbour is 1
    assert om.bf16_round(one + 3 * 2.0 ** -8) == one + 2.0 ** -6         # tie, even neighbour above
    assert om.bf16_round(one + 2.0 ** -8 + 2.0 ** -20) == one + 2.0 ** -7
    assert om.bf16_round(-(one + 2.0 ** -8 + 2.0 ** -20)) == -(one + 2.0 ** -7)
    x = np.random.default_rng(5).standard_normal(20000) * np.exp(np.random.default_rng(6).uniform(-20, 20, 20000))
    x = x.astype(np.float32).astype(np.float64)
    r = om.bf16_round(x)
    assert np.max(np.abs(r - x) / np.abs(x)) <= 2.0 ** -8
    t = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(r, t)
