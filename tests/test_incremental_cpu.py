"""The factorisation behind the incremental mixed-precision exchange, checked on the CPU.

K is linear in the density, so the exchange of a new occupied projector P_n = C_n C_n^T
(orthonormal columns) follows from that of the previous one, P_p, plus K[P_n - P_p].  The
SCF writes the change as U+ U+^T - U- U-^T from the principal vectors of the two occupied
spaces: with M = C_p^T C_n = Y cos(theta) W^T, B = C_n W and A = C_p M W / cos pair up, and
for each pair (a, b) of unit vectors b b^T - a a^T = u+ u+^T - u- u-^T with
u+- = sqrt(s/2) (p +- m), p = (b + a)/|b + a|, m = (b - a)/|b - a|, s = |b - a||b + a|/2.

These tests restate that construction in numpy and pin it to what the mathematics fixes:
the factors reproduce P_n - P_p to rounding at every size of change, s are the sines of the
principal angles (scipy.linalg.subspace_angles, an independent library routine), and the
squared factor norm is 2 sum(s), so a mixed-precision build of the factors makes an error
proportional to the change.
"""
import numpy as np
import pytest
from scipy.linalg import subspace_angles


def _orth(A):
    q, _ = np.linalg.qr(A)
    return q


def factors(Cp, Cn):
    M = Cp.T @ Cn
    c2, W = np.linalg.eigh(M.T @ M)
    A = Cp @ (M @ W)
    B = Cn @ W
    k = Cp.shape[1]
    Up, Um, s = np.zeros_like(Cp), np.zeros_like(Cp), np.zeros(k)
    for j in range(k):
        a = A[:, j] / np.linalg.norm(A[:, j])
        b = B[:, j] / np.linalg.norm(B[:, j])
        nm, npl = np.linalg.norm(b - a), np.linalg.norm(b + a)
        if nm == 0.0:
            continue
        s[j] = 0.5 * nm * npl
        f = np.sqrt(0.5 * s[j])
        Up[:, j] = f * ((b + a) / npl + (b - a) / nm)
        Um[:, j] = f * ((b + a) / npl - (b - a) / nm)
    return Up, Um, s, c2


@pytest.mark.parametrize("scale", [3e-1, 1e-2, 1e-5, 1e-9, 0.0])
def test_factors_reproduce_projector_change(scale):
    rng = np.random.default_rng(17)
    n, k = 48, 9
    Cp = _orth(rng.standard_normal((n, k)))
    G = scale * rng.standard_normal((n, k))
    Cn = _orth(Cp + G - Cp @ (Cp.T @ G)) @ _orth(rng.standard_normal((k, k)))
    dP = Cn @ Cn.T - Cp @ Cp.T
    Up, Um, s, c2 = factors(Cp, Cn)
    assert np.abs(Up @ Up.T - Um @ Um.T - dP).max() <= 2e-15
    # the sines are those of the principal angles where cos^2 resolves them (angles far above
    # sqrt(eps)); below that, vectors of a near-degenerate cluster pair up in any order, the
    # factorisation stays exact and the total stays of the size of the change
    theta = np.sort(subspace_angles(Cp, Cn))
    if scale >= 1e-5:
        assert np.allclose(np.sort(s), np.sort(np.sin(theta)), atol=1e-12)
    assert np.sum(s) <= 1.5 * np.sum(np.sin(theta)) + 1e-13
    assert abs(np.sum(Up ** 2) + np.sum(Um ** 2) - 2 * np.sum(s)) <= 1e-12 * max(1.0, np.sum(s))
    # Frobenius norm of the change: sqrt(2 sum s^2) (eigenvalues +-s)
    assert abs(np.linalg.norm(dP) - np.sqrt(2 * np.sum(s ** 2))) <= 1e-12


def test_sign_of_the_change_is_kept():
    # rotating a single occupied orbital by theta gives eigenvalues +-sin(theta)
    n = 6
    Cp = np.eye(n)[:, :2]
    t = 0.3
    Cn = Cp.copy()
    Cn[:, 1] = np.cos(t) * np.eye(n)[:, 1] + np.sin(t) * np.eye(n)[:, 4]
    Up, Um, s, _ = factors(Cp, Cn)
    ev = np.linalg.eigvalsh(Up @ Up.T - Um @ Um.T)
    assert np.isclose(ev.max(), np.sin(t)) and np.isclose(ev.min(), -np.sin(t))
    assert np.isclose(np.max(s), np.sin(t)) and np.isclose(np.min(s), 0.0)
