"""The exact orbital rotation of the Newton (second-order) SCF steps, checked on the CPU.

For kappa [nvir][nocc] the rotation exp(A), A = [[0, -kappa^T], [kappa, 0]], is applied in
closed form from k^T k = V diag(s^2) V^T:
  C_o <- C_o V cos(s) V^T + C_v k V sinc(s) V^T,
  C_v <- C_v (1 + k V ((cos(s) - 1)/s^2) V^T k^T) - C_o V sinc(s) V^T k^T.
This restates it in numpy and pins it to scipy.linalg.expm (an independent library routine)
and to orthonormality, including the small-angle series the kernel uses below s = 1e-4.
"""
import numpy as np
import pytest
from scipy.linalg import expm


def funcs(s2):
    s = np.sqrt(np.clip(s2, 0, None))
    small = s < 1e-4
    c = np.where(small, 1 - 0.5 * s2, np.cos(s))
    sc = np.where(small, 1 - s2 / 6, np.sin(s) / np.where(small, 1, s))
    d = np.where(small, -0.5 + s2 / 24, (np.cos(s) - 1) / np.where(small, 1, s2))
    return c, sc, d


def rotate(Co, Cv, k):
    s2, V = np.linalg.eigh(k.T @ k)
    c, sc, d = funcs(s2)
    Pc, Ps, Pd = (V * c) @ V.T, (V * sc) @ V.T, (V * d) @ V.T
    Co_new = Co @ Pc + Cv @ (k @ Ps)
    Cv_new = Cv @ (np.eye(k.shape[0]) + k @ Pd @ k.T) - Co @ (Ps @ k.T)
    return Co_new, Cv_new


@pytest.mark.parametrize("scale", [0.5, 1e-2, 1e-6, 1e-10])
def test_rotation_matches_expm(scale):
    rng = np.random.default_rng(3)
    n, no = 14, 4
    C, _ = np.linalg.qr(rng.standard_normal((n, n)))
    k = scale * rng.standard_normal((n - no, no))
    A = np.zeros((n, n))
    A[no:, :no] = k
    A[:no, no:] = -k.T
    ref = C @ expm(A)
    Co, Cv = rotate(C[:, :no], C[:, no:], k)
    assert np.abs(Co - ref[:, :no]).max() <= 1e-14
    assert np.abs(Cv - ref[:, no:]).max() <= 1e-14
    full = np.hstack([Co, Cv])
    assert np.abs(full.T @ full - np.eye(n)).max() <= 1e-14


def test_newton_direction_lowers_energy_model():
    # on a quadratic model E(k) = <g, k> + 1/2 <k, H k> with H positive definite, the
    # preconditioned CG that the Newton step runs reaches the minimiser -H^-1 g
    rng = np.random.default_rng(4)
    m = 30
    Q = rng.standard_normal((m, m))
    H = Q @ Q.T + m * np.eye(m)
    g = rng.standard_normal(m)
    h = np.diag(H).copy()
    x = np.zeros(m)
    r = -g
    z = r / h
    p = z.copy()
    rz = r @ z
    for _ in range(m):
        Ap = H @ p
        a = rz / (p @ Ap)
        x += a * p
        r -= a * Ap
        z = r / h
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    assert np.allclose(x, -np.linalg.solve(H, g), atol=1e-10)
