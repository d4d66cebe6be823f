"""The finite-difference orbital Hessian that pins the GPU stability analysis, checked on the
CPU against independent routes: second differences of the oracle's energy give the same
matrix, and on the stretched ten-centre ring the oracle's own SCF shows the saddle point and
the lower minimum that the GPU tests expect."""
import numpy as np

import gen
from oracle import scf as oscf
from stability_fd import energy_fd_hessian, escape, fd_hessian, h10_ring


def test_gradient_differences_match_energy_differences():
    mol = gen.make_molecule(2, gen.molecules.box_for(2), 3)
    sysm = oscf.build_system(mol)
    ref = oscf.rhf(sysm)
    assert ref.converged
    Hg, _ = fd_hessian(sysm, ref.D)
    He = energy_fd_hessian(sysm, ref.D)
    lg, le = np.linalg.eigvalsh(Hg), np.linalg.eigvalsh(He)
    assert np.max(np.abs(lg - le)) <= 1e-4 * np.max(np.abs(le)), (lg[:3], le[:3])
    assert lg[0] > 0                      # the ground state of two centres is a minimum


def test_ring_saddle_and_escape_in_the_oracle():
    sysm = oscf.build_system(h10_ring())
    sad = oscf.rhf(sysm)
    assert sad.converged
    H, XC = fd_hessian(sysm, sad.D)
    lam = np.linalg.eigvalsh(H)
    assert lam[0] < -0.05 and lam[1] > 0  # one negative direction: a saddle point
    lows = [escape(sysm, sad.D, H, XC, angle=a) for a in (0.3, -0.3)]
    for low in lows:
        assert low.converged and low.energy < sad.energy - 1e-3
    # the two bond-alternation patterns are images of each other under the ring's symmetry
    assert abs(lows[0].energy - lows[1].energy) <= 1e-8
    assert np.linalg.eigvalsh(fd_hessian(sysm, lows[0].D)[0])[0] > 0
