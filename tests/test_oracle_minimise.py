"""Pins of the oracle's velocity-projection minimiser and of the Hopf-map input texture."""
import numpy as np

import oracle
from oracle.models import oracle_model
from workloads import cubic_cell, hopf_ansatz, random_spins

C = oracle.constants()


def test_vp_descends_and_keeps_unit_spins():
    n = (6, 5, 4)
    m, w = oracle_model("sc_j123", n, pbc=(1, 1, 1), B=[0.0, 0.0, 2.0])
    S = random_spins(1, n, 3)
    e = [m.energy(S)]
    state = None
    for _ in range(20):
        S, state = m.vp(S, 0.05, 10, state)
        e.append(m.energy(S))
        assert np.abs(np.sqrt((S.reshape(3, -1) ** 2).sum(0)) - 1).max() < 1e-14
    assert all(b <= a + 1e-12 for a, b in zip(e, e[1:]))
    assert e[-1] < e[0] - 1.0


def test_vp_relaxes_ferromagnet_to_closed_form_ground_state():
    # J1 > 0 with a field along z: the ground state is S = z everywhere with
    # energy per site -1/2 * 6 J1 - mu mu_B B
    n = (5, 5, 5)
    m = oracle.Model(n, (1, 1, 1), cubic_cell(), [[0, 0, 0]], [1.0])
    m.add_shell_exchange(1, 1.0)
    m.set_zeeman([0.0, 0.0, 1.0])
    m.build()
    S = random_spins(1, n, 4)
    S[2] = np.abs(S[2]) + 0.2          # start in the upper hemisphere
    S /= np.sqrt((S * S).sum(0))
    S, _ = m.vp(S, 0.1, 3000)
    e = m.energy(S) / 125
    assert abs(e - (-3.0 - C["mu_B"])) < 1e-9
    assert m.torque_max(S) < 1e-6


def test_hopf_ansatz_geometry():
    n, R = (33, 33, 33), 12.0
    S = hopf_ansatz(n, R)
    assert np.abs(np.sqrt((S ** 2).sum(0)) - 1).max() < 1e-12
    c = 16
    assert np.allclose(S[:, 0, c, c, 0], [0, 0, 1])                 # far field
    assert np.allclose(S[:, 0, c, c, c], [0, 0, 1])                 # centre maps to the pole too
    assert S[2, 0, c, c, c + 6] < -0.999                            # ring r = R/2 in the mid plane
    assert S[2, 0, c, c + 6, c] < -0.999
    assert S[2].min() < -0.999 and (S[2] < 0).sum() > 100
