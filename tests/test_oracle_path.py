"""Pins for the oracle's minimum-energy-path methods ("Static optimization and minimum-energy
paths"): the geodesic metric, GNEB, climbing-image GNEB and the string method, checked against
closed forms that do not come from the oracle:

* geodesic distance of rigid rotations (sqrt(N) theta), antipodes (pi), symmetry and the
  triangle inequality of the product-sphere metric;
* a single spin with easy-axis anisotropy K along z in a transverse field h = mu mu_B B along x
  (Stoner-Wohlfarth): minima at sin(theta0) = h/(2K) on the +x side, saddle at +x with E = -h,
  barrier K (1 - h/(2K))^2, and the minimum-energy path is the x-z meridian through +x;
* a small strongly coupled ferromagnetic cluster (exchange >> anisotropy), whose minimum-energy
  path is coherent rotation with barrier N K.
"""
import numpy as np
import pytest

import oracle
from workloads import cubic_cell, nlerp_chain, polar_chain, random_spins, uniform_spins

K = 1.0
H = 0.6  # mu mu_B B in meV
THETA0 = np.arcsin(H / (2 * K))


def macrospin():
    c = oracle.constants()
    m = oracle.Model((1, 1, 1), (0, 0, 0), cubic_cell(), [[0, 0, 0]], [1.0])
    m.set_zeeman([H / c["mu_B"], 0.0, 0.0])
    m.set_anisotropy(0, K, [0.0, 0.0, 1.0])
    m.build()
    return m


def energy_theta(t):
    # S = (sin t, 0, cos t): E = -K cos^2 t - h sin t
    return -K * np.cos(t) ** 2 - H * np.sin(t)


def test_geodesic_rigid_rotation_and_antipodes():
    n = (4, 3, 2)
    A = uniform_spins(1, n, [0, 0, 1])
    for th in (1e-3, 0.3, 1.2, 2.9):
        B = uniform_spins(1, n, [np.sin(th), 0.0, np.cos(th)])
        assert oracle.geodesic(A, B) == pytest.approx(np.sqrt(24) * th, rel=1e-12)
    assert oracle.geodesic(A, uniform_spins(1, n, [0, 0, -1])) == pytest.approx(np.sqrt(24) * np.pi, rel=1e-15)
    assert oracle.geodesic(A, A) == 0.0


def test_geodesic_is_a_metric():
    n = (5, 4, 3)
    X, Y, Z = (random_spins(2, n, s) for s in (1, 2, 3))
    dxy, dyz, dxz = oracle.geodesic(X, Y), oracle.geodesic(Y, Z), oracle.geodesic(X, Z)
    assert dxy == pytest.approx(oracle.geodesic(Y, X), rel=1e-15)
    assert dxz <= dxy + dyz + 1e-12
    # one site differing by a right angle contributes (pi/2)^2
    Y2 = X.copy()
    Y2[:, 0, 0, 0, 0] = [-X[1, 0, 0, 0, 0], X[0, 0, 0, 0, 0], 0.0]
    Y2[:, 0, 0, 0, 0] /= np.linalg.norm(Y2[:, 0, 0, 0, 0])
    # pick a vector orthogonal to the site spin
    s = X[:, 0, 0, 0, 0]
    u = np.cross(s, [0.0, 0.0, 1.0])
    u /= np.linalg.norm(u)
    Y2[:, 0, 0, 0, 0] = u
    assert oracle.geodesic(X, Y2) == pytest.approx(np.pi / 2, rel=1e-14)


def test_ci_gneb_finds_stoner_wohlfarth_saddle():
    m = macrospin()
    chain = polar_chain(THETA0, np.pi - THETA0, 9, phi_bulge=0.8)
    img, E, fmax = m.gneb(chain, dt=0.1, k=1.0, niter=4000, climbing=True)
    S = img.reshape(9, 3)
    assert fmax < 1e-9
    top = int(np.argmax(E[1:-1])) + 1
    assert np.abs(S[top] - [1.0, 0.0, 0.0]).max() < 1e-8
    assert E[top] == pytest.approx(-H, abs=1e-12)
    assert E[top] - E[0] == pytest.approx(K * (1 - H / (2 * K)) ** 2, abs=1e-12)
    assert np.abs(S[:, 1]).max() < 1e-8  # path on the x-z meridian
    assert np.all(S[:, 0] > 0)  # through +x, not the higher saddle at -x
    # endpoints untouched
    assert np.array_equal(img[0], chain[0]) and np.array_equal(img[-1], chain[-1])


def test_gneb_spaces_images_evenly_on_the_meridian():
    m = macrospin()
    M = 9
    chain = polar_chain(THETA0, np.pi - THETA0, M, phi_bulge=0.5)
    # an uneven start along the meridian too
    img, E, fmax = m.gneb(chain, dt=0.1, k=1.0, niter=6000, climbing=False)
    S = img.reshape(M, 3)
    assert fmax < 1e-9
    theta = np.arctan2(S[:, 0], S[:, 2])
    expect = THETA0 + (np.pi - 2 * THETA0) * np.arange(M) / (M - 1)
    assert np.abs(theta - expect).max() < 1e-8
    assert np.abs(E - energy_theta(expect)).max() < 1e-10
    d = [oracle.geodesic(img[n], img[n + 1]) for n in range(M - 1)]
    assert max(d) - min(d) < 1e-8


def test_string_method_converges_to_equal_arc_length_meridian():
    m = macrospin()
    M = 9
    chain = polar_chain(THETA0, np.pi - THETA0, M, phi_bulge=0.8)
    img, E, fmax = m.string(chain, dt=0.1, niter=3000)
    S = img.reshape(M, 3)
    theta = np.arctan2(S[:, 0], S[:, 2])
    expect = THETA0 + (np.pi - 2 * THETA0) * np.arange(M) / (M - 1)
    assert np.abs(S[:, 1]).max() < 1e-8
    assert np.abs(theta - expect).max() < 1e-8
    # the middle image sits on the saddle by symmetry
    assert E[M // 2] == pytest.approx(-H, abs=1e-12)
    # on the converged path only the tangential part of the force is left (|f| = |dE/dtheta|)
    assert fmax == pytest.approx(np.abs(2 * K * np.cos(expect) * np.sin(expect) - H * np.cos(expect))[1:-1].max(),
                                 rel=1e-6)


def test_ci_gneb_coherent_rotation_barrier_of_a_stiff_cluster():
    n = (2, 2, 2)
    Kc = 0.1
    m = oracle.Model(n, (0, 0, 0), cubic_cell(), [[0, 0, 0]], [1.0])
    m.add_shell_exchange(1, 10.0)
    m.set_anisotropy(0, Kc, [0.0, 0.0, 1.0])
    m.build()
    A = uniform_spins(1, n, [0, 0, 1])
    B = uniform_spins(1, n, [0, 0, -1])
    chain = nlerp_chain(A, B, 7, jitter=0.05, seed=3)
    img, E, fmax = m.gneb(chain, dt=0.02, k=1.0, niter=6000, climbing=True)
    assert fmax < 1e-8
    top = int(np.argmax(E[1:-1])) + 1
    assert E[top] - E[0] == pytest.approx(8 * Kc, abs=1e-9)
    St = img[top].reshape(3, -1)
    assert np.abs(St[2]).max() < 1e-8  # in-plane
    assert np.abs(St - St[:, :1]).max() < 1e-8  # uniform


def test_chain_arguments_are_checked():
    m = macrospin()
    with pytest.raises(ValueError):
        m.gneb(polar_chain(0.1, 3.0, 2), dt=0.1, k=1.0, niter=1)


def _log_map(S, T):
    """Tangent u at S with R_exp(S, u) = T (inverse of the exponential map on the unit sphere)."""
    d = float(np.dot(S, T))
    w = T - d * S
    nw = np.linalg.norm(w)
    return np.zeros(3) if nw == 0 else np.arctan2(nw, d) * w / nw


@pytest.mark.parametrize("thetas,upwind", [((THETA0 + 0.1, THETA0 + 0.4, THETA0 + 0.8), "plus"),
                                           ((1.8, 2.1, 2.5), "minus")])
def test_gneb_force_uses_the_upwind_tangent_on_monotonic_energies(thetas, upwind):
    # one GNEB iteration on a 3-image single-spin chain; the force is read back from the step through
    # the inverse exponential map and compared with the analytic field b = 2K S_z z + h x:
    # F - f must be parallel to the tangent towards the higher-energy neighbour, with
    # (F - f).tau = k (d+ - d-) - f.tau
    m = macrospin()
    ph = (0.0, 0.15, 0.0)
    chain = np.array([[np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)] for t, p in zip(thetas, ph)])
    E = [energy_theta(t) for t in thetas]
    assert (E[0] < E[1] < E[2]) if upwind == "plus" else (E[0] > E[1] > E[2])
    dt, k = 1e-3, 0.7
    img, _, _ = m.gneb(chain.reshape(3, 3, 1, 1, 1, 1), dt=dt, k=k, niter=1, climbing=False)
    S0, S1, S2 = chain
    F = _log_map(S1, img[1].reshape(3)) / dt
    P = lambda x: x - np.dot(x, S1) * S1
    b = np.array([H, 0.0, 2 * K * S1[2]])
    f = P(b)
    t = P(S2 - S1) if upwind == "plus" else P(S1 - S0)
    tau = t / np.linalg.norm(t)
    dplus, dminus = oracle.geodesic(S1, S2), oracle.geodesic(S0, S1)
    G = F - f
    assert np.linalg.norm(np.cross(G, tau)) < 1e-10
    assert np.dot(G, tau) == pytest.approx(k * (dplus - dminus) - np.dot(f, tau), abs=1e-10)


def test_gneb_tangent_is_continuous_across_an_energy_extremum():
    # the middle image is a local maximum only by a hair (E1 - E2 ~ 1e-5 meV, E1 - E0 ~ 0.4 meV):
    # the energy-weighted tangent must then lie almost along the difference towards the higher
    # neighbour, as on the monotonic side of the switch
    m = macrospin()
    thetas = (THETA0 + 0.1, np.pi / 2 - 0.01, np.pi / 2 + 0.011)
    ph = (-0.6, 0.15, 0.15)
    chain = np.array([[np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)] for t, p in zip(thetas, ph)])
    E = [m.energy(c.reshape(3, 1, 1, 1, 1)) for c in chain]
    assert E[1] > E[2] > E[0] and E[1] - E[2] < 1e-4
    dt = 1e-3
    img, _, _ = m.gneb(chain.reshape(3, 3, 1, 1, 1, 1), dt=dt, k=0.7, niter=1, climbing=False)
    S0, S1, S2 = chain
    F = _log_map(S1, img[1].reshape(3)) / dt
    P = lambda x: x - np.dot(x, S1) * S1
    G = F - P(np.array([H, 0.0, 2 * K * S1[2]]))
    tp, tm = P(S2 - S1), P(S1 - S0)
    ang = lambda x, y: np.arccos(min(1.0, abs(np.dot(x, y)) / (np.linalg.norm(x) * np.linalg.norm(y))))
    assert ang(tp, tm) > 0.2
    assert ang(G, tp) < 1e-3


def test_vp_ci_gneb_finds_the_same_stoner_wohlfarth_saddle_faster():
    m = macrospin()
    chain = polar_chain(THETA0, np.pi - THETA0, 9, phi_bulge=0.8)
    img, E, fmax, state = m.gneb_vp(chain, dt=0.1, k=1.0, niter=400, climbing=True)
    S = img.reshape(9, 3)
    assert fmax < 1e-12
    top = int(np.argmax(E[1:-1])) + 1
    assert np.abs(S[top] - [1.0, 0.0, 0.0]).max() < 1e-8
    assert E[top] - E[0] == pytest.approx(K * (1 - H / (2 * K)) ** 2, abs=1e-12)
    assert np.abs(S[:, 1]).max() < 1e-8
    # after 100 iterations steepest descent with the same step is still far behind
    _, _, f100, _ = m.gneb_vp(chain, dt=0.1, k=1.0, niter=100, climbing=True)
    _, _, fsd = m.gneb(chain, dt=0.1, k=1.0, niter=100, climbing=True)
    assert f100 < 1e-5 and fsd > 100 * f100


def test_vp_gneb_first_iteration_is_the_half_dt_squared_step_and_state_carries_over():
    m = macrospin()
    chain = polar_chain(THETA0, np.pi - THETA0, 7, phi_bulge=0.6)
    dt = 0.05
    one, _, _, st1 = m.gneb_vp(chain, dt=dt, k=1.0, niter=1)
    # v = 0 on the first iteration, so the move is R_exp(S, dt^2/2 F): the same as a steepest-descent step of
    # dt^2/2
    sd, _, _ = m.gneb(chain, dt=0.5 * dt * dt, k=1.0, niter=1)
    assert np.abs(one - sd).max() < 1e-15
    # two calls of 5 with the carried state equal one call of 10
    a, _, _, st = m.gneb_vp(chain, dt=dt, k=1.0, niter=5)
    a, _, _, st = m.gneb_vp(a, dt=dt, k=1.0, niter=5, state=st)
    b, _, _, _ = m.gneb_vp(chain, dt=dt, k=1.0, niter=10)
    assert np.abs(a - b).max() < 1e-15
